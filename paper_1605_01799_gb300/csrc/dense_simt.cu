// Dense A, FP32 on the CUDA cores: the paper's split Bregman form.
//
// Per iteration k, for every query (a column of the n x B block):
//   r^{k-1} = y + lambda (2 p^{k-1} - u^{k-1})      (= y + lambda (d - b))
//   v^k     = M r^{k-1},  M = (A + lambda I)^{-1}    (eq. 3.4(a))
//   u^k     = v^k + u^{k-1} - p^{k-1}                 (= v^k + b^{k-1})
//   p^k     = prox_{(t/lambda) H}(u^k)                (eq. 3.4(b))
// with p^0 = u^0 = y.  b never needs storing: b^k = u^k - p^k (eq. 3.4(c)).
//
// One persistent cooperative launch runs all iterations.  Work item =
// (128-row tile of n, 128-query column tile).  The B-operand loader forms r
// from u and y on the fly; the epilogue updates u and writes per-(row tile,
// query) partial sums of |u^k - u^{k-1}|^2 and |u^k|^2.  u^k lives in buffer
// k & 1: an item's GEMM reads u^{k-1} over all rows of its column while the
// epilogues of the column's other row tiles write u^k, so the two may not
// share storage.  A grid barrier ends
// each iteration; the next iteration decides each query's convergence from the
// partials (every CTA reaches the same decision from the same data) and skips
// column tiles with no active query.  After the last iteration one more GEMM
// with A gives <p, A p> for phi.
#include "common.cuh"
#include "hopf_internal.h"

namespace hopf {

hopf_status dense_init(hopf_handle h, DenseWs& w, const float* x, const float* t, cudaStream_t s);
hopf_status dense_finalize(hopf_handle h, DenseWs& w, double* phi, float* dphidt, int32_t* iters, uint8_t* qstatus,
                           cudaStream_t s);

namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;
constexpr int PADS = 4;  // smem row padding (floats)

struct SimtArgs {
  const float* M;   // [np][np] (A + lambda I)^{-1}
  const float* A;   // [np][np] A (final phi pass)
  const float* w;   // [np] weights (1 when unweighted / padding)
  int n, np, rt, ct, h_kind, max_iter;
  float lam, tol;
  long long wait_limit;  // clock cycles of every bounded wait
  DenseWs ws;
  float* grad;      // [B][n] user output
  const float* x;   // [B][n] the caller's queries (terminal point)
  float* beta;      // optional: control in dH(grad phi) [B][n]
  float* xfin;      // optional: terminal point x - t beta [B][n]
  float* U[2];      // u^k in U[k & 1] (U[0] holds u^0 = y)
};

// Per-query data of the current column tile, decided at the start of an item.
struct TileQ {
  float tau[BN];
  float scale[BN];  // l2: shrink_2 scale of u^{k-1}
  int act[BN];      // 1 = update this query in this iteration
  int ub[BN];       // final pass: the buffer of the query's last iterate
  int first;        // iteration 1: p^0 = y
};

__device__ __forceinline__ float prox_of(float u, float w, float tau, float scale, int h_kind) {
  return h_kind == H_L2 ? scale * u : shrink1(u, tau * w);
}

// Decide, for the 128 queries of column tile c at iteration k, which are
// still active (convergence of iteration k-1 from its partials).  The CTA
// owning row tile 0 records the decisions.  Returns the active count.
__device__ int decide(const SimtArgs& a, int k, int c, int r, TileQ& tq) {
  const DenseWs& W = a.ws;
  const int par = (k - 1) & 1;
  int cnt = 0;
  for (int j = threadIdx.x; j < BN; j += blockDim.x) {
    const int64_t q = (int64_t)c * BN + j;
    const int done = W.qdone[q];
    float du2 = 0.f, nu2 = 0.f;
    if (k > 1) {
      for (int rr = 0; rr < a.rt; ++rr) {
        du2 += W.part[((int64_t)(par * 2 + 0) * a.rt + rr) * W.B_pad + q];
        nu2 += W.part[((int64_t)(par * 2 + 1) * a.rt + rr) * W.B_pad + q];
      }
    }
    int act = 0;
    if (!done) {
      const int kprev = k - 1;
      if (kprev >= 2 && du2 <= a.tol * fmaxf(1.f, nu2)) {
        if (r == 0) {
          W.qdone[q] = 1;
          W.qiter[q] = kprev;
        }
      } else if (kprev >= a.max_iter) {
        if (r == 0) {
          W.qdone[q] = 2;
          W.qiter[q] = a.max_iter;
        }
      } else {
        act = 1;
      }
    }
    tq.act[j] = act;
    tq.tau[j] = W.tau[q];
    // l2: shrink_2 scale of u^{k-1}, its norm from the partials of iteration k-1
    tq.scale[j] = k == 1 ? 1.f : shrink2_scale(sqrtf(nu2), tq.tau[j]);
    cnt += act;
  }
  tq.first = k == 1;
  return cnt;
}

__device__ __forceinline__ int block_sum_int(int v, int* red) {
  v = __reduce_add_sync(0xffffffffu, v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int s = 0;
  for (int i = 0; i < NT / 32; ++i) s += red[i];
  return s;
}

// One 128x128 tile: D = Mat[rows of r-tile][:] * Rhs[:, queries of c-tile],
// where Rhs is formed by the loader.  mode 0: step (r = y + lam (2p - u));
// mode 1: final (rhs = p).
template <int MODE>
__device__ void gemm_tile(const SimtArgs& a, const float* __restrict__ Mat, int r, int c, const TileQ& tq,
                          const float* __restrict__ Uin, float (*As)[BK][BM + PADS], float (*Bs)[BK][BN + PADS],
                          float acc[8][8]) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const DenseWs& W = a.ws;
  const int np = a.np;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  float4 ra[2], rb[2];
  auto load_a = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int f = tid + h * NT, row = f >> 2, c4 = f & 3;
      ra[h] = *reinterpret_cast<const float4*>(Mat + (int64_t)(r * BM + row) * np + k0 + c4 * 4);
    }
  };
  auto load_b = [&](int k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int f = tid + h * NT, j = f >> 2, c4 = f & 3;
      const int64_t q = (int64_t)c * BN + j;
      const int64_t off = q * np + k0 + c4 * 4;
      // step: u^{k-1} of every query; final: each query's last iterate
      const float* Uq = MODE == 0 ? Uin : a.U[tq.ub[j]];
      const float4 u4 = *reinterpret_cast<const float4*>(Uq + off);
      float4 o;
      if (MODE == 0) {
        const float4 y4 = *reinterpret_cast<const float4*>(W.y + off);
        const float4 w4 = *reinterpret_cast<const float4*>(a.w + k0 + c4 * 4);
        const float tau = tq.tau[j], sc = tq.scale[j], lam = a.lam;
        if (tq.first) {
          o = make_float4(y4.x + lam * y4.x, y4.y + lam * y4.y, y4.z + lam * y4.z, y4.w + lam * y4.w);
        } else {
          o.x = y4.x + lam * (2.f * prox_of(u4.x, w4.x, tau, sc, a.h_kind) - u4.x);
          o.y = y4.y + lam * (2.f * prox_of(u4.y, w4.y, tau, sc, a.h_kind) - u4.y);
          o.z = y4.z + lam * (2.f * prox_of(u4.z, w4.z, tau, sc, a.h_kind) - u4.z);
          o.w = y4.w + lam * (2.f * prox_of(u4.w, w4.w, tau, sc, a.h_kind) - u4.w);
        }
      } else {
        const float4 w4 = *reinterpret_cast<const float4*>(a.w + k0 + c4 * 4);
        const float tau = tq.tau[j], sc = tq.scale[j];
        o.x = prox_of(u4.x, w4.x, tau, sc, a.h_kind);
        o.y = prox_of(u4.y, w4.y, tau, sc, a.h_kind);
        o.z = prox_of(u4.z, w4.z, tau, sc, a.h_kind);
        o.w = prox_of(u4.w, w4.w, tau, sc, a.h_kind);
      }
      rb[h] = o;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int f = tid + h * NT, row = f >> 2, c4 = f & 3;
      As[buf][c4 * 4 + 0][row] = ra[h].x;
      As[buf][c4 * 4 + 1][row] = ra[h].y;
      As[buf][c4 * 4 + 2][row] = ra[h].z;
      As[buf][c4 * 4 + 3][row] = ra[h].w;
      Bs[buf][c4 * 4 + 0][row] = rb[h].x;
      Bs[buf][c4 * 4 + 1][row] = rb[h].y;
      Bs[buf][c4 * 4 + 2][row] = rb[h].z;
      Bs[buf][c4 * 4 + 3][row] = rb[h].w;
    }
  };
  const int nk = np / BK;
  load_a(0);
  load_b(0);
  __syncthreads();  // previous users of the smem buffers are done
  store(0);
  __syncthreads();
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) {
      load_a((kt + 1) * BK);
      load_b((kt + 1) * BK);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (kt + 1 < nk) {
      store(cur ^ 1);
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(NT, 1) k_dense_simt(SimtArgs a) {
  // one buffer: the two GEMM operand tiles, reused as reduction scratch
  __shared__ __align__(16) float smem[2 * BK * (BM + PADS) + 2 * BK * (BN + PADS)];
  auto As = reinterpret_cast<float(*)[BK][BM + PADS]>(smem);
  auto Bs = reinterpret_cast<float(*)[BK][BN + PADS]>(smem + 2 * BK * (BM + PADS));
  __shared__ TileQ tq;
  __shared__ int red[NT / 32];
  const DenseWs& W = a.ws;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int items = a.rt * a.ct;
  float acc[8][8];

  for (int k = 1;; ++k) {
    if (blockIdx.x == 0 && tid == 0) atomicExch(W.bar + 2 + ((k + 1) % 3), 0u);
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      const int r = it % a.rt, c = it / a.rt;
      __syncthreads();
      int cnt = decide(a, k, c, r, tq);
      cnt = block_sum_int(cnt, red);
      if (r == 0 && tid == 0 && cnt > 0) atomicAdd(W.bar + 2 + (k % 3), (unsigned)cnt);
      if (cnt == 0 || k > a.max_iter) continue;
      const float* Uold = a.U[(k - 1) & 1];
      float* Unew = a.U[k & 1];
      gemm_tile<0>(a, a.M, r, c, tq, Uold, As, Bs, acc);
      // epilogue: u^k = v^k + u^{k-1} - p^{k-1}; partials of |du|^2, |u|^2
      float pdu[8], pnu[8];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = (jj < 4 ? tx * 4 + jj : 64 + tx * 4 + (jj - 4));
        const int64_t q = (int64_t)c * BN + j;
        pdu[jj] = 0.f;
        pnu[jj] = 0.f;
        const bool act = tq.act[j];
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int row0 = r * BM + hh * 64 + ty * 4;
          const float4 u4 = *reinterpret_cast<const float4*>(Uold + q * a.np + row0);
          const float4 w4 = *reinterpret_cast<const float4*>(a.w + row0);
          const float uo[4] = {u4.x, u4.y, u4.z, u4.w}, wv[4] = {w4.x, w4.y, w4.z, w4.w};
          float un[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float p = tq.first ? uo[e] : prox_of(uo[e], wv[e], tq.tau[j], tq.scale[j], a.h_kind);
            const float v = acc[hh * 4 + e][jj];
            un[e] = v + uo[e] - p;
            const float du = un[e] - uo[e];
            pdu[jj] += du * du;
            pnu[jj] += un[e] * un[e];
          }
          if (act) *reinterpret_cast<float4*>(Unew + q * a.np + row0) = make_float4(un[0], un[1], un[2], un[3]);
        }
      }
      // reduce the partials over the 16 row groups (ty) of the tile
      __syncthreads();
      float* rs = smem;  // 16 x 128 x 2 floats
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = (jj < 4 ? tx * 4 + jj : 64 + tx * 4 + (jj - 4));
        rs[(ty * BN + j) * 2 + 0] = pdu[jj];
        rs[(ty * BN + j) * 2 + 1] = pnu[jj];
      }
      __syncthreads();
      if (tid < BN) {
        float s0 = 0.f, s1 = 0.f;
        for (int t2 = 0; t2 < 16; ++t2) {
          s0 += rs[(t2 * BN + tid) * 2 + 0];
          s1 += rs[(t2 * BN + tid) * 2 + 1];
        }
        const int64_t q = (int64_t)c * BN + tid;
        if (tq.act[tid]) {
          const int par = k & 1;
          W.part[((int64_t)(par * 2 + 0) * a.rt + r) * W.B_pad + q] = s0;
          W.part[((int64_t)(par * 2 + 1) * a.rt + r) * W.B_pad + q] = s1;
        }
      }
    }
    if (!grid_barrier(W.bar, gridDim.x, W.err, a.wait_limit)) return;
    const unsigned active = ld_acquire_u32(W.bar + 2 + (k % 3));
    if (active == 0) break;
  }

  // Final pass: D = A p for every query; phi partials and the gradient.
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int r = it % a.rt, c = it / a.rt;
    __syncthreads();
    // per-query prox data of the last iterate
    for (int j = tid; j < BN; j += blockDim.x) {
      const int64_t q = (int64_t)c * BN + j;
      tq.tau[j] = W.tau[q];
      tq.act[j] = q < W.B;
      const int kl = W.qiter[q];
      float nu2 = 0.f;
      if (kl >= 1)
        for (int rr = 0; rr < a.rt; ++rr) nu2 += W.part[((int64_t)((kl & 1) * 2 + 1) * a.rt + rr) * W.B_pad + q];
      tq.scale[j] = kl >= 1 ? shrink2_scale(sqrtf(nu2), tq.tau[j]) : 1.f;
      tq.ub[j] = kl & 1;
    }
    tq.first = 0;
    __syncthreads();
    int any = 0;
    for (int j = 0; j < BN; ++j) any |= tq.act[j];
    if (!any) continue;
    gemm_tile<1>(a, a.A, r, c, tq, nullptr, As, Bs, acc);
    double f0[8], f1[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = (jj < 4 ? tx * 4 + jj : 64 + tx * 4 + (jj - 4));
      const int64_t q = (int64_t)c * BN + j;
      f0[jj] = 0.0;
      f1[jj] = 0.0;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int row0 = r * BM + hh * 64 + ty * 4;
        const float4 u4 = *reinterpret_cast<const float4*>(a.U[tq.ub[j]] + q * a.np + row0);
        const float4 y4 = *reinterpret_cast<const float4*>(W.y + q * a.np + row0);
        const float4 w4 = *reinterpret_cast<const float4*>(a.w + row0);
        const float uo[4] = {u4.x, u4.y, u4.z, u4.w}, yv[4] = {y4.x, y4.y, y4.z, y4.w};
        const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float p = prox_of(uo[e], wv[e], tq.tau[j], tq.scale[j], a.h_kind);
          const double pd = p;
          f0[jj] += (double)yv[e] * pd - 0.5 * pd * (double)acc[hh * 4 + e][jj];
          f1[jj] += a.h_kind == H_L2 ? pd * pd : (double)wv[e] * fabs(pd);
          const int row = row0 + e;
          if (tq.act[j] && row < a.n) {
            a.grad[q * a.n + row] = p;
            if (a.beta) {
              // control (y - A p) / t = (u - p) / tau at the fixed point
              const float tau = tq.tau[j];
              const float bt = tau > 0.f ? (uo[e] - p) / tau : 0.f;
              a.beta[q * a.n + row] = bt;
              if (a.xfin) a.xfin[q * a.n + row] = a.x[q * a.n + row] - tau * a.lam * bt;
            }
          }
        }
      }
    }
    __syncthreads();
    double* rs = reinterpret_cast<double*>(smem);  // 16 x 128 x 2 doubles
    static_assert(sizeof(smem) >= 16 * BN * 2 * sizeof(double), "reduction scratch");
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = (jj < 4 ? tx * 4 + jj : 64 + tx * 4 + (jj - 4));
      rs[(ty * BN + j) * 2 + 0] = f0[jj];
      rs[(ty * BN + j) * 2 + 1] = f1[jj];
    }
    __syncthreads();
    if (tid < BN) {
      double s0 = 0.0, s1 = 0.0;
      for (int t2 = 0; t2 < 16; ++t2) {
        s0 += rs[(t2 * BN + tid) * 2 + 0];
        s1 += rs[(t2 * BN + tid) * 2 + 1];
      }
      const int64_t q = (int64_t)c * BN + tid;
      W.fpart[(int64_t)r * W.B_pad + q] = s0;
      W.fpart[(int64_t)(a.rt + r) * W.B_pad + q] = s1;
    }
  }
}

}  // namespace

hopf_status dense_eval_simt(hopf_handle h, DenseWs& w, const float* x, const float* t, double* phi, float* grad,
                            float* dphidt, int32_t* iters, uint8_t* qstatus, cudaStream_t stream, float* beta,
                            float* xfin) {
  hopf_status s = dense_init(h, w, x, t, stream);
  if (s != HOPF_OK) return s;
  SimtArgs a;
  a.M = h->d_M32;
  a.A = h->d_A32;
  a.w = h->d_wf;
  a.n = h->n;
  a.np = h->n_pad;
  a.rt = h->n_pad / BM;
  a.ct = (int)(w.B_pad / BN);
  a.h_kind = h->h_kind;
  a.max_iter = h->max_iter;
  a.wait_limit = h->wait_limit > 0 ? h->wait_limit : kWaitLimitCycles;
  a.lam = (float)h->lambda;
  a.tol = (float)h->tol;
  a.ws = w;
  a.grad = grad;
  a.x = x;
  a.beta = beta;
  a.xfin = xfin;
  a.U[0] = w.u;
  a.U[1] = w.u_b;
  int per_sm = 0;
  HOPF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_simt, NT, 0));
  if (per_sm < 1) return fail(HOPF_ECUDA, "dense FP32 solver: kernel does not fit on an SM");
  int grid = per_sm * h->num_sms;
  // under a cap (ragged batches) at most one CTA per SM of the share, so that
  // any unplaced CTA always finds an SM free of other cooperative CTAs
  if (h->grid_cap > 0 && grid > h->grid_cap) grid = h->grid_cap;
  const int items = a.rt * a.ct;
  if (grid > items) grid = items;
  void* args[] = {&a};
  if (h->prof_start) HOPF_CUDA(cudaEventRecord(h->prof_start, stream));
  HOPF_CUDA(cudaLaunchCooperativeKernel((const void*)k_dense_simt, dim3(grid), dim3(NT), args, 0, stream));
  if (h->prof_stop) HOPF_CUDA(cudaEventRecord(h->prof_stop, stream));
  return dense_finalize(h, w, phi, dphidt, iters, qstatus, stream);
}

}  // namespace hopf
