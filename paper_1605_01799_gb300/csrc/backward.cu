// Backward pass by the envelope theorem.
//
// phi(x, t; A) = max_v -F(v; x, t, A) with F the objective of eq. 3.3, and the
// maximiser v* is grad_x phi (Section 1).  Differentiating at fixed v*:
//   d phi/dx = v*,  d phi/dt = -H(v*),  d phi/dA = -1/2 v* v*^T
// (J*(v) = 1/2 v^T A v + ...).  With upstream weights g_q per query:
//   g_x[q] = g_q v*_q,  g_t[q] = -g_q H(v*_q),
//   g_A = -1/2 sum_q g_q v*_q v*_q^T = -1/2 V^T diag(g) V   (V = [B][n])
// and for diagonal A only the diagonal -1/2 sum_q g_q v*_{qi}^2.
#include "common.cuh"
#include "hopf_internal.h"

namespace hopf {
namespace {

// g_x and g_t: one warp per query.
__global__ void k_bwd_xt(const float* __restrict__ g, const float* __restrict__ V, const float* __restrict__ w,
                         const float* __restrict__ P, int n, int64_t B, int h_kind, float* __restrict__ gx,
                         float* __restrict__ gt) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= B) return;
  const float gq = g[q];
  double h = 0.0;  // H(v): sum (l1 kinds), sum of squares (l2 kinds), max (l_inf)
  for (int i = lane; i < n; i += 32) {
    const float v = V[q * n + i];
    if (gx) gx[q * n + i] = gq * v;
    const double av = fabs((double)v);
    if (h_kind == H_L2) h += av * av;
    else if (h_kind == H_DNORM) h += (double)w[i] * av * av;
    else if (h_kind == H_LINF) h = av > h ? av : h;
    else if (h_kind != H_ANORM) h += (double)w[i] * av;
  }
  if (h_kind == H_ANORM) {
    // sqrt(<v, M v>) = sqrt(sum_k l_k ((P^T v)_k)^2), l the weights
    for (int k = lane; k < n; k += 32) {
      double r = 0.0;
      for (int i = 0; i < n; ++i) r += (double)P[(int64_t)i * n + k] * (double)V[q * n + i];
      h += (double)w[k] * r * r;
    }
  }
  if (h_kind == H_LINF) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
  } else {
    h = warp_sum(h);
  }
  if (h_kind == H_L2 || h_kind == H_DNORM || h_kind == H_ANORM) h = sqrt(h);
  if (lane == 0 && gt) gt[q] = (float)(-(double)gq * h);
}

// Diagonal g_A: column sums over the batch.
__global__ void k_bwd_diagA(const float* __restrict__ g, const float* __restrict__ V, int n, int64_t B,
                            float* __restrict__ gA) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int64_t q = 0; q < B; ++q) {
    const double v = V[q * n + i];
    s += (double)g[q] * v * v;
  }
  gA[i] = (float)(-0.5 * s);
}

// Dense g_A: 128 x 128 output tile per CTA, K = the batch.  Both operands are
// rows of V (contiguous along the output index), so no transpose is needed.
constexpr int BM = 128, BK = 16, NT = 256, PADS = 4;

// g_A is symmetric, so only the tiles (bi, bj) with bi <= bj are computed and
// an off-diagonal tile is written twice (as itself and transposed): T (T + 1) / 2
// blocks for T = ceil(n / 128) tile rows.  The next k-tile of the batch is
// loaded into registers while the current one is multiplied.
__global__ void __launch_bounds__(NT, 2) k_bwd_denseA(const float* __restrict__ g, const float* __restrict__ V, int n,
                                                      int64_t B, float* __restrict__ gA) {
  __shared__ __align__(16) float As[2][BK][BM + PADS];
  __shared__ __align__(16) float Bs[2][BK][BM + PADS];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int T = (n + BM - 1) / BM;
  int bi = 0, rem = blockIdx.x;
  while (rem >= T - bi) {
    rem -= T - bi;
    ++bi;
  }
  const int bj = bi + rem;
  const int i0 = bi * BM, j0 = bj * BM;
  float acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
  // each thread stages 8 elements of each operand tile (16 batch rows x 128)
  float ra[8], rb[8];
  auto load = [&](int64_t q0) {
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int f = tid + h * NT, kk = f >> 7, col = f & 127;
      const int64_t q = q0 + kk;
      const bool okq = q < B;
      const float gq = okq ? g[q] : 0.f;
      const int ia = i0 + col, jb = j0 + col;
      ra[h] = (okq && ia < n) ? V[q * n + ia] * gq : 0.f;
      rb[h] = (okq && jb < n) ? V[q * n + jb] : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int f = tid + h * NT, kk = f >> 7, col = f & 127;
      As[buf][kk][col] = ra[h];
      Bs[buf][kk][col] = rb[h];
    }
  };
  load(0);
  store(0);
  __syncthreads();
  int cur = 0;
  for (int64_t q0 = 0; q0 < B; q0 += BK) {
    const bool more = q0 + BK < B;
    if (more) load(q0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    if (more) {
      store(cur ^ 1);  // the other buffer: its last readers finished before the previous barrier
      __syncthreads();
      cur ^= 1;
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = i0 + (a < 4 ? ty * 4 + a : 64 + ty * 4 + a - 4);
    if (i >= n) continue;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int j = j0 + (b < 4 ? tx * 4 + b : 64 + tx * 4 + b - 4);
      if (j < n) {
        const float v = -0.5f * acc[a][b];
        gA[(int64_t)i * n + j] = v;
        if (bi != bj) gA[(int64_t)j * n + i] = v;
      }
    }
  }
}

// Column sums over the batch for the parameter gradients: thread i owns
// column i and walks the batch in order (FP64 sums, deterministic).
__global__ void k_bwd_params(const float* __restrict__ g, const float* __restrict__ V, const float* __restrict__ t,
                             const float* __restrict__ dphidt, int n, int64_t B, int h_kind,
                             float* __restrict__ g_c, float* __restrict__ g_w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sc = 0.0, sw = 0.0;
  for (int64_t q = 0; q < B; ++q) {
    const double v = V[q * n + i], gq = g[q];
    sc -= gq * v;
    if (g_w) {
      if (h_kind == H_WL1) {
        sw -= gq * (double)t[q] * fabs(v);
      } else {  // H_DNORM: H_q = -dphidt[q]
        const double H = -(double)dphidt[q];
        if (H > 0.0) sw -= gq * (double)t[q] * v * v / (2.0 * H);
      }
    }
  }
  if (g_c) g_c[i] = (float)sc;
  if (g_w) g_w[i] = (float)sw;
}

// dL/dc0 = -sum_q g_q: one block, a fixed reduction order.
__global__ void k_bwd_c0(const float* __restrict__ g, int64_t B, float* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t q = threadIdx.x; q < B; q += blockDim.x) s -= g[q];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (float)red[0];
}

}  // namespace

hopf_status backward_params(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, const float* t,
                            const float* dphidt, float* g_c, float* g_c0, float* g_w, cudaStream_t stream) {
  const int n = h->n;
  if (g_c || g_w) {
    k_bwd_params<<<(n + 127) / 128, 128, 0, stream>>>(g_phi, vstar, t, dphidt, n, batch, h->h_kind, g_c, g_w);
    HOPF_CUDA(cudaGetLastError());
  }
  if (g_c0) {
    k_bwd_c0<<<1, 256, 0, stream>>>(g_phi, batch, g_c0);
    HOPF_CUDA(cudaGetLastError());
  }
  return HOPF_OK;
}

hopf_status backward(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, float* g_x, float* g_t,
                     float* g_A, cudaStream_t stream) {
  const int n = h->n;
  if (g_x || g_t) {
    k_bwd_xt<<<(unsigned)((batch * 32 + 255) / 256), 256, 0, stream>>>(g_phi, vstar, h->d_wf, h->d_Pf, n, batch,
                                                                        h->h_kind, g_x, g_t);
    HOPF_CUDA(cudaGetLastError());
  }
  if (g_A) {
    if (h->a_kind == HOPF_A_DIAG) {
      k_bwd_diagA<<<(n + 255) / 256, 256, 0, stream>>>(g_phi, vstar, n, batch, g_A);
    } else {
      const int T = (n + BM - 1) / BM;
      k_bwd_denseA<<<(unsigned)(T * (T + 1) / 2), NT, 0, stream>>>(g_phi, vstar, n, batch, g_A);
    }
    HOPF_CUDA(cudaGetLastError());
  }
  return HOPF_OK;
}

}  // namespace hopf
