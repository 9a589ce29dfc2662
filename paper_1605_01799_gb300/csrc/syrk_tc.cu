// Backward g_A = -1/2 V^T diag(g) V on the tensor cores (tcgen05 + TMA + TMEM).
//
// The envelope theorem applied to eq. 3.3 gives d phi / dA = -1/2 v* v*^T for
// each query (J*(v) = 1/2 v^T A v + ...), so with upstream weights g_q the
// batch gradient is the symmetric rank-B product
//     g_A[i][j] = -1/2 sum_q g_q V[q][i] V[q][j]        (V = [B][n], v* by rows)
// a contraction over the queries: C = X^T Y with X = diag(g) V, Y = V.
//
// Precision.  Both operands go in as two-term FP16 splits (x = x_hi +
// 2^-11 x_lo', ~2^-22), three MMAs per K = 16 step: X_hi Y_hi into a chunk
// accumulator, X_hi Y_lo' + X_lo' Y_hi into a correction accumulator scaled
// exactly by 2^-11.  The tensor cores' FP32 accumulation truncates; over the
// 2,048 K steps of 32,768 queries its bias would reach ~1e-4, so the main
// product is promoted to registers every 512 queries (one of three rotating
// TMEM chunk slots), and the partial products of the K ranges are summed in
// FP64.  g is scaled by a power of two into FP16's range first (exact).
//
// Layout.  A prep kernel writes the four operand planes transposed, K-major in
// the query: P[i][q] for i < n_pad (zero padded), q < K_pad = round_up(B, 64).
// Work items are (tile on or above the diagonal, K range of 4,096 queries),
// the K range slowest so that the CTAs in flight share one K range of the
// planes (64 MB at n = 2048, resident in L2).  A reduce kernel sums the K
// ranges in FP64, scales by -1/2 and writes each tile and its mirror.
//
// One persistent launch, one CTA per SM, 576 threads: warp 0 TMA producer
// (3-stage ring of {X_hi, X_lo', Y_hi, Y_lo'} 128 x 64 tiles, 128-byte
// swizzle), warp 1 TMEM owner and MMA issuer, warps 2-17 epilogue (four per
// TMEM lane quadrant, 32 columns each).  Every wait is bounded; on timeout the
// CTA records an error word, drains its copies and MMAs, frees TMEM and leaves.
#include <cuda_fp16.h>

#include <cstring>

#include "common.cuh"
#include "hopf_internal.h"
#include "tc_ptx.cuh"

namespace hopf {
namespace syrk {
using namespace tcx;

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 3;
constexpr int TILE = BM * BK * 2;         // 16 KB
constexpr int STAGE = 4 * TILE;           // X_hi, X_lo', Y_hi, Y_lo'
constexpr int KSPLIT_KB = 64;             // k-blocks per work item (4,096 queries)
constexpr int CHUNK_KB = 8;               // k-blocks per promoted chunk (512 queries)
constexpr int EPI_WARPS = 16;
constexpr int NT = 64 + 32 * EPI_WARPS;
constexpr int CPW = BN / (EPI_WARPS / 4);  // columns per epilogue warp
constexpr float kLo = 2048.f;              // 2^11

struct Args {
  CUtensorMap mXh, mXl, mYh, mYl;  // [n_pad][K_pad] FP16, K = query
  float* part;                     // [nsplit][n_pad][n_pad] partial products
  int np, nt, nsplit, nkb, ntiles, items;
  int* err;
  long long wait_limit;
};

struct Smem {
  uint64_t full[STAGES], empty[STAGES], cfull[3], cempty[3], dfull, dempty, drain;
  uint32_t tmem_base;
  int abort;
};

// item -> (tile row ti <= tile column tj, K range sp); the K range is slowest
__device__ __forceinline__ void item_of(const Args& a, int it, int& ti, int& tj, int& sp) {
  sp = it / a.ntiles;
  int rem = it - sp * a.ntiles, I = 0;
  while (rem >= a.nt - I) {
    rem -= a.nt - I;
    ++I;
  }
  ti = I;
  tj = I + rem;
}

__device__ __forceinline__ void kb_range(const Args& a, int sp, int& kb0, int& kb1) {
  kb0 = sp * KSPLIT_KB;
  kb1 = min(a.nkb, kb0 + KSPLIT_KB);
}

__device__ __forceinline__ bool wait_(uint32_t bar, uint32_t par, const Args& a, Smem& S) {
  return mbar_wait_lim(bar, par, a.err, &S.abort, a.wait_limit);
}

__global__ void __launch_bounds__(NT, 1) k_syrk_tc(const __grid_constant__ Args a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* stages = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Smem& S = *reinterpret_cast<Smem*>(stages + STAGES * STAGE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(sa(&S.full[s]), 1);
      mbar_init(sa(&S.empty[s]), 1);
    }
    for (int c = 0; c < 3; ++c) {
      mbar_init(sa(&S.cfull[c]), 1);
      mbar_init(sa(&S.cempty[c]), EPI_WARPS);
    }
    mbar_init(sa(&S.dfull), 1);
    mbar_init(sa(&S.dempty), EPI_WARPS);
    mbar_init(sa(&S.drain), 1);
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(sa(&S.tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();

  // producer state (for the drain)
  uint32_t p_st = 0, last_par[STAGES] = {0, 0, 0};
  bool used[STAGES] = {false, false, false};
  bool issued = false;

  if (warp == 0) {
    if (lane == 0) {
      for (int it = blockIdx.x; it < a.items && !S.abort; it += gridDim.x) {
        int ti, tj, sp, kb0, kb1;
        item_of(a, it, ti, tj, sp);
        kb_range(a, sp, kb0, kb1);
        bool ok = true;
        for (int kb = kb0; kb < kb1; ++kb, ++p_st) {
          const uint32_t s = p_st % STAGES, use = p_st / STAGES;
          if (!(ok = wait_(sa(&S.empty[s]), (use & 1) ^ 1, a, S))) break;
          const uint32_t full = sa(&S.full[s]);
          mbar_expect_tx(full, STAGE);
          const uint32_t base = sa(stages + (size_t)s * STAGE);
          tma_load(base, &a.mXh, full, kb * BK, ti * BM);
          tma_load(base + TILE, &a.mXl, full, kb * BK, ti * BM);
          tma_load(base + 2 * TILE, &a.mYh, full, kb * BK, tj * BN);
          tma_load(base + 3 * TILE, &a.mYl, full, kb * BK, tj * BN);
          last_par[s] = use & 1;
          used[s] = true;
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_f16_mn(0, BM, BN);
      uint32_t m_st = 0, rot = 0, ce[3] = {0, 0, 0}, de = 0;
      for (int it = blockIdx.x; it < a.items && !S.abort; it += gridDim.x) {
        int ti, tj, sp, kb0, kb1;
        item_of(a, it, ti, tj, sp);
        kb_range(a, sp, kb0, kb1);
        if (!wait_(sa(&S.dempty), (de & 1) ^ 1, a, S)) break;
        ++de;
        tc_fence_after();
        const uint32_t d2 = S.tmem_base + 384;
        uint32_t slot = 0, d1 = 0;
        bool ok = true;
        for (int kb = kb0; kb < kb1; ++kb, ++m_st) {
          const int local = kb - kb0;
          if (local % CHUNK_KB == 0) {
            slot = rot % 3;
            if (!(ok = wait_(sa(&S.cempty[slot]), (ce[slot] & 1) ^ 1, a, S))) break;
            ++ce[slot];
            tc_fence_after();
            d1 = S.tmem_base + slot * BN;
          }
          const uint32_t s = m_st % STAGES, use = m_st / STAGES;
          if (!(ok = wait_(sa(&S.full[s]), use & 1, a, S))) break;
          tc_fence_after();
          const uint32_t base = sa(stages + (size_t)s * STAGE);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint64_t x0 = smem_desc(base) + (uint64_t)(kk * 2);
            const uint64_t x1 = smem_desc(base + TILE) + (uint64_t)(kk * 2);
            const uint64_t y0 = smem_desc(base + 2 * TILE) + (uint64_t)(kk * 2);
            const uint64_t y1 = smem_desc(base + 3 * TILE) + (uint64_t)(kk * 2);
            mma_f16(d1, x0, y0, idesc, (local % CHUNK_KB == 0 && kk == 0) ? 0u : 1u);  // a chunk starts afresh
            mma_f16(d2, x0, y1, idesc, (local == 0 && kk == 0) ? 0u : 1u);
            mma_f16(d2, x1, y0, idesc, 1u);
          }
          issued = true;
          mma_commit(sa(&S.empty[s]));
          if (local % CHUNK_KB == CHUNK_KB - 1 || kb == kb1 - 1) {
            mma_commit(sa(&S.cfull[slot]));
            ++rot;
          }
        }
        if (!ok) break;
        mma_commit(sa(&S.dfull));
      }
    }
  } else {
    const int qd = warp & 3;
    const int jbase = ((warp - 2) >> 2) * CPW;
    const int rloc = qd * 32 + lane;
    const uint32_t lb = S.tmem_base + ((uint32_t)(qd * 32) << 16);
    uint32_t rot = 0, cf[3] = {0, 0, 0}, df = 0;
    for (int it = blockIdx.x; it < a.items; it += gridDim.x) {
      if (*((volatile int*)&S.abort)) break;
      int ti, tj, sp, kb0, kb1;
      item_of(a, it, ti, tj, sp);
      kb_range(a, sp, kb0, kb1);
      const int nch = (kb1 - kb0 + CHUNK_KB - 1) / CHUNK_KB;
      float acc[CPW];
#pragma unroll
      for (int j = 0; j < CPW; ++j) acc[j] = 0.f;
      bool good = true;
      for (int ch = 0; ch < nch; ++ch) {
        const uint32_t slot = rot % 3;
        ++rot;
        good = good && wait_(sa(&S.cfull[slot]), cf[slot] & 1, a, S);
        ++cf[slot];
        if (good) {
          tc_fence_after();
#pragma unroll
          for (int j0 = 0; j0 < CPW; j0 += 16) {
            float v[16];
            tmem_ld16(lb + slot * BN + jbase + j0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j0 + j] += v[j];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(sa(&S.cempty[slot]));
      }
      good = good && wait_(sa(&S.dfull), df & 1, a, S);
      ++df;
      if (good) {
        tc_fence_after();
#pragma unroll
        for (int j0 = 0; j0 < CPW; j0 += 16) {
          float v[16];
          tmem_ld16(lb + 384 + jbase + j0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j0 + j] += v[j] * (1.f / kLo);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(sa(&S.dempty));
      if (!good) break;
      float* dst = a.part + ((size_t)sp * a.np + (size_t)(ti * BM + rloc)) * a.np + tj * BN + jbase;
#pragma unroll
      for (int j0 = 0; j0 < CPW; j0 += 4)
        *reinterpret_cast<float4*>(dst + j0) = make_float4(acc[j0], acc[j0 + 1], acc[j0 + 2], acc[j0 + 3]);
    }
  }

  // drain: no copy or MMA of this CTA may be in flight when TMEM is freed
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < STAGES; ++s)
      if (used[s]) {
        const long long t0 = clock64();
        while (!mbar_test(sa(&S.full[s]), last_par[s]) && clock64() - t0 < (1ll << 31)) {
        }
      }
  }
  if (warp == 1 && lane == 0 && issued) {
    mma_commit(sa(&S.drain));
    const long long t0 = clock64();
    while (!mbar_test(sa(&S.drain), 0) && clock64() - t0 < (1ll << 31)) {
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(S.tmem_base) : "memory");
}

// A power of two s with s max|g| in [0.5, 1) (1 when g = 0): the scale that
// brings g V into FP16's range without rounding.
__global__ void k_syrk_gscale(const float* __restrict__ g, int64_t B, float* __restrict__ scale) {
  float m = 0.f;
  for (int64_t q = threadIdx.x; q < B; q += blockDim.x) m = fmaxf(m, fabsf(g[q]));
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    int e = 0;
    if (m > 0.f && isfinite(m)) frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
    *scale = ldexpf(1.f, -e);
  }
}

// Transposed two-term FP16 splits: X = s g_q V[q][i], Y = V[q][i] into
// planes [i][q] (i < n_pad, q < K_pad, zero padded).  32 x 32 tiles.
__global__ void k_syrk_prep(const float* __restrict__ g, const float* __restrict__ V, int n, int64_t B, int np,
                            int64_t kp, const float* __restrict__ scale, uint16_t* __restrict__ xh,
                            uint16_t* __restrict__ xl, uint16_t* __restrict__ yh, uint16_t* __restrict__ yl) {
  __shared__ float tv[32][33];
  __shared__ float tg[32];
  const int64_t q0 = (int64_t)blockIdx.x * 32;
  const int i0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t q = q0 + r;
    const int i = i0 + tx;
    tv[r][tx] = (q < B && i < n) ? V[q * n + i] : 0.f;
  }
  if (ty == 0) tg[tx] = q0 + tx < B ? g[q0 + tx] * *scale : 0.f;
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r;
    const int64_t q = q0 + tx;
    const float y = tv[tx][r];
    const float x = tg[tx] * y;
    const __half yh1 = __float2half_rn(y), xh1 = __float2half_rn(x);
    const size_t o = (size_t)i * kp + q;
    yh[o] = __half_as_ushort(yh1);
    yl[o] = __half_as_ushort(__float2half_rn((y - __half2float(yh1)) * kLo));
    xh[o] = __half_as_ushort(xh1);
    xl[o] = __half_as_ushort(__float2half_rn((x - __half2float(xh1)) * kLo));
  }
}

// g_A = -1/2 (1/s) sum over K ranges, FP64, each tile on or above the
// diagonal and its mirror.
// A bounded wait that gave up (err set) leaves NaN in g_A.
__global__ void k_syrk_reduce(const float* __restrict__ part, int nsplit, int n, int np, int nt,
                              const float* __restrict__ scale, const int* __restrict__ err, float* __restrict__ gA) {
  int rem = blockIdx.x, I = 0;
  while (rem >= nt - I) {
    rem -= nt - I;
    ++I;
  }
  const int J = I + rem;
  const double f = -0.5 / (double)*scale;
  const bool failed = *err != ERR_NONE;
  for (int e = threadIdx.x; e < BM * BN; e += blockDim.x) {
    // a diagonal tile gives its entries on and above the diagonal and their
    // mirrors (its two halves come from differently rounded operands), so
    // g_A is exactly symmetric
    if (I == J && e / BN > e % BN) continue;
    const int i = I * BM + e / BN, j = J * BN + e % BN;
    if (i >= n || j >= n) continue;
    double v = 0.0;
    for (int s = 0; s < nsplit; ++s) v += (double)part[((size_t)s * np + i) * np + j];
    const float o = failed ? __int_as_float(0x7fc00000) : (float)(v * f);
    gA[(size_t)i * n + j] = o;
    if (i != j) gA[(size_t)j * n + i] = o;
  }
}

}  // namespace syrk

static int64_t syrk_kpad(int64_t batch) { return round_up(batch > 0 ? batch : 1, syrk::BK); }
static int syrk_nsplit(int64_t batch) {
  return (int)((syrk_kpad(batch) / syrk::BK + syrk::KSPLIT_KB - 1) / syrk::KSPLIT_KB);
}

size_t syrk_workspace(const hopf_handle h, int64_t batch) {
  const size_t np = (size_t)h->n_pad, kp = (size_t)syrk_kpad(batch);
  return 4 * round_up(np * kp * 2, 256) + round_up((size_t)syrk_nsplit(batch) * np * np * 4, 256) + 256;
}

size_t syrk_smem_bytes() { return 1024 + (size_t)syrk::STAGES * syrk::STAGE + sizeof(syrk::Smem); }

hopf_status syrk_prepare() {
  static bool done[256] = {};
  int dev = 0;
  HOPF_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 256 && !done[dev]) {
    HOPF_CUDA(cudaFuncSetAttribute(syrk::k_syrk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)syrk_smem_bytes()));
    done[dev] = true;
  }
  return HOPF_OK;
}

hopf_status backward_dense_tc(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, float* g_A,
                              void* ws, size_t ws_bytes, cudaStream_t stream) {
  using namespace syrk;
  if (ws_bytes < syrk_workspace(h, batch)) return fail(HOPF_EINVAL, "hopf_backward_ws: workspace too small");
  if (((uintptr_t)ws & 255) != 0) return fail(HOPF_EINVAL, "hopf_backward_ws: workspace must be 256-byte aligned");
  const int n = h->n, np = h->n_pad;
  const int64_t kp = syrk_kpad(batch);
  char* p = (char*)ws;
  const size_t plane = round_up((size_t)np * kp * 2, 256);
  uint16_t* xh = (uint16_t*)p;
  uint16_t* xl = (uint16_t*)(p + plane);
  uint16_t* yh = (uint16_t*)(p + 2 * plane);
  uint16_t* yl = (uint16_t*)(p + 3 * plane);
  float* part = (float*)(p + 4 * plane);
  const int nsplit = syrk_nsplit(batch);
  float* scale = (float*)(p + 4 * plane + round_up((size_t)nsplit * np * np * 4, 256));
  {
    const hopf_status st = syrk_prepare();
    if (st != HOPF_OK) return st;
  }
  k_syrk_gscale<<<1, 1024, 0, stream>>>(g_phi, batch, scale);
  dim3 pg((unsigned)(kp / 32), (unsigned)(np / 32));
  k_syrk_prep<<<pg, 256, 0, stream>>>(g_phi, vstar, n, batch, np, kp, scale, xh, xl, yh, yl);
  HOPF_CUDA(cudaGetLastError());
  Args a;
  memset(&a, 0, sizeof(a));
  if (!tc_encode_f16(&a.mXh, xh, np, kp) || !tc_encode_f16(&a.mXl, xl, np, kp) ||
      !tc_encode_f16(&a.mYh, yh, np, kp) || !tc_encode_f16(&a.mYl, yl, np, kp))
    return fail(HOPF_ECUDA, "cuTensorMapEncodeTiled failed");
  a.part = part;
  a.np = np;
  a.nt = np / BM;
  a.nsplit = nsplit;
  a.nkb = (int)(kp / BK);
  a.ntiles = a.nt * (a.nt + 1) / 2;
  a.items = a.ntiles * nsplit;
  a.err = (int*)(scale + 1);
  a.wait_limit = h->wait_limit > 0 ? h->wait_limit : kWaitLimitCycles;
  HOPF_CUDA(cudaMemsetAsync(a.err, 0, sizeof(int), stream));
  const int grid = a.items < h->num_sms ? a.items : h->num_sms;
  k_syrk_tc<<<grid, NT, syrk_smem_bytes(), stream>>>(a);
  HOPF_CUDA(cudaGetLastError());
  k_syrk_reduce<<<(unsigned)a.ntiles, 256, 0, stream>>>(part, nsplit, n, np, a.nt, scale, a.err, g_A);
  HOPF_CUDA(cudaGetLastError());
  return HOPF_OK;
}

}  // namespace hopf
