// Shared device helpers for the Hopf-formula kernels (sm_103a).
//
// The method (Darbon & Osher, Section 3.1) evaluates
//   phi(x,t) = -min_v { J*(v) + t H(v) - <x,v> }            (eq. 3.3)
// by split Bregman (eq. 3.4(a)-(c)).  With J(x) = 1/2 (x-c)^T A^{-1} (x-c) - c0
// the v-update is v = (A + lambda I)^{-1} (y + lambda (d - b)), y = x - c, and
// the d-update is the prox of (t/lambda) H: shrink_1 per coordinate (l1,
// weighted l1) or shrink_2 (l2), both defined in Section 1.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hopf {

enum : int { H_L1 = 0, H_WL1 = 1, H_L2 = 2, H_LINF = 3, H_DNORM = 4, H_ANORM = 5 };
enum : int { J_QUAD = 0, J_L1SQ = 2, J_LINFSQ = 3 };
enum : int { STOP_PAPER = 0, STOP_UREL = 1 };
enum : uint8_t { Q_OK = 0, Q_NOT_CONVERGED = 1, Q_NONFINITE = 2, Q_ABORTED = 3, Q_BAD_INPUT = 4 };

// Error words a kernel can leave in its device error flag (never a trap).
enum : int { ERR_NONE = 0, ERR_BARRIER_TIMEOUT = 1, ERR_MBAR_TIMEOUT = 2, ERR_NOT_SPD = 3, ERR_TMEM = 4 };

// shrink_1(z, a): z - a if z > a, 0 if |z| <= a, z + a if z < -a (Section 1).
template <typename T>
__device__ __forceinline__ T shrink1(T z, T a) {
  return z > a ? z - a : (z < -a ? z + a : T(0));
}

// Scale s of shrink_2(z, tau) = s z with s = max(|z| - tau, 0)/|z| (0 at z = 0).
template <typename T>
__device__ __forceinline__ T shrink2_scale(T norm, T tau) {
  return norm > T(0) ? (norm > tau ? (norm - tau) / norm : T(0)) : T(0);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Default limit of every bounded device-side wait, in SM clock cycles (about
// two seconds at 2 GHz); a handle may set its own (hopf_set_wait_limit).
constexpr long long kWaitLimitCycles = 1ll << 32;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).
// bar[0] counts arrivals, bar[1] is the generation.  The wait is bounded by
// `limit` clock cycles: on timeout the CTA records ERR_BARRIER_TIMEOUT in *err
// and returns false, and the caller leaves its loop; nothing spins forever.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* err,
                                             long long limit = kWaitLimitCycles) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    s_ok = 1;
    unsigned gen = ld_acquire_u32(bar + 1);
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == nblocks) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      const long long t0 = clock64();
      while (ld_acquire_u32(bar + 1) == gen) {
        ++spins;
        if (clock64() - t0 > limit) {
          atomicExch(err, ERR_BARRIER_TIMEOUT);
          s_ok = 0;
          break;
        }
        if ((spins & 255u) == 0 && *((volatile int*)err) != ERR_NONE) {
          s_ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*((volatile int*)err) != ERR_NONE) s_ok = 0;
  }
  __syncthreads();
  return s_ok != 0;
}

__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

}  // namespace hopf
