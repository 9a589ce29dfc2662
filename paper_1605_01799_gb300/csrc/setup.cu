// Dense setup, once per handle: M = (A + lambda I)^{-1} on the GPU (FP64 for
// the forms that apply it as the paper's v-update, FP32 where it only
// preconditions the defect correction), then the padded copies each precision
// needs.
//
// The v-update of eq. 3.4(a) is the prox of the quadratic J*: with
// J*(v) = 1/2 v^T A v + <c,v> + c0 it solves (A + lambda I) v = y + lambda (d - b)
// (Section 3.1: the resolvent of 1/2 <., A .> is (I + alpha A)^{-1}).  Forming
// the inverse once turns every later v-update into a matrix product.
//
// Inverse by the symmetric sweep operator: sweeping pivot k maps S to S' with
//   S'_kk = -1/S_kk,  S'_kj = S_kj/S_kk,  S'_ik = S_ik/S_kk,
//   S'_ij = S_ij - S_ik S_kj / S_kk            (i, j != k),
// and sweeping every pivot of an SPD matrix yields -S^{-1}.  The pivots are the
// Schur complements, so a non-positive pivot proves A + lambda I is not SPD.
// The pivots go 64 at a time (a block sweep): n / 64 rounds of three
// launches, the bulk of the 2 n^3 FP64 flop in a symmetric rank-64 update.
//
// Device memory of a handle comes from cudaMalloc, or from the allocator the
// caller installed with hopf_set_allocator (captured by each handle, which
// frees with it).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "common.cuh"
#include "hopf_internal.h"

namespace hopf {

template <typename T>
__global__ void k_load_shifted(const double* __restrict__ A, T* __restrict__ S, int n, double lam) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  int i = (int)(idx / n), j = (int)(idx % n);
  // symmetrise the input: the method assumes A symmetric
  double a = 0.5 * (A[(int64_t)i * n + j] + A[(int64_t)j * n + i]);
  S[idx] = (T)(a + (i == j ? lam : 0.0));
}

// ---- blocked sweep ----------------------------------------------------------
// Sweeping a block K of pivots at once is the composition of its single-pivot
// sweeps:
//   S'_KK = -S_KK^{-1},  S'_KJ = S_KK^{-1} S_KJ,  S'_IK = S_IK S_KK^{-1},
//   S'_IJ = S_IJ - S_IK S_KK^{-1} S_KJ = S_IJ - S_KI^T T_KJ  (T = S_KK^{-1} S_K:),
// which keeps S symmetric.  Per block of kSB pivots: one CTA sweeps the pivot
// block in shared memory (checking each pivot), a second kernel forms T and
// keeps the old rows of K, and a third applies the rank-kSB update to the
// tiles on and above the diagonal, writing each tile and its mirror.
constexpr int kSB = 64;  // pivots per block = tile edge of the update

// Sweep the pivots of the diagonal block K = [k0, k0 + nb) in shared memory;
// out = -S_KK^{-1} (nb x nb, leading dimension kSB).
template <typename T>
__global__ void __launch_bounds__(256) k_sweep_block_inv(const T* __restrict__ S, int n, int k0, int nb,
                                                         T* __restrict__ out, int* err) {
  __shared__ T B[kSB][kSB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    B[i][j] = S[(int64_t)(k0 + i) * n + k0 + j];
  }
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    const T dkk = B[k][k];
    if (!(dkk > T(0))) {  // a Schur-complement pivot of A + lambda I: not SPD
      if (threadIdx.x == 0) {
        bad = 1;
        atomicExch(err, ERR_NOT_SPD);
      }
      break;  // dkk is the same for every thread: all leave together
    }
    const T inv = T(1) / dkk;
    // each thread owns the entries e = threadIdx.x + 256 r (static indices:
    // the new values stay in registers until every thread has read the old)
    constexpr int R = kSB * kSB / 256;
    T nv[R];
    if (nb == kSB) {
      // a full block: entry e is row (tid >> 6) + 4 r, column tid & 63, so
      // no index arithmetic runs per pivot (the same operations as below)
      const int j = threadIdx.x & (kSB - 1), i0 = threadIdx.x >> 6;
      const T bkj = B[k][j];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int i = i0 + 4 * r;
        if (i == k && j == k) nv[r] = -inv;
        else if (i == k) nv[r] = bkj * inv;
        else if (j == k) nv[r] = B[i][k] * inv;
        else nv[r] = B[i][j] - B[i][k] * bkj * inv;
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < R; ++r) B[i0 + 4 * r][j] = nv[r];
      __syncthreads();
      continue;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = threadIdx.x + 256 * r;
      nv[r] = T(0);
      if (e < nb * nb) {
        const int i = e / nb, j = e % nb;
        if (i == k && j == k) nv[r] = -inv;
        else if (i == k) nv[r] = B[k][j] * inv;
        else if (j == k) nv[r] = B[i][k] * inv;
        else nv[r] = B[i][j] - B[i][k] * B[k][j] * inv;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int e = threadIdx.x + 256 * r;
      if (e < nb * nb) B[e / nb][e % nb] = nv[r];
    }
    __syncthreads();
  }
  if (bad) return;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) out[(e / nb) * kSB + e % nb] = B[e / nb][e % nb];
}

// T[:, J] = -Kneg S[K, J] for one 64-column tile J (T = S_KK^{-1} S_K:), and the
// old rows of K kept in Sold.  Both nb x n, leading dimension n.
template <typename E>
__global__ void __launch_bounds__(256) k_sweep_block_T(const E* __restrict__ S, int n, int k0, int nb,
                                                       const E* __restrict__ Kneg, E* __restrict__ T,
                                                       E* __restrict__ Sold, const int* err) {
  if (*((volatile const int*)err) != ERR_NONE) return;
  __shared__ E Sk[kSB][kSB + 1];
  const int j0 = blockIdx.x * kSB;
  const int w = min(kSB, n - j0);
  for (int e = threadIdx.x; e < nb * kSB; e += blockDim.x) {
    const int k = e / kSB, j = e % kSB;
    const E v = j < w ? S[(int64_t)(k0 + k) * n + j0 + j] : E(0);
    Sk[k][j] = v;
    if (j < w) Sold[(int64_t)k * n + j0 + j] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nb * kSB; e += blockDim.x) {
    const int i = e / kSB, j = e % kSB;
    if (j >= w) continue;
    E acc = E(0);
    for (int k = 0; k < nb; ++k) acc += __ldg(Kneg + i * kSB + k) * Sk[k][j];
    T[(int64_t)i * n + j0 + j] = -acc;
  }
}

// Rank-nb update of tile (I, J), I <= J, 64 x 64, with its mirror (J, I):
//   I, J != K:  S_IJ -= Sold_K,I^T T_K,J
//   J == K:     S_IK = T_K,I^T  (I != K);  S_KK = Kneg
// Each thread owns a 4 x 4 block of the tile.
template <typename E>
__global__ void __launch_bounds__(256) k_sweep_block_update(E* __restrict__ S, int n, int kt, int nb,
                                                            const E* __restrict__ Kneg,
                                                            const E* __restrict__ T,
                                                            const E* __restrict__ Sold, const int* err) {
  if (*((volatile const int*)err) != ERR_NONE) return;
  // blockIdx.x enumerates the tiles on and above the diagonal, row by row
  const int nt = (n + kSB - 1) / kSB;
  int I = 0, rem = blockIdx.x;
  while (rem >= nt - I) {
    rem -= nt - I;
    ++I;
  }
  const int J = I + rem;
  const int i0 = I * kSB, j0 = J * kSB;
  const int hi = min(kSB, n - i0), wj = min(kSB, n - j0);
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  E out[4][4];
  if (I == kt || J == kt) {
    // row / column block K: copies of T (or -S_KK^{-1} on the diagonal)
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = 4 * ty + r, j = 4 * tx + c;
        E v = E(0);
        if (i < hi && j < wj) {
          if (I == kt && J == kt) v = Kneg[i * kSB + j];
          else if (I == kt) v = T[(int64_t)i * n + j0 + j];  // S_KJ = T_KJ
          else v = T[(int64_t)j * n + i0 + i];                // S_IK = T_KI^T
        }
        out[r][c] = v;
      }
  } else {
    constexpr int KC = 32;            // k rows staged per round (32 KB of shared memory)
    __shared__ E As[KC][kSB];    // As[k][i] = Sold[kc + k][i0 + i]
    __shared__ E Bs[KC][kSB];    // Bs[k][j] = T[kc + k][j0 + j]
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = 4 * ty + r, j = 4 * tx + c;
        out[r][c] = (i < hi && j < wj) ? S[(int64_t)(i0 + i) * n + j0 + j] : E(0);
      }
    for (int kc = 0; kc < nb; kc += KC) {
      __syncthreads();
      for (int e = threadIdx.x; e < KC * kSB; e += blockDim.x) {
        const int k = e / kSB, c = e % kSB;
        const bool kin = kc + k < nb;
        As[k][c] = (kin && c < hi) ? Sold[(int64_t)(kc + k) * n + i0 + c] : E(0);
        Bs[k][c] = (kin && c < wj) ? T[(int64_t)(kc + k) * n + j0 + c] : E(0);
      }
      __syncthreads();
      for (int k = 0; k < KC; ++k) {
        E a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = As[k][4 * ty + r];
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = Bs[k][4 * tx + c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) out[r][c] = fma(-a[r], b[c], out[r][c]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int i = 4 * ty + r, j = 4 * tx + c;
      if (i < hi && j < wj) {
        S[(int64_t)(i0 + i) * n + j0 + j] = out[r][c];
        if (I != J) S[(int64_t)(j0 + j) * n + i0 + i] = out[r][c];
      }
    }
}

// M = -(swept) symmetrised, padded to np x np with zeros; FP32/BF16 copies
// and (SPLIT form) the two-term FP16 split M = hi + lo * 2^-11 with
// hi = fp16(M), lo = fp16((M - hi) 2^11).
template <typename T>
__global__ void k_finish_inverse(const T* __restrict__ S, double* __restrict__ M64, float* __restrict__ M32,
                                 uint16_t* __restrict__ Mbf, uint16_t* __restrict__ Mh, uint16_t* __restrict__ Ml,
                                 int n, int np) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)np * np) return;
  int i = (int)(idx / np), j = (int)(idx % np);
  double m = 0.0;
  if (i < n && j < n) m = -0.5 * ((double)S[(int64_t)i * n + j] + (double)S[(int64_t)j * n + i]);
  if (M64) M64[idx] = m;
  if (M32) M32[idx] = (float)m;
  if (Mbf) Mbf[idx] = __bfloat16_as_ushort(__double2bfloat16(m));
  if (Mh) {
    const __half hi = __double2half(m);
    Mh[idx] = __half_as_ushort(hi);
    Ml[idx] = __half_as_ushort(__double2half((m - (double)__half2float(hi)) * 2048.0));
  }
}

// Copies of A: FP32, BF16, and the three-term FP16 split
// A = hi + lo * 2^-11 + lo2 * 2^-22 with hi = fp16(A), lo = fp16((A - hi) 2^11),
// lo2 = fp16((A - hi - lo 2^-11) 2^22), padded with zeros.
__global__ void k_cast_A(const double* __restrict__ A, float* __restrict__ A32, uint16_t* __restrict__ Abf,
                         uint16_t* __restrict__ Ah, uint16_t* __restrict__ Al, uint16_t* __restrict__ Al2, int n,
                         int np) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)np * np) return;
  int i = (int)(idx / np), j = (int)(idx % np);
  double a = 0.0;
  if (i < n && j < n) a = 0.5 * (A[(int64_t)i * n + j] + A[(int64_t)j * n + i]);
  if (A32) A32[idx] = (float)a;
  if (Abf) Abf[idx] = __bfloat16_as_ushort(__double2bfloat16(a));
  if (Ah) {
    const __half hi = __double2half(a);
    const double r1 = a - (double)__half2float(hi);
    const __half lo = __double2half(r1 * 2048.0);
    const double r2 = r1 - (double)__half2float(lo) / 2048.0;
    Ah[idx] = __half_as_ushort(hi);
    Al[idx] = __half_as_ushort(lo);
    Al2[idx] = __half_as_ushort(__double2half(r2 * 4194304.0));
  }
}

static std::mutex g_alloc_mu;
static Allocator g_alloc = {nullptr, nullptr, nullptr};

hopf_status set_allocator(hopf_alloc_fn alloc, hopf_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(HOPF_EINVAL, "hopf_set_allocator: give both functions, or neither (cudaMalloc / cudaFree)");
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc = {alloc, release, ctx};
  return HOPF_OK;
}

Allocator current_allocator() {
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  return g_alloc;
}

cudaError_t dev_alloc(const Allocator& a, void** p, size_t bytes) {
  if (!a.alloc) return cudaMalloc(p, bytes);
  *p = a.alloc(bytes, a.ctx);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

void dev_free(const Allocator& a, void* p) {
  if (!p) return;
  if (a.release) a.release(p, a.ctx);
  else cudaFree(p);
}

// The block sweep of A + lambda I in element type T into S (n x n); err
// receives ERR_NOT_SPD at a non-positive pivot.  Buffers as in dense_setup.
template <typename T>
static cudaError_t sweep_inverse(const double* dA, int n, double lam, void* S, void* Tm, void* Sold, void* Kneg,
                                 int* err, cudaStream_t stream) {
  const size_t nn = (size_t)n * n;
  const int tb = 256;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  k_load_shifted<T><<<(unsigned)((nn + tb - 1) / tb), tb, 0, stream>>>(dA, (T*)S, n, lam);
  const int nt = (n + kSB - 1) / kSB;
  const unsigned upper = (unsigned)(nt * (nt + 1) / 2);
  for (int kt = 0; kt < nt; ++kt) {
    const int k0 = kt * kSB, nb = n - k0 < kSB ? n - k0 : kSB;
    k_sweep_block_inv<T><<<1, 256, 0, stream>>>((const T*)S, n, k0, nb, (T*)Kneg, err);
    k_sweep_block_T<T><<<(unsigned)nt, 256, 0, stream>>>((const T*)S, n, k0, nb, (const T*)Kneg, (T*)Tm, (T*)Sold,
                                                         err);
    k_sweep_block_update<T><<<upper, 256, 0, stream>>>((T*)S, n, kt, nb, (const T*)Kneg, (const T*)Tm,
                                                       (const T*)Sold, err);
  }
  return cudaGetLastError();
}

hopf_status dense_setup(hopf_handle h, const double* A_host, cudaStream_t stream) {
  const int n = h->n, np = h->n_pad;
  const size_t nn = (size_t)n * n, pp = (size_t)np * np;
  const Allocator& al = h->alloc;
  double *S0 = nullptr, *Tm = nullptr, *Sold = nullptr, *Kneg = nullptr;
  int* err = nullptr;
  hopf_status st = HOPF_OK;
  auto cleanup = [&]() {
    dev_free(al, S0);
    dev_free(al, Tm);
    dev_free(al, Sold);
    dev_free(al, Kneg);
    dev_free(al, err);
  };
#define S_CALL(call)                   \
  do {                                 \
    cudaError_t e_ = (call);           \
    if (e_ != cudaSuccess) {           \
      cleanup();                       \
      return cuda_fail(e_, #call);     \
    }                                  \
  } while (0)
#define S_ALLOC(ptr, bytes) S_CALL(dev_alloc(al, (void**)&(ptr), (bytes)))
  S_ALLOC(h->d_A, nn * sizeof(double));
  S_CALL(cudaMemcpyAsync(h->d_A, A_host, nn * sizeof(double), cudaMemcpyHostToDevice, stream));
  S_ALLOC(S0, nn * sizeof(double));
  S_ALLOC(Tm, (size_t)kSB * n * sizeof(double));
  S_ALLOC(Sold, (size_t)kSB * n * sizeof(double));
  S_ALLOC(Kneg, (size_t)kSB * kSB * sizeof(double));
  S_ALLOC(err, sizeof(int));
  // M in FP32 where it only preconditions: the MIXED form's fixed point
  // (g = y - A p - lambda (u - p) = 0) uses A itself, and the BF16 form
  // rounds M to BF16; the FP32 and SPLIT forms apply M as the paper's
  // v-update, so their M comes from the FP64 sweep.  A non-positive FP32
  // pivot is checked again in FP64 before the handle reports HOPF_ENOTSPD.
  bool f32 = h->precision == HOPF_P_MIXED || h->precision == HOPF_P_BF16;
  int herr = 0;
  for (;;) {
    S_CALL(f32 ? sweep_inverse<float>(h->d_A, n, h->lambda, S0, Tm, Sold, Kneg, err, stream)
               : sweep_inverse<double>(h->d_A, n, h->lambda, S0, Tm, Sold, Kneg, err, stream));
    S_CALL(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    S_CALL(cudaStreamSynchronize(stream));
    if (herr != ERR_NOT_SPD || !f32) break;
    f32 = false;
  }
  if (herr == ERR_NOT_SPD) {
    cleanup();
    return fail(HOPF_ENOTSPD, "hopf_create: A + lambda I is not symmetric positive definite");
  }
  const int tb = 256;
  const bool simt = h->precision == HOPF_P_FP32;
  S_ALLOC(h->d_M32, pp * sizeof(float));
  S_ALLOC(h->d_A32, pp * sizeof(float));
  if (!simt) {
    S_ALLOC(h->d_Mbf, pp * sizeof(uint16_t));
    S_ALLOC(h->d_Ah16, pp * sizeof(uint16_t));
    S_ALLOC(h->d_Al16, pp * sizeof(uint16_t));
    S_ALLOC(h->d_Al2, pp * sizeof(uint16_t));
    S_ALLOC(h->d_Abf, pp * sizeof(uint16_t));
  }
  // the FP16 split of M: the SPLIT form, and the SPLIT first stage of MIXED
  // (l1, weighted l1)
  if (h->precision == HOPF_P_SPLIT || (h->precision == HOPF_P_MIXED && h->h_kind != HOPF_H_L2)) {
    S_ALLOC(h->d_Mh16, pp * sizeof(uint16_t));
    S_ALLOC(h->d_Ml16, pp * sizeof(uint16_t));
  }
  if (f32)
    k_finish_inverse<float><<<(unsigned)((pp + tb - 1) / tb), tb, 0, stream>>>((const float*)S0, nullptr, h->d_M32,
                                                                              h->d_Mbf, h->d_Mh16, h->d_Ml16, n, np);
  else
    k_finish_inverse<double><<<(unsigned)((pp + tb - 1) / tb), tb, 0, stream>>>(S0, nullptr, h->d_M32, h->d_Mbf,
                                                                               h->d_Mh16, h->d_Ml16, n, np);
  k_cast_A<<<(unsigned)((pp + tb - 1) / tb), tb, 0, stream>>>(h->d_A, h->d_A32, h->d_Abf, h->d_Ah16, h->d_Al16,
                                                               h->d_Al2, n, np);
  S_CALL(cudaGetLastError());
  S_CALL(cudaStreamSynchronize(stream));
  cleanup();
#undef S_ALLOC
#undef S_CALL
  return st;
}

}  // namespace hopf
