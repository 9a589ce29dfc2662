// Dense setup, once per handle: M = (A + lambda I)^{-1} in FP64 on the GPU,
// then the padded copies each precision needs.
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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "hopf_internal.h"

namespace hopf {

__global__ void k_load_shifted(const double* __restrict__ A, double* __restrict__ S, int n, double lam) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * n) return;
  int i = (int)(idx / n), j = (int)(idx % n);
  // symmetrise the input: the method assumes A symmetric
  double a = 0.5 * (A[(int64_t)i * n + j] + A[(int64_t)j * n + i]);
  S[idx] = a + (i == j ? lam : 0.0);
}

__global__ void k_sweep(const double* __restrict__ S, double* __restrict__ D, int n, int k, int* err) {
  if (*((volatile int*)err) != ERR_NONE) return;
  const double dkk = S[(int64_t)k * n + k];
  if (!(dkk > 0.0)) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) atomicExch(err, ERR_NOT_SPD);
    return;
  }
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const double inv = 1.0 / dkk;
  const double aik = S[(int64_t)i * n + k], akj = S[(int64_t)k * n + j];
  double out;
  if (i == k && j == k) out = -inv;
  else if (i == k) out = akj * inv;
  else if (j == k) out = aik * inv;
  else out = S[(int64_t)i * n + j] - aik * akj * inv;
  D[(int64_t)i * n + j] = out;
}

// M = -(swept) symmetrised, padded to np x np with zeros; FP32/BF16 copies
// and (SPLIT form) the two-term FP16 split M = hi + lo * 2^-11 with
// hi = fp16(M), lo = fp16((M - hi) 2^11).
__global__ void k_finish_inverse(const double* __restrict__ S, double* __restrict__ M64, float* __restrict__ M32,
                                 uint16_t* __restrict__ Mbf, uint16_t* __restrict__ Mh, uint16_t* __restrict__ Ml,
                                 int n, int np) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)np * np) return;
  int i = (int)(idx / np), j = (int)(idx % np);
  double m = 0.0;
  if (i < n && j < n) m = -0.5 * (S[(int64_t)i * n + j] + S[(int64_t)j * n + i]);
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

hopf_status dense_setup(hopf_handle h, const double* A_host, cudaStream_t stream) {
  const int n = h->n, np = h->n_pad;
  const size_t nn = (size_t)n * n, pp = (size_t)np * np;
  double *S0 = nullptr, *S1 = nullptr;
  int* err = nullptr;
  hopf_status st = HOPF_OK;
  auto cleanup = [&]() {
    if (S0) cudaFree(S0);
    if (S1) cudaFree(S1);
    if (err) cudaFree(err);
  };
#define S_CALL(call)                   \
  do {                                 \
    cudaError_t e_ = (call);           \
    if (e_ != cudaSuccess) {           \
      cleanup();                       \
      return cuda_fail(e_, #call);     \
    }                                  \
  } while (0)
  S_CALL(cudaMalloc(&h->d_A, nn * sizeof(double)));
  S_CALL(cudaMemcpyAsync(h->d_A, A_host, nn * sizeof(double), cudaMemcpyHostToDevice, stream));
  S_CALL(cudaMalloc(&S0, nn * sizeof(double)));
  S_CALL(cudaMalloc(&S1, nn * sizeof(double)));
  S_CALL(cudaMalloc(&err, sizeof(int)));
  S_CALL(cudaMemsetAsync(err, 0, sizeof(int), stream));
  const int tb = 256;
  k_load_shifted<<<(unsigned)((nn + tb - 1) / tb), tb, 0, stream>>>(h->d_A, S0, n, h->lambda);
  dim3 blk(32, 8), grd((n + 31) / 32, (n + 7) / 8);
  for (int k = 0; k < n; ++k) {
    k_sweep<<<grd, blk, 0, stream>>>(S0, S1, n, k, err);
    double* tmp = S0;
    S0 = S1;
    S1 = tmp;
  }
  S_CALL(cudaGetLastError());
  int herr = 0;
  S_CALL(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  S_CALL(cudaStreamSynchronize(stream));
  if (herr == ERR_NOT_SPD) {
    cleanup();
    return fail(HOPF_ENOTSPD, "hopf_create: A + lambda I is not symmetric positive definite");
  }
  const bool simt = h->precision == HOPF_P_FP32;
  S_CALL(cudaMalloc(&h->d_M32, pp * sizeof(float)));
  S_CALL(cudaMalloc(&h->d_A32, pp * sizeof(float)));
  if (!simt) {
    S_CALL(cudaMalloc(&h->d_Mbf, pp * sizeof(uint16_t)));
    S_CALL(cudaMalloc(&h->d_Ah16, pp * sizeof(uint16_t)));
    S_CALL(cudaMalloc(&h->d_Al16, pp * sizeof(uint16_t)));
    S_CALL(cudaMalloc(&h->d_Al2, pp * sizeof(uint16_t)));
    S_CALL(cudaMalloc(&h->d_Abf, pp * sizeof(uint16_t)));
  }
  if (h->precision == HOPF_P_SPLIT) {
    S_CALL(cudaMalloc(&h->d_Mh16, pp * sizeof(uint16_t)));
    S_CALL(cudaMalloc(&h->d_Ml16, pp * sizeof(uint16_t)));
  }
  k_finish_inverse<<<(unsigned)((pp + tb - 1) / tb), tb, 0, stream>>>(S0, nullptr, h->d_M32, h->d_Mbf, h->d_Mh16,
                                                                       h->d_Ml16, n, np);
  k_cast_A<<<(unsigned)((pp + tb - 1) / tb), tb, 0, stream>>>(h->d_A, h->d_A32, h->d_Abf, h->d_Ah16, h->d_Al16,
                                                               h->d_Al2, n, np);
  S_CALL(cudaGetLastError());
  S_CALL(cudaStreamSynchronize(stream));
  cleanup();
#undef S_CALL
  return st;
}

}  // namespace hopf
