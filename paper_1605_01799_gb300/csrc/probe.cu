// Throughput probes of the pipes the solvers run on, for roofline
// denominators measured on the GPU at hand (the paper has no counterpart).
//
//   FP32: chains of fused multiply-adds, 8 independent chains per thread and
//         enough warps per SM to cover the FMA latency: 2 flop per FMA.
//   FP64: the same with doubles.
//   L2:   repeated streaming reads of a buffer that fits in L2 (32 MiB, a
//         quarter of GB300's), 16-byte loads, summed so that nothing is
//         optimised away.
//
// Every kernel runs a fixed amount of work: nothing waits on anything else.
#include "common.cuh"
#include "hopf_internal.h"

namespace hopf {

constexpr int kProbeChains = 8;

template <typename T>
__global__ void __launch_bounds__(512) k_probe_fma(int iters, T m, T c, T* out) {
  T acc[kProbeChains];
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) acc[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < kProbeChains; ++j) acc[j] = fma(acc[j], m, c);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < kProbeChains; ++j) s += acc[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(512) k_probe_l2(const float4* __restrict__ buf, size_t n4, int passes,
                                                  float* out) {
  float s = 0.f;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      s += v.x + v.y + v.z + v.w;
    }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

size_t probe_scratch_bytes() { return ((size_t)32 << 20) + ((size_t)4 << 20); }

hopf_status measure_pipes(void* scratch, size_t bytes, double* fp32_tflops, double* fp64_tflops, double* l2_gbs,
                          cudaStream_t stream) {
  if (bytes < probe_scratch_bytes()) return fail(HOPF_EINVAL, "hopf_measure_pipes: scratch too small");
  int dev = 0;
  HOPF_CUDA(cudaGetDevice(&dev));
  const int sms = sm_count(dev);
  const int blocks = sms * 4, threads = 512;  // 64 warps per SM
  char* base = (char*)scratch;
  const size_t l2_bytes = (size_t)32 << 20;
  float* outf = (float*)(base + l2_bytes);
  double* outd = (double*)(base + l2_bytes);
  if ((size_t)blocks * threads * sizeof(double) > ((size_t)4 << 20))
    return fail(HOPF_EUNSUPPORTED, "hopf_measure_pipes: too many SMs for the output area");
  cudaEvent_t e0, e1;
  HOPF_CUDA(cudaEventCreate(&e0));
  HOPF_CUDA(cudaEventCreate(&e1));
  hopf_status st = HOPF_OK;
  auto timed = [&](auto launch, int reps) -> double {
    launch();  // warm-up
    cudaEventRecord(e0, stream);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return (double)ms / reps;
  };
  if (fp32_tflops) {
    const int iters = 4096;
    const double ms = timed([&] { k_probe_fma<float><<<blocks, threads, 0, stream>>>(iters, 0.9999f, 1e-4f, outf); }, 5);
    const double flop = 2.0 * kProbeChains * 16.0 * iters * (double)blocks * threads;
    *fp32_tflops = ms > 0 ? flop / (ms * 1e-3) / 1e12 : 0.0;
  }
  if (fp64_tflops) {
    const int iters = 64;
    const double ms = timed([&] { k_probe_fma<double><<<blocks, threads, 0, stream>>>(iters, 0.9999, 1e-4, outd); }, 3);
    const double flop = 2.0 * kProbeChains * 16.0 * iters * (double)blocks * threads;
    *fp64_tflops = ms > 0 ? flop / (ms * 1e-3) / 1e12 : 0.0;
  }
  if (l2_gbs) {
    cudaMemsetAsync(base, 0, l2_bytes, stream);
    const int passes = 20;
    const double ms = timed(
        [&] { k_probe_l2<<<blocks, threads, 0, stream>>>((const float4*)base, l2_bytes / 16, passes, outf); }, 5);
    *l2_gbs = ms > 0 ? (double)passes * l2_bytes / (ms * 1e-3) / 1e9 : 0.0;
  }
  if (cudaGetLastError() != cudaSuccess) st = fail(HOPF_ECUDA, "hopf_measure_pipes: a probe kernel failed");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

}  // namespace hopf
