// Diagonal-A path: plain evaluation (one query per thread, warp or CTA; the
// state and solver are in diag_query.cuh).
#include "diag_query.cuh"

namespace hopf {

// Lanes of a thread-per-query warp still iterating when at most this many
// remain hand their query to the whole warp (the runtime kinds, whose
// iteration counts run on a heavy tail: 1/2|x|_1^2 needs 10^2 iterations on
// average and 10^5 at worst).  FP64 only: there one lane's iteration is a
// long chain of FP64 operations, which GB300 issues at a small fraction of
// its FP32 rate, and spreading it over the warp shortens the tail 4-6x; in
// FP32 the warp's reductions cost as much as they save.
constexpr int kHandoverLanes = 4;

template <typename T, int G, int VPT, bool GEN>
__global__ void __launch_bounds__(block_of<G>()) k_diag_eval(DiagEvalArgs<T> A) {
  constexpr bool TAIL = GEN && G == 1 && sizeof(T) == 8;
  int64_t q = G == 1 ? (int64_t)blockIdx.x * blockDim.x + threadIdx.x
                     : (G == 32 ? ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5 : (int64_t)blockIdx.x);
  const bool live = q < A.batch;
  if constexpr (!TAIL) {
    if (!live) return;  // whole groups leave together
  } else {
    if (!live) q = A.batch - 1;  // in-bounds loads for the warp's votes; nothing is written
  }
  Query<T, G, VPT> Q;
  Q.load(A.P, A.x + q * A.n, A.n);
  Q.cold_start();
  const T tq = A.t[q];
  bool conv, pending = false;
  int k;
  if constexpr (TAIL) k = Q.solve_generic(A.P, tq, &conv, 0, kHandoverLanes, live, &pending);
  else k = Q.template solve<GEN>(A.P, tq, &conv);
  if (live && !pending) emit<GEN>(A, Q, q, tq, k, conv);
  if constexpr (TAIL) {
    // the warp takes over its last queries one at a time, coordinate i on
    // lane i (n <= VPT <= 32), from the state they stopped at
    static_assert(VPT <= 32, "the warp holds one coordinate per lane");
    const int lane = threadIdx.x & 31;
    unsigned pend = __ballot_sync(0xffffffffu, pending);
    while (pend) {
      const int L = __ffs(pend) - 1;
      pend &= pend - 1;
      Query<T, 32, 1> W;
      W.n = A.n;
      W.a = Q.a;
      W.w = Q.w;
      W.y[0] = W.ia[0] = W.v[0] = W.d[0] = W.b[0] = T(0);
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        const T y = __shfl_sync(0xffffffffu, Q.y[j], L), ia = __shfl_sync(0xffffffffu, Q.ia[j], L);
        const T v = __shfl_sync(0xffffffffu, Q.v[j], L), d = __shfl_sync(0xffffffffu, Q.d[j], L);
        const T b = __shfl_sync(0xffffffffu, Q.b[j], L);
        if (lane == j) {
          W.y[0] = y;
          W.ia[0] = ia;
          W.v[0] = v;
          W.d[0] = d;
          W.b[0] = b;
        }
      }
      const int kL = __shfl_sync(0xffffffffu, k, L);
      const T tL = __shfl_sync(0xffffffffu, tq, L);
      const long long qL = __shfl_sync(0xffffffffu, (long long)q, L);
      bool convL;
      const int k2 = W.solve_generic(A.P, tL, &convL, kL);
      emit<GEN>(A, W, (int64_t)qL, tL, k2, convL);
    }
  }
}

template <typename T, int G, int VPT, bool GEN>
static void launch_eval_kind(const DiagEvalArgs<T>& a, cudaStream_t s) {
  if constexpr (G == 1) {
    k_diag_eval<T, 1, VPT, GEN><<<(unsigned)((a.batch + 127) / 128), 128, 0, s>>>(a);
  } else if constexpr (G == 32) {
    k_diag_eval<T, 32, VPT, GEN><<<(unsigned)((a.batch + 3) / 4), 128, 0, s>>>(a);
  } else {
    k_diag_eval<T, G, VPT, GEN><<<(unsigned)a.batch, G, 0, s>>>(a);
  }
}

template <typename T, int G, int VPT>
static void launch_eval(const DiagEvalArgs<T>& a, cudaStream_t s) {
  if (generic_kind(a.P)) launch_eval_kind<T, G, VPT, true>(a, s);
  else launch_eval_kind<T, G, VPT, false>(a, s);
}

// Pick the group shape from n.
template <typename T>
static hopf_status dispatch_eval(const DiagEvalArgs<T>& a, cudaStream_t s) {
  const int n = a.n;
  if (n <= 4) launch_eval<T, 1, 4>(a, s);  // thread per query; the paper's n = 4..16 (Section 4.5)
  else if (n <= 8) launch_eval<T, 1, 8>(a, s);
  else if (n <= 16) launch_eval<T, 1, 16>(a, s);
  else if (n <= 64) launch_eval<T, 32, 2>(a, s);
  else if (n <= 256) launch_eval<T, 32, 8>(a, s);
  else if (n <= 512) launch_eval<T, 32, 16>(a, s);
  else if (n <= 4096) launch_eval<T, 256, 16>(a, s);
  else launch_eval<T, 512, 16>(a, s);
  HOPF_CUDA(cudaGetLastError());
  return HOPF_OK;
}

size_t diag_workspace(const hopf_handle, int64_t) { return 0; }

hopf_status diag_eval_f32(hopf_handle h, int64_t batch, const float* x, const float* t, double* phi, float* grad,
                          float* dphidt, int32_t* iters, uint8_t* qstatus, cudaStream_t stream, float* beta,
                          float* xfin) {
  DiagEvalArgs<float> a{part_of<float>(h), h->n, batch, x, t, phi, grad, dphidt, iters, qstatus, beta, xfin};
  if (h->prof_start) HOPF_CUDA(cudaEventRecord(h->prof_start, stream));
  hopf_status s = dispatch_eval(a, stream);
  if (h->prof_stop) HOPF_CUDA(cudaEventRecord(h->prof_stop, stream));
  return s;
}

hopf_status diag_eval_f64(hopf_handle h, int64_t batch, const double* x, const double* t, double* phi, double* grad,
                          double* dphidt, int32_t* iters, uint8_t* qstatus, cudaStream_t stream) {
  DiagEvalArgs<double> a{part_of<double>(h), h->n, batch, x, t, phi, grad, dphidt, iters, qstatus};
  if (h->prof_start) HOPF_CUDA(cudaEventRecord(h->prof_start, stream));
  hopf_status s = dispatch_eval(a, stream);
  if (h->prof_stop) HOPF_CUDA(cudaEventRecord(h->prof_stop, stream));
  return s;
}

}  // namespace hopf
