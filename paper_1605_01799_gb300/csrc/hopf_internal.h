// Internal declarations shared by the translation units of libhopf_gb300.
#pragma once
#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/hopf.h"

// Device allocator of handle memory: cudaMalloc / cudaFree, or the functions
// installed by hopf_set_allocator.
struct Allocator {
  hopf_alloc_fn alloc;
  hopf_free_fn release;
  void* ctx;
};

struct hopf_handle_s {
  int n = 0;          // problem dimension
  int n_pad = 0;      // leading dimension of padded device arrays (multiple of 128)
  int a_kind = 0, h_kind = 0, precision = 0, stop_rule = 0, max_iter = 0;
  double c0 = 0, lambda = 1, tol = 0;
  int device = 0, num_sms = 0;
  // initial data on the diagonal path: 0 quadratic (diagonal A), or
  // HOPF_J_L1SQ / HOPF_J_LINFSQ (A unused)
  int j_kind = 0;
  // SMs one cooperative dense launch may occupy (0: all).  A ragged batch sets
  // it to its per-stream share so that the dense solvers running side by side
  // on different streams fit on the GPU together.
  int grid_cap = 0;
  // device copies (FP64 inputs)
  double* d_A = nullptr;       // diagonal: [n]; dense: [n][n]
  double* d_c = nullptr;       // [n] or null
  double* d_w = nullptr;       // [n] (ones when not weighted)
  float* d_cf = nullptr;       // [n_pad] centre as float (zeros when none)
  float* d_wf = nullptr;       // [n_pad] weights as float (padding 1)
  float* d_af = nullptr;       // diagonal A as float [n_pad]
  // H = sqrt(<p, M p>): M = P diag(l) P^T, l stored as the weights d_w / d_wf
  double* d_P = nullptr;       // [n][n] row-major, column k the k-th eigenvector
  double* d_PT = nullptr;      // P^T
  float* d_Pf = nullptr;       // FP32 copies
  float* d_PTf = nullptr;
  // dense derived operands, padded to n_pad x n_pad, row-major
  double* d_M64 = nullptr;     // (A + lambda I)^{-1}, FP64
  float* d_M32 = nullptr;      // FP32 copy of M
  float* d_A32 = nullptr;      // FP32 copy of A
  uint16_t* d_Mbf = nullptr;   // BF16(M)
  uint16_t* d_Ah16 = nullptr;  // FP16(A)
  uint16_t* d_Al16 = nullptr;  // FP16((A - FP16(A)) * 2^11)
  uint16_t* d_Al2 = nullptr;   // FP16((A - hi - lo * 2^-11) * 2^22): third term of the split
  uint16_t* d_Abf = nullptr;   // BF16(A) (for the BF16 form's final phi pass)
  uint16_t* d_Mh16 = nullptr;  // FP16(M) (SPLIT form)
  uint16_t* d_Ml16 = nullptr;  // FP16((M - FP16(M)) * 2^11) (SPLIT form)
  cudaEvent_t prof_start = nullptr, prof_stop = nullptr;  // optional instrumentation
  int compact = 1;  // tensor-core path: pack active queries as others converge
  long long wait_limit = 0;  // clock cycles of the dense solvers' bounded waits (0: the default)
  int tc_pairs = 0;  // tensor-core path: SM pairs (cta_group::2) when the row tiles pair up (off: measured slower)
  double split_start = 0.0;  // MIXED form, l1 / weighted l1: SPLIT iterations down to this change first (0: off)
  Allocator alloc = {nullptr, nullptr, nullptr};  // the allocator this handle's memory came from
};

namespace hopf {

// thread-local last error
void set_error(const std::string& msg);
hopf_status fail(hopf_status s, const std::string& msg);
hopf_status cuda_fail(cudaError_t e, const char* what);

#define HOPF_CUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return hopf::cuda_fail(e_, #call); \
  } while (0)

// ---- setup (setup.cu) ----
hopf_status dense_setup(hopf_handle h, const double* A_host, cudaStream_t stream);
hopf_status set_allocator(hopf_alloc_fn alloc, hopf_free_fn release, void* ctx);
Allocator current_allocator();
cudaError_t dev_alloc(const Allocator& a, void** p, size_t bytes);
void dev_free(const Allocator& a, void* p);

// ---- diagonal path (diag.cu) ----
size_t diag_workspace(const hopf_handle h, int64_t batch);
hopf_status diag_eval_f32(hopf_handle h, int64_t batch, const float* x, const float* t, double* phi, float* grad,
                          float* dphidt, int32_t* iters, uint8_t* qstatus, cudaStream_t stream, float* beta = nullptr,
                          float* xfin = nullptr);
hopf_status diag_eval_f64(hopf_handle h, int64_t batch, const double* x, const double* t, double* phi, double* grad,
                          double* dphidt, int32_t* iters, uint8_t* qstatus, cudaStream_t stream);
size_t union_workspace(int K, int n, int64_t batch);
// maximize: pick the largest phi_i (maximum over Hamiltonians) instead of the smallest
hopf_status union_eval(const hopf_handle* parts, int K, int64_t batch, const float* x, const float* t, double* phi,
                       float* grad, int32_t* argmin, int32_t* iters, uint8_t* qstatus, void* ws, size_t ws_bytes,
                       cudaStream_t stream, bool maximize = false);
hopf_status union_closest(const hopf_handle* parts, int K, int64_t batch, const float* x, float s_tol,
                          int max_newton, float* dist, float* closest, int32_t* argmin, int32_t* newton,
                          uint8_t* qstatus, void* ws, size_t ws_bytes, cudaStream_t stream);
size_t noalloc_scratch_bytes();
hopf_status union_closest_noalloc(const hopf_handle* parts, int K, int64_t batch, const float* x, float s_tol,
                                  int max_newton, float* dist, float* closest, int32_t* argmin, int32_t* newton,
                                  uint8_t* qstatus, cudaStream_t stream);

// ---- dense path ----
// Workspace shared by the dense solvers.
struct DenseWs {
  int64_t B = 0, B_pad = 0;  // batch and its padding to the column tile
  int rt = 0;                // number of 128-row tiles of n_pad
  float* y = nullptr;        // [B_pad][n_pad] x - c
  float* u = nullptr;        // [B_pad][n_pad] d-update argument
  uint16_t* ph = nullptr;    // [B_pad][n_pad] tensor-core operand 1 (BF16 r, or FP16 split of p)
  uint16_t* pl = nullptr;    // [B_pad][n_pad] tensor-core operand 2 (FP16 split of p, scaled)
  uint16_t* g = nullptr;     // [B_pad][n_pad] BF16 residual g
  float* part = nullptr;     // [set][2][2][rt][B_pad] residual / norm partials by parity (tensor-core solver: by buffer set)
  double* fpart = nullptr;   // [2][rt][B_pad] final phi partials
  float* tau = nullptr;      // [B_pad] t / lambda
  float* tq = nullptr;       // [B_pad] t
  float* scale = nullptr;    // [B_pad] l2 prox scale of the current iterate
  int* qiter = nullptr;      // [B_pad]
  int* qdone = nullptr;      // [B_pad]
  int* qact = nullptr;       // [2][B_pad] by parity of the decision
  int* tile_act = nullptr;   // [2][B_pad / 128] per column tile (tensor-core solver: last decision with active slots; count)
  // tensor-core path: slots (columns of the operand planes) are compacted as
  // queries converge; a second buffer set receives the packed slots, and a
  // converged query's u and l2 scale are retired to query-indexed arrays
  float* y_b = nullptr;      // [B_pad][n_pad]
  float* u_b = nullptr;      // [B_pad][n_pad] (FP32 solver: u^k of odd k; u^k of even k is in u)
  uint16_t* ph_b = nullptr;  // [B_pad][n_pad]
  uint16_t* pl_b = nullptr;  // [B_pad][n_pad]
  float* scale_b = nullptr;  // [B_pad]
  float* taus = nullptr;     // [2][B_pad] t / lambda by slot (moves with its query)
  int* qact_b = nullptr;     // [2][B_pad]
  int* sq = nullptr;         // [2][B_pad] slot -> query
  float* ufin = nullptr;     // [B_pad][n_pad] u of converged queries, by query
  float* sfin = nullptr;     // [B_pad] l2 scale of converged queries, by query
  // SPLIT form: r^k lives in the operand planes of parity k & 1; parity 0 is
  // (ph, pl) / (ph_b, pl_b), parity 1 these (one pair per buffer set)
  uint16_t* qh = nullptr;    // [B_pad][n_pad]
  uint16_t* ql = nullptr;
  uint16_t* qh_b = nullptr;
  uint16_t* ql_b = nullptr;
  int* qiter0 = nullptr;     // [B_pad] two-stage solve: iterations of the first stage
  unsigned* bar = nullptr;   // [4] grid barrier + counters
  int* err = nullptr;        // [1]
};
size_t dense_workspace(const hopf_handle h, int64_t batch);
bool two_stage(const hopf_handle h);
hopf_status dense_init_warm(hopf_handle h, DenseWs& w, const float* x, const float* t, cudaStream_t s);
hopf_status dense_carve(const hopf_handle h, int64_t batch, void* ws, size_t ws_bytes, DenseWs* d);
hopf_status dense_eval_simt(hopf_handle h, DenseWs& w, const float* x, const float* t, double* phi, float* grad,
                            float* dphidt, int32_t* iters, uint8_t* qstatus, cudaStream_t stream, float* beta = nullptr,
                          float* xfin = nullptr);
size_t tc_smem_bytes();
hopf_status dense_tc_prepare();
hopf_status dense_eval_tc(hopf_handle h, DenseWs& w, const float* x, const float* t, double* phi, float* grad,
                          float* dphidt, int32_t* iters, uint8_t* qstatus, cudaStream_t stream, float* beta = nullptr,
                          float* xfin = nullptr);

// ---- ragged batches in one persistent launch (dense_tc.cu) ----
size_t ragged_dense_record_bytes();
size_t ragged_diag_record_bytes();
hopf_status ragged_build_dense(hopf_handle h, DenseWs& w, const float* x, const float* t, double* phi, float* grad,
                               float* dphidt, int32_t* iters, uint8_t* qstatus, void* rec);
int ragged_diag_class(hopf_handle h);  // work-list shape class of a diagonal instance, -1: its own launch
void ragged_build_diag(hopf_handle h, int64_t B, const float* x, const float* t, double* phi, float* grad,
                       float* dphidt, int32_t* iters, uint8_t* qstatus, void* rec);
hopf_status ragged_prepare();
hopf_status ragged_launch(const void* dense, const int4* sched, const int* sched_off, int grid, const void* diag,
                          const int4* dinfo, int n_diag, int n_items, unsigned* ctr, cudaStream_t stream);

// ---- backward on the tensor cores (syrk_tc.cu) ----
size_t syrk_workspace(const hopf_handle h, int64_t batch);
hopf_status backward_dense_tc(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, float* g_A,
                              void* ws, size_t ws_bytes, cudaStream_t stream);

// ---- backward (backward.cu) ----
hopf_status backward(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, float* g_x, float* g_t,
                     float* g_A, cudaStream_t stream);
hopf_status backward_params(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, const float* t,
                            const float* dphidt, float* g_c, float* g_c0, float* g_w, cudaStream_t stream);

int sm_count(int device);

// ---- pipe probes (probe.cu) ----
size_t probe_scratch_bytes();
hopf_status measure_pipes(void* scratch, size_t bytes, double* fp32_tflops, double* fp64_tflops, double* l2_gbs,
                          cudaStream_t stream);

// ---- ragged batches (batch.cu) ----
hopf_status batch_create(const hopf_desc* descs, int32_t count, hopf_batch* out, cudaStream_t stream);
void batch_destroy(hopf_batch b);
size_t batch_workspace(hopf_batch b, const int64_t* counts);
size_t batch_count(hopf_batch b);
hopf_status batch_eval(hopf_batch b, const int64_t* counts, const float* x, const float* t, double* phi, float* grad,
                       float* dphidt, int32_t* iters, uint8_t* qstatus, void* ws, size_t ws_bytes,
                       cudaStream_t stream);
hopf_status batch_info(hopf_batch b, int32_t* nstreams, int32_t* used_graph, float* tuned_ms);
void batch_set_mode(hopf_batch b, int mode);

}  // namespace hopf
