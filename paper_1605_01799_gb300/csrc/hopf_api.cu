// C ABI entry points: argument checks, handle lifetime, dispatch to kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "hopf_internal.h"

namespace hopf {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

hopf_status fail(hopf_status s, const std::string& msg) {
  set_error(msg);
  return s;
}

hopf_status cuda_fail(cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  set_error(buf);
  return e == cudaErrorMemoryAllocation ? HOPF_ENOMEM : HOPF_ECUDA;
}

int sm_count(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
  return v;
}

// Symmetric eigendecomposition M = P diag(l) P^T by the cyclic Jacobi method
// (row-by-row sweeps of plane rotations, each zeroing one off-diagonal pair;
// Golub and Van Loan, Matrix Computations, the cyclic Jacobi algorithm).  P is
// row-major with the k-th eigenvector in column k.  Returns false when 60
// sweeps leave the off-diagonal mass above 1e-30 of the total.
static bool sym_eig(int n, const double* M, std::vector<double>& P, std::vector<double>& l) {
  std::vector<double> a((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) a[(size_t)i * n + j] = 0.5 * (M[(size_t)i * n + j] + M[(size_t)j * n + i]);
  P.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) P[(size_t)i * n + i] = 1.0;
  bool ok = false;
  for (int sweep = 0; sweep < 60 && !ok; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v = a[(size_t)i * n + j] * a[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) {
      ok = true;
      break;
    }
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (apq == 0.0) continue;
        // rotation [c s; -s c] in the (p, q) plane with (J^T A J)_pq = 0
        const double theta = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q of A J
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q of J^T (A J)
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // P J
          const double pkp = P[(size_t)k * n + p], pkq = P[(size_t)k * n + q];
          P[(size_t)k * n + p] = c * pkp - s * pkq;
          P[(size_t)k * n + q] = s * pkp + c * pkq;
        }
      }
  }
  l.resize(n);
  for (int i = 0; i < n; ++i) l[i] = a[(size_t)i * n + i];
  return ok;
}

static void free_handle(hopf_handle h) {
  if (!h) return;
  void* ptrs[] = {h->d_A, h->d_c, h->d_w, h->d_cf, h->d_wf, h->d_af, h->d_M64, h->d_M32, h->d_A32,
                  h->d_Mbf, h->d_Ah16, h->d_Al16, h->d_Al2, h->d_Abf, h->d_Mh16, h->d_Ml16, h->d_P, h->d_PT,
                  h->d_Pf, h->d_PTf};
  for (void* p : ptrs) dev_free(h->alloc, p);
  delete h;
}

}  // namespace hopf

using namespace hopf;

extern "C" {

const char* hopf_last_error(void) { return g_last_error.c_str(); }

hopf_status hopf_batch_create(const hopf_desc* descs, int32_t count, hopf_batch* out, cudaStream_t stream) {
  set_error("");
  if (!descs || !out || count < 1) return fail(HOPF_EINVAL, "hopf_batch_create: need descs, out and count >= 1");
  *out = nullptr;
  return batch_create(descs, count, out, stream);
}

void hopf_batch_destroy(hopf_batch b) { batch_destroy(b); }

static hopf_status check_counts(hopf_batch b, const int64_t* counts) {
  if (!b || !counts) return fail(HOPF_EINVAL, "hopf_batch: null batch or counts");
  for (size_t i = 0; i < batch_count(b); ++i)
    if (counts[i] < 0 || counts[i] > ((int64_t)1 << 31)) return fail(HOPF_EINVAL, "hopf_batch: bad query count");
  return HOPF_OK;
}

hopf_status hopf_batch_workspace_size(hopf_batch b, const int64_t* counts, size_t* bytes) {
  set_error("");
  hopf_status s = check_counts(b, counts);
  if (s != HOPF_OK) return s;
  if (!bytes) return fail(HOPF_EINVAL, "hopf_batch_workspace_size: null bytes");
  *bytes = batch_workspace(b, counts);
  return HOPF_OK;
}

hopf_status hopf_batch_eval(hopf_batch b, const int64_t* counts, const float* x, const float* t, double* phi,
                            float* grad, float* dphidt, int32_t* iters, uint8_t* qstatus, void* workspace,
                            size_t ws_bytes, cudaStream_t stream) {
  set_error("");
  hopf_status s = check_counts(b, counts);
  if (s != HOPF_OK) return s;
  if (!x || !t || !phi || !grad) return fail(HOPF_EINVAL, "hopf_batch_eval: null x, t, phi or grad");
  const size_t need = batch_workspace(b, counts);
  if (need > 0 && (!workspace || ws_bytes < need)) return fail(HOPF_EINVAL, "hopf_batch_eval: workspace too small");
  if (need > 0 && ((uintptr_t)workspace & 255u)) return fail(HOPF_EINVAL, "hopf_batch_eval: workspace must be 256-byte aligned");
  return batch_eval(b, counts, x, t, phi, grad, dphidt, iters, qstatus, workspace, ws_bytes, stream);
}

hopf_status hopf_batch_set_mode(hopf_batch b, int32_t mode) {
  set_error("");
  if (!b || mode < 0 || mode > 2) return fail(HOPF_EINVAL, "hopf_batch_set_mode: bad batch or mode");
  batch_set_mode(b, mode);
  return HOPF_OK;
}

hopf_status hopf_batch_info(hopf_batch b, int32_t* nstreams, int32_t* used_graph, float* tuned_ms) {
  set_error("");
  if (!b) return fail(HOPF_EINVAL, "hopf_batch_info: null batch");
  return batch_info(b, nstreams, used_graph, tuned_ms);
}

hopf_status hopf_set_wait_limit(hopf_handle h, int64_t cycles) {
  set_error("");
  if (!h) return fail(HOPF_EINVAL, "hopf_set_wait_limit: null handle");
  if (cycles < 0) return fail(HOPF_EINVAL, "hopf_set_wait_limit: cycles must be >= 0");
  h->wait_limit = cycles;
  return HOPF_OK;
}

hopf_status hopf_set_split_start(hopf_handle h, double tol_switch) {
  set_error("");
  if (!h) return fail(HOPF_EINVAL, "hopf_set_split_start: null handle");
  if (!(tol_switch >= 0.0) || !std::isfinite(tol_switch))
    return fail(HOPF_EINVAL, "hopf_set_split_start: tol_switch must be finite and >= 0");
  if (tol_switch > 0.0 && (h->precision != HOPF_P_MIXED || h->h_kind == HOPF_H_L2))
    return fail(HOPF_EUNSUPPORTED, "hopf_set_split_start: MIXED precision with H = l1 or weighted l1 only");
  h->split_start = tol_switch;
  return HOPF_OK;
}

hopf_status hopf_set_tc_pairs(hopf_handle h, int32_t on) {
  set_error("");
  if (!h) return fail(HOPF_EINVAL, "hopf_set_tc_pairs: null handle");
  h->tc_pairs = on ? 1 : 0;
  return HOPF_OK;
}

hopf_status hopf_set_allocator(hopf_alloc_fn alloc, hopf_free_fn release, void* ctx) {
  set_error("");
  return set_allocator(alloc, release, ctx);
}

hopf_status hopf_set_compaction(hopf_handle h, int32_t on) {
  set_error("");
  if (!h) return fail(HOPF_EINVAL, "hopf_set_compaction: null handle");
  h->compact = on ? 1 : 0;
  return HOPF_OK;
}

hopf_status hopf_profile_events(hopf_handle h, cudaEvent_t start, cudaEvent_t stop) {
  set_error("");
  if (!h) return fail(HOPF_EINVAL, "hopf_profile_events: null handle");
  if ((start == nullptr) != (stop == nullptr)) return fail(HOPF_EINVAL, "hopf_profile_events: give both events or none");
  h->prof_start = start;
  h->prof_stop = stop;
  return HOPF_OK;
}

const char* hopf_version(void) { return "hopf-gb300 0.2 (sm_103a)"; }

size_t hopf_measure_pipes_scratch(void) { return probe_scratch_bytes(); }

hopf_status hopf_measure_pipes(void* scratch, size_t scratch_bytes, double* fp32_tflops, double* fp64_tflops,
                               double* l2_read_gbs, cudaStream_t stream) {
  set_error("");
  if (!scratch) return fail(HOPF_EINVAL, "hopf_measure_pipes: null scratch");
  return measure_pipes(scratch, scratch_bytes, fp32_tflops, fp64_tflops, l2_read_gbs, stream);
}

hopf_status hopf_create(const hopf_desc* desc, hopf_handle* out, cudaStream_t stream) {
  set_error("");
  if (!desc || !out) return fail(HOPF_EINVAL, "hopf_create: null desc or out");
  *out = nullptr;
  const hopf_desc& d = *desc;
  if (d.a_kind != HOPF_A_DIAG && d.a_kind != HOPF_A_DENSE && d.a_kind != HOPF_J_L1SQ && d.a_kind != HOPF_J_LINFSQ)
    return fail(HOPF_EINVAL, "hopf_create: bad a_kind");
  const bool jnorm = d.a_kind == HOPF_J_L1SQ || d.a_kind == HOPF_J_LINFSQ;  // no matrix: the diagonal path
  const int nmax = d.a_kind == HOPF_A_DENSE ? 4096 : 8192;
  if (d.n < 1 || d.n > nmax) return fail(HOPF_EINVAL, "hopf_create: n out of range");
  if (!d.A && !jnorm) return fail(HOPF_EINVAL, "hopf_create: null A");
  if (d.h_kind != HOPF_H_L1 && d.h_kind != HOPF_H_WL1 && d.h_kind != HOPF_H_L2 && d.h_kind != HOPF_H_LINF &&
      d.h_kind != HOPF_H_DNORM && d.h_kind != HOPF_H_ANORM)
    return fail(HOPF_EINVAL, "hopf_create: bad h_kind");
  const bool weighted = d.h_kind == HOPF_H_WL1 || d.h_kind == HOPF_H_DNORM;
  const bool anorm = d.h_kind == HOPF_H_ANORM;
  if (weighted && !d.w) return fail(HOPF_EINVAL, "hopf_create: weighted l1 and sqrt(sum w p^2) need w");
  if (anorm && !d.w) return fail(HOPF_EINVAL, "hopf_create: sqrt(<p, M p>) needs M in w");
  if (anorm && d.n > 512) return fail(HOPF_EUNSUPPORTED, "hopf_create: sqrt(<p, M p>) needs n <= 512");
  if (d.a_kind == HOPF_A_DENSE && (d.h_kind == HOPF_H_LINF || d.h_kind == HOPF_H_DNORM || anorm))
    return fail(HOPF_EUNSUPPORTED,
                "hopf_create: H = l_inf, sqrt(sum w p^2) and sqrt(<p, M p>) run on the diagonal path only");
  if (!(d.lambda > 0) || !std::isfinite(d.lambda)) return fail(HOPF_EINVAL, "hopf_create: lambda must be > 0");
  if (!(d.tol > 0) || !std::isfinite(d.tol)) return fail(HOPF_EINVAL, "hopf_create: tol must be > 0");
  if (d.max_iter < 1) return fail(HOPF_EINVAL, "hopf_create: max_iter must be >= 1");
  if (d.stop_rule != HOPF_STOP_PAPER && d.stop_rule != HOPF_STOP_UREL)
    return fail(HOPF_EINVAL, "hopf_create: bad stop_rule");
  if (d.precision != HOPF_P_FP64 && d.precision != HOPF_P_FP32 && d.precision != HOPF_P_BF16 &&
      d.precision != HOPF_P_SPLIT && d.precision != HOPF_P_MIXED)
    return fail(HOPF_EINVAL, "hopf_create: bad precision");
  if (d.a_kind == HOPF_A_DENSE && d.precision == HOPF_P_FP64)
    return fail(HOPF_EUNSUPPORTED, "hopf_create: FP64 is implemented for diagonal A only");
  if (d.a_kind == HOPF_A_DENSE && d.stop_rule == HOPF_STOP_PAPER)
    return fail(HOPF_EUNSUPPORTED, "hopf_create: dense A uses the relative u stop rule (HOPF_STOP_UREL)");
  const int n = d.n;
  for (int i = 0; i < n; ++i) {
    if (weighted && !(d.w[i] > 0 && std::isfinite(d.w[i]))) return fail(HOPF_EINVAL, "hopf_create: weights must be > 0");
    if (d.centre && !std::isfinite(d.centre[i])) return fail(HOPF_EINVAL, "hopf_create: non-finite centre");
    if (d.a_kind == HOPF_A_DIAG && !(d.A[i] > 0 && std::isfinite(d.A[i])))
      return fail(HOPF_ENOTSPD, "hopf_create: diagonal A must be positive");
  }

  // H = sqrt(<p, M p>): symmetric M, eigendecomposition, positive spectrum
  std::vector<double> eP, el;
  if (anorm) {
    double mx = 0.0;
    for (size_t i = 0; i < (size_t)n * n; ++i) {
      if (!std::isfinite(d.w[i])) return fail(HOPF_EINVAL, "hopf_create: non-finite M");
      mx = std::fmax(mx, std::fabs(d.w[i]));
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j)
        if (std::fabs(d.w[(size_t)i * n + j] - d.w[(size_t)j * n + i]) > 1e-12 * mx)
          return fail(HOPF_EINVAL, "hopf_create: M must be symmetric");
    if (!sym_eig(n, d.w, eP, el)) return fail(HOPF_ENOTSPD, "hopf_create: eigendecomposition of M did not converge");
    for (int i = 0; i < n; ++i)
      if (!(el[i] > 0.0)) return fail(HOPF_ENOTSPD, "hopf_create: M must be positive definite");
  }

  hopf_handle h = new hopf_handle_s();
  h->alloc = current_allocator();
  h->n = n;
  h->n_pad = (int)round_up(n, 128);
  h->a_kind = jnorm ? HOPF_A_DIAG : d.a_kind;
  h->j_kind = jnorm ? d.a_kind : 0;
  h->h_kind = d.h_kind;
  h->precision = d.precision;
  h->stop_rule = d.stop_rule;
  h->max_iter = d.max_iter;
  h->c0 = d.c0;
  h->lambda = d.lambda;
  h->tol = d.tol;
  // MIXED, l1 / weighted l1: SPLIT iterations until the change is within ten
  // times the tolerance, then the defect correction to the tolerance
  h->split_start = d.precision == HOPF_P_MIXED && d.h_kind != HOPF_H_L2 ? 10.0 * d.tol : 0.0;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    free_handle(h);
    return cuda_fail(e, "cudaGetDevice");
  }
  h->num_sms = sm_count(h->device);

#define H_ALLOC(ptr, bytes)                           \
  do {                                                \
    cudaError_t e2 = dev_alloc(h->alloc, (void**)&(ptr), (bytes)); \
    if (e2 != cudaSuccess) {                          \
      free_handle(h);                                 \
      return cuda_fail(e2, "cudaMalloc");             \
    }                                                 \
  } while (0)
#define H_CALL(call)                                  \
  do {                                                \
    cudaError_t e2 = (call);                          \
    if (e2 != cudaSuccess) {                          \
      free_handle(h);                                 \
      return cuda_fail(e2, #call);                    \
    }                                                 \
  } while (0)

  const int np = h->n_pad;
  std::vector<double> wv(n, 1.0);
  if (weighted)
    for (int i = 0; i < n; ++i) wv[i] = d.w[i];
  if (anorm) {  // the eigenvalues serve as the weights of the rotated problem
    wv = el;
    std::vector<double> PT((size_t)n * n);
    std::vector<float> Pf((size_t)n * n), PTf((size_t)n * n);
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < n; ++k) {
        const double v = eP[(size_t)i * n + k];
        PT[(size_t)k * n + i] = v;
        Pf[(size_t)i * n + k] = (float)v;
        PTf[(size_t)k * n + i] = (float)v;
      }
    const size_t b64 = sizeof(double) * n * n, b32 = sizeof(float) * n * n;
    H_ALLOC(h->d_P, b64);
    H_ALLOC(h->d_PT, b64);
    H_ALLOC(h->d_Pf, b32);
    H_ALLOC(h->d_PTf, b32);
    H_CALL(cudaMemcpyAsync(h->d_P, eP.data(), b64, cudaMemcpyHostToDevice, stream));
    H_CALL(cudaMemcpyAsync(h->d_PT, PT.data(), b64, cudaMemcpyHostToDevice, stream));
    H_CALL(cudaMemcpyAsync(h->d_Pf, Pf.data(), b32, cudaMemcpyHostToDevice, stream));
    H_CALL(cudaMemcpyAsync(h->d_PTf, PTf.data(), b32, cudaMemcpyHostToDevice, stream));
    H_CALL(cudaStreamSynchronize(stream));  // the host vectors die at the end of this block
  }
  std::vector<float> wf(np, 1.0f), cf(np, 0.0f);
  for (int i = 0; i < n; ++i) {
    wf[i] = (float)wv[i];
    cf[i] = d.centre ? (float)d.centre[i] : 0.0f;
  }
  H_ALLOC(h->d_w, sizeof(double) * n);
  H_CALL(cudaMemcpyAsync(h->d_w, wv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, stream));
  H_ALLOC(h->d_wf, sizeof(float) * np);
  H_CALL(cudaMemcpyAsync(h->d_wf, wf.data(), sizeof(float) * np, cudaMemcpyHostToDevice, stream));
  H_ALLOC(h->d_cf, sizeof(float) * np);
  H_CALL(cudaMemcpyAsync(h->d_cf, cf.data(), sizeof(float) * np, cudaMemcpyHostToDevice, stream));
  if (d.centre) {
    H_ALLOC(h->d_c, sizeof(double) * n);
    H_CALL(cudaMemcpyAsync(h->d_c, d.centre, sizeof(double) * n, cudaMemcpyHostToDevice, stream));
  }
  if (jnorm) {
    H_CALL(cudaStreamSynchronize(stream));  // no matrix: the data copies only
  } else if (d.a_kind == HOPF_A_DIAG) {
    H_ALLOC(h->d_A, sizeof(double) * n);
    H_CALL(cudaMemcpyAsync(h->d_A, d.A, sizeof(double) * n, cudaMemcpyHostToDevice, stream));
    std::vector<float> af(np, 1.0f);
    for (int i = 0; i < n; ++i) af[i] = (float)d.A[i];
    H_ALLOC(h->d_af, sizeof(float) * np);
    H_CALL(cudaMemcpyAsync(h->d_af, af.data(), sizeof(float) * np, cudaMemcpyHostToDevice, stream));
    H_CALL(cudaStreamSynchronize(stream));
  } else {
    hopf_status s = dense_setup(h, d.A, stream);
    if (s == HOPF_OK && d.precision != HOPF_P_FP32) s = dense_tc_prepare();
    if (s != HOPF_OK) {
      free_handle(h);
      return s;
    }
  }
#undef H_ALLOC
#undef H_CALL
  *out = h;
  return HOPF_OK;
}

void hopf_destroy(hopf_handle h) { free_handle(h); }

hopf_status hopf_workspace_size(hopf_handle h, int64_t batch, size_t* bytes) {
  set_error("");
  if (!h || !bytes || batch < 0) return fail(HOPF_EINVAL, "hopf_workspace_size: bad argument");
  *bytes = h->a_kind == HOPF_A_DIAG ? diag_workspace(h, batch) : dense_workspace(h, batch);
  return HOPF_OK;
}

static hopf_status check_eval(hopf_handle h, int64_t batch, const void* x, const void* t, const void* phi,
                              const void* grad, void* ws, size_t ws_bytes) {
  if (!h) return fail(HOPF_EINVAL, "hopf_eval: null handle");
  if (batch < 0) return fail(HOPF_EINVAL, "hopf_eval: negative batch");
  if (batch > (int64_t)1 << 31) return fail(HOPF_EINVAL, "hopf_eval: batch too large");
  if (batch == 0) return HOPF_OK;
  if (!x || !t || !phi || !grad) return fail(HOPF_EINVAL, "hopf_eval: null x, t, phi or grad");
  size_t need = h->a_kind == HOPF_A_DIAG ? diag_workspace(h, batch) : dense_workspace(h, batch);
  if (need > 0 && (!ws || ws_bytes < need)) return fail(HOPF_EINVAL, "hopf_eval: workspace too small");
  if (need > 0 && ((uintptr_t)ws & 255u)) return fail(HOPF_EINVAL, "hopf_eval: workspace must be 256-byte aligned");
  return HOPF_OK;
}

hopf_status hopf_eval(hopf_handle h, int64_t batch, const float* x, const float* t, double* phi, float* grad,
                      float* dphidt, int32_t* iters, uint8_t* qstatus, void* workspace, size_t ws_bytes,
                      cudaStream_t stream) {
  set_error("");
  hopf_status s = check_eval(h, batch, x, t, phi, grad, workspace, ws_bytes);
  if (s != HOPF_OK || batch == 0) return s;
  if (h->precision == HOPF_P_FP64) return fail(HOPF_EINVAL, "hopf_eval: FP64 handle needs hopf_eval_f64");
  if (h->a_kind == HOPF_A_DIAG) return diag_eval_f32(h, batch, x, t, phi, grad, dphidt, iters, qstatus, stream);
  DenseWs w;
  s = dense_carve(h, batch, workspace, ws_bytes, &w);
  if (s != HOPF_OK) return s;
  if (h->precision == HOPF_P_FP32) return dense_eval_simt(h, w, x, t, phi, grad, dphidt, iters, qstatus, stream);
  return dense_eval_tc(h, w, x, t, phi, grad, dphidt, iters, qstatus, stream);
}

hopf_status hopf_eval_control(hopf_handle h, int64_t batch, const float* x, const float* t, double* phi, float* grad,
                              float* dphidt, int32_t* iters, uint8_t* qstatus, float* beta, float* x_final,
                              void* workspace, size_t ws_bytes, cudaStream_t stream) {
  set_error("");
  hopf_status s = check_eval(h, batch, x, t, phi, grad, workspace, ws_bytes);
  if (s != HOPF_OK || batch == 0) return s;
  if (!beta) return fail(HOPF_EINVAL, "hopf_eval_control: null beta");
  if (h->precision == HOPF_P_FP64) return fail(HOPF_EUNSUPPORTED, "hopf_eval_control: FP32-output handles only");
  if (h->a_kind == HOPF_A_DIAG)
    return diag_eval_f32(h, batch, x, t, phi, grad, dphidt, iters, qstatus, stream, beta, x_final);
  DenseWs w;
  s = dense_carve(h, batch, workspace, ws_bytes, &w);
  if (s != HOPF_OK) return s;
  if (h->precision == HOPF_P_FP32)
    return dense_eval_simt(h, w, x, t, phi, grad, dphidt, iters, qstatus, stream, beta, x_final);
  return dense_eval_tc(h, w, x, t, phi, grad, dphidt, iters, qstatus, stream, beta, x_final);
}

hopf_status hopf_eval_f64(hopf_handle h, int64_t batch, const double* x, const double* t, double* phi, double* grad,
                          double* dphidt, int32_t* iters, uint8_t* qstatus, void* workspace, size_t ws_bytes,
                          cudaStream_t stream) {
  set_error("");
  hopf_status s = check_eval(h, batch, x, t, phi, grad, workspace, ws_bytes);
  if (s != HOPF_OK || batch == 0) return s;
  if (h->precision != HOPF_P_FP64 || h->a_kind != HOPF_A_DIAG)
    return fail(HOPF_EINVAL, "hopf_eval_f64: needs a diagonal FP64 handle");
  return diag_eval_f64(h, batch, x, t, phi, grad, dphidt, iters, qstatus, stream);
}

static hopf_status check_parts(const hopf_handle* parts, int32_t K, bool need_l2, bool same_h = true) {
  if (!parts || K < 1) return fail(HOPF_EINVAL, "hopf_union: need K >= 1 parts");
  for (int i = 0; i < K; ++i) {
    if (!parts[i]) return fail(HOPF_EINVAL, "hopf_union: null part");
    if (parts[i]->a_kind != HOPF_A_DIAG || parts[i]->precision != HOPF_P_FP32)
      return fail(HOPF_EUNSUPPORTED, "hopf_union: parts must be diagonal FP32 handles");
    if (parts[i]->n != parts[0]->n || (same_h && parts[i]->h_kind != parts[0]->h_kind))
      return fail(HOPF_EINVAL, "hopf_union: parts must share n and h_kind");
    if (need_l2 && (parts[i]->h_kind != HOPF_H_L2 || parts[i]->j_kind != 0))
      return fail(HOPF_EINVAL, "hopf_union_closest: parts must use H = l2 and a quadratic J");
  }
  return HOPF_OK;
}

hopf_status hopf_union_workspace_size(const hopf_handle* parts, int32_t K, int64_t batch, size_t* bytes) {
  set_error("");
  hopf_status s = check_parts(parts, K, false, false);  // (the size does not depend on H)
  if (s != HOPF_OK) return s;
  if (!bytes || batch < 0) return fail(HOPF_EINVAL, "hopf_union_workspace_size: bad argument");
  *bytes = union_workspace(K, parts[0]->n, batch);
  return HOPF_OK;
}

hopf_status hopf_union_eval(const hopf_handle* parts, int32_t K, int64_t batch, const float* x, const float* t,
                            double* phi, float* grad, int32_t* argmin, int32_t* iters, uint8_t* qstatus,
                            void* workspace, size_t ws_bytes, cudaStream_t stream) {
  set_error("");
  hopf_status s = check_parts(parts, K, false);
  if (s != HOPF_OK) return s;
  if (batch < 0) return fail(HOPF_EINVAL, "hopf_union_eval: negative batch");
  if (batch == 0) return HOPF_OK;
  if (!x || !t || !phi || !grad || !argmin) return fail(HOPF_EINVAL, "hopf_union_eval: null output");
  if (!workspace || ws_bytes < union_workspace(K, parts[0]->n, batch))
    return fail(HOPF_EINVAL, "hopf_union_eval: workspace too small");
  return union_eval(parts, K, batch, x, t, phi, grad, argmin, iters, qstatus, workspace, ws_bytes, stream);
}

hopf_status hopf_maxH_eval(const hopf_handle* parts, int32_t K, int64_t batch, const float* x, const float* t,
                           double* phi, float* grad, int32_t* argmax, int32_t* iters, uint8_t* qstatus,
                           void* workspace, size_t ws_bytes, cudaStream_t stream) {
  set_error("");
  hopf_status s = check_parts(parts, K, false, false);
  if (s != HOPF_OK) return s;
  if (batch < 0) return fail(HOPF_EINVAL, "hopf_maxH_eval: negative batch");
  if (batch == 0) return HOPF_OK;
  if (!x || !t || !phi || !grad || !argmax) return fail(HOPF_EINVAL, "hopf_maxH_eval: null output");
  if (!workspace || ws_bytes < union_workspace(K, parts[0]->n, batch))
    return fail(HOPF_EINVAL, "hopf_maxH_eval: workspace too small");
  return union_eval(parts, K, batch, x, t, phi, grad, argmax, iters, qstatus, workspace, ws_bytes, stream, true);
}

hopf_status hopf_union_closest(const hopf_handle* parts, int32_t K, int64_t batch, const float* x, float s_tol,
                               int32_t max_newton, float* dist, float* closest, int32_t* argmin, int32_t* newton,
                               uint8_t* qstatus, void* workspace, size_t ws_bytes, cudaStream_t stream) {
  set_error("");
  hopf_status s = check_parts(parts, K, true);
  if (s != HOPF_OK) return s;
  if (batch < 0 || max_newton < 1 || !(s_tol > 0)) return fail(HOPF_EINVAL, "hopf_union_closest: bad argument");
  if (batch == 0) return HOPF_OK;
  if (!x || !dist || !argmin) return fail(HOPF_EINVAL, "hopf_union_closest: null x, dist or argmin");
  if (!workspace || ws_bytes < union_workspace(K, parts[0]->n, batch))
    return fail(HOPF_EINVAL, "hopf_union_closest: workspace too small");
  return union_closest(parts, K, batch, x, s_tol, max_newton, dist, closest, argmin, newton, qstatus, workspace,
                       ws_bytes, stream);
}

hopf_status hopf_union_closest_noalloc(const hopf_handle* parts, int32_t K, int64_t batch, const float* x,
                                       float s_tol, int32_t max_newton, float* dist, float* closest, int32_t* argmin,
                                       int32_t* newton, uint8_t* qstatus, cudaStream_t stream) {
  set_error("");
  hopf_status s = check_parts(parts, K, true);
  if (s != HOPF_OK) return s;
  if (batch < 0 || max_newton < 1 || !(s_tol > 0)) return fail(HOPF_EINVAL, "hopf_union_closest_noalloc: bad argument");
  if (batch == 0) return HOPF_OK;
  if (!x || !dist || !argmin) return fail(HOPF_EINVAL, "hopf_union_closest_noalloc: null x, dist or argmin");
  return union_closest_noalloc(parts, K, batch, x, s_tol, max_newton, dist, closest, argmin, newton, qstatus, stream);
}

hopf_status hopf_backward_params(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar,
                                 const float* t, const float* dphidt, float* g_c, float* g_c0, float* g_w,
                                 cudaStream_t stream) {
  set_error("");
  if (!h || batch < 0) return fail(HOPF_EINVAL, "hopf_backward_params: bad argument");
  if (g_w && h->h_kind != HOPF_H_WL1 && h->h_kind != HOPF_H_DNORM)
    return fail(HOPF_EUNSUPPORTED, "hopf_backward_params: g_w needs weights (HOPF_H_WL1 or HOPF_H_DNORM)");
  if (batch == 0) {
    if (g_c) HOPF_CUDA(cudaMemsetAsync(g_c, 0, sizeof(float) * h->n, stream));
    if (g_w) HOPF_CUDA(cudaMemsetAsync(g_w, 0, sizeof(float) * h->n, stream));
    if (g_c0) HOPF_CUDA(cudaMemsetAsync(g_c0, 0, sizeof(float), stream));
    return HOPF_OK;
  }
  if (!g_phi || ((g_c || g_w) && !vstar)) return fail(HOPF_EINVAL, "hopf_backward_params: null g_phi or vstar");
  if (g_w && !t) return fail(HOPF_EINVAL, "hopf_backward_params: g_w needs t");
  if (g_w && h->h_kind == HOPF_H_DNORM && !dphidt)
    return fail(HOPF_EINVAL, "hopf_backward_params: g_w for sqrt(sum w p^2) needs dphidt");
  return backward_params(h, batch, g_phi, vstar, t, dphidt, g_c, g_c0, g_w, stream);
}

hopf_status hopf_backward(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, float* g_x,
                          float* g_t, float* g_A, cudaStream_t stream) {
  set_error("");
  if (!h || batch < 0) return fail(HOPF_EINVAL, "hopf_backward: bad argument");
  if (g_A && h->j_kind != 0)
    return fail(HOPF_EUNSUPPORTED, "hopf_backward: g_A needs initial data with a matrix A");
  if (batch == 0) {
    if (g_A) {
      size_t m = h->a_kind == HOPF_A_DENSE ? (size_t)h->n * h->n : (size_t)h->n;
      HOPF_CUDA(cudaMemsetAsync(g_A, 0, m * sizeof(float), stream));
    }
    return HOPF_OK;
  }
  if (!g_phi || !vstar) return fail(HOPF_EINVAL, "hopf_backward: null g_phi or vstar");
  return backward(h, batch, g_phi, vstar, g_x, g_t, g_A, stream);
}

hopf_status hopf_backward_workspace_size(hopf_handle h, int64_t batch, size_t* bytes) {
  set_error("");
  if (!h || !bytes || batch < 0) return fail(HOPF_EINVAL, "hopf_backward_workspace_size: bad argument");
  *bytes = h->a_kind == HOPF_A_DENSE && h->j_kind == 0 ? syrk_workspace(h, batch) : 0;
  return HOPF_OK;
}

hopf_status hopf_backward_ws(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, float* g_x,
                             float* g_t, float* g_A, void* workspace, size_t ws_bytes, cudaStream_t stream) {
  set_error("");
  if (!h || batch < 0) return fail(HOPF_EINVAL, "hopf_backward_ws: bad argument");
  if (!g_A || h->a_kind != HOPF_A_DENSE || h->j_kind != 0 || batch == 0)
    return hopf_backward(h, batch, g_phi, vstar, g_x, g_t, g_A, stream);
  if (!g_phi || !vstar) return fail(HOPF_EINVAL, "hopf_backward_ws: null g_phi or vstar");
  if (!workspace) return fail(HOPF_EINVAL, "hopf_backward_ws: null workspace");
  if (g_x || g_t) {
    hopf_status st = backward(h, batch, g_phi, vstar, g_x, g_t, nullptr, stream);
    if (st != HOPF_OK) return st;
  }
  return backward_dense_tc(h, batch, g_phi, vstar, g_A, workspace, ws_bytes, stream);
}

}  // extern "C"
