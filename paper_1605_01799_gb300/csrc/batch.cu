// Ragged batch: many instances (each its own A, H, n and query count) in one
// CUDA graph replay.
//
// The method evaluates every query on its own, with no shared state (Section
// 1; Section 4.5 runs queries one per core), so a batch of instances is a set
// of independent evaluations.  hopf_batch_eval records, for every instance, the
// same kernels a single hopf_eval would launch (the diagonal per-query kernel,
// or the dense tensor-core / FP32 solver) into one CUDA graph, forked from the
// caller's stream onto worker streams and joined back; the schedule is
// described at enqueue().  The number of lanes is picked by a small autotuner
// on the first call: each candidate schedule is captured and timed, the
// fastest is kept.  Later calls with the same buffers and counts replay it.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "hopf_internal.h"

struct hopf_batch_s {
  std::vector<hopf_handle> inst;
  // lanes 0..15 for the side-by-side work, the last stream for wide solves
  static constexpr int kMaxStreams = 17;
  cudaStream_t workers[kMaxStreams] = {};
  cudaStream_t origin = nullptr;  // capture origin (the caller's stream may be the legacy default stream)
  cudaEvent_t fork = nullptr, wide_done = nullptr, join[kMaxStreams] = {}, t0 = nullptr, t1 = nullptr;
  int nstreams = 0;          // tuned number of worker streams (0: not tuned yet)
  float tuned_ms[5] = {0, 0, 0, 0, 0};
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> key;  // buffers and counts of the captured call
  int used_graph = 0;
};

namespace hopf {

namespace {

struct Call {
  const int64_t* counts;
  const float* x;
  const float* t;
  double* phi;
  float* grad;
  float* dphidt;
  int32_t* iters;
  uint8_t* qstatus;
  char* ws;
};

// Work estimate of one instance (queries x the cost of one iteration per query).
double cost_of(hopf_handle h, int64_t B) {
  const double n = h->n;
  return h->a_kind == HOPF_A_DIAG ? (double)B * n : (double)B * n * n + 2.0 * n * n;
}

size_t ws_of(hopf_handle h, int64_t B) {
  return round_up(h->a_kind == HOPF_A_DIAG ? diag_workspace(h, B) : dense_workspace(h, B), 256);
}

hopf_status launch_one(hopf_handle h, int64_t B, const Call& c, int64_t qoff, int64_t xoff, size_t wsoff,
                       cudaStream_t s) {
  if (B == 0) return HOPF_OK;
  const float* x = c.x + xoff;
  const float* t = c.t + qoff;
  double* phi = c.phi + qoff;
  float* grad = c.grad + xoff;
  float* dphidt = c.dphidt ? c.dphidt + qoff : nullptr;
  int32_t* iters = c.iters ? c.iters + qoff : nullptr;
  uint8_t* qs = c.qstatus ? c.qstatus + qoff : nullptr;
  if (h->a_kind == HOPF_A_DIAG) return diag_eval_f32(h, B, x, t, phi, grad, dphidt, iters, qs, s);
  DenseWs w;
  hopf_status st = dense_carve(h, B, c.ws + wsoff, ws_of(h, B), &w);
  if (st != HOPF_OK) return st;
  if (h->precision == HOPF_P_FP32) return dense_eval_simt(h, w, x, t, phi, grad, dphidt, iters, qs, s);
  return dense_eval_tc(h, w, x, t, phi, grad, dphidt, iters, qs, s);
}

// 128 x 128 output tiles of one dense solve (the unit the persistent grid
// distributes over its CTAs).
int64_t tiles_of(hopf_handle h, int64_t B) { return (int64_t)(h->n_pad / 128) * ((B + 127) / 128); }

// Longest-first assignment of the instances in `ids` to `ns` lanes, each to
// the least loaded lane so far; returns the lane of every instance.
void assign(const std::vector<int>& ids, const std::vector<double>& cost, int ns, std::vector<int>* lane,
            std::vector<int>* order) {
  std::vector<int> o(ids);
  std::stable_sort(o.begin(), o.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  std::vector<double> load(ns, 0.0);
  for (int i : o) {
    const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    (*lane)[i] = s;
    load[s] += cost[i];
  }
  order->insert(order->end(), o.begin(), o.end());
}

// Enqueue the whole batch from `stream`.
//
// Dense solves are persistent cooperative kernels whose CTAs wait for each
// other at grid barriers, so the schedule never lets dense grids that are in
// flight together need more SMs than the GPU has:
//   * wide dense instances (at least one tile per SM) run one after another
//     on their own stream with the full grid;
//   * once they are done, the narrow dense instances run on `ns` lanes, each
//     capped at num_sms / ns CTAs, so the grids of the lanes fit side by side;
//   * diagonal instances (plain kernels that never wait on other CTAs) are
//     spread over the lanes ahead of the narrow dense work and overlap the
//     wide phase.
hopf_status enqueue(hopf_batch b, const Call& c, int ns, cudaStream_t stream) {
  const int m = (int)b->inst.size();
  std::vector<int64_t> qoff(m + 1, 0), xoff(m + 1, 0);
  std::vector<size_t> wsoff(m + 1, 0);
  std::vector<double> cost(m);
  std::vector<int> wide, narrow, diag;
  for (int i = 0; i < m; ++i) {
    hopf_handle h = b->inst[i];
    qoff[i + 1] = qoff[i] + c.counts[i];
    xoff[i + 1] = xoff[i] + c.counts[i] * h->n;
    wsoff[i + 1] = wsoff[i] + ws_of(h, c.counts[i]);
    cost[i] = cost_of(h, c.counts[i]);
    if (c.counts[i] == 0) continue;
    if (h->a_kind == HOPF_A_DIAG) diag.push_back(i);
    else if (tiles_of(h, c.counts[i]) >= h->num_sms) wide.push_back(i);
    else narrow.push_back(i);
  }
  std::vector<int> lane(m, 0), order_d, order_n;
  assign(diag, cost, ns, &lane, &order_d);
  assign(narrow, cost, ns, &lane, &order_n);
  std::stable_sort(wide.begin(), wide.end(), [&](int a, int d) { return cost[a] > cost[d]; });
  cudaStream_t ws = b->workers[hopf_batch_s::kMaxStreams - 1];

  HOPF_CUDA(cudaEventRecord(b->fork, stream));
  HOPF_CUDA(cudaStreamWaitEvent(ws, b->fork, 0));
  for (int s = 0; s < ns; ++s) HOPF_CUDA(cudaStreamWaitEvent(b->workers[s], b->fork, 0));
  for (int i : wide) {
    b->inst[i]->grid_cap = 0;
    hopf_status st = launch_one(b->inst[i], c.counts[i], c, qoff[i], xoff[i], wsoff[i], ws);
    if (st != HOPF_OK) return st;
  }
  HOPF_CUDA(cudaEventRecord(b->wide_done, ws));
  for (int i : order_d) {
    hopf_status st = launch_one(b->inst[i], c.counts[i], c, qoff[i], xoff[i], wsoff[i], b->workers[lane[i]]);
    if (st != HOPF_OK) return st;
  }
  if (!narrow.empty())
    for (int s = 0; s < ns; ++s) HOPF_CUDA(cudaStreamWaitEvent(b->workers[s], b->wide_done, 0));
  for (int i : order_n) {
    hopf_handle h = b->inst[i];
    h->grid_cap = std::max(1, h->num_sms / ns);
    hopf_status st = launch_one(h, c.counts[i], c, qoff[i], xoff[i], wsoff[i], b->workers[lane[i]]);
    if (st != HOPF_OK) return st;
  }
  for (int s = 0; s < ns; ++s) {
    HOPF_CUDA(cudaEventRecord(b->join[s], b->workers[s]));
    HOPF_CUDA(cudaStreamWaitEvent(stream, b->join[s], 0));
  }
  HOPF_CUDA(cudaStreamWaitEvent(stream, b->wide_done, 0));
  return HOPF_OK;
}

// Capture the batch as a graph on the batch's own origin stream (capture is
// not allowed on the legacy default stream); the graph is launched on the
// caller's stream.  On failure the capture is abandoned cleanly.
hopf_status capture(hopf_batch b, const Call& c, int ns, cudaGraphExec_t* exec) {
  *exec = nullptr;
  cudaStream_t o = b->origin;
  HOPF_CUDA(cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal));
  hopf_status st = enqueue(b, c, ns, o);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(o, &g);
  if (st != HOPF_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return HOPF_OK;
}

std::vector<uintptr_t> key_of(hopf_batch b, const Call& c, size_t ws_bytes) {
  std::vector<uintptr_t> k = {(uintptr_t)c.x,    (uintptr_t)c.t,     (uintptr_t)c.phi,     (uintptr_t)c.grad,
                              (uintptr_t)c.dphidt, (uintptr_t)c.iters, (uintptr_t)c.qstatus, (uintptr_t)c.ws,
                              (uintptr_t)ws_bytes};
  for (size_t i = 0; i < b->inst.size(); ++i) k.push_back((uintptr_t)c.counts[i]);
  return k;
}

void free_batch(hopf_batch b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (int s = 0; s < hopf_batch_s::kMaxStreams; ++s) {
    if (b->workers[s]) cudaStreamDestroy(b->workers[s]);
    if (b->join[s]) cudaEventDestroy(b->join[s]);
  }
  if (b->origin) cudaStreamDestroy(b->origin);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->wide_done) cudaEventDestroy(b->wide_done);
  if (b->t0) cudaEventDestroy(b->t0);
  if (b->t1) cudaEventDestroy(b->t1);
  for (hopf_handle h : b->inst) hopf_destroy(h);
  delete b;
}

}  // namespace

hopf_status batch_create(const hopf_desc* descs, int32_t count, hopf_batch* out, cudaStream_t stream) {
  for (int i = 0; i < count; ++i)
    if (descs[i].precision == HOPF_P_FP64)
      return fail(HOPF_EUNSUPPORTED, "hopf_batch_create: instance " + std::to_string(i) +
                                         ": FP64 instances are not batched");
  hopf_batch b = new hopf_batch_s();
  for (int i = 0; i < count; ++i) {
    hopf_handle h = nullptr;
    hopf_status st = hopf_create(&descs[i], &h, stream);
    if (st != HOPF_OK) {
      const std::string msg = std::string("hopf_batch_create: instance ") + std::to_string(i) + ": " + hopf_last_error();
      free_batch(b);
      return fail(st, msg);
    }
    b->inst.push_back(h);
  }
#define B_CALL(call)                     \
  do {                                   \
    cudaError_t e_ = (call);             \
    if (e_ != cudaSuccess) {             \
      free_batch(b);                     \
      return cuda_fail(e_, #call);       \
    }                                    \
  } while (0)
  for (int s = 0; s < hopf_batch_s::kMaxStreams; ++s) {
    B_CALL(cudaStreamCreateWithFlags(&b->workers[s], cudaStreamNonBlocking));
    B_CALL(cudaEventCreateWithFlags(&b->join[s], cudaEventDisableTiming));
  }
  B_CALL(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking));
  B_CALL(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  B_CALL(cudaEventCreateWithFlags(&b->wide_done, cudaEventDisableTiming));
  B_CALL(cudaEventCreate(&b->t0));
  B_CALL(cudaEventCreate(&b->t1));
#undef B_CALL
  *out = b;
  return HOPF_OK;
}

void batch_destroy(hopf_batch b) { free_batch(b); }

size_t batch_count(hopf_batch b) { return b->inst.size(); }

size_t batch_workspace(hopf_batch b, const int64_t* counts) {
  size_t s = 0;
  for (size_t i = 0; i < b->inst.size(); ++i) s += ws_of(b->inst[i], counts[i]);
  return s;
}

hopf_status batch_eval(hopf_batch b, const int64_t* counts, const float* x, const float* t, double* phi, float* grad,
                       float* dphidt, int32_t* iters, uint8_t* qstatus, void* ws, size_t ws_bytes,
                       cudaStream_t stream) {
  Call c{counts, x, t, phi, grad, dphidt, iters, qstatus, (char*)ws};
  const std::vector<uintptr_t> key = key_of(b, c, ws_bytes);
  if (b->exec && key == b->key) {
    HOPF_CUDA(cudaGraphLaunch(b->exec, stream));
    return HOPF_OK;
  }
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->nstreams == 0) {
    // autotune the number of worker streams on this call: capture and time
    // each candidate schedule (the second replay of each), keep the fastest
    const int cand[5] = {1, 2, 4, 8, 16};
    float best = 0.f;
    for (int ci = 0; ci < 5; ++ci) {
      cudaGraphExec_t ex = nullptr;
      hopf_status st = capture(b, c, cand[ci], &ex);
      if (st != HOPF_OK) return st;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        cudaError_t e = cudaEventRecord(b->t0, stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(ex, stream);
        if (e == cudaSuccess) e = cudaEventRecord(b->t1, stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(b->t1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->t0, b->t1);
        if (e != cudaSuccess) {
          cudaGraphExecDestroy(ex);
          return cuda_fail(e, "batch autotune replay");
        }
      }
      b->tuned_ms[ci] = ms;
      if (b->nstreams == 0 || ms < best) {
        best = ms;
        b->nstreams = cand[ci];
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = ex;
      } else {
        cudaGraphExecDestroy(ex);
      }
    }
    b->key = key;
    b->used_graph = 1;
    return HOPF_OK;  // the kept graph has already produced this call's results
  }
  hopf_status st = capture(b, c, b->nstreams, &b->exec);
  if (st != HOPF_OK) return st;
  b->key = key;
  b->used_graph = 1;
  HOPF_CUDA(cudaGraphLaunch(b->exec, stream));
  return HOPF_OK;
}

hopf_status batch_info(hopf_batch b, int32_t* nstreams, int32_t* used_graph, float* tuned_ms) {
  if (nstreams) *nstreams = b->nstreams;
  if (used_graph) *used_graph = b->used_graph;
  if (tuned_ms) std::memcpy(tuned_ms, b->tuned_ms, sizeof(b->tuned_ms));
  return HOPF_OK;
}

}  // namespace hopf
