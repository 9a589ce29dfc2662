// Ragged batch: many instances (each its own A, H, n and query count) in one
// CUDA graph replay.
//
// The method evaluates every query on its own, with no shared state (Section
// 1; Section 4.5 runs queries one per core), so a batch of instances is a set
// of independent evaluations.  Two schedules:
//   * persistent (enqueue_persistent): one cooperative launch of the ragged
//     solver (k_ragged) runs every tensor-core dense instance on a schedule
//     of CTA groups (wide instances on the whole grid, the others on lanes of
//     it) and then every diagonal instance from a shared work list; the
//     graph holds that launch, a copy of the schedule and the instances'
//     arguments from pinned host memory, and a memset of their barrier words;
//   * streams (enqueue): the kernels a single hopf_eval would launch, per
//     instance, forked onto worker streams and joined back.
// Instances the persistent solver does not take (dense FP32 CUDA-core, the
// diagonal runtime kinds, diagonal n > 4096) run their own launches beside
// it.  The autotuner on the first call captures and times candidate graphs
// (the persistent schedule with 4 to 32 lanes, with some CTAs starting on the
// diagonal work list, or with every dense instance on lanes; the stream
// schedule with 8 and 16 lanes, or with 1 to 16 when only streams are
// allowed) and keeps the fastest.  Later calls with the same buffers and
// counts replay it.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "hopf_internal.h"

struct hopf_batch_s {
  std::vector<hopf_handle> inst;
  // lanes 0..15 for the side-by-side work, the last stream for wide solves
  static constexpr int kMaxStreams = 17;  // (the persistent schedule's 32 lanes are CTA groups, not streams)
  cudaStream_t workers[kMaxStreams] = {};
  cudaStream_t origin = nullptr;  // capture origin (the caller's stream may be the legacy default stream)
  cudaEvent_t fork = nullptr, wide_done = nullptr, join[kMaxStreams] = {}, t0 = nullptr, t1 = nullptr;
  int nstreams = 0;          // tuned number of lanes (0: not tuned yet)
  int mode = 0;              // 0: tune both schedules, 1: persistent only, 2: streams only
  int chosen = 0;            // schedule of the kept graph: 1 persistent, 2 streams
  bool wide_on_lanes = false;  // persistent: wide dense instances on lanes too
  int reserve = 0;             // persistent: CTAs that start on the diagonal work list
  float tuned_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float streams_ms = 0.f;
  void* staging = nullptr;   // pinned host copy of the persistent schedule and arguments
  size_t staging_bytes = 0;
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

// The persistent schedule's area at the end of the batch workspace (and the
// same layout in the pinned staging buffer): instance records, the per-CTA
// schedule, the diagonal work descriptors, then the barrier words (zeroed by
// every replay).
struct RagLayout {
  size_t dense, diag, sched, sched_off, dinfo, ctrl, total;
};

RagLayout rag_layout(hopf_batch b) {
  const size_t m = b->inst.size();
  const int grid = b->inst.empty() ? 1 : b->inst[0]->num_sms;
  RagLayout L;
  size_t o = 0;
  L.dense = o;
  o += round_up(m * ragged_dense_record_bytes(), 256);
  L.diag = o;
  o += round_up(m * ragged_diag_record_bytes(), 256);
  L.sched = o;
  o += round_up((size_t)grid * m * sizeof(int4), 256);
  L.sched_off = o;
  o += round_up((size_t)(grid + 1) * sizeof(int), 256);
  L.dinfo = o;
  o += round_up(m * sizeof(int4), 256);
  L.ctrl = o;
  o += round_up(m * 128 + 64, 256);
  L.total = o;
  return L;
}

size_t inst_ws_total(hopf_batch b, const int64_t* counts) {
  size_t s = 0;
  for (size_t i = 0; i < b->inst.size(); ++i) s += ws_of(b->inst[i], counts[i]);
  return round_up(s, 256);
}

// Enqueue the batch as one persistent launch (plus the own launches of the
// instances it does not take, on a side stream).
hopf_status enqueue_persistent(hopf_batch b, const Call& c, int ns, bool wide_on_lanes, int reserve,
                               cudaStream_t stream) {
  const int m = (int)b->inst.size();
  const int grid = b->inst[0]->num_sms;
  // the last `reserve` CTAs start on the diagonal work list; the dense
  // schedule runs on the others (every CTA takes diagonal work when its own
  // list is done)
  const int gd = std::max(1, grid - std::max(0, reserve));
  std::vector<int64_t> qoff(m + 1, 0), xoff(m + 1, 0);
  std::vector<size_t> wsoff(m + 1, 0);
  std::vector<double> cost(m);
  std::vector<int> wide, narrow, diag, own;
  for (int i = 0; i < m; ++i) {
    hopf_handle h = b->inst[i];
    qoff[i + 1] = qoff[i] + c.counts[i];
    xoff[i + 1] = xoff[i] + c.counts[i] * h->n;
    wsoff[i + 1] = wsoff[i] + ws_of(h, c.counts[i]);
    cost[i] = cost_of(h, c.counts[i]);
    if (c.counts[i] == 0) continue;
    if (h->a_kind == HOPF_A_DIAG) {
      if (ragged_diag_class(h) >= 0) diag.push_back(i);
      else own.push_back(i);
    } else if (h->precision == HOPF_P_FP32) {
      own.push_back(i);
    } else if (!wide_on_lanes && tiles_of(h, c.counts[i]) >= gd) {
      wide.push_back(i);
    } else {
      narrow.push_back(i);
    }
  }
  const RagLayout L = rag_layout(b);
  char* st = (char*)b->staging;
  char* dev = c.ws + inst_ws_total(b, c.counts);
  std::memset(st, 0, L.ctrl);
  // dense records: wide ones first, longest first, then the lanes' ones
  std::stable_sort(wide.begin(), wide.end(), [&](int a, int d) { return cost[a] > cost[d]; });
  ns = std::max(1, std::min(ns, gd));
  std::vector<int> lane(m, 0), order_n;
  assign(narrow, cost, ns, &lane, &order_n);
  std::vector<int> dense_ids(wide);
  dense_ids.insert(dense_ids.end(), order_n.begin(), order_n.end());
  std::vector<int> slot(m, -1);
  for (size_t j = 0; j < dense_ids.size(); ++j) {
    const int i = dense_ids[j];
    hopf_handle h = b->inst[i];
    slot[i] = (int)j;
    DenseWs w;
    hopf_status s = dense_carve(h, c.counts[i], c.ws + wsoff[i], ws_of(h, c.counts[i]), &w);
    if (s != HOPF_OK) return s;
    w.bar = (unsigned*)(dev + L.ctrl + j * 128);
    w.err = (int*)(dev + L.ctrl + j * 128 + 64);
    s = ragged_build_dense(h, w, c.x + xoff[i], c.t + qoff[i], c.phi + qoff[i], c.grad + xoff[i],
                           c.dphidt ? c.dphidt + qoff[i] : nullptr, c.iters ? c.iters + qoff[i] : nullptr,
                           c.qstatus ? c.qstatus + qoff[i] : nullptr, st + L.dense + j * ragged_dense_record_bytes());
    if (s != HOPF_OK) return s;
  }
  // per-CTA schedule: every wide instance on the gd dense CTAs, then the
  // lane's instances in order on the lane (lane l holds CTAs [l gd / ns,
  // (l + 1) gd / ns))
  int4* sched = (int4*)(st + L.sched);
  int* soff = (int*)(st + L.sched_off);
  int e = 0;
  for (int l = 0, cta = 0; l < ns; ++l) {
    const int l0 = (int)((int64_t)l * gd / ns), l1 = (int)((int64_t)(l + 1) * gd / ns);
    for (; cta < l1; ++cta) {
      soff[cta] = e;
      for (int i : wide) sched[e++] = make_int4(slot[i], cta, gd, 0);
      for (int i : order_n)
        if (lane[i] == l) sched[e++] = make_int4(slot[i], cta - l0, l1 - l0, 0);
    }
  }
  for (int cta = gd; cta <= grid; ++cta) soff[cta] = e;
  // diagonal work: instances longest first; items of 256 queries (a thread
  // each), 8 (a warp each) or 1 (256 threads) by the instance's group shape
  std::stable_sort(diag.begin(), diag.end(), [&](int a, int d) { return cost[a] > cost[d]; });
  int4* dinfo = (int4*)(st + L.dinfo);
  int items = 0;
  for (size_t d = 0; d < diag.size(); ++d) {
    const int i = diag[d];
    hopf_handle h = b->inst[i];
    const int cls = ragged_diag_class(h);
    const int per = cls <= 2 ? 256 : cls <= 5 ? 8 : 1;
    ragged_build_diag(h, c.counts[i], c.x + xoff[i], c.t + qoff[i], c.phi + qoff[i], c.grad + xoff[i],
                      c.dphidt ? c.dphidt + qoff[i] : nullptr, c.iters ? c.iters + qoff[i] : nullptr,
                      c.qstatus ? c.qstatus + qoff[i] : nullptr, st + L.diag + d * ragged_diag_record_bytes());
    dinfo[d] = make_int4((int)c.counts[i], per, cls, items);
    items += (int)((c.counts[i] + per - 1) / per);
  }
  cudaStream_t side = b->workers[0];
  HOPF_CUDA(cudaMemcpyAsync(dev, st, L.ctrl, cudaMemcpyHostToDevice, stream));
  HOPF_CUDA(cudaMemsetAsync(dev + L.ctrl, 0, L.total - L.ctrl, stream));
  if (!own.empty()) {
    HOPF_CUDA(cudaEventRecord(b->fork, stream));
    HOPF_CUDA(cudaStreamWaitEvent(side, b->fork, 0));
    for (int i : own) {
      b->inst[i]->grid_cap = 0;
      hopf_status s = launch_one(b->inst[i], c.counts[i], c, qoff[i], xoff[i], wsoff[i], side);
      if (s != HOPF_OK) return s;
    }
    HOPF_CUDA(cudaEventRecord(b->join[0], side));
  }
  if (!dense_ids.empty() || items > 0) {
    hopf_status s = ragged_launch(dev + L.dense, (const int4*)(dev + L.sched), (const int*)(dev + L.sched_off), grid,
                                  dev + L.diag, (const int4*)(dev + L.dinfo), (int)diag.size(), items,
                                  (unsigned*)(dev + L.ctrl + (size_t)m * 128), stream);
    if (s != HOPF_OK) return s;
  }
  if (!own.empty()) HOPF_CUDA(cudaStreamWaitEvent(stream, b->join[0], 0));
  return HOPF_OK;
}

// Capture the batch as a graph on the batch's own origin stream (capture is
// not allowed on the legacy default stream); the graph is launched on the
// caller's stream.  On failure the capture is abandoned cleanly.
hopf_status capture(hopf_batch b, const Call& c, int ns, bool persistent, bool wide_on_lanes, int reserve,
                    cudaGraphExec_t* exec) {
  *exec = nullptr;
  cudaStream_t o = b->origin;
  HOPF_CUDA(cudaStreamBeginCapture(o, cudaStreamCaptureModeThreadLocal));
  hopf_status st = persistent ? enqueue_persistent(b, c, ns, wide_on_lanes, reserve, o) : enqueue(b, c, ns, o);
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
  if (b->staging) cudaFreeHost(b->staging);
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
  b->staging_bytes = rag_layout(b).total;
  B_CALL(cudaHostAlloc(&b->staging, b->staging_bytes, cudaHostAllocDefault));
#undef B_CALL
  *out = b;
  return HOPF_OK;
}

void batch_destroy(hopf_batch b) { free_batch(b); }

size_t batch_count(hopf_batch b) { return b->inst.size(); }

size_t batch_workspace(hopf_batch b, const int64_t* counts) { return inst_ws_total(b, counts) + rag_layout(b).total; }

void batch_set_mode(hopf_batch b, int mode) {
  b->mode = mode;
  b->nstreams = 0;  // tune again on the next call
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->key.clear();
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
    // autotune on this call: capture and time (the second replay of each)
    // the persistent schedule with 4, 8, 16 and 32 lanes (wide dense
    // instances on the whole grid), with 8 and 16 lanes and 8 or 16 CTAs
    // starting on the diagonal work list, and with 8 lanes taking every
    // dense instance (so that the instances' last iterations overlap); then
    // the stream schedule with 8 and 16 lanes; keep the fastest
    struct Cand {
      int ns;
      bool persistent, wide_on_lanes;
      int reserve;
    };
    std::vector<Cand> cands;
    if (b->mode != 2)
      for (Cand cd : {Cand{4, true, false, 0}, Cand{8, true, false, 0}, Cand{16, true, false, 0},
                      Cand{32, true, false, 0}, Cand{8, true, false, 8}, Cand{16, true, false, 8},
                      Cand{16, true, false, 16}, Cand{8, true, true, 0}})
        cands.push_back(cd);
    else
      for (int ns : {1, 2, 4, 8, 16}) cands.push_back(Cand{ns, false, false, 0});
    float best = 0.f;
    auto trial = [&](const Cand& cd, float* out_ms) -> hopf_status {
      cudaGraphExec_t ex = nullptr;
      hopf_status st = capture(b, c, cd.ns, cd.persistent, cd.wide_on_lanes, cd.reserve, &ex);
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
      *out_ms = ms;
      if (b->nstreams == 0 || ms < best) {
        best = ms;
        b->nstreams = cd.ns;
        b->chosen = cd.persistent ? 1 : 2;
        b->wide_on_lanes = cd.wide_on_lanes;
        b->reserve = cd.reserve;
        if (b->exec) cudaGraphExecDestroy(b->exec);
        b->exec = ex;
      } else {
        cudaGraphExecDestroy(ex);
      }
      return HOPF_OK;
    };
    for (size_t ci = 0; ci < cands.size(); ++ci) {
      hopf_status st = trial(cands[ci], &b->tuned_ms[ci]);
      if (st != HOPF_OK) return st;
    }
    if (b->mode == 0) {
      // the stream schedule at 8 and 16 lanes (its best lane count need not be
      // the persistent schedule's)
      float ms8 = 0.f, ms16 = 0.f;
      hopf_status st = trial(Cand{8, false, false, 0}, &ms8);
      if (st == HOPF_OK) st = trial(Cand{16, false, false, 0}, &ms16);
      if (st != HOPF_OK) return st;
      b->streams_ms = ms8 < ms16 ? ms8 : ms16;
    }
    if (b->chosen == 1) {
      // the persistent graph copies its schedule from the staging buffer,
      // which the later candidates overwrote: capture the kept one again
      // (the outputs of this call are complete already)
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
      hopf_status st = capture(b, c, b->nstreams, true, b->wide_on_lanes, b->reserve, &b->exec);
      if (st != HOPF_OK) return st;
    }
    b->key = key;
    b->used_graph = b->chosen;
    return HOPF_OK;
  }
  hopf_status st = capture(b, c, b->nstreams, b->chosen != 2, b->wide_on_lanes, b->reserve, &b->exec);
  if (st != HOPF_OK) return st;
  b->key = key;
  b->used_graph = b->chosen == 2 ? 2 : 1;
  HOPF_CUDA(cudaGraphLaunch(b->exec, stream));
  return HOPF_OK;
}

hopf_status batch_info(hopf_batch b, int32_t* nstreams, int32_t* used_graph, float* tuned_ms) {
  if (nstreams) *nstreams = b->nstreams;
  if (used_graph) *used_graph = b->used_graph;
  if (tuned_ms) std::memcpy(tuned_ms, b->tuned_ms, sizeof(b->tuned_ms));  // 8 floats
  return HOPF_OK;
}

}  // namespace hopf
