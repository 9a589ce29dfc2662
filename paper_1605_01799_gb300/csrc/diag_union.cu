// Unions of initial data, the maximum over Hamiltonians and the closest point
// to a union (Sections 2.2 and 3.2) on the diagonal path.
#include <mutex>

#include "diag_query.cuh"

namespace hopf {

// ---------------------------------------------------------------------------
// Union of initial data (Section 2.2): phi = min_i phi_i.  Pass 1 evaluates
// every (query, part) pair; pass 2 picks the minimising part (ties to the
// smallest index) and re-runs it to write its gradient.
constexpr int kMaxParts = 64;

struct UnionArgs {
  DiagPart<float> parts[kMaxParts];  // by value: the launch needs no host copy
  int K, n;
  int64_t batch;
  const float* x;
  const float* t;       // time per query (union eval) or null (closest point)
  double* phi_parts;    // [batch][K]
  float* s_parts;       // [batch][K] Newton root per part (closest point)
  int32_t* it_parts;    // [batch][K]
  uint8_t* st_parts;    // [batch][K]
  unsigned* best;       // [batch] smallest root found so far (float bits; closest point)
  int maximize;         // phi pass: keep the largest phi_i (maximum over Hamiltonians)
  float s_tol;
  int max_newton;
  // outputs
  double* phi;
  float* grad;
  int32_t* argmin;
  int32_t* iters;
  uint8_t* qstatus;
  float* dist;
  float* closest;
};

template <int G>
__device__ __forceinline__ int64_t group_index() {
  if constexpr (G == 32) return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  else return (int64_t)blockIdx.x;
}

template <int G, int VPT, bool GEN>
__global__ void __launch_bounds__(block_of<G>()) k_union_parts(UnionArgs U) {
  const int64_t pair = group_index<G>();
  if (pair >= U.batch * U.K) return;
  const int64_t q = pair / U.K;
  const int part = (int)(pair % U.K);
  const DiagPart<float> P = U.parts[part];
  Query<float, G, VPT> Q;
  Q.load(P, U.x + q * U.n, U.n);
  Q.cold_start();
  bool conv;
  const int k = Q.template solve<GEN>(P, U.t[q], &conv);
  double H;
  const double phi = Q.template objective<GEN>(P, (double)U.t[q], &H);
  if (group_lane<G>() == 0) {
    U.phi_parts[pair] = phi;
    U.it_parts[pair] = k;
    U.st_parts[pair] = !isfinite(phi) ? Q_NONFINITE : (conv ? Q_OK : Q_NOT_CONVERGED);
  }
}

template <int G, int VPT, bool GEN>
__global__ void __launch_bounds__(block_of<G>()) k_union_pick(UnionArgs U) {
  const int64_t q = group_index<G>();
  if (q >= U.batch) return;
  // the minimum over initial data (unions) or the maximum over Hamiltonians;
  // ties go to the smallest index
  int best = 0;
  double bv = U.phi_parts[q * U.K];
  for (int i = 1; i < U.K; ++i) {
    const double v = U.phi_parts[q * U.K + i];
    const bool better = U.maximize ? v > bv : v < bv;
    if (better || (isnan(bv) && !isnan(v))) {
      bv = v;
      best = i;
    }
  }
  const DiagPart<float> P = U.parts[best];
  Query<float, G, VPT> Q;
  Q.load(P, U.x + q * U.n, U.n);
  Q.cold_start();
  bool conv;
  Q.template solve<GEN>(P, U.t[q], &conv);
  const int l = group_lane<G>();
#pragma unroll
  for (int j = 0; j < VPT; ++j) {
    const int i = l + G * j;
    if (i < U.n) U.grad[q * U.n + i] = Q.d[j];
  }
  if (l == 0) {
    U.phi[q] = bv;
    U.argmin[q] = best;
    if (U.iters) U.iters[q] = U.it_parts[q * U.K + best];
    if (U.qstatus) U.qstatus[q] = !(U.t[q] >= 0.f) ? Q_BAD_INPUT : U.st_parts[q * U.K + best];
  }
}

// Newton on s for psi_i(y, s) = 0 (Section 3.2), warm-started solves.
template <int G, int VPT>
__global__ void __launch_bounds__(block_of<G>()) k_closest_parts(UnionArgs U) {
  const int64_t pair = group_index<G>();
  if (pair >= U.batch * U.K) return;
  const int64_t q = pair / U.K;
  const int part = (int)(pair % U.K);
  const DiagPart<float> P = U.parts[part];
  Query<float, G, VPT> Q;
  Q.load(P, U.x + q * U.n, U.n);
  Q.cold_start();
  double s = 0.0;
  bool ok = false, finite = true, pruned = false;
  int l;
  for (l = 0; l < U.max_newton; ++l) {
    bool conv;
    Q.template solve<false>(P, (float)s, &conv);
    double H;
    const double psi = Q.template objective<false>(P, s, &H);
    // |grad psi| = |d| (H = l2 here)
    if (!(H > 0.0) || !isfinite(psi)) {
      finite = isfinite(psi);
      break;
    }
    const double ds = psi / H;
    s += ds;
    if (fabs(ds) <= (double)U.s_tol * (s > 1.0 ? s : 1.0)) {
      ok = true;
      ++l;
      if (group_lane<G>() == 0 && s >= 0.0) atomicMin(U.best + q, __float_as_uint((float)s));
      break;
    }
    // psi is convex and non-increasing in s (a maximum of affine functions of
    // s with slopes -H(v) <= 0), so Newton from s = 0 rises monotonically to
    // the part's root: an iterate already past another part's root by a
    // clear margin (1e-3, far above the Newton tolerance) cannot be the
    // nearest part's, and the part stops.  The decision is the group's first
    // thread's, so the group stays together.
    float bs = __uint_as_float(*((volatile unsigned*)(U.best + q)));
    bs = Group<G, float>::bcast0(bs);
    if (s > (double)bs + 1e-3 * ((double)bs > 1.0 ? (double)bs : 1.0)) {
      pruned = true;
      ++l;
      break;
    }
  }
  if (group_lane<G>() == 0) {
    U.s_parts[pair] = (float)s;
    U.phi_parts[pair] = pruned ? INFINITY : s;  // a pruned part is not the nearest
    U.it_parts[pair] = l;
    U.st_parts[pair] = !finite ? Q_NONFINITE : (ok ? Q_OK : Q_NOT_CONVERGED);
  }
}

template <int G, int VPT>
__global__ void __launch_bounds__(block_of<G>()) k_closest_pick(UnionArgs U) {
  const int64_t q = group_index<G>();
  if (q >= U.batch) return;
  int best = 0;
  double bv = U.phi_parts[q * U.K];
  for (int i = 1; i < U.K; ++i) {
    const double v = U.phi_parts[q * U.K + i];
    if (v < bv || (isnan(bv) && !isnan(v))) {
      bv = v;
      best = i;
    }
  }
  const float s = U.s_parts[q * U.K + best];
  const int l = group_lane<G>();
  if (U.closest) {
    const DiagPart<float> P = U.parts[best];
    Query<float, G, VPT> Q;
    Q.load(P, U.x + q * U.n, U.n);
    Q.cold_start();
    bool conv;
    Q.template solve<false>(P, s, &conv);
    float nn = 0.f;
#pragma unroll
    for (int j = 0; j < VPT; ++j) nn += Q.d[j] * Q.d[j];
    nn = sqrtf(Group<G, float>::sum(nn));
    const float inv = nn > 0.f ? 1.f / nn : 0.f;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const int i = l + G * j;
      if (i < U.n) U.closest[q * U.n + i] = U.x[q * U.n + i] - s * Q.d[j] * inv;  // eq. projection_when_s_known
    }
  }
  if (l == 0) {
    U.dist[q] = s;
    U.argmin[q] = best;
    if (U.iters) U.iters[q] = U.it_parts[q * U.K + best];
    if (U.qstatus) U.qstatus[q] = U.st_parts[q * U.K + best];
  }
}

size_t union_workspace(int K, int n, int64_t batch) {
  (void)n;
  size_t b = (size_t)batch * K;
  return round_up(b * 8, 256) + round_up(b * 4, 256) + round_up(b * 4, 256) + round_up(b, 256) +
         round_up((size_t)batch * 4, 256);
}

static hopf_status carve_union(const hopf_handle* parts, int K, int64_t batch, void* ws, UnionArgs* U) {
  if (K > kMaxParts) return fail(HOPF_EUNSUPPORTED, "hopf_union: at most 64 parts");
  char* p = (char*)ws;
  size_t b = (size_t)batch * K;
  U->phi_parts = (double*)p;
  p += round_up(b * 8, 256);
  U->s_parts = (float*)p;
  p += round_up(b * 4, 256);
  U->it_parts = (int32_t*)p;
  p += round_up(b * 4, 256);
  U->st_parts = (uint8_t*)p;
  p += round_up(b, 256);
  U->best = (unsigned*)p;
  for (int i = 0; i < K; ++i) U->parts[i] = part_of<float>(parts[i]);
  U->K = K;
  U->n = parts[0]->n;
  U->batch = batch;
  return HOPF_OK;
}

template <int G, int VPT>
static void launch_union(UnionArgs& U, bool closest, cudaStream_t s) {
  const int64_t pairs = U.batch * U.K;
  const unsigned bx = G == 32 ? 128 : G;
  const int per = G == 32 ? 4 : 1;
  bool gen = false;
  for (int i = 0; i < U.K; ++i) gen = gen || generic_kind(U.parts[i]);
  if (!closest && gen) {
    k_union_parts<G, VPT, true><<<(unsigned)((pairs + per - 1) / per), bx, 0, s>>>(U);
    k_union_pick<G, VPT, true><<<(unsigned)((U.batch + per - 1) / per), bx, 0, s>>>(U);
  } else if (!closest) {
    k_union_parts<G, VPT, false><<<(unsigned)((pairs + per - 1) / per), bx, 0, s>>>(U);
    k_union_pick<G, VPT, false><<<(unsigned)((U.batch + per - 1) / per), bx, 0, s>>>(U);
  } else {
    k_closest_parts<G, VPT><<<(unsigned)((pairs + per - 1) / per), bx, 0, s>>>(U);
    k_closest_pick<G, VPT><<<(unsigned)((U.batch + per - 1) / per), bx, 0, s>>>(U);
  }
}

static hopf_status dispatch_union(UnionArgs& U, bool closest, cudaStream_t s) {
  const int n = U.n;
  if (n <= 64) launch_union<32, 2>(U, closest, s);
  else if (n <= 256) launch_union<32, 8>(U, closest, s);
  else if (n <= 512) launch_union<32, 16>(U, closest, s);
  else if (n <= 4096) launch_union<256, 16>(U, closest, s);
  else launch_union<512, 16>(U, closest, s);
  HOPF_CUDA(cudaGetLastError());
  return HOPF_OK;
}

hopf_status union_eval(const hopf_handle* parts, int K, int64_t batch, const float* x, const float* t, double* phi,
                       float* grad, int32_t* argmin, int32_t* iters, uint8_t* qstatus, void* ws, size_t,
                       cudaStream_t stream, bool maximize) {
  UnionArgs U{};
  hopf_status s = carve_union(parts, K, batch, ws, &U);
  if (s != HOPF_OK) return s;
  U.maximize = maximize ? 1 : 0;
  U.x = x;
  U.t = t;
  U.phi = phi;
  U.grad = grad;
  U.argmin = argmin;
  U.iters = iters;
  U.qstatus = qstatus;
  return dispatch_union(U, false, stream);
}

hopf_status union_closest(const hopf_handle* parts, int K, int64_t batch, const float* x, float s_tol,
                          int max_newton, float* dist, float* closest, int32_t* argmin, int32_t* newton,
                          uint8_t* qstatus, void* ws, size_t, cudaStream_t stream) {
  UnionArgs U{};
  hopf_status s = carve_union(parts, K, batch, ws, &U);
  if (s != HOPF_OK) return s;
  U.x = x;
  U.t = nullptr;
  U.s_tol = s_tol;
  U.max_newton = max_newton;
  U.dist = dist;
  U.closest = closest;
  U.argmin = argmin;
  U.iters = newton;
  U.qstatus = qstatus;
  // best roots start at a huge positive float (bytes 0x7f: 3.4e38)
  HOPF_CUDA(cudaMemsetAsync(U.best, 0x7f, (size_t)batch * 4, stream));
  return dispatch_union(U, true, stream);
}

// ---------------------------------------------------------------------------
// Allocation-free distance / closest point.
//
// Some callers must not allocate device memory once they are running: a
// controller that queries the distance to a set of obstacles at a fixed rate,
// code inside a region whose memory budget is fixed in advance, or a host
// that hands this library no allocator at all.  For them the scratch of
// union_closest lives in one static device array that every GPU loading the
// library holds until the process exits.  The device address of that array
// is looked up once per device, with the device current, on the first call
// there; calls that overlap on the GPU share the array and race.  No entry of
// the scratch needs to start at zero: every slot a call reads is written
// earlier in the same call.
constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[256];

static hopf_status noalloc_scratch(void** out) {
  int dev = 0;
  HOPF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) return fail(HOPF_EUNSUPPORTED, "no-alloc scratch: device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_noalloc_addr[dev] = ptr;
  }
  *out = g_noalloc_addr[dev];
  return HOPF_OK;
}

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

hopf_status union_closest_noalloc(const hopf_handle* parts, int K, int64_t batch, const float* x, float s_tol,
                                  int max_newton, float* dist, float* closest, int32_t* argmin, int32_t* newton,
                                  uint8_t* qstatus, cudaStream_t stream) {
  const size_t need = union_workspace(K, parts[0]->n, batch);
  if (need > kNoAllocScratchBytes)
    return fail(HOPF_EINVAL, "hopf_union_closest_noalloc: batch * (17 parts + 4) bytes exceed the 8 MiB static "
                             "scratch (about 399,000 queries with one part, 30,000 with 16)");
  void* ws = nullptr;
  hopf_status s = noalloc_scratch(&ws);
  if (s != HOPF_OK) return s;
  return union_closest(parts, K, batch, x, s_tol, max_newton, dist, closest, argmin, newton, qstatus, ws, need,
                       stream);
}

}  // namespace hopf
