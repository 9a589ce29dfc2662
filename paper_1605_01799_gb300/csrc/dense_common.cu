// Dense-A path: workspace layout, query initialisation and the final reduction.
//
// State of one query in the batched solver (both forms):
//   y = x - c and u, where u^k = v^k + b^{k-1} is the argument of the d-update
//   (eq. 3.4(b)); d^k = prox(u^k) and b^k = u^k - d^k follow from it, so u is
//   the whole split Bregman state after the first step.  The start
//   v^0 = d^0 = y, b^0 = 0 (Section 3.1) is u^0 = d^0 = y with the first step
//   taking p^0 = y instead of prox(u^0).
#include <cuda_fp16.h>

#include "common.cuh"
#include "hopf_internal.h"

namespace hopf {

// The MIXED form starts with SPLIT iterations (l1 and weighted l1).
bool two_stage(const hopf_handle h) {
  return h->precision == HOPF_P_MIXED && h->split_start > 0.0 && h->h_kind != HOPF_H_L2;
}

static size_t carve_sizes(const hopf_handle h, int64_t batch, size_t* out /* 32 */) {
  const int64_t B_pad = round_up(batch > 0 ? batch : 1, 256);
  const int64_t np = h->n_pad;
  const int rt = (int)(np / 128);
  const bool tc = h->precision != HOPF_P_FP32;
  size_t s[32] = {0};
  s[0] = B_pad * np * 4;                 // y
  s[1] = B_pad * np * 4;                 // u
  s[2] = tc ? B_pad * np * 2 : 0;        // ph
  s[3] = tc ? B_pad * np * 2 : 0;        // pl
  s[4] = tc ? B_pad * np * 2 : 0;        // g
  s[5] = (size_t)2 * 2 * 2 * rt * B_pad * 4; // part (two buffer sets; the FP32 solver uses the first)
  s[6] = (size_t)2 * rt * B_pad * 8;     // fpart
  s[7] = B_pad * 4;                      // tau
  s[8] = B_pad * 4;                      // tq
  s[9] = B_pad * 4;                      // scale
  s[10] = B_pad * 4;                     // qiter
  s[11] = B_pad * 4;                     // qdone
  s[12] = 64;                            // bar (16 unsigned)
  s[13] = 64;                            // err
  s[14] = 2 * B_pad * 4;                 // qact (by decision parity)
  s[15] = 2 * (B_pad / 128) * 4;         // tile_act (tensor-core solver: last decision with active slots, and its count)
  s[16] = tc ? B_pad * np * 4 : 0;       // y_b
  s[17] = B_pad * np * 4;                // u_b (FP32 solver: u of odd iterations)
  s[18] = tc ? B_pad * np * 2 : 0;       // ph_b
  s[19] = tc ? B_pad * np * 2 : 0;       // pl_b
  s[20] = B_pad * 4;                     // scale_b
  s[21] = 2 * B_pad * 4;                 // qact_b (by decision parity)
  s[22] = 2 * B_pad * 4;                 // sq
  s[23] = tc ? B_pad * np * 4 : 0;       // ufin
  s[24] = B_pad * 4;                     // sfin
  s[25] = 2 * B_pad * 4;                 // taus
  const bool split = h->precision == HOPF_P_SPLIT || two_stage(h);
  for (int i = 26; i < 30; ++i) s[i] = split ? B_pad * np * 2 : 0;  // qh, ql, qh_b, ql_b
  s[30] = tc ? B_pad * 4 : 0;            // qiter0 (two-stage solve: iterations of the first stage)
  size_t total = 0;
  for (int i = 0; i < 31; ++i) {
    if (out) out[i] = total;
    total += round_up(s[i], 256);
  }
  return total;
}

size_t dense_workspace(const hopf_handle h, int64_t batch) { return carve_sizes(h, batch, nullptr); }

hopf_status dense_carve(const hopf_handle h, int64_t batch, void* ws, size_t ws_bytes, DenseWs* d) {
  size_t off[32];
  size_t total = carve_sizes(h, batch, off);
  if (ws_bytes < total) return fail(HOPF_EINVAL, "hopf_eval: workspace too small");
  char* p = (char*)ws;
  d->B = batch;
  d->B_pad = round_up(batch, 256);
  d->rt = h->n_pad / 128;
  d->y = (float*)(p + off[0]);
  d->u = (float*)(p + off[1]);
  const bool tc = h->precision != HOPF_P_FP32;
  d->ph = tc ? (uint16_t*)(p + off[2]) : nullptr;
  d->pl = tc ? (uint16_t*)(p + off[3]) : nullptr;
  d->g = tc ? (uint16_t*)(p + off[4]) : nullptr;
  d->part = (float*)(p + off[5]);
  d->fpart = (double*)(p + off[6]);
  d->tau = (float*)(p + off[7]);
  d->tq = (float*)(p + off[8]);
  d->scale = (float*)(p + off[9]);
  d->qiter = (int*)(p + off[10]);
  d->qdone = (int*)(p + off[11]);
  d->bar = (unsigned*)(p + off[12]);
  d->err = (int*)(p + off[13]);
  d->qact = (int*)(p + off[14]);
  d->tile_act = (int*)(p + off[15]);
  d->y_b = tc ? (float*)(p + off[16]) : nullptr;
  d->u_b = (float*)(p + off[17]);
  d->ph_b = tc ? (uint16_t*)(p + off[18]) : nullptr;
  d->pl_b = tc ? (uint16_t*)(p + off[19]) : nullptr;
  d->scale_b = (float*)(p + off[20]);
  d->qact_b = (int*)(p + off[21]);
  d->sq = (int*)(p + off[22]);
  d->ufin = tc ? (float*)(p + off[23]) : nullptr;
  d->sfin = (float*)(p + off[24]);
  d->taus = (float*)(p + off[25]);
  const bool split = h->precision == HOPF_P_SPLIT || two_stage(h);
  d->qh = split ? (uint16_t*)(p + off[26]) : nullptr;
  d->ql = split ? (uint16_t*)(p + off[27]) : nullptr;
  d->qh_b = split ? (uint16_t*)(p + off[28]) : nullptr;
  d->ql_b = split ? (uint16_t*)(p + off[29]) : nullptr;
  d->qiter0 = tc ? (int*)(p + off[30]) : nullptr;
  return HOPF_OK;
}

// y = x - c, u = y in the padded layout; per-query time data; padding
// queries start done.
__global__ void k_dense_init(const float* __restrict__ x, const float* __restrict__ t, const float* __restrict__ c,
                             int n, int np, int64_t B, int64_t B_pad, float lam, float* __restrict__ y,
                             float* __restrict__ u, float* __restrict__ tau, float* __restrict__ tq,
                             int* __restrict__ qiter, int* __restrict__ qdone, int* __restrict__ sq,
                             float* __restrict__ taus) {
  const int64_t q = blockIdx.x;  // one CTA per query (1-D grid: no 65,535 limit)
  if (q >= B_pad) return;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    float v = 0.f;
    if (q < B && i < n) v = x[q * n + i] - c[i];
    y[q * np + i] = v;
    u[q * np + i] = v;
  }
  if (threadIdx.x == 0) {
    const float tt = q < B ? t[q] : 0.f;
    tq[q] = tt;
    tau[q] = tt / lam;
    taus[q] = tt / lam;
    qiter[q] = 0;
    qdone[q] = q < B ? 0 : 1;
    sq[q] = (int)q;  // slot q starts with query q
  }
}

// Second stage of the two-stage solve: every slot plane is rebuilt from the
// query-indexed results of the first (whose compactions moved the slots):
// y = x - c, u = the query's last u, the operand planes the FP16 split of
// p = prox(u) (l1 and weighted l1 shrink by (t / lambda) w), slot q holding
// query q.  The first stage's iteration count moves to qiter0; a query it
// stopped at max_iter stays stopped (qdone 2, its count kept).
__global__ void k_dense_init_warm(const float* __restrict__ x, const float* __restrict__ t,
                                  const float* __restrict__ c, const float* __restrict__ wt,
                                  const float* __restrict__ ufin, int n, int np, int64_t B, int64_t B_pad, float lam,
                                  int max_iter, float* __restrict__ y, float* __restrict__ u, uint16_t* __restrict__ ph,
                                  uint16_t* __restrict__ pl, float* __restrict__ tau, float* __restrict__ tq,
                                  int* __restrict__ qiter, int* __restrict__ qiter0, int* __restrict__ qdone,
                                  int* __restrict__ sq, float* __restrict__ taus) {
  const int64_t q = blockIdx.x;  // one CTA per query
  if (q >= B_pad) return;
  const float tt = q < B ? t[q] : 0.f;
  const float tl = tt / lam;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    float yv = 0.f, uv = 0.f;
    if (q < B && i < n) {
      yv = x[q * n + i] - c[i];
      uv = ufin[q * np + i];
    }
    const float pv = shrink1(uv, tl * wt[i]);
    const __half hi = __float2half_rn(pv);
    y[q * np + i] = yv;
    u[q * np + i] = uv;
    ph[q * np + i] = __half_as_ushort(hi);
    pl[q * np + i] = __half_as_ushort(__float2half_rn((pv - __half2float(hi)) * 2048.f));  // 2^11: the split's scale
  }
  if (threadIdx.x == 0) {
    const int k1 = q < B ? qiter[q] : 0;
    const bool capped = q < B && k1 >= max_iter;
    tq[q] = tt;
    tau[q] = tl;
    taus[q] = tl;
    qiter0[q] = k1;
    qiter[q] = capped ? k1 : 0;
    qdone[q] = q >= B ? 1 : capped ? 2 : 0;
    sq[q] = (int)q;
  }
}

hopf_status dense_init_warm(hopf_handle h, DenseWs& w, const float* x, const float* t, cudaStream_t s) {
  // the error word carries over: a first stage that gave up aborts the second
  HOPF_CUDA(cudaMemsetAsync(w.bar, 0, 64, s));
  HOPF_CUDA(cudaMemsetAsync(w.tile_act, 0, (size_t)2 * (w.B_pad / 128) * 4, s));
  k_dense_init_warm<<<(unsigned)w.B_pad, 256, 0, s>>>(x, t, h->d_cf, h->d_wf, w.ufin, h->n, h->n_pad, w.B, w.B_pad,
                                                      (float)h->lambda, h->max_iter, w.y, w.u, w.ph, w.pl, w.tau,
                                                      w.tq, w.qiter, w.qiter0, w.qdone, w.sq, w.taus);
  HOPF_CUDA(cudaGetLastError());
  return HOPF_OK;
}

hopf_status dense_init(hopf_handle h, DenseWs& w, const float* x, const float* t, cudaStream_t s) {
  HOPF_CUDA(cudaMemsetAsync(w.bar, 0, 64, s));
  HOPF_CUDA(cudaMemsetAsync(w.err, 0, 64, s));
  HOPF_CUDA(cudaMemsetAsync(w.tile_act, 0, (size_t)2 * (w.B_pad / 128) * 4, s));
  k_dense_init<<<(unsigned)w.B_pad, 256, 0, s>>>(x, t, h->d_cf, h->n, h->n_pad, w.B, w.B_pad, (float)h->lambda, w.y,
                                                 w.u, w.tau, w.tq, w.qiter, w.qdone, w.sq, w.taus);
  HOPF_CUDA(cudaGetLastError());
  return HOPF_OK;
}

// phi = sum_r fpart0 - c0 - t H, H = sum_r fpart1 (l1) or its square root (l2).
__global__ void k_dense_finalize(const double* __restrict__ fpart, const int* __restrict__ qiter,
                                 const int* __restrict__ qdone, const float* __restrict__ tq, int rt, int64_t B,
                                 int64_t B_pad, double c0, int h_kind, const int* __restrict__ err, double* phi,
                                 float* dphidt, int32_t* iters, uint8_t* qstatus) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B) return;
  double s = 0.0, hh = 0.0;
  for (int r = 0; r < rt; ++r) {
    s += fpart[(int64_t)r * B_pad + q];
    hh += fpart[(int64_t)(rt + r) * B_pad + q];
  }
  const double H = h_kind == H_L2 ? sqrt(hh) : hh;
  const double p = s - c0 - (double)tq[q] * H;
  phi[q] = p;
  if (dphidt) dphidt[q] = (float)(-H);
  if (iters) iters[q] = qiter[q];
  if (qstatus) {
    uint8_t st = qdone[q] == 1 ? Q_OK : Q_NOT_CONVERGED;
    if (!isfinite(p)) st = Q_NONFINITE;
    if (!(tq[q] >= 0.f)) st = Q_BAD_INPUT;  // t < 0 or NaN
    if (*err != ERR_NONE) st = Q_ABORTED;
    qstatus[q] = st;
  }
}

hopf_status dense_finalize(hopf_handle h, DenseWs& w, double* phi, float* dphidt, int32_t* iters, uint8_t* qstatus,
                           cudaStream_t s) {
  k_dense_finalize<<<(unsigned)((w.B + 255) / 256), 256, 0, s>>>(w.fpart, w.qiter, w.qdone, w.tq, w.rt, w.B,
                                                                  w.B_pad, h->c0, h->h_kind, w.err, phi, dphidt,
                                                                  iters, qstatus);
  HOPF_CUDA(cudaGetLastError());
  return HOPF_OK;
}

}  // namespace hopf
