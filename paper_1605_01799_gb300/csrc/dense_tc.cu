// Dense A on the 5th-generation tensor cores (tcgen05 + TMA + TMEM), sm_103a.
//
// Three forms of the split Bregman iteration (eq. 3.4(a)-(c)) in terms of the
// d-update argument u (u^k = v^k + b^{k-1}; p = prox_{(t/lambda)H}(u) is d,
// b = u - p):
//
//  SPLIT (the paper's v-update with split operands, one phase per iteration).
//     v^{k+1} = M r^k,  r^k = y + lambda (2 p^k - u^k),  u^{k+1} = v^{k+1} + b^k
//  with M and r both two-term FP16 splits, M r ~ M_hi r_hi
//  + 2^-11 (M_hi r_lo' + M_lo' r_hi), the correction terms in a second TMEM
//  accumulator scaled exactly in the epilogue (~2^-22 per product).  For
//  H = l2 the prox is s u with a scale s known only once |u| is summed over
//  all row tiles, so the operand holds u itself and linearity gives
//  v^{k+1} = M y + lambda (2 s - 1) M u^k; the first iteration's product
//  (operand y) is M y, which then replaces y in the slot's y plane.
//
//  MIXED (defect correction).  With M = (A + lambda I)^{-1} and the identity
//  M (A + lambda I) = I, the v-update of eq. 3.4(a) becomes
//     u^{k+1} = u^k + M g^k,   g^k = y - A p^k - lambda (u^k - p^k),
//  so the fixed point is g = 0 whatever approximation of M the step uses:
//    phase A:  A p on the tensor cores as a two-term FP16 split,
//              A p ~ A_hi p_hi + 2^-11 (A_hi p_lo' + A_lo' p_hi)
//              (A_lo' = fp16((A - A_hi) 2^11), p_lo' likewise), the correction
//              terms in a second TMEM accumulator scaled exactly in the
//              epilogue; the epilogue forms g and stores it in BF16;
//    phase B:  M g with BF16 operands (K = 16 steps alternating between two
//              accumulators, so consecutive MMAs do not wait on one another),
//              the epilogue updates u, stores the FP16 split of the next p and
//              the residual partial sums.
//  BF16 (the paper's form, v = M r with r = y + lambda (2p - u) in BF16): one
//  phase per iteration.  Its fixed point carries the BF16 error of M r.
//
// The start v^0 = d^0 = y, b^0 = 0 (Section 3.1) is u^0 = p^0 = y.  After the
// last iteration a final pass computes A p for
// phi = <y,p> - 1/2 <p, A p> - c0 - t H(p) (FP64 partial sums) with a
// three-term FP16 split of both A and p (about 33 bits: the two-term split's
// 2^-22 would leave ~1e-6 in phi, where <y,p> and <p,Ap>/2 cancel):
//   A p ~ D1 + 2^-11 D2 + 2^-22 D3,  D1 = A1 p1,  D2 = A1 p2 + A2 p1,
//   D3 = A1 p3 + A2 p2 + A3 p1,
// two ring stages per k-block and both TMEM buffers per tile.
//
// One persistent cooperative launch, one CTA per SM, 64 + 32 EPI_WARPS threads
// (576 with the default 16 epilogue warps):
//   warp 0   TMA producer (one elected lane), 3-stage shared-memory ring
//   warp 1   TMEM owner and MMA issuer (one elected lane)
//   warps 2.. epilogue: TMEM -> registers -> elementwise update -> global;
//            EPI_WARPS / 4 warps per TMEM lane quadrant, each taking
//            128 / (EPI_WARPS / 4) of the tile's columns
// Work item = (128-row tile of n, 128-query column tile); items of a phase
// are dealt round-robin over CTAs; grid barriers separate the phases.  Every
// wait is bounded: on timeout the CTA records an error word, drains its own
// copies and MMAs, frees TMEM and leaves.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <new>

#include "common.cuh"
#include "diag_query.cuh"
#include "hopf_internal.h"
#include "tc_ptx.cuh"

namespace hopf {

hopf_status dense_init(hopf_handle h, DenseWs& w, const float* x, const float* t, cudaStream_t s);
hopf_status dense_init_warm(hopf_handle h, DenseWs& w, const float* x, const float* t, cudaStream_t s);
hopf_status dense_finalize(hopf_handle h, DenseWs& w, double* phi, float* dphidt, int32_t* iters, uint8_t* qstatus,
                           cudaStream_t s);

namespace tc {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int TILE_BYTES = BM * BK * 2;        // 16 KB: 128 rows x 128 bytes
// The ring by CG, the number of CTAs per MMA: CG = 1, one CTA per 128 x 128
// tile, three stages of 64 KB; CG = 2, an SM pair (a cluster of two CTAs) per
// 256 x 128 tile, each CTA holding its 128 rows of A and 64 of the 128 B rows,
// four stages of 48 KB.  A stage holds two A tiles and two B tiles.
template <int CG>
struct Ring {
  static constexpr int STAGES = CG == 1 ? 3 : 4;
  static constexpr int BH = BN / CG;                         // B rows held by one CTA
  static constexpr int B_BYTES = BH * BK * 2;                // one B tile
  static constexpr int STAGE_BYTES = 2 * TILE_BYTES + 2 * B_BYTES;
  static constexpr uint32_t A1 = TILE_BYTES >> 4;            // descriptor offsets within a stage
  static constexpr uint32_t B0 = (2 * TILE_BYTES) >> 4;
  static constexpr uint32_t B1 = (2 * TILE_BYTES + B_BYTES) >> 4;
};
constexpr int MAX_STAGES = 4;
constexpr int RING_BYTES = 3 * 4 * TILE_BYTES;
static_assert(Ring<1>::STAGES * Ring<1>::STAGE_BYTES == RING_BYTES, "ring size");
static_assert(Ring<2>::STAGES * Ring<2>::STAGE_BYTES == RING_BYTES, "ring size");
#ifndef HOPF_TC_EPI_WARPS
#define HOPF_TC_EPI_WARPS 16
#endif
constexpr int EPI_WARPS = HOPF_TC_EPI_WARPS;   // a multiple of 4: the same number per TMEM lane quadrant
constexpr int NEPI = EPI_WARPS * 32;           // epilogue threads
constexpr int NT = 64 + NEPI;                  // 2 role warps + the epilogue warps
constexpr int CPW = BN / (EPI_WARPS / 4);      // tile columns per epilogue warp
constexpr int TMEM_COLS = 512;                 // 2 buffers x 2 accumulators x 128 columns
constexpr int FORM_MIXED = 0, FORM_BF16 = 1, FORM_SPLIT = 2;
constexpr int PH_A = 0, PH_B = 1, PH_P = 2, PH_F = 3, PH_S = 4;
constexpr float kLoScale = 2048.f;             // 2^11: FP16 split scale
constexpr float kLo2Scale = 4194304.f;         // 2^22: third term of the split

// Slot-indexed state comes in two buffer sets ([0], [1]); compaction packs the
// active slots of one set into the other.  Query-indexed: tau, qiter, qdone,
// ufin, sfin, fpart, the final-pass operand planes.
struct TcArgs {
  CUtensorMap mAh, mAl, mAl2, mM, mP1, mP2, mP1b, mP2b, mG, mP3;  // mP3: the g plane read as the third split of p
  CUtensorMap mU[2];  // the FP32 u planes, for L2 prefetch of the epilogue's tiles
  CUtensorMap mMh, mMl;           // SPLIT: the two-term FP16 split of M
  CUtensorMap mQ1[2], mQ2[2];     // SPLIT: r^k of odd k, by buffer set (even k: mP1/mP2, mP1b/mP2b)
  float* y[2];
  float* u[2];
  uint16_t* p1[2];
  uint16_t* p2[2];
  uint16_t* q1[2];    // SPLIT: odd-parity operand planes by set
  uint16_t* q2[2];
  float* taus[2];     // t / lambda by slot
  int* qact[2][2];    // [set][parity of the decision]: 1 active, 2 retiring in this decision, 0 otherwise
  int* sq[2];         // slot -> query
  uint16_t* g;
  float* part[2];     // by set: [parity][2][rt][B_pad] partial sums of |du|^2, |u|^2
  double* fpart;
  float* tau;
  int* qiter;
  int* qdone;
  int* tile_k;        // per column tile: the last decision that found active slots in it
  int* tile_cnt;      // per column tile: the number it found
  float* ufin;
  float* sfin;
  const float* x;     // the caller's queries [B][n] (final pass: y = x - c)
  const float* cf;    // centre, padded
  unsigned* bar;
  int* err;
  const float* w;
  float* grad;
  float* beta;        // optional: control in dH(grad phi) [B][n]
  float* xfin;        // optional: terminal point x - t beta [B][n]
  int64_t B, B_pad;
  int n, np, rt, ct, h_kind, max_iter, form, compact;
  float lam, tol;
  long long wait_limit;  // clock cycles of every bounded wait
  // Two-stage solve (SPLIT iterations, then MIXED from where each query left
  // off): the first stage skips the final pass (no_final); the second starts
  // warm (u from that stage, no first-iteration rule, a stop allowed from the
  // first decision) and counts on from iter_base[q] iterations (also against
  // max_iter).  Both zero / null for a one-stage solve.
  int warm, no_final;
  int* iter_base;  // (the ragged kernel's in-kernel set-up of a second stage writes it)
};

// Per-CTA view of the slot layout; every CTA updates it identically.
struct Ctx {
  int cb;     // current buffer set
  int ct_on;  // column tiles in use (the active prefix)
  int fresh;  // compacted before this iteration: every tile below ct_on holds active slots
  int k;      // iteration
  int par;    // parity of this iteration's decision (k & 1)
  int gr, gs; // this CTA's rank in the group of CTAs solving the instance, and the group's size
};

// ---------------------------------------------------------------- PTX helpers
using namespace tcx;

// kind::f16 instruction descriptor: D F32, K-major A and B, M = 128, N = 128.
__host__ __device__ constexpr uint32_t idesc_f16(uint32_t ab_fmt /* 0 = F16, 1 = BF16 */) {
  return idesc_f16_mn(ab_fmt, BM, BN);
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(NEPI) : "memory"); }
// the first 128 epilogue threads only (one per slot of a tile)
__device__ __forceinline__ void epi_sync_half() { asm volatile("bar.sync 2, 128;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

__device__ __forceinline__ float prox1(float u, float w, float tau, float sc, int h_kind) {
  return h_kind == H_L2 ? sc * u : shrink1(u, tau * w);
}

// -------------------------------------------------------------- shared state
struct Smem {
  uint64_t full[MAX_STAGES], empty[MAX_STAGES], tfull[2], tempty[2], drain;
  uint64_t pfull[MAX_STAGES];  // SM pairs: the second CTA's stage is full (arrivals from the pair's CTA 1)
  uint64_t cfull[2], cempty[2];  // final pass: hand-off of the D1 chunks
  uint32_t tmem_base;
  int abort;
  // [2]: by item parity in the per-iteration epilogues (slot 0 in the final
  // pass and the compaction)
  int epi_abort[2];  // snapshot of abort read by all epilogue warps after a barrier
  int cnt[2][4];     // active slots per warp of the decision (row tile 0)
  alignas(16) float qtau[2][BN];
  alignas(16) float qscale[2][BN];
  int qact[2][BN];
  int qid[2][BN];
  int base[1024];  // compaction: first new slot of each column tile
  float red[2][4][BN][2];  // by item parity: an item's row sums are read after the next item's barrier
  double redd[4][BN][2];
};

struct PhaseCfg {
  int na, nb, nterm;
  int ta[3], tb[3], td[3];
  uint32_t idesc;
};

template <int CG>
__device__ __forceinline__ PhaseCfg phase_cfg(int ph) {
  PhaseCfg c{};
  if (ph == PH_A || ph == PH_F || ph == PH_S) {
    c.na = 2; c.nb = 2; c.nterm = 3;
    c.ta[0] = 0; c.tb[0] = 0; c.td[0] = 0;   // A_hi p_hi     -> D1
    c.ta[1] = 0; c.tb[1] = 1; c.td[1] = 1;   // A_hi p_lo'    -> D2
    c.ta[2] = 1; c.tb[2] = 0; c.td[2] = 1;   // A_lo' p_hi    -> D2
    c.idesc = idesc_f16_mn(0, BM * CG, BN);  // (PH_S: M_hi r_hi, M_hi r_lo', M_lo' r_hi)
  } else {
    c.na = 1; c.nb = 1; c.nterm = 1;
    c.ta[0] = 0; c.tb[0] = 0; c.td[0] = 0;   // M (g or r)    -> D1
    c.idesc = idesc_f16_mn(1, BM * CG, BN);
  }
  return c;
}

// Decision k is taken in the epilogue of phase A (or P) of iteration k, by
// every row tile of a column from the same partial sums; row tile 0 records
// it.  tile_k[c] only grows (row tile 0 sets it to k when decision k finds
// active slots in column c), so a column that has emptied stays out:
// phase A of iteration k runs the columns with tile_k >= k - 1 (all of them in
// the first iteration and right after a compaction), phase B those with
// tile_k == k.  Values left from before a compaction are older than the
// iteration, so they never count.
__device__ __forceinline__ int tile_count(const TcArgs& a, const Ctx& x, int c) {
  return a.tile_k[c] == x.k ? a.tile_cnt[c] : 0;
}
__device__ __forceinline__ bool tile_on(const TcArgs& a, const Ctx& x, int ph, int c) {
  if (ph == PH_F) return (int64_t)c * BN < a.B;
  if (c >= x.ct_on) return false;
  if (ph == PH_B) return a.tile_k[c] == x.k;
  return x.k == 1 || x.fresh || a.tile_k[c] >= x.k - 1;
}
// The items of a phase, dealt round-robin over the group's CTAs (CG = 1) or
// SM pairs (CG = 2): item it is column tile it / (rt / CG) and row tile
// CG (it % (rt / CG)) + (gr % CG), so the two CTAs of a pair take the two
// row tiles of one 256-row block of the same column tile.
template <int CG>
__device__ __forceinline__ int phase_items(const TcArgs& a, const Ctx& x, int ph) {
  return (a.rt / CG) * (ph == PH_F ? a.ct : x.ct_on);
}

// ------------------------------------------------------------ role: producer
struct ProdState {
  uint32_t kb = 0;                 // k-blocks issued so far (ring position)
  uint32_t last_par[MAX_STAGES];   // parity of the last load issued into each stage
  bool used[MAX_STAGES];
};

// BF16 form: r^{k-1} lives in buffer (k-1) & 1 (p1 = buffer 0, p2 = buffer 1)
// and the epilogue of iteration k writes r^k into the other one, so no CTA
// overwrites an operand another CTA may still be loading.
template <int CG>
__device__ void producer_phase(const TcArgs& a, Smem& S, uint8_t* stages, int ph, int k, const Ctx& x,
                               ProdState& st) {
  using R = Ring<CG>;
  const PhaseCfg cfg = phase_cfg<CG>(ph);
  const CUtensorMap* A0 = (ph == PH_A || ph == PH_F) ? &a.mAh : ph == PH_S ? &a.mMh : &a.mM;
  const CUtensorMap* A1 = ph == PH_S ? &a.mMl : &a.mAl;
  const CUtensorMap* B0 = ph == PH_A ? (x.cb ? &a.mP1b : &a.mP1)
                          : ph == PH_F ? &a.mP1
                          : ph == PH_B ? &a.mG
                                       : (((k - 1) & 1) ? &a.mP2 : &a.mP1);
  const CUtensorMap* B1 = (ph == PH_A && x.cb) ? &a.mP2b : &a.mP2;
  if (ph == PH_S) {
    // r^{k-1}: parity (k - 1) & 1 of the current buffer set
    const bool odd = ((k - 1) & 1) != 0;
    B0 = odd ? &a.mQ1[x.cb] : (x.cb ? &a.mP1b : &a.mP1);
    B1 = odd ? &a.mQ2[x.cb] : (x.cb ? &a.mP2b : &a.mP2);
  }
  // phases with one operand pair (B, P) fill a stage with two k-blocks
  const int kstep = cfg.na == 1 ? 2 : 1;
  const uint32_t bytes = R::STAGE_BYTES;
  const int nk = a.np / BK, items = phase_items<CG>(a, x, ph), rpc = a.rt / CG, rank = x.gr % CG;
  const int nsub = ph == PH_F ? 2 : 1;  // PH_F: {A1, A2 | p1, p2} then {A1, A3 | p3, p1}
  for (int it = x.gr / CG; it < items; it += x.gs / CG) {
    const int r = CG * (it % rpc) + rank, c = it / rpc;
    if (!tile_on(a, x, ph, c)) continue;
    const int cq = c * BN + rank * R::BH;  // the first B row (query) this CTA loads
    // the epilogue of this item reads u of its tile one to two items from
    // now: start the DRAM reads now (a prefetch of y as well measured slower)
    if (ph != PH_F) tma_prefetch_l2(&a.mU[x.cb], r * BM, c * BN);
    for (int kb = 0; kb < nk; kb += kstep) {
      for (int sub = 0; sub < nsub; ++sub, ++st.kb) {
        const uint32_t s = st.kb % R::STAGES, use = st.kb / R::STAGES;
        if (!mbar_wait_lim(sa(&S.empty[s]), (use & 1) ^ 1, a.err, &S.abort, a.wait_limit)) return;
        const uint32_t full = sa(&S.full[s]);
        mbar_expect_tx(full, bytes);
        uint8_t* base = stages + (size_t)s * R::STAGE_BYTES;
        uint8_t* bt0 = base + 2 * TILE_BYTES;
        uint8_t* bt1 = bt0 + R::B_BYTES;
        const int kx = kb * BK;
        if (kstep == 2) {
          // {M_kb, M_kb+1 | g_kb, g_kb+1}
          tma_load(sa(base), A0, full, kx, r * BM);
          tma_load(sa(base + TILE_BYTES), A0, full, kx + BK, r * BM);
          tma_load(sa(bt0), B0, full, kx, cq);
          tma_load(sa(bt1), B0, full, kx + BK, cq);
        } else {
          const CUtensorMap* a1 = sub ? &a.mAl2 : A1;
          const CUtensorMap* b0 = sub ? &a.mP3 : B0;
          const CUtensorMap* b1 = sub ? &a.mP1 : B1;
          tma_load(sa(base), A0, full, kx, r * BM);
          tma_load(sa(base + TILE_BYTES), a1, full, kx, r * BM);
          tma_load(sa(bt0), b0, full, kx, cq);
          tma_load(sa(bt1), b1, full, kx, cq);
        }
        st.last_par[s] = use & 1;
        st.used[s] = true;
      }
    }
  }
}

// ----------------------------------------------------------------- role: MMA
// TMEM: two buffers of 256 columns; each tile normally takes one buffer
// (alternating), the final pass takes both.  Per-buffer counts of empty waits
// and full commits give the mbarrier parities.
struct MmaState {
  uint32_t kb = 0;       // ring stages consumed
  uint32_t nb = 0;       // buffer of the next ordinary tile
  uint32_t ue[2] = {0, 0}, uf[2] = {0, 0};
  uint32_t ce[2] = {0, 0}, cf[2] = {0, 0};  // final-pass chunk slots
  bool issued = false;
  uint64_t sdesc[MAX_STAGES];  // shared-memory descriptor of each ring stage's first tile
};

// The ordinary phases with as few instructions per MMA as possible: one
// thread issues every MMA of the CTA, on a sub-partition it shares with
// epilogue warps, and each instruction it spends delays the tensor pipe.
// Descriptors are the stage's precomputed base plus constants (a tile is
// 16 KB = 1024 descriptor units, a K = 16 step 32 bytes = 2 units), the
// terms are fixed at compile time, and the next item's column check is
// loaded while this item's MMAs are issued.
//   THREE: phases A and S, one k-block per stage {A0, A1 | B0, B1}:
//          A0 B0 -> D1, A0 B1 + A1 B0 -> D2;
//   else:  phases B and P, two k-blocks per stage {M_kb, M_kb+1 | g_kb, g_kb+1},
//          K steps alternating between D1 and D2.
//   SM pairs: CTA 0 of the pair issues M = 256 MMAs over both CTAs' stages
//   once its own stage and the other CTA's are full (CTA 1's MMA thread
//   relays its full barriers to CTA 0's pfull); the commits arrive in both
//   CTAs, and both CTAs' epilogues release the accumulator to CTA 0.
template <int CG, bool THREE>
__device__ __forceinline__ void mma_items(const TcArgs& a, Smem& S, int ph, const Ctx& x, MmaState& st,
                                          uint32_t idesc) {
  using R = Ring<CG>;
  const int nst = THREE ? a.np / BK : a.np / (2 * BK);  // stages per item
  const int items = phase_items<CG>(a, x, ph), rpc = a.rt / CG, step = x.gs / CG;
  const bool lead = CG == 1 || x.gr % CG == 0;
  int it = x.gr / CG;
  while (it < items && !tile_on(a, x, ph, it / rpc)) it += step;
  uint32_t s = st.kb % R::STAGES, suse = st.kb / R::STAGES;
  while (it < items) {
    const int nx = it + step;
    const bool nx_on = nx < items && tile_on(a, x, ph, nx / rpc);  // used after this item
    if (!lead) {
      for (int j = 0; j < nst; ++j) {
        if (!mbar_wait_lim(sa(&S.full[s]), suse & 1, a.err, &S.abort, a.wait_limit)) return;
        mbar_arrive_rank(sa(&S.pfull[s]), 0);
        if (++s == R::STAGES) {
          s = 0;
          ++suse;
        }
      }
      st.kb += nst;
    } else {
      const uint32_t buf = st.nb;
      st.nb ^= 1;
      const uint32_t tpar = (st.ue[buf] & 1) ^ 1;
      if (!mbar_wait_lim(sa(&S.tempty[buf]), tpar, a.err, &S.abort, a.wait_limit)) return;
      ++st.ue[buf];
      tc_fence_after();
      const uint32_t d1 = S.tmem_base + buf * 256, d2 = d1 + BN;
      for (int j = 0; j < nst; ++j) {
        if (!mbar_wait_lim(sa(&S.full[s]), suse & 1, a.err, &S.abort, a.wait_limit)) return;
        if (CG == 2 && !mbar_wait_lim(sa(&S.pfull[s]), suse & 1, a.err, &S.abort, a.wait_limit)) return;
        tc_fence_after();
        const uint64_t b = st.sdesc[s];
        if constexpr (THREE) {
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            mma_f16_cg<CG>(d1, b + kk * 2, b + R::B0 + kk * 2, idesc, (j == 0 && kk == 0) ? 0u : 1u);
            mma_f16_cg<CG>(d2, b + kk * 2, b + R::B1 + kk * 2, idesc, (j == 0 && kk == 0) ? 0u : 1u);
            mma_f16_cg<CG>(d2, b + R::A1 + kk * 2, b + R::B0 + kk * 2, idesc, 1u);
          }
        } else {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              mma_f16_cg<CG>((kk & 1) ? d2 : d1, b + h * R::A1 + kk * 2, b + (h ? R::B1 : R::B0) + kk * 2, idesc,
                             (j == 0 && h == 0 && kk < 2) ? 0u : 1u);
        }
        st.issued = true;
        mma_commit_cg<CG>(sa(&S.empty[s]));  // frees the stage (in both CTAs) once these MMAs have read it
        if (++s == R::STAGES) {
          s = 0;
          ++suse;
        }
      }
      st.kb += nst;
      mma_commit_cg<CG>(sa(&S.tfull[buf]));  // accumulator ready for the epilogue(s)
      ++st.uf[buf];
    }
    it = nx;
    if (!nx_on)
      while (it < items && !tile_on(a, x, ph, it / rpc)) it += step;
  }
}

template <int CG>
__device__ void mma_phase(const TcArgs& a, Smem& S, uint8_t* stages, int ph, const Ctx& x, MmaState& st) {
  using R = Ring<CG>;
  const PhaseCfg cfg = phase_cfg<CG>(ph);
  if (ph == PH_A || ph == PH_S) return mma_items<CG, true>(a, S, ph, x, st, cfg.idesc);
  if (ph == PH_B || ph == PH_P) return mma_items<CG, false>(a, S, ph, x, st, cfg.idesc);
  // the final pass (PH_F): both TMEM buffers per item
  const int nk = a.np / BK, items = phase_items<CG>(a, x, PH_F), rpc = a.rt / CG;
  const bool lead = CG == 1 || x.gr % CG == 0;
  const uint32_t idesc = idesc_f16_mn(0, BM * CG, BN);
  for (int it = x.gr / CG; it < items; it += x.gs / CG) {
    const int c = it / rpc;
    if (!tile_on(a, x, PH_F, c)) continue;
    if (!lead) {
      for (int kb = 0; kb < nk; ++kb)
        for (int sub = 0; sub < 2; ++sub, ++st.kb) {
          const uint32_t s = st.kb % R::STAGES, suse = st.kb / R::STAGES;
          if (!mbar_wait_lim(sa(&S.full[s]), suse & 1, a.err, &S.abort, a.wait_limit)) return;
          mbar_arrive_rank(sa(&S.pfull[s]), 0);
        }
      continue;
    }
    for (uint32_t b = 0; b < 2; ++b) {
      const uint32_t tpar = (st.ue[b] & 1) ^ 1;
      if (!mbar_wait_lim(sa(&S.tempty[b]), tpar, a.err, &S.abort, a.wait_limit)) return;
      ++st.ue[b];
    }
    tc_fence_after();
    for (int kb = 0; kb < nk; ++kb) {
      // The main term D1 = A1 p1 goes into one of two 128-column slots per
      // 128-wide K chunk (two k-blocks); the epilogue adds the chunks up in
      // registers, so no TMEM accumulator sums more than 8 products of
      // K = 16.  D2 and D3 (scaled by 2^-11, 2^-22) accumulate over all of K
      // in the second buffer.  TMEM: D1 slots at 0 and 128, D2 at 256, D3 at 384.
      const uint32_t chunk = kb >> 1, slot = chunk & 1;
      if ((kb & 1) == 0) {
        const uint32_t cpar = (st.ce[slot] & 1) ^ 1;
        if (!mbar_wait_lim(sa(&S.cempty[slot]), cpar, a.err, &S.abort, a.wait_limit)) return;
        ++st.ce[slot];
        tc_fence_after();
      }
      const uint32_t d1 = S.tmem_base + slot * BN, d2 = S.tmem_base + 256, d3 = S.tmem_base + 384;
      // sub-stage X: {A1, A2 | p1, p2};  sub-stage Y: {A1, A3 | p3, p1}
      for (int sub = 0; sub < 2; ++sub, ++st.kb) {
        const uint32_t s = st.kb % R::STAGES, suse = st.kb / R::STAGES;
        if (!mbar_wait_lim(sa(&S.full[s]), suse & 1, a.err, &S.abort, a.wait_limit)) return;
        if (CG == 2 && !mbar_wait_lim(sa(&S.pfull[s]), suse & 1, a.err, &S.abort, a.wait_limit)) return;
        tc_fence_after();
        const uint64_t b = st.sdesc[s];
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t a0 = b + kk * 2, a1 = b + R::A1 + kk * 2;
          const uint64_t b0 = b + R::B0 + kk * 2, b1 = b + R::B1 + kk * 2;
          const uint32_t fc = ((kb & 1) == 0 && kk == 0) ? 0u : 1u;  // chunk start overwrites D1
          const uint32_t fi = (kb == 0 && kk == 0) ? 0u : 1u;        // item start overwrites D2, D3
          if (sub == 0) {
            mma_f16_cg<CG>(d1, a0, b0, idesc, fc);    // D1 += A1 p1
            mma_f16_cg<CG>(d2, a0, b1, idesc, fi);    // D2 += A1 p2
            mma_f16_cg<CG>(d2, a1, b0, idesc, 1u);    // D2 += A2 p1
            mma_f16_cg<CG>(d3, a1, b1, idesc, fi);    // D3 += A2 p2
          } else {
            mma_f16_cg<CG>(d3, a0, b0, idesc, 1u);    // D3 += A1 p3
            mma_f16_cg<CG>(d3, a1, b1, idesc, 1u);    // D3 += A3 p1
          }
        }
        st.issued = true;
        mma_commit_cg<CG>(sa(&S.empty[s]));
      }
      if (kb & 1) {
        mma_commit_cg<CG>(sa(&S.cfull[slot]));  // this chunk of D1 is ready
        ++st.cf[slot];
      }
    }
    mma_commit_cg<CG>(sa(&S.tfull[0]));  // D2, D3 ready for the epilogue(s)
    ++st.uf[0];
  }
}

// ------------------------------------------------------------ role: epilogue
struct EpiState {
  uint32_t nb = 0;  // buffer of the next ordinary tile
  uint32_t ue[2] = {0, 0}, uf[2] = {0, 0};
  uint32_t ce[2] = {0, 0}, cf[2] = {0, 0};  // final-pass chunk slots
};

// Load the per-query data of column tile c into shared memory.
// Final pass: the per-query data of column tile c (query-indexed).
__device__ void epi_stage_final(const TcArgs& a, Smem& S, int c, int et) {
  if (et >= BN) return;
  const int64_t q = (int64_t)c * BN + et;
  S.qtau[0][et] = a.tau[q];
  S.qscale[0][et] = a.sfin[q];
  S.qact[0][et] = q < a.B;
}

// Transpose-reduce over 16 columns: lane L holds v[0..15] (one value per
// column for its row).  Four halving steps (8 + 4 + 2 + 1 shuffles) leave lane
// L with column (L & 15) summed over the 16 lanes that share bit 4 of L; one
// more exchange across bit 4 completes the sum over all 32 rows.  On return
// v[0] of lanes L and L ^ 16 holds the total of column L & 15.
__device__ __forceinline__ void transpose_reduce16(float v[16], int lane) {
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = up ? v[i] : v[i + o];
      const float keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// The same for V doubles: lane l ends with the warp total of value l & (V - 1).
template <int V>
__device__ __forceinline__ void transpose_reduce_d(double v[V], int lane) {
#pragma unroll
  for (int o = V / 2; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const double send = up ? v[i] : v[i + o];
      const double keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int o = V; o < 32; o <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
}

// Per-slot data of an item's column: t / lambda, query, prox scale and state.
// Phases A and P take decision k here from the partial sums of iteration
// k - 1 (every row tile of the column alike):  0 inactive, 1 active,
// 2 stops converged, 3 stops at max_iter.  Phase B reads the recorded state.
__device__ __forceinline__ void slot_data(const TcArgs& a, const Ctx& x, int ph, int64_t sl, float& tau, float& sc,
                                          int& act, int& qid) {
  const int cb = x.cb;
  tau = a.taus[cb][sl];
  qid = a.sq[cb][sl];
  sc = 1.f;
  if (ph == PH_B) {
    act = a.qact[cb][x.par][sl];
    return;
  }
  if (x.k == 1) {
    // a warm start leaves out the queries the first stage stopped at max_iter
    act = qid < a.B && (!a.warm || a.qdone[qid] == 0) ? 1 : 0;
    return;
  }
  // every load issued before any is used (one memory latency)
  const int prev = a.qact[cb][x.par ^ 1][sl];
  const float* P = a.part[cb] + (int64_t)((x.par ^ 1) * 2) * a.rt * a.B_pad + sl;
  const int64_t rs = a.B_pad, ns = (int64_t)a.rt * a.B_pad;
  float dv[8], nv[8];
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    dv[rr] = rr < a.rt ? P[rr * rs] : 0.f;
    nv[rr] = rr < a.rt ? P[ns + rr * rs] : 0.f;
  }
  float du2 = 0.f, nu2 = 0.f;
#pragma unroll
  for (int rr = 0; rr < 8; ++rr) {
    du2 += dv[rr];
    nu2 += nv[rr];
  }
  for (int rr = 8; rr < a.rt; ++rr) {
    du2 += P[rr * rs];
    nu2 += P[ns + rr * rs];
  }
  act = 0;
  if (prev != 1) return;
  sc = shrink2_scale(sqrtf(nu2), tau);
  const int kprev = x.k - 1;
  const int done_before = a.iter_base ? a.iter_base[qid] : 0;
  if (kprev >= 2 - a.warm && du2 <= a.tol * fmaxf(1.f, nu2)) act = 2;
  else if (kprev + done_before >= a.max_iter) act = 3;
  else act = 1;
}

// Ask L1 for the slot data that slot_data() will read for slot sl.
__device__ __forceinline__ void slot_prefetch(const TcArgs& a, const Ctx& x, int ph, int64_t sl) {
  const int cb = x.cb;
  asm volatile("prefetch.global.L1 [%0];" ::"l"(a.taus[cb] + sl));
  asm volatile("prefetch.global.L1 [%0];" ::"l"(a.sq[cb] + sl));
  if (ph == PH_B) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a.qact[cb][x.par] + sl));
    return;
  }
  if (x.k == 1) return;
  asm volatile("prefetch.global.L1 [%0];" ::"l"(a.qact[cb][x.par ^ 1] + sl));
  const float* P = a.part[cb] + (int64_t)((x.par ^ 1) * 2) * a.rt * a.B_pad + sl;
  for (int rr = 0; rr < 2 * a.rt; ++rr) asm volatile("prefetch.global.L1 [%0];" ::"l"(P + (int64_t)rr * a.B_pad));
}

template <int CG, int ph>
__device__ void epilogue_phase(const TcArgs& a, Smem& S, int k, const Ctx& x, EpiState& st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int et = threadIdx.x - 64;      // 0..255
  const int qd = warp & 3;              // TMEM lane quadrant of this warp
  const int jbase = ((warp - 2) >> 2) * CPW;  // this warp's share of the columns
  const int rloc = qd * 32 + lane;      // row within the tile
  const int items = phase_items<CG>(a, x, ph), rpc = a.rt / CG, rank = x.gr % CG, step = x.gs / CG;
  const int np = a.np, hk = a.h_kind;
  const float lam = a.lam;
  const int cb = x.cb;
  // the slot data (and, in phases A and P, the decision) of the next item is
  // loaded into registers while the current item is processed
  int it = x.gr / CG;
  while (it < items && !tile_on(a, x, ph, it / rpc)) it += step;
  float pf_tau = 0.f, pf_sc = 1.f;
  int pf_act = 0, pf_qid = 0;
  if (it < items && et < BN) slot_data(a, x, ph, (int64_t)(it / rpc) * BN + et, pf_tau, pf_sc, pf_act, pf_qid);
  // One named barrier per item: the shared query data and row sums are
  // double-buffered by item parity ib.  A warp that writes item i + 1's has
  // passed item i's barrier, so every warp has finished reading item i - 1's.
  // Phases B and P: an item's row sums go to the partial-sum array after the
  // next item's barrier (or after the loop).
  int ib = 0, prev_par = 0, prev_r = 0, prev_c = -1;
  bool prev_on = false;
  auto flush_part = [&]() {
    if (prev_c >= 0 && prev_on) {
      const int64_t q = (int64_t)prev_c * BN + et;
      const float s0 = S.red[prev_par][0][et][0] + S.red[prev_par][1][et][0] + S.red[prev_par][2][et][0] +
                       S.red[prev_par][3][et][0];
      const float s1 = S.red[prev_par][0][et][1] + S.red[prev_par][1][et][1] + S.red[prev_par][2][et][1] +
                       S.red[prev_par][3][et][1];
      const int par = k & 1;
      a.part[cb][((int64_t)(par * 2 + 0) * a.rt + prev_r) * a.B_pad + q] = s0;
      a.part[cb][((int64_t)(par * 2 + 1) * a.rt + prev_r) * a.B_pad + q] = s1;
    }
  };
  while (it < items) {
    const int r = CG * (it % rpc) + rank, c = it / rpc;
    int it_next = it + step;
    while (it_next < items && !tile_on(a, x, ph, it_next / rpc)) it_next += step;
    const uint32_t buf = st.nb;
    st.nb ^= 1;
    const uint32_t use = st.uf[buf]++;
    const bool record = ph != PH_B && r == 0;  // row tile 0 records decision k
    if (et < BN) {
      S.qtau[ib][et] = pf_tau;
      S.qscale[ib][et] = pf_sc;
      S.qact[ib][et] = pf_act;
      S.qid[ib][et] = pf_qid;
      if (record) {
        const int64_t sl = (int64_t)c * BN + et;
        a.qact[cb][x.par][sl] = pf_act >= 2 ? 2 : pf_act;
        if (pf_act >= 2) {
          a.qdone[pf_qid] = pf_act == 2 ? 1 : 2;
          a.qiter[pf_qid] = pf_act == 2 ? k - 1 + (a.iter_base ? a.iter_base[pf_qid] : 0) : a.max_iter;
          a.sfin[pf_qid] = pf_sc;
        }
        const int cnt = __reduce_add_sync(0xffffffffu, pf_act == 1 ? 1 : 0);
        if ((et & 31) == 0) S.cnt[ib][et >> 5] = cnt;
      }
      // one lane in 32 asks for each 128-byte line of the next item's slot data
      if (it_next < items && (et & 31) == 0)
        slot_prefetch(a, x, ph, (int64_t)(it_next / rpc) * BN + et);
    }
    if (et == 0) S.epi_abort[ib] = S.abort;
    epi_sync();
    if (S.epi_abort[ib]) return;  // the same decision in all epilogue warps
    if constexpr (ph != PH_A) {
      if (et < BN) flush_part();
    }
    if (record && et == 0) {
      const int tot = S.cnt[ib][0] + S.cnt[ib][1] + S.cnt[ib][2] + S.cnt[ib][3];
      if (tot) {
        a.tile_cnt[c] = tot;
        a.tile_k[c] = k;
        atomicAdd(a.bar + 2 + (k % 3), (unsigned)tot);
      }
    }
    const int row = r * BM + rloc;
    const float wr = a.w[row];
    const uint32_t tbase = S.tmem_base + ((uint32_t)(qd * 32) << 16) + buf * 256;
    const bool first = k == 1 && !a.warm;
    // The state a chunk reads from global memory does not depend on this
    // item's products: the first chunk's loads go out before the wait for
    // the accumulator, each later chunk's when its predecessor is done.
    // am: active slots of the 16-column chunk, rm (phases A and P): slots
    // that stop in this decision (lanes 0-15 vote).
    float uu[16], yy[16];
    uint32_t am = 0, rm = 0;
    auto load = [&](int j0) {
      const int qa = lane < 16 ? S.qact[ib][j0 + (lane & 15)] : 0;
      am = __ballot_sync(0xffffffffu, qa == 1);
      rm = ph == PH_B ? 0u : __ballot_sync(0xffffffffu, qa >= 2);
      const int64_t col0 = ((int64_t)c * BN + j0) * np + row;
      const float* ucol = a.u[cb] + col0;
      const float* ycol = a.y[cb] + col0;
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        uu[jj] = ((am | rm) >> jj & 1u) ? ucol[(int64_t)jj * np] : 0.f;
        if constexpr (ph != PH_B) yy[jj] = (am >> jj & 1u) ? __ldg(ycol + (int64_t)jj * np) : 0.f;
      }
    };
    load(jbase);
    // a failed wait skips the work of this item but keeps the warp in step
    // with the others at the named barriers below
    const bool good = mbar_wait_lim(sa(&S.tfull[buf]), use & 1, a.err, &S.abort, a.wait_limit);
    if (good) tc_fence_after();
    for (int j0 = jbase; good && j0 < jbase + CPW; j0 += 16) {
      if (j0 != jbase) load(j0);
      float d1[16];
      {
        // A p (PH_A), M r (PH_S) = D1 + 2^-11 D2; M g (PH_B) and M r (PH_P)
        // = D1 + D2, the two accumulators of alternating K steps
        float d2[16];
        tmem_ld16(tbase + j0, d1);
        tmem_ld16(tbase + BN + j0, d2);
        const float s2 = (ph == PH_A || ph == PH_S) ? 1.f / kLoScale : 1.f;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) d1[jj] += d2[jj] * s2;
      }
      const int64_t col0 = ((int64_t)c * BN + j0) * np + row;
      if (rm) {
        // a stopping slot leaves its u^{k-1} row segment in the final array
#pragma unroll
        for (int jj = 0; jj < 16; ++jj)
          if (rm >> jj & 1u) a.ufin[(int64_t)S.qid[ib][j0 + jj] * np + row] = uu[jj];
      }
      if constexpr (ph == PH_A) {
        // b = u - prox(u) in place of u, column by column (the branches are
        // uniform): l1 and weighted l1 shrink by tau w, l2 scales u (and A u)
        // by the query's s; in the first iteration p = y
        if (first) {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) uu[jj] -= yy[jj];
        } else if (hk == H_L2) {
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const float4 s4 = *reinterpret_cast<const float4*>(&S.qscale[ib][j0 + 4 * q4]);
            const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              uu[4 * q4 + e] -= sv[e] * uu[4 * q4 + e];
              d1[4 * q4 + e] *= sv[e];  // the operand held u: A p = s A u
            }
          }
        } else {
#pragma unroll
          for (int q4 = 0; q4 < 4; ++q4) {
            const float4 t4 = *reinterpret_cast<const float4*>(&S.qtau[ib][j0 + 4 * q4]);
            const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) uu[4 * q4 + e] -= shrink1(uu[4 * q4 + e], tv[e] * wr);
          }
        }
        uint16_t* gcol = a.g + col0;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const float g = yy[jj] - d1[jj] - lam * uu[jj];
          if (am >> jj & 1u) gcol[(int64_t)jj * np] = __bfloat16_as_ushort(__float2bfloat16_rn(g));
        }
      } else if constexpr (ph == PH_B) {
        // d1 becomes |u^k - u^{k-1}|^2 and uu becomes |u^k|^2 in place
        float* U = a.u[cb] + col0;
        uint16_t* P1 = a.p1[cb] + col0;
        uint16_t* P2 = a.p2[cb] + col0;
        // the operand planes hold p (l1, weighted l1) or u itself (l2)
        const bool l2 = hk == H_L2;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float4 t4 = *reinterpret_cast<const float4*>(&S.qtau[ib][j0 + 4 * q4]);
          const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int jj = 4 * q4 + e;
            const bool on = am >> jj & 1u;
            const float du = on ? d1[jj] : 0.f;
            const float un = uu[jj] + du;
            if (on) {
              const float pn = l2 ? un : shrink1(un, tv[e] * wr);
              const __half hi = __float2half_rn(pn);
              P1[(int64_t)jj * np] = __half_as_ushort(hi);
              P2[(int64_t)jj * np] = __half_as_ushort(__float2half_rn((pn - __half2float(hi)) * kLoScale));
              U[(int64_t)jj * np] = un;
            }
            d1[jj] = du * du;
            uu[jj] = on ? un * un : 0.f;
          }
        }
        transpose_reduce16(d1, lane);
        transpose_reduce16(uu, lane);
        if (lane < 16) {
          S.red[ib][qd][j0 + lane][0] = d1[0];
          S.red[ib][qd][j0 + lane][1] = uu[0];
        }
      } else if constexpr (ph == PH_S) {
        // d1 holds v^k = M r^{k-1} (l2: M u^{k-1}, or M y when k = 1);
        // u^k = v^k + b^{k-1}, then the split of r^k (l2: of u^k) goes to the
        // planes of parity k & 1; d1 and uu become |u^k - u^{k-1}|^2, |u^k|^2
        float* U = a.u[cb] + col0;
        const bool odd = (k & 1) != 0;
        uint16_t* R1 = (odd ? a.q1[cb] : a.p1[cb]) + col0;
        uint16_t* R2 = (odd ? a.q2[cb] : a.p2[cb]) + col0;
        float* Y = a.y[cb] + col0;
        const bool l2 = hk == H_L2;
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
          const float4 t4 = *reinterpret_cast<const float4*>(&S.qtau[ib][j0 + 4 * q4]);
          const float4 s4 = *reinterpret_cast<const float4*>(&S.qscale[ib][j0 + 4 * q4]);
          const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
          const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int jj = 4 * q4 + e;
            const bool on = am >> jj & 1u;
            float du = 0.f, un = 0.f;
            if (on) {
              const float th = tv[e] * wr;
              float v, b;
              if (l2) {
                if (first) {
                  v = (1.f + lam) * d1[jj];  // r^0 = (1 + lambda) y
                  b = 0.f;
                  Y[(int64_t)jj * np] = d1[jj];  // M y, for every later iteration
                } else {
                  v = yy[jj] + lam * (2.f * sv[e] - 1.f) * d1[jj];
                  b = (1.f - sv[e]) * uu[jj];
                }
              } else {
                v = d1[jj];
                b = first ? 0.f : uu[jj] - shrink1(uu[jj], th);  // b^0 = 0
              }
              un = v + b;
              du = un - uu[jj];
              const float rn = l2 ? un : yy[jj] + lam * (2.f * shrink1(un, th) - un);
              const __half hi = __float2half_rn(rn);
              R1[(int64_t)jj * np] = __half_as_ushort(hi);
              R2[(int64_t)jj * np] = __half_as_ushort(__float2half_rn((rn - __half2float(hi)) * kLoScale));
              U[(int64_t)jj * np] = un;
            }
            d1[jj] = du * du;
            uu[jj] = un * un;
          }
        }
        transpose_reduce16(d1, lane);
        transpose_reduce16(uu, lane);
        if (lane < 16) {
          S.red[ib][qd][j0 + lane][0] = d1[0];
          S.red[ib][qd][j0 + lane][1] = uu[0];
        }
      } else if constexpr (ph == PH_P) {
        float* U = a.u[cb] + col0;
        uint16_t* rbuf = ((k & 1) ? a.p2[cb] : a.p1[cb]) + col0;  // BF16 form: no compaction, set 0
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          float du = 0.f, un = 0.f;
          if (am >> jj & 1u) {
            const int j = j0 + jj;
            const float tau = S.qtau[ib][j];
            const float p = first ? yy[jj] : prox1(uu[jj], wr, tau, S.qscale[ib][j], hk);
            un = d1[jj] + uu[jj] - p;
            du = un - uu[jj];
            const float pn = prox1(un, wr, tau, 1.f, hk);
            rbuf[(int64_t)jj * np] = __bfloat16_as_ushort(__float2bfloat16_rn(yy[jj] + lam * (2.f * pn - un)));
            U[(int64_t)jj * np] = un;
          }
          d1[jj] = du * du;
          uu[jj] = un * un;
        }
        transpose_reduce16(d1, lane);
        transpose_reduce16(uu, lane);
        if (lane < 16) {
          S.red[ib][qd][j0 + lane][0] = d1[0];
          S.red[ib][qd][j0 + lane][1] = uu[0];
        }
      }
    }
    // release the accumulator buffer to the MMA warp (of the pair's CTA 0)
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      if (CG == 1) mbar_arrive(sa(&S.tempty[buf]));
      else mbar_arrive_rank(sa(&S.tempty[buf]), 0);
    }
    ++st.ue[buf];
    if constexpr (ph != PH_A) {
      prev_on = et < BN && S.qact[ib][et] == 1;
      prev_c = c;
      prev_r = r;
      prev_par = ib;
    }
    // the next item's slot data (and decision), from lines asked for above
    if (et < BN && it_next < items) slot_data(a, x, ph, (int64_t)(it_next / rpc) * BN + et, pf_tau, pf_sc, pf_act, pf_qid);
    it = it_next;
    ib ^= 1;
  }
  if constexpr (ph != PH_A) {
    epi_sync();
    if (et < BN) flush_part();
  }
}

// The final pass runs once per call: kept out of line so its FP64 registers do
// not weigh on the per-iteration epilogues.
template <int CG>
__device__ __noinline__ void epilogue_final(const TcArgs& a, Smem& S, const Ctx& x, EpiState& st) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int et = threadIdx.x - 64;
  const int qd = warp & 3;
  const int jbase = ((warp - 2) >> 2) * CPW;
  const int rloc = qd * 32 + lane;
  const int items = phase_items<CG>(a, x, PH_F), nk = a.np / BK, rpc = a.rt / CG;
  const int np = a.np, hk = a.h_kind;
  for (int it = x.gr / CG; it < items; it += x.gs / CG) {
    const int r = CG * (it % rpc) + x.gr % CG, c = it / rpc;
    if (!tile_on(a, x, PH_F, c)) continue;
    epi_sync();
    epi_stage_final(a, S, c, et);
    if (et == 0) S.epi_abort[0] = S.abort;
    epi_sync();
    if (S.epi_abort[0]) return;
    const uint32_t lanebase = S.tmem_base + ((uint32_t)(qd * 32) << 16);
    // promote each 128-wide K chunk of D1 into FP32 registers (round to nearest)
    float acc[CPW];
#pragma unroll
    for (int j = 0; j < CPW; ++j) acc[j] = 0.f;
    bool good = true;
    for (int chunk = 0; chunk < nk / 2; ++chunk) {
      const uint32_t slot = chunk & 1;
      good = good && mbar_wait_lim(sa(&S.cfull[slot]), st.cf[slot] & 1, a.err, &S.abort, a.wait_limit);
      ++st.cf[slot];
      if (good) {
        tc_fence_after();
#pragma unroll
        for (int j0 = 0; j0 < CPW; j0 += 16) {
          float v[16];
          tmem_ld16(lanebase + slot * BN + jbase + j0, v);
#pragma unroll
          for (int j = 0; j < 16; ++j) acc[j0 + j] += v[j];
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (CG == 1) mbar_arrive(sa(&S.cempty[slot]));
        else mbar_arrive_rank(sa(&S.cempty[slot]), 0);
      }
      ++st.ce[slot];
    }
    const uint32_t use = st.uf[0]++;
    good = good && mbar_wait_lim(sa(&S.tfull[0]), use & 1, a.err, &S.abort, a.wait_limit);
    if (good) tc_fence_after();
    const int row = r * BM + rloc;
    const float wr = a.w[row];
#pragma unroll
    for (int g = 0; g < CPW / 16; ++g) {
      if (!good) break;
      const int j0 = jbase + 16 * g;
      float d2[16], d3[16];
      tmem_ld16(lanebase + 256 + j0, d2);
      tmem_ld16(lanebase + 384 + j0, d3);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
      // the FP64 objective terms of 8 columns, summed over the warp's 32 rows
      // by one transpose-reduction (9 FP64 adds per lane for 8 columns)
      double f0v[8], f1v[8];
#pragma unroll
      for (int jh = 0; jh < 8; ++jh) {
        const int jj = 8 * h + jh;
        const int j = j0 + jj;
        // A p = D1 + 2^-11 D2 + 2^-22 D3
        const float ap = acc[16 * g + jj] + (d2[jj] + d3[jj] * (1.f / kLoScale)) * (1.f / kLoScale);
        double f0 = 0.0, f1 = 0.0;
        if (S.qact[0][j]) {
          const int64_t q = (int64_t)c * BN + j;
          const int64_t off = q * np + row;
          const float uu = a.ufin[off];
          const float yy = row < a.n ? a.x[q * a.n + row] - a.cf[row] : 0.f;  // y = x - c, as at the start
          const float p = prox1(uu, wr, S.qtau[0][j], S.qscale[0][j], hk);
          const double pd = p;
          f0 = (double)yy * pd - 0.5 * pd * (double)ap;
          f1 = hk == H_L2 ? pd * pd : (double)wr * fabs(pd);
          if (row < a.n) {
            a.grad[q * a.n + row] = p;
            if (a.beta) {
              // control (y - A p) / t = (u - p) / tau at the fixed point, an
              // element of dH(p) by the prox (u - prox(u) in tau dH)
              const float tau = S.qtau[0][j];
              const float bt = tau > 0.f ? (uu - p) / tau : 0.f;
              a.beta[q * a.n + row] = bt;
              if (a.xfin) a.xfin[q * a.n + row] = a.x[q * a.n + row] - tau * a.lam * bt;
            }
          }
        }
        f0v[jh] = f0;
        f1v[jh] = f1;
      }
      transpose_reduce_d<8>(f0v, lane);
      transpose_reduce_d<8>(f1v, lane);
      if (lane < 8) {
        S.redd[qd][j0 + 8 * h + lane][0] = f0v[0];
        S.redd[qd][j0 + 8 * h + lane][1] = f1v[0];
      }
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) {
      if (CG == 1) {
        mbar_arrive(sa(&S.tempty[0]));
        mbar_arrive(sa(&S.tempty[1]));
      } else {
        mbar_arrive_rank(sa(&S.tempty[0]), 0);
        mbar_arrive_rank(sa(&S.tempty[1]), 0);
      }
    }
    ++st.ue[0];
    ++st.ue[1];
    epi_sync();
    if (et < BN) {
      const int64_t q = (int64_t)c * BN + et;
      const double s0 = S.redd[0][et][0] + S.redd[1][et][0] + S.redd[2][et][0] + S.redd[3][et][0];
      const double s1 = S.redd[0][et][1] + S.redd[1][et][1] + S.redd[2][et][1] + S.redd[3][et][1];
      a.fpart[(int64_t)r * a.B_pad + q] = s0;
      a.fpart[(int64_t)(a.rt + r) * a.B_pad + q] = s1;
    }
  }
}

// Compaction after phase B of iteration k: the slots active after decision k
// move, in order, to the front of the other buffer set: y, u and the FP16
// split of p by rows, with the slot's query, t / lambda, state and the partial
// sums of iteration k (decision k + 1 reads them).  Every CTA scans the
// per-tile active counts itself; tile c's active slots start at base[c].
// Slots past the active count in the last new tile are marked inactive.
__device__ __noinline__ void compact(const TcArgs& a, Smem& S, const Ctx& x, int n_active) {
  const int et = threadIdx.x - 64;
  const int cb = x.cb, nb = cb ^ 1, par = x.par;
  if (et == 0) {
    int acc = 0;
    for (int c = 0; c < x.ct_on; ++c) {
      S.base[c] = acc;
      acc += tile_count(a, x, c);
    }
  }
  epi_sync();
  const int np = a.np, rt = a.rt;
  const int64_t pstride = (int64_t)rt * a.B_pad;
  // operand planes to carry: MIXED the split of p (one pair per set), SPLIT
  // r^k in the pair of parity k & 1
  const bool odd = a.form == FORM_SPLIT && (x.k & 1);
  const uint16_t* o1 = odd ? a.q1[cb] : a.p1[cb];
  const uint16_t* o2 = odd ? a.q2[cb] : a.p2[cb];
  uint16_t* d1p = odd ? a.q1[nb] : a.p1[nb];
  uint16_t* d2p = odd ? a.q2[nb] : a.p2[nb];
  for (int c = x.gr; c < x.ct_on; c += x.gs) {
    if (tile_count(a, x, c) == 0) continue;  // the same for every thread
    if (et < BN) {
      const int64_t sl = (int64_t)c * BN + et;
      const bool act = a.qact[cb][par][sl] == 1;
      const unsigned m = __ballot_sync(0xffffffffu, act);
      if ((et & 31) == 0) S.red[0][et >> 5][1][0] = __int_as_float(__popc(m));
      epi_sync_half();
      int rank = __popc(m & ((1u << (et & 31)) - 1u));
      for (int wv = 0; wv < (et >> 5); ++wv) rank += __float_as_int(S.red[0][wv][1][0]);
      S.qact[0][et] = act ? S.base[c] + rank : -1;  // destination slot
      if (act) {
        const int d = S.base[c] + rank;
        a.sq[nb][d] = a.sq[cb][sl];
        a.taus[nb][d] = a.taus[cb][sl];
        a.qact[nb][par][d] = 1;
        const float* P0 = a.part[cb] + (int64_t)(par * 2) * pstride;
        float* P1 = a.part[nb] + (int64_t)(par * 2) * pstride;
        for (int rr = 0; rr < 2 * rt; ++rr) P1[rr * a.B_pad + d] = P0[rr * a.B_pad + sl];
      }
    }
    epi_sync();
    // all active rows of the tile at once: the epilogue threads stream (slot, 4-element)
    // pieces, so many loads are in flight
    const int per_row = np / 4, total = BN * per_row;
    for (int e0 = et; e0 < total; e0 += 4 * NEPI) {
      float4 yv[4], uv[4];
      uint2 p1v[4], p2v[4];
      int64_t dst[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) {  // loads of four pieces first
        const int e = e0 + b * NEPI;
        dst[b] = -1;
        if (e >= total) continue;
        const int j = e / per_row, i = (e - j * per_row) * 4;
        const int d = S.qact[0][j];
        if (d < 0) continue;
        const int64_t so = ((int64_t)c * BN + j) * np + i;
        dst[b] = (int64_t)d * np + i;
        yv[b] = *reinterpret_cast<const float4*>(a.y[cb] + so);
        uv[b] = *reinterpret_cast<const float4*>(a.u[cb] + so);
        p1v[b] = *reinterpret_cast<const uint2*>(o1 + so);
        p2v[b] = *reinterpret_cast<const uint2*>(o2 + so);
      }
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        if (dst[b] < 0) continue;
        *reinterpret_cast<float4*>(a.y[nb] + dst[b]) = yv[b];
        *reinterpret_cast<float4*>(a.u[nb] + dst[b]) = uv[b];
        *reinterpret_cast<uint2*>(d1p + dst[b]) = p1v[b];
        *reinterpret_cast<uint2*>(d2p + dst[b]) = p2v[b];
      }
    }
    epi_sync();
  }
  // the tail of the last new tile
  const int need = (n_active + BN - 1) / BN;
  for (int64_t sl = (int64_t)n_active + x.gr * NEPI + et; sl < (int64_t)need * BN; sl += (int64_t)x.gs * NEPI) {
    a.qact[nb][par][sl] = 0;
    a.sq[nb][sl] = 0;
    a.taus[nb][sl] = 0.f;
  }
}

// Before the final pass: the three-term FP16 split of p = prox(u) for every
// query (query-indexed p1 and p2 planes of buffer set 0, the third term in the
// g plane), from the retired u.
__device__ __noinline__ void prep_final_operand(const TcArgs& a, const Ctx& x) {
  // four consecutive rows of one query per piece (np is a multiple of 128),
  // two pieces per thread in flight
  const int per_q = a.np / 4;
  const int64_t total = a.B_pad * per_q;
  const int64_t stride = (int64_t)x.gs * NEPI;
  for (int64_t i0 = (int64_t)x.gr * NEPI + (threadIdx.x - 64); i0 < total; i0 += 2 * stride) {
    float4 uv[2];
    int64_t q[2];
    int row[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int64_t i4 = i0 + b * stride;
      q[b] = i4 / per_q;
      row[b] = (int)(i4 - q[b] * per_q) * 4;
      uv[b] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i4 < total && q[b] < a.B) uv[b] = *reinterpret_cast<const float4*>(a.ufin + i4 * 4);
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int64_t i4 = i0 + b * stride;
      if (i4 >= total) break;
      const bool live = q[b] < a.B;
      const float tq = live ? (a.h_kind == H_L2 ? a.sfin[q[b]] : a.tau[q[b]]) : 0.f;
      const float4 w4 = *reinterpret_cast<const float4*>(a.w + row[b]);
      const float u4[4] = {uv[b].x, uv[b].y, uv[b].z, uv[b].w};
      const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
      unsigned short h1[4], h2[4], h3[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float pn = 0.f;
        if (live) pn = a.h_kind == H_L2 ? tq * u4[e] : shrink1(u4[e], tq * wv[e]);
        const __half x1 = __float2half_rn(pn);
        const float r1 = pn - __half2float(x1);  // exact
        const __half x2 = __float2half_rn(r1 * kLoScale);
        const float r2 = r1 - __half2float(x2) * (1.f / kLoScale);  // exact
        h1[e] = __half_as_ushort(x1);
        h2[e] = __half_as_ushort(x2);
        h3[e] = __half_as_ushort(__float2half_rn(r2 * kLo2Scale));
      }
      const uint2 o1 = make_uint2(h1[0] | ((unsigned)h1[1] << 16), h1[2] | ((unsigned)h1[3] << 16));
      const uint2 o2 = make_uint2(h2[0] | ((unsigned)h2[1] << 16), h2[2] | ((unsigned)h2[3] << 16));
      const uint2 o3 = make_uint2(h3[0] | ((unsigned)h3[1] << 16), h3[2] | ((unsigned)h3[3] << 16));
      *reinterpret_cast<uint2*>(a.p1[0] + i4 * 4) = o1;
      *reinterpret_cast<uint2*>(a.p2[0] + i4 * 4) = o2;
      *reinterpret_cast<uint2*>(a.g + i4 * 4) = o3;
    }
  }
}

// One instance solved by a group of gs CTAs (this one has rank gr) that share
// the instance's barrier words: the whole grid for hopf_eval, a lane of the
// grid in a ragged batch.  The ring, the TMEM and the role states carry over
// from one instance to the next.  Returns false when a wait gave up.
template <int CG>
__device__ bool solve_instance(const TcArgs& a, Smem& S, uint8_t* stages, ProdState& ps, MmaState& ms, EpiState& es,
                               int gr, int gs) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0 && lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&a.mAh)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&a.mM)) : "memory");
  }
  Ctx cx;
  cx.cb = 0;
  cx.ct_on = a.ct;
  cx.fresh = 0;
  cx.k = 0;
  cx.par = 0;
  cx.gr = gr;
  cx.gs = gs;
  auto run = [&](int ph, int k) {
    if (warp == 0) {
      if (lane == 0) {
        proxy_fence_global();  // generic-proxy writes of the last phase, then TMA reads
        producer_phase<CG>(a, S, stages, ph, k, cx, ps);
      }
    } else if (warp == 1) {
      if (lane == 0) mma_phase<CG>(a, S, stages, ph, cx, ms);
    } else {
      if (ph == PH_A) epilogue_phase<CG, PH_A>(a, S, k, cx, es);
      else if (ph == PH_S) epilogue_phase<CG, PH_S>(a, S, k, cx, es);
      else if (ph == PH_B) epilogue_phase<CG, PH_B>(a, S, k, cx, es);
      else if (ph == PH_P) epilogue_phase<CG, PH_P>(a, S, k, cx, es);
      else epilogue_final<CG>(a, S, cx, es);
      proxy_fence_global();
    }
  };

  // Iteration k: phase A (decision k in its epilogue, then g), barrier,
  // phase B (u, p and the partial sums), barrier, and a compaction when it
  // frees a quarter of the column tiles in use.  The SPLIT form has the
  // single phase S (decision k, u^k, r^k and the partial sums) before the
  // same compaction; the BF16 form the single phase P, without compaction.
  bool ok = true;
  for (int k = 1; ok; ++k) {
    cx.k = k;
    cx.par = k & 1;
    // the count slot that decision k + 1 fills (last read at iteration
    // k - 2, which every CTA has left)
    if (gr == 0 && threadIdx.x == 0) atomicExch(a.bar + 2 + ((k + 1) % 3), 0u);
    run(a.form == FORM_MIXED ? PH_A : a.form == FORM_SPLIT ? PH_S : PH_P, k);
    if (!(ok = grid_barrier(a.bar, gs, a.err, a.wait_limit))) break;
    const int n_active = (int)ld_acquire_u32(a.bar + 2 + (k % 3));
    if (n_active == 0) break;
    if (a.form == FORM_BF16) continue;
    if (a.form == FORM_MIXED) {
      run(PH_B, k);
      if (!(ok = grid_barrier(a.bar, gs, a.err, a.wait_limit))) break;
    }
    // every CTA takes the same decision from the same count: compact when it
    // frees a quarter of the column tiles in use and shortens each phase by
    // at least one round of items over the group (a sixteenth, an eighth, a
    // third and a half were each measured slower)
    const int need = (n_active + BN - 1) / BN;
    const bool fewer_rounds = (need * a.rt + gs - 1) / gs < (cx.ct_on * a.rt + gs - 1) / gs;
    // (the packing offsets of the column tiles live in shared memory)
    if (a.compact && cx.ct_on <= (int)(sizeof(S.base) / sizeof(S.base[0])) &&
        need + (cx.ct_on + 3) / 4 <= cx.ct_on && fewer_rounds) {
      if (warp >= 2) compact(a, S, cx, n_active);
      proxy_fence_global();
      if (!(ok = grid_barrier(a.bar, gs, a.err, a.wait_limit))) break;
      cx.cb ^= 1;
      cx.ct_on = need;
      cx.fresh = 1;
    } else {
      cx.fresh = 0;
    }
  }
  if (ok && !a.no_final) {
    if (warp >= 2) prep_final_operand(a, cx);
    proxy_fence_global();
    ok = grid_barrier(a.bar, gs, a.err, a.wait_limit);
    if (ok) run(PH_F, 0);
  }
  return ok;
}

// Shared memory, mbarriers and TMEM of a solver CTA (set up once per launch).
// SM pairs: the accumulator-empty barriers of CTA 0 count both CTAs'
// epilogue warps; the TMEM is allocated by one warp of each CTA together, and
// neither CTA goes on before the other's barriers exist.
template <int CG>
__device__ __forceinline__ Smem& tc_setup(uint8_t*& stages) {
  extern __shared__ uint8_t smem_raw[];
  stages = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Smem& S = *reinterpret_cast<Smem*>(stages + RING_BYTES);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    for (int s = 0; s < MAX_STAGES; ++s) {
      mbar_init(sa(&S.full[s]), 1);
      mbar_init(sa(&S.empty[s]), 1);
      mbar_init(sa(&S.pfull[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(sa(&S.tfull[b]), 1);
      mbar_init(sa(&S.tempty[b]), EPI_WARPS * CG);
    }
    mbar_init(sa(&S.drain), 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(sa(&S.cfull[b]), 1);
      mbar_init(sa(&S.cempty[b]), EPI_WARPS * CG);
    }
    S.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    if constexpr (CG == 1) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&S.tmem_base)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&S.tmem_base)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
  }
  __syncthreads();
  if constexpr (CG == 2) cluster_sync_all();
  tc_fence_after();
  return S;
}

// Drain (no copy or MMA of this CTA may be in flight when TMEM is freed) and
// free the TMEM.  SM pairs: CTA 0 commits the drain in both CTAs (its MMAs
// read CTA 1's shared memory and write its TMEM), and both CTAs pass a
// cluster barrier before either frees its TMEM or leaves.
template <int CG>
__device__ __forceinline__ void tc_teardown(Smem& S, const ProdState& ps, const MmaState& ms, bool lead = true) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < MAX_STAGES; ++s)
      if (ps.used[s]) {
        const long long t0 = clock64();
        while (!mbar_test(sa(&S.full[s]), ps.last_par[s]) && clock64() - t0 < (1ll << 31)) {
        }
      }
  }
  if (warp == 1 && lane == 0 && (CG == 2 || ms.issued)) {
    if (lead) mma_commit_cg<CG>(sa(&S.drain));
    const long long t0 = clock64();
    while (!mbar_test(sa(&S.drain), 0) && clock64() - t0 < (1ll << 31)) {
    }
  }
  tc_fence_before();
  __syncthreads();
  if constexpr (CG == 2) cluster_sync_all();
  tc_fence_after();
  if (warp == 1) {
    if constexpr (CG == 1)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(TMEM_COLS)
                   : "memory");
  }
}

// Registers: each of the 4 sub-partitions holds 16,384, shared by the warps
// placed on it (warp w on sub-partition w % 4): 18 warps put 5 on two of them,
// hence at most 96 per thread; 10 warps allow 168.
// CG = 2 runs in clusters of two CTAs (consecutive blocks: rank = block & 1).
template <int CG>
__global__ void __launch_bounds__(NT, 1) k_dense_tc(const __grid_constant__ TcArgs a) {
  uint8_t* stages;
  Smem& S = tc_setup<CG>(stages);
  ProdState ps;
  for (int s = 0; s < MAX_STAGES; ++s) ps.used[s] = false;
  MmaState ms;
  for (int s = 0; s < Ring<CG>::STAGES; ++s) ms.sdesc[s] = smem_desc(sa(stages + (size_t)s * Ring<CG>::STAGE_BYTES));
  EpiState es;
  solve_instance<CG>(a, S, stages, ps, ms, es, blockIdx.x, gridDim.x);
  tc_teardown<CG>(S, ps, ms, blockIdx.x % CG == 0);
}

// ------------------------------------------------------------------- host side
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
  }
  return fn;
}

// 2-D tensor [rows][np] of 16-bit elements, box 128 rows x 64 elements.
static bool encode(CUtensorMap* m, const void* ptr, int64_t rows, int np, bool bf16, int box_rows = 128) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)np * 2};
  cuuint32_t box[2] = {BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                  const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 2-D tensor [rows][np] of FP32, box 128 rows x 128 elements, no swizzle
// (used for L2 prefetch only).
static bool encode_f32(CUtensorMap* m, const void* ptr, int64_t rows, int np) {
  EncodeTiled fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)np, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)np * 4};
  cuuint32_t box[2] = {128, 128};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// FP16 split of y (MIXED: p^0 = y; SPLIT with H = l2: the operand u^0 = y),
// of r^0 = y + lambda y (SPLIT, l1 and weighted l1), or BF16 r^0 (BF16 form).
__global__ void k_tc_init_operand(const float* __restrict__ y, uint16_t* __restrict__ p1, uint16_t* __restrict__ p2,
                                  int64_t total, int form, float lam, int h_kind) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    float v = y[i];
    if (form == FORM_SPLIT && h_kind != H_L2) v = v + lam * v;
    if (form != FORM_BF16) {
      const __half hi = __float2half_rn(v);
      p1[i] = __half_as_ushort(hi);
      p2[i] = __half_as_ushort(__float2half_rn((v - __half2float(hi)) * kLoScale));
    } else {
      p1[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v + lam * v));
    }
  }
}


// ------------------------------------------------------------ ragged batches
// One persistent cooperative launch runs a whole ragged batch (hopf_batch_*):
// the dense instances by a schedule of CTA groups, then the diagonal
// instances from a shared work list.
//
// Dense.  Every CTA walks its own list of (instance, rank, group size)
// entries.  A group is the whole grid for a wide instance (at least one tile
// per SM) and a lane of the grid for the others; all CTAs of a group hold the
// same instances in the same order, so each instance's barrier words are used
// by exactly its group.  Per instance the group initialises the state (what
// k_dense_init and k_tc_init_operand do for hopf_eval), solves it with
// solve_instance, and writes phi, d phi / dt, the iteration count and the
// status (what k_dense_finalize does): the arithmetic of every query is that
// of hopf_eval, so the results are the same bit for bit.  A CTA whose wait
// gave up (its ring and TMEM state are then unusable) marks every later
// instance of its list aborted, and their groups report HOPF_Q_ABORTED.
//
// Diagonal.  When its list is done, each CTA's first 256 threads take work
// items (instance, first query, query count, group shape) from an atomic
// counter: 256 queries of a thread-per-query instance, 8 of a warp-per-query
// one, or one query of a 256-thread one; the group shape is the one hopf_eval
// picks for the instance's n, so again the results are the same.
struct alignas(128) RagDense {
  TcArgs a;
  TcArgs a2;          // staged MIXED (staged != 0): the defect-correction stage after a's SPLIT one
  int staged;
  const float* t;     // the caller's t for the instance
  float* tq;          // [B_pad] t by query
  double* phi;
  float* dphidt;
  int32_t* iters;
  uint8_t* qstatus;
  double c0;
};

struct RagDiag {
  DiagEvalArgs<float> e;
};

struct RaggedArgs {
  const RagDense* dense;
  const int4* sched;      // per CTA entries (instance, rank, size, -)
  const int* sched_off;   // [grid + 1]
  const RagDiag* diag;
  const int4* dinfo;      // per diagonal instance (queries, queries per item, shape class, first item)
  int n_diag, n_items;
  unsigned* ctr;          // work-list counter (zero before the launch)
};

__device__ void rag_init(const RagDense& d, int gr, int gs) {
  const TcArgs& a = d.a;
  const int64_t nthr = (int64_t)gs * NT, tid = (int64_t)gr * NT + threadIdx.x;
  const int np = a.np;
  const float lam = a.lam;
  // a warp per row, 8 independent loads in flight per lane: with one CTA per
  // SM there are too few threads to hide the load latency one element at a time
  constexpr int U = 8;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = (int64_t)gs * (NT / 32), wid = (int64_t)gr * (NT / 32) + (threadIdx.x >> 5);
  for (int64_t q = wid; q < a.B_pad; q += nwarp) {
    const float* xr = q < a.B ? a.x + q * a.n : nullptr;
    for (int i0 = 0; i0 < np; i0 += 32 * U) {
      float v[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int i = i0 + j * 32 + lane;
        v[j] = (xr && i < a.n) ? xr[i] - a.cf[i] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int i = i0 + j * 32 + lane;
        if (i >= np) break;
        const int64_t e = q * np + i;
        a.y[0][e] = v[j];
        a.u[0][e] = v[j];
        // the first operand: the FP16 split of y (MIXED; SPLIT with l2), of
        // r^0 = y + lambda y (SPLIT), or BF16 r^0 (BF16 form)
        float o = v[j];
        if (a.form == FORM_SPLIT && a.h_kind != H_L2) o = v[j] + lam * v[j];
        if (a.form != FORM_BF16) {
          const __half hi = __float2half_rn(o);
          a.p1[0][e] = __half_as_ushort(hi);
          a.p2[0][e] = __half_as_ushort(__float2half_rn((o - __half2float(hi)) * kLoScale));
        } else {
          a.p1[0][e] = __bfloat16_as_ushort(__float2bfloat16_rn(v[j] + lam * v[j]));
        }
      }
    }
  }
  for (int64_t q = tid; q < a.B_pad; q += nthr) {
    const float tt = q < a.B ? d.t[q] : 0.f;
    d.tq[q] = tt;
    a.tau[q] = tt / lam;
    a.taus[0][q] = tt / lam;
    a.qiter[q] = 0;
    a.qdone[q] = q < a.B ? 0 : 1;
    a.sq[0][q] = (int)q;
  }
  for (int64_t c = tid; c < a.B_pad / BN; c += nthr) {
    a.tile_k[c] = 0;
    a.tile_cnt[c] = 0;
  }
  proxy_fence_global();  // the operand planes are read by TMA
}

// The second stage of a staged instance, set up in-kernel by its group (what
// k_dense_init_warm does for hopf_eval, in the same arithmetic): every slot
// plane rebuilt from the first stage's query-indexed results, the iteration
// counts so far kept in qiter0, the tile and decision counters cleared.
__device__ void rag_init_warm(const RagDense& d, int gr, int gs) {
  const TcArgs& a = d.a2;
  const int64_t nthr = (int64_t)gs * NT, tid = (int64_t)gr * NT + threadIdx.x;
  const int np = a.np;
  const float lam = a.lam;
  constexpr int U = 8;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = (int64_t)gs * (NT / 32), wid = (int64_t)gr * (NT / 32) + (threadIdx.x >> 5);
  for (int64_t q = wid; q < a.B_pad; q += nwarp) {
    const bool live = q < a.B;
    const float tl = (live ? d.t[q] : 0.f) / lam;
    const float* xr = live ? a.x + q * a.n : nullptr;
    const float* ur = a.ufin + q * np;
    for (int i0 = 0; i0 < np; i0 += 32 * U) {
      float yv[U], uv[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int i = i0 + j * 32 + lane;
        const bool in = xr && i < a.n;
        yv[j] = in ? xr[i] - a.cf[i] : 0.f;
        uv[j] = in ? ur[i] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const int i = i0 + j * 32 + lane;
        if (i >= np) break;
        const int64_t e = q * np + i;
        const float pv = shrink1(uv[j], tl * a.w[i]);
        const __half hi = __float2half_rn(pv);
        a.y[0][e] = yv[j];
        a.u[0][e] = uv[j];
        a.p1[0][e] = __half_as_ushort(hi);
        a.p2[0][e] = __half_as_ushort(__float2half_rn((pv - __half2float(hi)) * kLoScale));
      }
    }
  }
  for (int64_t q = tid; q < a.B_pad; q += nthr) {
    const int k1 = q < a.B ? a.qiter[q] : 0;
    const bool capped = q < a.B && k1 >= a.max_iter;
    const float tl = (q < a.B ? d.t[q] : 0.f) / lam;
    a.tau[q] = tl;
    a.taus[0][q] = tl;
    a.iter_base[q] = k1;
    a.qiter[q] = capped ? k1 : 0;
    a.qdone[q] = q >= a.B ? 1 : capped ? 2 : 0;
    a.sq[0][q] = (int)q;
  }
  for (int64_t c = tid; c < a.B_pad / BN; c += nthr) {
    a.tile_k[c] = 0;
    a.tile_cnt[c] = 0;
  }
  if (gr == 0 && threadIdx.x == 0)
    for (int j = 2; j < 5; ++j) atomicExch(a.bar + j, 0u);  // the decision counts (not the barrier's own words)
  proxy_fence_global();  // the operand planes are read by TMA
}

__device__ void rag_finalize(const RagDense& d, int gr, int gs) {
  const TcArgs& a = d.a;
  const int64_t nthr = (int64_t)gs * NT, tid = (int64_t)gr * NT + threadIdx.x;
  const bool aborted = *((volatile int*)a.err) != ERR_NONE;
  for (int64_t q = tid; q < a.B; q += nthr) {
    double sum = 0.0, hh = 0.0;
    for (int r = 0; r < a.rt; ++r) {
      sum += a.fpart[(int64_t)r * a.B_pad + q];
      hh += a.fpart[(int64_t)(a.rt + r) * a.B_pad + q];
    }
    const double H = a.h_kind == H_L2 ? sqrt(hh) : hh;
    const double ph = sum - d.c0 - (double)d.tq[q] * H;
    d.phi[q] = ph;
    if (d.dphidt) d.dphidt[q] = (float)(-H);
    if (d.iters) d.iters[q] = a.qiter[q];
    if (d.qstatus) {
      uint8_t st = a.qdone[q] == 1 ? Q_OK : Q_NOT_CONVERGED;
      if (!isfinite(ph)) st = Q_NONFINITE;
      if (!(d.tq[q] >= 0.f)) st = Q_BAD_INPUT;
      if (aborted) st = Q_ABORTED;
      d.qstatus[q] = st;
    }
  }
}

template <int G, int VPT>
__device__ void rag_diag_item(const RagDiag& D, int64_t q0, int nq) {
  const int qi = G == 1 ? (int)threadIdx.x : (G == 32 ? (int)(threadIdx.x >> 5) : 0);
  if (qi >= nq) return;  // whole groups leave together
  const int64_t q = q0 + qi;
  Query<float, G, VPT> Q;
  Q.load(D.e.P, D.e.x + q * D.e.n, D.e.n);
  Q.cold_start();
  const float tq = D.e.t[q];
  bool conv;
  const int k = Q.template solve<false>(D.e.P, tq, &conv);
  emit<false>(D.e, Q, q, tq, k, conv);
}

__device__ void rag_diag_loop(const RaggedArgs& r) {
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(r.ctr, 1u);
    group_sync<256>();
    const int it = s_item;
    group_sync<256>();
    if (it >= r.n_items) break;
    // the instance whose item range holds `it` (first items ascending)
    int lo = 0, hi = r.n_diag - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (r.dinfo[mid].w <= it) lo = mid;
      else hi = mid - 1;
    }
    const int4 w = r.dinfo[lo];
    const RagDiag& D = r.diag[lo];
    const int64_t q0 = (int64_t)(it - w.w) * w.y;
    const int nq = (int)min((int64_t)w.y, (int64_t)w.x - q0);
    switch (w.z) {
      case 0: rag_diag_item<1, 4>(D, q0, nq); break;
      case 1: rag_diag_item<1, 8>(D, q0, nq); break;
      case 2: rag_diag_item<1, 16>(D, q0, nq); break;
      case 3: rag_diag_item<32, 2>(D, q0, nq); break;
      case 4: rag_diag_item<32, 8>(D, q0, nq); break;
      case 5: rag_diag_item<32, 16>(D, q0, nq); break;
      default: rag_diag_item<256, 16>(D, q0, nq); break;
    }
  }
}

__global__ void __launch_bounds__(NT, 1) k_ragged(const __grid_constant__ RaggedArgs r) {
  uint8_t* stages;
  Smem& S = tc_setup<1>(stages);
  ProdState ps;
  for (int s = 0; s < MAX_STAGES; ++s) ps.used[s] = false;
  MmaState ms;
  for (int s = 0; s < Ring<1>::STAGES; ++s) ms.sdesc[s] = smem_desc(sa(stages + (size_t)s * Ring<1>::STAGE_BYTES));
  EpiState es;
  bool alive = true;
  for (int e = r.sched_off[blockIdx.x]; e < r.sched_off[blockIdx.x + 1]; ++e) {
    const int4 w = r.sched[e];
    const RagDense& d = r.dense[w.x];
    const TcArgs& a = d.a;
    if (!alive && threadIdx.x == 0) atomicExch(a.err, ERR_MBAR_TIMEOUT);
    rag_init(d, w.y, w.z);
    bool ok = grid_barrier(a.bar, w.z, a.err, a.wait_limit);
    if (ok) ok = solve_instance<1>(a, S, stages, ps, ms, es, w.y, w.z);
    if (d.staged) {
      if (ok) ok = grid_barrier(a.bar, w.z, a.err, a.wait_limit);
      if (ok) rag_init_warm(d, w.y, w.z);
      if (ok) ok = grid_barrier(a.bar, w.z, a.err, a.wait_limit);
      if (ok) ok = solve_instance<1>(d.a2, S, stages, ps, ms, es, w.y, w.z);
    }
    if (ok) ok = grid_barrier(a.bar, w.z, a.err, a.wait_limit);
    else __syncthreads();
    rag_finalize(d, w.y, w.z);
    if (S.abort) alive = false;
  }
  if (threadIdx.x < 256) rag_diag_loop(r);
  tc_teardown<1>(S, ps, ms);
}
}  // namespace tc

bool tc_encode_f16(CUtensorMap* m, const void* ptr, int64_t rows, int64_t cols) {
  tc::EncodeTiled fn = tc::encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {tc::BK, 128};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


size_t tc_smem_bytes() { return 1024 + (size_t)tc::RING_BYTES + sizeof(tc::Smem); }

// Raise the kernel's dynamic shared memory limit once (at handle creation, so
// that later evaluations stay capturable in a CUDA graph).
hopf_status dense_tc_prepare() {
  static bool done[256] = {};
  int dev = 0;
  HOPF_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 256 && !done[dev]) {
    HOPF_CUDA(cudaFuncSetAttribute(tc::k_dense_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes()));
    HOPF_CUDA(cudaFuncSetAttribute(tc::k_dense_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes()));
    done[dev] = true;
  }
  return HOPF_OK;
}

// cg: CTAs per MMA (the B operand maps copy 128 / cg query rows per tile).
static hopf_status build_tc_args(hopf_handle h, DenseWs& w, const float* x, float* grad, float* beta, float* xfin,
                                 int form, int cg, tc::TcArgs* out) {
  using namespace tc;
  TcArgs& a = *out;
  memset(&a, 0, sizeof(a));
  const int np = h->n_pad;
  const int bh = BN / cg;
  bool ok = encode(&a.mAh, h->d_Ah16, np, np, false) && encode(&a.mAl, h->d_Al16, np, np, false) &&
            encode(&a.mAl2, h->d_Al2, np, np, false) && encode(&a.mP3, w.g, w.B_pad, np, false, bh) &&
            encode(&a.mM, h->d_Mbf, np, np, true) &&
            encode(&a.mP1, w.ph, w.B_pad, np, form == FORM_BF16, bh) &&
            encode(&a.mP2, w.pl, w.B_pad, np, false, bh) && encode(&a.mP1b, w.ph_b, w.B_pad, np, false, bh) &&
            encode(&a.mP2b, w.pl_b, w.B_pad, np, false, bh) && encode(&a.mG, w.g, w.B_pad, np, true, bh) &&
            encode_f32(&a.mU[0], w.u, w.B_pad, np) &&
            encode_f32(&a.mU[1], form != FORM_BF16 ? w.u_b : w.u, w.B_pad, np);
  if (ok && form == FORM_SPLIT)
    ok = encode(&a.mMh, h->d_Mh16, np, np, false) && encode(&a.mMl, h->d_Ml16, np, np, false) &&
         encode(&a.mQ1[0], w.qh, w.B_pad, np, false, bh) && encode(&a.mQ2[0], w.ql, w.B_pad, np, false, bh) &&
         encode(&a.mQ1[1], w.qh_b, w.B_pad, np, false, bh) && encode(&a.mQ2[1], w.ql_b, w.B_pad, np, false, bh);
  if (!ok) return fail(HOPF_ECUDA, "cuTensorMapEncodeTiled failed");
  a.y[0] = w.y;
  a.y[1] = w.y_b;
  a.u[0] = w.u;
  a.u[1] = w.u_b;
  a.p1[0] = w.ph;
  a.p1[1] = w.ph_b;
  a.p2[0] = w.pl;
  a.p2[1] = w.pl_b;
  a.q1[0] = w.qh;
  a.q1[1] = w.qh_b;
  a.q2[0] = w.ql;
  a.q2[1] = w.ql_b;
  a.taus[0] = w.taus;
  a.taus[1] = w.taus + w.B_pad;
  a.qact[0][0] = w.qact;
  a.qact[0][1] = w.qact + w.B_pad;
  a.qact[1][0] = w.qact_b;
  a.qact[1][1] = w.qact_b + w.B_pad;
  a.sq[0] = w.sq;
  a.sq[1] = w.sq + w.B_pad;
  a.g = w.g;
  a.part[0] = w.part;
  a.part[1] = w.part + (int64_t)2 * 2 * w.rt * w.B_pad;
  a.fpart = w.fpart;
  a.tau = w.tau;
  a.qiter = w.qiter;
  a.qdone = w.qdone;
  a.tile_k = w.tile_act;
  a.tile_cnt = w.tile_act + w.B_pad / 128;
  a.ufin = w.ufin;
  a.sfin = w.sfin;
  a.x = x;
  a.cf = h->d_cf;
  a.bar = w.bar;
  a.err = w.err;
  a.w = h->d_wf;
  a.grad = grad;
  a.beta = beta;
  a.xfin = xfin;
  a.B = w.B;
  a.B_pad = w.B_pad;
  a.n = h->n;
  a.np = np;
  a.rt = np / BM;
  a.ct = (int)(w.B_pad / BN);
  a.h_kind = h->h_kind;
  a.max_iter = h->max_iter;
  a.wait_limit = h->wait_limit > 0 ? h->wait_limit : kWaitLimitCycles;
  a.form = form;
  // the BF16 form keeps its r double buffer in set 0 and runs without compaction
  a.compact = form != FORM_BF16 && h->compact && a.ct <= 1024;  // the scan table holds 1,024 tiles
  a.lam = (float)h->lambda;
  a.tol = (float)h->tol;

  return HOPF_OK;
}

// One launch of the persistent solver for the arguments a (built for cg CTAs
// per MMA), on one CTA per SM and no more CTAs than tiles: small problems
// leave the other SMs to concurrent work.
static hopf_status launch_tc(hopf_handle h, const tc::TcArgs& a, int cg, int64_t tiles, int sms, cudaStream_t stream) {
  using namespace tc;
  const size_t smem = tc_smem_bytes();
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  at[1].id = cudaLaunchAttributeClusterDimension;
  at[1].val.clusterDim.x = cg;
  at[1].val.clusterDim.y = 1;
  at[1].val.clusterDim.z = 1;
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  int grid = (int)(tiles < sms ? (tiles > 0 ? tiles : 1) : sms);
  if (cg == 1) {
    int per_sm = 0;
    HOPF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_tc<1>, NT, smem));
    if (per_sm < 1) return fail(HOPF_ECUDA, "dense tensor-core solver: kernel does not fit on an SM");
  } else {
    // whole clusters of two, as many as fit at once (the grid barrier needs
    // every CTA resident)
    static int max_pairs[256] = {};
    int dev = 0;
    HOPF_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(HOPF_ECUDA, "dense tensor-core solver: device index");
    if (max_pairs[dev] == 0) {
      cfg.gridDim = dim3(2 * (h->num_sms / 2));
      cfg.numAttrs = 1;  // the occupancy query takes the cluster shape alone
      cfg.attrs = at + 1;
      int n = 0;
      HOPF_CUDA(cudaOccupancyMaxActiveClusters(&n, (const void*)k_dense_tc<2>, &cfg));
      cfg.attrs = at;
      cfg.numAttrs = 2;
      max_pairs[dev] = n > 0 ? n : -1;
    }
    if (max_pairs[dev] < 0) return fail(HOPF_ECUDA, "dense tensor-core solver: no SM pair fits");
    grid = grid / 2 < max_pairs[dev] ? grid / 2 : max_pairs[dev];
    grid = 2 * (grid > 0 ? grid : 1);
  }
  cfg.gridDim = dim3(grid);
  if (cg == 2) HOPF_CUDA(cudaLaunchKernelEx(&cfg, k_dense_tc<2>, a));
  else HOPF_CUDA(cudaLaunchKernelEx(&cfg, k_dense_tc<1>, a));
  return HOPF_OK;
}

hopf_status dense_eval_tc(hopf_handle h, DenseWs& w, const float* x, const float* t, double* phi, float* grad,
                          float* dphidt, int32_t* iters, uint8_t* qstatus, cudaStream_t stream, float* beta,
                          float* xfin) {
  using namespace tc;
  const int form = h->precision == HOPF_P_MIXED ? FORM_MIXED : h->precision == HOPF_P_SPLIT ? FORM_SPLIT : FORM_BF16;
  if (form == FORM_BF16 && h->h_kind == HOPF_H_L2)
    return fail(HOPF_EUNSUPPORTED, "dense BF16 form: H = l2 needs the MIXED form");
  // MIXED in two stages: the SPLIT form (one phase per iteration) until each
  // query's squared relative change is within split_start, then the defect
  // correction from where it stopped to the tolerance (its fixed point, g = 0,
  // does not depend on the start)
  const bool staged = form == FORM_MIXED && two_stage(h) && w.qh && w.qiter0 && h->d_Mh16;
  const int form1 = staged ? FORM_SPLIT : form;
  hopf_status s = dense_init(h, w, x, t, stream);
  if (s != HOPF_OK) return s;
  const int64_t total = w.B_pad * h->n_pad;
  k_tc_init_operand<<<1024, 256, 0, stream>>>(w.y, w.ph, w.pl, total, form1, (float)h->lambda, h->h_kind);
  HOPF_CUDA(cudaGetLastError());

  // SM pairs: an even number of 128-row tiles, and room for at least two CTAs
  const int rt = h->n_pad / BM;
  const int64_t tiles = (int64_t)rt * (w.B_pad / BN);
  const int sms = h->grid_cap > 0 && h->grid_cap < h->num_sms ? h->grid_cap : h->num_sms;
  const int cg = h->tc_pairs && rt % 2 == 0 && sms >= 2 && tiles >= 2 ? 2 : 1;
  TcArgs a;
  s = build_tc_args(h, w, x, grad, beta, xfin, form1, cg, &a);
  if (s != HOPF_OK) return s;
  if (staged) {
    a.tol = (float)h->split_start;
    a.no_final = 1;
  }
  if (h->prof_start) HOPF_CUDA(cudaEventRecord(h->prof_start, stream));
  s = launch_tc(h, a, cg, tiles, sms, stream);
  if (s != HOPF_OK) return s;
  if (staged) {
    s = dense_init_warm(h, w, x, t, stream);
    if (s != HOPF_OK) return s;
    s = build_tc_args(h, w, x, grad, beta, xfin, FORM_MIXED, cg, &a);
    if (s != HOPF_OK) return s;
    a.warm = 1;
    a.iter_base = w.qiter0;
    s = launch_tc(h, a, cg, tiles, sms, stream);
    if (s != HOPF_OK) return s;
  }
  if (h->prof_stop) HOPF_CUDA(cudaEventRecord(h->prof_stop, stream));
  return dense_finalize(h, w, phi, dphidt, iters, qstatus, stream);
}


size_t ragged_dense_record_bytes() { return sizeof(tc::RagDense); }
size_t ragged_diag_record_bytes() { return sizeof(tc::RagDiag); }

hopf_status ragged_build_dense(hopf_handle h, DenseWs& w, const float* x, const float* t, double* phi, float* grad,
                               float* dphidt, int32_t* iters, uint8_t* qstatus, void* rec) {
  using namespace tc;
  const int form = h->precision == HOPF_P_MIXED ? FORM_MIXED : h->precision == HOPF_P_SPLIT ? FORM_SPLIT : FORM_BF16;
  if (form == FORM_BF16 && h->h_kind == HOPF_H_L2)
    return fail(HOPF_EUNSUPPORTED, "dense BF16 form: H = l2 needs the MIXED form");
  RagDense* d = new (rec) RagDense();
  // MIXED in two stages, as hopf_eval runs it: the SPLIT stage in a, the
  // defect correction (warm) in a2
  const bool staged = form == FORM_MIXED && two_stage(h) && w.qh && w.qiter0 && h->d_Mh16;
  hopf_status s = build_tc_args(h, w, x, grad, nullptr, nullptr, staged ? FORM_SPLIT : form, 1, &d->a);
  if (s != HOPF_OK) return s;
  if (staged) {
    d->a.tol = (float)h->split_start;
    d->a.no_final = 1;
    s = build_tc_args(h, w, x, grad, nullptr, nullptr, FORM_MIXED, 1, &d->a2);
    if (s != HOPF_OK) return s;
    d->a2.warm = 1;
    d->a2.iter_base = w.qiter0;
    d->staged = 1;
  }
  d->t = t;
  d->tq = w.tq;
  d->phi = phi;
  d->dphidt = dphidt;
  d->iters = iters;
  d->qstatus = qstatus;
  d->c0 = h->c0;
  return HOPF_OK;
}

int ragged_diag_class(hopf_handle h) {
  if (h->precision == HOPF_P_FP64 || h->j_kind != 0 || h->h_kind > HOPF_H_L2) return -1;  // runtime kinds: own launch
  const int n = h->n;
  return n <= 4 ? 0 : n <= 8 ? 1 : n <= 16 ? 2 : n <= 64 ? 3 : n <= 256 ? 4 : n <= 512 ? 5 : n <= 4096 ? 6 : -1;
}

void ragged_build_diag(hopf_handle h, int64_t B, const float* x, const float* t, double* phi, float* grad,
                       float* dphidt, int32_t* iters, uint8_t* qstatus, void* rec) {
  tc::RagDiag* d = new (rec) tc::RagDiag();
  d->e = DiagEvalArgs<float>{part_of<float>(h), h->n, B, x, t, phi, grad, dphidt, iters, qstatus, nullptr, nullptr};
}

hopf_status ragged_prepare() {
  static bool done[256] = {};
  int dev = 0;
  HOPF_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 256 && !done[dev]) {
    HOPF_CUDA(cudaFuncSetAttribute(tc::k_ragged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes()));
    done[dev] = true;
  }
  return HOPF_OK;
}

hopf_status ragged_launch(const void* dense, const int4* sched, const int* sched_off, int grid, const void* diag,
                          const int4* dinfo, int n_diag, int n_items, unsigned* ctr, cudaStream_t stream) {
  HOPF_CUDA(ragged_prepare() == HOPF_OK ? cudaSuccess : cudaErrorUnknown);
  tc::RaggedArgs r;
  r.dense = (const tc::RagDense*)dense;
  r.sched = sched;
  r.sched_off = sched_off;
  r.diag = (const tc::RagDiag*)diag;
  r.dinfo = dinfo;
  r.n_diag = n_diag;
  r.n_items = n_items;
  r.ctr = ctr;
  void* args[] = {&r};
  HOPF_CUDA(cudaLaunchCooperativeKernel((const void*)tc::k_ragged, dim3(grid), dim3(tc::NT), args, tc_smem_bytes(),
                                        stream));
  return HOPF_OK;
}
}  // namespace hopf
