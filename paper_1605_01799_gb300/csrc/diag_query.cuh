// Per-query split Bregman state and solver of the diagonal path, shared by
// the plain evaluation (diag.cu) and the unions, maximum over Hamiltonians and
// closest point (diag_union.cu): the whole split Bregman iteration of one
// query on chip.
//
// For A = diag(a) the v-update of eq. 3.4(a) is elementwise,
//   v_i = (y_i + lambda (d_i - b_i)) / (a_i + lambda),
// the d-update (eq. 3.4(b)) is shrink_1 with threshold (t/lambda) w_i or
// shrink_2 with threshold t/lambda, and the b-update (eq. 3.4(c)) is
// b = b + v - d.  A group of G threads owns one query; each thread keeps VPT
// coordinates of y, v, d, b in registers (index i = lane + G * j), so the state
// never leaves the SM (the paper's "very low memory" remark, Section 4.5).
// G = 1 is the paper's own setting (n = 4..16, one evaluation per core);
// G = 32 is a warp per query; G = 256 / 512 is a CTA per query for large n
// (n <= 8192).
#pragma once

#include <cmath>

#include "common.cuh"
#include "hopf_internal.h"

namespace hopf {

template <typename T>
struct DiagPart {
  const T* a;    // [n] diagonal of A
  const T* c;    // [n] centre or null
  const T* w;    // [n] weights (ones when unweighted); eigenvalues of M for H_ANORM
  double c0;
  T lam, tol;
  int max_iter, stop_rule, h_kind;
  int jk;        // initial data: J_QUAD (uses a), J_L1SQ, J_LINFSQ
  const T* P;    // H_ANORM: eigenvectors of M, [n][n] row-major (column k the k-th)
  const T* PT;   // H_ANORM: their transpose
  const double* P64;  // H_ANORM: the FP64 eigenvectors (H in the objective)
};

// Barrier over the G threads of a query group larger than a warp: named
// barrier 15 with G threads (the whole block in the plain kernels, whose
// blocks are one group; the first G threads of a persistent solver CTA that
// runs diagonal work next to its other roles).
template <int G>
__device__ __forceinline__ void group_sync() {
  asm volatile("bar.sync 15, %0;" ::"n"(G) : "memory");
}

// Sum of three values over the G threads of a query group.
template <int G, typename T>
struct Group {
  __device__ static void sum3(T& a, T& b, T& c) {
    if constexpr (G == 1) {
      return;
    } else if constexpr (G == 32) {
      a = warp_sum(a);
      b = warp_sum(b);
      c = warp_sum(c);
    } else {
      __shared__ T s[3][G / 32];
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      a = warp_sum(a);
      b = warp_sum(b);
      c = warp_sum(c);
      group_sync<G>();
      if (lane == 0) {
        s[0][wid] = a;
        s[1][wid] = b;
        s[2][wid] = c;
      }
      group_sync<G>();
      a = T(0);
      b = T(0);
      c = T(0);
#pragma unroll
      for (int k = 0; k < G / 32; ++k) {
        a += s[0][k];
        b += s[1][k];
        c += s[2][k];
      }
    }
  }
  // Maximum over the group.
  __device__ static T max(T a) {
    if constexpr (G == 1) {
      return a;
    } else if constexpr (G == 32) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
      return a;
    } else {
      __shared__ T sm[G / 32];
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
      group_sync<G>();
      if (lane == 0) sm[wid] = a;
      group_sync<G>();
      a = sm[0];
#pragma unroll
      for (int k = 1; k < G / 32; ++k) a = fmax(a, sm[k]);
      return a;
    }
  }
  // Value of the group's first thread, in every thread of the group.
  __device__ static T bcast0(T a) {
    if constexpr (G == 1) {
      return a;
    } else if constexpr (G == 32) {
      return __shfl_sync(0xffffffffu, a, 0);
    } else {
      __shared__ T s0;
      group_sync<G>();
      if (threadIdx.x == 0) s0 = a;
      group_sync<G>();
      return s0;
    }
  }
  // Sum of two values (the two shuffle chains run side by side).
  __device__ static void sum2(T& a, T& b) {
    if constexpr (G == 1) {
      return;
    } else if constexpr (G == 32) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
      }
    } else {
      T c = T(0);
      sum3(a, b, c);
    }
  }
  __device__ static T sum(T a) {
    T b = T(0), c = T(0);
    sum3(a, b, c);
    return a;
  }
};

template <int G>
__device__ __forceinline__ int group_lane() {
  if constexpr (G == 1) return 0;
  else if constexpr (G == 32) return threadIdx.x & 31;
  else return threadIdx.x;
}

template <typename T, int G, int VPT>
struct Query {
  T y[VPT], ia[VPT], v[VPT], d[VPT], b[VPT];  // ia = 1 / (a_i + lambda)
  const T* a;
  const T* w;
  int n;

  __device__ void load(const DiagPart<T>& P, const T* x, int n_) {
    n = n_;
    a = P.a;
    w = P.w;
    const int l = group_lane<G>();
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const int i = l + G * j;
      const bool in = i < n;
      const T xi = in ? x[i] : T(0);
      y[j] = in ? xi - (P.c ? P.c[i] : T(0)) : T(0);
      ia[j] = in && P.jk == J_QUAD ? T(1) / (P.a[i] + P.lam) : T(0);
    }
  }
  __device__ T wt(int j) const {
    const int i = group_lane<G>() + G * j;
    return i < n ? __ldg(w + i) : T(1);
  }
  __device__ T at(int j) const {
    const int i = group_lane<G>() + G * j;
    return i < n && a ? __ldg(a + i) : T(0);
  }
  // The paper's start: v^0 = d^0 = y, b^0 = 0 (Section 3.1).
  __device__ void cold_start() {
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      v[j] = y[j];
      d[j] = y[j];
      b[j] = T(0);
    }
  }

  // Runs split Bregman at time t from the current (v, d, b); returns the
  // iteration count, sets *conv.  One loop per Hamiltonian family (shrink_1
  // thresholds or the l2 scale) and stop rule, so each keeps only the state
  // it reads.  GEN selects the runtime-kind loop (solve_generic), compiled
  // into kernels of its own so the common kinds keep their register budget.
  template <bool GEN>
  __device__ int solve(const DiagPart<T>& P, T t, bool* conv) {
    if constexpr (GEN) return solve_generic(P, t, conv);
    if (P.h_kind == H_L2) {
      return P.stop_rule == STOP_PAPER ? solve_rule<true, true>(P, t, conv) : solve_rule<true, false>(P, t, conv);
    }
    return P.stop_rule == STOP_PAPER ? solve_rule<false, true>(P, t, conv) : solve_rule<false, false>(P, t, conv);
  }

  template <bool L2, bool PAPER>
  __device__ int solve_rule(const DiagPart<T>& P, T t, bool* conv) {
    const T lam = P.lam, tau = t / P.lam;
    T thr[VPT];  // shrink_1 thresholds tau w_i
    if constexpr (!L2) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) thr[j] = tau * wt(j);
    }
    int k;
    *conv = false;
    for (k = 1; k <= P.max_iter; ++k) {
      T vn[VPT], z[VPT];
      T zz = T(0);
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        vn[j] = (y[j] + lam * (d[j] - b[j])) * ia[j];  // eq. 3.4(a)
        z[j] = vn[j] + b[j];                                  // u^k = v^k + b^{k-1}
        zz += z[j] * z[j];
      }
      if constexpr (!PAPER) {
        // relative rule: |u^k - u^{k-1}|^2 and |u^k|^2 are both known before
        // the prox, so one group reduction serves the l2 scale and the test
        T r1 = T(0);
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          const T du = vn[j] - d[j];  // u^k - u^{k-1} = (v^k + b^{k-1}) - (d^{k-1} + b^{k-1})
          r1 += du * du;
        }
        Group<G, T>::sum2(r1, zz);
        T s2 = T(1);
        if constexpr (L2) s2 = shrink2_scale(sqrt(zz), tau);
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          T dn;
          if constexpr (L2) dn = s2 * z[j];            // eq. 3.4(b)
          else dn = shrink1(z[j], thr[j]);
          b[j] = z[j] - dn;  // eq. 3.4(c): b^{k-1} + v^k - d^k = u^k - d^k
          d[j] = dn;
        }
        if (k >= 2 && r1 <= P.tol * (zz > T(1) ? zz : T(1))) {
          *conv = true;
          break;
        }
      } else {
        T s2 = T(1);
        if constexpr (L2) s2 = shrink2_scale(sqrt(Group<G, T>::sum(zz)), tau);
        T r1 = T(0), r2 = T(0), r3 = T(0);
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          T dn;
          if constexpr (L2) dn = s2 * z[j];            // eq. 3.4(b)
          else dn = shrink1(z[j], thr[j]);
          r1 += (vn[j] - v[j]) * (vn[j] - v[j]);
          r2 += (dn - d[j]) * (dn - d[j]);
          r3 += (dn - vn[j]) * (dn - vn[j]);
          b[j] = z[j] - dn;  // eq. 3.4(c): b^{k-1} + v^k - d^k = u^k - d^k
          d[j] = dn;
          v[j] = vn[j];
        }
        Group<G, T>::sum3(r1, r2, r3);
        if (r1 <= P.tol && r2 <= P.tol && r3 <= P.tol) {
          *conv = true;
          break;
        }
      }
    }
    // (v is kept only by the paper rule, the one reader of it)
    return k > P.max_iter ? P.max_iter : k;
  }

  // ---- the initial data and Hamiltonians of Sections 4.2-4.4 ----------

  // The root s of f(s) = alpha |shrink_1(z, s)|_1 - gamma s - r, a convex,
  // piecewise-affine, decreasing function of s >= 0 with breakpoints |z_i|:
  //   beta of the 1/2|.|^2 proxes of Section 4.4 (alpha, gamma, r) = (alpha, 1, 0),
  //   mu of the l1-ball projection of Section 4.2  (alpha, gamma, r) = (1, 0, r).
  // Newton's method from s0 (the previous iteration's root): from the left of
  // the root it rises monotonically, from the right its first step lands on
  // the left (convexity), and the iterate is exact once two consecutive
  // points lie on one affine piece (the same count of active coordinates).
  // Near convergence the active set changes little between split Bregman
  // iterations, so one or two steps suffice; at most n + 3 steps, one group
  // reduction of the active sum and count each.
  __device__ T breakpoint_root(const T z[VPT], T alpha, T gamma, T r, T s0) const {
    T s = s0 > T(0) ? s0 : T(0);
    T cprev = T(-1);
    bool left = false;  // a point with f > 0 has been visited
    for (int it = 0; it <= n + 3; ++it) {
      T S = T(0), c = T(0);
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        const T m = fabs(z[j]) - s;
        if (m > T(0)) {
          S += m;
          c += T(1);
        }
      }
      Group<G, T>::sum2(S, c);
      const T f = alpha * S - gamma * s - r;
      if (c == cprev || f == T(0)) break;  // on the previous point's piece: its root
      if (!(f > T(0)) && left) break;      // from the left only rounding passes the root
      const T slope = alpha * c + gamma;
      if (!(slope > T(0))) {  // beyond every breakpoint with gamma = 0: restart from 0
        s = T(0);
        cprev = T(-1);
        continue;
      }
      if (f > T(0)) left = true;
      cprev = c;
      s += f / slope;
      if (s < T(0)) s = T(0);
    }
    return s;
  }

  // prox of tau H at u for any H kind (eq. 3.4(b)); l_inf and
  // sqrt(sum w p^2) by Moreau's identity: u minus the projection of u on tau
  // times the dual unit ball (the l1 ball; the ellipsoid sum y_i^2 / w_i <= 1,
  // Section 4.3: Newton on its multiplier).  mu carries the multiplier from
  // one call to the next as Newton's starting point.
  __device__ void prox_any(const DiagPart<T>& P, T tau, const T u[VPT], const T wv[VPT], T out[VPT],
                           T& mu) const {
    if (P.h_kind == H_L1 || P.h_kind == H_WL1) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) out[j] = shrink1(u[j], tau * wv[j]);
    } else if (P.h_kind == H_L2) {
      T uu = T(0);
#pragma unroll
      for (int j = 0; j < VPT; ++j) uu += u[j] * u[j];
      const T s2 = shrink2_scale(sqrt(Group<G, T>::sum(uu)), tau);
#pragma unroll
      for (int j = 0; j < VPT; ++j) out[j] = s2 * u[j];
    } else if (P.h_kind == H_LINF) {
      T l1 = T(0);
#pragma unroll
      for (int j = 0; j < VPT; ++j) l1 += fabs(u[j]);
      l1 = Group<G, T>::sum(l1);
      if (l1 <= tau) {
#pragma unroll
        for (int j = 0; j < VPT; ++j) out[j] = T(0);
      } else {
        mu = breakpoint_root(u, T(1), T(0), tau, mu);
#pragma unroll
        for (int j = 0; j < VPT; ++j) out[j] = u[j] - shrink1(u[j], mu);  // sign(u) min(|u|, mu)
      }
    } else if (P.h_kind == H_DNORM) {
      dnorm_prox(tau, u, wv, out, mu);
    } else {  // H_ANORM: the H_DNORM prox in M's eigenbasis (Section 4.3)
      if constexpr (G <= 32) {
        T ur[VPT], pr[VPT];
        matvec_cols(P.P, u, ur);  // P^T u
        dnorm_prox(tau, ur, wv, pr, mu);
        matvec_cols(P.PT, pr, out);  // P pr
      }
    }
  }

  // prox of tau sqrt(sum w p^2) at u: u minus the projection of u on the
  // ellipsoid sum y_i^2 / (tau^2 w_i) <= 1 (Moreau's identity, Section 4.3),
  // Newton on the multiplier from mu0 (0, or the previous call's root).
  // F'(mu) = 1 - sum s2 u^2 / (s2 + mu)^2 is increasing and concave, so from
  // the left Newton rises monotonically and from the right its first step
  // lands on the left.
  __device__ void dnorm_prox(T tau, const T u[VPT], const T wv[VPT], T out[VPT], T& mu0) const {
    if (!(tau > T(0))) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) out[j] = u[j];
      return;
    }
    T ins = T(0);
#pragma unroll
    for (int j = 0; j < VPT; ++j) ins += wv[j] > T(0) ? u[j] * u[j] / (tau * tau * wv[j]) : T(0);
    ins = Group<G, T>::sum(ins);
    if (ins <= T(1)) {
#pragma unroll
      for (int j = 0; j < VPT; ++j) out[j] = T(0);
      return;
    }
    const T eps = sizeof(T) == 8 ? T(1e-14) : T(1e-6);
    T mu = mu0 > T(0) ? mu0 : T(0);
    for (int it = 0; it < 100; ++it) {
      T f1 = T(0), f2 = T(0);
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        const T s2 = tau * tau * wv[j];
        const T q = s2 + mu;
        const T e = q > T(0) ? s2 * u[j] * u[j] / (q * q) : T(0);
        f1 += e;
        f2 += q > T(0) ? T(2) * e / q : T(0);
      }
      Group<G, T>::sum2(f1, f2);
      f1 = T(1) - f1;
      if (!(f2 > T(0))) break;
      const T dmu = -f1 / f2;
      mu += dmu;
      if (mu < T(0)) mu = T(0);  // (a first step from the right may overshoot 0)
      // relative: the root can be far below 1 (small tau^2 w), and the
      // projection's error follows the relative error of mu
      if (fabs(dmu) <= eps * mu) break;
    }
    mu0 = mu;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const T s2 = tau * tau * wv[j];
      out[j] = s2 + mu > T(0) ? u[j] * mu / (s2 + mu) : T(0);
    }
  }

  // out_r = sum_c C[c n + r] in_c over the query's n coordinates, r and c
  // laid out like the state (coordinate lane + G j): the thread's own values
  // for G = 1, warp shuffles for G = 32.  Reads of C are coalesced along r.
  template <typename C_T = T, typename A = T>
  __device__ void matvec_cols(const C_T* __restrict__ C, const T in[VPT], A out[VPT]) const {
#pragma unroll
    for (int j = 0; j < VPT; ++j) out[j] = A(0);
    if constexpr (G == 1) {
#pragma unroll
      for (int c = 0; c < VPT; ++c) {
        if (c < n) {
#pragma unroll
          for (int j = 0; j < VPT; ++j)
            if (j < n) out[j] += (A)__ldg(C + c * n + j) * (A)in[c];
        }
      }
    } else if constexpr (G == 32) {
      const int lane = threadIdx.x & 31;
#pragma unroll
      for (int jc = 0; jc < VPT; ++jc) {
#pragma unroll 2
        for (int l = 0; l < 32; ++l) {
          const int c = l + 32 * jc;
          if (c >= n) break;  // the same for every lane
          const A v = (A)__shfl_sync(0xffffffffu, in[jc], l);
#pragma unroll
          for (int j = 0; j < VPT; ++j) {
            const int r = lane + 32 * j;
            if (r < n) out[j] += (A)__ldg(C + (size_t)c * n + r) * v;
          }
        }
      }
    }
  }

  // Split Bregman for any initial data and Hamiltonian (runtime kinds).  The
  // v-update of eq. 3.4(a) for J = 1/2|x-c|_inf^2 is the prox of
  // (1/(2 lambda)) |.|_1^2 at z = (d - b) + y / lambda: shrink_1(z, beta);
  // for J = 1/2|x-c|_1^2 it is z minus the prox of (lambda / 2) |.|_1^2 at z
  // (Moreau's identity with the scale 1 / lambda).
  //
  // k0 iterations are already done (a continuation from the current state).
  // With handover > 0 (thread per query only) the loop runs in step across
  // the warp, every lane to the same trip count, and ends once at most
  // `handover` lanes still iterate; those set *pending and keep their state
  // for a continuation by the whole warp.  run = false: a lane with no query
  // that only takes part in the warp's votes.
  __device__ int solve_generic(const DiagPart<T>& P, T t, bool* conv, int k0 = 0, int handover = 0,
                               bool run = true, bool* pending = nullptr) {
    const T lam = P.lam, tau = t / P.lam;
    const bool paper = P.stop_rule == STOP_PAPER;
    T wv[VPT];
#pragma unroll
    for (int j = 0; j < VPT; ++j) wv[j] = wt(j);
    T beta_w = T(0), mu_w = T(0);  // Newton's starting points, carried across iterations
    int k = k0;
    bool done = !run;
    *conv = false;
    for (int kk = k0 + 1; kk <= P.max_iter; ++kk) {
      if (!done) {
        k = kk;
        T vn[VPT], z[VPT];
        if (P.jk == J_QUAD) {
#pragma unroll
          for (int j = 0; j < VPT; ++j) vn[j] = (y[j] + lam * (d[j] - b[j])) * ia[j];
        } else {
#pragma unroll
          for (int j = 0; j < VPT; ++j) z[j] = (d[j] - b[j]) + y[j] / lam;
          beta_w = breakpoint_root(z, P.jk == J_LINFSQ ? T(1) / lam : lam, T(1), T(0), beta_w);
#pragma unroll
          for (int j = 0; j < VPT; ++j) {
            const T sh = shrink1(z[j], beta_w);
            vn[j] = P.jk == J_LINFSQ ? sh : z[j] - sh;
          }
        }
#pragma unroll
        for (int j = 0; j < VPT; ++j) z[j] = vn[j] + b[j];  // u^k = v^k + b^{k-1}
        T dn[VPT];
        prox_any(P, tau, z, wv, dn, mu_w);                  // eq. 3.4(b)
        T r1 = T(0), r2 = T(0), r3 = T(0);
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          if (paper) {
            r1 += (vn[j] - v[j]) * (vn[j] - v[j]);
            r2 += (dn[j] - d[j]) * (dn[j] - d[j]);
            r3 += (dn[j] - vn[j]) * (dn[j] - vn[j]);
          } else {
            const T du = vn[j] - d[j];  // u^k - u^{k-1} = (v^k + b^{k-1}) - (d^{k-1} + b^{k-1})
            r1 += du * du;
            r2 += z[j] * z[j];
          }
          b[j] = z[j] - dn[j];  // eq. 3.4(c): b^{k-1} + v^k - d^k = u^k - d^k
          d[j] = dn[j];
          v[j] = vn[j];
        }
        Group<G, T>::sum3(r1, r2, r3);
        if (paper ? (r1 <= P.tol && r2 <= P.tol && r3 <= P.tol)
                  : (kk >= 2 && r1 <= P.tol * (r2 > T(1) ? r2 : T(1)))) {
          *conv = true;
          done = true;
        }
      }
      if constexpr (G == 1) {
        if (handover > 0) {
          const unsigned m = __ballot_sync(0xffffffffu, !done);
          if (m == 0u) break;
          if (__popc(m) <= handover && kk < P.max_iter) {
            if (!done && pending) *pending = true;
            break;
          }
          continue;
        }
      }
      if (done) break;
    }
    return k;
  }

  // phi = <y, d> - 1/2 d^T A d - c0 - t H(d), FP64 accumulation; returns H(d).
  template <bool GEN>
  __device__ double objective(const DiagPart<T>& P, double t, double* H) {
    if constexpr (GEN) return objective_generic(P, t, H);
    double s = 0.0, h = 0.0, z = 0.0;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const double dj = (double)d[j];
      s += (double)y[j] * dj - 0.5 * (double)at(j) * dj * dj;
      if (P.h_kind == H_L2) h += dj * dj;
      else h += (double)wt(j) * fabs(dj);
    }
    Group<G, double>::sum3(s, h, z);
    *H = P.h_kind == H_L2 ? sqrt(h) : h;
    return s - P.c0 - t * (*H);
  }

  // The same for any kind: J*(d) without <c, d> + c0 is 1/2 d^T A d
  // (quadratic J), 1/2 |d|_inf^2 (J = 1/2|.|_1^2) or 1/2 |d|_1^2
  // (J = 1/2|.|_inf^2).
  __device__ double objective_generic(const DiagPart<T>& P, double t, double* H) {
    double s = 0.0, h = 0.0, q = 0.0, m = 0.0;
    if (P.h_kind == H_ANORM) {  // H(d) = sqrt(sum_k l_k ((P^T d)_k)^2), FP64 P and sums
      if constexpr (G <= 32) {
        double r[VPT];
        matvec_cols<double, double>(P.P64, d, r);
#pragma unroll
        for (int j = 0; j < VPT; ++j) h += (double)wt(j) * r[j] * r[j];
      }
    }
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const double dj = (double)d[j];
      if (P.jk == J_QUAD) s += (double)y[j] * dj - 0.5 * (double)at(j) * dj * dj;
      else s += (double)y[j] * dj;
      if (P.jk == J_LINFSQ) q += fabs(dj);
      if (P.h_kind == H_L2) h += dj * dj;
      else if (P.h_kind == H_DNORM) h += (double)wt(j) * dj * dj;
      else if (P.h_kind == H_L1 || P.h_kind == H_WL1) h += (double)wt(j) * fabs(dj);
      m = fabs(dj) > m ? fabs(dj) : m;
    }
    Group<G, double>::sum3(s, h, q);
    if (P.jk == J_L1SQ || P.h_kind == H_LINF) m = Group<G, double>::max(m);
    if (P.jk == J_LINFSQ) s -= 0.5 * q * q;
    else if (P.jk == J_L1SQ) s -= 0.5 * m * m;
    *H = P.h_kind == H_L2 || P.h_kind == H_DNORM || P.h_kind == H_ANORM ? sqrt(h) : (P.h_kind == H_LINF ? m : h);
    return s - P.c0 - t * (*H);
  }
};

template <int G>
constexpr int block_of() { return G == 1 || G == 32 ? 128 : G; }

// The H and J kinds that need the runtime-kind loop.
template <typename T>
__host__ __device__ inline bool generic_kind(const DiagPart<T>& P) {
  return P.jk != J_QUAD || P.h_kind == H_LINF || P.h_kind == H_DNORM || P.h_kind == H_ANORM;
}

// The device view of a diagonal-path handle.
template <typename T>
DiagPart<T> part_of(hopf_handle h);

template <>
inline DiagPart<float> part_of<float>(hopf_handle h) {
  return DiagPart<float>{h->d_af, h->d_c ? h->d_cf : nullptr, h->d_wf, h->c0, (float)h->lambda, (float)h->tol,
                         h->max_iter, h->stop_rule, h->h_kind, h->j_kind, h->d_Pf, h->d_PTf, h->d_P};
}
template <>
inline DiagPart<double> part_of<double>(hopf_handle h) {
  return DiagPart<double>{h->d_A, h->d_c, h->d_w, h->c0,        h->lambda,
                          h->tol, h->max_iter, h->stop_rule, h->h_kind, h->j_kind, h->d_P, h->d_PT, h->d_P};
}

// Arguments of a plain diagonal evaluation and the write-out of one query's
// results (shared by the per-instance kernels and the ragged work list).
template <typename T>
struct DiagEvalArgs {
  DiagPart<T> P;
  int n;
  int64_t batch;
  const T* x;
  const T* t;
  double* phi;
  T* grad;
  T* dphidt;
  int32_t* iters;
  uint8_t* qstatus;
  T* beta;  // optional: control in dH(grad phi), [batch][n]
  T* xfin;  // optional: terminal point x - t beta, [batch][n]
};

// Writes one query's outputs from its final state (any group shape).
template <bool GEN, typename T, int G, int VPT>
__device__ void emit(const DiagEvalArgs<T>& A, Query<T, G, VPT>& Q, int64_t q, T tq, int k, bool conv) {
  double H;
  const double phi = Q.template objective<GEN>(A.P, (double)tq, &H);
  const int l = group_lane<G>();
  const bool finite = isfinite(phi);
#pragma unroll
  for (int j = 0; j < VPT; ++j) {
    const int i = l + G * j;
    if (i < A.n) A.grad[q * A.n + i] = Q.d[j];
  }
  if (A.beta) {
    // at the fixed point lambda b = y - A d, so the control
    // (y - A p) / t = b / tau lies in dH(p) (b = u - prox(u) in tau dH)
    const T tau = tq / A.P.lam;
#pragma unroll
    for (int j = 0; j < VPT; ++j) {
      const int i = l + G * j;
      if (i < A.n) {
        const T bt = tau > T(0) ? Q.b[j] / tau : T(0);
        A.beta[q * A.n + i] = bt;
        if (A.xfin) A.xfin[q * A.n + i] = A.x[q * A.n + i] - tq * bt;
      }
    }
  }
  if (l == 0) {
    A.phi[q] = phi;
    if (A.dphidt) A.dphidt[q] = (T)(-H);
    if (A.iters) A.iters[q] = k;
    if (A.qstatus)
      A.qstatus[q] = !(tq >= T(0)) ? Q_BAD_INPUT : (!finite ? Q_NONFINITE : (conv ? Q_OK : Q_NOT_CONVERGED));
  }
}

}  // namespace hopf
