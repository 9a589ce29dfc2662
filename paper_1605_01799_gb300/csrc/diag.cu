// Diagonal-A path: the whole split Bregman iteration of one query on chip.
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
#include <cmath>
#include <mutex>

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
      __syncthreads();
      if (lane == 0) {
        s[0][wid] = a;
        s[1][wid] = b;
        s[2][wid] = c;
      }
      __syncthreads();
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
      __syncthreads();
      if (lane == 0) sm[wid] = a;
      __syncthreads();
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
      __syncthreads();
      if (threadIdx.x == 0) s0 = a;
      __syncthreads();
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
          const T du = z[j] - (d[j] + b[j]);  // u^{k-1} = d^{k-1} + b^{k-1}
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
          b[j] = b[j] + vn[j] - dn;  // eq. 3.4(c)
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
          b[j] = b[j] + vn[j] - dn;  // eq. 3.4(c)
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

  // beta with beta = alpha |shrink_1(z, beta)|_1 (Section 4.4).  g(beta) =
  // alpha |shrink_1(z, beta)|_1 - beta is convex, piecewise affine and
  // decreasing, so Newton's method from beta = 0 rises to the root and is
  // exact once a step stays on one affine piece (the count of active
  // coordinates stops changing): at most n + 1 steps, one group reduction of
  // the active sum and count each.
  __device__ T l1sq_root(const T z[VPT], T alpha) const {
    T beta = T(0);
    T cprev = T(-1);
    for (int it = 0; it <= n + 1; ++it) {
      T S = T(0), c = T(0);
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        const T m = fabs(z[j]) - beta;
        if (m > T(0)) {
          S += m;
          c += T(1);
        }
      }
      Group<G, T>::sum2(S, c);
      const T g = alpha * S - beta;
      if (!(g > T(0)) || c == cprev) break;
      cprev = c;
      beta += g / (alpha * c + T(1));
    }
    return beta;
  }

  // mu with |shrink_1(z, mu)|_1 = r for |z|_1 > r (Section 4.2, eq.
  // condition_mu_linfty), by the same Newton iteration on the convex,
  // piecewise affine |shrink_1(z, mu)|_1 - r.
  __device__ T l1ball_mu(const T z[VPT], T r) const {
    T mu = T(0);
    T cprev = T(-1);
    for (int it = 0; it <= n + 1; ++it) {
      T S = T(0), c = T(0);
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        const T m = fabs(z[j]) - mu;
        if (m > T(0)) {
          S += m;
          c += T(1);
        }
      }
      Group<G, T>::sum2(S, c);
      const T h = S - r;
      if (!(h > T(0)) || !(c > T(0)) || c == cprev) break;
      cprev = c;
      mu += h / c;
    }
    return mu;
  }

  // prox of tau H at u for any H kind (eq. 3.4(b)); l_inf and
  // sqrt(sum w p^2) by Moreau's identity: u minus the projection of u on tau
  // times the dual unit ball (the l1 ball; the ellipsoid sum y_i^2 / w_i <= 1,
  // Section 4.3: Newton on its multiplier from 0).
  __device__ void prox_any(const DiagPart<T>& P, T tau, const T u[VPT], const T wv[VPT], T out[VPT]) const {
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
        const T mu = l1ball_mu(u, tau);
#pragma unroll
        for (int j = 0; j < VPT; ++j) out[j] = u[j] - shrink1(u[j], mu);  // sign(u) min(|u|, mu)
      }
    } else if (P.h_kind == H_DNORM) {
      dnorm_prox(tau, u, wv, out);
    } else {  // H_ANORM: the H_DNORM prox in M's eigenbasis (Section 4.3)
      if constexpr (G <= 32) {
        T ur[VPT], pr[VPT];
        matvec_cols(P.P, u, ur);  // P^T u
        dnorm_prox(tau, ur, wv, pr);
        matvec_cols(P.PT, pr, out);  // P pr
      }
    }
  }

  // prox of tau sqrt(sum w p^2) at u: u minus the projection of u on the
  // ellipsoid sum y_i^2 / (tau^2 w_i) <= 1 (Moreau's identity, Section 4.3),
  // Newton on the multiplier from 0.
  __device__ void dnorm_prox(T tau, const T u[VPT], const T wv[VPT], T out[VPT]) const {
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
    T mu = T(0);
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
      // relative: the root can be far below 1 (small tau^2 w), and the
      // projection's error follows the relative error of mu
      if (fabs(dmu) <= eps * mu) break;
    }
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
  __device__ int solve_generic(const DiagPart<T>& P, T t, bool* conv) {
    const T lam = P.lam, tau = t / P.lam;
    const bool paper = P.stop_rule == STOP_PAPER;
    T wv[VPT];
#pragma unroll
    for (int j = 0; j < VPT; ++j) wv[j] = wt(j);
    int k;
    *conv = false;
    for (k = 1; k <= P.max_iter; ++k) {
      T vn[VPT], z[VPT];
      if (P.jk == J_QUAD) {
#pragma unroll
        for (int j = 0; j < VPT; ++j) vn[j] = (y[j] + lam * (d[j] - b[j])) * ia[j];
      } else {
#pragma unroll
        for (int j = 0; j < VPT; ++j) z[j] = (d[j] - b[j]) + y[j] / lam;
        const T beta = l1sq_root(z, P.jk == J_LINFSQ ? T(1) / lam : lam);
#pragma unroll
        for (int j = 0; j < VPT; ++j) {
          const T sh = shrink1(z[j], beta);
          vn[j] = P.jk == J_LINFSQ ? sh : z[j] - sh;
        }
      }
#pragma unroll
      for (int j = 0; j < VPT; ++j) z[j] = vn[j] + b[j];  // u^k = v^k + b^{k-1}
      T dn[VPT];
      prox_any(P, tau, z, wv, dn);                        // eq. 3.4(b)
      T r1 = T(0), r2 = T(0), r3 = T(0);
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        if (paper) {
          r1 += (vn[j] - v[j]) * (vn[j] - v[j]);
          r2 += (dn[j] - d[j]) * (dn[j] - d[j]);
          r3 += (dn[j] - vn[j]) * (dn[j] - vn[j]);
        } else {
          const T du = z[j] - (d[j] + b[j]);  // u^k - u^{k-1}
          r1 += du * du;
          r2 += z[j] * z[j];
        }
        b[j] = b[j] + vn[j] - dn[j];  // eq. 3.4(c)
        d[j] = dn[j];
        v[j] = vn[j];
      }
      Group<G, T>::sum3(r1, r2, r3);
      if (paper) {
        if (r1 <= P.tol && r2 <= P.tol && r3 <= P.tol) {
          *conv = true;
          break;
        }
      } else if (k >= 2 && r1 <= P.tol * (r2 > T(1) ? r2 : T(1))) {
        *conv = true;
        break;
      }
    }
    return k > P.max_iter ? P.max_iter : k;
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

// ---------------------------------------------------------------------------
// Plain evaluation.
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

template <int G>
constexpr int block_of() { return G == 1 || G == 32 ? 128 : G; }

template <typename T, int G, int VPT, bool GEN>
__global__ void __launch_bounds__(block_of<G>()) k_diag_eval(DiagEvalArgs<T> A) {
  const int64_t q = G == 1 ? (int64_t)blockIdx.x * blockDim.x + threadIdx.x
                           : (G == 32 ? ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5 : (int64_t)blockIdx.x);
  if (q >= A.batch) return;  // whole groups leave together
  Query<T, G, VPT> Q;
  Q.load(A.P, A.x + q * A.n, A.n);
  Q.cold_start();
  const T tq = A.t[q];
  bool conv;
  const int k = Q.template solve<GEN>(A.P, tq, &conv);
  double H;
  const double phi = Q.template objective<GEN>(A.P, (double)tq, &H);
  const int l = group_lane<G>();
  bool finite = isfinite(phi);
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
    if (A.qstatus) A.qstatus[q] = !finite ? Q_NONFINITE : (conv ? Q_OK : Q_NOT_CONVERGED);
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

// The H and J kinds that need the runtime-kind loop.
template <typename T>
__host__ __device__ inline bool generic_kind(const DiagPart<T>& P) {
  return P.jk != J_QUAD || P.h_kind == H_LINF || P.h_kind == H_DNORM || P.h_kind == H_ANORM;
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
  if (n <= 16) launch_eval<T, 1, 16>(a, s);
  else if (n <= 64) launch_eval<T, 32, 2>(a, s);
  else if (n <= 256) launch_eval<T, 32, 8>(a, s);
  else if (n <= 512) launch_eval<T, 32, 16>(a, s);
  else if (n <= 4096) launch_eval<T, 256, 16>(a, s);
  else launch_eval<T, 512, 16>(a, s);
  HOPF_CUDA(cudaGetLastError());
  return HOPF_OK;
}

size_t diag_workspace(const hopf_handle, int64_t) { return 0; }

template <typename T>
static DiagPart<T> part_of(hopf_handle h);

template <>
DiagPart<float> part_of<float>(hopf_handle h) {
  return DiagPart<float>{h->d_af, h->d_c ? h->d_cf : nullptr, h->d_wf, h->c0, (float)h->lambda, (float)h->tol,
                         h->max_iter, h->stop_rule, h->h_kind, h->j_kind, h->d_Pf, h->d_PTf, h->d_P};
}
template <>
DiagPart<double> part_of<double>(hopf_handle h) {
  return DiagPart<double>{h->d_A, h->d_c, h->d_w, h->c0,        h->lambda,
                          h->tol, h->max_iter, h->stop_rule, h->h_kind, h->j_kind, h->d_P, h->d_PT, h->d_P};
}

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
    if (U.qstatus) U.qstatus[q] = U.st_parts[q * U.K + best];
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
    return fail(HOPF_EINVAL, "hopf_union_closest_noalloc: batch * parts needs more than the 8 MiB static scratch "
                             "(at most about 490,000 query-part pairs)");
  void* ws = nullptr;
  hopf_status s = noalloc_scratch(&ws);
  if (s != HOPF_OK) return s;
  return union_closest(parts, K, batch, x, s_tol, max_newton, dist, closest, argmin, newton, qstatus, ws, need,
                       stream);
}

}  // namespace hopf
