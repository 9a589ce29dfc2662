/*
 * hopf.h - C ABI of the GB300 (sm_103a) Hopf-formula evaluator.
 *
 * The library evaluates, for many queries (x, t) at once, the viscosity
 * solution of the Hamilton-Jacobi initial value problem
 *     d phi/dt + H(grad_x phi) = 0,  phi(x, 0) = J(x)       (eqs. 1.1a-1.1b)
 * through the Hopf formula
 *     phi(x, t) = -min_v { J*(v) + t H(v) - <x, v> }         (eq. 1.2, eq. 3.3)
 * of Darbon & Osher, "Algorithms for overcoming the curse of dimensionality
 * for certain Hamilton-Jacobi equations arising in control theory and
 * elsewhere".  The minimisation runs split Bregman (eq. 3.4(a)-(c)).
 *
 * Initial data (quadratic, Section 4: J = 1/2 <., D^{-1} .> generalised):
 *     J(x) = 1/2 (x - c)^T A^{-1} (x - c) - c0,
 *     J*(v) = 1/2 v^T A v + <c, v> + c0,
 * with A symmetric positive definite, given either by its diagonal or as a
 * dense matrix.  Hamiltonians (positively 1-homogeneous, Section 2.1):
 *     H(p) = sum |p_i| (l1), sum w_i |p_i| (weighted l1, w_i > 0), |p|_2 (l2).
 * Outputs per query: phi, grad_x phi = the minimiser v* (Section 1: the
 * gradient is the unique minimiser of eq. 1.2), d phi/dt = -H(v*) (eq. 1.1a),
 * the split Bregman iteration count and a status byte.
 *
 * Conventions for every entry point:
 *   - All array arguments of hopf_eval* / hopf_union_* / hopf_backward are
 *     DEVICE pointers owned by the caller, row-major, query-major: x[q*n + i].
 *     hopf_desc arrays are HOST pointers, read during hopf_create only.
 *   - Work is enqueued on `stream`; calls return once the work is enqueued.
 *     The caller synchronises the stream before reading results.
 *   - Errors in arguments or CUDA calls return a non-OK status; the message
 *     is in hopf_last_error() (thread-local).  Numerical outcomes per query
 *     (no convergence, non-finite values) never fail the call: they are
 *     reported in qstatus.
 *   - batch == 0 is a valid no-op.
 *   - No entry point below allocates memory except hopf_create (the handle's
 *     own copies of the data); scratch comes from the caller's workspace,
 *     whose size hopf_workspace_size reports.
 */
#ifndef HOPF_GB300_H
#define HOPF_GB300_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hopf_handle_s* hopf_handle;

typedef enum {
  HOPF_OK = 0,
  HOPF_EINVAL = 1,        /* bad argument (null pointer, size, ...) */
  HOPF_ENOMEM = 2,        /* device allocation failed in hopf_create */
  HOPF_ECUDA = 3,         /* a CUDA runtime or driver call failed */
  HOPF_ENOTSPD = 4,       /* A + lambda I (or M of HOPF_H_ANORM) is not SPD */
  HOPF_EUNSUPPORTED = 5,  /* valid request this build does not implement */
  HOPF_ETIMEOUT = 6       /* a bounded device-side wait gave up (no hang) */
} hopf_status;

/* Initial data J.  Quadratic, J(x) = 1/2 (x-c)^T A^{-1} (x-c) - c0, with a
 * diagonal or dense SPD A; or the norms of Section 4.4 (no A):
 * HOPF_J_L1SQ J = 1/2 |x-c|_1^2 - c0, HOPF_J_LINFSQ J = 1/2 |x-c|_inf^2 - c0
 * (both run on the diagonal path: per-query state in registers). */
enum { HOPF_A_DIAG = 0, HOPF_A_DENSE = 1, HOPF_J_L1SQ = 2, HOPF_J_LINFSQ = 3 };
/* Hamiltonians: |p|_1, sum w_i |p_i|, |p|_2 (Section 1), |p|_inf (Section
 * 4.2: prox by Moreau's identity and the projection on the l1 ball),
 * sqrt(sum w_i p_i^2) (Section 4.3, diagonal D = diag(w): prox by the
 * projection on an ellipsoid, Newton on its multiplier) and sqrt(<p, M p>)
 * with M symmetric positive definite (Section 4.3: the same projection in
 * M's eigenbasis; hopf_create computes M = P diag(l) P^T once, and each
 * iteration rotates by P^T and back by P).  l_inf, sqrt(sum w p^2) and
 * sqrt(<p, M p>) need the diagonal path; sqrt(<p, M p>) needs n <= 512. */
enum { HOPF_H_L1 = 0, HOPF_H_WL1 = 1, HOPF_H_L2 = 2, HOPF_H_LINF = 3, HOPF_H_DNORM = 4, HOPF_H_ANORM = 5 };

/* Arithmetic of the v-update (eq. 3.4(a)).
 *   FP64   diagonal A only; use hopf_eval_f64.
 *   FP32   diagonal: FP32 per-query kernel.  Dense: the paper's form
 *          v = (A + lambda I)^{-1} r as an FP32 CUDA-core GEMM per iteration.
 *   BF16   dense: the same form with M = (A + lambda I)^{-1} and r in BF16 on
 *          the tensor cores (tcgen05), FP32 accumulation.  Fast, ~1e-2 error.
 *   SPLIT  dense: the paper's form v = M r on the tensor cores with both
 *          operands as two-term FP16 splits, M = M_hi + 2^-11 M_lo and
 *          r = r_hi + 2^-11 r_lo, three MMAs per k-step
 *          (M_hi r_hi, then M_hi r_lo + M_lo r_hi in a second accumulator
 *          scaled exactly by 2^-11), FP32 accumulation: ~2^-22 per product,
 *          FP32-class results in one phase per iteration.
 *   MIXED  dense: tensor-core defect-correction form u <- u + M g(u) with
 *          g = y - A p - lambda (u - p), A p from a two-term FP16 split with
 *          an exactly scaled correction accumulator, M g in BF16.  Its fixed
 *          point depends only on the accuracy of g: FP32-class results, two
 *          phases (four MMAs) per iteration.  With H = l1 or weighted l1 it
 *          starts with SPLIT iterations (hopf_set_split_start).
 * SPLIT does three n x n MMA passes per iteration in one phase, MIXED four in
 * two.  The tensor cores' FP32 accumulation truncates; in SPLIT that error
 * reaches the fixed point amplified by |A + lambda I|, in MIXED it enters
 * through g alone, so at the same tolerance SPLIT's gradient is a few times
 * less accurate (about 1e-5 against 3e-6 relative for a condition number of
 * 100 at n = 1024).
 */
enum { HOPF_P_FP64 = 0, HOPF_P_FP32 = 1, HOPF_P_BF16 = 2, HOPF_P_SPLIT = 4, HOPF_P_MIXED = 5 };

/* Stopping rules.
 *   PAPER: |v^k - v^{k-1}|^2, |d^k - d^{k-1}|^2, |d^k - v^k|^2 all <= tol
 *          (Section 4.5).  Diagonal A only.
 *   UREL:  |u^k - u^{k-1}|^2 <= tol * max(1, |u^k|^2) for k >= 2, where
 *          u^k = v^k + b^{k-1} is the argument of the d-update. */
enum { HOPF_STOP_PAPER = 0, HOPF_STOP_UREL = 1 };

/* Per-query status bytes.  ABORTED: a bounded device-side wait of the dense
 * solver gave up (it never hangs); every query of that call carries it.
 * BAD_INPUT: the query's t is negative or NaN (t lives on the device, so the
 * call cannot refuse it); its outputs carry no meaning.
 * NONFINITE: phi came out NaN or infinite (e.g. a NaN or infinite coordinate
 * of x); such a query's residual never passes the stop test, so it runs to
 * max_iter.  Queries are independent: a bad query leaves every other query's
 * outputs bit-identical. */
enum { HOPF_Q_OK = 0, HOPF_Q_NOT_CONVERGED = 1, HOPF_Q_NONFINITE = 2, HOPF_Q_ABORTED = 3, HOPF_Q_BAD_INPUT = 4 };

/* Problem description for hopf_create (host memory, copied).
 *   n          dimension, 1 <= n <= 8192 (diagonal) or 4096 (dense)
 *   a_kind     HOPF_A_DIAG: A points to n doubles > 0;
 *              HOPF_A_DENSE: A points to n*n doubles, row-major, symmetric;
 *              HOPF_J_L1SQ / HOPF_J_LINFSQ: A ignored (may be NULL)
 *   centre     n doubles, or NULL for c = 0
 *   c0         constant of J
 *   h_kind     HOPF_H_L1 / HOPF_H_WL1 / HOPF_H_L2 / HOPF_H_LINF / HOPF_H_DNORM /
 *              HOPF_H_ANORM
 *   w          n doubles > 0 for HOPF_H_WL1 and HOPF_H_DNORM; for HOPF_H_ANORM
 *              M, n*n doubles, row-major, symmetric positive definite (else
 *              HOPF_ENOTSPD); else ignored (may be NULL)
 *   lambda     split Bregman parameter, > 0 (the paper uses 1)
 *   tol        stopping tolerance for stop_rule, > 0
 *   max_iter   cap on split Bregman iterations, >= 1
 *   precision  HOPF_P_*
 *   stop_rule  HOPF_STOP_* */
typedef struct {
  int32_t n;
  int32_t a_kind;
  const double* A;
  const double* centre;
  double c0;
  int32_t h_kind;
  const double* w;
  double lambda;
  double tol;
  int32_t max_iter;
  int32_t precision;
  int32_t stop_rule;
} hopf_desc;

/* Build a handle: copies A, c, w to the device and, for dense A, forms
 * M = (A + lambda I)^{-1} on the GPU (the prox of the quadratic J*,
 * Section 3.1 / Section 4.1: (I + alpha A)^{-1}) with the casts the chosen
 * precision needs: in FP64 for HOPF_P_FP32 and HOPF_P_SPLIT, which apply M
 * as the v-update; in FP32 for HOPF_P_MIXED, where M only preconditions the
 * defect correction (whose fixed point uses A itself), and HOPF_P_BF16, which
 * rounds M to BF16.  Returns HOPF_ENOTSPD when a pivot of A + lambda I is not
 * positive (an FP32 pivot that is not is checked again in FP64).  The handle
 * is immutable afterwards: hopf_eval may run on several streams at once with
 * distinct workspaces.  Synchronises `stream`. */
hopf_status hopf_create(const hopf_desc* desc, hopf_handle* out, cudaStream_t stream);

/* Release the handle and its device memory (NULL is a no-op). */
void hopf_destroy(hopf_handle h);

/* Bytes of device workspace hopf_eval / hopf_eval_f64 need for `batch`
 * queries (256-byte aligned pointer expected), with the handle's current
 * settings (the two-stage MIXED solve, hopf_set_split_start, needs the SPLIT
 * form's operand planes too). */
hopf_status hopf_workspace_size(hopf_handle h, int64_t batch, size_t* bytes);

/* Evaluate `batch` queries (FP32 interface; any precision but FP64).
 *   x       [batch][n] float, device      t      [batch] float >= 0, device
 *   phi     [batch] double (FP64-accumulated phi), device
 *   grad    [batch][n] float: grad_x phi = d^K (eq. 3.4(b) iterate), device
 *   dphidt  [batch] float: -H(grad), device, may be NULL
 *   iters   [batch] int32: split Bregman iterations, device, may be NULL
 *   qstatus [batch] uint8: HOPF_Q_*, device, may be NULL
 * t must be >= 0 (a query with t < 0 or NaN reports HOPF_Q_BAD_INPUT); t = 0
 * gives phi = J(x) (eq. 1.1b).  The split Bregman start
 * is v^0 = d^0 = x - c, b^0 = 0 (Section 3.1). */
hopf_status hopf_eval(hopf_handle h, int64_t batch, const float* x, const float* t, double* phi, float* grad,
                      float* dphidt, int32_t* iters, uint8_t* qstatus, void* workspace, size_t ws_bytes,
                      cudaStream_t stream);

/* Same with FP64 queries and gradients; requires precision HOPF_P_FP64 and a
 * diagonal A (the paper's own setting: FP64, n = 4..16, Section 4.5). */
hopf_status hopf_eval_f64(hopf_handle h, int64_t batch, const double* x, const double* t, double* phi, double* grad,
                          double* dphidt, int32_t* iters, uint8_t* qstatus, void* workspace, size_t ws_bytes,
                          cudaStream_t stream);

/* Optimal control and terminal point (Section 2: the control of the optimal
 * trajectory is beta = grad H(grad_x phi); for a 1-homogeneous H the terminal
 * point is the Hopf-Lax minimiser x - t beta).  Same call as hopf_eval, plus
 *   beta    [batch][n] float: the control.  At the fixed point the optimality
 *           condition of eq. 3.3 gives lambda b = y - A p (for the norm
 *           initial data, y - lambda b lies in dJ*(p)), so the library
 *           returns beta = b / (t / lambda) = (u - prox(u)) / (t / lambda),
 *           which lies in the subdifferential dH(p) (equal to grad H(p)
 *           where H is differentiable); 0 when t = 0.  Device, required.
 *   x_final [batch][n] float: x - t beta (device, may be NULL).
 * FP32-output handles (diagonal FP32, dense FP32 / SPLIT / MIXED / BF16); FP64
 * handles return HOPF_EUNSUPPORTED.  Workspace as for hopf_eval. */
hopf_status hopf_eval_control(hopf_handle h, int64_t batch, const float* x, const float* t, double* phi, float* grad,
                              float* dphidt, int32_t* iters, uint8_t* qstatus, float* beta, float* x_final,
                              void* workspace, size_t ws_bytes, cudaStream_t stream);

/* Maximum over Hamiltonians (Section 2.2: for one convex initial data J and
 * Hamiltonians H_1..H_K, max_i phi_i solves the HJ equation with the
 * Hamiltonian min_i H_i).  parts: K diagonal FP32 handles that share n and
 * J (A, centre, c0; not checked beyond n) and may differ in h_kind and
 * weights.  phi [batch] double = max_i phi_i; grad [batch][n] = the gradient
 * of the maximising part; argmax [batch] int32 (ties -> smallest i); iters
 * [batch] (iterations of that part, may be NULL); qstatus [batch] (may be
 * NULL); all device.  workspace: hopf_union_workspace_size(parts, K, batch)
 * bytes. */
hopf_status hopf_maxH_eval(const hopf_handle* parts, int32_t K, int64_t batch, const float* x, const float* t,
                           double* phi, float* grad, int32_t* argmax, int32_t* iters, uint8_t* qstatus,
                           void* workspace, size_t ws_bytes, cudaStream_t stream);

/* Union of initial data (Section 2.2: the pointwise minimum of the solutions
 * for convex J_i solves the problem with initial data min_i J_i).
 * parts: K handles, all diagonal FP32 with the same n and h_kind
 * (hopf_union_workspace_size asks for the same n only).
 *   phi [batch] double = min_i phi_i; grad [batch][n] float = grad of the
 *   minimising part; argmin [batch] int32 (ties -> smallest i); iters [batch]
 *   (iterations of the minimising part), qstatus [batch]; all device.
 * workspace: hopf_union_workspace_size bytes. */
hopf_status hopf_union_workspace_size(const hopf_handle* parts, int32_t K, int64_t batch, size_t* bytes);
hopf_status hopf_union_eval(const hopf_handle* parts, int32_t K, int64_t batch, const float* x, const float* t,
                            double* phi, float* grad, int32_t* argmin, int32_t* iters, uint8_t* qstatus,
                            void* workspace, size_t ws_bytes, cudaStream_t stream);

/* Distance and closest point to the union of the sets {J_i <= 0}
 * (Section 3.2).  For each part, Newton's method on s for psi_i(y, s) = 0,
 * psi_i the eikonal (H = l2) solution with initial data J_i:
 *     s <- s + psi_i(y, s) / |grad psi_i(y, s)|   (eq. Newton_zero with
 *     d psi/ds = -|grad psi|), s_0 = 0,
 * stopping when |delta s| <= s_tol * max(1, s) or after max_newton steps, each
 * step one split Bregman solve warm-started from the previous one.  Then
 * dist = min_i s_i and closest = y - s grad psi / |grad psi| for the nearest
 * part (eq. projection_when_s_known).  parts: diagonal quadratic J, h_kind HOPF_H_L2, same
 * n.  Queries must lie outside every set (J_i(x) > 0).
 *   dist [batch] float, closest [batch][n] float (may be NULL), argmin [batch]
 *   int32, newton [batch] int32 Newton steps of the nearest part (may be
 *   NULL), qstatus [batch] (may be NULL); all device. */
hopf_status hopf_union_closest(const hopf_handle* parts, int32_t K, int64_t batch, const float* x, float s_tol,
                               int32_t max_newton, float* dist, float* closest, int32_t* argmin, int32_t* newton,
                               uint8_t* qstatus, void* workspace, size_t ws_bytes, cudaStream_t stream);

/* hopf_union_closest without any allocation, for callers that may not call
 * cudaMalloc once running: a controller that queries distances to obstacles
 * at a fixed rate, code inside a fixed memory budget, or a host that gives the
 * library no allocator.  (The paper has no counterpart: this is a property of
 * the library, not of the method.)  Same arguments and results as
 * hopf_union_closest, minus the workspace: the scratch is one static 8 MiB
 * device array that every GPU which loads the library holds until the
 * process exits.  A call needs batch * (17 K + 4) bytes of it (five regions,
 * each rounded up to 256 bytes), so batch may not exceed about 399,000
 * queries with one part, or about 30,000 with 16 (larger requests return
 * HOPF_EINVAL and launch nothing).  The first call on
 * a device looks up the array's device address with that device current;
 * make that first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents (nothing in it needs to start at
 * zero): calls that overlap on the GPU race, so serialise them. */
hopf_status hopf_union_closest_noalloc(const hopf_handle* parts, int32_t K, int64_t batch, const float* x,
                                       float s_tol, int32_t max_newton, float* dist, float* closest, int32_t* argmin,
                                       int32_t* newton, uint8_t* qstatus, cudaStream_t stream);

/* Gradients of phi with respect to the data by the envelope theorem applied
 * to eq. 3.3 (v* = grad, the minimiser): with upstream weights g_phi[q],
 *   g_x[q]  = g_phi[q] v*_q                  ([batch][n] float, may be NULL)
 *   g_t[q]  = -g_phi[q] H(v*_q)              ([batch] float, may be NULL)
 *   g_A     = -1/2 sum_q g_phi[q] v*_q v*_q^T   (dense: [n][n] float; diagonal:
 *             [n] float, the diagonal only; may be NULL; overwritten)
 * All device pointers.  Dense g_A is a batched outer-product GEMM. */
hopf_status hopf_backward(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, float* g_x,
                          float* g_t, float* g_A, cudaStream_t stream);

/* hopf_backward with the dense g_A on the tensor cores (tcgen05): the same
 * outputs, with g_A = -1/2 V^T diag(g) V computed from two-term FP16 splits of
 * g V and V (about 2^-22 per product), the main product promoted from tensor
 * memory to registers every 512 queries and the partial products of each
 * 4,096-query range summed in FP64.  workspace: device memory of at least
 * hopf_backward_workspace_size bytes (256-byte aligned), owned by the caller;
 * nothing is allocated.  Without a dense A (or with g_A NULL or batch 0) it
 * is hopf_backward.  A bounded device wait that gives up (see
 * hopf_set_wait_limit) leaves NaN in g_A. */
hopf_status hopf_backward_workspace_size(hopf_handle h, int64_t batch, size_t* bytes);
hopf_status hopf_backward_ws(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar, float* g_x,
                             float* g_t, float* g_A, void* workspace, size_t ws_bytes, cudaStream_t stream);

/* Gradients of L = sum_q g_phi[q] phi_q with respect to the problem's other
 * parameters, by the same envelope argument (phi = <x - c, p> - J*_0(p) - c0
 * - t H(p) at the minimiser p = vstar):
 *   g_c  [n] float   dL/dc    = -sum_q g_phi[q] vstar[q]                (may be NULL)
 *   g_c0 [1] float   dL/dc0   = -sum_q g_phi[q]                         (may be NULL)
 *   g_w  [n] float   dL/dw_i  = -sum_q g_phi[q] t[q] |vstar[q][i]|      (HOPF_H_WL1)
 *                             = -sum_q g_phi[q] t[q] vstar[q][i]^2 / (2 H_q)
 *                               with H_q = -dphidt[q] (HOPF_H_DNORM; 0 where H_q = 0)
 *                    (may be NULL; requested for another h_kind: HOPF_EUNSUPPORTED)
 * t [batch] is needed for g_w, dphidt [batch] (the forward's output) for g_w
 * with HOPF_H_DNORM.  All device pointers, float sums accumulated in FP64 in a
 * fixed order (the result does not depend on the launch).  batch = 0 writes
 * zeros. */
hopf_status hopf_backward_params(hopf_handle h, int64_t batch, const float* g_phi, const float* vstar,
                                 const float* t, const float* dphidt, float* g_c, float* g_c0, float* g_w,
                                 cudaStream_t stream);

/* ---- ragged batches -----------------------------------------------------
 * Many independent instances (each with its own A, H, n and number of
 * queries) evaluated together.  Queries share no state (Section 1; Section
 * 4.5 runs them one per core), so the batch is a set of single evaluations,
 * recorded into one CUDA graph and replayed by later calls that pass the same
 * buffers and counts.  Two schedules:
 *   persistent  one cooperative launch of the ragged solver: the dense
 *               tensor-core instances run on a schedule of CTA groups (an
 *               instance with at least one 128 x 128 tile per SM on the whole
 *               GPU, the others side by side on "lanes" of the SMs, longest
 *               first to the least loaded lane), then every diagonal instance
 *               from a shared work list (256 queries of a thread-per-query
 *               instance, 8 of a warp-per-query one or one query of a
 *               256-thread one per item).  The arithmetic of every query is
 *               that of hopf_eval: results are the same bit for bit.
 *   streams     per instance the kernels hopf_eval launches, forked onto
 *               worker streams ("lanes", the dense solvers capped at an equal
 *               share of the SMs).
 * Instances the persistent solver does not take (dense FP32, the diagonal
 * runtime kinds, diagonal n > 4096) run their own launches beside it.
 *
 * Layout: instance i has counts[i] queries.  Per-query arrays (t, phi, dphidt,
 * iters, qstatus) hold the instances one after another: instance i starts at
 * row sum_{j<i} counts[j].  x and grad hold instance i's rows of length n_i
 * starting at element sum_{j<i} counts[j] * n_j.  counts is a HOST array;
 * everything else is device memory, as for hopf_eval.
 *
 * The first hopf_batch_eval call tunes the schedule: it captures and times
 * the persistent schedule with 4 to 32 lanes, wide instances on the whole GPU
 * or on lanes too, some SMs starting on the diagonal instances, and the stream
 * schedule with 8 and 16 lanes, and keeps the fastest (so it synchronises
 * `stream`; its results are complete when it returns); hopf_batch_info
 * reports the choice.  Instances with FP64 precision are not accepted.
 * hopf_batch_create keeps a pinned host copy of the persistent schedule
 * (O(instances x SMs) bytes). */
typedef struct hopf_batch_s* hopf_batch;
hopf_status hopf_batch_create(const hopf_desc* descs, int32_t count, hopf_batch* out, cudaStream_t stream);
void hopf_batch_destroy(hopf_batch b);
hopf_status hopf_batch_workspace_size(hopf_batch b, const int64_t* counts, size_t* bytes);
hopf_status hopf_batch_eval(hopf_batch b, const int64_t* counts, const float* x, const float* t, double* phi,
                            float* grad, float* dphidt, int32_t* iters, uint8_t* qstatus, void* workspace,
                            size_t ws_bytes, cudaStream_t stream);
/* nstreams: lanes chosen (0 before the first eval); used_graph: 0 before the
 * first eval, 1 when the batch replays the persistent schedule's graph, 2 the
 * stream schedule's; tuned_ms[8]: the timed candidates (may be NULL): the
 * persistent schedule with 4, 8, 16, 32 lanes (wide dense instances on the
 * whole GPU), 8 and 16 lanes with 8 SMs and 16 lanes with 16 SMs starting on
 * the diagonal work list, and 8 lanes taking every dense instance; with
 * mode 2 the stream schedule with 1, 2, 4, 8, 16 lanes in the first five. */
hopf_status hopf_batch_info(hopf_batch b, int32_t* nstreams, int32_t* used_graph, float* tuned_ms);

/* Schedule the tuner may pick: 0 either (the default), 1 persistent only,
 * 2 streams only.  Drops the current graph; the next hopf_batch_eval tunes
 * again. */
hopf_status hopf_batch_set_mode(hopf_batch b, int32_t mode);

/* Instrumentation: when `start` and `stop` are non-NULL CUDA events, every
 * later hopf_eval on this handle records `start` on its stream immediately
 * before the main solver kernel and `stop` immediately after it, so a caller
 * can time that kernel alone (cudaEventElapsedTime).  NULL, NULL turns it off.
 * Not thread-safe with concurrent hopf_eval calls on the same handle. */
hopf_status hopf_profile_events(hopf_handle h, cudaEvent_t start, cudaEvent_t stop);

/* Limit of every bounded device-side wait of the dense solvers (their grid
 * barriers and, on the tensor-core path, the waits on the TMA ring and the
 * accumulator hand-offs), in SM clock cycles; 0 restores the default of 2^32
 * (about two seconds).  A wait that runs out makes the kernel record an
 * error word, drain its copies and MMAs, free its tensor memory and return:
 * the call's queries then report HOPF_Q_ABORTED, and the handle stays usable.
 * (The paper has no counterpart: this bounds the library's own waits.)  Not
 * thread-safe with concurrent evaluations on the same handle. */
hopf_status hopf_set_wait_limit(hopf_handle h, int64_t cycles);

/* Dense A on the tensor cores: with on != 0 a call whose padded n is a
 * multiple of 256 runs each MMA over an SM pair (a cluster of two CTAs,
 * tcgen05 cta_group::2: a 256 x 128 tile per pair, each CTA bringing in its
 * own 128 rows of A and half of the 128 query rows of the operand); on == 0
 * (the default: on GB300 the pairs measured 5-9 % slower on the dense
 * workloads) keeps one CTA per 128 x 128 tile.  Both compute every product in
 * the same K order, so the outputs agree bit for bit.  Takes effect at the
 * next evaluation; ragged batches always use single CTAs.  (The paper has no
 * counterpart.) */
hopf_status hopf_set_tc_pairs(hopf_handle h, int32_t on);

/* HOPF_P_MIXED with H = l1 or weighted l1 solves in two stages: the
 * HOPF_P_SPLIT iteration (one tensor-core phase per iteration) until each
 * query's squared relative change |u^k - u^{k-1}|^2 / max(1, |u^k|^2) is at
 * most tol_switch, then the defect correction (two phases per iteration) from
 * where that query stopped until the handle's tolerance.  The defect
 * correction's fixed point (g = 0) does not depend on its start, so the
 * results keep the MIXED form's accuracy; the second stage corrects the
 * SPLIT fixed point's bias.  Reported iterations count both stages, and
 * max_iter caps their sum.  tol_switch = 0 runs the defect correction alone;
 * the default is ten times the handle's tolerance.  A workspace must be sized
 * (hopf_workspace_size) after the last call: the first stage needs the SPLIT
 * form's operand planes.  Ragged batches run their MIXED instances the same
 * way (both schedules), with each instance's switch as created.
 * Errors: HOPF_EINVAL for a null handle or a negative or non-finite
 * tol_switch; HOPF_EUNSUPPORTED for tol_switch > 0 with another precision or
 * H.  (The switch is this library's; the paper's iteration is unchanged.) */
hopf_status hopf_set_split_start(hopf_handle h, double tol_switch);

/* Device allocator for the memory hopf_create and hopf_batch_create keep (the
 * handle's copies of A, M and the weights, and their set-up scratch).
 * alloc(bytes, ctx) returns device memory or NULL (then the create call
 * frees what it already took and returns HOPF_ENOMEM); release(ptr, ctx)
 * gives it back.  Both NULL restores cudaMalloc / cudaFree; exactly one NULL
 * is HOPF_EINVAL.  Process-wide; each handle remembers the allocator it was
 * made with and frees through it in hopf_destroy.  Install it while no create
 * call runs on another thread.  (The paper has no counterpart.) */
typedef void* (*hopf_alloc_fn)(size_t bytes, void* ctx);
typedef void (*hopf_free_fn)(void* ptr, void* ctx);
hopf_status hopf_set_allocator(hopf_alloc_fn alloc, hopf_free_fn release, void* ctx);

/* Query compaction of the dense tensor-core (MIXED) solver: as queries
 * converge, the still-active ones are packed into fewer column tiles so the
 * tensor cores work only on unconverged queries.  On by default; off gives the
 * same results (each query's arithmetic does not depend on its column), only
 * slower.  Other paths ignore it. */
hopf_status hopf_set_compaction(hopf_handle h, int32_t on);

/* Roofline denominators measured on the current device (the paper has no
 * counterpart: a calibration utility for reporting throughput against the
 * hardware at hand).  Runs fixed-size probe kernels on `stream` and waits for
 * them (it synchronises the stream):
 *   fp32_tflops  chains of FP32 fused multiply-adds, 2 flop each (may be NULL)
 *   fp64_tflops  the same in FP64 (may be NULL)
 *   l2_read_gbs  repeated 16-byte reads of a 32 MiB buffer, which stays in L2
 *                (may be NULL)
 * scratch: device memory of at least hopf_measure_pipes_scratch() bytes,
 * owned by the caller; its contents are overwritten.  Changes no setting of
 * the GPU. */
size_t hopf_measure_pipes_scratch(void);
hopf_status hopf_measure_pipes(void* scratch, size_t scratch_bytes, double* fp32_tflops, double* fp64_tflops,
                               double* l2_read_gbs, cudaStream_t stream);

/* Message of the last failed call on this thread ("" if none). */
const char* hopf_last_error(void);

/* Library version string. */
const char* hopf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HOPF_GB300_H */
