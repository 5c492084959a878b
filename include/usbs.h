/*
 * usbs.h -- C ABI of libusbs, the GB300 (sm_103a) hot path of USBS, the unified
 * spectral bundle method with sketching of Angell & McCallum (arXiv 2312.11801).
 *
 * Problem (Sec. 2.1, programs (P) and (D)):
 *     maximise <C, X>  s.t.  <A_c, X> = b_c (c not in I),  <A_c, X> <= b_c (c in I),  X PSD
 * with C symmetric n x n and A_1..A_m symmetric.  USBS minimises the penalised dual
 * f(y) = alpha [lambda_max(C - A*(y))]_+ + <b, y> over y_I >= 0 (eq. pen-D) by the
 * proximal bundle iteration of Algorithm 1 (Sec. 3), keeping the primal implicit
 * (<C, Xbar>, tr Xbar, A Xbar; App. C) and, when r > 0, a Nystrom sketch P = Xbar Psi
 * (Sec. 4).
 *
 * Conventions shared by every call
 *  - Return value: USBS_OK (0) or a negative USBS_E* code.  No exception crosses the
 *    ABI.  usbs_last_error(ctx) gives a message for the last failing call on ctx
 *    (usbs_last_error(NULL) for failures of usbs_create itself).
 *  - Indices are 0-based.  Matrices are row-major.
 *  - Host pointers are read during the call only; the library copies what it keeps.
 *  - The library owns all device memory it allocates; it is released by usbs_destroy.
 *  - All work is queued on usbs_params.stream (a cudaStream_t; NULL = a stream the
 *    context creates).  Calls that return host data synchronise that stream.
 *  - A context is not thread-safe: one host thread at a time per context.
 *  - Units: inputs and outputs are in the units of the problem as given.  Internally
 *    the problem is scaled so that ||C||_F = tr(X*) = 1 and alpha = 2 (App. E);
 *    the stopping gates are evaluated in those scaled units, as in the paper.
 */
#ifndef USBS_H
#define USBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define USBS_ABI_VERSION 5   /* 2: usbs_eig_info.reruns, usbs_nystrom_round;
                                3: certification of f(y) and the objective-relative gate;
                                4: the App. B.1 model-value IPM, usbs_selftest_tile_wait;
                                5: usbs_selftest_tf32_round */

/* status codes */
#define USBS_OK          0
#define USBS_EINVAL     -1   /* bad argument: sizes, index ranges, NULL where required */
#define USBS_ENOMEM     -2   /* device allocation failed */
#define USBS_ECUDA      -3   /* a CUDA runtime call failed (message has the CUDA error) */
#define USBS_ETIMEOUT   -4   /* a bounded device-side wait ran out */
#define USBS_ENOTCONV   -5   /* usbs_solve hit max_iters before both gates passed */
#define USBS_EBUSY      -6   /* server or batch has no free slot / budget */
#define USBS_ENUMERIC   -7   /* non-finite value in an FP64 reduction or the IPM */

/* arithmetic of the bulk (n-sized) work; k-sized work is FP64 in both modes */
#define USBS_PRECISION_FP64   0  /* SpMM, Lanczos basis and V in FP64 */
#define USBS_PRECISION_MIXED  1  /* SpMM, reorthogonalisation and V in FP32 */
/* The sketch P and its test matrix Psi are stored in FP32 in both modes (sums in FP64). */

typedef struct usbs_ctx usbs_ctx;

typedef struct usbs_params {
  double alpha;            /* trace bound after scaling; 0 = 2 (App. E) */
  double rho;              /* proximal parameter (eq. proposal_step); default 0.01 */
  double beta;             /* descent fraction (eq. descent_cond); default 0.25 */
  int    k_c;              /* current eigenvectors kept in V, 1..8; default 8 */
  int    k_p;              /* past-information columns (Sec. 3, eqs. model_update_
                              eigendecomposition, x_bar_def, v_next_def): V holds
                              k_c + k_p <= 8 columns; the k_p leading eigenvectors of S stay
                              in V and leave Xbar.  Default 0 (Xbar = X) */
  int    r;                /* sketch rank (Sec. 4); 0 = no sketch */
  int    precision;        /* USBS_PRECISION_*; default MIXED */
  int    lanczos_basis;    /* block Lanczos basis columns J: 16, 32 or 64 (at most n - 16) */
  int    lanczos_restarts; /* Rayleigh-Ritz cycles per eigen solve (App. E: 10) */
  double lanczos_tol;      /* stop when the top-k_c Ritz residuals <= tol * |theta|_max */
  double ipm_mu_tol;       /* IPM stops once mu < ipm_mu_tol (App. B.1: 1e-7) */
  int    ipm_max_iter;     /* Newton steps per IPM call; default 100 */
  int    max_alt;          /* alternating-maximisation passes (eq. small_quad_sdp); 50 */
  double alt_tol;          /* stop alternation when ||d nu|| <= alt_tol (1 + ||b||) */
  double trace_hint;       /* tr(X*) before scaling; 0 = derive from diag equalities */
  int    max_iters;        /* iteration cap of usbs_solve; default 1000 */
  uint64_t seed;           /* seeds the random start/deflation vectors of Lanczos */
  void*  stream;           /* cudaStream_t to run on; NULL = own stream */
  int    device;           /* CUDA device ordinal; -1 = current device */
  /* Certification of the dual value (usbs_solve).  f(y) = alpha lambda_max(C - A*(y))_+
   * + <b, y> bounds the optimum from above only through the exact lambda_max (eq.
   * objective_subopt_upper_bound), and a Ritz value of a budgeted eigen solve is a lower
   * estimate of it.  With certify_restarts > 0, once both gates pass, usbs_solve first
   * recomputes f at the centre y by an eigen solve with a 64-column basis (at most n - 16),
   * at most certify_restarts cycles and residual tolerance certify_tol, keeps the larger of
   * the two values of f(y), and re-evaluates the gates with it; the solve goes on if they
   * no longer pass.  0 = off (the default). */
  int    certify_restarts;
  double certify_tol;      /* 0 = 1e-7 (MIXED) or 1e-10 (FP64) */
  /* When > 0, convergence also needs |f(y) - <C,X>| / |<C,X>| <= obj_gap_tol: the gap
   * relative to the objective itself, beside the paper's 1 + |<C,X>| denominator. */
  double obj_gap_tol;
  /* 1 = compute the model value f^_t(y~) of the descent test (Sec. 3) by the interior
   * point method of App. B.1 (a linear SDP over the model set) instead of its closed form
   * (the maximum over the vertices 0, alpha Xbar / tr Xbar and alpha v v^T, v in range V);
   * usbs_step_info carries both.  0 = closed form (the default). */
  int    model_value_ipm;
} usbs_params;

typedef struct usbs_eig_info {
  int    cycles;           /* Rayleigh-Ritz cycles run */
  int    matvecs;          /* single-vector products with C - A*(y) (block size x SpMMs) */
  int    converged;        /* 1 if every top-k_c residual met lanczos_tol */
  double max_residual;     /* max over top k_c of ||M v - theta v|| (scaled units) */
  int    jacobi_sweeps;    /* Jacobi sweeps of the Rayleigh-Ritz steps, summed */
  int    reruns;           /* cycles run again with the masked deflation passes, summed
                              over the context's life (a speculative cycle met a deficient
                              column); 0 with USBS_NO_SPECULATE=1 in the environment */
} usbs_eig_info;

typedef struct usbs_step_info {
  int    t;                /* iteration index after the step */
  int    descent;          /* 1 = descent step, 0 = null step (Algorithm 1) */
  int    n_alt;            /* alternating-maximisation passes used */
  int    ipm_iters;        /* Newton steps summed over the passes */
  int    matvecs;          /* Lanczos products at the candidate */
  double f_y;              /* f(y_{t+1}), scaled units */
  double f_cand;           /* f(y~_{t+1}) */
  double f_hat;            /* model value f^_t(y~_{t+1}) */
  double lambda_max;       /* lambda_max(C - A*(y~_{t+1})), scaled */
  double cx;               /* <C, X_{t+1}>, scaled */
  double trx;              /* tr X_{t+1}, scaled */
  double eta;              /* weight on Xbar_t in X_{t+1} */
  double relgap;           /* |f(y) - <C,X>| / (1 + |<C,X>|), scaled (App. E) */
  double relinf;           /* dist(A X, K) / (1 + ||b||), scaled (eq. relative_error_tol) */
  double relinf_max;       /* ||A X - proj_K(A X)||_inf, scaled */
  double objective;        /* <C, X_{t+1}> in the units of the given problem */
  double dual_bound;       /* f(y_{t+1}) in the units of the given problem */
  double f_hat_closed;     /* the closed-form model value (equals f_hat unless model_value_ipm) */
  int    ipm_iters_b1;     /* Newton steps of the App. B.1 IPM (model_value_ipm = 1) */
} usbs_step_info;

typedef struct usbs_result {
  int    iters;            /* iterations run by this call */
  int    converged;        /* both gates <= tol (and the objective-relative gap, if asked) */
  int    descent_steps;
  long long matvecs;       /* total Lanczos single-vector products (certification included) */
  usbs_step_info last;     /* diagnostics of the last iteration (f_y, relgap and dual_bound
                              after certification when it ran) */
  int    certifications;   /* certifying eigen solves run (usbs_params.certify_restarts) */
  double cert_residual;    /* max top-k_c Ritz residual of the last one (scaled units) */
  double obj_gap;          /* |f(y) - <C,X>| / |<C,X>| of the last iterate */
} usbs_result;

/* Fill *p with the defaults listed above. */
void usbs_params_default(usbs_params* p);

/* Version of this ABI (USBS_ABI_VERSION). */
int usbs_abi_version(void);

/* Message of the last failure on ctx (NULL ctx: last failure of usbs_create).
 * The string stays valid until the next call on ctx. */
const char* usbs_last_error(const usbs_ctx* ctx);

/*
 * usbs_create -- copy one problem (C, A, b, I) of Sec. 2.1 to the device and set the
 * state to the cold start y_0 = 0, Xbar_0 = 0 (the first solve computes V_0).
 *
 *  n        : order of C and X (n >= 32).
 *  C_rowptr : n+1 int64, C_col : nnz int32, C_val : nnz FP64.  C as CSR with BOTH
 *             triangles; diagonal entries allowed; duplicates are summed.
 *  m        : number of constraints; nnzA entries (A_con[e], A_i[e], A_j[e], A_val[e])
 *             each add A_val[e] * X_ij to <A_con[e], X>.  For i != j the entry stands for
 *             the symmetric matrix (v/2)(e_i e_j^T + e_j e_i^T); i > j is swapped.
 *  b        : m FP64.  is_ineq : m uint8, nonzero = row is <A_c, X> <= b_c.
 *  Psi      : n x r FP32 row-major sketch test matrix (Sec. 4), required iff p->r > 0.
 *  p        : parameters (NULL = defaults).
 * Errors: USBS_EINVAL (sizes, index ranges, r > 0 without Psi, n < 32, k_c + k_p > 8,
 * unknown trace), USBS_ENOMEM, USBS_ECUDA.  *out is NULL on failure.
 */
int usbs_create(usbs_ctx** out, int64_t n, const int64_t* C_rowptr, const int32_t* C_col,
                const double* C_val, int64_t m, int64_t nnzA, const int32_t* A_con,
                const int32_t* A_i, const int32_t* A_j, const double* A_val,
                const double* b, const uint8_t* is_ineq, const float* Psi,
                const usbs_params* p);

/* Release every device allocation of ctx.  NULL is allowed. */
int usbs_destroy(usbs_ctx* ctx);

/*
 * usbs_extreme_eigs -- top-k_c eigenpairs of the dual slack matrix C - A*(y)
 * (Sec. 3: the cost of each f evaluation; App. E: thick-restart Lanczos), by block
 * Lanczos with classical Gram-Schmidt reorthogonalisation (two passes) and thick
 * restart.  Scaled units: the matrix is (C - A*(y_o)) / ||C||_F for y_o given in the
 * problem's units.
 *  y      : m FP64 host, in the problem's units; NULL = the context's current y.
 *  kc     : 1..k_c eigenpairs wanted.
 *  evals  : kc FP64 host, descending, scaled units (multiply by ||C||_F to unscale).
 *  evecs  : n x kc FP64 host row-major orthonormal eigenvectors, or NULL.
 *  info   : optional.
 * The context's V is not changed.
 */
int usbs_extreme_eigs(usbs_ctx* ctx, const double* y, int kc, double* evals,
                      double* evecs, usbs_eig_info* info);

/* One iteration of Algorithm 1 (the body of its loop).  If the context has no iterate yet the
 * cold start (y_0 = 0, Xbar_0 = 0, V_0 = top eigenvectors of C) is made first. */
int usbs_step(usbs_ctx* ctx, usbs_step_info* info);

/*
 * usbs_solve -- iterate until relgap <= tol and relinf <= tol (App. E gates, scaled
 * units) or max_iters.  warm_start = 0 restarts from the cold start; 1 continues from
 * the current state (after usbs_set_state, usbs_grow or earlier steps).  With
 * usbs_params.certify_restarts > 0 the gates are accepted only after f(y) has been
 * recomputed by a certifying eigen solve (see usbs_params); with obj_gap_tol > 0 the
 * objective-relative gap must pass too.
 * Returns USBS_OK when converged, USBS_ENOTCONV at the cap (out is filled either way).
 */
int usbs_solve(usbs_ctx* ctx, int warm_start, double tol, usbs_result* out);

/* Sketch and implicit primal (Sec. 4, App. C), in the problem's units:
 *  P       : n x r FP32 host, X Psi (may be NULL),  Psi : n x r FP32 host (may be NULL),
 *  scalars : 2 FP64 host {<C, Xbar>, tr Xbar} (may be NULL). */
int usbs_get_sketch(usbs_ctx* ctx, float* P, float* Psi, double* scalars);

/*
 * usbs_nystrom_round -- rank-r reconstruction of the primal from its sketch and MaxCut
 * rounding (App. C, eq. nystrom_approx; App. E, rounding).
 * From the context's sketch P = Xbar Psi and test matrix Psi (n x r), by the stable method
 * of Tropp, Yurtsever, Udell and Cevher (2017, Algorithm 3):
 *   nu = sqrt(n) eps(||P||_2) with eps the FP32 spacing (the sketch is stored in FP32),
 *   Y = P + nu Psi, Psi^T Y = R^T R, Y R^-1 = U Sigma W^T, lam = max(Sigma^2 - nu, 0),
 * so that X_hat = U diag(lam) U^T approximates Xbar in the problem's units.  Every column
 * u_k of U gives the sign vector z_k = sgn(u_k) (0 counted as +1), valued <C, z_k z_k^T>
 * (for C = L/4 the weight of the cut z_k); the best column is reported.
 *   lam    : r FP64 host, descending (required).
 *   U      : n x r FP64 host, row-major, orthonormal columns; NULL to skip the copy.
 *   values : r FP64 host, the value of every column's sign vector; may be NULL.
 *   best   : host int, the index of the column with the largest value; may be NULL.
 *   signs  : n int8 host, the best column's sign vector (+1 / -1); may be NULL.
 * Computed on the device in FP64 from the FP32 sketch; allocates n x r doubles of scratch
 * for the call.  Errors: USBS_EINVAL without a sketch (r = 0), USBS_ENUMERIC if Psi^T Y is
 * not positive definite, USBS_ECUDA / USBS_ENOMEM from the device.
 */
int usbs_nystrom_round(usbs_ctx* ctx, double* lam, double* U, double* values, int* best, int8_t* signs);

/*
 * usbs_qap_round -- QAP rounding of the sketch (App. E, QAP: Rounding) for a problem built as
 * the QAP relaxation of eq. qap_sdp, whose primal is indexed by [1; vec(Pi)] (n = nq^2 + 1,
 * vec stacking columns).  From U of usbs_nystrom_round, every column u_k is oriented so that
 * its first entry is non-negative, that entry is dropped, the rest is reshaped column by
 * column into M_k (nq x nq), and the permutation Pi_k maximising <M_k, Pi_k> is found by the
 * Hungarian method on the device; its cost is tr(W Pi_k D Pi_k^T).
 *   W, D   : nq x nq FP64 host, row-major (flows and distances).
 *   costs  : r FP64 host, the cost of every column's permutation (required).
 *   scores : r FP64 host, <M_k, Pi_k>; may be NULL.
 *   perms  : r x nq int host, perms[k nq + i] = the column j with Pi_k(i, j) = 1; may be NULL.
 *   best   : host int, the column of least cost (smallest index on ties); may be NULL.
 * Errors: USBS_EINVAL if n != nq^2 + 1, nq > 64 or r = 0; those of usbs_nystrom_round.
 */
int usbs_qap_round(usbs_ctx* ctx, int nq, const double* W, const double* D, double* costs,
                   double* scores, int* perms, int* best);

/* Current dual iterate y_t (m FP64 host), problem units. */
int usbs_get_dual(usbs_ctx* ctx, double* y);

/* Current primal constraint values A Xbar (m FP64 host), problem units. */
int usbs_get_primal_constraints(usbs_ctx* ctx, double* ax);

/*
 * Complete iterate state (USBS has no iteration-dependent parameters, Sec. 3, so this
 * is a checkpoint and the warm-start input).  Layout of the FP64 host buffer, problem
 * units: [y (m), A Xbar (m), <C,Xbar>, tr Xbar, f(y), V (n*(k_c+k_p) row-major), P (n*r)].
 * usbs_state_size gives its length in doubles.
 */
int64_t usbs_state_size(const usbs_ctx* ctx);
int usbs_get_state(usbs_ctx* ctx, double* state);
int usbs_set_state(usbs_ctx* ctx, const double* state);

/*
 * usbs_grow -- warm start of a grown instance (Sec. 5.1: pad the smaller solution with
 * zeros and rescale).  The new problem must keep the old vertices 0..n_old-1 and
 * constraints 0..m_old-1 in place.  y, A Xbar, tr Xbar and P are unscaled with the old
 * scaling, zero-padded, and rescaled with the new one; <C, Xbar> adds the change of C
 * on old-old entries when that change is diagonal and each changed X_ii is fixed by a
 * one-entry constraint (MaxCut growth), otherwise the implicit primal restarts at 0.
 * V is padded with zero rows.  Psi_new (n_new x r) must extend the old Psi.
 * Arguments after ctx_old are those of usbs_create for the new problem.
 */
int usbs_grow(usbs_ctx* ctx_old, usbs_ctx** out, int64_t n, const int64_t* C_rowptr,
              const int32_t* C_col, const double* C_val, int64_t m, int64_t nnzA,
              const int32_t* A_con, const int32_t* A_i, const int32_t* A_j,
              const double* A_val, const double* b, const uint8_t* is_ineq,
              const float* Psi_new);

/* ---------------------------------------------------------------------------------
 * Single-operation entry points on device buffers (the rows of one iteration run
 * alone, for testing and composition).  All pointers are DEVICE pointers; the
 * operation is queued on the context's stream and the call does not synchronise.
 * Precision of T-typed buffers follows the context: float (MIXED) or double (FP64).
 * --------------------------------------------------------------------------------- */

/* Y = (C - A*(y)) X / ||C||_F for X, Y n x 8 row-major (T); y is m FP64 in scaled
 * units, i.e. the problem's y divided by ||C||_F (usbs_scaling).  The operator of
 * eq. pen-D. */
int usbs_op_matmul(usbs_ctx* ctx, const double* y_scaled_dev, const void* X_dev,
                   void* Y_dev);

/* z = A(V S V^T) (App. C): V n x k_c (T, row-major, k_c columns), S k_c x k_c FP64
 * row-major, z m FP64; scaled operator, so z is in the units of A. */
int usbs_op_constraint_eval(usbs_ctx* ctx, const void* V_dev, const double* S_dev,
                            double* z_dev);

/* Sketch update of Sec. 4 with k_p = 0: P <- eta P + V (S (V^T Psi)), V n x k_c (T),
 * S k_c x k_c FP64, P and Psi n x r FP32.  eta is a host scalar. */
int usbs_op_sketch_update(usbs_ctx* ctx, const void* V_dev, const double* S_dev,
                          const float* Psi_dev, float* P_dev, double eta);

/* ---------------------------------------------------------------------------------
 * Measurement.  With profiling on, every kernel launch of the context is bracketed by
 * two CUDA events on its stream and the elapsed device time is added to one of the
 * kinds below (the events add a few microseconds of host time per launch).
 * --------------------------------------------------------------------------------- */
#define USBS_KIND_SPMM      0  /* (C - A*(y)) X, the Lanczos matvec */
#define USBS_KIND_REORTH    1  /* Gram-Schmidt projection H = Q^T W (and V^T C V) */
#define USBS_KIND_RESTART   2  /* thick-restart and Ritz-vector products Q Y */
#define USBS_KIND_CONSTR    3  /* per-constraint kernels: G^T G, A(V S V^T), alternation */
#define USBS_KIND_SMALL     4  /* one-CTA FP64 kernels: IPM, Cholesky-QR factor, model value */
#define USBS_KIND_REDUCE    5  /* cross-CTA reductions */
#define USBS_KIND_SKETCH    6  /* V^T Psi and the sketch update */
#define USBS_KIND_SETUP     7  /* operator set-up for a new y */
#define USBS_KIND_REORTH_UPDATE 8  /* X = W - Q H with H2 = Q^T X and X^T X (second pass) */
#define USBS_KIND_REORTH_FINAL  9  /* (X - Q H2) R^-1: the new orthonormal block */
#define USBS_KIND_RITZ      10 /* Rayleigh-Ritz of the projected J x J matrix (one CTA) */
#define USBS_NUM_KINDS      11

/* Turn event timing on (1) or off (0); turning it on clears the totals. */
int usbs_profile(usbs_ctx* ctx, int on);
/* Device time (ms), launch count and algorithmic bytes (every input of a launch read
 * once, every output written once; 0 for the one-CTA kinds) of one kind since profiling
 * was turned on.  Synchronises the stream.  Any output pointer may be NULL. */
int usbs_kernel_stats(usbs_ctx* ctx, int kind, double* total_ms, long long* launches,
                      double* bytes);
/* Kernels this context has launched since usbs_create (profiling on or off). */
long long usbs_launch_count(const usbs_ctx* ctx);

/*
 * usbs_selftest_tile_wait -- runs the bounded wait of the staged Gram-Schmidt tiles alone
 * (one CTA on the current device; no context).  Every wait of a tile kernel on its staged
 * copies polls at most 2^20 times with a short sleep (about 0.1 s); when it runs out the
 * kernel writes USBS_ETIMEOUT to the Lanczos status word, waits (bounded again) for copies
 * still in flight, releases its barriers and returns, so the device stays usable and the
 * eigen solve returns USBS_ETIMEOUT.  deliver = 0 arms the barrier for a copy that is never
 * issued, so the wait must run out: returns USBS_ETIMEOUT.  deliver = 1 issues the copy:
 * returns USBS_OK.  USBS_ENOMEM / USBS_ECUDA on a failed allocation or launch.  The paper has
 * no counterpart: this checks the failure path of the library's own waits without a fault.
 */
int usbs_selftest_tile_wait(int deliver);

/*
 * usbs_selftest_tf32_round -- the TF32 rounding of the FP32 Gram-Schmidt tiles (each
 * operand is split into a TF32 high part and a TF32 low part before its m16n8k8 MMAs),
 * run on the current device for `count` values x (host, FP32): ours[i] receives the bits of
 * the tiles' rounding of x[i], ref[i] those of the PTX conversion cvt.rna.tf32.f32 (round to
 * nearest, ties away from zero).  All three arrays are host memory of `count` elements,
 * owned by the caller.  count = 0 is a no-op.  Returns USBS_OK, USBS_EINVAL (count < 0 or a
 * NULL array with count > 0), USBS_ENOMEM or USBS_ECUDA.
 */
int usbs_selftest_tf32_round(int64_t count, const float* x, uint32_t* ours, uint32_t* ref);

/*
 * usbs_sketch_update_static -- the sketch update of usbs_op_sketch_update,
 * P <- eta P + V (S (V^T Psi)), without a context and without allocating anything.
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, for example a serving process that has handed all of HBM to its own
 * memory pool up front, or code that must not take the device-wide synchronisation
 * that cudaMalloc and cudaFree may cause while other work is in flight.
 *
 *  n   : rows (1 <= n < 2^31).   r : sketch rank, 1 <= r <= 32 (USBS_EINVAL beyond).
 *  V_dev   : n x 8 FP32 row-major (columns past k_c zero), device.
 *  S_dev   : 8 x 8 FP64 row-major, device.
 *  Psi_dev : n x r FP32 row-major, device.   P_dev : n x r FP32, updated in place.
 *  stream  : cudaStream_t to run on (NULL = the legacy default stream).
 * The call only queues work; it does not synchronise.  Returns USBS_OK, USBS_EINVAL
 * or USBS_ECUDA (no message is recorded).
 * Its scratch is one static device array of 264,192 bytes (partial sums of V^T Psi and
 * their total), which every GPU that loads the library holds until the process exits.
 * The first call on a device looks the array's address up (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All calls on a
 * device share the array and it keeps the last call's contents; each call writes every
 * scratch entry it reads, so nothing needs clearing, but calls that overlap on the GPU
 * (different streams, or different host threads) race on it and must be serialised.
 */
int usbs_sketch_update_static(int64_t n, int r, const float* V_dev, const double* S_dev,
                              const float* Psi_dev, float* P_dev, double eta, void* stream);

/* ---------------------------------------------------------------------------------
 * Serving and batching.  The paper has no counterpart for these: they are the service
 * forms built around its solver.  Requests enter a FIFO queue; one is admitted when a
 * solve slot is free and its device footprint fits the memory budget.  Each slot is a
 * host thread and each instance owns a CUDA stream, so admitted solves overlap on the
 * GPU (continuous batching).  Finished instances stay device-resident in an LRU cache; a
 * request that names a cached instance as its parent is warm-started from it with
 * usbs_grow, as the paper warm-starts grown instances (Sec. 5.1).
 * --------------------------------------------------------------------------------- */
typedef struct usbs_server usbs_server;

typedef struct usbs_server_params {
  uint64_t hbm_budget_bytes; /* device bytes for resident instances; 0 = 80% of free memory */
  int      max_slots;        /* solves running at once (1..256); default 8 */
  int      cache_entries;    /* finished instances kept for warm starts; default 16 */
  int      dry_run;          /* 1 = no GPU: a request holds its slot for fake_service_s */
  usbs_params solver;        /* parameters of every instance (the stream field is ignored) */
} usbs_server_params;

typedef struct usbs_completion {
  int64_t  request_id;
  int64_t  parent_id;        /* -1 = cold start requested */
  int      status;           /* USBS_OK, USBS_ENOTCONV, USBS_EBUSY (never fits), or an error */
  int      warm;             /* 1 = warm-started from the resident parent */
  int      iters;            /* USBS iterations of the solve */
  int      slot;             /* solve slot that ran it */
  double   objective, dual_bound, relgap, relinf;
  double   t_arrival, t_admit, t_finish;   /* seconds since usbs_server_create */
  uint64_t bytes;            /* device bytes reserved for the instance */
} usbs_completion;

typedef struct usbs_server_stats {
  uint64_t used_bytes, peak_bytes, budget_bytes;
  int      pending, running, peak_running, cached;
  int64_t  finished, rejected;
} usbs_server_stats;

/* Device footprint of one context, as usbs_create allocates it (an upper bound). */
uint64_t usbs_instance_bytes(int64_t n, int64_t nnzC, int64_t m, int64_t nnzA, int r,
                             int precision);

void usbs_server_params_default(usbs_server_params* p);
int usbs_server_create(usbs_server** out, const usbs_server_params* p);

/* Queue one solve.  The problem arguments are those of usbs_create (copied).  parent_id
 * >= 0 asks for a warm start from that finished request if it is still resident (the new
 * problem must extend the parent's as usbs_grow requires); otherwise the solve is cold.
 * fake_service_s is used only in dry-run mode. */
int usbs_server_submit(usbs_server* s, int64_t request_id, int64_t parent_id, int64_t n,
                       const int64_t* C_rowptr, const int32_t* C_col, const double* C_val,
                       int64_t m, int64_t nnzA, const int32_t* A_con, const int32_t* A_i,
                       const int32_t* A_j, const double* A_val, const double* b,
                       const uint8_t* is_ineq, const float* Psi, double tol,
                       double fake_service_s);

/* Move up to max finished requests into out (waiting up to wait_ms for the first one).
 * Returns how many were written, or a negative status. */
int usbs_server_poll(usbs_server* s, usbs_completion* out, int max, int wait_ms);
int usbs_server_get_stats(usbs_server* s, usbs_server_stats* st);
/* Finish every queued and running request, then free the server and its cache. */
int usbs_server_destroy(usbs_server* s);

/* Solve `count` contexts from their cold start, up to max_concurrency at a time (each on
 * its own stream and host thread).  results[i] and status[i] (may be NULL) per context;
 * returns the first hard error, else USBS_OK. */
int usbs_batch_solve(usbs_ctx** ctxs, int count, double tol, int max_concurrency,
                     usbs_result* results, int* status);

/* Scaling of the problem: c = ||C||_F and tau = tr(X*) (App. E). */
int usbs_scaling(const usbs_ctx* ctx, double* c_scale, double* tau);

/* Sizes the context was built with: n, m, k_c, r, precision, J. */
int usbs_dims(const usbs_ctx* ctx, int64_t* n, int64_t* m, int* k_c, int* r,
              int* precision, int* basis);

#ifdef __cplusplus
}
#endif

#endif /* USBS_H */
