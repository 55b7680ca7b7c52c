/*
 * gn.h — C ABI of the GB300 Gauss-Newton library for sparse polynomial systems
 * in complex double, double double and quad double arithmetic.
 *
 * The operations follow J. Verschelde and X. Yu, "GPU acceleration of Newton's
 * method for large systems of polynomial equations in double double and quad
 * double arithmetic" (2014):
 *   - systems are given in sparse distributed form (Section 1, Problem
 *     Statement): fully expanded, only monomials with a nonzero coefficient;
 *   - evaluation and differentiation use common factors (Section 2.1, eq. 1),
 *     the Speelpenning product and gradient (Section 2.2) and term sums
 *     (Section 2.3);
 *   - the least-squares update comes from modified Gram-Schmidt on [A b]
 *     (Section 3, eq. 2) and back substitution (eq. 5);
 *   - a Newton step is A = J_f(x0), b = -f(x0), A dx = b, x1 = x0 + dx
 *     (Section 4), taken in the least-squares sense (Gauss-Newton).
 *
 * Conventions shared by every call:
 *   - A complex number at precision L (L = 1, 2, 4) is 2L doubles: the L limbs
 *     of the real part, then the L limbs of the imaginary part.  Each part is
 *     a cascade of doubles (limb l+1 holds what limbs 0..l leave over).  For
 *     L = 1 this is the layout of C99 double complex.
 *   - Pointers named d_* are device pointers the caller owns; pointers named
 *     h_* are host pointers the caller owns.  The library never frees them.
 *   - Every call is stream-ordered on the given CUDA stream (NULL = legacy
 *     default stream) and returns a status; errors never cross the ABI in any
 *     other form.  Device-side failures (a singular pivot, a NaN) are recorded
 *     in a status word that the call reads back after its kernels, so calls
 *     that report such conditions synchronize the stream.
 *   - One gn_system may be used from one host thread and one stream at a time.
 *   - Link with -lgn (libgn.so); the library needs only the CUDA runtime.
 */
#ifndef GN_H
#define GN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Working precision; the value is the number of limbs L. */
typedef enum { GN_D = 1, GN_DD = 2, GN_QD = 4 } gn_prec;

typedef enum {
  GN_OK = 0,
  GN_EINVAL = 1,     /* invalid argument or malformed system */
  GN_ENOMEM = 2,     /* device or host allocation failed */
  GN_ECUDA = 3,      /* a CUDA runtime call failed */
  GN_ESINGULAR = 4,  /* rank-deficient Jacobian: r_kk <= 2^(8-50L) ||a_k|| */
  GN_ENOCONV = 5,    /* tolerance not reached within the allowed steps */
  GN_ENONFINITE = 6, /* NaN or Inf in the inputs (x, coefficients, [A b]), f, J or the update */
  GN_ETIMEOUT = 7    /* a bounded device-side wait gave up */
} gn_status;

/* Opaque, library-owned handle holding a system in device memory. */
typedef struct gn_system gn_system;

#define GN_REPORT_MAX 64

/* Per-step record of gn_newton, host-owned. */
typedef struct {
  int32_t steps_done;               /* steps whose update was applied */
  int32_t status;                   /* gn_status of the run */
  double res_norm[GN_REPORT_MAX];   /* ||f(x_k)||_2 before step k (leading limbs) */
  double dx_norm[GN_REPORT_MAX];    /* ||dx_k||_2 of step k (leading limbs) */
} gn_report;

/*
 * Load a system in sparse distributed form (Section 1).  All arrays are host
 * arrays read once; the caller keeps ownership.
 *   N, n        : number of polynomials and of variables, N >= n >= 1.
 *   T           : total number of monomials (terms) over all polynomials.
 *   h_poly_ptr  : [N+1], monomials of polynomial i are [h_poly_ptr[i], h_poly_ptr[i+1]).
 *   h_mono_ptr  : [T+1], the support of monomial t is h_var[h_mono_ptr[t] ..
 *                 h_mono_ptr[t+1]) with exponents h_exp[...]; an empty support
 *                 is a constant term.
 *   h_var       : variable indices in [0, n); no variable twice in one monomial.
 *   h_exp       : exponents d >= 1 (eq. 1: the monomial is x_{i1}^{d1} ... x_{ik}^{dk}).
 *   h_coef      : [T][2][coef_limbs] doubles: re limbs then im limbs per term.
 *   coef_limbs  : 1, 2 or 4; a run at precision L uses the first min(L, coef_limbs)
 *                 limbs of each part (higher ones taken as 0).
 * Limits: n < 2^24, exponents <= 255, total support length < 2^31.
 * Returns GN_EINVAL for N < n, a variable out of range or repeated within a
 * monomial, an exponent of 0, non-monotone pointers, or null pointers.
 * On success *out owns device memory until gn_system_destroy.
 */
gn_status gn_system_create(gn_system **out, int32_t N, int32_t n, int64_t T,
                           const int64_t *h_poly_ptr, const int64_t *h_mono_ptr,
                           const int32_t *h_var, const uint8_t *h_exp,
                           const double *h_coef, int32_t coef_limbs);

/* Free a system and all workspaces it holds (synchronizes the device). */
gn_status gn_system_destroy(gn_system *s);

/*
 * Arithmetic of evaluation (Section 2) and least squares (Section 3) at every
 * precision.  Inputs and outputs keep the cascade layout either way.
 *   GN_ARITH_INT : integer mantissas with one binary exponent per complex
 *                  value (evaluation) or per column (MGS and back
 *                  substitution); 62, 126 and 254 mantissa bits for L = 1, 2, 4,
 *                  so at least the precision of the cascades; products and
 *                  sums run on the integer pipe.
 *   GN_ARITH_FP64: the cascades themselves, combined by error-free
 *                  transformations of doubles (the paper's double double and
 *                  quad double arithmetic) on the FP64 pipe, with MGS as one
 *                  launch per pivot.
 *   GN_ARITH_AUTO (default): the faster of the two per step on this GPU:
 *                  FP64 evaluation in double precision, integer evaluation in
 *                  DD and QD, integer least squares at every precision.
 * All three meet the accuracy stated for gn_eval, gn_lstsq and gn_newton.
 * Changing it discards the Newton step graphs the system has captured.
 * Returns GN_EINVAL for a null system or an unknown value.
 */
typedef enum { GN_ARITH_AUTO = 0, GN_ARITH_INT = 1, GN_ARITH_FP64 = 2 } gn_arith;
gn_status gn_system_set_arith(gn_system *s, gn_arith arith);

/* Basic facts about a loaded system (any pointer may be NULL). */
gn_status gn_system_info(const gn_system *s, int32_t *N, int32_t *n, int64_t *T,
                         int64_t *nnz, int32_t *max_support);

/*
 * Evaluate and differentiate (Section 2): f(x) and the Jacobian J(x).
 *   d_x : [n] complex at precision prec (2*prec doubles each).
 *   d_f : [N] complex, output; may be NULL to skip f.
 *   d_J : N x n complex, column-major (entry (i, v) at index v*ldJ + i),
 *         output; entries no term touches are set to 0.  May be NULL.
 *   ldJ : leading dimension of d_J in entries, >= N.
 * Stream-ordered; does not synchronize.  Uses workspace owned by s.
 */
gn_status gn_eval(gn_system *s, gn_prec prec, const double *d_x, double *d_f,
                  double *d_J, int64_t ldJ, void *cuda_stream);

/*
 * Least squares by modified Gram-Schmidt on the augmented matrix [A b]
 * (Section 3, figure "The modified Gram-Schmidt orthogonalization algorithm",
 * eq. 2), then back substitution R dx = y (eq. 5).
 *   d_Ab : m x (n+1) complex, column-major with leading dimension ldAb >= m;
 *          columns 0..n-1 are A, column n is b.  Overwritten: columns 0..n-1
 *          by Q, column n by b - Q y (its norm is z of eq. 2).
 *   d_R  : (n+1) x (n+1) complex, column-major, ld n+1, output (not NULL);
 *          R[k][k] real positive, R[0:n, n] = y, R[n][n] = z, zeros below
 *          the diagonal.
 *   d_dx : [n] complex, output: the least-squares solution of A dx = b.
 * Returns GN_ESINGULAR (after synchronizing) when a pivot r_kk, k < n, is at
 * most 2^(8-50L) times the original norm of column k (under GN_ARITH_INT the
 * test compares bit lengths, so the threshold holds within a factor of 2),
 * and GN_ENONFINITE when [A b] holds a NaN or an infinity.
 */
gn_status gn_lstsq(gn_system *s, gn_prec prec, int32_t m, int32_t n, double *d_Ab,
                   int64_t ldAb, double *d_R, double *d_dx, void *cuda_stream);

/*
 * The factorisation of gn_lstsq alone: modified Gram-Schmidt on [A b]
 * (Section 3, eq. 2) without the back substitution, fully stream-ordered.
 *   d_Ab, ldAb, d_R : as for gn_lstsq (Q and b - Q y overwrite d_Ab; R into d_R).
 *   d_status : device int32 the caller owns; when the kernels finish it holds
 *              GN_OK, GN_ESINGULAR (the rank test of gn_lstsq), GN_ENONFINITE
 *              (a NaN or an infinity in [A b]) or GN_ETIMEOUT.
 * Requires n <= the system's number of variables (it uses the system's
 * workspace).  Does not synchronize: check *d_status after the stream does.
 */
gn_status gn_mgs(gn_system *s, gn_prec prec, int32_t m, int32_t n, double *d_Ab, int64_t ldAb,
                 double *d_R, int32_t *d_status, void *cuda_stream);

/*
 * Take up to `steps` Gauss-Newton steps (Section 4) in place on d_x:
 * evaluate f and J (Section 2), solve [J, -f] by MGS least squares (Section 3),
 * x <- x + dx.  The whole loop stays on the device; the host reads back only
 * the per-step norms once at the end (or once per step when tol > 0, to test
 * ||dx|| <= tol * ||x||).
 *   d_x    : [n] complex at precision prec, updated in place.
 *   steps  : 1 .. GN_REPORT_MAX.
 *   tol    : 0 to always take `steps` steps; > 0 to stop early, GN_ENOCONV if
 *            never reached.
 *   report : host-owned, may be NULL.
 * Synchronizes the stream before returning.  A step that fails (GN_ESINGULAR;
 * GN_ENONFINITE for a NaN or an infinity in x or a coefficient, which
 * reaches f and J; GN_ETIMEOUT) leaves x as the previous step left it.
 */
gn_status gn_newton(gn_system *s, gn_prec prec, double *d_x, int32_t steps, double tol,
                    gn_report *report, void *cuda_stream);

/*
 * Gauss-Newton with the factorisation in double precision and the residuals
 * at precision prec (GN_DD or GN_QD).  Section 5.2 of the paper finds the
 * linear solve dominant when evaluation is cheap and suggests iterative
 * methods in double arithmetic; this call is such a method:
 *   1. d_steps Gauss-Newton steps (Section 4) in double precision on the
 *      leading limbs of x (as gn_newton with GN_D);
 *   2. refine_steps refinement steps with the last double factorisation
 *      [J, -f] = Q R (Section 3) frozen: b = -f(x) at precision prec
 *      (Section 2), y = Q^H b in double, R dx = y in double, x <- x + dx at
 *      precision prec.
 * Under GN_ARITH_INT or GN_ARITH_AUTO with 32 <= n <= 1024 the double
 * factorisation is CholeskyQR: R from the Cholesky factor of the Gram
 * matrix of [J, -f] (scaled by its columns' powers of two, in float-float
 * arithmetic on the FP32 pipe: about 47 significant bits), Q never formed,
 * and the refinement's y = R^-H (J^H b); the triangular solves run on the
 * float-float factor too (blocked, on one 8-CTA cluster); its error, about kappa(J)^2 2^-47,
 * suits Jacobians with kappa(J)^2 2^-47 << 1, and a pivot below 2^-20 of its
 * column's norm is reported as GN_ESINGULAR.  The Gram matrix is exact for the columns
 * rounded at their scales, then rounded once to doubles: on the tensor
 * cores (BF16 products of 7-bit digit planes, 56-bit columns) for N <= 2048,
 * else on the integer pipe (62-bit columns).  The first such call on a
 * system allocates the tensor-core form's scratch, kept until
 * gn_system_destroy: 32 Np nq + 2^22 nb (nb + 1) bytes (Np = N rounded up to
 * 64, nb = ceil((n+1)/128), nq = 128 nb; 434 MB at N = 1536, n = 1024); if
 * it cannot be allocated the integer-pipe form runs instead.  With
 * CholeskyQR the double step and the refinement step are each captured once
 * as a CUDA graph and then replayed (kept with the system; the refinement's
 * is captured again for another d_x), and the Cholesky's panels run one
 * ahead on a second, high-priority stream that the system owns.  Otherwise
 * the double phase is MGS.
 * Phase 2 gains about -log10(kappa(J) u_double) digits per step, so for a
 * consistent system (f(x*) = 0) it reaches the root at precision prec:
 * quad double from a double start takes three or four steps for
 * kappa(J) up to about 1e4.
 *   d_x          : [n] complex at precision prec, updated in place (after
 *                  phase 1 its lower limbs are those of the double iterate).
 *   d_steps      : >= 1; refine_steps >= 0; d_steps + refine_steps <= GN_REPORT_MAX.
 *   tol          : 0 to take every refinement step; > 0 to stop the
 *                  refinement once ||dx|| <= tol ||x|| (GN_ENOCONV if never).
 *   report       : host-owned, may be NULL: the double steps first, then
 *                  the refinement steps.
 * Synchronizes the stream.  Returns GN_EINVAL for an unknown precision or
 * step counts, and the status of phase 1 (GN_ESINGULAR, ...) if it fails.
 * The paper has no counterpart of this entry point.
 */
gn_status gn_newton_mixed(gn_system *s, gn_prec prec, double *d_x, int32_t d_steps,
                          int32_t refine_steps, double tol, gn_report *report, void *cuda_stream);

/*
 * Replace the coefficients of a loaded system from device memory (the
 * supports stay).  d_coef: [T][2][coef_limbs] doubles, the layout of
 * gn_system_create's h_coef, caller-owned; coef_limbs 1, 2 or 4.  Stream-
 * ordered: calls issued later on the same stream see the new coefficients,
 * and captured Newton step graphs stay valid (they read the coefficients
 * when they run).  Returns GN_EINVAL for a null system or pointer or an
 * unknown coef_limbs.
 */
gn_status gn_system_set_coef(gn_system *s, const double *d_coef, int32_t coef_limbs,
                             void *cuda_stream);

/*
 * Gradient of a real loss with respect to every coefficient at a root x.
 * The paper's Newton's method (Section 4) is the forward solve; this is its
 * adjoint by the implicit function theorem at the Gauss-Newton fixed point:
 * at a root with J of full column rank the root moves by dx = -J^+ (df/dc) dc,
 * J^+ = R^-1 Q^H for J = QR (Section 3), so for a loss gradient
 * g = dL/dRe x + i dL/dIm x the coefficient gradient is
 *   grad_t = dL/dRe c_t + i dL/dIm c_t = -lambda_i conj(x^{a_t}),
 *   lambda = Q w with R^H w = g,
 * for term t of polynomial i.  Every coefficient, constant terms included,
 * counts as an independent input.
 *   d_x      : [n] complex at precision prec, a root of the system (the
 *              result of gn_newton); the formula is the derivative of the
 *              root only where f(x) = 0.
 *   d_g      : [n] complex, the loss gradient at x (2x for L = sum |x_j|^2).
 *   d_grad   : [T] complex, output.
 *   d_lambda : [N] complex, output, may be NULL.
 *   flags    : 0 evaluates [J, -f] at x (Section 2) and factors it by MGS
 *              (Section 3) in the system's arithmetic; GN_ADJ_REUSE instead
 *              takes the factorisation the last gn_newton (of J at the
 *              iterate before its result) or gn_adjoint call at this
 *              precision left, and returns GN_EINVAL when another call
 *              (gn_lstsq, gn_mgs, gn_system_set_coef, gn_system_set_arith, a
 *              failed step) has replaced it since.  After a converged run the
 *              last step moved x by about the working precision, so the two
 *              Jacobians agree to that precision; with a larger last step the
 *              gradient is off by about that step's relative size.
 * Then R^H w = g, lambda = Q w and the gradients follow in the cascade
 * arithmetic of precision prec.  Synchronizes the stream.  Returns
 * GN_ESINGULAR for a rank-deficient J (the rank test of gn_lstsq), and then
 * leaves d_grad and d_lambda undefined.
 */
#define GN_ADJ_REUSE 1
gn_status gn_adjoint(gn_system *s, gn_prec prec, const double *d_x, const double *d_g,
                     double *d_grad, double *d_lambda, int32_t flags, void *cuda_stream);

/*
 * Batches: many independent square systems (N_s = n_s <= 128) advanced
 * together (Section 4 steps on every system of the batch).  The systems are
 * stored back to back in sparse distributed form (Section 1):
 *   S          : number of systems.
 *   h_sys_n    : [S], n_s in 1 .. 128; system s owns polynomials
 *                [P_s, P_s + n_s) and variables [X_s, X_s + n_s) of the
 *                concatenated vectors (P_s = X_s = n_0 + ... + n_{s-1}).
 *   T          : total number of terms over all polynomials.
 *   h_poly_ptr : [X+1] (X = sum of n_s) term ranges of the polynomials.
 *   h_mono_ptr, h_exp, h_coef, coef_limbs : as for gn_system_create.
 *   h_var      : variable indices LOCAL to each system, in [0, n_s).
 * Returns GN_EINVAL for a malformed batch (as gn_system_create, per system).
 * The paper treats one system at a time; batching is this library's.
 */
typedef struct gn_batch gn_batch;
gn_status gn_batch_create(gn_batch **out, int32_t S, const int64_t *h_sys_n, int64_t T,
                          const int64_t *h_poly_ptr, const int64_t *h_mono_ptr,
                          const int32_t *h_var, const uint8_t *h_exp, const double *h_coef,
                          int32_t coef_limbs);
gn_status gn_batch_destroy(gn_batch *b);
gn_status gn_batch_info(const gn_batch *b, int32_t *S, int64_t *X, int64_t *T, int64_t *nnz,
                        int32_t *max_n);
/*
 * Take `steps` Gauss-Newton steps on every system of the batch, in place on
 * d_x ([X] complex at precision prec, the systems' variables back to back).
 * Each step is one CUDA graph: evaluation of all systems (integer mantissa
 * arithmetic), then one persistent launch that solves every system's least
 * squares problem by MGS and back substitution and adds dx.
 *   d_status : [S] device int32, caller-owned, GN_OK on entry for the systems
 *              to advance; a system whose least squares problem fails gets
 *              GN_ESINGULAR or GN_ENONFINITE and is left alone afterwards.
 *   d_norms  : [steps][S][2] device doubles (may be NULL): ||f(x_k)|| and
 *              ||dx_k|| of each system at each step.
 * Stream-ordered; does not synchronize.  The first call per precision tunes
 * the launch on the batch (gn_batch_tuning: six evaluations and up to four
 * solves on a copy of x, synchronizing) and keeps the fastest choices.
 */
gn_status gn_batch_newton(gn_batch *b, gn_prec prec, double *d_x, int32_t steps, double *d_norms,
                          int32_t *d_status, void *cuda_stream);

/*
 * The launch choices the first gn_batch_newton call at precision prec made
 * by timing the candidates on the batch (host-owned outputs, any may be
 * NULL):
 *   eval_block    : CTA size of the per-term evaluation kernel (64, 128, 256);
 *   eval_lanes    : lanes per term of that kernel: 1 (the product chain of
 *                   Section 2.2 on one lane) or 2 (its forward and backward
 *                   products on a lane pair);
 *   solve_threads : CTA size of the persistent solver (128 or 256);
 *   solve_grid    : its CTAs (SMs x resident CTAs);
 *   largest_first : 1 when its work queue takes the largest systems first,
 *                   0 when it takes them as stored.
 * Returns GN_EINVAL for a null batch, an unknown precision or a precision
 * not yet stepped.  Batching and its tuning are this library's, not the
 * paper's.
 */
gn_status gn_batch_tuning(const gn_batch *b, gn_prec prec, int32_t *eval_block, int32_t *eval_lanes,
                          int32_t *solve_threads, int32_t *solve_grid, int32_t *largest_first);

/*
 * gn_eval_noalloc — the same evaluation as gn_eval, for callers that may not
 * allocate device memory when they evaluate (a host thread inside a CUDA
 * stream capture it does not own, a real-time loop that forbids allocator
 * calls, a process whose device memory is a fixed pool handed out
 * elsewhere).  gn_eval allocates its workspace on first use; this call
 * allocates nothing: it calls no cudaMalloc, no cudaFree and no allocating
 * library routine.  Its scratch is one static device array of
 * GN_NOALLOC_SCRATCH_BYTES inside the library, which every process that
 * loads the library holds on each GPU it uses until it exits.
 *   It always evaluates with the GN_ARITH_FP64 kernels (cascades combined
 *   by error-free transformations), whatever gn_system_set_arith chose; the
 *   results meet the accuracy stated for gn_eval.
 *   Arguments, layouts and outputs are those of gn_eval; d_x, d_f and d_J
 *   remain caller memory and the system must already be loaded (loading it
 *   allocates).  Like gn_eval it is stream-ordered, does not synchronize and
 *   reports no device-side condition: a NaN or infinite input comes out as
 *   NaN or infinite entries of f and J.
 *   Returns GN_EINVAL for a system with a monomial of more than 64
 *   variables (gn_eval accepts those, e.g. cyclic n-roots for n > 64), and
 *   when the scratch the system needs — 256 bytes plus 16 * prec bytes per
 *   power-table entry (n x max(dmax-1, 1)), per term (T) and per variable
 *   occurrence (nnz), each part rounded up to 256 bytes — exceeds
 *   GN_NOALLOC_SCRATCH_BYTES.
 *   The first call on a device looks up the scratch address on that device
 *   (cudaGetSymbolAddress) and loads the kernels of all three precisions
 *   (under lazy module loading a kernel's first launch may allocate); make
 *   that first call, in any precision, before any stream capture.
 *   All calls share the one array and it keeps the last call's contents:
 *   calls whose work overlaps on the GPU (other streams, other host threads)
 *   race on it and must be serialized by the caller.
 * The paper has no counterpart of this entry point.
 */
#define GN_NOALLOC_SCRATCH_BYTES (64u << 20)
gn_status gn_eval_noalloc(const gn_system *s, gn_prec prec, const double *d_x, double *d_f,
                          double *d_J, int64_t ldJ, void *cuda_stream);

/*
 * Bound of one device-side wait of the MGS kernel (the cluster reductions
 * and the pivot flags of Section 3's factorisation, which the kernel runs
 * as one persistent launch), in SM clock cycles, on the current device.
 * A wait that runs out records GN_ETIMEOUT in the call's status word; every
 * other wait of the launch then gives up at once and the kernel returns, so
 * a lost message costs about one bound and leaves the device usable.
 *   cycles   : > 0 sets the bound; 0 restores the default (2e9 cycles,
 *              about one second at the GB300's clock).
 *   previous : host int64, may be NULL: the bound before this call.
 * Applies to launches issued after the call (also replays of captured
 * Newton graphs, which read the bound when they run).  Not stream-ordered:
 * change it while no factorisation is in flight.  Returns GN_EINVAL for
 * cycles < 0, GN_ECUDA if the device copy cannot be read or written.
 * For tests of the failure path and for callers that prefer a prompt
 * GN_ETIMEOUT over a long wait; the paper has no counterpart.
 */
gn_status gn_set_wait_limit(int64_t cycles, int64_t *previous);

/* Human-readable name of a status. */
const char *gn_status_str(gn_status st);

/* Library version as major*10000 + minor*100 + patch. */
int32_t gn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GN_H */
