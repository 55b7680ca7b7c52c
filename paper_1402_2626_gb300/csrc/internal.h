// internal.h — library-internal declarations shared by the .cu files.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/gn.h"

namespace gn {

// An NVTX range over a host-side phase of an entry point (named "gn_newton:
// capture" and so on), for timelines of a profiler; without a profiler
// attached the calls do nothing.  Device work inside a captured graph shows
// under the kernels' own names.
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

// One workspace per precision, allocated on first use.
struct Workspace {
  bool ready = false;
  double *pow = nullptr;        // [pmax][n] complex: plane p holds x^(p+1)
  double *stage_val = nullptr;  // [T] complex: value of each term
  double *stage_d = nullptr;    // [nnz] complex: d_s * partial of each occurrence
  double *Ab = nullptr;         // N x (n+1) complex, column-major, ld N
  double *R = nullptr;          // (n+1) x (n+1) complex, column-major
  double *dx = nullptr;         // [n] complex
  double *lam = nullptr;        // [N] complex: multipliers of the coefficient gradient
  double *xmix = nullptr;       // [n] complex: the double iterate of mixed-precision Newton
  double *rinv = nullptr;       // [(n+1) L] 1 / r_kk, [n+1] original column norms, [n+1] exponents
  double *norms = nullptr;      // [3 * GN_REPORT_MAX]: |f|, |dx|, |x| per step
  int32_t *status = nullptr;    // sticky device status word
  uint32_t *flags = nullptr;    // [(n+1) * 8] pivot publication flags of the MGS kernel
  double *Rm = nullptr;         // mantissas of R (layout of R)
  double *Zs = nullptr;         // [(n+1) (L+1)] mantissas and exponents of 1/r_jj
  double *Xinv = nullptr;       // inverses of R's 16 x 16 diagonal blocks (blocked back substitution)
  void *cq_scratch = nullptr;   // CholeskyQR's tensor-core Gram scratch (allocated on first use)
  size_t cq_bytes = 0;
  cudaStream_t cq_side = nullptr;          // CholeskyQR's lookahead: the panels' stream
  cudaEvent_t cq_ev[2] = {nullptr, nullptr};  // and its two events (created on first use)
  double *h_norms = nullptr;    // pinned host copy of norms
  int32_t *h_status = nullptr;  // pinned host copy of status
  // what Ab, R, Rm, Zs and rinv hold: 0 nothing reusable; 1 / 2 the
  // factorisation of the last gn_newton step, integer mantissas / cascades
  int fact = 0;
  int fact_int = 0;  // that factorisation came from the integer MGS (Rm, Zs valid)
  // CUDA graph of one Newton step for a given x pointer and stream
  cudaGraphExec_t step_exec = nullptr;
  const double *graph_x = nullptr;
  cudaGraphExec_t cq_exec = nullptr;   // the mixed solver's CholeskyQR double step (L = 1)
  cudaGraphExec_t ref_exec = nullptr;  // the mixed solver's refinement step, for x at ref_x
  const double *ref_x = nullptr;
  cudaStream_t graph_stream = nullptr;
};

}  // namespace gn

struct gn_system {
  int32_t N = 0, n = 0;
  int64_t T = 0, nnz = 0;
  int32_t kmax = 0, dmax = 1, pmax = 1;
  int32_t arith = GN_ARITH_AUTO;  // gn_arith of evaluation and least squares
  int32_t *d_poly_ptr = nullptr;  // [N+1] term ranges
  int32_t *d_mono_off = nullptr;  // [T+1] occurrence offsets
  uint32_t *d_occ = nullptr;      // [nnz] (var << 8) | exp
  double *d_coef = nullptr;       // [4 limbs][2 parts][T] limb-planar coefficients
  int32_t *d_long = nullptr;      // [nlong] terms with more than 64 variables
  int64_t nlong = 0;
  // Jacobian pattern in column-major order (by column, then row)
  int64_t nz = 0;
  int32_t *d_jz_row = nullptr;  // [nz]
  int32_t *d_jz_col = nullptr;  // [nz]
  int32_t *d_jz_ptr = nullptr;  // [nz+1] into d_jz_occ
  int32_t *d_jz_occ = nullptr;  // [nnz] occurrence indices, term order within an entry
  gn::Workspace ws[5];
};

namespace gn {

gn_status workspace_get(gn_system *s, int L, Workspace **out);

// eval.cu: cascades of doubles with error-free transformations (FP64 pipe)
gn_status launch_eval(gn_system *s, int L, const double *d_x, double *d_f, int neg_f,
                      double *d_J, int64_t ldJ, cudaStream_t st);
// eval_int.cu: integer mantissas with one exponent per complex value
gn_status launch_eval_int(gn_system *s, int L, const double *d_x, double *d_f, int neg_f,
                          double *d_J, int64_t ldJ, cudaStream_t st);
// every array of one evaluation, for callers with their own layout (batches)
struct EvalArgs {
  const double *x = nullptr;  // [nvar] complex
  int64_t nvar = 0;
  int32_t pmax = 1, kmax = 0;
  double *pow = nullptr, *stage_val = nullptr, *stage_d = nullptr;
  int64_t T = 0;
  const int32_t *mono_off = nullptr;
  const uint32_t *occ = nullptr;  // (variable << 8) | exponent, variables in [0, nvar)
  const double *coef = nullptr;   // [4][2][T]
  const int32_t *long_terms = nullptr;  // terms with supports longer than 64 (one warp each)
  int64_t nlong = 0;
  int64_t nz = 0, nocc = 0;  // Jacobian entries, partials summed into them
  const int32_t *jz_row = nullptr, *jz_col = nullptr, *jz_ptr = nullptr, *jz_occ = nullptr;
  const int64_t *jz_out = nullptr;  // complex-entry offsets of the J entries (or null: col ldJ + row)
  double *J = nullptr;
  int64_t ldJ = 0;
  int64_t npoly = 0;
  const int32_t *poly_ptr = nullptr;
  double *f = nullptr;
  const int64_t *f_out = nullptr;  // complex-entry offsets of f (or null: i)
  int neg_f = 0;
  const int32_t *status = nullptr;
  int block = 128;  // CTA size of the per-term kernel (64, 128 or 256)
  // lanes per term of the integer per-term kernel: 1, 2 (the forward and
  // backward products side by side), or 0 to choose by the longest support
  // (1 up to 16 variables, 2 beyond)
  int lanes = 0;
};
gn_status launch_eval_int_raw(int L, const EvalArgs &a, cudaStream_t st);
// whether the system's arithmetic evaluates (eval_int) or solves (lstsq) on
// integer mantissas at precision L
// (supports longer than 64 variables evaluate on integer mantissas always)
inline bool eval_int(const gn_system *s, int L) {
  return s->kmax > 64 || s->arith == GN_ARITH_INT || (s->arith == GN_ARITH_AUTO && L > 1);
}
inline bool lstsq_int(const gn_system *s) { return s->arith != GN_ARITH_FP64; }
// the evaluation the system's arithmetic selects
inline gn_status launch_eval_sel(gn_system *s, int L, const double *d_x, double *d_f, int neg_f,
                                 double *d_J, int64_t ldJ, cudaStream_t st) {
  return eval_int(s, L) ? launch_eval_int(s, L, d_x, d_f, neg_f, d_J, ldJ, st)
                        : launch_eval(s, L, d_x, d_f, neg_f, d_J, ldJ, st);
}
// words of one staged complex value: 2L limbs (cascades) or 2L mantissa limbs
// and an exponent (integer evaluation)
inline size_t stage_words(int L) { return 2 * (size_t)L + 1; }

// lstsq.cu
// want_q: convert Q back to L-limb cascades (gn_lstsq); the Newton step skips it.
// d_dx NULL: factorisation only (no back substitution).
// Xinv: scratch of the blocked back substitution (NULL: one level at a time).
gn_status launch_lstsq(gn_system *s, int L, int32_t m, int32_t n, double *d_Ab, int64_t ldAb,
                       double *d_R, double *rinv, uint32_t *flags, double *Rm, double *Zs,
                       double *Xinv, double *d_dx, int32_t *d_status, cudaStream_t st, bool want_q);
// whether launch_lstsq takes the integer-mantissa path for an m x (n+1) [A b]
bool lstsq_int_path(const gn_system *s, int L, int32_t m, int32_t n);
gn_status launch_backsub_int(int L, const double *Rm, int64_t ldr, int32_t n, const double *Zs,
                             const double *rinv, double *Xinv, double *dx, int32_t *status,
                             cudaStream_t st);
// query (once) whether the cluster back substitution can be placed; never
// call during a stream capture
void backsub_prepare(int L);
// R^H w = g (cascades in and out) on the integer mantissas of R, blocked on
// a cluster (the adjoint's forward substitution); available for 32 <= n <= 1024
bool fwdsub_int_available(int L, int32_t n);
gn_status launch_fwdsub_int(int L, const double *Rm, int64_t ldr, int32_t n, const double *Zs,
                            const double *rinv, double *Xinv, const double *g, double *w,
                            int32_t *status, cudaStream_t st);
// doubles of the inverse diagonal blocks (16 x 16, one complex value with an
// exponent each: 2L+1 words) for n unknowns
inline size_t bs_inv_doubles(int32_t n, int L) {
  return (size_t)((n + 15) / 16) * 256 * (2 * (size_t)L + 1);
}
constexpr int BACKSUB_INT_MAX_N = 1024;
// CholeskyQR of [A b] (double complex, N x (n+1), leading dimension N) for the
// mixed solver: R^ (float-float in the double-complex slots of R, upper,
// leading dimension n+1; the inverses of its 32 x 32 diagonal blocks below
// the diagonal), with R = R^ D,
// D = diag(2^(s_j + 62)); the column norms and exponents s_j at rinv + n+1 and
// rinv + 2(n+1)
bool cholqr_available(const gn_system *s);
gn_status launch_cholqr(int32_t N, int32_t n, const double *A, double *R, double *rinv, void *scratch,
                        int32_t *status, cudaStream_t st, cudaStream_t side = nullptr,
                        cudaEvent_t ev_panel = nullptr, cudaEvent_t ev_trail = nullptr);
// Solves with that factor, dx double complex [n]: R dx = y (y = the factor's
// last column; refine = false), or R^H w = c then R dx = w (refine = true, c
// double complex [n]); sexp = rinv + 2(n+1)
gn_status launch_cq_solve(bool refine, int32_t n, const double *R, const double *sexp, const double *c,
                          double *dx, int32_t *status, cudaStream_t st);
// The Gram matrix G = A^H A (upper triangle, double complex, leading
// dimension nc) of A (N x nc, leading dimension N) on the tensor cores,
// exact for the columns rounded to 56 bits at their scales 2^sexp_j;
// scratch of gram_tc_scratch_bytes (digit planes and per-pair products)
bool gram_tc_available(int32_t N, int32_t nc);
size_t gram_tc_scratch_bytes(int32_t N, int32_t nc);
gn_status launch_gram_tc(int32_t N, int32_t nc, const double *A, const double *sexp, double *G, void *scratch,
                         int32_t *status, cudaStream_t st);
// R and 1/r_kk as cascades from the mantissas the MGS launch left
gn_status launch_mgs_r_out(int L, double *R, const double *Rm, int64_t ldr, int32_t ncols,
                           double *rinv, const int32_t *status, cudaStream_t st);
gn_status launch_mgs_to_cascade(int L, double *A, int32_t m, int64_t lda, int32_t ncols,
                                const double *rinv, const int32_t *status, cudaStream_t st);
// doubles of the per-solve scratch: 1/r_kk (L per column), original norms, column exponents
inline size_t lstsq_scratch_doubles(int32_t n, int L) { return (size_t)(n + 1) * (L + 2); }

// mgs.cu: MGS as one launch of thread-block clusters (0 clusters: unavailable)
int mgs_flow_clusters(int L);
// whether an m x ncols matrix fits the launch's shared-memory layout
bool mgs_flow_fits(int L, int32_t m, int32_t ncols);
gn_status launch_mgs_flow(int L, double *A, int32_t m, int64_t lda, int32_t ncols, double *R,
                          int64_t ldr, double *rinv, uint32_t *flags, int32_t *status, double *Rm,
                          double *Zs, cudaStream_t st);
constexpr int MGS_FLAGS_PER_COLUMN = 8;
// R[0:n,0:n] dx = R[0:n, n] in the cascade arithmetic (one CTA, 1/r_ll from rinv)
gn_status launch_backsub_fp64(int L, const double *R, int64_t ldr, int32_t n, const double *rinv,
                              double *dx, const int32_t *status, cudaStream_t st);
gn_status launch_update(int L, int32_t n, double *d_x, const double *d_dx, const double *d_fnorm,
                        double *d_norms, int32_t *d_status, cudaStream_t st);

}  // namespace gn
