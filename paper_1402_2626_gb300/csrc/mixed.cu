// mixed.cu — Gauss-Newton with the factorisation in double precision and the
// residuals in double double or quad double.
//
// Section 5.2 of Verschelde & Yu observes that when evaluation is cheap the
// linear solve dominates a Newton step, and that iterative methods in double
// arithmetic may do well.  Here that becomes a two-phase solver:
//   1. Gauss-Newton steps (Section 4) in double precision from the leading
//      limbs of x: evaluation, MGS on [J, -f] and back substitution, each
//      step one replay of the double-precision step graph;
//   2. refinement at precision L with the last double factorisation frozen:
//      b = -f(x) evaluated at precision L (Section 2), y = Q^H b in double,
//      R dx = y by back substitution (the blocked solve on the integer
//      mantissas the double MGS left, or in double after an FP64 one),
//      x <- x + dx at precision L.
// Phase 2 converges linearly, by about kappa(J) times the unit roundoff of
// double per step, to the precision of the residuals; for a consistent
// system this is the root at precision L.  The factorisation, the cost the
// paper finds dominant, runs once per double step instead of once per step
// at precision L.
//
// With the integer arithmetic and 32 .. 1024 unknowns the double
// factorisation is CholeskyQR (cholqr.cu) instead of MGS: each double step
// is the evaluation, the exact Gram matrix of [J, -f], its Cholesky factor
// (whose last column is y = R^-H J^H (-f)), R dx = y and x += dx; each
// refinement forms c = J^H b with the frozen J, R^H w = c, then R dx = w
// (the normal equations through the Cholesky factor, kappa(J)^2 u_double
// per step, which the refinement tolerates for kappa(J)^2 u << 1).  Both
// solves run on the float-float factor itself, on one cluster (cholqr.cu).
#include <string.h>

#include "internal.h"
#include "mw.cuh"

namespace gn {

constexpr int MIX_THREADS = 256;

// leading limbs of x (precision L) into xd (double)
template <int L>
__global__ void k_mix_lead(int32_t n, const double *__restrict__ x, double *__restrict__ xd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  xd[2 * i] = x[(int64_t)i * 2 * L];
  xd[2 * i + 1] = x[(int64_t)i * 2 * L + L];
}

// a double complex vector as a cascade of precision L (lower limbs 0)
template <int L>
__global__ void k_mix_spread(int32_t n, const double *__restrict__ xd, double *__restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double *o = x + (int64_t)i * 2 * L;
#pragma unroll
  for (int l = 0; l < L; l++) {
    o[l] = l ? 0.0 : xd[2 * i];
    o[L + l] = l ? 0.0 : xd[2 * i + 1];
  }
}

// y_k = sum_i conj(q_ik) b_i in double, b = the leading limbs of -f (stored
// at precision L), into column n of R (the place of y in the factor of
// [A b]); one CTA per column k, partial sums over rows i = tid, tid + 256,
// ... added in a fixed tree.  CTA 0 also forms ||f||_2 (leading limbs).
template <int L>
__global__ void __launch_bounds__(MIX_THREADS) k_mix_qhb(const double *__restrict__ Q, int64_t ldq,
                                                         int32_t m, int32_t n,
                                                         const double *__restrict__ negf,
                                                         double *__restrict__ R, int64_t ldr,
                                                         double *__restrict__ fnorm,
                                                         const int32_t *__restrict__ status) {
  __shared__ double sre[MIX_THREADS], sim[MIX_THREADS], sf[MIX_THREADS];
  if (*status != GN_OK) return;
  const int k = blockIdx.x;
  double re = 0.0, im = 0.0, ff = 0.0;
  for (int i = threadIdx.x; i < m; i += MIX_THREADS) {
    const double qr = Q[((int64_t)k * ldq + i) * 2], qi = Q[((int64_t)k * ldq + i) * 2 + 1];
    const double br = negf[(int64_t)i * 2 * L], bi = negf[(int64_t)i * 2 * L + L];
    re = fma(qr, br, fma(qi, bi, re));
    im = fma(qr, bi, fma(-qi, br, im));
    ff = fma(br, br, fma(bi, bi, ff));
  }
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  sf[threadIdx.x] = ff;
  __syncthreads();
#pragma unroll
  for (int h = MIX_THREADS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sre[threadIdx.x] += sre[threadIdx.x + h];
      sim[threadIdx.x] += sim[threadIdx.x + h];
      sf[threadIdx.x] += sf[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    R[((int64_t)n * ldr + k) * 2] = sre[0];
    R[((int64_t)n * ldr + k) * 2 + 1] = sim[0];
    if (k == 0) *fnorm = sqrt(sf[0]);
  }
}

// c_k = sum_i conj(a_ik) b_i in double for the frozen J (column-major, ld N)
// and b = the leading limbs of -f (stored at precision L), into c; CTA 0
// also forms ||f||_2 (leading limbs).  One CTA per column k, partial sums
// over rows i = tid, tid + 256, ... added in a fixed tree.
template <int L>
__global__ void __launch_bounds__(MIX_THREADS) k_mix_ahb(const double *__restrict__ A, int64_t lda,
                                                         int32_t m, const double *__restrict__ negf,
                                                         double *__restrict__ c, double *__restrict__ fnorm,
                                                         const int32_t *__restrict__ status) {
  __shared__ double sre[MIX_THREADS], sim[MIX_THREADS], sf[MIX_THREADS];
  if (*status != GN_OK) return;
  const int k = blockIdx.x;
  double re = 0.0, im = 0.0, ff = 0.0;
  for (int i = threadIdx.x; i < m; i += MIX_THREADS) {
    const double ar = A[((int64_t)k * lda + i) * 2], ai = A[((int64_t)k * lda + i) * 2 + 1];
    const double br = negf[(int64_t)i * 2 * L], bi = negf[(int64_t)i * 2 * L + L];
    re = fma(ar, br, fma(ai, bi, re));
    im = fma(ar, bi, fma(-ai, br, im));
    ff = fma(br, br, fma(bi, bi, ff));
  }
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  sf[threadIdx.x] = ff;
  __syncthreads();
#pragma unroll
  for (int h = MIX_THREADS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      sre[threadIdx.x] += sre[threadIdx.x + h];
      sim[threadIdx.x] += sim[threadIdx.x + h];
      sf[threadIdx.x] += sf[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    c[2 * k] = sre[0];
    c[2 * k + 1] = sim[0];
    if (k == 0) *fnorm = sqrt(sf[0]);
  }
}

// y (double complex, y_i at y + 2 i: column n of the cascade R, or a
// vector) into column n of the mantissas Rm as one-limb fixed point at a
// common scale 2^sig, |y| / 2^sig < 2^61 (the format MGS leaves its last
// column in), sig into sexp[n]; one CTA.
__global__ void __launch_bounds__(MIX_THREADS) k_mix_y_fixed(const double *__restrict__ yv,
                                                            double *__restrict__ Rm, int64_t ldr,
                                                            int32_t n, double *__restrict__ sexp,
                                                            const int32_t *__restrict__ status) {
  __shared__ double smax[MIX_THREADS];
  if (*status != GN_OK) return;
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += MIX_THREADS) {
    const double *y = yv + 2 * (int64_t)i;
    m = fmax(m, fmax(fabs(y[0]), fabs(y[1])));
  }
  smax[threadIdx.x] = m;
  __syncthreads();
  for (int h = MIX_THREADS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + h]);
    __syncthreads();
  }
  int e = 0;
  if (smax[0] > 0.0) frexp(smax[0], &e);  // max |y| < 2^e
  const int sig = e - 61;
  for (int i = threadIdx.x; i < n; i += MIX_THREADS) {
    const double *y = yv + 2 * (int64_t)i;
    long long *d = (long long *)(Rm + ((int64_t)n * ldr + i) * 2);
    d[0] = llrint(ldexp(y[0], -sig));
    d[1] = llrint(ldexp(y[1], -sig));
  }
  if (threadIdx.x == 0) sexp[n] = (double)sig;
}

template <int L>
static gn_status refine_step(gn_system *s, Workspace *w1, Workspace *wL, double *d_x, bool int_fact,
                             cudaStream_t st) {
  const int32_t N = s->N, n = s->n;
  const int64_t W = 2 * L;
  double *negf = wL->Ab + (int64_t)n * N * W;
  double *fnorm = wL->rinv;  // the refinement factors nothing at precision L
  gn_status e = launch_eval_sel(s, L, d_x, negf, 1, nullptr, N, st);
  if (e) return e;
  k_mix_qhb<L><<<(unsigned)n, MIX_THREADS, 0, st>>>(w1->Ab, N, N, n, negf, w1->R, n + 1, fnorm,
                                                    wL->status);
  if (int_fact && n <= BACKSUB_INT_MAX_N) {
    // the integer factors of the last double step are still in place: the
    // blocked back substitution on them
    double *sexp = w1->rinv + 2 * (size_t)(n + 1);
    k_mix_y_fixed<<<1, MIX_THREADS, 0, st>>>(w1->R + (int64_t)n * (n + 1) * 2, w1->Rm, n + 1, n, sexp,
                                             wL->status);
    e = launch_backsub_int(1, w1->Rm, n + 1, n, w1->Zs, w1->rinv, w1->Xinv, w1->dx, wL->status, st);
  } else {
    e = launch_backsub_fp64(1, w1->R, n + 1, n, w1->rinv, w1->dx, wL->status, st);
  }
  if (e) return e;
  k_mix_spread<L><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, w1->dx, wL->dx);
  return launch_update(L, n, d_x, wL->dx, fnorm, wL->norms, wL->status, st);
}

// One refinement step with the frozen CholeskyQR factors of the last double
// step (cholqr.cu): b = -f(x) at precision L, c = J^H b, R^H w = c, R dx = w
// (both substitutions in one launch on the float-float factor), x += dx at
// precision L.
template <int L>
static gn_status refine_step_cq(gn_system *s, Workspace *w1, Workspace *wL, double *d_x, cudaStream_t st) {
  const int32_t N = s->N, n = s->n;
  const int64_t W = 2 * L;
  double *negf = wL->Ab + (int64_t)n * N * W;
  double *fnorm = wL->rinv;
  double *c = w1->lam;  // [n] double complex (lam holds N >= n entries)
  const double *sexp = w1->rinv + 2 * (size_t)(n + 1);
  gn_status e = launch_eval_sel(s, L, d_x, negf, 1, nullptr, N, st);
  if (e) return e;
  k_mix_ahb<L><<<(unsigned)n, MIX_THREADS, 0, st>>>(w1->Ab, N, N, negf, c, fnorm, wL->status);
  e = launch_cq_solve(true, n, w1->R, sexp, c, w1->dx, wL->status, st);
  if (e) return e;
  k_mix_spread<L><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, w1->dx, wL->dx);
  return launch_update(L, n, d_x, wL->dx, fnorm, wL->norms, wL->status, st);
}

// d_steps Gauss-Newton steps in double on w1->xmix with CholeskyQR
// factorisations: evaluation into [J, -f], the factor R of [J, -f] (its last
// column is y), R dx = y, x += dx; the factors of the last step stay in w1.
// A CUDA graph of the work fn(stream) enqueues (its launches, and any side
// stream it forks from that stream and joins back), instantiated into *exec;
// on failure *exec stays null and the caller launches directly.
template <class F>
static void capture_graph(cudaGraphExec_t *exec, F &&fn) {
  *exec = nullptr;
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    ok = fn(cap) == GN_OK;
    ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && ok;
  }
  if (ok && cudaGraphInstantiate(exec, g, 0) != cudaSuccess) {
    ok = false;
    *exec = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (!ok) cudaGetLastError();
}

static gn_status cholqr_steps(gn_system *s, Workspace *w1, int32_t d_steps, gn_report *r1,
                              cudaStream_t st) {
  const int32_t N = s->N, n = s->n;
  w1->fact = 0;
  if (cudaMemsetAsync(w1->status, 0, sizeof(int32_t) * 2, st) != cudaSuccess ||
      cudaMemsetAsync(w1->norms, 0, sizeof(double) * 3 * GN_REPORT_MAX, st) != cudaSuccess)
    return GN_ECUDA;
  const double *fnorm = w1->rinv + (n + 1) + n;  // ||b|| = ||f||: the b column's norm
  // scratch of the tensor-core Gram matrix, kept with the workspace; without
  // it (no memory) the Gram matrix is formed on the integer pipe
  if (gram_tc_available(N, n + 1) && !w1->cq_scratch) {
    const size_t need = gram_tc_scratch_bytes(N, n + 1);
    if (cudaMalloc(&w1->cq_scratch, need) == cudaSuccess) {
      w1->cq_bytes = need;
    } else {
      cudaGetLastError();
      w1->cq_scratch = nullptr;
    }
  }
  // the Cholesky's lookahead stream (at the highest priority) and events,
  // kept with the workspace; without them the panels run on st alone
  if (!w1->cq_side) {
    cudaStream_t side = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
        cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, hi) == cudaSuccess &&
        cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming) == cudaSuccess) {
      w1->cq_side = side;
      w1->cq_ev[0] = ev[0];
      w1->cq_ev[1] = ev[1];
    } else {
      if (ev[0]) cudaEventDestroy(ev[0]);
      if (side) cudaStreamDestroy(side);
      cudaGetLastError();
    }
  }
  // one double step; captured once as a graph (its pointers are the
  // workspace's), so the host does not pace the chain of panel launches
  auto step = [&](cudaStream_t cs) {
    gn_status e = launch_eval_sel(s, 1, w1->xmix, w1->Ab + (int64_t)n * N * 2, 1, w1->Ab, N, cs);
    if (!e)
      e = launch_cholqr(N, n, w1->Ab, w1->R, w1->rinv, w1->cq_scratch, w1->status, cs, w1->cq_side,
                        w1->cq_ev[0], w1->cq_ev[1]);
    if (!e) e = launch_cq_solve(false, n, w1->R, w1->rinv + 2 * (size_t)(n + 1), nullptr, w1->dx, w1->status, cs);
    if (!e) e = launch_update(1, n, w1->xmix, w1->dx, fnorm, w1->norms, w1->status, cs);
    return e;
  };
  if (!w1->cq_exec) capture_graph(&w1->cq_exec, step);
  for (int32_t k = 0; k < d_steps; k++) {
    const gn_status e = w1->cq_exec ? (cudaGraphLaunch(w1->cq_exec, st) == cudaSuccess ? GN_OK : GN_ECUDA)
                                    : step(st);
    if (e) return e;
  }
  if (cudaMemcpyAsync(w1->h_status, w1->status, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(w1->h_norms, w1->norms, sizeof(double) * 3 * GN_REPORT_MAX, cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GN_ECUDA;
  memset(r1, 0, sizeof(*r1));
  r1->status = w1->h_status[0];
  r1->steps_done = w1->h_status[1];
  for (int32_t k = 0; k < r1->steps_done && k < GN_REPORT_MAX; k++) {
    r1->res_norm[k] = w1->h_norms[3 * k];
    r1->dx_norm[k] = w1->h_norms[3 * k + 1];
  }
  return (gn_status)w1->h_status[0];
}

}  // namespace gn

using namespace gn;

extern "C" gn_status gn_newton_mixed(gn_system *s, gn_prec prec, double *d_x, int32_t d_steps,
                                     int32_t refine_steps, double tol, gn_report *report,
                                     void *cuda_stream) {
  gn::Range nvtx_range("gn_newton_mixed");
  if (!s || (prec != GN_DD && prec != GN_QD) || !d_x || d_steps < 1 || refine_steps < 0 ||
      d_steps + refine_steps > GN_REPORT_MAX || !(tol >= 0.0))
    return GN_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int L = prec;
  const int32_t n = s->n;
  Workspace *w1, *wL;
  gn_status e = workspace_get(s, 1, &w1);
  if (!e) e = workspace_get(s, L, &wL);
  if (e) return e;
  if (report) memset(report, 0, sizeof(*report));
  const unsigned nb = (unsigned)((n + 127) / 128);
  // phase 1: double-precision Gauss-Newton on the leading limbs
  switch (L) {
    case 2: k_mix_lead<2><<<nb, 128, 0, st>>>(n, d_x, w1->xmix); break;
    case 4: k_mix_lead<4><<<nb, 128, 0, st>>>(n, d_x, w1->xmix); break;
  }
  if (cudaPeekAtLastError() != cudaSuccess) return GN_ECUDA;
  gn_report r1;
  const bool cq = cholqr_available(s);
  e = cq ? cholqr_steps(s, w1, d_steps, &r1, st) : gn_newton(s, GN_D, w1->xmix, d_steps, 0.0, &r1, cuda_stream);
  if (report) {
    report->steps_done = r1.steps_done;
    for (int k = 0; k < r1.steps_done; k++) {
      report->res_norm[k] = r1.res_norm[k];
      report->dx_norm[k] = r1.dx_norm[k];
    }
    report->status = e;
  }
  if (e) return e;
  // the last step's factors as doubles (MGS), or in place (CholeskyQR)
  const bool int_fact = w1->fact == 1;
  if (!cq && w1->fact == 1) {
    e = launch_mgs_to_cascade(1, w1->Ab, s->N, s->N, n + 1, w1->rinv, w1->status, st);
    if (!e) e = launch_mgs_r_out(1, w1->R, w1->Rm, n + 1, n + 1, w1->rinv, w1->status, st);
    if (e) return e;
    w1->fact = 2;
  }
  if (!cq && w1->fact != 2) return GN_EINVAL;
  switch (L) {
    case 2: k_mix_spread<2><<<nb, 128, 0, st>>>(n, w1->xmix, d_x); break;
    case 4: k_mix_spread<4><<<nb, 128, 0, st>>>(n, w1->xmix, d_x); break;
  }
  // phase 2: refinement with frozen factors
  wL->fact = 0;
  if (cudaMemsetAsync(wL->status, 0, sizeof(int32_t) * 2, st) != cudaSuccess ||
      cudaMemsetAsync(wL->norms, 0, sizeof(double) * 3 * GN_REPORT_MAX, st) != cudaSuccess)
    return GN_ECUDA;
  bool converged = false;
  // the refinement step with CholeskyQR factors, captured once per x as a graph
  auto rstep = [&](cudaStream_t cs) {
    return L == 2 ? refine_step_cq<2>(s, w1, wL, d_x, cs) : refine_step_cq<4>(s, w1, wL, d_x, cs);
  };
  if (cq && refine_steps > 0 && (!wL->ref_exec || wL->ref_x != d_x)) {
    if (wL->ref_exec) cudaGraphExecDestroy(wL->ref_exec);
    capture_graph(&wL->ref_exec, rstep);
    wL->ref_x = wL->ref_exec ? d_x : nullptr;
  }
  for (int32_t k = 0; k < refine_steps; k++) {
    if (cq)
      e = wL->ref_exec ? (cudaGraphLaunch(wL->ref_exec, st) == cudaSuccess ? GN_OK : GN_ECUDA) : rstep(st);
    else
      e = L == 2 ? refine_step<2>(s, w1, wL, d_x, int_fact, st) : refine_step<4>(s, w1, wL, d_x, int_fact, st);
    if (e) return e;
    if (tol > 0.0) {
      if (cudaMemcpyAsync(wL->h_status, wL->status, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaMemcpyAsync(wL->h_norms, wL->norms, sizeof(double) * 3 * GN_REPORT_MAX,
                          cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return GN_ECUDA;
      if (wL->h_status[0] != GN_OK) break;
      if (wL->h_norms[3 * k + 1] <= tol * wL->h_norms[3 * k + 2]) {
        converged = true;
        break;
      }
    }
  }
  if (cudaMemcpyAsync(wL->h_status, wL->status, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(wL->h_norms, wL->norms, sizeof(double) * 3 * GN_REPORT_MAX,
                      cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GN_ECUDA;
  gn_status run = (gn_status)wL->h_status[0];
  const int32_t done = wL->h_status[1];
  if (run == GN_OK && tol > 0.0 && !converged && refine_steps > 0) run = GN_ENOCONV;
  if (report) {
    report->status = run;
    for (int32_t k = 0; k < done && r1.steps_done + k < GN_REPORT_MAX; k++) {
      report->res_norm[r1.steps_done + k] = wL->h_norms[3 * k];
      report->dx_norm[r1.steps_done + k] = wL->h_norms[3 * k + 1];
    }
    report->steps_done = r1.steps_done + done;
  }
  return run;
}
