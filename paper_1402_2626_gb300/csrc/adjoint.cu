// adjoint.cu — gradient of a real loss with respect to the coefficients at a
// root of the system, and coefficient updates on the device.
//
// The paper's Newton's method (Section 4) is the forward solve.  Its adjoint
// follows from the implicit function theorem at the Gauss-Newton fixed point:
// at a root x of f(x; c) = 0 with J of full column rank, the root moves by
// dx = -J^+ (df/dc) dc, J^+ = R^-1 Q^H for the factors J = QR of Section 3.
// For a real loss with gradient g = dL/dRe x + i dL/dIm x, the gradient with
// respect to a coefficient c_t of polynomial i is
//   grad_t = sum_j g_j conj(dx_j / dc_t) = -lambda_i conj(x^{a_t}),
//   lambda = (J^+)^H g = Q w,  R^H w = g.
// Three launches after the factorisation (evaluation and MGS are the Newton
// step's own kernels, on [J, -f] at x):
//   R^H w = g by forward substitution: blocked on R's integer mantissas
//                 (k_fwdsub_cl, with the inverse diagonal blocks) when the
//                 factorisation came from the integer MGS, else k_adj_fwdsub
//                 (one CTA, cascade arithmetic),
//   k_adj_lambda  lambda = Q w (one CTA per row),
//   k_adj_grad    grad_t = -lambda_i conj(x^{a_t}) (one thread per term).
// The arithmetic is the cascade arithmetic of mw.cuh at precision L.
#include "internal.h"
#include "mw.cuh"

namespace gn {

constexpr int ADJ_THREADS = 256;

// w_l = (g_l - sum_{j<l} conj(r_jl) w_j) / r_ll for l = 0 .. n-1, column
// oriented: once w_l is known every thread subtracts conj(r_li) w_l from its
// w_i (i > l); r_li is row l of R, entry (l, i) of the column-major factor.
// w_l itself is formed by one thread while the FP64 pipe is otherwise idle
// (a lookahead that forms w_{l+1} during the updates measured slower: its
// dependent chain then queues behind the other rows' updates).
template <int L>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_fwdsub(const double *__restrict__ R, int64_t ldr,
                                                            int32_t n, const double *__restrict__ rinv,
                                                            const double *__restrict__ g,
                                                            double *__restrict__ w,
                                                            const int32_t *__restrict__ status) {
  __shared__ cx<L> s_w;
  if (*status != GN_OK) return;
  const int64_t W = 2 * L;
  for (int i = threadIdx.x; i < n; i += blockDim.x) c_store<L>(w + i * W, c_load<L>(g + i * W));
  __syncthreads();
  for (int l = 0; l < n; l++) {
    if (threadIdx.x == 0) {
      rl<L> inv;
#pragma unroll
      for (int q = 0; q < L; q++) inv.v[q] = rinv[(int64_t)l * L + q];
      cx<L> wl = c_mul_real<L>(c_load<L>(w + l * W), inv);
      c_store<L>(w + l * W, wl);
      s_w = wl;
    }
    __syncthreads();
    const cx<L> wl = s_w;
    for (int i = l + 1 + threadIdx.x; i < n; i += blockDim.x) {
      cx<L> p = c_conj_mul<L>(c_load<L>(R + ((int64_t)i * ldr + l) * W), wl);
      c_store<L>(w + i * W, c_sub<L>(c_load<L>(w + i * W), p));
    }
    __syncthreads();
  }
}

// lambda_i = sum_l q_il w_l, one CTA per row: thread c sums l = c, c + 256,
// ... and the partial sums meet in a fixed tree, so the result does not
// depend on scheduling.
template <int L>
__global__ void __launch_bounds__(ADJ_THREADS) k_adj_lambda(const double *__restrict__ Q, int64_t ldq,
                                                            int32_t m, int32_t n,
                                                            const double *__restrict__ w,
                                                            double *__restrict__ lam,
                                                            const int32_t *__restrict__ status) {
  __shared__ cx<L> part[ADJ_THREADS];
  if (*status != GN_OK) return;
  const int64_t W = 2 * L;
  const int i = blockIdx.x;
  cx<L> acc = c_zero<L>();
  for (int l = threadIdx.x; l < n; l += ADJ_THREADS)
    acc = c_add<L>(acc, c_mul<L>(c_load<L>(Q + ((int64_t)l * ldq + i) * W), c_load<L>(w + l * W)));
  part[threadIdx.x] = acc;
  __syncthreads();
#pragma unroll
  for (int h = ADJ_THREADS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) part[threadIdx.x] = c_add<L>(part[threadIdx.x], part[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) c_store<L>(lam + i * W, part[0]);
}

// x^d by square and multiply (d >= 1)
template <int L>
__device__ cx<L> c_pow(cx<L> a, int d) {
  cx<L> r = c_one<L>();
  bool first = true;
  while (d) {
    if (d & 1) {
      r = first ? a : c_mul<L>(r, a);
      first = false;
    }
    d >>= 1;
    if (d) a = c_mul<L>(a, a);
  }
  return r;
}

// grad_t = -lambda_i conj(m_t), m_t = prod over the support of x_v^d
// (1 for a constant term); i is the polynomial of term t, found by bisection
// of the term ranges.
template <int L>
__global__ void __launch_bounds__(128) k_adj_grad(int64_t T, int32_t N, const int32_t *__restrict__ poly_ptr,
                                                  const int32_t *__restrict__ mono_off,
                                                  const uint32_t *__restrict__ occ,
                                                  const double *__restrict__ x,
                                                  const double *__restrict__ lam,
                                                  double *__restrict__ grad,
                                                  const int32_t *__restrict__ status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T || *status != GN_OK) return;
  const int64_t W = 2 * L;
  int lo = 0, hi = N - 1;  // last i with poly_ptr[i] <= t
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(poly_ptr + mid) <= t) lo = mid;
    else hi = mid - 1;
  }
  cx<L> m = c_one<L>();
  const int o1 = __ldg(mono_off + t + 1);
  for (int o = __ldg(mono_off + t); o < o1; o++) {
    uint32_t vd = __ldg(occ + o);
    m = c_mul<L>(m, c_pow<L>(c_load<L>(x + (int64_t)(vd >> 8) * W), (int)(vd & 255u)));
  }
  c_store<L>(grad + t * W, c_neg<L>(c_conj_mul<L>(m, c_load<L>(lam + (int64_t)lo * W))));
}

// Limb-planar coefficients [4][2][T] from a device cascade [T][2][cl].
__global__ void k_set_coef(int64_t T, const double *__restrict__ src, int32_t cl,
                           double *__restrict__ dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
#pragma unroll
  for (int part = 0; part < 2; part++)
#pragma unroll
    for (int l = 0; l < 4; l++)
      dst[(int64_t)(2 * l + part) * T + t] = l < cl ? src[(t * 2 + part) * cl + l] : 0.0;
}

template <int L>
static gn_status adjoint_tail(gn_system *s, Workspace *ws, const double *d_x, const double *d_g,
                              double *d_grad, double *lam, bool int_fact, cudaStream_t st) {
  const int32_t N = s->N, n = s->n;
  if (int_fact && fwdsub_int_available(L, n)) {
    // blocked on the integer mantissas of R (the diagonal blocks' inverses)
    gn_status e = launch_fwdsub_int(L, ws->Rm, n + 1, n, ws->Zs, ws->rinv, ws->Xinv, d_g, ws->dx,
                                    ws->status, st);
    if (e) return e;
  } else {
    k_adj_fwdsub<L><<<1, ADJ_THREADS, 0, st>>>(ws->R, n + 1, n, ws->rinv, d_g, ws->dx, ws->status);
  }
  k_adj_lambda<L><<<(unsigned)N, ADJ_THREADS, 0, st>>>(ws->Ab, N, N, n, ws->dx, lam, ws->status);
  if (s->T > 0)
    k_adj_grad<L><<<(unsigned)((s->T + 127) / 128), 128, 0, st>>>(
        s->T, N, s->d_poly_ptr, s->d_mono_off, s->d_occ, d_x, lam, d_grad, ws->status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

}  // namespace gn

using namespace gn;

extern "C" gn_status gn_adjoint(gn_system *s, gn_prec prec, const double *d_x, const double *d_g,
                                double *d_grad, double *d_lambda, int32_t flags, void *cuda_stream) {
  gn::Range nvtx_range("gn_adjoint");
  if (!s || (prec != 1 && prec != 2 && prec != 4) || !d_x || !d_g || (s->T > 0 && !d_grad) ||
      (flags & ~GN_ADJ_REUSE))
    return GN_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Workspace *ws;
  gn_status e = workspace_get(s, prec, &ws);
  if (e) return e;
  const int64_t W = 2 * prec;
  const int32_t N = s->N, n = s->n;
  double *lam = d_lambda ? d_lambda : ws->lam;
  const bool reuse = (flags & GN_ADJ_REUSE) != 0;
  if (reuse && ws->fact == 0) return GN_EINVAL;
  if (cudaMemsetAsync(ws->status, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return GN_ECUDA;
  if (reuse) {
    // Q and R of the last Newton step: integer mantissas to cascades
    if (ws->fact == 1) {
      e = launch_mgs_to_cascade(prec, ws->Ab, N, N, n + 1, ws->rinv, ws->status, st);
      if (!e) e = launch_mgs_r_out(prec, ws->R, ws->Rm, n + 1, n + 1, ws->rinv, ws->status, st);
    }
  } else {
    // [J, -f] at x and its factorisation, Q and R as cascades
    ws->fact = 0;
    ws->fact_int = lstsq_int_path(s, prec, N, n) ? 1 : 0;
    e = launch_eval_sel(s, prec, d_x, ws->Ab + (int64_t)n * N * W, 1, ws->Ab, N, st);
    if (!e)
      e = launch_lstsq(s, prec, N, n, ws->Ab, N, ws->R, ws->rinv, ws->flags, ws->Rm, ws->Zs, nullptr,
                       nullptr, ws->status, st, true);
  }
  if (!e) {
    switch (prec) {
      case 1: e = adjoint_tail<1>(s, ws, d_x, d_g, d_grad, lam, ws->fact_int != 0, st); break;
      case 2: e = adjoint_tail<2>(s, ws, d_x, d_g, d_grad, lam, ws->fact_int != 0, st); break;
      case 4: e = adjoint_tail<4>(s, ws, d_x, d_g, d_grad, lam, ws->fact_int != 0, st); break;
    }
  }
  if (e) return e;
  if (cudaMemcpyAsync(ws->h_status, ws->status, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GN_ECUDA;
  // Q and R are cascades now (the tail kernels leave them alone): reusable
  ws->fact = ws->h_status[0] == GN_OK ? 2 : 0;
  return (gn_status)ws->h_status[0];
}

extern "C" gn_status gn_system_set_coef(gn_system *s, const double *d_coef, int32_t coef_limbs,
                                        void *cuda_stream) {
  if (!s || (coef_limbs != 1 && coef_limbs != 2 && coef_limbs != 4) || (s->T > 0 && !d_coef))
    return GN_EINVAL;
  for (Workspace &w : s->ws) w.fact = 0;  // a factorisation of the old J
  if (s->T == 0) return GN_OK;
  k_set_coef<<<(unsigned)((s->T + 127) / 128), 128, 0, (cudaStream_t)cuda_stream>>>(
      s->T, d_coef, coef_limbs, s->d_coef);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}
