// lstsq.cu — least squares by modified Gram-Schmidt on [A b] and back
// substitution (Section 3 of Verschelde & Yu), and the Newton update
// x <- x + dx (Section 4).
//
// MGS follows the figure "The modified Gram-Schmidt orthogonalization
// algorithm" (right-looking): for each pivot k, one CTA forms
// r_kk = sqrt(a_k^H a_k) and q_k = a_k / r_kk, then one CTA per trailing
// column j forms r_kj = q_k^H a_j and a_j <- a_j - r_kj q_k.  The right-hand
// side b rides along as the last column (eq. 2), which gives y = Q^H b in
// R[0:n, n] and z in R[n][n]; b itself is not normalised.  Inner products are
// summed by a fixed tree inside the CTA, so results are reproducible.
//
// The K20C version delayed each normalisation by one step because blocks of
// one launch could read a half-normalised pivot; here the normalisation and
// the updates are separate launches in stream (or CUDA-graph) order, so the
// same arithmetic runs without that device.
#include <math.h>

#include "internal.h"
#include "mw.cuh"

namespace gn {

constexpr int MGS_THREADS = 256;

template <int L>
__device__ __forceinline__ cx<L> shfl_xor_c(const cx<L> &a, int m) {
  cx<L> r;
#pragma unroll
  for (int l = 0; l < L; l++) {
    r.re[l] = __shfl_xor_sync(0xffffffffu, a.re[l], m);
    r.im[l] = __shfl_xor_sync(0xffffffffu, a.im[l], m);
  }
  return r;
}

// Deterministic CTA-wide sum (butterfly in each warp, then warp 0 sums the
// warp partials).  Every thread gets the result.
template <int L>
__device__ cx<L> block_sum(cx<L> v, cx<L> *sh /* >= 32 entries */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = c_add<L>(v, shfl_xor_c<L>(v, m));
  __syncthreads();  // sh may still be read by a previous call
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    cx<L> w = lane < nw ? sh[lane] : c_zero<L>();
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) w = c_add<L>(w, shfl_xor_c<L>(w, m));
    if (lane == 0) sh[0] = w;
  }
  __syncthreads();
  return sh[0];
}

// Double estimates of the original column norms, for the rank test.
template <int L>
__global__ void k_colnorms(const double *__restrict__ A, int32_t m, int64_t lda, int32_t ncols,
                           double *__restrict__ nrm0, int32_t *__restrict__ status) {
  int j = blockIdx.x;
  if (j >= ncols) return;
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double *a = A + ((int64_t)j * lda + i) * 2 * L;
    s = fma(a[0], a[0], fma(a[L], a[L], s));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); w++) t += sh[w];
    nrm0[j] = sqrt(t);
    // a NaN or an infinity in the column, reported before any pivot runs
    if (!isfinite(t)) atomicCAS(status, GN_OK, GN_ENONFINITE);
  }
}

// Pivot k: r_kk = sqrt(a_k^H a_k); for k < ncols-1 test the rank and
// normalise a_k in place; for the last column store z = r_nn only.
template <int L>
__global__ void __launch_bounds__(MGS_THREADS) k_mgs_pivot(double *__restrict__ A, int32_t m,
                                                           int64_t lda, int32_t ncols, int32_t k,
                                                           double *__restrict__ R, int64_t ldr,
                                                           double *__restrict__ rinv,
                                                           const double *__restrict__ nrm0,
                                                           int32_t *__restrict__ status) {
  __shared__ cx<L> sh[32];
  __shared__ rl<L> s_inv;
  __shared__ int s_ok;
  if (*status != GN_OK) return;
  const int64_t W = 2 * L;
  double *ak = A + (int64_t)k * lda * W;
  cx<L> acc = c_zero<L>();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    rl<L> p = c_abs2<L>(c_load<L>(ak + i * W));
    cx<L> pc = c_zero<L>();
#pragma unroll
    for (int l = 0; l < L; l++) pc.re[l] = p.v[l];
    acc = c_add<L>(acc, pc);
  }
  cx<L> tot = block_sum<L>(acc, sh);
  if (threadIdx.x == 0) {
    rl<L> ss;
#pragma unroll
    for (int l = 0; l < L; l++) ss.v[l] = tot.re[l];
    rl<L> r = r_sqrt<L>(ss);
    cx<L> rc = c_zero<L>();
#pragma unroll
    for (int l = 0; l < L; l++) rc.re[l] = r.v[l];
    c_store<L>(R + ((int64_t)k * ldr + k) * W, rc);
    int ok = 1;
    if (!isfinite(ss.v[0]) || !isfinite(r.v[0])) {
      ok = 0;
      atomicCAS(status, GN_OK, GN_ENONFINITE);
    } else if (k < ncols - 1) {
      double thresh = ldexp(nrm0[k], 8 - 50 * L);
      if (!(r.v[0] > thresh)) {
        ok = 0;
        atomicCAS(status, GN_OK, GN_ESINGULAR);
      } else {
        s_inv = r_recip<L>(r);
#pragma unroll
        for (int l = 0; l < L; l++) rinv[(int64_t)k * L + l] = s_inv.v[l];
      }
    } else {
      ok = 0;  // b is not normalised
    }
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return;
  rl<L> inv = s_inv;
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    c_store<L>(ak + i * W, c_mul_real<L>(c_load<L>(ak + i * W), inv));
}

// Trailing update for pivot k: CTA b handles column j = k + 1 + b.
template <int L>
__global__ void __launch_bounds__(MGS_THREADS) k_mgs_update(double *__restrict__ A, int32_t m,
                                                            int64_t lda, int32_t ncols, int32_t k,
                                                            double *__restrict__ R, int64_t ldr,
                                                            const int32_t *__restrict__ status) {
  __shared__ cx<L> sh[32];
  if (*status != GN_OK) return;
  const int j = k + 1 + blockIdx.x;
  if (j >= ncols) return;
  const int64_t W = 2 * L;
  const double *qk = A + (int64_t)k * lda * W;
  double *aj = A + (int64_t)j * lda * W;
  cx<L> acc = c_zero<L>();
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    acc = c_add<L>(acc, c_conj_mul<L>(c_load<L>(qk + i * W), c_load<L>(aj + i * W)));
  cx<L> r = block_sum<L>(acc, sh);
  if (threadIdx.x == 0) c_store<L>(R + ((int64_t)j * ldr + k) * W, r);
  cx<L> nr = c_neg<L>(r);
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    c_store<L>(aj + i * W, c_add<L>(c_load<L>(aj + i * W), c_mul<L>(nr, c_load<L>(qk + i * W))));
}

// Back substitution R[0:n,0:n] dx = y, y = R[0:n, n]:
//   dx_l = (y_l - sum_{j>l} r_lj dx_j) / r_ll, l = n-1 .. 0,
// column-oriented in one CTA: after dx_l is known every thread subtracts
// r_il dx_l from its y_i (i < l).  y is kept in dx.
template <int L>
__global__ void __launch_bounds__(MGS_THREADS) k_backsub(const double *__restrict__ R, int64_t ldr,
                                                         int32_t n, const double *__restrict__ rinv,
                                                         double *__restrict__ dx,
                                                         const int32_t *__restrict__ status) {
  __shared__ cx<L> s_x;
  if (*status != GN_OK) return;
  const int64_t W = 2 * L;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    c_store<L>(dx + i * W, c_load<L>(R + ((int64_t)n * ldr + i) * W));
  __syncthreads();
  for (int l = n - 1; l >= 0; l--) {
    if (threadIdx.x == 0) {
      rl<L> inv;
#pragma unroll
      for (int q = 0; q < L; q++) inv.v[q] = rinv[(int64_t)l * L + q];
      cx<L> xl = c_mul_real<L>(c_load<L>(dx + l * W), inv);
      c_store<L>(dx + l * W, xl);
      s_x = xl;
    }
    __syncthreads();
    cx<L> nx = c_neg<L>(s_x);
    for (int i = threadIdx.x; i < l; i += blockDim.x)
      c_store<L>(dx + i * W,
                 c_add<L>(c_load<L>(dx + i * W),
                          c_mul<L>(nx, c_load<L>(R + ((int64_t)l * ldr + i) * W))));
    __syncthreads();
  }
}

// x <- x + dx (Section 4); records ||f|| (the original norm of the b = -f
// column, taken before MGS overwrote it), ||dx|| and ||x|| in double for the
// report, flags non-finite values and counts applied steps (status[1]).
template <int L>
__global__ void __launch_bounds__(MGS_THREADS) k_update(int32_t n, double *__restrict__ x,
                                                        const double *__restrict__ dx,
                                                        const double *__restrict__ fnorm,
                                                        double *__restrict__ norms,
                                                        int32_t *__restrict__ status) {
  __shared__ double sh[2][32];
  if (*status != GN_OK) return;
  const int64_t W = 2 * L;
  double sx = 0.0, sd = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    cx<L> d = c_load<L>(dx + i * W);
    sd = fma(d.re[0], d.re[0], fma(d.im[0], d.im[0], sd));
    cx<L> xn = c_add<L>(c_load<L>(x + i * W), d);
    sx = fma(xn.re[0], xn.re[0], fma(xn.im[0], xn.im[0], sx));
    c_store<L>(x + i * W, xn);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sd += __shfl_xor_sync(0xffffffffu, sd, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = sx;
    sh[1][threadIdx.x >> 5] = sd;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); w++) {
      a += sh[0][w];
      b += sh[1][w];
    }
    int step = status[1];
    if (step >= 0 && step < GN_REPORT_MAX) {
      norms[3 * step + 0] = *fnorm;
      norms[3 * step + 1] = sqrt(b);
      norms[3 * step + 2] = sqrt(a);
    }
    if (!isfinite(a) || !isfinite(b))
      atomicCAS(status, GN_OK, GN_ENONFINITE);
    else
      status[1] = step + 1;
  }
}

template <int L>
static gn_status lstsq_impl(bool use_int, int32_t m, int32_t n, double *A, int64_t lda, double *R,
                            double *rinv, double *nrm0, uint32_t *flags, double *Rm, double *Zs,
                            double *Xinv, double *dx, int32_t *status, cudaStream_t st, bool want_q) {
  const int32_t ncols = n + 1;
  const int64_t ldr = ncols;
  if (use_int && flags && Rm && Zs && mgs_flow_clusters(L) > 0 && mgs_flow_fits(L, m, ncols)) {
    const bool int_bs = dx && n <= BACKSUB_INT_MAX_N;
    gn_status e = launch_mgs_flow(L, A, m, lda, ncols, R, ldr, rinv, flags, status, Rm, Zs, st);
    if (e) return e;
    if (want_q) {
      e = launch_mgs_to_cascade(L, A, m, lda, ncols, rinv, status, st);
      if (e) return e;
    }
    // R as cascades: for the caller, or for the FP64 back substitution
    if (want_q || (dx && !int_bs)) {
      e = launch_mgs_r_out(L, R, Rm, ldr, ncols, rinv, status, st);
      if (e) return e;
    }
    if (!dx) return GN_OK;
    if (int_bs) return launch_backsub_int(L, Rm, ldr, n, Zs, rinv, Xinv, dx, status, st);
    k_backsub<L><<<1, MGS_THREADS, 0, st>>>(R, ldr, n, rinv, dx, status);
    return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
  }
  if (cudaMemsetAsync(R, 0, sizeof(double) * 2 * L * ldr * ncols, st) != cudaSuccess) return GN_ECUDA;
  // one launch per pivot and one per trailing update (devices without clusters)
  k_colnorms<L><<<ncols, 128, 0, st>>>(A, m, lda, ncols, nrm0, status);
  for (int k = 0; k < ncols; k++) {
    k_mgs_pivot<L><<<1, MGS_THREADS, 0, st>>>(A, m, lda, ncols, k, R, ldr, rinv, nrm0, status);
    if (k < ncols - 1)
      k_mgs_update<L><<<ncols - 1 - k, MGS_THREADS, 0, st>>>(A, m, lda, ncols, k, R, ldr, status);
  }
  if (dx) k_backsub<L><<<1, MGS_THREADS, 0, st>>>(R, ldr, n, rinv, dx, status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

bool lstsq_int_path(const gn_system *s, int L, int32_t m, int32_t n) {
  return lstsq_int(s) && mgs_flow_clusters(L) > 0 && mgs_flow_fits(L, m, n + 1);
}

gn_status launch_lstsq(gn_system *s, int L, int32_t m, int32_t n, double *d_Ab, int64_t ldAb,
                       double *d_R, double *rinv, uint32_t *flags, double *Rm, double *Zs,
                       double *Xinv, double *d_dx, int32_t *d_status, cudaStream_t st, bool want_q) {
  double *nrm0 = rinv + (int64_t)(n + 1) * L;
  const bool ui = lstsq_int(s);
  switch (L) {
    case 1: return lstsq_impl<1>(ui, m, n, d_Ab, ldAb, d_R, rinv, nrm0, flags, Rm, Zs, Xinv, d_dx, d_status, st, want_q);
    case 2: return lstsq_impl<2>(ui, m, n, d_Ab, ldAb, d_R, rinv, nrm0, flags, Rm, Zs, Xinv, d_dx, d_status, st, want_q);
    case 4: return lstsq_impl<4>(ui, m, n, d_Ab, ldAb, d_R, rinv, nrm0, flags, Rm, Zs, Xinv, d_dx, d_status, st, want_q);
  }
  return GN_EINVAL;
}

gn_status launch_backsub_fp64(int L, const double *R, int64_t ldr, int32_t n, const double *rinv,
                              double *dx, const int32_t *status, cudaStream_t st) {
  switch (L) {
    case 1: k_backsub<1><<<1, MGS_THREADS, 0, st>>>(R, ldr, n, rinv, dx, status); break;
    case 2: k_backsub<2><<<1, MGS_THREADS, 0, st>>>(R, ldr, n, rinv, dx, status); break;
    case 4: k_backsub<4><<<1, MGS_THREADS, 0, st>>>(R, ldr, n, rinv, dx, status); break;
    default: return GN_EINVAL;
  }
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

gn_status launch_update(int L, int32_t n, double *d_x, const double *d_dx, const double *d_fnorm,
                        double *d_norms, int32_t *d_status, cudaStream_t st) {
  switch (L) {
    case 1: k_update<1><<<1, MGS_THREADS, 0, st>>>(n, d_x, d_dx, d_fnorm, d_norms, d_status); break;
    case 2: k_update<2><<<1, MGS_THREADS, 0, st>>>(n, d_x, d_dx, d_fnorm, d_norms, d_status); break;
    case 4: k_update<4><<<1, MGS_THREADS, 0, st>>>(n, d_x, d_dx, d_fnorm, d_norms, d_status); break;
    default: return GN_EINVAL;
  }
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

}  // namespace gn
