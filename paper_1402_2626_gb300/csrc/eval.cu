// eval.cu — evaluation and differentiation of a sparse polynomial system
// (Section 2 of Verschelde & Yu): table of pure powers (Section 2.1), common
// factor (eq. 1), Speelpenning product and gradient (Section 2.2),
// coefficient x common factor x exponent and term sums (Section 2.3).
//
// GB300 design (FP64-issue bound for DD and QD):
//   * one thread per monomial.  The sequential reverse mode costs 3k + l - 3
//     complex multiplications for k variables of which l have exponent >= 2
//     (the coefficient and common factor are folded into the forward
//     products), the fewest of any schedule; a warp-level tree would do
//     O(k log k) work on a pipe that has none to spare;
//   * terms and partials are staged per occurrence, then summed by their
//     owner (one thread per Jacobian entry, one warp per polynomial) in term
//     order: no atomics (multiword values have none) and bitwise
//     reproducible results.
#include <mutex>

#include "internal.h"
#include "mw.cuh"

namespace gn {

constexpr int KMAX = 64;  // longest support handled with a local forward-product stack

// x^p for p = 1..pmax, plane p-1 of pow; one thread per variable.
template <int L>
__global__ void k_powers(const double *__restrict__ x, int32_t n, int32_t pmax,
                         double *__restrict__ pow, const int32_t *__restrict__ status) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n || *status != GN_OK) return;
  const int64_t W = 2 * L;
  cx<L> xv = c_load<L>(x + v * W);
  cx<L> p = xv;
  c_store<L>(pow + (int64_t)v * W, p);
  for (int q = 1; q < pmax; q++) {
    p = c_mul<L>(p, xv);
    c_store<L>(pow + ((int64_t)q * n + v) * W, p);
  }
}

template <int L>
__device__ __forceinline__ cx<L> load_coef(const double *__restrict__ coef, int64_t T, int64_t t) {
  cx<L> c;
#pragma unroll
  for (int l = 0; l < L; l++) {
    c.re[l] = __ldg(coef + (int64_t)(2 * l + 0) * T + t);
    c.im[l] = __ldg(coef + (int64_t)(2 * l + 1) * T + t);
  }
  return c;
}

// Phase 1: one thread per monomial t.
//   a = c * prod_{d_s >= 2} x_{v_s}^{d_s - 1}           (common factor, eq. 1)
//   F_s = a * x_{v_0} ... x_{v_{s-1}}, s = 0..k-1        (forward products)
//   value = F_{k-1} * x_{v_{k-1}}
//   partial_s = d_s * F_s * (x_{v_{s+1}} ... x_{v_{k-1}}) (one running backward product)
template <int L>
__global__ void __launch_bounds__(128) k_monomials(
    const int32_t *__restrict__ mono_off, const uint32_t *__restrict__ occ,
    const double *__restrict__ coef, int64_t T, const double *__restrict__ pow, int32_t n,
    double *__restrict__ stage_val, double *__restrict__ stage_d,
    const int32_t *__restrict__ status) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T || *status != GN_OK) return;
  const int64_t W = 2 * L;
  const int o0 = __ldg(mono_off + t);
  const int k = __ldg(mono_off + t + 1) - o0;
  cx<L> a = load_coef<L>(coef, T, t);
  for (int s = 0; s < k; s++) {
    uint32_t w = __ldg(occ + o0 + s);
    int d = (int)(w & 255u);
    if (d >= 2) {
      int v = (int)(w >> 8);
      a = c_mul<L>(a, c_load<L>(pow + ((int64_t)(d - 2) * n + v) * W));
    }
  }
  if (k == 0) {
    c_store<L>(stage_val + t * W, a);
    return;
  }
  cx<L> F[KMAX];
  F[0] = a;
  for (int s = 1; s < k; s++) {
    int v = (int)(__ldg(occ + o0 + s - 1) >> 8);
    F[s] = c_mul<L>(F[s - 1], c_load<L>(pow + (int64_t)v * W));
  }
  uint32_t wl = __ldg(occ + o0 + k - 1);
  cx<L> B = c_load<L>(pow + (int64_t)(wl >> 8) * W);
  c_store<L>(stage_val + t * W, c_mul<L>(F[k - 1], B));
  c_store<L>(stage_d + (int64_t)(o0 + k - 1) * W, c_scale_int<L>(F[k - 1], (int)(wl & 255u)));
  for (int s = k - 2; s >= 0; s--) {
    uint32_t w = __ldg(occ + o0 + s);
    cx<L> p = c_mul<L>(F[s], B);
    c_store<L>(stage_d + (int64_t)(o0 + s) * W, c_scale_int<L>(p, (int)(w & 255u)));
    if (s > 0) B = c_mul<L>(B, c_load<L>(pow + (int64_t)(w >> 8) * W));
  }
}

// Phase 2a: J entries, one thread per structural nonzero (column-major order),
// contributions summed in term order.
template <int L>
__global__ void k_sum_jacobian(int64_t nz, const int32_t *__restrict__ jz_row,
                               const int32_t *__restrict__ jz_col,
                               const int32_t *__restrict__ jz_ptr,
                               const int32_t *__restrict__ jz_occ,
                               const double *__restrict__ stage_d, double *__restrict__ J,
                               int64_t ldJ, const int32_t *__restrict__ status) {
  int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz || *status != GN_OK) return;
  const int64_t W = 2 * L;
  int p0 = __ldg(jz_ptr + z), p1 = __ldg(jz_ptr + z + 1);
  cx<L> acc = c_load<L>(stage_d + (int64_t)__ldg(jz_occ + p0) * W);
  for (int p = p0 + 1; p < p1; p++) acc = c_add<L>(acc, c_load<L>(stage_d + (int64_t)__ldg(jz_occ + p) * W));
  c_store<L>(J + ((int64_t)__ldg(jz_col + z) * ldJ + __ldg(jz_row + z)) * W, acc);
}

template <int L>
__device__ __forceinline__ cx<L> shfl_down(const cx<L> &a, int off) {
  cx<L> r;
#pragma unroll
  for (int l = 0; l < L; l++) {
    r.re[l] = __shfl_down_sync(0xffffffffu, a.re[l], off);
    r.im[l] = __shfl_down_sync(0xffffffffu, a.im[l], off);
  }
  return r;
}

// Phase 2b: f_i, one warp per polynomial; lane-strided partial sums, then a
// fixed shuffle tree.  neg = 1 stores -f (the right-hand side b of Section 4).
template <int L>
__global__ void k_sum_f(int32_t N, const int32_t *__restrict__ poly_ptr,
                        const double *__restrict__ stage_val, double *__restrict__ f, int neg,
                        const int32_t *__restrict__ status) {
  int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (i >= N || *status != GN_OK) return;
  const int64_t W = 2 * L;
  int t0 = __ldg(poly_ptr + i), t1 = __ldg(poly_ptr + i + 1);
  cx<L> acc = c_zero<L>();
  for (int t = t0 + lane; t < t1; t += 32) acc = c_add<L>(acc, c_load<L>(stage_val + (int64_t)t * W));
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc = c_add<L>(acc, shfl_down<L>(acc, off));
  if (lane == 0) c_store<L>(f + (int64_t)i * W, neg ? c_neg<L>(acc) : acc);
}

template <int L>
static gn_status eval_impl(gn_system *s, const double *d_x, double *d_f, int neg_f, double *d_J,
                           int64_t ldJ, cudaStream_t st) {
  Workspace *ws;
  gn_status e = workspace_get(s, L, &ws);
  if (e) return e;
  const int64_t W = 2 * L;
  k_powers<L><<<(s->n + 127) / 128, 128, 0, st>>>(d_x, s->n, s->pmax, ws->pow, ws->status);
  if (s->T > 0)
    k_monomials<L><<<(unsigned)((s->T + 127) / 128), 128, 0, st>>>(
        s->d_mono_off, s->d_occ, s->d_coef, s->T, ws->pow, s->n, ws->stage_val, ws->stage_d,
        ws->status);
  if (d_J) {
    // entries outside the structural pattern are zero
    if (s->nz < (int64_t)s->N * s->n &&
        cudaMemset2DAsync(d_J, sizeof(double) * W * ldJ, 0, sizeof(double) * W * s->N, s->n, st) !=
            cudaSuccess)
      return GN_ECUDA;
    if (s->nz > 0)
      k_sum_jacobian<L><<<(unsigned)((s->nz + 127) / 128), 128, 0, st>>>(
          s->nz, s->d_jz_row, s->d_jz_col, s->d_jz_ptr, s->d_jz_occ, ws->stage_d, d_J, ldJ,
          ws->status);
  }
  if (d_f) k_sum_f<L><<<(s->N + 3) / 4, 128, 0, st>>>(s->N, s->d_poly_ptr, ws->stage_val, d_f, neg_f, ws->status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

gn_status launch_eval(gn_system *s, int L, const double *d_x, double *d_f, int neg_f, double *d_J,
                      int64_t ldJ, cudaStream_t st) {
  if (s->kmax > KMAX) return GN_EINVAL;
  switch (L) {
    case 1: return eval_impl<1>(s, d_x, d_f, neg_f, d_J, ldJ, st);
    case 2: return eval_impl<2>(s, d_x, d_f, neg_f, d_J, ldJ, st);
    case 4: return eval_impl<4>(s, d_x, d_f, neg_f, d_J, ldJ, st);
  }
  return GN_EINVAL;
}

}  // namespace gn

// ---------------------------------------------------------------------------
// gn_eval_noalloc: evaluation with library-static scratch instead of the
// per-system workspace, for callers that cannot allocate device memory at
// the time they evaluate.  The paper has no counterpart of this entry point.
// ---------------------------------------------------------------------------

namespace gn {

// Scratch for the power table, the staged terms and partials, and a status
// word.  Every process that loads the library holds this much device memory
// on each GPU it uses, until it exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GN_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static unsigned char *g_noalloc_ptr[kMaxDevices];  // device address of the scratch, per device

// the kernels of gn_eval_noalloc at precision L, loaded now: under lazy
// module loading (the CUDA default) a kernel's code is loaded, which may
// allocate device memory, at its first launch, and that first launch may be
// a later call in another precision
template <int L>
static bool noalloc_load_kernels() {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, k_powers<L>) == cudaSuccess &&
         cudaFuncGetAttributes(&fa, k_monomials<L>) == cudaSuccess &&
         cudaFuncGetAttributes(&fa, k_sum_jacobian<L>) == cudaSuccess &&
         cudaFuncGetAttributes(&fa, k_sum_f<L>) == cudaSuccess;
}

// Host code must not hand g_noalloc_scratch to a kernel: on the host that
// name is a stand-in, not a device address.  Look the address up once per
// device, with that device current, and load the kernels of every precision.
static gn_status noalloc_scratch(unsigned char **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GN_ECUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p ||
        !noalloc_load_kernels<1>() || !noalloc_load_kernels<2>() || !noalloc_load_kernels<4>()) {
      cudaGetLastError();
      return GN_ECUDA;
    }
    g_noalloc_ptr[dev] = (unsigned char *)p;
  }
  *out = g_noalloc_ptr[dev];
  return GN_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <int L>
static gn_status eval_noalloc_impl(const gn_system *s, const double *d_x, double *d_f, double *d_J,
                                   int64_t ldJ, cudaStream_t st) {
  const size_t W = 2 * L;
  const size_t b_status = 256;
  const size_t b_pow = align256(sizeof(double) * W * (size_t)s->n * s->pmax);
  const size_t b_val = align256(sizeof(double) * W * (size_t)(s->T > 0 ? s->T : 1));
  const size_t b_d = align256(sizeof(double) * W * (size_t)(s->nnz > 0 ? s->nnz : 1));
  if (b_status + b_pow + b_val + b_d > (size_t)GN_NOALLOC_SCRATCH_BYTES) return GN_EINVAL;
  unsigned char *base;
  gn_status e = noalloc_scratch(&base);
  if (e) return e;
  int32_t *status = (int32_t *)base;
  double *pow = (double *)(base + b_status);
  double *stage_val = (double *)(base + b_status + b_pow);
  double *stage_d = (double *)(base + b_status + b_pow + b_val);
  // The scratch keeps the previous call's contents.  The status word only
  // gates the kernels (each returns at once on a bad status, none sets one),
  // so it must start at GN_OK; like gn_eval, the call reports no device-side
  // condition (a NaN input comes out as NaN in f and J).
  if (cudaMemsetAsync(status, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return GN_ECUDA;
  k_powers<L><<<(s->n + 127) / 128, 128, 0, st>>>(d_x, s->n, s->pmax, pow, status);
  if (s->T > 0)
    k_monomials<L><<<(unsigned)((s->T + 127) / 128), 128, 0, st>>>(
        s->d_mono_off, s->d_occ, s->d_coef, s->T, pow, s->n, stage_val, stage_d, status);
  if (d_J) {
    if (s->nz < (int64_t)s->N * s->n &&
        cudaMemset2DAsync(d_J, sizeof(double) * W * ldJ, 0, sizeof(double) * W * s->N, s->n, st) !=
            cudaSuccess)
      return GN_ECUDA;
    if (s->nz > 0)
      k_sum_jacobian<L><<<(unsigned)((s->nz + 127) / 128), 128, 0, st>>>(
          s->nz, s->d_jz_row, s->d_jz_col, s->d_jz_ptr, s->d_jz_occ, stage_d, d_J, ldJ, status);
  }
  if (d_f) k_sum_f<L><<<(s->N + 3) / 4, 128, 0, st>>>(s->N, s->d_poly_ptr, stage_val, d_f, 0, status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

}  // namespace gn

extern "C" gn_status gn_eval_noalloc(const gn_system *s, gn_prec prec, const double *d_x,
                                     double *d_f, double *d_J, int64_t ldJ, void *cuda_stream) {
  if (!s || !d_x || (d_J && ldJ < s->N) || s->kmax > gn::KMAX) return GN_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  switch (prec) {
    case GN_D: return gn::eval_noalloc_impl<1>(s, d_x, d_f, d_J, ldJ, st);
    case GN_DD: return gn::eval_noalloc_impl<2>(s, d_x, d_f, d_J, ldJ, st);
    case GN_QD: return gn::eval_noalloc_impl<4>(s, d_x, d_f, d_J, ldJ, st);
  }
  return GN_EINVAL;
}
