// eval_int.cu — evaluation and differentiation (Section 2) with
// integer-mantissa complex arithmetic (cf.cuh): the same schedule as eval.cu
// (power table, common factor folded into the forward products, one running
// backward product, exponent factors, owner-computed term sums), with every
// product and sum on the integer pipe instead of FP64 error-free
// transformations.  Term sums align the contributions to the largest
// exponent among them and add the mantissas exactly.
#include "cf.cuh"
#include "internal.h"
#include "mw.cuh"

namespace gn {

constexpr int KMAXI = 64;

// words (8 bytes) per staged complex value: re mantissa, im mantissa, exponent
template <int L>
struct CfStore {
  static constexpr int WORDS = 2 * L + 1;
};

template <int K>
__device__ __forceinline__ void cf_st(double *p, const cf<K> &z) {
  uint64_t *q = (uint64_t *)p;
#pragma unroll
  for (int w = 0; w < K; w++) {
    q[w] = z.re.w[w];
    q[K + w] = z.im.w[w];
  }
  q[2 * K] = (uint64_t)(int64_t)z.e;
}

template <int K>
__device__ __forceinline__ cf<K> cf_ld(const double *p) {
  const uint64_t *q = (const uint64_t *)p;
  cf<K> z;
#pragma unroll
  for (int w = 0; w < K; w++) {
    z.re.w[w] = __ldg(q + w);
    z.im.w[w] = __ldg(q + K + w);
  }
  z.e = (int)(int64_t)__ldg(q + 2 * K);
  return z;
}

// the exponent factor d of Section 2.3 (d = 1: the normalised input itself,
// which is what a scaling by 1 returns)
template <int K>
__device__ __forceinline__ cf<K> cf_scale_d(const cf<K> &a, uint32_t d) {
  return d == 1 ? a : cf_scale_int<K>(a, d);
}

template <int L>
__global__ void k_powers_cf(const double *__restrict__ x, int32_t n, int32_t pmax,
                            double *__restrict__ pow, const int32_t *__restrict__ status) {
  constexpr int WS = CfStore<L>::WORDS;
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n || *status != GN_OK) return;
  double re[L], im[L];
#pragma unroll
  for (int l = 0; l < L; l++) {
    re[l] = x[(int64_t)v * 2 * L + l];
    im[l] = x[(int64_t)v * 2 * L + L + l];
  }
  const cf<L> xv = cf_from_cascade<L, L>(re, im);
  cf<L> p = xv;
  cf_st<L>(pow + (int64_t)v * WS, p);
  for (int q = 1; q < pmax; q++) {
    p = cf_mul<L>(p, xv);
    cf_st<L>(pow + ((int64_t)q * n + v) * WS, p);
  }
}

// KM: the longest support the launch handles (the forward products of one
// monomial live in a KM-entry per-thread array)
template <int L, int KM>
__global__ void __launch_bounds__(256) k_monomials_cf(
    const int32_t *__restrict__ mono_off, const uint32_t *__restrict__ occ,
    const double *__restrict__ coef, int64_t T, const double *__restrict__ pow, int32_t n,
    double *__restrict__ stage_val, double *__restrict__ stage_d,
    const int32_t *__restrict__ status) {
  constexpr int WS = CfStore<L>::WORDS;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T || *status != GN_OK) return;
  const int o0 = __ldg(mono_off + t);
  const int k = __ldg(mono_off + t + 1) - o0;
  if (k > KM) return;  // a long support: k_monomials_long_cf
  double cre[L], cim[L];
#pragma unroll
  for (int l = 0; l < L; l++) {
    cre[l] = __ldg(coef + (int64_t)(2 * l + 0) * T + t);
    cim[l] = __ldg(coef + (int64_t)(2 * l + 1) * T + t);
  }
  cf<L> a = cf_from_cascade<L, L>(cre, cim);
  for (int s = 0; s < k; s++) {
    uint32_t w = __ldg(occ + o0 + s);
    int d = (int)(w & 255u);
    if (d >= 2) a = cf_mul<L>(a, cf_ld<L>(pow + ((int64_t)(d - 2) * n + (w >> 8)) * WS));
  }
  if (k == 0) {
    cf_st<L>(stage_val + t * WS, a);
    return;
  }
  cf<L> F[KM];
  F[0] = a;
  for (int s = 1; s < k; s++) {
    int v = (int)(__ldg(occ + o0 + s - 1) >> 8);
    F[s] = cf_mul<L>(F[s - 1], cf_ld<L>(pow + (int64_t)v * WS));
  }
  uint32_t wl = __ldg(occ + o0 + k - 1);
  cf<L> B = cf_ld<L>(pow + (int64_t)(wl >> 8) * WS);
  cf_st<L>(stage_val + t * WS, cf_mul<L>(F[k - 1], B));
  cf_st<L>(stage_d + (int64_t)(o0 + k - 1) * WS, cf_scale_d<L>(F[k - 1], wl & 255u));
  for (int s = k - 2; s >= 0; s--) {
    uint32_t w = __ldg(occ + o0 + s);
    cf_st<L>(stage_d + (int64_t)(o0 + s) * WS, cf_scale_d<L>(cf_mul<L>(F[s], B), w & 255u));
    if (s > 0) B = cf_mul<L>(B, cf_ld<L>(pow + (int64_t)(w >> 8) * WS));
  }
}

// the value of the other lane of a pair (lanes 2p, 2p + 1 of the warp)
template <int K>
__device__ __forceinline__ cf<K> cf_pair_swap(const cf<K> &a) {
  const unsigned mask = 3u << (threadIdx.x & 30);
  cf<K> r;
#pragma unroll
  for (int w = 0; w < K; w++) {
    r.re.w[w] = __shfl_xor_sync(mask, (unsigned long long)a.re.w[w], 1);
    r.im.w[w] = __shfl_xor_sync(mask, (unsigned long long)a.im.w[w], 1);
  }
  r.e = __shfl_xor_sync(mask, a.e, 1);
  return r;
}

// The schedule of k_monomials_cf on a lane pair per term, the same products
// in the same order (so the same bits), with the two chains side by side:
// lane 0 of the pair forms the coefficient times the common factor and the
// forward products F_s = a x_0 .. x_{s-1}; lane 1 the backward products
// B_s = x_{s+1} .. x_{k-1} (the running product from the end).  Then the
// pair forms the partials d_s F_s B_s two at a time, lane 0 the even s and
// lane 1 the odd s, each taking the factor it lacks from the other lane by
// one shuffle.  The dependent chain per term is the common factor plus k - 1
// products plus k / 2, against the common factor plus 3k - 3 on one lane.
// The terms' values alone, for an evaluation of f without J (the
// refinement steps of the mixed solver): the common factor and then the
// forward chain of k_monomials_cf, the same products in the same order (so
// the same bits), and none of the partial derivatives.  Supports longer than
// KMAXI are left to k_monomials_long_cf, as there.
template <int L>
__global__ void __launch_bounds__(256) k_monomial_values_cf(
    const int32_t *__restrict__ mono_off, const uint32_t *__restrict__ occ,
    const double *__restrict__ coef, int64_t T, const double *__restrict__ pow, int32_t n,
    double *__restrict__ stage_val, const int32_t *__restrict__ status) {
  constexpr int WS = CfStore<L>::WORDS;
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T || *status != GN_OK) return;
  const int o0 = __ldg(mono_off + t);
  const int k = __ldg(mono_off + t + 1) - o0;
  if (k > KMAXI) return;  // a long support: k_monomials_long_cf
  double cre[L], cim[L];
#pragma unroll
  for (int l = 0; l < L; l++) {
    cre[l] = __ldg(coef + (int64_t)(2 * l + 0) * T + t);
    cim[l] = __ldg(coef + (int64_t)(2 * l + 1) * T + t);
  }
  cf<L> a = cf_from_cascade<L, L>(cre, cim);
  for (int s = 0; s < k; s++) {
    uint32_t w = __ldg(occ + o0 + s);
    int d = (int)(w & 255u);
    if (d >= 2) a = cf_mul<L>(a, cf_ld<L>(pow + ((int64_t)(d - 2) * n + (w >> 8)) * WS));
  }
  for (int s = 0; s < k; s++) a = cf_mul<L>(a, cf_ld<L>(pow + (int64_t)(__ldg(occ + o0 + s) >> 8) * WS));
  cf_st<L>(stage_val + t * WS, a);
}

template <int L, int KM>
__global__ void __launch_bounds__(256) k_monomials2_cf(
    const int32_t *__restrict__ mono_off, const uint32_t *__restrict__ occ,
    const double *__restrict__ coef, int64_t T, const double *__restrict__ pow, int32_t n,
    double *__restrict__ stage_val, double *__restrict__ stage_d,
    const int32_t *__restrict__ status) {
  constexpr int WS = CfStore<L>::WORDS;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t t = g >> 1;
  const int side = (int)(g & 1);
  if (t >= T || *status != GN_OK) return;  // both lanes of a pair alike
  const int o0 = __ldg(mono_off + t);
  const int k = __ldg(mono_off + t + 1) - o0;
  if (k > KM) return;  // a long support: k_monomials_long_cf
  cf<L> P[KM];  // lane 0: F_s; lane 1: B_s
  if (side == 0) {
    double cre[L], cim[L];
#pragma unroll
    for (int l = 0; l < L; l++) {
      cre[l] = __ldg(coef + (int64_t)(2 * l + 0) * T + t);
      cim[l] = __ldg(coef + (int64_t)(2 * l + 1) * T + t);
    }
    cf<L> a = cf_from_cascade<L, L>(cre, cim);
    for (int s = 0; s < k; s++) {
      uint32_t w = __ldg(occ + o0 + s);
      int d = (int)(w & 255u);
      if (d >= 2) a = cf_mul<L>(a, cf_ld<L>(pow + ((int64_t)(d - 2) * n + (w >> 8)) * WS));
    }
    if (k == 0) {
      cf_st<L>(stage_val + t * WS, a);
      return;
    }
    P[0] = a;
    for (int s = 1; s < k; s++) {
      int v = (int)(__ldg(occ + o0 + s - 1) >> 8);
      P[s] = cf_mul<L>(P[s - 1], cf_ld<L>(pow + (int64_t)v * WS));
    }
    const uint32_t wl = __ldg(occ + o0 + k - 1);
    cf_st<L>(stage_val + t * WS, cf_mul<L>(P[k - 1], cf_ld<L>(pow + (int64_t)(wl >> 8) * WS)));
  } else {
    if (k == 0) return;
    if (k >= 2) {
      cf<L> B = cf_ld<L>(pow + (int64_t)(__ldg(occ + o0 + k - 1) >> 8) * WS);
      for (int s = k - 2; s >= 0; s--) {
        P[s] = B;
        if (s > 0) B = cf_mul<L>(B, cf_ld<L>(pow + (int64_t)(__ldg(occ + o0 + s) >> 8) * WS));
      }
    }
  }
  // partials: step q takes s0 = 2q on lane 0 and s1 = 2q + 1 on lane 1; lane 0
  // sends F_s1, lane 1 sends B_s0 (what the other lane lacks)
  for (int s0 = 0; s0 < k; s0 += 2) {
    const int s1 = s0 + 1;
    const int mine = side == 0 ? s0 : s1;
    const int give = side == 0 ? s1 : s0;
    const cf<L> got = cf_pair_swap<L>(P[give < k ? give : mine]);
    if (mine >= k) continue;
    const uint32_t w = __ldg(occ + o0 + mine);
    // lane 0 holds F_mine and receives B_mine; lane 1 holds B_mine and receives F_mine
    const cf<L> F = side == 0 ? P[mine] : got;
    cf<L> dv;
    if (mine == k - 1) {
      dv = cf_scale_d<L>(F, w & 255u);  // B_{k-1} is the empty product
    } else {
      const cf<L> B = side == 0 ? got : P[mine];
      dv = cf_scale_d<L>(cf_mul<L>(F, B), w & 255u);
    }
    cf_st<L>(stage_d + (int64_t)(o0 + mine) * WS, dv);
  }
}

// a cf<K> value and whether it holds anything (the empty product)
template <int K>
struct cfo {
  cf<K> v;
  int has;
};

template <int K>
__device__ __forceinline__ cfo<K> cfo_mul(const cfo<K> &a, const cfo<K> &b) {
  if (!a.has) return b;
  if (!b.has) return a;
  return {cf_mul<K>(a.v, b.v), 1};
}

template <int K>
__device__ __forceinline__ cfo<K> cfo_shfl(const cfo<K> &a, int src, int mode /* 0 idx, 1 up, 2 down */,
                                           int delta) {
  cfo<K> r;
  auto sh = [&](uint64_t w) -> uint64_t {
    return mode == 0 ? __shfl_sync(0xffffffffu, (unsigned long long)w, src)
           : mode == 1 ? __shfl_up_sync(0xffffffffu, (unsigned long long)w, delta)
                       : __shfl_down_sync(0xffffffffu, (unsigned long long)w, delta);
  };
  auto shi = [&](int w) -> int {
    return mode == 0 ? __shfl_sync(0xffffffffu, w, src)
           : mode == 1 ? __shfl_up_sync(0xffffffffu, w, delta)
                       : __shfl_down_sync(0xffffffffu, w, delta);
  };
#pragma unroll
  for (int w = 0; w < K; w++) {
    r.v.re.w[w] = sh(a.v.re.w[w]);
    r.v.im.w[w] = sh(a.v.im.w[w]);
  }
  r.v.e = shi(a.v.e);
  r.has = shi(a.has);
  return r;
}

// a staged value written by this thread earlier in the launch (not __ldg:
// the read-only path need not see this launch's own stores)
template <int K>
__device__ __forceinline__ cf<K> cf_ld_own(const double *p) {
  const uint64_t *q = (const uint64_t *)p;
  cf<K> z;
#pragma unroll
  for (int w = 0; w < K; w++) {
    z.re.w[w] = q[w];
    z.im.w[w] = q[K + w];
  }
  z.e = (int)(int64_t)q[2 * K];
  return z;
}

// Terms whose support is longer than KMAXI: one warp per term, the
// Speelpenning product and gradient of Section 2.2 split over the lanes.
// Lane l owns the support positions [l c, l c + c), c = ceil(k / 32), and
// forms the product of its x's; two warp scans give every lane the product
// of the lanes before it (E) and after it (S); then, within the chunk,
//   left_s  = a E  prod_{r < s in chunk} x_r   (forward, parked in stage_d)
//   right_s = prod_{r > s in chunk} x_r  S     (backward, running)
// and stage_d[s] = d_s left_s right_s, stage_val = a prod_all x.  The
// coefficient times the common factor prod x^(d-1) (Section 2.1), a, is the
// product of lane partials reduced to lane 0 in a fixed tree.  The cyclic
// n-roots system of Section 5.3 has supports up to n.
template <int L>
__global__ void __launch_bounds__(128) k_monomials_long_cf(
    const int32_t *__restrict__ long_terms, int64_t nlong, const int32_t *__restrict__ mono_off,
    const uint32_t *__restrict__ occ, const double *__restrict__ coef, int64_t T,
    const double *__restrict__ pow, int32_t n, double *__restrict__ stage_val,
    double *__restrict__ stage_d, const int32_t *__restrict__ status) {
  constexpr int WS = CfStore<L>::WORDS;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= nlong || *status != GN_OK) return;  // uniform across the warp
  const int64_t t = __ldg(long_terms + wid);
  const int o0 = __ldg(mono_off + t);
  const int k = __ldg(mono_off + t + 1) - o0;
  const int c = (k + 31) >> 5;
  const int s0 = lane * c < k ? lane * c : k;
  const int s1 = s0 + c < k ? s0 + c : k;
  // a = coefficient x common factor
  cfo<L> a = {cf_zero<L>(), 0};
  if (lane == 0) {
    double cre[L], cim[L];
#pragma unroll
    for (int l = 0; l < L; l++) {
      cre[l] = __ldg(coef + (int64_t)(2 * l + 0) * T + t);
      cim[l] = __ldg(coef + (int64_t)(2 * l + 1) * T + t);
    }
    a = {cf_from_cascade<L, L>(cre, cim), 1};
  }
  cfo<L> p = {cf_zero<L>(), 0};
  for (int s = s0; s < s1; s++) {
    const uint32_t w = __ldg(occ + o0 + s);
    const int d = (int)(w & 255u);
    if (d >= 2) a = cfo_mul<L>(a, {cf_ld<L>(pow + ((int64_t)(d - 2) * n + (w >> 8)) * WS), 1});
    p = cfo_mul<L>(p, {cf_ld<L>(pow + (int64_t)(w >> 8) * WS), 1});
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const cfo<L> u = cfo_shfl<L>(a, 0, 2, off);
    if (lane < off) a = cfo_mul<L>(a, u);
  }
  a = cfo_shfl<L>(a, 0, 0, 0);
  // inclusive prefix and suffix products of the lane partials
  cfo<L> pre = p, suf = p;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const cfo<L> u = cfo_shfl<L>(pre, 0, 1, off);
    const cfo<L> v = cfo_shfl<L>(suf, 0, 2, off);
    if (lane >= off) pre = cfo_mul<L>(u, pre);
    if (lane + off < 32) suf = cfo_mul<L>(suf, v);
  }
  const cfo<L> total = cfo_shfl<L>(pre, 31, 0, 0);
  cfo<L> E = cfo_shfl<L>(pre, 0, 1, 1);
  cfo<L> S = cfo_shfl<L>(suf, 0, 2, 1);
  if (lane == 0) E.has = 0;
  if (lane == 31) S.has = 0;
  if (lane == 0) cf_st<L>(stage_val + t * WS, cfo_mul<L>(a, total).v);
  cfo<L> left = cfo_mul<L>(a, E);
  for (int s = s0; s < s1; s++) {
    cf_st<L>(stage_d + (int64_t)(o0 + s) * WS, left.v);
    left = cfo_mul<L>(left, {cf_ld<L>(pow + (int64_t)(__ldg(occ + o0 + s) >> 8) * WS), 1});
  }
  cfo<L> right = S;
  for (int s = s1 - 1; s >= s0; s--) {
    const uint32_t w = __ldg(occ + o0 + s);
    const cfo<L> g = cfo_mul<L>({cf_ld_own<L>(stage_d + (int64_t)(o0 + s) * WS), 1}, right);
    cf_st<L>(stage_d + (int64_t)(o0 + s) * WS, cf_scale_d<L>(g.v, w & 255u));
    right = cfo_mul<L>(right, {cf_ld<L>(pow + (int64_t)(w >> 8) * WS), 1});
  }
}

template <int L>
__device__ __forceinline__ void cf_store_cascade(double *dst, const fx<L + 1> &re, const fx<L + 1> &im,
                                                 int E, bool neg) {
  double r[L], i[L];
  if (E == CF_EZERO) {
#pragma unroll
    for (int l = 0; l < L; l++) r[l] = i[l] = 0.0;
  } else if (E > CF_ENAN / 2) {  // a non-finite input reached this sum
#pragma unroll
    for (int l = 0; l < L; l++) r[l] = i[l] = __longlong_as_double(0x7FF8000000000000ll);
  } else {
    fx_to_cascade<L + 1, L>(re, 64 - E, r);
    fx_to_cascade<L + 1, L>(im, 64 - E, i);
  }
#pragma unroll
  for (int l = 0; l < L; l++) {
    dst[l] = neg ? -r[l] : r[l];
    dst[L + l] = neg ? -i[l] : i[l];
  }
}

// J entry z goes to J[(col ldJ + row)], or to J[jz_out[z]] (complex entries)
// when jz_out is given (the blocks of a batch)
template <int L>
__global__ void k_sum_jacobian_cf(int64_t nz, const int32_t *__restrict__ jz_row,
                                  const int32_t *__restrict__ jz_col,
                                  const int32_t *__restrict__ jz_ptr,
                                  const int32_t *__restrict__ jz_occ,
                                  const int64_t *__restrict__ jz_out,
                                  const double *__restrict__ stage_d, double *__restrict__ J,
                                  int64_t ldJ, const int32_t *__restrict__ status) {
  constexpr int WS = CfStore<L>::WORDS;
  int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nz || *status != GN_OK) return;
  const int p0 = __ldg(jz_ptr + z), p1 = __ldg(jz_ptr + z + 1);
  int emax = CF_EZERO;
  for (int p = p0; p < p1; p++) {
    const int e = (int)(int64_t)__ldg((const uint64_t *)(stage_d + (int64_t)__ldg(jz_occ + p) * WS) + 2 * L);
    emax = e > emax ? e : emax;
  }
  const int E = cf_sum_exponent(emax, p1 - p0);
  fx<L + 1> re, im;
  fx_zero<L + 1>(re);
  fx_zero<L + 1>(im);
  for (int p = p0; p < p1; p++) cf_accumulate<L>(re, im, cf_ld<L>(stage_d + (int64_t)__ldg(jz_occ + p) * WS), E);
  const int64_t at = jz_out ? __ldg(jz_out + z) : (int64_t)__ldg(jz_col + z) * ldJ + __ldg(jz_row + z);
  cf_store_cascade<L>(J + at * 2 * L, re, im, E, false);
}

// The same sums with one warp per entry, for systems whose entries gather
// many partials (the dense Jacobian of cyclic n-roots: up to n - 1 per
// entry): lanes stride over the entry's partials, the largest exponent and
// the exact aligned sum are reduced over the warp.
template <int L>
__global__ void __launch_bounds__(128) k_sum_jacobian_warp_cf(
    int64_t nz, const int32_t *__restrict__ jz_row, const int32_t *__restrict__ jz_col,
    const int32_t *__restrict__ jz_ptr, const int32_t *__restrict__ jz_occ,
    const int64_t *__restrict__ jz_out, const double *__restrict__ stage_d, double *__restrict__ J,
    int64_t ldJ, const int32_t *__restrict__ status) {
  constexpr int WS = CfStore<L>::WORDS;
  const int64_t z = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (z >= nz || *status != GN_OK) return;  // uniform over the warp
  const int p0 = __ldg(jz_ptr + z), p1 = __ldg(jz_ptr + z + 1);
  int emax = CF_EZERO;
  for (int p = p0 + lane; p < p1; p += 32) {
    const int e = (int)(int64_t)__ldg((const uint64_t *)(stage_d + (int64_t)__ldg(jz_occ + p) * WS) + 2 * L);
    emax = e > emax ? e : emax;
  }
  const int E = cf_sum_exponent(__reduce_max_sync(0xffffffffu, emax), p1 - p0);
  fx<L + 1> re, im;
  fx_zero<L + 1>(re);
  fx_zero<L + 1>(im);
  for (int p = p0 + lane; p < p1; p += 32)
    cf_accumulate<L>(re, im, cf_ld<L>(stage_d + (int64_t)__ldg(jz_occ + p) * WS), E);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fx<L + 1> u, v;
#pragma unroll
    for (int w = 0; w <= L; w++) {
      u.w[w] = __shfl_xor_sync(0xffffffffu, re.w[w], o);
      v.w[w] = __shfl_xor_sync(0xffffffffu, im.w[w], o);
    }
    re = ix_add<L + 1>(re, u);
    im = ix_add<L + 1>(im, v);
  }
  if (lane == 0) {
    const int64_t at = jz_out ? __ldg(jz_out + z) : (int64_t)__ldg(jz_col + z) * ldJ + __ldg(jz_row + z);
    cf_store_cascade<L>(J + at * 2 * L, re, im, E, false);
  }
}

// f_i goes to f[i], or to f[f_out[i]] (complex entries) when f_out is given
template <int L>
__global__ void k_sum_f_cf(int32_t N, const int32_t *__restrict__ poly_ptr,
                           const double *__restrict__ stage_val, double *__restrict__ f,
                           const int64_t *__restrict__ f_out, int neg,
                           const int32_t *__restrict__ status) {
  constexpr int WS = CfStore<L>::WORDS;
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (i >= N || *status != GN_OK) return;
  const int t0 = __ldg(poly_ptr + i), t1 = __ldg(poly_ptr + i + 1);
  int emax = CF_EZERO;
  for (int t = t0 + lane; t < t1; t += 32) {
    const int e = (int)(int64_t)__ldg((const uint64_t *)(stage_val + (int64_t)t * WS) + 2 * L);
    emax = e > emax ? e : emax;
  }
  const int E = cf_sum_exponent(__reduce_max_sync(0xffffffffu, emax), t1 - t0);
  fx<L + 1> re, im;
  fx_zero<L + 1>(re);
  fx_zero<L + 1>(im);
  for (int t = t0 + lane; t < t1; t += 32) cf_accumulate<L>(re, im, cf_ld<L>(stage_val + (int64_t)t * WS), E);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fx<L + 1> u, v;
#pragma unroll
    for (int w = 0; w <= L; w++) {
      u.w[w] = __shfl_xor_sync(0xffffffffu, re.w[w], o);
      v.w[w] = __shfl_xor_sync(0xffffffffu, im.w[w], o);
    }
    re = ix_add<L + 1>(re, u);
    im = ix_add<L + 1>(im, v);
  }
  if (lane == 0) cf_store_cascade<L>(f + (f_out ? __ldg(f_out + i) : (int64_t)i) * 2 * L, re, im, E, neg != 0);
}

template <int L>
static gn_status eval_int_raw(const EvalArgs &a, cudaStream_t st) {
  if (a.nvar > 0)
    k_powers_cf<L><<<(unsigned)((a.nvar + 127) / 128), 128, 0, st>>>(a.x, (int32_t)a.nvar, a.pmax, a.pow,
                                                                      a.status);
  if (a.T > 0) {
    const int bt = (a.block == 64 || a.block == 256) ? a.block : 128;
    // one lane per term where the product chain is short (the kernel is
    // bound by its ALU instructions: gn256, k = 16, DD 0.205 ms against
    // 0.260 ms on pairs), a lane pair where it is long (k = 40, DD 0.148
    // against 0.173 ms); batches time both
    const int lanes = a.lanes == 1 || a.lanes == 2 ? a.lanes : (a.kmax <= 16 ? 1 : 2);
    const unsigned nb = (unsigned)((lanes * a.T + bt - 1) / bt);
    if (!a.J) {  // f alone: the values, no partials
      k_monomial_values_cf<L><<<(unsigned)((a.T + bt - 1) / bt), bt, 0, st>>>(
          a.mono_off, a.occ, a.coef, a.T, a.pow, (int32_t)a.nvar, a.stage_val, a.status);
    } else if (lanes == 1) {
      if (a.kmax <= 16)
        k_monomials_cf<L, 16><<<nb, bt, 0, st>>>(a.mono_off, a.occ, a.coef, a.T, a.pow, (int32_t)a.nvar,
                                                 a.stage_val, a.stage_d, a.status);
      else
        k_monomials_cf<L, KMAXI><<<nb, bt, 0, st>>>(a.mono_off, a.occ, a.coef, a.T, a.pow, (int32_t)a.nvar,
                                                    a.stage_val, a.stage_d, a.status);
    } else {
      if (a.kmax <= 16)
        k_monomials2_cf<L, 16><<<nb, bt, 0, st>>>(a.mono_off, a.occ, a.coef, a.T, a.pow, (int32_t)a.nvar,
                                                  a.stage_val, a.stage_d, a.status);
      else
        k_monomials2_cf<L, KMAXI><<<nb, bt, 0, st>>>(a.mono_off, a.occ, a.coef, a.T, a.pow,
                                                     (int32_t)a.nvar, a.stage_val, a.stage_d, a.status);
    }
  }
  if (a.nlong > 0)
    k_monomials_long_cf<L><<<(unsigned)((a.nlong + 3) / 4), 128, 0, st>>>(
        a.long_terms, a.nlong, a.mono_off, a.occ, a.coef, a.T, a.pow, (int32_t)a.nvar, a.stage_val,
        a.stage_d, a.status);
  if (a.J && a.nz > 0) {
    if (a.nocc >= 24 * a.nz)  // many partials per entry: a warp each
      k_sum_jacobian_warp_cf<L><<<(unsigned)((a.nz + 3) / 4), 128, 0, st>>>(
          a.nz, a.jz_row, a.jz_col, a.jz_ptr, a.jz_occ, a.jz_out, a.stage_d, a.J, a.ldJ, a.status);
    else
      k_sum_jacobian_cf<L><<<(unsigned)((a.nz + 127) / 128), 128, 0, st>>>(
          a.nz, a.jz_row, a.jz_col, a.jz_ptr, a.jz_occ, a.jz_out, a.stage_d, a.J, a.ldJ, a.status);
  }
  if (a.f && a.npoly > 0)
    k_sum_f_cf<L><<<(unsigned)((a.npoly + 3) / 4), 128, 0, st>>>((int32_t)a.npoly, a.poly_ptr, a.stage_val,
                                                                 a.f, a.f_out, a.neg_f, a.status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

gn_status launch_eval_int_raw(int L, const EvalArgs &a, cudaStream_t st) {
  if (a.kmax > KMAXI && !a.long_terms) return GN_EINVAL;
  switch (L) {
    case 1: return eval_int_raw<1>(a, st);
    case 2: return eval_int_raw<2>(a, st);
    case 4: return eval_int_raw<4>(a, st);
  }
  return GN_EINVAL;
}

gn_status launch_eval_int(gn_system *s, int L, const double *d_x, double *d_f, int neg_f,
                          double *d_J, int64_t ldJ, cudaStream_t st) {
  Workspace *ws;
  gn_status e = workspace_get(s, L, &ws);
  if (e) return e;
  const int64_t W = 2 * L;
  if (d_J && s->nz < (int64_t)s->N * s->n &&
      cudaMemset2DAsync(d_J, sizeof(double) * W * ldJ, 0, sizeof(double) * W * s->N, s->n, st) !=
          cudaSuccess)
    return GN_ECUDA;
  EvalArgs a;
  a.x = d_x;
  a.nvar = s->n;
  a.pmax = s->pmax;
  a.kmax = s->kmax;
  a.long_terms = s->d_long;
  a.nlong = s->nlong;
  a.pow = ws->pow;
  a.T = s->T;
  a.mono_off = s->d_mono_off;
  a.occ = s->d_occ;
  a.coef = s->d_coef;
  a.stage_val = ws->stage_val;
  a.stage_d = ws->stage_d;
  a.nz = s->nz;
  a.nocc = s->nnz;
  a.jz_row = s->d_jz_row;
  a.jz_col = s->d_jz_col;
  a.jz_ptr = s->d_jz_ptr;
  a.jz_occ = s->d_jz_occ;
  a.J = d_J;
  a.ldJ = ldJ;
  a.npoly = s->N;
  a.poly_ptr = s->d_poly_ptr;
  a.f = d_f;
  a.neg_f = neg_f;
  a.status = ws->status;
  return launch_eval_int_raw(L, a, st);
}

}  // namespace gn
