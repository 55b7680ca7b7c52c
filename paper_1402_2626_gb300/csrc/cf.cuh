// cf.cuh — complex numbers with integer mantissas and one binary exponent.
//
// A value (re + i im) 2^e holds re and im as K-limb two's-complement
// integers (K = 1, 2, 4 for double, double double and quad double: 62, 126
// and 254 significant bits), normalised so that max(|re|, |im|) lies in
// [2^(64K-3), 2^(64K-2)] (zero: both mantissas 0).  A product is four
// truncated K x K-limb integer products, two additions and a renormalising
// shift of a few bits; the error of each operation is below 2^(-64K+4)
// relative to |a| |b| (normwise, as for complex floating-point products).
//
// On GB300 this runs on the integer pipe, which issues 38 times more lane
// operations per cycle than the FP64 pipe a double-double or quad-double
// product would need (measured: 19 T INT32 vs 0.5 T FP64 lane-ops/s).
#pragma once

#include <math.h>

#include "ifx.cuh"

namespace gn {

constexpr int CF_EZERO = -(1 << 28);  // exponent of zero

// Exponent of a value that stands for a NaN or an infinity (cf_from_cascade
// of a non-finite input).  Products stay at or near it (cf_mul saturates
// there), sums align to it and drop every finite term, and cf_store_cascade
// writes NaN for it, so a non-finite input reaches f and J as NaN, as it
// would in floating point; one that meets an exact zero factor vanishes.
// Finite values stay far below it (|e| < 2^17 for values in the double
// range and products of a few hundred of them).
constexpr int CF_ENAN = 1 << 24;

template <int K>
struct cf {
  fx<K> re, im;
  int e;
};

template <int K>
FX_HD cf<K> cf_zero() {
  cf<K> z;
  fx_zero<K>(z.re);
  fx_zero<K>(z.im);
  z.e = CF_EZERO;
  return z;
}

// the low K limbs of floor(x / 2^(r - 8)) for a signed (K+1)-limb x with
// |x| < 2^(64K + 55) and 0 <= r < 64: x 2^8 (exact), then one funnel shift
// right by r (a shift left by 8 - r when r < 8); no branch on the direction
template <int K>
FX_HD fx<K> cf_shift8(const fx<K + 1> &x, int r) {
  fx<K + 1> t;
#pragma unroll
  for (int i = 0; i <= K; i++) t.w[i] = (x.w[i] << 8) | (i > 0 ? x.w[i - 1] >> 56 : 0);
  fx<K> o;
#pragma unroll
  for (int i = 0; i < K; i++) o.w[i] = (t.w[i] >> r) | ((t.w[i + 1] << 1) << (63 - r));
  return o;
}

// shift a (K+1)-limb signed value so that max bit length lands on 64K-2,
// then narrow to K limbs; returns the exponent adjustment
template <int K>
FX_HD int cf_normalize(fx<K + 1> &re, fx<K + 1> &im, fx<K> &ore, fx<K> &oim) {
  uint64_t n1, n2;
  const ux<K + 1> ur = ix_abs<K + 1>(re, n1), ui = ix_abs<K + 1>(im, n2);
  // the bit length of max(|re|, |im|) is that of |re| | |im|
  fx<K + 1> am;
#pragma unroll
  for (int w = 0; w <= K; w++) am.w[w] = ur.w[w] | ui.w[w];
  const int B = ix_bitlen<K + 1>(am);
  if (B == 0) {
    fx_zero<K>(ore);
    fx_zero<K>(oim);
    return CF_EZERO;
  }
  const int sh = B - (64 * K - 2);  // > 0: shift right
  if (sh >= -8 && sh < 56) {
    // every normalised product, scaling and conversion lands here
    ore = cf_shift8<K>(re, sh + 8);
    oim = cf_shift8<K>(im, sh + 8);
    return sh;
  }
  if (sh >= 0) {
    re = ix_sar<K + 1>(re, sh);
    im = ix_sar<K + 1>(im, sh);
  } else {
    // shift left by -sh (< 64 K)
    re = ix_shl<K + 1>(re, -sh);
    im = ix_shl<K + 1>(im, -sh);
  }
  ore = ix_narrow<K>(re);
  oim = ix_narrow<K>(im);
  return sh;
}

// a * b.  Each part is the same value as the difference (sum) of the two
// signed truncated products ix_mul_shift forms, s1 T1 -+ s2 T2, taken as
// s1 (T1 -+ s1 s2 T2) on the magnitudes T: one addition with a conditional
// complement and one conditional negation instead of two negations and an
// addition.
template <int K>
FX_HD cf<K> cf_mul(const cf<K> &a, const cf<K> &b) {
  uint64_t nar, nai, nbr, nbi;
  const ux<K> uar = ix_abs<K>(a.re, nar), uai = ix_abs<K>(a.im, nai);
  const ux<K> ubr = ix_abs<K>(b.re, nbr), ubi = ix_abs<K>(b.im, nbi);
  // re = s_rr T_rr - s_ii T_ii = s_rr (T_rr - s_rr s_ii T_ii)
  const uint64_t srr = nar ^ nbr, sii = nai ^ nbi;
  fx<K + 1> re = ix_add_cneg<K + 1>(ix_umul_shift<K>(uar, ubr), ix_umul_shift<K>(uai, ubi), 1 ^ srr ^ sii);
  ix_cneg<K + 1>(re, srr);
  // im = s_ri T_ri + s_ir T_ir = s_ri (T_ri + s_ri s_ir T_ir)
  const uint64_t sri = nar ^ nbi, sir = nai ^ nbr;
  fx<K + 1> im = ix_add_cneg<K + 1>(ix_umul_shift<K>(uar, ubi), ix_umul_shift<K>(uai, ubr), sri ^ sir);
  ix_cneg<K + 1>(im, sri);
  cf<K> r;
  const int sh = cf_normalize<K>(re, im, r.re, r.im);
  const int e = a.e + b.e + (64 * K - 2) + sh;
  r.e = (sh == CF_EZERO || a.e == CF_EZERO || b.e == CF_EZERO) ? CF_EZERO : (e < CF_ENAN ? e : CF_ENAN);
  return r;
}

// d * a for an integer 0 < d < 2^32
template <int K>
FX_HD cf<K> cf_scale_int(const cf<K> &a, uint32_t d) {
  fx<K + 1> re, im;
  uint64_t n1, n2;
  const ux<K> ur = ix_abs<K>(a.re, n1), ui = ix_abs<K>(a.im, n2);
  u128_t c1 = 0, c2 = 0;
#pragma unroll
  for (int w = 0; w < K; w++) {
    c1 += (u128_t)ur.w[w] * d;
    c2 += (u128_t)ui.w[w] * d;
    re.w[w] = (uint64_t)c1;
    im.w[w] = (uint64_t)c2;
    c1 >>= 64;
    c2 >>= 64;
  }
  re.w[K] = (uint64_t)c1;
  im.w[K] = (uint64_t)c2;
  ix_cneg<K + 1>(re, n1);
  ix_cneg<K + 1>(im, n2);
  cf<K> r;
  const int sh = cf_normalize<K>(re, im, r.re, r.im);
  r.e = (sh == CF_EZERO || a.e == CF_EZERO) ? CF_EZERO : a.e + sh;
  return r;
}

// from the [re limbs | im limbs] cascade of L doubles
template <int K, int L>
FX_HD cf<K> cf_from_cascade(const double (&re)[L], const double (&im)[L]) {
  bool finite = true;
#pragma unroll
  for (int l = 0; l < L; l++) finite &= isfinite(re[l]) && isfinite(im[l]);
  if (!finite) {
    cf<K> z;  // any normalised mantissas, exponent CF_ENAN
    fx_zero<K>(z.re);
    fx_zero<K>(z.im);
    z.re.w[K - 1] = z.im.w[K - 1] = 1ull << 61;
    z.e = CF_ENAN;
    return z;
  }
  const double m = fabs(re[0]) > fabs(im[0]) ? fabs(re[0]) : fabs(im[0]);
  if (!(m > 0.0)) return cf_zero<K>();
  // |value| < 2^(E+1) with E the exponent of the leading limb (one bit of
  // room for the lower limbs), mantissas at 2^(64K - 3 - E)
  const int E = fx_exponent_of(m);
  const int F = 64 * K - 3 - E;
  fx<K + 1> r, i;
  fx_zero<K + 1>(r);
  fx_zero<K + 1>(i);
#pragma unroll
  for (int l = 0; l < L; l++) {
    fx_add_double<K + 1>(r, re[l], F);
    fx_add_double<K + 1>(i, im[l], F);
  }
  cf<K> z;
  const int sh = cf_normalize<K>(r, i, z.re, z.im);
  z.e = (sh == CF_EZERO) ? CF_EZERO : sh - F;
  return z;
}

template <int K, int L>
FX_HD void cf_to_cascade(const cf<K> &z, double (&re)[L], double (&im)[L]) {
  if (z.e == CF_EZERO) {
#pragma unroll
    for (int l = 0; l < L; l++) re[l] = im[l] = 0.0;
    return;
  }
  fx_to_cascade<K, L>(z.re, -z.e, re);
  fx_to_cascade<K, L>(z.im, -z.e, im);
}

// Exact-alignment term sums (Section 2.3).  The common exponent E is the
// largest exponent among the terms plus the bit length of their count, so
// that the sum cannot overflow; each K-limb mantissa goes to the top K limbs
// of a (K+1)-limb accumulator (64 guard bits) and shifts right by E - e.  The
// accumulator then holds the sum in units of 2^(E - 64), and the only error
// is the truncation of each term below that unit.
template <int K>
FX_HD void cf_accumulate(fx<K + 1> &re, fx<K + 1> &im, const cf<K> &z, int E) {
  if (z.e == CF_EZERO) return;
  const int s = E - z.e;
  if (s >= 64 * K + 62) return;  // entirely below the accumulator's unit
  fx<K + 1> a, b;
  a.w[0] = 0;
  b.w[0] = 0;
#pragma unroll
  for (int w = 0; w < K; w++) {
    a.w[w + 1] = z.re.w[w];
    b.w[w + 1] = z.im.w[w];
  }
  re = ix_add<K + 1>(re, ix_sar<K + 1>(a, s));
  im = ix_add<K + 1>(im, ix_sar<K + 1>(b, s));
}

// exponent of the sums of c terms whose largest exponent is emax
FX_HD int cf_sum_exponent(int emax, int c) {
  return emax == CF_EZERO ? CF_EZERO : emax + (64 - fx_clz64((uint64_t)(c > 0 ? c : 1)));
}

}  // namespace gn
