// mwfx.cuh — products of multiword numbers summed exactly on the integer pipe.
//
// A product of two L-limb reals is split by FP64 TwoProd into exact pieces
// (all pieces down to order 2^(-53 L) relative; the few of lower order are
// summed in FP64, their rounding sits below 2^(-53 (L+1))).  The pieces go
// into an fx accumulator, which sums them exactly.  So an inner product, an
// axpy or a renormalised product costs a handful of FP64 instructions per
// term plus integer work, instead of the dozens of FP64 instructions a
// double-double or quad-double addition takes (see mw.cuh).
#pragma once

#include "fx.cuh"
#include "mw.cuh"

namespace gn {

// Limbs and scale headroom of the accumulator per precision.  Values bounded
// by 2^E are accumulated at F = BITS - E: the resolution is 2^(E - BITS)
// (far below 2^(-53 L) of the bound) and up to 2^(64 NL - 2 - BITS) such
// values can be summed.
template <int L>
struct FxCfg;
template <>
struct FxCfg<1> {
  static constexpr int NL = 2, BITS = 110;
};
template <>
struct FxCfg<2> {
  static constexpr int NL = 3, BITS = 170;
};
template <>
struct FxCfg<4> {
  static constexpr int NL = 5, BITS = 290;
};

// acc += (neg ? -1 : 1) * d * 2^F
template <int NL>
GN_DEV bool fx_addd(fx<NL> &acc, double d, int F, bool neg) {
  return fx_add_bits<NL>(acc, fx_dbits(d) ^ (neg ? 0x8000000000000000ull : 0ull), F);
}

// acc += s * x * y for reals x, y at precision L (s = -1 when neg)
template <int L, int NL>
GN_DEV bool fx_add_prod(fx<NL> &acc, const double (&x)[L], const double (&y)[L], bool neg, int F) {
  bool ok = true;
  if constexpr (L == 1) {
    double p, e;
    two_prod(x[0], y[0], p, e);
    ok &= fx_addd<NL>(acc, p, F, neg);
    ok &= fx_addd<NL>(acc, e, F, neg);
  } else if constexpr (L == 2) {
    double p, e;
    two_prod(x[0], y[0], p, e);
    double lo = __fma_rn(x[0], y[1], e);
    lo = __fma_rn(x[1], y[0], lo);
    ok &= fx_addd<NL>(acc, p, F, neg);
    ok &= fx_addd<NL>(acc, lo, F, neg);
  } else {
    double p00, e00, p01, e01, p10, e10, p02, e02, p11, e11, p20, e20;
    two_prod(x[0], y[0], p00, e00);
    two_prod(x[0], y[1], p01, e01);
    two_prod(x[1], y[0], p10, e10);
    two_prod(x[0], y[2], p02, e02);
    two_prod(x[1], y[1], p11, e11);
    two_prod(x[2], y[0], p20, e20);
    double s3 = __dadd_rn(__dadd_rn(e02, e11), e20);
    s3 = __fma_rn(x[0], y[3], s3);
    s3 = __fma_rn(x[1], y[2], s3);
    s3 = __fma_rn(x[2], y[1], s3);
    s3 = __fma_rn(x[3], y[0], s3);
    ok &= fx_addd<NL>(acc, p00, F, neg);
    ok &= fx_addd<NL>(acc, e00, F, neg);
    ok &= fx_addd<NL>(acc, p01, F, neg);
    ok &= fx_addd<NL>(acc, e01, F, neg);
    ok &= fx_addd<NL>(acc, p10, F, neg);
    ok &= fx_addd<NL>(acc, e10, F, neg);
    ok &= fx_addd<NL>(acc, p02, F, neg);
    ok &= fx_addd<NL>(acc, p11, F, neg);
    ok &= fx_addd<NL>(acc, p20, F, neg);
    ok &= fx_addd<NL>(acc, s3, F, neg);
  }
  return ok;
}

// acc += s * x for a real x at precision L
template <int L, int NL>
GN_DEV bool fx_add_limbs(fx<NL> &acc, const double (&x)[L], bool neg, int F) {
  bool ok = true;
#pragma unroll
  for (int l = 0; l < L; l++) ok &= fx_addd<NL>(acc, x[l], F, neg);
  return ok;
}

// re += Re(conj(q) a), im += Im(conj(q) a)
template <int L, int NL>
GN_DEV bool fx_add_conj_prod(fx<NL> &re, fx<NL> &im, const cx<L> &q, const cx<L> &a, int F) {
  bool ok = true;
  ok &= fx_add_prod<L, NL>(re, q.re, a.re, false, F);
  ok &= fx_add_prod<L, NL>(re, q.im, a.im, false, F);
  ok &= fx_add_prod<L, NL>(im, q.re, a.im, false, F);
  ok &= fx_add_prod<L, NL>(im, q.im, a.re, true, F);
  return ok;
}

// re += s Re(r q), im += s Im(r q)
template <int L, int NL>
GN_DEV bool fx_add_cprod(fx<NL> &re, fx<NL> &im, const cx<L> &r, const cx<L> &q, bool neg, int F) {
  bool ok = true;
  ok &= fx_add_prod<L, NL>(re, r.re, q.re, neg, F);
  ok &= fx_add_prod<L, NL>(re, r.im, q.im, !neg, F);
  ok &= fx_add_prod<L, NL>(im, r.re, q.im, neg, F);
  ok &= fx_add_prod<L, NL>(im, r.im, q.re, neg, F);
  return ok;
}

// a - r q, exact sum rounded (truncated) to L limbs per part
template <int L>
GN_DEV cx<L> fx_axpy(const cx<L> &a, const cx<L> &r, const cx<L> &q, int F, bool &ok) {
  constexpr int NL = FxCfg<L>::NL;
  fx<NL> re, im;
  fx_zero<NL>(re);
  fx_zero<NL>(im);
  ok &= fx_add_limbs<L, NL>(re, a.re, false, F);
  ok &= fx_add_limbs<L, NL>(im, a.im, false, F);
  ok &= fx_add_cprod<L, NL>(re, im, r, q, true, F);
  cx<L> out;
  fx_to_cascade<NL, L>(re, F, out.re);
  fx_to_cascade<NL, L>(im, F, out.im);
  return out;
}

// a * s for a real s, rounded (truncated) to L limbs per part
template <int L>
GN_DEV cx<L> fx_scale_real(const cx<L> &a, const double (&s)[L], int F, bool &ok) {
  constexpr int NL = FxCfg<L>::NL;
  fx<NL> re, im;
  fx_zero<NL>(re);
  fx_zero<NL>(im);
  ok &= fx_add_prod<L, NL>(re, a.re, s, false, F);
  ok &= fx_add_prod<L, NL>(im, a.im, s, false, F);
  cx<L> out;
  fx_to_cascade<NL, L>(re, F, out.re);
  fx_to_cascade<NL, L>(im, F, out.im);
  return out;
}

template <int NL>
GN_DEV fx<NL> fx_shfl_xor(const fx<NL> &a, int m) {
  fx<NL> r;
#pragma unroll
  for (int i = 0; i < NL; i++) r.w[i] = __shfl_xor_sync(0xffffffffu, a.w[i], m);
  return r;
}

// warp-wide exact sum; every lane gets it
template <int NL>
GN_DEV fx<NL> fx_warp_sum(fx<NL> a) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    fx<NL> b = fx_shfl_xor<NL>(a, m);
    fx_add_to<NL>(a, b);
  }
  return a;
}

}  // namespace gn
