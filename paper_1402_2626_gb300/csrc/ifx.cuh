// ifx.cuh — signed multiword integer products for block-floating-point
// linear algebra on the integer pipe.
//
// Modified Gram-Schmidt (Section 3) runs with one binary exponent per column
// and K-limb two's-complement integer mantissas per real part (K = 1, 2, 4
// for double, double double and quad double: 62, 126 and 254 bits, more
// than the 53, 106 and 212 bits of the floating-point formats).  A product
// of two K-limb mantissas is formed from 64 x 64 -> 128-bit integer
// multiplications; on GB300 these issue about 16 times faster per lane than
// the FP64 instructions of a double-double product (and the FP64 pipe is
// the scarce one), with a latency of a few cycles instead of 64.
//
// Conventions: fx<K> (fx.cuh) holds a signed value; "scale" exponents are
// tracked by the caller.
#pragma once

#include "fx.cuh"

namespace gn {

typedef unsigned __int128 u128_t;

template <int N>
struct ux {
  uint64_t w[N];
};

// |a| and the sign of a (two's complement)
template <int K>
FX_HD ux<K> ix_abs(const fx<K> &a, uint64_t &neg) {
  neg = a.w[K - 1] >> 63;
  const uint64_t m = 0 - neg;  // all ones when negative
  ux<K> r;
  u128_t c = neg;
#pragma unroll
  for (int i = 0; i < K; i++) {
    c += (u128_t)(a.w[i] ^ m);
    r.w[i] = (uint64_t)c;
    c >>= 64;
  }
  return r;
}

// |a| as a signed N-limb value (a >= -2^(64N-1) + 1)
template <int N>
FX_HD fx<N> ix_abs_fx(const fx<N> &a) {
  uint64_t n;
  const ux<N> u = ix_abs<N>(a, n);
  fx<N> r;
#pragma unroll
  for (int i = 0; i < N; i++) r.w[i] = u.w[i];
  return r;
}

// conditional two's-complement negation of an N-limb value
template <int N>
FX_HD void ix_cneg(fx<N> &a, uint64_t neg) {
  const uint64_t m = 0 - neg;
  u128_t c = neg;
#pragma unroll
  for (int i = 0; i < N; i++) {
    c += (u128_t)(a.w[i] ^ m);
    a.w[i] = (uint64_t)c;
    c >>= 64;
  }
}

// Product of unsigned K-limb numbers as 2K limbs.  Exact for K <= 2; for
// K = 4 the partial products a_i b_j with i + j < 2 are left out (they are
// below 2^130, far under the bits the callers keep).
template <int K>
FX_HD ux<2 * K> ix_umul(const ux<K> &a, const ux<K> &b) {
  ux<2 * K> p;
#pragma unroll
  for (int i = 0; i < 2 * K; i++) p.w[i] = 0;
#pragma unroll
  for (int i = 0; i < K; i++) {
    u128_t carry = 0;
#pragma unroll
    for (int j = 0; j < K; j++) {
      if (K == 4 && i + j < 2) continue;
      u128_t t = (u128_t)a.w[i] * b.w[j] + p.w[i + j] + carry;
      p.w[i + j] = (uint64_t)t;
      carry = t >> 64;
    }
    // propagate the row's carry
#pragma unroll
    for (int t = i + K; t < 2 * K; t++) {
      u128_t s = (u128_t)p.w[t] + carry;
      p.w[t] = (uint64_t)s;
      carry = s >> 64;
    }
  }
  return p;
}

// floor(a * b / 2^(64K - 2)) for signed K-limb a, b, as K+1 limbs (signed).
// |result| <= |a| |b| / 2^(64K-2); exact up to the K = 4 truncation above
// (an error below one unit).
template <int K>
FX_HD fx<K + 1> ix_mul_shift(const fx<K> &a, const fx<K> &b) {
  uint64_t na, nb;
  ux<K> ua = ix_abs<K>(a, na), ub = ix_abs<K>(b, nb);
  ux<2 * K> p = ix_umul<K>(ua, ub);
  fx<K + 1> r;
  // bits [64K - 2, 128K) of p: limb t = (p[K-1+t] >> 62) | (p[K+t] << 2)
#pragma unroll
  for (int t = 0; t <= K; t++) {
    uint64_t lo = p.w[K - 1 + t] >> 62;
    uint64_t hi = (K + t < 2 * K) ? (p.w[K + t] << 2) : 0;
    r.w[t] = lo | hi;
  }
  ix_cneg<K + 1>(r, na ^ nb);
  return r;
}

// |a| |b| / 2^(64K - 2) truncated, for unsigned K-limb |a|, |b|: the
// magnitude ix_mul_shift negates (K+1 limbs)
template <int K>
FX_HD fx<K + 1> ix_umul_shift(const ux<K> &ua, const ux<K> &ub) {
  const ux<2 * K> p = ix_umul<K>(ua, ub);
  fx<K + 1> r;
#pragma unroll
  for (int t = 0; t <= K; t++) {
    const uint64_t lo = p.w[K - 1 + t] >> 62;
    const uint64_t hi = (K + t < 2 * K) ? (p.w[K + t] << 2) : 0;
    r.w[t] = lo | hi;
  }
  return r;
}

// a + b when neg = 0, a - b when neg = 1 (N limbs, mod 2^(64N)): b's
// complement and the carry-in of its +1 go into the one addition
template <int N>
FX_HD fx<N> ix_add_cneg(const fx<N> &a, const fx<N> &b, uint64_t neg) {
  const uint64_t m = 0 - neg;
  fx<N> r;
  u128_t c = neg;
#pragma unroll
  for (int i = 0; i < N; i++) {
    c += (u128_t)a.w[i] + (u128_t)(b.w[i] ^ m);
    r.w[i] = (uint64_t)c;
    c >>= 64;
  }
  return r;
}

// a * b exactly for signed KA- and KB-limb values, as KA+KB limbs (signed)
template <int KA, int KB>
FX_HD fx<KA + KB> ix_mul_full(const fx<KA> &a, const fx<KB> &b) {
  uint64_t na, nb;
  const ux<KA> ua = ix_abs<KA>(a, na);
  const ux<KB> ub = ix_abs<KB>(b, nb);
  fx<KA + KB> p;
#pragma unroll
  for (int i = 0; i < KA + KB; i++) p.w[i] = 0;
#pragma unroll
  for (int i = 0; i < KA; i++) {
    u128_t carry = 0;
#pragma unroll
    for (int j = 0; j < KB; j++) {
      u128_t t = (u128_t)ua.w[i] * ub.w[j] + p.w[i + j] + carry;
      p.w[i + j] = (uint64_t)t;
      carry = t >> 64;
    }
    p.w[i + KB] = (uint64_t)carry;
  }
  ix_cneg<KA + KB>(p, na ^ nb);
  return p;
}

// |a|^2 exactly as 2K+1 limbs (unsigned, top limb zero)
template <int K>
FX_HD fx<2 * K + 1> ix_square(const fx<K> &a) {
  uint64_t n;
  ux<K> u = ix_abs<K>(a, n);
  ux<2 * K> p;
  if constexpr (K == 4) {
    // exact square: all 16 partial products
#pragma unroll
    for (int i = 0; i < 2 * K; i++) p.w[i] = 0;
#pragma unroll
    for (int i = 0; i < K; i++) {
      u128_t carry = 0;
#pragma unroll
      for (int j = 0; j < K; j++) {
        u128_t t = (u128_t)u.w[i] * u.w[j] + p.w[i + j] + carry;
        p.w[i + j] = (uint64_t)t;
        carry = t >> 64;
      }
#pragma unroll
      for (int t = i + K; t < 2 * K; t++) {
        u128_t s = (u128_t)p.w[t] + carry;
        p.w[t] = (uint64_t)s;
        carry = s >> 64;
      }
    }
  } else {
    p = ix_umul<K>(u, u);
  }
  fx<2 * K + 1> r;
#pragma unroll
  for (int i = 0; i < 2 * K; i++) r.w[i] = p.w[i];
  r.w[2 * K] = 0;
  return r;
}

// a + b and a - b for signed N-limb values (mod 2^(64N))
template <int N>
FX_HD fx<N> ix_add(fx<N> a, const fx<N> &b) {
  u128_t c = 0;
#pragma unroll
  for (int i = 0; i < N; i++) {
    c += (u128_t)a.w[i] + b.w[i];
    a.w[i] = (uint64_t)c;
    c >>= 64;
  }
  return a;
}

template <int N>
FX_HD fx<N> ix_sub(fx<N> a, const fx<N> &b) {
  u128_t c = 1;
#pragma unroll
  for (int i = 0; i < N; i++) {
    c += (u128_t)a.w[i] + (u128_t)(~b.w[i]);
    a.w[i] = (uint64_t)c;
    c >>= 64;
  }
  return a;
}

// the low K limbs of a signed (K+1)-limb value (caller guarantees it fits)
template <int K>
FX_HD fx<K> ix_narrow(const fx<K + 1> &a) {
  fx<K> r;
#pragma unroll
  for (int i = 0; i < K; i++) r.w[i] = a.w[i];
  return r;
}

// the low N limbs of an M-limb value (caller guarantees it fits)
template <int N, int M>
FX_HD fx<N> ix_low(const fx<M> &a) {
  fx<N> r;
#pragma unroll
  for (int i = 0; i < N; i++) r.w[i] = a.w[i];
  return r;
}

// sign-extend a K-limb value to N limbs
template <int K, int N>
FX_HD fx<N> ix_widen(const fx<K> &a) {
  fx<N> r;
  const uint64_t s = 0 - (a.w[K - 1] >> 63);
#pragma unroll
  for (int i = 0; i < N; i++) r.w[i] = i < K ? a.w[i] : s;
  return r;
}

// bit length of a nonnegative value (0 for zero)
template <int N>
FX_HD int ix_bitlen(const fx<N> &a) {
  int p = 0;
#pragma unroll
  for (int i = N - 1; i >= 0; i--)
    if (p == 0 && a.w[i]) p = 64 * i + 64 - fx_clz64(a.w[i]);
  return p;
}

// a >> s (arithmetic) for 0 <= s < 64 N.  The limb part of the shift is a
// logarithmic barrel (one stage per bit of s / 64, each a select between
// fixed limb positions), so a run-time s never indexes the register array.
template <int N>
FX_HD fx<N> ix_sar(const fx<N> &a, int s) {
  const int q = s >> 6, r = s & 63;
  const uint64_t sign = 0 - (a.w[N - 1] >> 63);
  fx<N> t = a;
#pragma unroll
  for (int m = 1; m < N; m <<= 1) {
    const bool on = (q & m) != 0;
#pragma unroll
    for (int i = 0; i < N; i++) {
      const uint64_t v = (i + m < N) ? t.w[i + m] : sign;
      t.w[i] = on ? v : t.w[i];
    }
  }
  fx<N> o;
#pragma unroll
  for (int i = 0; i < N; i++) {
    const uint64_t hi = (i + 1 < N) ? t.w[i + 1] : sign;
    o.w[i] = r ? ((t.w[i] >> r) | (hi << (64 - r))) : t.w[i];
  }
  return o;
}

// a << s (bits shifted out of the top are lost) for 0 <= s < 64 N, with the
// same barrel structure as ix_sar
template <int N>
FX_HD fx<N> ix_shl(const fx<N> &a, int s) {
  const int q = s >> 6, r = s & 63;
  fx<N> t = a;
#pragma unroll
  for (int m = 1; m < N; m <<= 1) {
    const bool on = (q & m) != 0;
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
      const uint64_t v = (i - m >= 0) ? t.w[i - m] : 0;
      t.w[i] = on ? v : t.w[i];
    }
  }
  fx<N> o;
#pragma unroll
  for (int i = 0; i < N; i++) {
    const uint64_t lo = (i - 1 >= 0) ? t.w[i - 1] : 0;
    o.w[i] = r ? ((t.w[i] << r) | (lo >> (64 - r))) : t.w[i];
  }
  return o;
}

// One Newton step y <- y + y (1 - t y^2) / 2 for y ~ 1/sqrt(t) in K-limb
// fixed point: Y = y 2^(64K-2), tt = t 2^(64K) with t in [1/4, 1).  The
// number of correct bits roughly doubles, up to the resolution of K limbs.
template <int K>
FX_HD void ix_rsqrt_step(const ux<K> &tt, ux<K> &Y) {
  constexpr int S = 64 * K - 2;
  // W = Y^2 / 2^S  (value y^2, scale 2^S), K+1 limbs
  ux<2 * K> y2 = ix_umul<K>(Y, Y);
  ux<K + 1> Wv;
#pragma unroll
  for (int t = 0; t <= K; t++) {
    uint64_t lo = y2.w[K - 1 + t] >> 62;
    uint64_t hi = (K + t < 2 * K) ? (y2.w[K + t] << 2) : 0;
    Wv.w[t] = lo | hi;
  }
  // V = t * W = tt * W / 2^(64K)  (value t y^2 ~ 1, scale 2^S)
  ux<K> Wk;
#pragma unroll
  for (int i = 0; i < K; i++) Wk.w[i] = Wv.w[i];
  ux<2 * K> tw = ix_umul<K>(tt, Wk);
  // tw / 2^(64K): limbs K..2K-1, plus tt * Wv.w[K] (W's top limb) at weight 2^(64K)
  ux<K> V;
#pragma unroll
  for (int i = 0; i < K; i++) V.w[i] = tw.w[K + i];
  {
    u128_t c = 0;
#pragma unroll
    for (int i = 0; i < K; i++) {
      c += (u128_t)V.w[i] + (u128_t)tt.w[i] * Wv.w[K];
      V.w[i] = (uint64_t)c;
      c >>= 64;
    }
  }
  // e = 2^S - V (signed, small), Y <- Y + Y e / 2^(S+1)
  fx<K> one;
#pragma unroll
  for (int i = 0; i < K; i++) one.w[i] = (i == (S >> 6)) ? (1ull << (S & 63)) : 0;
  fx<K> Vf;
#pragma unroll
  for (int i = 0; i < K; i++) Vf.w[i] = V.w[i];
  fx<K> e = ix_sub<K>(one, Vf);
  uint64_t ne;
  ux<K> ue = ix_abs<K>(e, ne);
  ux<2 * K> ye = ix_umul<K>(Y, ue);
  // ye / 2^(S+1) = ye >> (64K - 1)
  fx<K> d;
#pragma unroll
  for (int t = 0; t < K; t++) {
    uint64_t lo = ye.w[K - 1 + t] >> 63;
    uint64_t hi = (K + t < 2 * K) ? (ye.w[K + t] << 1) : 0;
    d.w[t] = lo | hi;
  }
  ix_cneg<K>(d, ne);
  fx<K> Yf;
#pragma unroll
  for (int i = 0; i < K; i++) Yf.w[i] = Y.w[i];
  Yf = ix_add<K>(Yf, d);
#pragma unroll
  for (int i = 0; i < K; i++) Y.w[i] = Yf.w[i];
}

// One higher-order step in K limbs (scale S = 64K - 2): with e = 1 - t y^2,
// 1/sqrt(t) = y (1 - e)^(-1/2) = y (1 + e/2 + 3e^2/8 + 5e^3/16 + ...), so
// y <- y (1 + e/2 + 3e^2/8 + 5e^3/16) leaves a relative error of about
// (35/128) e^4: from |e| <= 2^-36 (one 1-limb Newton step from a seed good
// to 2^-20) below 2^-145, from |e| <= 2^-100 (a 2-limb result) far below
// 2^-256; under one unit of the result either way, where Newton would need
// two steps.  EB: the step applies when |e| < 2^-EB (else returns false and
// leaves Y as it was).  e^2 and e^3 are formed from the 64 bits of |e| below
// 2^(S-EB): eh = |e| / 2^(S-EB-64), e^2 / 2^S = eh^2 / 2^(2EB+128-S) (error
// below 2^(S-2EB-63) units), e^3 / 2^(2S) = (e^2 / 2^S) eh / 2^(EB+64).
template <int K, int EB>
FX_HD bool ix_rsqrt_step3(const ux<K> &tt, ux<K> &Y) {
  constexpr int S = 64 * K - 2;
  constexpr int LO = S - EB - 64;          // eh = |e| >> LO
  constexpr int SH = 2 * EB + 128 - S;     // e^2 / 2^S = eh^2 >> SH
  static_assert(LO >= 0 && SH >= 64 && SH < 128, "guard out of range");
  // W = Y^2 / 2^S (K+1 limbs), V = t W / 2^(64K), e = 2^S - V: as in ix_rsqrt_step
  const ux<2 * K> y2 = ix_umul<K>(Y, Y);
  ux<K + 1> Wv;
#pragma unroll
  for (int t = 0; t <= K; t++) {
    const uint64_t lo = y2.w[K - 1 + t] >> 62;
    const uint64_t hi = (K + t < 2 * K) ? (y2.w[K + t] << 2) : 0;
    Wv.w[t] = lo | hi;
  }
  ux<K> Wk;
#pragma unroll
  for (int i = 0; i < K; i++) Wk.w[i] = Wv.w[i];
  const ux<2 * K> tw = ix_umul<K>(tt, Wk);
  ux<K> V;
#pragma unroll
  for (int i = 0; i < K; i++) V.w[i] = tw.w[K + i];
  {
    u128_t c = 0;
#pragma unroll
    for (int i = 0; i < K; i++) {
      c += (u128_t)V.w[i] + (u128_t)tt.w[i] * Wv.w[K];
      V.w[i] = (uint64_t)c;
      c >>= 64;
    }
  }
  fx<K> one, Vf;
#pragma unroll
  for (int i = 0; i < K; i++) {
    one.w[i] = (i == (S >> 6)) ? (1ull << (S & 63)) : 0;
    Vf.w[i] = V.w[i];
  }
  const fx<K> e = ix_sub<K>(one, Vf);
  uint64_t ne;
  const ux<K> ue = ix_abs<K>(e, ne);
  // |e| < 2^(S-EB): no bit at or above S - EB
  {
    uint64_t hi = 0;
#pragma unroll
    for (int i = 0; i < K; i++) {
      const int b0 = 64 * i;  // limb i holds bits b0 .. b0 + 63
      if (b0 + 63 >= S - EB) hi |= (b0 >= S - EB) ? ue.w[i] : (ue.w[i] >> ((S - EB) - b0));
    }
    if (hi) return false;
  }
  // eh = bits LO .. LO + 63 of |e|
  uint64_t eh;
  {
    const int li = LO >> 6, lb = LO & 63;
    eh = ue.w[li] >> lb;
    if (lb && li + 1 < K) eh |= ue.w[li + 1] << (64 - lb);
  }
  const uint64_t e2 = (uint64_t)(((u128_t)eh * eh) >> SH);  // < 2^(128 - SH)
  // e2 eh < 2^118: for EB + 64 >= 128 (the 4-limb step) the term is zero
  uint64_t e3 = 0;  // < 2^(S - 2EB)
  if constexpr (EB + 64 < 128) e3 = (uint64_t)(((u128_t)e2 * eh) >> (EB + 64));
  // c = e/2 + 3 e^2 / 8 + 5 e^3 / 16 (signed, scale 2^S)
  fx<K> c = ix_sar<K>(e, 1);
  fx<K> t3, t5;
#pragma unroll
  for (int i = 0; i < K; i++) t3.w[i] = t5.w[i] = 0;
  t3.w[0] = (3 * e2) >> 3;
  t5.w[0] = (5 * e3) >> 4;
  ix_cneg<K>(t5, ne);
  c = ix_add<K>(c, t3);
  c = ix_add<K>(c, t5);
  uint64_t nc;
  const ux<K> uc = ix_abs<K>(c, nc);
  // Y <- Y + Y c / 2^S; Y c / 2^S = bits S .. S + 64K - 1 of the product
  const ux<2 * K> yc = ix_umul<K>(Y, uc);
  fx<K> d;
#pragma unroll
  for (int t = 0; t < K; t++) {
    const uint64_t lo = yc.w[K - 1 + t] >> 62;
    const uint64_t hi = yc.w[K + t] << 2;
    d.w[t] = lo | hi;
  }
  ix_cneg<K>(d, nc);
  fx<K> Yf;
#pragma unroll
  for (int i = 0; i < K; i++) Yf.w[i] = Y.w[i];
  Yf = ix_add<K>(Yf, d);
#pragma unroll
  for (int i = 0; i < K; i++) Y.w[i] = Yf.w[i];
  return true;
}

// the top KK limbs of tt, and Y from KK to 2 KK limbs (same value)
template <int K, int KK>
FX_HD ux<KK> ix_top(const ux<K> &tt) {
  ux<KK> r;
#pragma unroll
  for (int i = 0; i < KK; i++) r.w[i] = tt.w[K - KK + i];
  return r;
}

template <int KK>
FX_HD ux<2 * KK> ix_rsqrt_widen(const ux<KK> &Y) {
  ux<2 * KK> r;
#pragma unroll
  for (int i = 0; i < 2 * KK; i++) r.w[i] = i < KK ? 0 : Y.w[i - KK];
  return r;
}

// The steps after the seed: Y1 = y0 2^62 with y0 ~ 1/sqrt(t) to 2^-20 or
// better (one limb at scale 2^62; FP32 rsqrtf is within 2^-21.8).
template <int K>
FX_HD ux<K> ix_rsqrt_from_seed(const ux<K> &tt, ux<1> Y1) {
  static_assert(K == 1 || K == 2 || K == 4, "K = 1, 2 or 4 limbs");
  const ux<1> t1 = ix_top<K, 1>(tt);
  ix_rsqrt_step<1>(t1, Y1);  // ~43 bits
  if constexpr (K == 1) {
    ix_rsqrt_step<1>(t1, Y1);
    return Y1;
  } else {
    ux<2> Y2 = ix_rsqrt_widen<1>(Y1);
    const ux<2> t2 = ix_top<K, 2>(tt);
    if (!ix_rsqrt_step3<2, 36>(t2, Y2)) {  // ~128 bits; else two Newton steps
      ix_rsqrt_step<2>(t2, Y2);
      ix_rsqrt_step<2>(t2, Y2);
    }
    if constexpr (K == 2) {
      return Y2;
    } else {
      ux<4> Y4 = ix_rsqrt_widen<2>(Y2);
      if (!ix_rsqrt_step3<4, 100>(tt, Y4)) {  // ~256 bits
        ix_rsqrt_step<4>(tt, Y4);
        ix_rsqrt_step<4>(tt, Y4);
      }
      return Y4;
    }
  }
}

// Y = 2^(64K-2) / sqrt(t) for t = tt / 2^(64K) in [1/4, 1), tt a K-limb
// unsigned fraction: FP32 reciprocal square root seed (24 bits), then steps
// in as many limbs as their result needs: a Newton step in 1 limb (~43 bits),
// then one more (K = 1), or a third-order step in 2 limbs (~128 bits) and,
// for K = 4, a third-order step in 4 limbs.
// Y is in (2^(64K-2), 2^(64K-1)].
template <int K>
FX_HD ux<K> ix_rsqrt_frac(const ux<K> &tt) {
  // seed from the top 32 bits of t
  const float tf = (float)(uint32_t)(tt.w[K - 1] >> 32) * 2.3283064365386963e-10f;  // 2^-32
#if defined(__CUDA_ARCH__)
  const float y0 = rsqrtf(tf);
#else
  const float y0 = 1.0f / __builtin_sqrtf(tf);
#endif
  // y0 in (1, 2] with 24 significant bits, as one limb at scale 2^62
  ux<1> Y1;
  Y1.w[0] = (uint64_t)(y0 * 16777216.0f) << 38;
  return ix_rsqrt_from_seed<K>(tt, Y1);
}

#if defined(__CUDACC__)
// Exact sum over the warp of an N-limb two's-complement value (modulo
// 2^(64N)), in every lane: each limb in four 16-bit chunks, one warp
// reduction per chunk (sums below 2^21, so no chunk overflows), then one
// carry pass.  The 4N reductions are independent of one another, unlike the
// five dependent shuffle-and-add levels of a butterfly.
template <int N>
__device__ __forceinline__ fx<N> warp_sum_fx(const fx<N> &v) {
  uint32_t c[4 * N];
#pragma unroll
  for (int w = 0; w < N; w++)
#pragma unroll
    for (int h = 0; h < 4; h++)
      c[4 * w + h] = __reduce_add_sync(0xffffffffu, (uint32_t)((v.w[w] >> (16 * h)) & 0xFFFFu));
  fx<N> r;
  uint64_t carry = 0;
#pragma unroll
  for (int w = 0; w < N; w++) {
    const u128_t a = (u128_t)carry + c[4 * w] + ((u128_t)c[4 * w + 1] << 16) +
                     ((u128_t)c[4 * w + 2] << 32) + ((u128_t)c[4 * w + 3] << 48);
    r.w[w] = (uint64_t)a;
    carry = (uint64_t)(a >> 64);
  }
  return r;
}

#endif

}  // namespace gn
