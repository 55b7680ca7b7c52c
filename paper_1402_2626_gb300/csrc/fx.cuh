// fx.cuh — exact fixed-point accumulation of doubles on the integer pipe.
//
// A value V * 2^-F is held as a two's-complement integer V of NL 64-bit limbs
// (little-endian).  Adding a double is exact except that bits below 2^-F are
// dropped (truncation toward zero of the addend's magnitude); additions of
// accumulators are exact and associative, so sums do not depend on their
// order.  Converting back yields a cascade of doubles, each the top 53 bits of
// what the previous ones leave (truncated), so L limbs carry the value to
// within 2^(-52 L) relative.
//
// Why: on GB300 an FP64 warp instruction occupies its SM sub-partition for 64
// cycles, while integer instructions issue about 32 times faster.  Every sum
// of multiword values (inner products, norms, term sums) is therefore formed
// here, in integers, from the exact pieces that FP64 TwoProd gives for each
// product; only the products stay on the FP64 pipe.
//
// The caller picks F from a bound on the magnitudes involved (for instance
// the original norm of a column): with |every partial sum| < 2^(64 NL - 1 - F)
// nothing overflows.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define FX_HD __host__ __device__ __forceinline__
#else
#define FX_HD inline
#endif

namespace gn {

template <int NL>
struct fx {
  uint64_t w[NL];
};

template <int NL>
FX_HD void fx_zero(fx<NL> &a) {
#pragma unroll
  for (int i = 0; i < NL; i++) a.w[i] = 0;
}

FX_HD uint64_t fx_dbits(double d) {
#if defined(__CUDA_ARCH__)
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  __builtin_memcpy(&b, &d, 8);
  return b;
#endif
}

FX_HD double fx_bitsd(uint64_t b) {
#if defined(__CUDA_ARCH__)
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, 8);
  return d;
#endif
}

FX_HD int fx_clz64(uint64_t x) {
#if defined(__CUDA_ARCH__)
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

// a += b + cin (mod 2^(64 NL))
template <int NL>
FX_HD void fx_add_to(fx<NL> &a, const fx<NL> &b, uint64_t cin = 0) {
#if defined(__CUDA_ARCH__)
  if constexpr (NL == 2) {
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;"
        : "+l"(a.w[0]), "+l"(a.w[1])
        : "l"(b.w[0]), "l"(b.w[1]));
  } else if constexpr (NL == 3) {
    asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, %4;\n\taddc.u64 %2, %2, %5;"
        : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2])
        : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]));
  } else if constexpr (NL == 5) {
    asm("add.cc.u64 %0, %0, %5;\n\taddc.cc.u64 %1, %1, %6;\n\taddc.cc.u64 %2, %2, %7;\n\t"
        "addc.cc.u64 %3, %3, %8;\n\taddc.u64 %4, %4, %9;"
        : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2]), "+l"(a.w[3]), "+l"(a.w[4])
        : "l"(b.w[0]), "l"(b.w[1]), "l"(b.w[2]), "l"(b.w[3]), "l"(b.w[4]));
  } else {
    unsigned __int128 c = cin;
    for (int i = 0; i < NL; i++) {
      c += (unsigned __int128)a.w[i] + b.w[i];
      a.w[i] = (uint64_t)c;
      c >>= 64;
    }
    return;
  }
  if (cin) {
    if constexpr (NL == 2) {
      asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, 0;" : "+l"(a.w[0]), "+l"(a.w[1]) : "l"(cin));
    } else if constexpr (NL == 3) {
      asm("add.cc.u64 %0, %0, %3;\n\taddc.cc.u64 %1, %1, 0;\n\taddc.u64 %2, %2, 0;"
          : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2])
          : "l"(cin));
    } else {
      asm("add.cc.u64 %0, %0, %5;\n\taddc.cc.u64 %1, %1, 0;\n\taddc.cc.u64 %2, %2, 0;\n\t"
          "addc.cc.u64 %3, %3, 0;\n\taddc.u64 %4, %4, 0;"
          : "+l"(a.w[0]), "+l"(a.w[1]), "+l"(a.w[2]), "+l"(a.w[3]), "+l"(a.w[4])
          : "l"(cin));
    }
  }
#else
  unsigned __int128 c = cin;
  for (int i = 0; i < NL; i++) {
    c += (unsigned __int128)a.w[i] + b.w[i];
    a.w[i] = (uint64_t)c;
    c >>= 64;
  }
#endif
}

// a += d * 2^F where b holds the bits of d (bits of the addend below 2^0 are
// dropped).  Subnormal and zero addends add nothing.  Returns false when the
// addend does not fit.
template <int NL>
FX_HD bool fx_add_bits(fx<NL> &a, uint64_t b, int F) {
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return true;
  uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  int s = e - 1075 + F;  // fixed-point value = m * 2^s
  if (s < 0) {
    if (s < -63) return true;
    m >>= -s;
    s = 0;
  }
  if (s > 64 * NL - 54) return false;  // top mantissa bit must stay below the sign bit
  const int q = s >> 6, r = s & 63;
  const uint64_t lo = m << r;
  const uint64_t hi = r ? (m >> (64 - r)) : 0;
  const uint64_t mask = (uint64_t)((int64_t)b >> 63);  // all ones for a negative addend
  fx<NL> v;
#pragma unroll
  for (int i = 0; i < NL; i++) {
    uint64_t x = (i == q) ? lo : ((i == q + 1) ? hi : 0);
    v.w[i] = x ^ mask;
  }
  fx_add_to<NL>(a, v, mask & 1);
  return true;
}

template <int NL>
FX_HD bool fx_add_double(fx<NL> &a, double d, int F) {
  return fx_add_bits<NL>(a, fx_dbits(d), F);
}

template <int NL>
FX_HD void fx_neg(fx<NL> &a) {
  fx<NL> z;
#pragma unroll
  for (int i = 0; i < NL; i++) {
    z.w[i] = ~a.w[i];
    a.w[i] = 0;
  }
  fx_add_to<NL>(a, z, 1);
}

// The value a * 2^-F as a cascade of L doubles: limb l is the double nearest
// to what limbs 0..l-1 leave over (ties away from zero), so each limb after
// the first is at most half an ulp of the one before and may have either
// sign.
template <int NL, int L>
FX_HD void fx_to_cascade(fx<NL> a, int F, double (&out)[L]) {
#pragma unroll
  for (int l = 0; l < L; l++) {
    const uint64_t sign = a.w[NL - 1] >> 63;
    fx<NL> u = a;
    if (sign) fx_neg<NL>(u);
    // position p of the top set bit of |a|
    int p = -1;
#pragma unroll
    for (int i = NL - 1; i >= 0; i--)
      if (p < 0 && u.w[i]) p = 64 * i + 63 - fx_clz64(u.w[i]);
    if (p < 0) {
      out[l] = 0.0;
      continue;
    }
    const int lo_bit = p - 52;
    uint64_t m;
    if (lo_bit > 0) {
      // the 53 bits [lo_bit, p], plus the bit below them rounded in
      const int li = lo_bit >> 6, off = lo_bit & 63;
      const int rb = lo_bit - 1, ri = rb >> 6, ro = rb & 63;
      uint64_t w0 = 0, w1 = 0, wr = 0;
#pragma unroll
      for (int i = 0; i < NL; i++) {
        if (i == li) w0 = u.w[i];
        if (i == li + 1) w1 = u.w[i];
        if (i == ri) wr = u.w[i];
      }
      m = ((w0 >> off) | (off ? (w1 << (64 - off)) : 0)) & ((1ull << 53) - 1);
      m += (wr >> ro) & 1;  // m in [2^52, 2^53]
      // u -= m 2^lo_bit (u may turn negative when rounded up)
      fx<NL> v;
#pragma unroll
      for (int i = 0; i < NL; i++) {
        uint64_t x = 0;
        if (i == li) x = m << off;
        if (i == li + 1 && off) x = m >> (64 - off);
        v.w[i] = ~x;
      }
      fx_add_to<NL>(u, v, 1);
    } else {
      m = u.w[0] << (-lo_bit);  // exact: nothing is left over
      fx_zero<NL>(u);
    }
    // a = sign(a) * (|a| - m 2^lo_bit)
    if (sign) fx_neg<NL>(u);
    a = u;
    int E = lo_bit - F;  // limb value m 2^E
    if (m >> 53) {
      m >>= 1;
      E += 1;
    }
    const int biased = E + 1075;
    if (biased <= 0) {
      out[l] = 0.0;  // below the normal range: not produced by the scales used here
      continue;
    }
    if (biased >= 2047) {
      out[l] = fx_bitsd(0x7FF8000000000000ull);  // beyond the double range: NaN
      continue;
    }
    out[l] = fx_bitsd((sign << 63) | ((uint64_t)biased << 52) | (m & 0xFFFFFFFFFFFFFull));
  }
}

// Scale exponent for values bounded by 2^E: F = bits - E, leaving headroom for
// sums of up to 2^(64 NL - 1 - bits) such values.
FX_HD int fx_exponent_of(double bound) {
  const uint64_t b = fx_dbits(bound);
  const int e = (int)((b >> 52) & 0x7FF);
  return e == 0 ? -1022 : e - 1022;  // bound < 2^returned
}

}  // namespace gn
