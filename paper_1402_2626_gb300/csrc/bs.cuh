// bs.cuh — the two steps of back substitution (Section 3, eq. 5) on the
// integer mantissas MGS leaves: x_l from y_l and 1/r_ll, and the update of a
// row's y by r_il x_l.  y is fixed point at the scale of the last column
// (K+2 limbs), x_l block floating point (K-limb mantissas, one exponent).
#pragma once

#include "ifx.cuh"

namespace gn {

// x = y 2^sig * Z 2^e as a K-limb mantissa per part and the exponent t
template <int K, int KY>
__device__ __forceinline__ void bs_solve(const fx<KY> &yr, const fx<KY> &yi, const fx<K> &Z, int e,
                                         int sig, fx<K> &Xr, fx<K> &Xi, int &t) {
  uint64_t nz;
  const ux<K> uz = ix_abs<K>(Z, nz);
  fx<KY + K> P[2];
  int B = 0;
#pragma unroll
  for (int part = 0; part < 2; part++) {
    uint64_t ny;
    const ux<KY> uy = ix_abs<KY>(part ? yi : yr, ny);
    // |y| |Z| as KY + K limbs
#pragma unroll
    for (int w = 0; w < KY + K; w++) P[part].w[w] = 0;
#pragma unroll
    for (int a = 0; a < KY; a++) {
      u128_t carry = 0;
#pragma unroll
      for (int b = 0; b < K; b++) {
        u128_t tt = (u128_t)uy.w[a] * uz.w[b] + P[part].w[a + b] + carry;
        P[part].w[a + b] = (uint64_t)tt;
        carry = tt >> 64;
      }
      P[part].w[a + K] = (uint64_t)carry;
    }
    const int bl = ix_bitlen<KY + K>(P[part]);
    B = bl > B ? bl : B;
    ix_cneg<KY + K>(P[part], ny ^ nz);
  }
  const int sh = B > 64 * K - 2 ? B - (64 * K - 2) : 0;
  const fx<KY + K> qr = ix_sar<KY + K>(P[0], sh), qi = ix_sar<KY + K>(P[1], sh);
#pragma unroll
  for (int w = 0; w < K; w++) {
    Xr.w[w] = qr.w[w];
    Xi.w[w] = qi.w[w];
  }
  t = sig + e + sh;
}

// (yr, yi) -= r x, with r x at scale 2^d relative to the units of y
template <int K, int KY>
__device__ __forceinline__ void bs_update(fx<KY> &yr, fx<KY> &yi, const fx<K> &rr, const fx<K> &ri,
                                          const fx<K> &xr, const fx<K> &xi, int d, int *sFail) {
  // re = rr xr - ri xi, im = rr xi + ri xr as 2K+1 limbs
  fx<2 * K + 1> pr, pi;
  {
    uint64_t n1, n2, n3, n4;
    ux<K> a1 = ix_abs<K>(rr, n1), b1 = ix_abs<K>(xr, n2);
    ux<K> a2 = ix_abs<K>(ri, n3), b2 = ix_abs<K>(xi, n4);
    ux<2 * K> p1 = ix_umul<K>(a1, b1), p2 = ix_umul<K>(a2, b2);
    ux<2 * K> p3 = ix_umul<K>(a1, b2), p4 = ix_umul<K>(a2, b1);
    fx<2 * K + 1> f1, f2, f3, f4;
#pragma unroll
    for (int w = 0; w < 2 * K; w++) {
      f1.w[w] = p1.w[w];
      f2.w[w] = p2.w[w];
      f3.w[w] = p3.w[w];
      f4.w[w] = p4.w[w];
    }
    f1.w[2 * K] = f2.w[2 * K] = f3.w[2 * K] = f4.w[2 * K] = 0;
    ix_cneg<2 * K + 1>(f1, n1 ^ n2);
    ix_cneg<2 * K + 1>(f2, n3 ^ n4);
    ix_cneg<2 * K + 1>(f3, n1 ^ n4);
    ix_cneg<2 * K + 1>(f4, n3 ^ n2);
    pr = ix_sub<2 * K + 1>(f1, f2);
    pi = ix_add<2 * K + 1>(f3, f4);
  }
  fx<KY> ur, ui;
  if (d <= 0) {
    const int s = -d;
    if (s >= 64 * (2 * K + 1)) {
      fx_zero<KY>(ur);
      fx_zero<KY>(ui);
    } else {
      const fx<2 * K + 1> qr = ix_sar<2 * K + 1>(pr, s), qi = ix_sar<2 * K + 1>(pi, s);
#pragma unroll
      for (int w = 0; w < KY; w++) {
        ur.w[w] = w < 2 * K + 1 ? qr.w[w] : (0 - (qr.w[2 * K] >> 63));
        ui.w[w] = w < 2 * K + 1 ? qi.w[w] : (0 - (qi.w[2 * K] >> 63));
      }
    }
  } else {
    // a product larger than the units of y by 2^d: only harmless when tiny
    if (ix_bitlen<2 * K + 1>(pr) + d > 64 * KY - 2 || ix_bitlen<2 * K + 1>(pi) + d > 64 * KY - 2)
      *sFail = 1;
#pragma unroll
    for (int w = 0; w < KY; w++) {
      ur.w[w] = w < 2 * K + 1 ? pr.w[w] : (0 - (pr.w[2 * K] >> 63));
      ui.w[w] = w < 2 * K + 1 ? pi.w[w] : (0 - (pi.w[2 * K] >> 63));
    }
    // shift left by d (d < 64 KY guaranteed by the check above when it succeeds)
    const int dd = d < 64 * KY ? d : 64 * KY - 1;
    ur = ix_shl<KY>(ur, dd);
    ui = ix_shl<KY>(ui, dd);
  }
  yr = ix_sub<KY>(yr, ur);
  yi = ix_sub<KY>(yi, ui);
}

}  // namespace gn
