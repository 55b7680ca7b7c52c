// mw.cuh — complex double (L=1), double double (L=2) and quad double (L=4)
// arithmetic for the device.
//
// The paper computes in double double and quad double (Section 1) but only
// cites their algorithms (Hida-Li-Bailey; Lu-He-Luo).  This file builds them
// from published error-free transformations:
//   TwoSum (Knuth), FastTwoSum (Dekker 1971), TwoProd with one FMA, and
//   renormalisation of a short expansion by cascades of TwoSum (Priest 1991,
//   Shewchuk 1997).
// Square roots and reciprocals start from the hardware double result and
// take Newton steps (Karp-Markstein 1997).
//
// GB300 has about 1/64 of its FP32 rate in FP64, so every routine here is
// written to minimise FP64 instructions (DADD, DMUL and DFMA each count one):
//   * a complex product forms each part as one sum of products of limbs,
//     with all error terms collected before a single renormalisation;
//   * additions are "sloppy" (limb-wise, error relative to |a| + |b|),
//     which is the error model every sum in this library needs: the
//     tolerances are relative to the sum of the magnitudes of the terms;
//   * multiplications by small integers (the exponents of Section 2.3) use
//     TwoProd on each limb.
//
// Layout: cx<L> holds re[L] and im[L]; limb 0 is the leading double.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gn {

#define GN_DEV __device__ __forceinline__

// ---------------------------------------------------------------------------
// error-free transformations (no contraction: explicit _rn intrinsics)
// ---------------------------------------------------------------------------

// s + e == a + b exactly (Knuth's TwoSum, 6 flops)
GN_DEV void two_sum(double a, double b, double &s, double &e) {
  s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// s + e == a + b exactly when exponent(a) >= exponent(b) (Dekker, 3 flops)
GN_DEV void fast_two_sum(double a, double b, double &s, double &e) {
  s = __dadd_rn(a, b);
  e = __dsub_rn(b, __dsub_rn(s, a));
}

// p + e == a * b exactly (2 flops)
GN_DEV void two_prod(double a, double b, double &p, double &e) {
  p = __dmul_rn(a, b);
  e = __fma_rn(a, b, -p);
}

template <int L>
struct cx {
  double re[L];
  double im[L];
};

template <int L>
struct rl {
  double v[L];
};

template <int L>
GN_DEV cx<L> c_zero() {
  cx<L> z;
#pragma unroll
  for (int l = 0; l < L; l++) z.re[l] = z.im[l] = 0.0;
  return z;
}

template <int L>
GN_DEV cx<L> c_one() {
  cx<L> z = c_zero<L>();
  z.re[0] = 1.0;
  return z;
}

template <int L>
GN_DEV cx<L> c_neg(const cx<L> &a) {
  cx<L> z;
#pragma unroll
  for (int l = 0; l < L; l++) {
    z.re[l] = -a.re[l];
    z.im[l] = -a.im[l];
  }
  return z;
}

// ---------------------------------------------------------------------------
// quad double building blocks
// ---------------------------------------------------------------------------

// Renormalise x0 + x1 + x2 + x3 (roughly decreasing, possibly overlapping)
// into 4 limbs; exact except for the last rounding (6 TwoSum, 36 flops).
GN_DEV void qd_renorm(double x0, double x1, double x2, double x3, double (&r)[4]) {
  double s, t0, t1, t2;
  two_sum(x2, x3, s, t2);
  two_sum(x1, s, s, t1);
  two_sum(x0, s, r[0], t0);
  two_sum(t1, t2, s, t2);
  two_sum(t0, s, r[1], t1);
  two_sum(t1, t2, r[2], r[3]);
}

// Sum of NP products sum_k a_k * b_k of quad doubles (signs folded into a).
// Products are grouped by order 2^(-53 j); groups 0..2 are summed with TwoSum
// chains whose errors move one group down; group 3 is summed in plain
// arithmetic (its rounding is of order 2^-212).  Products of order >= 4 are
// dropped (below 2^-212 relative).
template <int NP>
GN_DEV void qd_sum_of_products(const double (&a)[NP][4], const double (&b)[NP][4],
                               double (&r)[4]) {
  double s0, s1, s2, s3 = 0.0;
  double t;
  // order 0
  double p0[NP], e0[NP];
#pragma unroll
  for (int k = 0; k < NP; k++) two_prod(a[k][0], b[k][0], p0[k], e0[k]);
  s0 = p0[0];
  double g1_extra[NP];  // errors of the order-0 sum (order 1)
#pragma unroll
  for (int k = 1; k < NP; k++) {
    two_sum(s0, p0[k], s0, t);
    g1_extra[k] = t;
  }
  // order 1 terms: e0[k], a_k0 b_k1, a_k1 b_k0, g1_extra
  double p01[NP], e01[NP], p10[NP], e10[NP];
#pragma unroll
  for (int k = 0; k < NP; k++) {
    two_prod(a[k][0], b[k][1], p01[k], e01[k]);
    two_prod(a[k][1], b[k][0], p10[k], e10[k]);
  }
  // order 2 products
  double p02[NP], e02[NP], p11[NP], e11[NP], p20[NP], e20[NP];
#pragma unroll
  for (int k = 0; k < NP; k++) {
    two_prod(a[k][0], b[k][2], p02[k], e02[k]);
    two_prod(a[k][1], b[k][1], p11[k], e11[k]);
    two_prod(a[k][2], b[k][0], p20[k], e20[k]);
  }
  // order-3 group in plain arithmetic: products a_i b_j with i + j = 3 and the
  // TwoProd errors of the order-2 products
#pragma unroll
  for (int k = 0; k < NP; k++) {
    s3 = __fma_rn(a[k][0], b[k][3], s3);
    s3 = __fma_rn(a[k][1], b[k][2], s3);
    s3 = __fma_rn(a[k][2], b[k][1], s3);
    s3 = __fma_rn(a[k][3], b[k][0], s3);
    s3 = __dadd_rn(s3, e02[k]);
    s3 = __dadd_rn(s3, e11[k]);
    s3 = __dadd_rn(s3, e20[k]);
  }
  // order-1 group -> s1; its errors are order 2 and join group 2 through s2
  s1 = e0[0];
  s2 = 0.0;
  double u;
#pragma unroll
  for (int k = 0; k < NP; k++) {
    if (k > 0) {
      two_sum(s1, e0[k], s1, t);
      two_sum(s2, t, s2, u);
      s3 = __dadd_rn(s3, u);
      two_sum(s1, g1_extra[k], s1, t);
      two_sum(s2, t, s2, u);
      s3 = __dadd_rn(s3, u);
    }
    two_sum(s1, p01[k], s1, t);
    two_sum(s2, t, s2, u);
    s3 = __dadd_rn(s3, u);
    two_sum(s1, p10[k], s1, t);
    two_sum(s2, t, s2, u);
    s3 = __dadd_rn(s3, u);
  }
  // rest of the order-2 group
#pragma unroll
  for (int k = 0; k < NP; k++) {
    two_sum(s2, e01[k], s2, u);
    s3 = __dadd_rn(s3, u);
    two_sum(s2, e10[k], s2, u);
    s3 = __dadd_rn(s3, u);
    two_sum(s2, p02[k], s2, u);
    s3 = __dadd_rn(s3, u);
    two_sum(s2, p11[k], s2, u);
    s3 = __dadd_rn(s3, u);
    two_sum(s2, p20[k], s2, u);
    s3 = __dadd_rn(s3, u);
  }
  qd_renorm(s0, s1, s2, s3, r);
}

// a + b for quad doubles, limb-wise with carried errors (absolute error of
// order 2^-212 (|a| + |b|)).
GN_DEV void qd_add(const double (&a)[4], const double (&b)[4], double (&r)[4]) {
  double s0, s1, s2, s3, e0, e1, e2, t, u, w;
  two_sum(a[0], b[0], s0, e0);
  two_sum(a[1], b[1], s1, e1);
  two_sum(a[2], b[2], s2, e2);
  s3 = __dadd_rn(a[3], b[3]);
  two_sum(s1, e0, s1, t);
  two_sum(s2, e1, s2, u);
  two_sum(s2, t, s2, w);
  s3 = __dadd_rn(__dadd_rn(s3, e2), __dadd_rn(u, w));
  qd_renorm(s0, s1, s2, s3, r);
}

// d * a for a small integer d (exact products of each limb, then renormalise)
GN_DEV void qd_scale(const double (&a)[4], double d, double (&r)[4]) {
  double p0, p1, p2, p3, e0, e1, e2, s1, s2, t1, t2, t3, s3;
  two_prod(a[0], d, p0, e0);
  two_prod(a[1], d, p1, e1);
  two_prod(a[2], d, p2, e2);
  p3 = __dmul_rn(a[3], d);
  two_sum(p1, e0, s1, t1);
  two_sum(p2, e1, s2, t2);
  two_sum(s2, t1, s2, t3);
  s3 = __dadd_rn(__dadd_rn(p3, e2), __dadd_rn(t2, t3));
  qd_renorm(p0, s1, s2, s3, r);
}

// ---------------------------------------------------------------------------
// double double building blocks
// ---------------------------------------------------------------------------

// a0 b0 + c0 d0 + cross terms: one part of a complex double-double product.
// hi/lo limbs: (a0,a1) (b0,b1) (c0,c1) (d0,d1); error O(2^-104)(|ab| + |cd|).
GN_DEV void dd_two_products(double a0, double a1, double b0, double b1, double c0, double c1,
                            double d0, double d1, double &r0, double &r1) {
  double p1, e1, p2, e2, s, t, lo;
  two_prod(a0, b0, p1, e1);
  two_prod(c0, d0, p2, e2);
  two_sum(p1, p2, s, t);
  lo = __fma_rn(a0, b1, e1);
  lo = __fma_rn(a1, b0, lo);
  lo = __dadd_rn(lo, e2);
  lo = __fma_rn(c0, d1, lo);
  lo = __fma_rn(c1, d0, lo);
  lo = __dadd_rn(lo, t);
  fast_two_sum(s, lo, r0, r1);
}

GN_DEV void dd_add(double a0, double a1, double b0, double b1, double &r0, double &r1) {
  double s, e;
  two_sum(a0, b0, s, e);
  e = __dadd_rn(e, __dadd_rn(a1, b1));
  fast_two_sum(s, e, r0, r1);
}

GN_DEV void dd_mul(double a0, double a1, double b0, double b1, double &r0, double &r1) {
  double p, e;
  two_prod(a0, b0, p, e);
  e = __fma_rn(a0, b1, e);
  e = __fma_rn(a1, b0, e);
  fast_two_sum(p, e, r0, r1);
}

GN_DEV void dd_scale(double a0, double a1, double d, double &r0, double &r1) {
  double p, e;
  two_prod(a0, d, p, e);
  e = __fma_rn(a1, d, e);
  fast_two_sum(p, e, r0, r1);
}

// ---------------------------------------------------------------------------
// generic complex operations
// ---------------------------------------------------------------------------

// a * b
template <int L>
GN_DEV cx<L> c_mul(const cx<L> &a, const cx<L> &b) {
  cx<L> r;
  if constexpr (L == 1) {
    r.re[0] = __fma_rn(a.re[0], b.re[0], -__dmul_rn(a.im[0], b.im[0]));
    r.im[0] = __fma_rn(a.re[0], b.im[0], __dmul_rn(a.im[0], b.re[0]));
  } else if constexpr (L == 2) {
    dd_two_products(a.re[0], a.re[1], b.re[0], b.re[1], -a.im[0], -a.im[1], b.im[0], b.im[1],
                    r.re[0], r.re[1]);
    dd_two_products(a.re[0], a.re[1], b.im[0], b.im[1], a.im[0], a.im[1], b.re[0], b.re[1],
                    r.im[0], r.im[1]);
  } else {
    double A[2][4], B[2][4];
#pragma unroll
    for (int l = 0; l < 4; l++) {
      A[0][l] = a.re[l];
      B[0][l] = b.re[l];
      A[1][l] = -a.im[l];
      B[1][l] = b.im[l];
    }
    qd_sum_of_products<2>(A, B, r.re);
#pragma unroll
    for (int l = 0; l < 4; l++) {
      A[0][l] = a.re[l];
      B[0][l] = b.im[l];
      A[1][l] = a.im[l];
      B[1][l] = b.re[l];
    }
    qd_sum_of_products<2>(A, B, r.im);
  }
  return r;
}

// conj(a) * b (the inner products q^H a of Section 3)
template <int L>
GN_DEV cx<L> c_conj_mul(const cx<L> &a, const cx<L> &b) {
  cx<L> ac;
#pragma unroll
  for (int l = 0; l < L; l++) {
    ac.re[l] = a.re[l];
    ac.im[l] = -a.im[l];
  }
  return c_mul<L>(ac, b);
}

template <int L>
GN_DEV cx<L> c_add(const cx<L> &a, const cx<L> &b) {
  cx<L> r;
  if constexpr (L == 1) {
    r.re[0] = __dadd_rn(a.re[0], b.re[0]);
    r.im[0] = __dadd_rn(a.im[0], b.im[0]);
  } else if constexpr (L == 2) {
    dd_add(a.re[0], a.re[1], b.re[0], b.re[1], r.re[0], r.re[1]);
    dd_add(a.im[0], a.im[1], b.im[0], b.im[1], r.im[0], r.im[1]);
  } else {
    qd_add(a.re, b.re, r.re);
    qd_add(a.im, b.im, r.im);
  }
  return r;
}

template <int L>
GN_DEV cx<L> c_sub(const cx<L> &a, const cx<L> &b) {
  return c_add<L>(a, c_neg<L>(b));
}

// d * a for a small positive integer d
template <int L>
GN_DEV cx<L> c_scale_int(const cx<L> &a, int d) {
  cx<L> r;
  const double dd = (double)d;
  if constexpr (L == 1) {
    r.re[0] = __dmul_rn(a.re[0], dd);
    r.im[0] = __dmul_rn(a.im[0], dd);
  } else if constexpr (L == 2) {
    dd_scale(a.re[0], a.re[1], dd, r.re[0], r.re[1]);
    dd_scale(a.im[0], a.im[1], dd, r.im[0], r.im[1]);
  } else {
    qd_scale(a.re, dd, r.re);
    qd_scale(a.im, dd, r.im);
  }
  return r;
}

// a * s for a real s at precision L
template <int L>
GN_DEV cx<L> c_mul_real(const cx<L> &a, const rl<L> &s) {
  cx<L> r;
  if constexpr (L == 1) {
    r.re[0] = __dmul_rn(a.re[0], s.v[0]);
    r.im[0] = __dmul_rn(a.im[0], s.v[0]);
  } else if constexpr (L == 2) {
    dd_mul(a.re[0], a.re[1], s.v[0], s.v[1], r.re[0], r.re[1]);
    dd_mul(a.im[0], a.im[1], s.v[0], s.v[1], r.im[0], r.im[1]);
  } else {
    double A[1][4], B[1][4];
#pragma unroll
    for (int l = 0; l < 4; l++) {
      A[0][l] = a.re[l];
      B[0][l] = s.v[l];
    }
    qd_sum_of_products<1>(A, B, r.re);
#pragma unroll
    for (int l = 0; l < 4; l++) A[0][l] = a.im[l];
    qd_sum_of_products<1>(A, B, r.im);
  }
  return r;
}

// |a|^2 as a real at precision L
template <int L>
GN_DEV rl<L> c_abs2(const cx<L> &a) {
  rl<L> r;
  if constexpr (L == 1) {
    r.v[0] = __fma_rn(a.re[0], a.re[0], __dmul_rn(a.im[0], a.im[0]));
  } else if constexpr (L == 2) {
    dd_two_products(a.re[0], a.re[1], a.re[0], a.re[1], a.im[0], a.im[1], a.im[0], a.im[1],
                    r.v[0], r.v[1]);
  } else {
    double A[2][4];
#pragma unroll
    for (int l = 0; l < 4; l++) {
      A[0][l] = a.re[l];
      A[1][l] = a.im[l];
    }
    qd_sum_of_products<2>(A, A, r.v);
  }
  return r;
}

template <int L>
GN_DEV rl<L> r_add(const rl<L> &a, const rl<L> &b) {
  rl<L> r;
  if constexpr (L == 1) {
    r.v[0] = __dadd_rn(a.v[0], b.v[0]);
  } else if constexpr (L == 2) {
    dd_add(a.v[0], a.v[1], b.v[0], b.v[1], r.v[0], r.v[1]);
  } else {
    qd_add(a.v, b.v, r.v);
  }
  return r;
}

template <int L>
GN_DEV rl<L> r_mul(const rl<L> &a, const rl<L> &b) {
  rl<L> r;
  if constexpr (L == 1) {
    r.v[0] = __dmul_rn(a.v[0], b.v[0]);
  } else if constexpr (L == 2) {
    dd_mul(a.v[0], a.v[1], b.v[0], b.v[1], r.v[0], r.v[1]);
  } else {
    double A[1][4], B[1][4];
#pragma unroll
    for (int l = 0; l < 4; l++) {
      A[0][l] = a.v[l];
      B[0][l] = b.v[l];
    }
    qd_sum_of_products<1>(A, B, r.v);
  }
  return r;
}

// 1 / b: Newton steps y <- y + y (1 - b y) from the double reciprocal
template <int L>
GN_DEV rl<L> r_recip(const rl<L> &b) {
  rl<L> y;
#pragma unroll
  for (int l = 0; l < L; l++) y.v[l] = 0.0;
  y.v[0] = 1.0 / b.v[0];
  if constexpr (L > 1) {
    constexpr int iters = (L == 2) ? 1 : 2;
#pragma unroll
    for (int it = 0; it < iters + 1; it++) {
      rl<L> by = r_mul<L>(b, y);
      rl<L> one_minus;
#pragma unroll
      for (int l = 0; l < L; l++) one_minus.v[l] = -by.v[l];
      rl<L> one;
#pragma unroll
      for (int l = 0; l < L; l++) one.v[l] = 0.0;
      one.v[0] = 1.0;
      one_minus = r_add<L>(one, one_minus);
      y = r_add<L>(y, r_mul<L>(y, one_minus));
    }
  }
  return y;
}

// sqrt(a), a >= 0: Newton steps s <- s + (a - s^2) / (2 s) from the double sqrt
template <int L>
GN_DEV rl<L> r_sqrt(const rl<L> &a) {
  rl<L> s;
#pragma unroll
  for (int l = 0; l < L; l++) s.v[l] = 0.0;
  if (!(a.v[0] > 0.0)) return s;
  s.v[0] = sqrt(a.v[0]);
  if constexpr (L > 1) {
    constexpr int iters = (L == 2) ? 1 : 2;
#pragma unroll
    for (int it = 0; it < iters + 1; it++) {
      rl<L> ss = r_mul<L>(s, s);
#pragma unroll
      for (int l = 0; l < L; l++) ss.v[l] = -ss.v[l];
      rl<L> res = r_add<L>(a, ss);  // a - s^2
      rl<L> h;
#pragma unroll
      for (int l = 0; l < L; l++) h.v[l] = 0.0;
      h.v[0] = 0.5 / s.v[0];
      s = r_add<L>(s, r_mul<L>(res, h));
    }
  }
  return s;
}

// ---------------------------------------------------------------------------
// loads and stores of the [re limbs | im limbs] layout
// ---------------------------------------------------------------------------

template <int L>
GN_DEV cx<L> c_load(const double *p) {
  cx<L> z;
  if constexpr (L == 1) {
    double2 v = *reinterpret_cast<const double2 *>(p);
    z.re[0] = v.x;
    z.im[0] = v.y;
  } else if constexpr (L == 2) {
    double2 v0 = reinterpret_cast<const double2 *>(p)[0];
    double2 v1 = reinterpret_cast<const double2 *>(p)[1];
    z.re[0] = v0.x;
    z.re[1] = v0.y;
    z.im[0] = v1.x;
    z.im[1] = v1.y;
  } else {
#pragma unroll
    for (int h = 0; h < 2; h++) {
      double2 v0 = reinterpret_cast<const double2 *>(p)[2 * h];
      double2 v1 = reinterpret_cast<const double2 *>(p)[2 * h + 1];
      double *dst = h ? z.im : z.re;
      dst[0] = v0.x;
      dst[1] = v0.y;
      dst[2] = v1.x;
      dst[3] = v1.y;
    }
  }
  return z;
}

template <int L>
GN_DEV void c_store(double *p, const cx<L> &z) {
  if constexpr (L == 1) {
    *reinterpret_cast<double2 *>(p) = make_double2(z.re[0], z.im[0]);
  } else if constexpr (L == 2) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(z.re[0], z.re[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(z.im[0], z.im[1]);
  } else {
    reinterpret_cast<double2 *>(p)[0] = make_double2(z.re[0], z.re[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(z.re[2], z.re[3]);
    reinterpret_cast<double2 *>(p)[2] = make_double2(z.im[0], z.im[1]);
    reinterpret_cast<double2 *>(p)[3] = make_double2(z.im[2], z.im[3]);
  }
}

}  // namespace gn
