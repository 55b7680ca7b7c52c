// cholqr.cu — the double-precision factorisation of the mixed-precision
// solver as CholeskyQR: R of [A b] = QR from the Gram matrix G = [A b]^H [A b]
// = R^H R, without forming Q.
//
// Section 5.2 of Verschelde & Yu finds the linear solve dominant and points
// to methods in double arithmetic; the mixed solver (mixed.cu) needs one
// double factorisation per double Gauss-Newton step.  For a tall matrix MGS
// (Section 3) is a chain of n dependent pivots whose bulk updates of the
// later columns set its pace; here the O(m n^2) work becomes one
// throughput-bound contraction, the exact Gram matrix of the columns'
// mantissas: on the tensor cores as products of 7-bit digit planes
// (gram_tc.cu, the columns rounded to 56 bits), else on the integer pipe
// (k_cq_gram below, 62 bits), and only an O(n^3 / 3) Cholesky is left, in
// float-float on the FP32 pipe (below).  The factor's last column is y = R^-H A^H b and R_nn = ||b - A x||,
// as MGS on [A b] gives them (eq. 2), so the Gauss-Newton step is R dx = y;
// it and the refinement's R^H w = A^H b, R dx = w are blocked substitutions
// with the float-float factor on one cluster (below).
//
// Accuracy: R from the Cholesky of the Gram matrix has a relative error of
// about kappa(A)^2 u (against kappa u for MGS), u = 2^-47 for the
// float-float Cholesky; the refinement only needs the factors to contract,
// which they do for kappa(A)^2 u << 1 (the mixed workload's Jacobian has
// kappa = 15).  Rank: a pivot below
// 2^-40 of its column's squared norm (kappa above about 10^6, where the
// double refinement would not converge) is reported as GN_ESINGULAR.
#include <cooperative_groups.h>

#include <mutex>
#include <type_traits>

#include "ifx.cuh"
#include "internal.h"

namespace gn {

namespace cg = cooperative_groups;

constexpr int CQ_T = 32;        // tile width of the Gram matrix and of the Cholesky panels
constexpr int CQ_THREADS = 256;
constexpr int CQ_S = 62;        // mantissa scale of the one-limb columns: |M| < 2^62

// Column norms (double) and scale exponents of [A b] (double complex, N x nc,
// column-major, leading dimension N): s_j with ||a_j|| < 2^(62 + s_j), so
// every entry of column j is a 62-bit mantissa at 2^s_j; a NaN or an
// infinity anywhere is GN_ENONFINITE.  One warp per column.
__global__ void k_cq_scale(const double *__restrict__ A, int32_t N, int32_t nc, double *__restrict__ nrm0,
                           double *__restrict__ sexp, int32_t *__restrict__ status) {
  const int j = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (j >= nc) return;  // whole warps
  const double *a = A + (int64_t)j * N * 2;
  double s = 0.0;
  for (int i = lane; i < N; i += 32) s = fma(a[2 * i], a[2 * i], fma(a[2 * i + 1], a[2 * i + 1], s));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const double n0 = sqrt(s);
    if (!isfinite(n0)) atomicCAS(status, GN_OK, GN_ENONFINITE);
    nrm0[j] = n0;
    sexp[j] = (double)(fx_exponent_of(n0 * 1.0000001 + 1e-300) - CQ_S);
  }
}

// the tile (ib, jb), ib <= jb, of linear index t (column-by-column order)
__device__ __forceinline__ void cq_tile(int t, int &ib, int &jb) {
  int j = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((j + 1) * (j + 2) / 2 <= t) j++;
  while (j * (j + 1) / 2 > t) j--;
  jb = j;
  ib = t - j * (j + 1) / 2;
}

// acc (128-bit two's complement) += (hi, lo), one carry chain
__device__ __forceinline__ void cq_add(uint64_t (&acc)[2], uint64_t lo, uint64_t hi) {
  asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(acc[0]), "+l"(acc[1]) : "l"(lo), "l"(hi));
}

// acc += a b for signed 64-bit a, b: the 128-bit product from one low and one
// signed high multiply
__device__ __forceinline__ void cq_mac(uint64_t (&acc)[2], int64_t a, int64_t b) {
  cq_add(acc, (uint64_t)a * (uint64_t)b, (uint64_t)__mul64hi(a, b));
}

// G_ij = sum_r conj(a_ri) a_rj for i <= j (the upper triangle of G, column-
// major, leading dimension nc), exactly: the entries as 62-bit mantissas at
// their columns' scales (fx_add_double: |M| < 2^62 and, the scale coming
// from the column norm, sum_r |M_r|^2 < 2^124), the sums in 128-bit
// accumulators, rounded to a double once at the end.  Each complex product
// takes three real ones (Gauss): with s = ar - ai on the i side and
// d1 = bi - br, d2 = br + bi on the j side (all below 2^63),
//   conj(a) b = (br s + ai d2) + i (br s + ar d1),
// exact in integers.  By Cauchy-Schwarz every partial sum of br s, of ai d2
// and of ar d1 over rows is below 2^124.5 (|s|^2, |d1|^2, |d2|^2 sum to at
// most twice the column's), so each accumulated part stays below 2^126 and
// the 128-bit two's complement never wraps, for any N.  One CTA per 32 x 32 tile (ib <= jb) of 256 threads,
// thread (ty, tx) owning entries (2 ty + {0,1}, 2 tx + {0,1}); rows in
// chunks of 32 staged in shared memory as mantissas with those sums.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_gram(const double *__restrict__ A, int32_t N, int32_t nc,
                                                        const double *__restrict__ sexp,
                                                        double *__restrict__ G,
                                                        const int32_t *__restrict__ status) {
  __shared__ int64_t sI[CQ_T][CQ_T][3];  // [row][column of the i tile]: ar, ai, ar - ai
  __shared__ int64_t sJ[CQ_T][CQ_T][3];  // [row][column of the j tile]: br, bi - br, br + bi
  if (*status != GN_OK) return;
  int ib, jb;
  cq_tile(blockIdx.x, ib, jb);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  uint64_t cr[2][2][2], ci[2][2][2];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++)
#pragma unroll
      for (int w = 0; w < 2; w++) cr[a][b][w] = ci[a][b][w] = 0;
  for (int r0 = 0; r0 < N; r0 += CQ_T) {
    // stage rows r0 .. r0+31 of both tiles' columns: consecutive threads take
    // consecutive rows of one column (coalesced complex loads)
#pragma unroll
    for (int q = 0; q < (CQ_T * CQ_T) / CQ_THREADS; q++) {
      const int idx = tid + q * CQ_THREADS, rr = idx % CQ_T, cc = idx / CQ_T;
      const int r = r0 + rr;
#pragma unroll
      for (int side = 0; side < 2; side++) {
        const int col = (side ? jb : ib) * CQ_T + cc;
        fx<1> mr, mi;
        fx_zero<1>(mr);
        fx_zero<1>(mi);
        if (r < N && col < nc) {
          const double *e = A + ((int64_t)col * N + r) * 2;
          const int F = -(int)sexp[col];
          fx_add_double<1>(mr, e[0], F);
          fx_add_double<1>(mi, e[1], F);
        }
        const int64_t xr = (int64_t)mr.w[0], xi = (int64_t)mi.w[0];
        if (side) {
          sJ[rr][cc][0] = xr;
          sJ[rr][cc][1] = xi - xr;
          sJ[rr][cc][2] = xr + xi;
        } else {
          sI[rr][cc][0] = xr;
          sI[rr][cc][1] = xi;
          sI[rr][cc][2] = xr - xi;
        }
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < CQ_T; rr++) {
      int64_t ar[2], ai[2], as[2], br[2], d1[2], d2[2];
#pragma unroll
      for (int a = 0; a < 2; a++) {
        ar[a] = sI[rr][2 * ty + a][0];
        ai[a] = sI[rr][2 * ty + a][1];
        as[a] = sI[rr][2 * ty + a][2];
        br[a] = sJ[rr][2 * tx + a][0];
        d1[a] = sJ[rr][2 * tx + a][1];
        d2[a] = sJ[rr][2 * tx + a][2];
      }
#pragma unroll
      for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
          const uint64_t lo = (uint64_t)br[b] * (uint64_t)as[a];  // br s, shared by both parts
          const uint64_t hi = (uint64_t)__mul64hi(br[b], as[a]);
          cq_add(cr[a][b], lo, hi);
          cq_add(ci[a][b], lo, hi);
          cq_mac(cr[a][b], ai[a], d2[b]);
          cq_mac(ci[a][b], ar[a], d1[b]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const int i = ib * CQ_T + 2 * ty + a, j = jb * CQ_T + 2 * tx + b;
      if (i < nc && j < nc && i <= j) {
        const int F = -((int)sexp[i] + (int)sexp[j]);
        fx<3> vr, vi;
#pragma unroll
        for (int w = 0; w < 2; w++) {
          vr.w[w] = cr[a][b][w];
          vi.w[w] = ci[a][b][w];
        }
        vr.w[2] = (uint64_t)((int64_t)cr[a][b][1] >> 63);  // sign extension
        vi.w[2] = (uint64_t)((int64_t)ci[a][b][1] >> 63);
        double re[1], im[1];
        fx_to_cascade<3, 1>(vr, F, re);
        fx_to_cascade<3, 1>(vi, F, im);
        G[((int64_t)j * nc + i) * 2] = re[0];
        G[((int64_t)j * nc + i) * 2 + 1] = im[0];
      }
    }
}

// ---- float-float arithmetic on the FP32 pipe ----
//
// The Cholesky runs on values h + l of two floats (about 47 significant
// bits): GB300 issues 64 FP32 lanes for every FP64 lane, and the refinement
// needs the double factors only to contract (their error, about
// kappa^2 2^-47, stays far below the contraction the frozen Jacobian
// allows).  Sums follow Knuth's TwoSum with Dekker's renormalisation,
// products the FMA form of Dekker's TwoProduct (Dekker 1971; Knuth, TAOCP
// vol. 2, 4.2.2).  The Gram matrix is scaled by its columns' powers of two
// first, G^_ij = G_ij 2^-(s_i + 62) 2^-(s_j + 62), so every entry lies in
// [-1, 1] and the float exponent range holds it; then R = R^ D with
// D = diag(2^(s_j + 62)).

struct ffv {
  float h, l;
};
struct cff {
  ffv re, im;
};

__device__ __forceinline__ ffv ff_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

__device__ __forceinline__ double ff_to(ffv a) { return (double)a.h + (double)a.l; }

// (the _rn intrinsics are never fused into FMAs, which would break the
// error terms)
__device__ __forceinline__ ffv ff_add(ffv a, ffv b) {
  const float s = __fadd_rn(a.h, b.h), bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ ffv ff_neg(ffv a) { return {-a.h, -a.l}; }

__device__ __forceinline__ ffv ff_mul(ffv a, ffv b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float h = __fadd_rn(p, e);
  return {h, __fsub_rn(e, __fsub_rn(h, p))};
}

// 1 / sqrt(d) for d > 0: the FP32 estimate and two Newton steps
// y <- y + y (1 - d y^2) / 2 in float-float
__device__ __forceinline__ ffv ff_rsqrt(ffv d) {
  ffv y = {rsqrtf(d.h), 0.f};
#pragma unroll
  for (int it = 0; it < 2; it++) {
    const ffv e = ff_add({1.f, 0.f}, ff_neg(ff_mul(d, ff_mul(y, y))));
    const ffv t = ff_mul(y, e);
    y = ff_add(y, {__fmul_rn(0.5f, t.h), __fmul_rn(0.5f, t.l)});
  }
  return y;
}

// 1 / d for d > 0: the FP32 reciprocal and two Newton steps y += y (1 - d y)
__device__ __forceinline__ ffv ff_recip(ffv d) {
  ffv y = {__frcp_rn(d.h), 0.f};
#pragma unroll
  for (int it = 0; it < 2; it++) {
    const ffv e = ff_add({1.f, 0.f}, ff_neg(ff_mul(d, y)));
    y = ff_add(y, ff_mul(y, e));
  }
  return y;
}

// g -= conj(a) b
__device__ __forceinline__ void cff_sub_conj_mul(cff &g, const cff &a, const cff &b) {
  const ffv re = ff_add(ff_mul(a.re, b.re), ff_mul(a.im, b.im));
  const ffv im = ff_add(ff_mul(a.re, b.im), ff_neg(ff_mul(a.im, b.re)));
  g.re = ff_add(g.re, ff_neg(re));
  g.im = ff_add(g.im, ff_neg(im));
}

__device__ __forceinline__ cff cff_scale(const cff &a, ffv s) { return {ff_mul(a.re, s), ff_mul(a.im, s)}; }

// one complex entry of the scaled matrix: four floats where the double
// complex entry was
__device__ __forceinline__ cff cff_ld(const double *G, int64_t at) {
  const float4 v = *(const float4 *)(G + at * 2);
  return {{v.x, v.y}, {v.z, v.w}};
}

__device__ __forceinline__ void cff_st(double *G, int64_t at, const cff &a) {
  *(float4 *)(G + at * 2) = make_float4(a.re.h, a.re.l, a.im.h, a.im.l);
}

// G (double complex, upper triangle, leading dimension nc) into G^ in
// float-float, in place; thread per entry of the upper triangle's columns
__global__ void k_cq_to_ff(double *__restrict__ G, int32_t nc, const double *__restrict__ sexp,
                           const int32_t *__restrict__ status) {
  if (*status != GN_OK) return;
  const int j = blockIdx.x;
  const int sj = (int)sexp[j] + CQ_S;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const int64_t at = (int64_t)j * nc + i;
    const int sc = -(sj + (int)sexp[i] + CQ_S);
    const double re = ldexp(G[at * 2], sc), im = ldexp(G[at * 2 + 1], sc);
    cff_st(G, at, {ff_from(re), ff_from(im)});
  }
}

// The panel's diagonal block G^[p:pe, p:pe] = R11^H R11 (upper, in place)
// by one CTA in shared memory, right-looking on the unscaled rows: with
// pivot d_k = g_kk final, every g_ij with k < i <= j less conj(g_ki) g_kj / d_k
// (= conj(r_ki) r_kj), so a step needs the reciprocal of its pivot only; the
// square roots and the rows' scaling, r_kj = g_kj / sqrt(d_k), follow for all
// rows at once at the end.  The pairs (i, j), 1 <= i <= j < 32, are listed by
// decreasing i, so the pairs still to update after row k are the first
// (31 - k)(32 - k) / 2 of the list and a step's threads are packed into whole
// warps.  The thread of pair (k + 1, k + 1) takes the next pivot as soon as
// it has updated it: one barrier per step.  A pivot d_k <= 2^-40 ||a_k||^2
// (k < nchk; in the scaled units) records GN_ESINGULAR.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_potrf(double *__restrict__ G, int32_t nc, int32_t p,
                                                         const double *__restrict__ nrm0,
                                                         const double *__restrict__ sexp, int32_t nchk,
                                                         int32_t *__restrict__ status) {
  constexpr int NPAIR = (CQ_T - 1) * CQ_T / 2;  // 496 pairs with i >= 1
  static_assert(NPAIR <= 2 * CQ_THREADS, "two pairs per thread");
  __shared__ cff sB[CQ_T][CQ_T];           // [row][column]
  __shared__ unsigned short sPair[NPAIR];  // i << 8 | j
  __shared__ ffv sInv[CQ_T];               // 1 / d_k, then 1 / sqrt(d_k)
  __shared__ float sThr[CQ_T];             // the rank test's pivot thresholds
  __shared__ int sBad;
  if (*status != GN_OK) return;
  const int pb = min(CQ_T, nc - p);
  const int tid = threadIdx.x;
  if (tid < pb) {
    const float n0 = (float)ldexp(nrm0[p + tid], -((int)sexp[p + tid] + CQ_S));  // in (1/2, 1]
    sThr[tid] = ldexpf(n0 * n0, -40);
  }
  for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
    const int i = q % CQ_T, j = q / CQ_T;
    cff v = {{0.f, 0.f}, {0.f, 0.f}};
    if (i < pb && j < pb && i <= j) v = cff_ld(G, (int64_t)(p + j) * nc + p + i);
    sB[i][j] = v;
  }
  if (tid >= 1 && tid < CQ_T) {  // row i = tid starts after the rows below it
    const int i = tid, base = (CQ_T - 1 - i) * (CQ_T - i) / 2;
    for (int j = i; j < CQ_T; j++) sPair[base + j - i] = (unsigned short)(i << 8 | j);
  }
  if (tid == 0) sBad = 0;
  __syncthreads();
  // the pivot d_k (its thread only): the rank test and 1 / d_k
  auto pivot = [&](int k) {
    const ffv d = sB[k][k].re;
    const bool bad = !(d.h > sThr[k]);
    if (bad && p + k < nchk) {
      atomicCAS(status, GN_OK, GN_ESINGULAR);
      sBad = 1;
    }
    sInv[k] = d.h > 0.f ? ff_recip(d) : ffv{0.f, 0.f};
  };
  if (tid == 0) pivot(0);
  for (int k = 0; k + 1 < pb; k++) {
    __syncthreads();
    if (sBad) return;  // uniform: read after the barrier
    const ffv inv = sInv[k];
    const int np = (CQ_T - 1 - k) * (CQ_T - k) / 2, qk = (CQ_T - 2 - k) * (CQ_T - 1 - k) / 2;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int q = tid + h * CQ_THREADS;
      if (q < np) {
        const int pr = sPair[q], i = pr >> 8, j = pr & 255;
        cff g = sB[i][j];
        cff_sub_conj_mul(g, sB[k][i], cff_scale(sB[k][j], inv));
        sB[i][j] = g;
        if (q == qk) pivot(k + 1);  // pair (k + 1, k + 1)
      }
    }
  }
  __syncthreads();
  if (sBad) return;
  if (tid < pb) {  // 1 / sqrt(d_k)
    const ffv d = sB[tid][tid].re;
    sInv[tid] = d.h > 0.f ? ff_rsqrt(d) : ffv{0.f, 0.f};
  }
  __syncthreads();
  for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
    const int i = q % CQ_T, j = q / CQ_T;
    if (i < pb && j < pb && i <= j) {
      const cff v = sB[i][j];
      const cff r = i == j ? cff{ff_mul(v.re, sInv[i]), {0.f, 0.f}} : cff_scale(v, sInv[i]);
      cff_st(G, (int64_t)(p + j) * nc + p + i, r);
    }
  }
}

// The panel's rows to the right of its diagonal block: R12 = R11^-H G12, by
// forward substitution with R11^H (lower): one warp per column j >= pe,
// lane i holding row p + i; R11 and the reciprocals of its diagonal staged
// in shared memory by each CTA.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_trsm(double *__restrict__ G, int32_t nc, int32_t p,
                                                        const int32_t *__restrict__ status) {
  __shared__ cff sR[CQ_T][CQ_T];
  __shared__ ffv sInv[CQ_T];
  if (*status != GN_OK) return;
  const int pb = min(CQ_T, nc - p), pe = p + pb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
    const int i = q % CQ_T, j = q / CQ_T;
    cff v = {{0.f, 0.f}, {0.f, 0.f}};
    if (i < pb && j < pb && i <= j) v = cff_ld(G, (int64_t)(p + j) * nc + p + i);
    sR[i][j] = v;
  }
  __syncthreads();
  if (tid < CQ_T) {
    const ffv r = sR[tid][tid].re;
    sInv[tid] = r.h > 0.f ? ff_mul(ff_rsqrt(r), ff_rsqrt(r)) : ffv{0.f, 0.f};  // 1 / r_ii
  }
  __syncthreads();
  const int j = pe + blockIdx.x * (CQ_THREADS / 32) + warp;
  if (j >= nc) return;  // whole warps
  cff g = {{0.f, 0.f}, {0.f, 0.f}};
  if (lane < pb) g = cff_ld(G, (int64_t)j * nc + p + lane);
  for (int i = 0; i < pb; i++) {
    // x_i = g_i / r_ii (r_ii real), then g_k -= conj(r_ik) x_i for k > i
    cff xi = {{0.f, 0.f}, {0.f, 0.f}};
    if (lane == i) {
      g = cff_scale(g, sInv[i]);
      xi = g;
    }
    xi.re.h = __shfl_sync(0xffffffffu, xi.re.h, i);
    xi.re.l = __shfl_sync(0xffffffffu, xi.re.l, i);
    xi.im.h = __shfl_sync(0xffffffffu, xi.im.h, i);
    xi.im.l = __shfl_sync(0xffffffffu, xi.im.l, i);
    if (lane > i && lane < pb) cff_sub_conj_mul(g, sR[i][lane], xi);  // r_i,lane
  }
  if (lane < pb) cff_st(G, (int64_t)j * nc + p + lane, g);
}

// The trailing matrix: G^_ij -= sum_{k in the panel} conj(r_ki) r_kj for
// pe <= i <= j < nc, by 32 x 32 tiles (ib <= jb over the trailing range), 256
// threads of 2 x 2 entries, the panel's rows of both tiles' columns staged
// in shared memory.  part 0: every tile; 2: the tiles below the next
// panel's rows (ib >= 1), whose own update is k_cq_herk_rows.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_herk(double *__restrict__ G, int32_t nc, int32_t p,
                                                        int32_t part, const int32_t *__restrict__ status) {
  __shared__ cff sI[CQ_T][CQ_T];  // [panel row][column of the i tile]
  __shared__ cff sJ[CQ_T][CQ_T];
  if (*status != GN_OK) return;
  const int pb = min(CQ_T, nc - p), pe = p + pb;
  int ib, jb;
  cq_tile(blockIdx.x, ib, jb);
  if (part == 2) {  // every tile below the next panel's rows
    ib++;
    jb++;
  }
  const int i0 = pe + ib * CQ_T, j0 = pe + jb * CQ_T;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
    const int k = q % CQ_T, c = q / CQ_T;
    cff u = {{0.f, 0.f}, {0.f, 0.f}}, v = u;
    if (k < pb) {
      if (i0 + c < nc) u = cff_ld(G, (int64_t)(i0 + c) * nc + p + k);
      if (j0 + c < nc) v = cff_ld(G, (int64_t)(j0 + c) * nc + p + k);
    }
    sI[k][c] = u;
    sJ[k][c] = v;
  }
  __syncthreads();
  cff acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) acc[a][b] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int k = 0; k < pb; k++) {
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int b = 0; b < 2; b++) cff_sub_conj_mul(acc[a][b], sI[k][2 * ty + a], sJ[k][2 * tx + b]);
  }
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const int i = i0 + 2 * ty + a, j = j0 + 2 * tx + b;
      if (i < nc && j < nc && i <= j) {
        const int64_t at = (int64_t)j * nc + i;
        cff g = cff_ld(G, at);
        g.re = ff_add(g.re, acc[a][b].re);  // acc holds minus the sum
        g.im = ff_add(g.im, acc[a][b].im);
        cff_st(G, at, g);
      }
    }
}

// The trailing update of the next panel's rows alone, the step of the
// lookahead that the next panel waits for: the same sums as k_cq_herk for
// the tiles (0, jb), by 16 x 16 quarters of them, one entry per thread with
// two accumulation chains, so these few tiles spread over four times the
// CTAs and a thread's chain is half as long.
constexpr int CQ_H = 16;
__global__ void __launch_bounds__(CQ_H * CQ_H) k_cq_herk_rows(double *__restrict__ G, int32_t nc, int32_t p,
                                                             const int32_t *__restrict__ status) {
  __shared__ cff sI[CQ_T][CQ_H];  // [panel row][row of the quarter]
  __shared__ cff sJ[CQ_T][CQ_H];  // [panel row][column of the quarter]
  if (*status != GN_OK) return;
  const int pb = min(CQ_T, nc - p), pe = p + pb;
  const int jb = blockIdx.x >> 2, qd = blockIdx.x & 3;
  const int i0 = pe + (qd >> 1) * CQ_H, j0 = pe + jb * CQ_T + (qd & 1) * CQ_H;
  if (i0 > j0 + CQ_H - 1) return;  // a quarter below the diagonal: the whole CTA, before any barrier
  const int tid = threadIdx.x, ty = tid / CQ_H, tx = tid % CQ_H;
  for (int q = tid; q < CQ_T * CQ_H; q += CQ_H * CQ_H) {
    const int k = q % CQ_T, c = q / CQ_T;
    cff u = {{0.f, 0.f}, {0.f, 0.f}}, v = u;
    if (k < pb) {
      if (i0 + c < nc) u = cff_ld(G, (int64_t)(i0 + c) * nc + p + k);
      if (j0 + c < nc) v = cff_ld(G, (int64_t)(j0 + c) * nc + p + k);
    }
    sI[k][c] = u;
    sJ[k][c] = v;
  }
  __syncthreads();
  cff acc[2] = {{{0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}}};
#pragma unroll
  for (int k = 0; k < CQ_T; k++)
    if (k < pb) cff_sub_conj_mul(acc[k & 1], sI[k][ty], sJ[k][tx]);
  const int i = i0 + ty, j = j0 + tx;
  if (i < nc && j < nc && i <= j) {
    const int64_t at = (int64_t)j * nc + i;
    cff g = cff_ld(G, at);
    g.re = ff_add(g.re, ff_add(acc[0].re, acc[1].re));  // acc holds minus the sum
    g.im = ff_add(g.im, ff_add(acc[0].im, acc[1].im));
    cff_st(G, at, g);
  }
}

// ---- triangular solves with the float-float factor ----
//
// With R^ final, the Gauss-Newton step (R dx = y) and each refinement step
// (R^H w = c, then R dx = w) are triangular solves needed to double accuracy
// only: the refinement's corrections carry their own residual.  R = R^ D, so
// R dx = y is R^ z = y^ with z = D dx, and R^H w = c is (R^)^H w = D^-1 c.
// Blocked substitution on one cluster of CQC CTAs: R^ is cut into CQB x CQB
// diagonal blocks D_k whose inverses X_k = D_k^-1 are formed once per
// factorisation (k_cq_binv); block b of the unknowns lives in CTA b mod CQC.
// Per block, the owner of the next block brings that block's rows up to date
// with the newest unknowns, forms the next CQB unknowns as X times its rows
// and sends them to every CTA's shared memory; then every CTA updates its
// other rows, and one cluster barrier ends the step.  The right-hand side is
// scaled by a power of two first, its largest part in [1/2, 1), so the float
// exponent range holds every intermediate value.

constexpr int CQB = 32;                           // rows per block
constexpr int CQC = 8;                            // CTAs of the cluster
constexpr int CQC_THREADS = 512;
constexpr int CQC_MAXN = 1024;                    // unknowns
constexpr int CQC_OWN = CQC_MAXN / (CQB * CQC);   // blocks per CTA
constexpr size_t CQC_SMEM =
    sizeof(cff) * (CQC_OWN * CQB * CQB + 2 * CQC_OWN * CQB + 2 * CQB) + sizeof(double) * (CQC_THREADS / 32);


// acc += a x, or conj(a) x
template <bool CONJ>
__device__ __forceinline__ void cff_mac(cff &acc, const cff &a, const cff &x) {
  const ffv rr = ff_mul(a.re, x.re), ii = ff_mul(a.im, x.im);
  const ffv ri = ff_mul(a.re, x.im), ir = ff_mul(a.im, x.re);
  acc.re = ff_add(acc.re, CONJ ? ff_add(rr, ii) : ff_add(rr, ff_neg(ii)));
  acc.im = ff_add(acc.im, CONJ ? ff_add(ri, ff_neg(ir)) : ff_add(ri, ir));
}

// the sum over the G lanes of an aligned lane group, in each of them
template <int G>
__device__ __forceinline__ cff cff_group_sum(cff v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    cff u;
    u.re.h = __shfl_xor_sync(0xffffffffu, v.re.h, o);
    u.re.l = __shfl_xor_sync(0xffffffffu, v.re.l, o);
    u.im.h = __shfl_xor_sync(0xffffffffu, v.im.h, o);
    u.im.l = __shfl_xor_sync(0xffffffffu, v.im.l, o);
    v.re = ff_add(v.re, u.re);
    v.im = ff_add(v.im, u.im);
  }
  return v;
}

// X_k = D_k^-1 for the diagonal blocks of R^[0:n, 0:n] (upper), into the
// strictly lower triangle of the same blocks: X_rc (r < c) at the place of
// entry (b0 + c, b0 + r); X_rr = 1 / r_rr is formed where it is used.  One
// CTA per block, warp c forming column c by substitution (lane i holding
// row i: once x_l is known, rows i < l subtract d_il x_l and row l - 1 is
// divided by its pivot).
__global__ void __launch_bounds__(CQB * 32) k_cq_binv(double *__restrict__ R, int32_t nc, int32_t n,
                                                     const int32_t *__restrict__ status) {
  __shared__ cff sD[CQB][CQB + 1];  // [column][row]
  if (*status != GN_OK) return;
  const int b0 = blockIdx.x * CQB, bs = min(CQB, n - b0);
  const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
  if (lane <= c && c < bs) sD[c][lane] = cff_ld(R, (int64_t)(b0 + c) * nc + b0 + lane);
  __syncthreads();
  if (c >= bs) return;  // whole warps, after the only barrier
  ffv rinv = {0.f, 0.f};
  if (lane < bs && sD[lane][lane].re.h > 0.f) rinv = ff_recip(sD[lane][lane].re);
  cff x = {{0.f, 0.f}, {0.f, 0.f}};
  if (lane == c) x.re = rinv;
  for (int l = c; l >= 1; l--) {
    cff xl;
    xl.re.h = __shfl_sync(0xffffffffu, x.re.h, l);
    xl.re.l = __shfl_sync(0xffffffffu, x.re.l, l);
    xl.im.h = __shfl_sync(0xffffffffu, x.im.h, l);
    xl.im.l = __shfl_sync(0xffffffffu, x.im.l, l);
    if (lane < l) {
      cff p = {{0.f, 0.f}, {0.f, 0.f}};
      cff_mac<false>(p, sD[l][lane], xl);
      x.re = ff_add(x.re, ff_neg(p.re));
      x.im = ff_add(x.im, ff_neg(p.im));
      if (lane == l - 1) x = cff_scale(x, rinv);
    }
  }
  if (lane < c) cff_st(R, (int64_t)(b0 + lane) * nc + b0 + c, x);
}

// REFINE: R^H w = c, then R dx = w for c (double complex [n]); else R dx = y
// with y the factor's last column.  R^ in float-float (leading dimension
// nc = n + 1) with the block inverses of k_cq_binv; dx double complex [n].
template <bool REFINE>
__global__ void __launch_bounds__(CQC_THREADS, 1) k_cq_solve(const double *__restrict__ R, int32_t nc, int32_t n,
                                                             const double *__restrict__ sexp,
                                                             const double *__restrict__ c,
                                                             double *__restrict__ dx,
                                                             int32_t *__restrict__ status) {
  extern __shared__ __align__(16) float4 cq_sm[];
  cff *sXb = (cff *)cq_sm;              // [CQC_OWN][CQB][CQB] X of this CTA's blocks, [row][column]
  cff *sY = sXb + CQC_OWN * CQB * CQB;  // [CQC_OWN * CQB] the rows of this CTA's blocks
  cff *sU = sY + CQC_OWN * CQB;         // [CQC_OWN * CQB] the unknowns of this CTA's blocks
  cff *sX = sU + CQC_OWN * CQB;         // [2][CQB] the newest block of unknowns
  double *smax = (double *)(sX + 2 * CQB);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  // every CTA takes the same cluster barriers, whatever it reads here (only
  // the non-finite check below writes the status word before the end, and
  // then no CTA does any work)
  const bool run = *status == GN_OK;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (n + CQB - 1) / CQB;
  auto bsz = [&](int b) { return min(CQB, n - b * CQB); };
  auto rhs = [&](int i, double &vr, double &vi) {
    if (REFINE) {
      const int sc = -((int)sexp[i] + CQ_S);
      vr = ldexp(c[2 * i], sc);
      vi = ldexp(c[2 * i + 1], sc);
    } else {
      const cff y = cff_ld(R, (int64_t)n * nc + i);
      vr = ff_to(y.re);
      vi = ff_to(y.im);
    }
  };
  // the scale: every CTA forms max |v| over all n rows (the same value)
  double m = 0.0;
  if (run)
    for (int i = tid; i < n; i += CQC_THREADS) {
      double vr, vi;
      rhs(i, vr, vi);
      m = fmax(m, (isfinite(vr) && isfinite(vi)) ? fmax(fabs(vr), fabs(vi)) : HUGE_VAL);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) smax[warp] = m;
  __syncthreads();
  m = lane < CQC_THREADS / 32 ? smax[lane] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const bool go = run && isfinite(m);  // uniform over the cluster
  if (run && !go && rank == 0 && tid == 0) atomicCAS(status, GN_OK, GN_ENONFINITE);
  int e = 0;
  if (go && m > 0.0) frexp(m, &e);  // max |v| < 2^e
  const int nown = rank < nb ? (nb - 1 - rank) / CQC + 1 : 0;
  if (go) {
    for (int q = 0; q < nown; q++) {
      const int b = rank + CQC * q, b0 = b * CQB, bs = bsz(b);
      for (int r = tid; r < bs; r += CQC_THREADS) {
        double vr, vi;
        rhs(b0 + r, vr, vi);
        sY[q * CQB + r] = {ff_from(ldexp(vr, -e)), ff_from(ldexp(vi, -e))};
      }
      for (int idx = tid; idx < CQB * CQB; idx += CQC_THREADS) {
        const int r = idx / CQB, cc = idx % CQB;
        cff v = {{0.f, 0.f}, {0.f, 0.f}};
        if (r < bs && cc < bs) {
          if (r < cc) {
            v = cff_ld(R, (int64_t)(b0 + r) * nc + b0 + cc);
          } else if (r == cc) {
            const ffv d = cff_ld(R, (int64_t)(b0 + r) * nc + b0 + r).re;
            if (d.h > 0.f) v.re = ff_recip(d);
          }
        }
        sXb[(q * CQB + r) * CQB + cc] = v;
      }
    }
  }
  __syncthreads();
  cl.sync();  // rows loaded; every CTA started (the stores below may target it)

  // Rows of the owned blocks of slots [q0, q1) minus the product of block
  // column k (forward: conj(R^(k, rows))^T) with the unknowns in buffer buf,
  // G lanes per row, all rows in one pass.  The entries of R^ are loaded a
  // step ahead (load), before the cluster barrier, so the update waits for
  // no load.
  auto load = [&](auto gtag, bool fwd, int k, int q0, int q1, cff *ent) {
    constexpr int G = decltype(gtag)::value;
    const int k0 = k * CQB, kb = bsz(k), p = tid % G;
    const int s = q0 * CQB + tid / G, q = s / CQB, r = s % CQB;
    const int b = rank + CQC * q, i = b * CQB + r;
    const bool act = s < q1 * CQB && r < bsz(b);
#pragma unroll
    for (int t = 0; t < CQB / G; t++) {
      const int cc = p + G * t;
      ent[t] = {{0.f, 0.f}, {0.f, 0.f}};
      if (act && cc < kb)
        ent[t] = fwd ? cff_ld(R, (int64_t)i * nc + k0 + cc) : cff_ld(R, (int64_t)(k0 + cc) * nc + i);
    }
  };
  auto update = [&](auto gtag, bool fwd, int k, int buf, int q0, int q1, const cff *ent) {
    constexpr int G = decltype(gtag)::value;
    const int kb = bsz(k), p = tid % G;
    const int s = q0 * CQB + tid / G, q = s / CQB, r = s % CQB;
    const bool act = s < q1 * CQB && r < bsz(rank + CQC * q);
    cff acc[2] = {{{0.f, 0.f}, {0.f, 0.f}}, {{0.f, 0.f}, {0.f, 0.f}}};  // two chains
#pragma unroll
    for (int t = 0; t < CQB / G; t++) {
      const int cc = p + G * t;
      if (act && cc < kb) {
        if (fwd) {
          cff_mac<true>(acc[t & 1], ent[t], sX[buf * CQB + cc]);
        } else {
          cff_mac<false>(acc[t & 1], ent[t], sX[buf * CQB + cc]);
        }
      }
    }
    acc[0].re = ff_add(acc[0].re, acc[1].re);
    acc[0].im = ff_add(acc[0].im, acc[1].im);
    const cff sum = cff_group_sum<G>(acc[0]);
    if (act && p == 0) {
      cff y = sY[s];
      y.re = ff_add(y.re, ff_neg(sum.re));
      y.im = ff_add(y.im, ff_neg(sum.im));
      sY[s] = y;
    }
  };
  // the unknowns of owned block k (slot q) from its rows: X_k y (backward) or
  // X_k^H g (forward), 16 lanes per row; lane t < CQC of a row sends it to
  // buffer buf of CTA t, and it is kept in sU
  auto xstep = [&](bool fwd, int k, int buf) {
    constexpr int G = CQC_THREADS / CQB;
    static_assert(CQC < G, "a lane of the row's group for each CTA");
    const int q = (k - rank) / CQC, kb = bsz(k);
    const int r = tid / G, p = tid % G;
    cff acc = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
    for (int t = 0; t < CQB / G; t++) {
      const int cc = p + G * t;
      if (cc < kb) {
        if (fwd) {
          if (cc <= r) cff_mac<true>(acc, sXb[(q * CQB + cc) * CQB + r], sY[q * CQB + cc]);
        } else {
          if (cc >= r) cff_mac<false>(acc, sXb[(q * CQB + r) * CQB + cc], sY[q * CQB + cc]);
        }
      }
    }
    acc = cff_group_sum<G>(acc);
    if (r < kb) {
      const float4 v = make_float4(acc.re.h, acc.re.l, acc.im.h, acc.im.l);
      if (p < CQC) *((float4 *)cl.map_shared_rank(sX, p) + buf * CQB + r) = v;
      if (p == CQC) *((float4 *)sU + q * CQB + r) = v;
    }
  };
  using G4 = std::integral_constant<int, 4>;
  using G16 = std::integral_constant<int, CQC_THREADS / CQB>;
  static_assert(CQC_OWN * CQB * 4 <= CQC_THREADS, "the other rows in one pass of 4 lanes each");
  // the owned slots of blocks in [lo, hi)
  auto slot_lo = [&](int lo) { return lo <= rank ? 0 : (lo - rank + CQC - 1) / CQC; };
  auto slot_hi = [&](int hi) { return hi <= rank ? 0 : min(nown, (hi - rank + CQC - 1) / CQC); };
  auto slot_of = [&](int b) { return (b - rank) / CQC; };  // b owned
  // the entries of the next steps: e16 for this CTA's next turn as owner
  // (loaded right after its previous turn, CQC steps ahead), e4 for the
  // other rows of the next step
  cff e16[CQB / 16], e4[CQB / 4];
  if (REFINE) {
    // forward: w_k = X_k^H (g_k - sum_{j<k} R_jk^H w_j), blocks in order; step
    // k applies w_k to block k+1 (its owner first) and to the blocks after it
    auto owns = [&](int k) { return rank == (k + 1) % CQC; };
    auto fetch16 = [&](int k) { load(G16{}, true, k, slot_of(k + 1), slot_of(k + 1) + 1, e16); };
    auto fetch4 = [&](int k) { load(G4{}, true, k, slot_lo(k + 2), slot_hi(nb), e4); };
    if (go && nb > 1) {
      for (int k = 0; k + 1 < nb && k < CQC; k++)
        if (owns(k)) fetch16(k);
      fetch4(0);
    }
    if (go && rank == 0) xstep(true, 0, 0);
    cl.sync();
    for (int k = 0; k + 1 < nb; k++) {
      const int buf = k & 1;
      if (go) {
        if (owns(k)) {
          const int q = slot_of(k + 1);
          update(G16{}, true, k, buf, q, q + 1, e16);  // block k+1 first
          if (k + CQC + 1 < nb) fetch16(k + CQC);
          __syncthreads();
          xstep(true, k + 1, buf ^ 1);
        }
        update(G4{}, true, k, buf, slot_lo(k + 2), slot_hi(nb), e4);  // the other owned blocks below
        if (k + 2 < nb) fetch4(k + 1);
      }
      cl.sync();
    }
  }
  if (REFINE) {  // w is the backward solve's right-hand side
    for (int t = tid; t < nown * CQB; t += CQC_THREADS) sY[t] = sU[t];
    __syncthreads();
  }
  // backward: x_k = X_k (y_k - sum_{j>k} R_kj x_j), blocks from the last;
  // step k applies x_k to block k-1 (its owner first) and to the blocks above
  auto owns = [&](int k) { return rank == (k - 1) % CQC; };
  auto fetch16 = [&](int k) { load(G16{}, false, k, slot_of(k - 1), slot_of(k - 1) + 1, e16); };
  auto fetch4 = [&](int k) { load(G4{}, false, k, 0, slot_hi(k - 1), e4); };
  if (go && nb > 1) {
    for (int k = nb - 1; k >= 1 && k > nb - 1 - CQC; k--)
      if (owns(k)) fetch16(k);
    fetch4(nb - 1);
  }
  if (go && rank == (nb - 1) % CQC) xstep(false, nb - 1, (nb - 1) & 1);
  cl.sync();
  for (int k = nb - 1; k >= 1; k--) {
    const int buf = k & 1;
    if (go) {
      if (owns(k)) {
        const int q = slot_of(k - 1);
        update(G16{}, false, k, buf, q, q + 1, e16);  // block k-1 first
        if (k - CQC >= 1) fetch16(k - CQC);
        __syncthreads();
        xstep(false, k - 1, buf ^ 1);
      }
      update(G4{}, false, k, buf, 0, slot_hi(k - 1), e4);  // the other owned blocks above
      if (k - 1 >= 1) fetch4(k - 1);
    }
    cl.sync();
  }
  // dx of the owned rows: REFINE dx = D^-1 z, else dx = D^-1 z 2^(s_n + 62);
  // and the scale 2^e back
  if (go)
    for (int t = tid; t < nown * CQB; t += CQC_THREADS) {
      const int b = rank + CQC * (t / CQB), r = t % CQB, i = b * CQB + r;
      if (r >= bsz(b)) continue;
      const int sh = REFINE ? e - ((int)sexp[i] + CQ_S) : e + (int)sexp[n] - (int)sexp[i];
      const double xr = ldexp(ff_to(sU[t].re), sh), xi = ldexp(ff_to(sU[t].im), sh);
      if (!isfinite(xr) || !isfinite(xi)) atomicCAS(status, GN_OK, GN_ENONFINITE);
      dx[2 * i] = xr;
      dx[2 * i + 1] = xi;
    }
}

gn_status launch_cq_solve(bool refine, int32_t n, const double *R, const double *sexp, const double *c,
                          double *dx, int32_t *status, cudaStream_t st) {
  if (n < 1 || n > CQC_MAXN) return GN_EINVAL;
  // the kernels' shared-memory limit, raised once per device
  constexpr int kDevices = 64;
  static std::mutex mu;
  static signed char ready[kDevices] = {};  // 0 not yet, 1 done, -1 refused
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) return GN_ECUDA;
  {
    std::lock_guard<std::mutex> g(mu);
    if (ready[dev] == 0)
      ready[dev] = cudaFuncSetAttribute(k_cq_solve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)CQC_SMEM) == cudaSuccess &&
                           cudaFuncSetAttribute(k_cq_solve<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)CQC_SMEM) == cudaSuccess
                       ? 1
                       : -1;
  }
  if (ready[dev] != 1) return GN_ECUDA;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CQC);
  cfg.blockDim = dim3(CQC_THREADS);
  cfg.dynamicSmemBytes = CQC_SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = CQC;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  const int32_t nc = n + 1;
  const cudaError_t err = refine ? cudaLaunchKernelEx(&cfg, k_cq_solve<true>, R, nc, n, sexp, c, dx, status)
                                 : cudaLaunchKernelEx(&cfg, k_cq_solve<false>, R, nc, n, sexp, c, dx, status);
  return err == cudaSuccess ? GN_OK : GN_ECUDA;
}

bool cholqr_available(const gn_system *s) {
  // the cluster solves hold at most CQC_MAXN unknowns: 32 .. 1024
  return s->arith != GN_ARITH_FP64 && s->n >= 32 && s->n <= CQC_MAXN && s->N >= s->n;
}

// With a second stream (side, created at the highest priority) and two
// events the panels look one ahead: the panels' Cholesky, row block and the
// trailing update of the next panel's rows run on side, so the next panel
// follows at once, while the rest of each trailing update runs on st; the
// next panel's own trailing update waits for that rest (it updates the same
// rows).  The priority gives the panels' launches the SMs that free up
// while a large trailing update fills the GPU.
gn_status launch_cholqr(int32_t N, int32_t n, const double *A, double *R, double *rinv, void *scratch,
                        int32_t *status, cudaStream_t st, cudaStream_t side, cudaEvent_t ev_panel,
                        cudaEvent_t ev_trail) {
  const int32_t nc = n + 1;
  double *nrm0 = rinv + nc, *sexp = rinv + 2 * (size_t)nc;  // the layout of the one-limb rinv
  k_cq_scale<<<(unsigned)((nc * 32 + CQ_THREADS - 1) / CQ_THREADS), CQ_THREADS, 0, st>>>(A, N, nc, nrm0,
                                                                                      sexp, status);
  if (scratch && gram_tc_available(N, nc)) {
    const gn_status e = launch_gram_tc(N, nc, A, sexp, R, scratch, status, st);
    if (e) return e;
  } else {
    const int nb = (nc + CQ_T - 1) / CQ_T;
    k_cq_gram<<<(unsigned)(nb * (nb + 1) / 2), CQ_THREADS, 0, st>>>(A, N, nc, sexp, R, status);
  }
  k_cq_to_ff<<<(unsigned)nc, 128, 0, st>>>(R, nc, sexp, status);
  const bool ahead = side && ev_panel && ev_trail;
  cudaStream_t ps = st;  // the panels' stream
  if (ahead) {
    ps = side;
    if (cudaEventRecord(ev_trail, st) != cudaSuccess || cudaStreamWaitEvent(ps, ev_trail, 0) != cudaSuccess)
      return GN_ECUDA;
  }
  bool trail = false;  // a trailing update is in flight on st
  for (int p = 0; p < nc; p += CQ_T) {
    k_cq_potrf<<<1, CQ_THREADS, 0, ps>>>(R, nc, p, nrm0, sexp, n, status);
    const int pe = p + CQ_T < nc ? p + CQ_T : nc;
    if (pe >= nc) break;
    const int cols = nc - pe;
    k_cq_trsm<<<(unsigned)((cols + CQ_THREADS / 32 - 1) / (CQ_THREADS / 32)), CQ_THREADS, 0, ps>>>(R, nc, p,
                                                                                                status);
    const int tb = (cols + CQ_T - 1) / CQ_T;
    if (!ahead) {
      k_cq_herk<<<(unsigned)(tb * (tb + 1) / 2), CQ_THREADS, 0, st>>>(R, nc, p, 0, status);
      continue;
    }
    if (cudaEventRecord(ev_panel, ps) != cudaSuccess) return GN_ECUDA;  // the row block is done
    // the next panel's rows: after the previous rest, which updated them too
    if (trail && cudaStreamWaitEvent(ps, ev_trail, 0) != cudaSuccess) return GN_ECUDA;
    k_cq_herk_rows<<<(unsigned)(4 * tb), CQ_H * CQ_H, 0, ps>>>(R, nc, p, status);
    trail = tb > 1;
    if (trail) {
      if (cudaStreamWaitEvent(st, ev_panel, 0) != cudaSuccess) return GN_ECUDA;
      k_cq_herk<<<(unsigned)((tb - 1) * tb / 2), CQ_THREADS, 0, st>>>(R, nc, p, 2, status);
      if (cudaEventRecord(ev_trail, st) != cudaSuccess) return GN_ECUDA;
    }
  }
  if (ahead) {  // st continues after the last panel (its own rests are in order)
    if (cudaEventRecord(ev_panel, ps) != cudaSuccess || cudaStreamWaitEvent(st, ev_panel, 0) != cudaSuccess)
      return GN_ECUDA;
  }
  k_cq_binv<<<(unsigned)((n + CQB - 1) / CQB), CQB * 32, 0, st>>>(R, nc, n, status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

}  // namespace gn
