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
// as MGS on [A b] gives them (eq. 2), so the Gauss-Newton step and the
// refinement's y = R^-H (A^H b) reuse the blocked integer triangular solves
// (bsb.cuh) once R is in their mantissa format.
//
// Accuracy: R from the Cholesky of the Gram matrix has a relative error of
// about kappa(A)^2 u (against kappa u for MGS), u = 2^-47 for the
// float-float Cholesky; the refinement only needs the factors to contract,
// which they do for kappa(A)^2 u << 1 (the mixed workload's Jacobian has
// kappa = 15).  Rank: a pivot below
// 2^-40 of its column's squared norm (kappa above about 10^6, where the
// double refinement would not converge) is reported as GN_ESINGULAR.
#include "ifx.cuh"
#include "internal.h"

namespace gn {

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
// by one CTA in shared memory, right-looking: after row k is final (r_kk =
// sqrt(g_kk), the rest of the row times 1 / r_kk), every g_ij with
// k < i <= j less conj(r_ki) r_kj.  The pairs (i, j), 1 <= i <= j < 32, are
// listed by decreasing i, so the pairs still to update after row k are the
// first (31 - k)(32 - k) / 2 of the list and a step's threads are packed
// into whole warps.  The thread of pair (k + 1, k + 1) takes the next pivot
// as soon as it has updated it.  A pivot g_kk <= 2^-40 ||a_k||^2 (k < nchk;
// in the scaled units) records GN_ESINGULAR.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_potrf(double *__restrict__ G, int32_t nc, int32_t p,
                                                         const double *__restrict__ nrm0,
                                                         const double *__restrict__ sexp, int32_t nchk,
                                                         int32_t *__restrict__ status) {
  constexpr int NPAIR = (CQ_T - 1) * CQ_T / 2;  // 496 pairs with i >= 1
  static_assert(NPAIR <= 2 * CQ_THREADS, "two pairs per thread");
  __shared__ cff sB[CQ_T][CQ_T];           // [row][column]
  __shared__ unsigned short sPair[NPAIR];  // i << 8 | j
  __shared__ ffv sInv[CQ_T];
  __shared__ int sBad;
  if (*status != GN_OK) return;
  const int pb = min(CQ_T, nc - p);
  const int tid = threadIdx.x;
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
  // the pivot of row k (its thread only): r_kk, 1 / r_kk, the rank test
  auto pivot = [&](int k) {
    const ffv d = sB[k][k].re;
    const float n0 = (float)ldexp(nrm0[p + k], -((int)sexp[p + k] + CQ_S));  // in (1/2, 1]
    const bool bad = !(d.h > ldexpf(n0 * n0, -40));
    if (bad && p + k < nchk) {
      atomicCAS(status, GN_OK, GN_ESINGULAR);
      sBad = 1;
    }
    const ffv inv = d.h > 0.f ? ff_rsqrt(d) : ffv{0.f, 0.f};
    sB[k][k] = {ff_mul(d, inv), {0.f, 0.f}};
    sInv[k] = inv;
  };
  if (tid == 0) pivot(0);
  for (int k = 0;; k++) {
    __syncthreads();
    if (sBad) return;  // uniform: read after the barrier
    const ffv inv = sInv[k];
    for (int j = k + 1 + tid; j < CQ_T; j += CQ_THREADS) sB[k][j] = cff_scale(sB[k][j], inv);
    if (k + 1 >= pb) break;
    __syncthreads();
    const int np = (CQ_T - 1 - k) * (CQ_T - k) / 2, qk = (CQ_T - 2 - k) * (CQ_T - 1 - k) / 2;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int q = tid + h * CQ_THREADS;
      if (q < np) {
        const int pr = sPair[q], i = pr >> 8, j = pr & 255;
        cff g = sB[i][j];
        cff_sub_conj_mul(g, sB[k][i], sB[k][j]);
        sB[i][j] = g;
        if (q == qk) pivot(k + 1);  // pair (k + 1, k + 1)
      }
    }
  }
  __syncthreads();
  for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
    const int i = q % CQ_T, j = q / CQ_T;
    if (i < pb && j < pb && i <= j) cff_st(G, (int64_t)(p + j) * nc + p + i, sB[i][j]);
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
// in shared memory.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_herk(double *__restrict__ G, int32_t nc, int32_t p,
                                                        const int32_t *__restrict__ status) {
  __shared__ cff sI[CQ_T][CQ_T];  // [panel row][column of the i tile]
  __shared__ cff sJ[CQ_T][CQ_T];
  if (*status != GN_OK) return;
  const int pb = min(CQ_T, nc - p), pe = p + pb;
  int ib, jb;
  cq_tile(blockIdx.x, ib, jb);
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

// R = R^ D (R^ in float-float, upper, leading dimension nc) into the
// mantissa format of the integer triangular solves: column j's entries as
// one-limb mantissas at 2^s_j (r_kj 2^-s_j = r^_kj 2^62, |r^_kj| <= 1), 1/r_jj
// as a mantissa in [2^61, 2^62) and its exponent (Zs), 1/r_jj as a double
// too.  One CTA per column.
__global__ void k_cq_to_int(const double *__restrict__ R, int32_t nc, const double *__restrict__ sexp,
                            double *__restrict__ Rm, double *__restrict__ Zs, double *__restrict__ rinv,
                            const int32_t *__restrict__ status) {
  if (*status != GN_OK) return;
  const int j = blockIdx.x;
  for (int k = threadIdx.x; k <= j; k += blockDim.x) {
    const cff e = cff_ld(R, (int64_t)j * nc + k);
    long long *d = (long long *)(Rm + ((int64_t)j * nc + k) * 2);
    d[0] = llrint(ldexp(ff_to(e.re), CQ_S));
    d[1] = llrint(ldexp(ff_to(e.im), CQ_S));
  }
  if (threadIdx.x == 0 && j < nc - 1) {
    const double r = ff_to(cff_ld(R, (int64_t)j * nc + j).re);
    const double v = r > 0.0 ? ldexp(1.0 / r, -((int)sexp[j] + CQ_S)) : 0.0;  // 1 / (r^_jj 2^(s_j + 62))
    int ex = 0;
    const double f = frexp(v, &ex);  // v = f 2^ex, f in [1/2, 1)
    ((long long *)Zs)[(size_t)j * 2] = llrint(ldexp(f, 62));
    Zs[(size_t)j * 2 + 1] = (double)(ex - 62);
    rinv[j] = v;
  }
}

bool cholqr_available(const gn_system *s) {
  // the blocked integer solves it hands R to take 32 .. 1024 unknowns
  return s->arith != GN_ARITH_FP64 && s->n >= 32 && s->n <= BACKSUB_INT_MAX_N && s->N >= s->n &&
         fwdsub_int_available(1, s->n);
}

gn_status launch_cholqr(int32_t N, int32_t n, const double *A, double *R, double *rinv, double *Rm,
                        double *Zs, void *scratch, int32_t *status, cudaStream_t st) {
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
  for (int p = 0; p < nc; p += CQ_T) {
    k_cq_potrf<<<1, CQ_THREADS, 0, st>>>(R, nc, p, nrm0, sexp, n, status);
    const int pe = p + CQ_T < nc ? p + CQ_T : nc;
    if (pe >= nc) break;
    const int cols = nc - pe;
    k_cq_trsm<<<(unsigned)((cols + CQ_THREADS / 32 - 1) / (CQ_THREADS / 32)), CQ_THREADS, 0, st>>>(R, nc, p,
                                                                                                status);
    const int tb = (cols + CQ_T - 1) / CQ_T;
    k_cq_herk<<<(unsigned)(tb * (tb + 1) / 2), CQ_THREADS, 0, st>>>(R, nc, p, status);
  }
  k_cq_to_int<<<(unsigned)nc, 128, 0, st>>>(R, nc, sexp, Rm, Zs, rinv, status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

}  // namespace gn
