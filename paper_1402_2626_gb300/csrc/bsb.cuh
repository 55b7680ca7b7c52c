// bsb.cuh — blocked back substitution R x = y (Section 3, eq. 5) on the
// integer mantissas MGS leaves, with explicit inverses of the diagonal
// blocks.
//
// Solving one unknown at a time makes every level of the n-level chain a
// dependent multi-word product, a reciprocal scaling and a barrier (about
// 2 us per level in DD).  Here R is cut into BSB x BSB diagonal blocks D_k:
//   k_bs_inv        X_k = D_k^-1 for every block at once (one warp per block,
//                   lane c forms column c by substitution inside the block);
//   k_backsub_cl    for k = last .. 0: x_k = X_k y_k, then y_i -= R_ik x_k for
//                   the rows above (the rows of block k-1 first), on a
//                   cluster of CTAs.
// Both steps of a block are small matrix-vector products: every thread forms
// one product and 16 lanes add theirs exactly (integer sums), so a block
// costs two products and two 4-level reductions on the chain instead of 16
// levels.  The formats are those of bs.cuh: y fixed point at the scale of
// the last column with two limbs of headroom, x_l = X 2^t with K-limb X.
// Entries of X_k are complex values with one binary exponent (cf.cuh).
#pragma once

#include <cooperative_groups.h>

#include "bs.cuh"
#include "cf.cuh"
#include "internal.h"

namespace gn {

namespace cg = cooperative_groups;

constexpr int BSB = 16;              // block size
constexpr int BSB_THREADS = 512;     // threads of the solve (32 rows x 16 columns per pass)

// a complex value with N-limb integer parts at 2^e0 as cf<K>
template <int K, int N>
__device__ __forceinline__ cf<K> cf_from_fixed(const fx<N> &re, const fx<N> &im, int e0) {
  const int b1 = ix_bitlen<N>(ix_abs_fx<N>(re)), b2 = ix_bitlen<N>(ix_abs_fx<N>(im));
  const int B = b1 > b2 ? b1 : b2;
  cf<K> z;
  if (B == 0) return cf_zero<K>();
  const int sh = B - (64 * K - 2);
  fx<N> r = re, i = im;
  if (sh > 0) {
    r = ix_sar<N>(r, sh);
    i = ix_sar<N>(i, sh);
  } else if (sh < 0) {
    r = ix_shl<N>(r, -sh);
    i = ix_shl<N>(i, -sh);
  }
  z.re = ix_low<K, N>(r);
  z.im = ix_low<K, N>(i);
  z.e = e0 + sh;
  return z;
}

template <int K>
__device__ __forceinline__ cf<K> cf_neg(const cf<K> &a) {
  cf<K> r = a;
  fx<K> z;
  fx_zero<K>(z);
  r.re = ix_sub<K>(z, a.re);
  r.im = ix_sub<K>(z, a.im);
  return r;
}

template <int K>
__device__ __forceinline__ void cf_put(double *p, const cf<K> &z) {
  uint64_t *q = (uint64_t *)p;
#pragma unroll
  for (int w = 0; w < K; w++) {
    q[w] = z.re.w[w];
    q[K + w] = z.im.w[w];
  }
  q[2 * K] = (uint64_t)(int64_t)z.e;
}

template <int K>
__device__ __forceinline__ cf<K> cf_get(const double *p) {
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

// exact sum of up to 16 cf values (lanes of one 16-lane group; inactive
// lanes pass has = false), as cf<K> in every lane of the group
template <int K>
__device__ __forceinline__ cf<K> cf_group16_sum(const cf<K> &v, bool has) {
  int e = has ? v.e : CF_EZERO;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const int u = __shfl_xor_sync(0xffffffffu, e, o);
    e = u > e ? u : e;
  }
  const int E = cf_sum_exponent(e, 16);
  fx<K + 1> re, im;
  fx_zero<K + 1>(re);
  fx_zero<K + 1>(im);
  if (has) cf_accumulate<K>(re, im, v, E);
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    fx<K + 1> a, b;
#pragma unroll
    for (int w = 0; w <= K; w++) {
      a.w[w] = __shfl_xor_sync(0xffffffffu, re.w[w], o);
      b.w[w] = __shfl_xor_sync(0xffffffffu, im.w[w], o);
    }
    re = ix_add<K + 1>(re, a);
    im = ix_add<K + 1>(im, b);
  }
  if (E == CF_EZERO) return cf_zero<K>();
  // the accumulator counts units of 2^(E - 64)
  return cf_from_fixed<K, K + 1>(re, im, E - 64);
}

// X_k = D_k^-1 for the diagonal blocks of R[0:n, 0:n], one CTA of 256
// threads per block.  The block's entries r_ij (i <= j) and 1/r_ii are first
// converted to cf<K> in shared memory; then the 16-lane group c forms column
// c of the inverse, one row per step from the diagonal up:
//   X_cc = 1 / r_cc,  X_ic = -(1 / r_ii) sum_{j=i+1..c} r_ij X_jc  (i < c),
// lane j forming r_ij X_jc and the group adding the products exactly.
// Xinv[(k BSB + i) BSB + c] holds X_ic as cf<K> (2K+1 words), 0 below the
// diagonal.
template <int L>
__global__ void __launch_bounds__(BSB * BSB) k_bs_inv(const double *__restrict__ Rm, int64_t ldr,
                                                      int32_t n, const double *__restrict__ Zs,
                                                      const double *__restrict__ sexp,
                                                      double *__restrict__ Xinv,
                                                      const int32_t *__restrict__ status) {
  constexpr int K = L, W = 2 * L, CW = 2 * K + 1;
  __shared__ cf<K> sD[BSB][BSB];  // r_ij of the block
  __shared__ cf<K> sX[BSB][BSB];  // X_ic
  __shared__ cf<K> sZ[BSB];       // 1 / r_ii
  if (*status != GN_OK) return;
  const int k = blockIdx.x;
  const int b0 = k * BSB;
  const int bs = n - b0 < BSB ? n - b0 : BSB;
  const int t = threadIdx.x, a = t / BSB, b = t % BSB;
  sX[a][b] = cf_zero<K>();
  if (a <= b && b < bs) {
    const fx<K> *e = (const fx<K> *)(Rm + ((int64_t)(b0 + b) * ldr + b0 + a) * W);
    sD[a][b] = cf_from_fixed<K, K>(e[0], e[1], (int)sexp[b0 + b]);
  }
  if (t < bs) {
    const uint64_t *z = (const uint64_t *)(Zs + (size_t)(b0 + t) * (K + 1));
    fx<K> zr, zi;
#pragma unroll
    for (int w = 0; w < K; w++) zr.w[w] = z[w];
    fx_zero<K>(zi);
    sZ[t] = cf_from_fixed<K, K>(zr, zi, (int)Zs[(size_t)(b0 + t) * (K + 1) + K]);
  }
  __syncthreads();
  const int c = a, j = b;  // group c, lane j
  if (c < bs && j == 0) sX[c][c] = sZ[c];
  __syncwarp();
  for (int i = BSB - 2; i >= 0; i--) {
    const bool has = i < c && c < bs && j > i && j <= c;
    cf<K> p = cf_zero<K>();
    if (has) p = cf_mul<K>(sD[i][j], sX[j][c]);
    const cf<K> sum = cf_group16_sum<K>(p, has);
    if (i < c && c < bs && j == 0) sX[i][c] = cf_neg<K>(cf_mul<K>(sZ[i], sum));
    __syncwarp();
  }
  __syncthreads();  // column c was written by group c's warp
  cf_put<K>(Xinv + ((size_t)(k * BSB + a) * BSB + b) * CW, sX[a][b]);
}

// R x = y with y = R[0:n, n] on a cluster of BSC CTAs: block b of rows (and of y) lives
// in CTA b mod BSC.  Per block k, from the last: the owner of block k-1
// subtracts R_(k-1),k x_k from its rows and forms x_(k-1) = X_(k-1) y_(k-1)
// at once, storing it into every CTA's shared memory (double-buffered by the
// parity of the block); every CTA then subtracts R_ik x_k from its other
// rows; one cluster barrier ends the step.  The chain per block is one
// update pass, one inverse pass and a barrier; the bulk of the n^2/2
// products is split over the cluster's SMs.  Every CTA runs every barrier
// (no early exit after the first one).
constexpr int BSC = 8;
// rows of the blocks one CTA of the cluster owns, at most (block b in CTA b mod BSC)
__host__ __device__ constexpr int bsc_own_rows(int n) {
  return ((n + BSB - 1) / BSB + BSC - 1) / BSC * BSB;
}
static_assert(BSC < BSB, "a lane of each row's group per CTA, and one more");

template <int L>
__global__ void __launch_bounds__(BSB_THREADS, 1) k_backsub_cl(
    const double *__restrict__ Rm, int64_t ldr, int32_t n, const double *__restrict__ sexp,
    const double *__restrict__ Xinv, double *__restrict__ dx, int32_t *__restrict__ status) {
  constexpr int K = L, W = 2 * L, KY = K + 2, CW = 2 * K + 1;
  extern __shared__ __align__(16) unsigned char bsm[];
  fx<KY> *sY = (fx<KY> *)bsm;              // [n][2], the rows of this CTA's blocks
  fx<K> *sXc = (fx<K> *)(sY + 2 * n);      // [2][BSB][2] x of the current / next block
  cf<K> *sXo = (cf<K> *)(sXc + 2 * BSB * 2);  // x of this CTA's blocks, for dx at the end
  int *sTc = (int *)(sXo + bsc_own_rows(n));  // [2][BSB]
  int *sFail = sTc + 2 * BSB;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const bool run = *status == GN_OK;  // the same for every CTA: nothing writes it before the end
  const int tid = threadIdx.x;
  const int r = tid / BSB, c = tid % BSB;
  const int sig = (int)sexp[n];
  const int nb = (n + BSB - 1) / BSB;
  auto bsz = [&](int b) { return n - b * BSB < BSB ? n - b * BSB : BSB; };
  if (run)
    for (int b = rank; b < nb; b += BSC)
      for (int q = tid; q < bsz(b); q += BSB_THREADS) {
        const int i = b * BSB + q;
        const fx<K> *e = (const fx<K> *)(Rm + ((int64_t)n * ldr + i) * W);
        sY[2 * i] = ix_widen<K, KY>(e[0]);
        sY[2 * i + 1] = ix_widen<K, KY>(e[1]);
      }
  if (tid == 0) *sFail = 0;
  // x_k = X_k y_k for a block this CTA owns, into buffer buf of every CTA
  // and into dx
  auto xstep = [&](int k, int buf) {
    const int b0 = k * BSB, bs = bsz(k);
    if (r < BSB) {  // whole warps: the first BSB rows of pairs
      const bool has = r < bs && c >= r && c < bs;
      cf<K> p = cf_zero<K>();
      if (has) {
        const cf<K> xk = cf_get<K>(Xinv + ((size_t)(k * BSB + r) * BSB + c) * CW);
        const cf<K> yc = cf_from_fixed<K, KY>(sY[2 * (b0 + c)], sY[2 * (b0 + c) + 1], sig);
        p = cf_mul<K>(xk, yc);
      }
      const cf<K> sx = cf_group16_sum<K>(p, has);  // in every lane of the row's group
      if (r < bs) {
        if (c < BSC) {  // lane c sends x_r to CTA c
          fx<K> *rx = cl.map_shared_rank(sXc, c) + 2 * (buf * BSB + r);
          rx[0] = sx.re;
          rx[1] = sx.im;
          cl.map_shared_rank(sTc, c)[buf * BSB + r] = sx.e;
        } else if (c == BSC) {
          sXo[(k / BSC) * BSB + r] = sx;
        }
      }
    }
  };
  // rows of the owned blocks b with lo <= b < hi (b = rank mod BSC) minus
  // R[rows, block k] x_k (x_k in buffer buf); two blocks of rows per pass
  auto update = [&](int k, int buf, int lo, int hi) {
    const int j0 = k * BSB, jb = bsz(k);
    int first = lo + ((rank - lo) % BSC + BSC) % BSC;  // first owned block >= lo
    for (int b2 = first; b2 < hi; b2 += 2 * BSC) {
      const int b = b2 + (r / BSB) * BSC;  // this pair's block
      const int i = b * BSB + (r % BSB);
      const bool act = b < hi && (r % BSB) < bsz(b < nb ? b : 0) && c < jb;
      fx<KY> ur, ui;
      fx_zero<KY>(ur);
      fx_zero<KY>(ui);
      if (act) {
        const int j = j0 + c;
        const fx<K> *e = (const fx<K> *)(Rm + ((int64_t)j * ldr + i) * W);
        const int d = (int)sexp[j] + sTc[buf * BSB + c] - sig;
        bs_update<K, KY>(ur, ui, e[0], e[1], sXc[2 * (buf * BSB + c)], sXc[2 * (buf * BSB + c) + 1], d,
                         sFail);
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        fx<KY> a, bb;
#pragma unroll
        for (int w = 0; w < KY; w++) {
          a.w[w] = __shfl_xor_sync(0xffffffffu, ur.w[w], o);
          bb.w[w] = __shfl_xor_sync(0xffffffffu, ui.w[w], o);
        }
        ur = ix_add<KY>(ur, a);
        ui = ix_add<KY>(ui, bb);
      }
      if (c == 0 && b < hi && (r % BSB) < bsz(b < nb ? b : 0)) {
        sY[2 * i] = ix_add<KY>(sY[2 * i], ur);
        sY[2 * i + 1] = ix_add<KY>(sY[2 * i + 1], ui);
      }
    }
  };
  __syncthreads();
  cl.sync();  // rows loaded; every CTA started (DSMEM stores may target it)
  if (run && rank == (nb - 1) % BSC) xstep(nb - 1, (nb - 1) & 1);
  cl.sync();
  for (int k = nb - 1; k >= 1; k--) {
    const int buf = k & 1;
    if (run) {
      if (rank == (k - 1) % BSC) {
        update(k, buf, k - 1, k);  // block k-1 first
        __syncthreads();
        xstep(k - 1, buf ^ 1);
      }
      update(k, buf, 0, k - 1);  // the other owned blocks above
    }
    cl.sync();
  }
  // the owned rows' unknowns to L-limb cascades, off the steps' chain
  if (run)
    for (int t = tid; t < bsc_own_rows(n); t += BSB_THREADS) {
      const int b = rank + BSC * (t / BSB), r = t % BSB;
      if (b >= nb || r >= bsz(b)) continue;
      const cf<K> sx = sXo[t];
      double cr[L], ci[L];
      const bool z = sx.e == CF_EZERO;
      fx_to_cascade<K, L>(sx.re, z ? 0 : -sx.e, cr);
      fx_to_cascade<K, L>(sx.im, z ? 0 : -sx.e, ci);
#pragma unroll
      for (int q = 0; q < L; q++) {
        dx[(int64_t)(b * BSB + r) * W + q] = cr[q];
        dx[(int64_t)(b * BSB + r) * W + L + q] = ci[q];
      }
    }
  if (*sFail && tid == 0) atomicCAS(status, GN_OK, GN_ENONFINITE);
}

// R^H w = g (the adjoint's forward substitution) on the same cluster and the
// same inverse blocks: the diagonal blocks of R^H are D_k^H, with inverses
// X_k^H.  Blocks run forward; the owner of block k+1 subtracts
// (R^H)_(k+1),k w_k = conj(R_k,(k+1))^T w_k from its rows and forms
// w_(k+1) = X_(k+1)^H g_(k+1) at once.  g (L-limb cascades) is taken to
// fixed point at one scale 2^sig, max |g| < 2^(64K-3+sig), two limbs of
// headroom above it; the products conj(r_ji) w_j carry column i's exponent.
template <int L>
__global__ void __launch_bounds__(BSB_THREADS, 1) k_fwdsub_cl(
    const double *__restrict__ Rm, int64_t ldr, int32_t n, const double *__restrict__ sexp,
    const double *__restrict__ Xinv, const double *__restrict__ g, double *__restrict__ w,
    int32_t *__restrict__ status) {
  constexpr int K = L, W = 2 * L, KY = K + 2, CW = 2 * K + 1;
  extern __shared__ __align__(16) unsigned char bsm[];
  fx<KY> *sY = (fx<KY> *)bsm;              // [n][2], the rows of this CTA's blocks
  fx<K> *sXc = (fx<K> *)(sY + 2 * n);      // [2][BSB][2] w of the current / next block
  cf<K> *sXo = (cf<K> *)(sXc + 2 * BSB * 2);  // w of this CTA's blocks, for the output at the end
  int *sTc = (int *)(sXo + bsc_own_rows(n));  // [2][BSB]
  int *sFail = sTc + 2 * BSB;
  int *sE = sFail + 1;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const bool run = *status == GN_OK;
  const int tid = threadIdx.x;
  const int r = tid / BSB, c = tid % BSB;
  const int nb = (n + BSB - 1) / BSB;
  auto bsz = [&](int b) { return n - b * BSB < BSB ? n - b * BSB : BSB; };
  // the scale: the largest exponent of a leading limb (the same in every CTA)
  if (tid == 0) *sE = -100000;
  __syncthreads();
  {
    int em = -100000;
    for (int i = tid; i < n; i += BSB_THREADS) {
      const double a = fmax(fabs(g[(int64_t)i * W]), fabs(g[(int64_t)i * W + L]));
      if (a > 0.0) em = max(em, fx_exponent_of(a));
    }
    atomicMax(sE, em);
  }
  if (tid == 0) *sFail = 0;
  __syncthreads();
  // |g| < 2^(E+1) (one bit for the lower limbs); mantissas at 2^(64K-4-E)
  const int sig = (*sE == -100000) ? 0 : *sE + 4 - 64 * K;
  if (run)
    for (int b = rank; b < nb; b += BSC)
      for (int q = tid; q < bsz(b); q += BSB_THREADS) {
        const int i = b * BSB + q;
        fx<K> re, im;
        fx_zero<K>(re);
        fx_zero<K>(im);
#pragma unroll
        for (int l = 0; l < L; l++) {
          fx_add_double<K>(re, g[(int64_t)i * W + l], -sig);
          fx_add_double<K>(im, g[(int64_t)i * W + L + l], -sig);
        }
        sY[2 * i] = ix_widen<K, KY>(re);
        sY[2 * i + 1] = ix_widen<K, KY>(im);
      }
  auto xstep = [&](int k, int buf) {
    const int b0 = k * BSB, bs = bsz(k);
    if (r < BSB) {
      const bool has = r < bs && c <= r;
      cf<K> p = cf_zero<K>();
      if (has) {
        // (X_k^H)_rc = conj(X_k cr)
        cf<K> xk = cf_get<K>(Xinv + ((size_t)(k * BSB + c) * BSB + r) * CW);
        fx<K> z;
        fx_zero<K>(z);
        xk.im = ix_sub<K>(z, xk.im);
        const cf<K> yc = cf_from_fixed<K, KY>(sY[2 * (b0 + c)], sY[2 * (b0 + c) + 1], sig);
        p = cf_mul<K>(xk, yc);
      }
      const cf<K> sx = cf_group16_sum<K>(p, has);  // in every lane of the row's group
      if (r < bs) {
        if (c < BSC) {  // lane c sends w_r to CTA c
          fx<K> *rx = cl.map_shared_rank(sXc, c) + 2 * (buf * BSB + r);
          rx[0] = sx.re;
          rx[1] = sx.im;
          cl.map_shared_rank(sTc, c)[buf * BSB + r] = sx.e;
        } else if (c == BSC) {
          sXo[(k / BSC) * BSB + r] = sx;
        }
      }
    }
  };
  // rows of the owned blocks b with lo <= b < hi minus conj(R[block k, rows])^T w_k
  auto update = [&](int k, int buf, int lo, int hi) {
    const int j0 = k * BSB, jb = bsz(k);
    int first = lo + ((rank - lo) % BSC + BSC) % BSC;
    for (int b2 = first; b2 < hi; b2 += 2 * BSC) {
      const int b = b2 + (r / BSB) * BSC;
      const int i = b * BSB + (r % BSB);
      const bool rowok = b < hi && (r % BSB) < bsz(b < nb ? b : 0);
      const bool act = rowok && c < jb;
      fx<KY> ur, ui;
      fx_zero<KY>(ur);
      fx_zero<KY>(ui);
      if (act) {
        const int j = j0 + c;
        const fx<K> *e = (const fx<K> *)(Rm + ((int64_t)i * ldr + j) * W);  // r_ji, column i
        fx<K> z;
        fx_zero<K>(z);
        const int d = (int)sexp[i] + sTc[buf * BSB + c] - sig;
        bs_update<K, KY>(ur, ui, e[0], ix_sub<K>(z, e[1]), sXc[2 * (buf * BSB + c)],
                         sXc[2 * (buf * BSB + c) + 1], d, sFail);
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        fx<KY> a, bb;
#pragma unroll
        for (int q = 0; q < KY; q++) {
          a.w[q] = __shfl_xor_sync(0xffffffffu, ur.w[q], o);
          bb.w[q] = __shfl_xor_sync(0xffffffffu, ui.w[q], o);
        }
        ur = ix_add<KY>(ur, a);
        ui = ix_add<KY>(ui, bb);
      }
      if (c == 0 && rowok) {
        sY[2 * i] = ix_add<KY>(sY[2 * i], ur);
        sY[2 * i + 1] = ix_add<KY>(sY[2 * i + 1], ui);
      }
    }
  };
  __syncthreads();
  cl.sync();
  if (run && rank == 0 % BSC) xstep(0, 0);
  cl.sync();
  for (int k = 0; k < nb - 1; k++) {
    const int buf = k & 1;
    if (run) {
      if (rank == (k + 1) % BSC) {
        update(k, buf, k + 1, k + 2);  // block k+1 first
        __syncthreads();
        xstep(k + 1, buf ^ 1);
      }
      update(k, buf, k + 2, nb);  // the other owned blocks below
    }
    cl.sync();
  }
  // the owned rows' unknowns to L-limb cascades, off the steps' chain
  if (run)
    for (int t = tid; t < bsc_own_rows(n); t += BSB_THREADS) {
      const int b = rank + BSC * (t / BSB), r = t % BSB;
      if (b >= nb || r >= bsz(b)) continue;
      const cf<K> sx = sXo[t];
      double cr[L], ci[L];
      const bool z = sx.e == CF_EZERO;
      fx_to_cascade<K, L>(sx.re, z ? 0 : -sx.e, cr);
      fx_to_cascade<K, L>(sx.im, z ? 0 : -sx.e, ci);
#pragma unroll
      for (int q = 0; q < L; q++) {
        w[(int64_t)(b * BSB + r) * W + q] = cr[q];
        w[(int64_t)(b * BSB + r) * W + L + q] = ci[q];
      }
    }
  if (*sFail && tid == 0) atomicCAS(status, GN_OK, GN_ENONFINITE);
}

template <int L>
__host__ __device__ constexpr size_t bsc_smem_bytes(int n) {
  return sizeof(fx<L + 2>) * 2 * (size_t)(n > 0 ? n : 1) + sizeof(fx<L>) * 2 * 2 * BSB +
         sizeof(cf<L>) * (size_t)bsc_own_rows(n) + sizeof(int) * (2 * BSB + 4);
}

}  // namespace gn
