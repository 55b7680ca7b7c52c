// cholqr.cu — the double-precision factorisation of the mixed-precision
// solver as CholeskyQR: R of [A b] = QR from the Gram matrix G = [A b]^H [A b]
// = R^H R, without forming Q.
//
// Section 5.2 of Verschelde & Yu finds the linear solve dominant and points
// to methods in double arithmetic; the mixed solver (mixed.cu) needs one
// double factorisation per double Gauss-Newton step.  For a tall matrix MGS
// (Section 3) is a chain of n dependent pivots whose bulk updates of the
// later columns set its pace; here the O(m n^2) work becomes one
// throughput-bound contraction on the integer pipe (the exact Gram matrix of
// the columns' 62-bit mantissas), and only an O(n^3 / 3) Cholesky in FP64 is
// left.  The factor's last column is y = R^-H A^H b and R_nn = ||b - A x||,
// as MGS on [A b] gives them (eq. 2), so the Gauss-Newton step and the
// refinement's y = R^-H (A^H b) reuse the blocked integer triangular solves
// (bsb.cuh) once R is in their mantissa format.
//
// Accuracy: R from the Cholesky of the Gram matrix has a relative error of
// about kappa(A)^2 u_double (against kappa u for MGS); the refinement only
// needs the double factors to contract, which they do for kappa(A)^2 u << 1
// (the mixed workload's Jacobian has kappa = 15).  Rank: a pivot below
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

// G_ij = sum_r conj(a_ri) a_rj for i <= j (the upper triangle of G, column-
// major, leading dimension nc), exactly: the entries as 62-bit mantissas at
// their columns' scales, each product 124 bits, the sums (N < 2^30 terms) in
// three limbs, rounded to a double once at the end.  One CTA per 32 x 32
// tile (ib <= jb) of 256 threads, thread (ty, tx) owning entries
// (2 ty + {0,1}, 2 tx + {0,1}); rows in chunks of 32 staged in shared memory
// as mantissas.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_gram(const double *__restrict__ A, int32_t N, int32_t nc,
                                                        const double *__restrict__ sexp,
                                                        double *__restrict__ G,
                                                        const int32_t *__restrict__ status) {
  __shared__ int64_t sI[CQ_T][CQ_T][2];  // [row][column of the i tile][re, im]
  __shared__ int64_t sJ[CQ_T][CQ_T][2];
  if (*status != GN_OK) return;
  int ib, jb;
  cq_tile(blockIdx.x, ib, jb);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  fx<3> cr[2][2], ci[2][2];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      fx_zero<3>(cr[a][b]);
      fx_zero<3>(ci[a][b]);
    }
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
        int64_t(*dst)[CQ_T][2] = side ? sJ : sI;
        dst[rr][cc][0] = (int64_t)mr.w[0];
        dst[rr][cc][1] = (int64_t)mi.w[0];
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < CQ_T; rr++) {
      fx<1> ar[2], ai[2], br[2], bi[2];
#pragma unroll
      for (int a = 0; a < 2; a++) {
        ar[a].w[0] = (uint64_t)sI[rr][2 * ty + a][0];
        ai[a].w[0] = (uint64_t)sI[rr][2 * ty + a][1];
        br[a].w[0] = (uint64_t)sJ[rr][2 * tx + a][0];
        bi[a].w[0] = (uint64_t)sJ[rr][2 * tx + a][1];
      }
#pragma unroll
      for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 2; b++) {
          // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
          cr[a][b] = ix_add<3>(cr[a][b], ix_widen<2, 3>(ix_mul_full<1, 1>(ar[a], br[b])));
          cr[a][b] = ix_add<3>(cr[a][b], ix_widen<2, 3>(ix_mul_full<1, 1>(ai[a], bi[b])));
          ci[a][b] = ix_add<3>(ci[a][b], ix_widen<2, 3>(ix_mul_full<1, 1>(ar[a], bi[b])));
          ci[a][b] = ix_sub<3>(ci[a][b], ix_widen<2, 3>(ix_mul_full<1, 1>(ai[a], br[b])));
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
        double re[1], im[1];
        fx_to_cascade<3, 1>(cr[a][b], F, re);
        fx_to_cascade<3, 1>(ci[a][b], F, im);
        G[((int64_t)j * nc + i) * 2] = re[0];
        G[((int64_t)j * nc + i) * 2 + 1] = im[0];
      }
    }
}

// The panel's diagonal block G[p:pe, p:pe] = R11^H R11 (upper, in place) by
// one CTA in shared memory: for each k, r_kk = sqrt(g_kk), row k divided by
// r_kk, the block's trailing upper triangle less conj(r_ki) r_kj.  A pivot
// g_kk <= 2^-40 ||a_k||^2 (k < nchk) records GN_ESINGULAR.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_potrf(double *__restrict__ G, int32_t nc, int32_t p,
                                                         const double *__restrict__ nrm0, int32_t nchk,
                                                         int32_t *__restrict__ status) {
  __shared__ double2 sB[CQ_T][CQ_T];  // [row][column]
  __shared__ int sBad;
  if (*status != GN_OK) return;
  const int pb = min(CQ_T, nc - p);
  const int tid = threadIdx.x;
  for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
    const int i = q % CQ_T, j = q / CQ_T;
    double2 v = make_double2(0.0, 0.0);
    if (i < pb && j < pb && i <= j) {
      const double *e = G + ((int64_t)(p + j) * nc + p + i) * 2;
      v = make_double2(e[0], e[1]);
    }
    sB[i][j] = v;
  }
  if (tid == 0) sBad = 0;
  __syncthreads();
  for (int k = 0; k < pb; k++) {
    if (tid == 0) {
      const double d = sB[k][k].x;
      const double n0 = nrm0[p + k];
      const bool bad = !(d > ldexp(n0 * n0, -40));
      if (bad && p + k < nchk) {
        atomicCAS(status, GN_OK, GN_ESINGULAR);
        sBad = 1;
      }
      const double r = d > 0.0 ? sqrt(d) : 0.0;
      sB[k][k] = make_double2(r, 0.0);
    }
    __syncthreads();
    if (sBad) return;  // uniform: read after the barrier
    const double r = sB[k][k].x;
    const double inv = r > 0.0 ? 1.0 / r : 0.0;
    for (int j = k + 1 + tid; j < pb; j += CQ_THREADS) {
      sB[k][j].x *= inv;
      sB[k][j].y *= inv;
    }
    __syncthreads();
    // g_ij -= conj(r_ki) r_kj for k < i <= j < pb
    for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
      const int i = q % CQ_T, j = q / CQ_T;
      if (i > k && i <= j && j < pb) {
        const double2 a = sB[k][i], b = sB[k][j];
        sB[i][j].x -= a.x * b.x + a.y * b.y;
        sB[i][j].y -= a.x * b.y - a.y * b.x;
      }
    }
    __syncthreads();
  }
  for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
    const int i = q % CQ_T, j = q / CQ_T;
    if (i < pb && j < pb && i <= j) {
      double *e = G + ((int64_t)(p + j) * nc + p + i) * 2;
      e[0] = sB[i][j].x;
      e[1] = sB[i][j].y;
    }
  }
}

// The panel's rows to the right of its diagonal block: R12 = R11^-H G12, by
// forward substitution with R11^H (lower): one warp per column j >= pe,
// lane i holding row p + i; R11 staged in shared memory by each CTA.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_trsm(double *__restrict__ G, int32_t nc, int32_t p,
                                                        const int32_t *__restrict__ status) {
  __shared__ double2 sR[CQ_T][CQ_T];
  if (*status != GN_OK) return;
  const int pb = min(CQ_T, nc - p), pe = p + pb;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
    const int i = q % CQ_T, j = q / CQ_T;
    double2 v = make_double2(0.0, 0.0);
    if (i < pb && j < pb && i <= j) {
      const double *e = G + ((int64_t)(p + j) * nc + p + i) * 2;
      v = make_double2(e[0], e[1]);
    }
    sR[i][j] = v;
  }
  __syncthreads();
  const int j = pe + blockIdx.x * (CQ_THREADS / 32) + warp;
  if (j >= nc) return;  // whole warps
  double *col = G + (int64_t)j * nc * 2;
  double2 g = make_double2(0.0, 0.0);
  if (lane < pb) g = make_double2(col[2 * (p + lane)], col[2 * (p + lane) + 1]);
  for (int i = 0; i < pb; i++) {
    // x_i = g_i / r_ii (r_ii real), then g_k -= conj(r_ik) x_i for k > i
    const double rii = sR[i][i].x;
    const double inv = rii > 0.0 ? 1.0 / rii : 0.0;
    double2 xi = make_double2(0.0, 0.0);
    if (lane == i) {
      g.x *= inv;
      g.y *= inv;
      xi = g;
    }
    xi.x = __shfl_sync(0xffffffffu, xi.x, i);
    xi.y = __shfl_sync(0xffffffffu, xi.y, i);
    if (lane > i && lane < pb) {
      const double2 a = sR[i][lane];  // r_i,lane
      g.x -= a.x * xi.x + a.y * xi.y;
      g.y -= a.x * xi.y - a.y * xi.x;
    }
  }
  if (lane < pb) {
    col[2 * (p + lane)] = g.x;
    col[2 * (p + lane) + 1] = g.y;
  }
}

// The trailing matrix: G_ij -= sum_{k in the panel} conj(r_ki) r_kj for
// pe <= i <= j < nc, by 32 x 32 tiles (ib <= jb over the trailing range), 256
// threads of 2 x 2 entries, the panel's rows of both tiles' columns staged
// in shared memory.
__global__ void __launch_bounds__(CQ_THREADS) k_cq_herk(double *__restrict__ G, int32_t nc, int32_t p,
                                                        const int32_t *__restrict__ status) {
  __shared__ double2 sI[CQ_T][CQ_T];  // [panel row][column of the i tile]
  __shared__ double2 sJ[CQ_T][CQ_T];
  if (*status != GN_OK) return;
  const int pb = min(CQ_T, nc - p), pe = p + pb;
  int ib, jb;
  cq_tile(blockIdx.x, ib, jb);
  const int i0 = pe + ib * CQ_T, j0 = pe + jb * CQ_T;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int q = tid; q < CQ_T * CQ_T; q += CQ_THREADS) {
    const int k = q % CQ_T, c = q / CQ_T;
    double2 u = make_double2(0.0, 0.0), v = make_double2(0.0, 0.0);
    if (k < pb) {
      if (i0 + c < nc) {
        const double *e = G + ((int64_t)(i0 + c) * nc + p + k) * 2;
        u = make_double2(e[0], e[1]);
      }
      if (j0 + c < nc) {
        const double *e = G + ((int64_t)(j0 + c) * nc + p + k) * 2;
        v = make_double2(e[0], e[1]);
      }
    }
    sI[k][c] = u;
    sJ[k][c] = v;
  }
  __syncthreads();
  double2 acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) acc[a][b] = make_double2(0.0, 0.0);
  for (int k = 0; k < pb; k++) {
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
      for (int b = 0; b < 2; b++) {
        const double2 u = sI[k][2 * ty + a], v = sJ[k][2 * tx + b];
        acc[a][b].x = fma(u.x, v.x, fma(u.y, v.y, acc[a][b].x));
        acc[a][b].y = fma(u.x, v.y, fma(-u.y, v.x, acc[a][b].y));
      }
  }
#pragma unroll
  for (int a = 0; a < 2; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const int i = i0 + 2 * ty + a, j = j0 + 2 * tx + b;
      if (i < nc && j < nc && i <= j) {
        double *e = G + ((int64_t)j * nc + i) * 2;
        e[0] -= acc[a][b].x;
        e[1] -= acc[a][b].y;
      }
    }
}

// R (double, upper, leading dimension nc) into the mantissa format of the
// integer triangular solves: column j's entries as one-limb mantissas at
// 2^s_j (|r_kj| <= ||a_j|| < 2^(62 + s_j)), 1/r_jj as a mantissa in
// [2^61, 2^62) and its exponent (Zs), 1/r_jj as a double too.  One CTA per
// column.
__global__ void k_cq_to_int(const double *__restrict__ R, int32_t nc, const double *__restrict__ sexp,
                            double *__restrict__ Rm, double *__restrict__ Zs, double *__restrict__ rinv,
                            const int32_t *__restrict__ status) {
  if (*status != GN_OK) return;
  const int j = blockIdx.x;
  const int F = -(int)sexp[j];
  for (int k = threadIdx.x; k <= j; k += blockDim.x) {
    const double *e = R + ((int64_t)j * nc + k) * 2;
    long long *d = (long long *)(Rm + ((int64_t)j * nc + k) * 2);
    d[0] = llrint(ldexp(e[0], F));
    d[1] = llrint(ldexp(e[1], F));
  }
  if (threadIdx.x == 0 && j < nc - 1) {
    const double r = R[((int64_t)j * nc + j) * 2];
    const double v = r > 0.0 ? 1.0 / r : 0.0;
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
                        double *Zs, int32_t *status, cudaStream_t st) {
  const int32_t nc = n + 1;
  double *nrm0 = rinv + nc, *sexp = rinv + 2 * (size_t)nc;  // the layout of the one-limb rinv
  k_cq_scale<<<(unsigned)((nc * 32 + CQ_THREADS - 1) / CQ_THREADS), CQ_THREADS, 0, st>>>(A, N, nc, nrm0,
                                                                                      sexp, status);
  const int nb = (nc + CQ_T - 1) / CQ_T;
  k_cq_gram<<<(unsigned)(nb * (nb + 1) / 2), CQ_THREADS, 0, st>>>(A, N, nc, sexp, R, status);
  for (int p = 0; p < nc; p += CQ_T) {
    k_cq_potrf<<<1, CQ_THREADS, 0, st>>>(R, nc, p, nrm0, n, status);
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
