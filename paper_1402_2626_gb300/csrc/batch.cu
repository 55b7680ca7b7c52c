// batch.cu — Gauss-Newton steps (Section 4) on many independent square
// systems at once.
//
// The systems are stored back to back in sparse distributed form (Section 1).
// One step is a CUDA graph: the evaluation kernels of eval_int.cu run once
// over every term of every system (variables renumbered into one
// concatenated vector x, each system's J and -f scattered straight into its
// own augmented matrix [J, -f]), then one persistent launch solves the least
// squares problems: every CTA takes systems from a queue ordered by
// decreasing size (largest first, so the last CTAs do not wait on a big
// one), runs MGS on the system's matrix in block floating point (Section 3,
// figure "The modified Gram-Schmidt orthogonalization algorithm": a warp per
// trailing column, the column after the pivot first so that the next pivot
// starts while the other columns are still being updated), back
// substitution (eq. 5) and x += dx.  Systems are independent, so nothing is
// exchanged between CTAs.  The CTA size is chosen by timing the candidates
// on the batch itself before the step is captured.
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <numeric>
#include <vector>

#include "bs.cuh"
#include "ifx.cuh"
#include "internal.h"
#include "mw.cuh"

namespace gn {

constexpr int BT_MAX_N = 128;  // largest system of the persistent solver

struct BatchWs {
  bool ready = false;
  double *pow = nullptr, *stage_val = nullptr, *stage_d = nullptr;
  double *A = nullptr, *Rm = nullptr, *Zs = nullptr;
  int32_t *zero = nullptr;     // status word the evaluation kernels read (always GN_OK)
  int32_t *counter = nullptr;  // [0] work queue position, [1] step index
  int threads = 0, grid = 0;   // tuned launch of the solver
  int eval_block = 128;        // tuned CTA size of the per-term evaluation kernel
  int eval_lanes = 1;          // tuned lanes per term of that kernel (1 or 2)
  int sorted = 1;              // solver queue: largest systems first (1) or as stored (0)
  cudaGraphExec_t exec = nullptr;
  const double *gx = nullptr;
  double *gnorms = nullptr;
  int32_t *gstatus = nullptr;
  int32_t gsteps = 0;  // steps the captured step can report norms for
};

}  // namespace gn

struct gn_batch {
  int32_t S = 0, max_n = 0, kmax = 0, dmax = 1, pmax = 1;
  int64_t X = 0, P = 0, T = 0, nnz = 0, nz = 0;
  int64_t A_total = 0, R_total = 0, C_total = 0;  // complex entries; C: sum of (n+1)
  int32_t *d_poly_ptr = nullptr, *d_mono_off = nullptr;
  uint32_t *d_occ = nullptr;
  double *d_coef = nullptr;
  int32_t *d_jz_ptr = nullptr, *d_jz_occ = nullptr;
  int64_t *d_jz_out = nullptr, *d_f_out = nullptr;
  int32_t *d_sys_n = nullptr, *d_order = nullptr, *d_order_id = nullptr;
  int64_t *d_x_off = nullptr, *d_A_off = nullptr, *d_R_off = nullptr, *d_C_off = nullptr;
  gn::BatchWs ws[5];
};

namespace gn {

template <typename T>
static gn_status bdalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc((void **)p, sizeof(T) * count) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return GN_ENOMEM;
  }
  return GN_OK;
}

template <typename T>
static gn_status bupload(T **p, const T *h, size_t count) {
  gn_status e = bdalloc(p, count);
  if (e) return e;
  if (count && cudaMemcpy(*p, h, sizeof(T) * count, cudaMemcpyHostToDevice) != cudaSuccess)
    return GN_ECUDA;
  return GN_OK;
}

static void bws_free(BatchWs &w) {
  if (w.exec) cudaGraphExecDestroy(w.exec);
  cudaFree(w.pow);
  cudaFree(w.stage_val);
  cudaFree(w.stage_d);
  cudaFree(w.A);
  cudaFree(w.Rm);
  cudaFree(w.Zs);
  cudaFree(w.zero);
  cudaFree(w.counter);
  w = BatchWs();
}

struct BsArgs {
  double *A, *Rm, *Zs, *x;
  const int64_t *A_off, *R_off, *C_off, *x_off;
  const int32_t *sys_n, *order;
  int32_t S;
  int32_t *counter;      // [0] queue, [1] step index
  int32_t *status;       // [S] per-system status (sticky)
  double *norms;         // [steps][S][2]: ||f||, ||dx|| (may be null)
  int32_t max_steps;
};

// ---- per-warp pieces of the integer MGS (one CTA per system) -------------

// conj(q)^T a over the N rows, lanes over rows; all lanes get the total
template <int K>
__device__ __forceinline__ void bt_dot(const fx<K> *q, const fx<K> *a, int N, fx<K + 1> &dr,
                                       fx<K + 1> &di) {
  const int lane = threadIdx.x & 31;
  fx_zero<K + 1>(dr);
  fx_zero<K + 1>(di);
  for (int r = lane; r < N; r += 32) {
    const fx<K> qr = q[2 * r], qi = q[2 * r + 1], ar = a[2 * r], ai = a[2 * r + 1];
    dr = ix_add<K + 1>(dr, ix_mul_shift<K>(qr, ar));
    dr = ix_add<K + 1>(dr, ix_mul_shift<K>(qi, ai));
    di = ix_add<K + 1>(di, ix_mul_shift<K>(qr, ai));
    di = ix_sub<K + 1>(di, ix_mul_shift<K>(qi, ar));
  }
  dr = warp_sum_fx<K + 1>(dr);
  di = warp_sum_fx<K + 1>(di);
}

// a <- a - r q over the N rows
template <int K>
__device__ __forceinline__ void bt_axpy(const fx<K> *q, fx<K> *a, int N, const fx<K> &rr,
                                        const fx<K> &ri) {
  const int lane = threadIdx.x & 31;
  for (int r = lane; r < N; r += 32) {
    const fx<K> qr = q[2 * r], qi = q[2 * r + 1];
    fx<K + 1> xr = ix_widen<K, K + 1>(a[2 * r]);
    fx<K + 1> xi = ix_widen<K, K + 1>(a[2 * r + 1]);
    xr = ix_sub<K + 1>(xr, ix_mul_shift<K>(rr, qr));
    xr = ix_add<K + 1>(xr, ix_mul_shift<K>(ri, qi));
    xi = ix_sub<K + 1>(xi, ix_mul_shift<K>(rr, qi));
    xi = ix_sub<K + 1>(xi, ix_mul_shift<K>(ri, qr));
    a[2 * r] = ix_narrow<K>(xr);
    a[2 * r + 1] = ix_narrow<K>(xi);
  }
}

template <int L>
__global__ void __launch_bounds__(256) k_batch_solve(BsArgs a) {
  constexpr int K = L, W = 2 * L, S = 64 * K - 2, KY = K + 2;
  __shared__ int sS[BT_MAX_N + 1];   // column exponents s_j
  __shared__ int sTb[BT_MAX_N + 1];  // rank-test bit lengths
  __shared__ fx<K> sZ[BT_MAX_N];     // mantissas of 1/r_jj
  __shared__ int sZe[BT_MAX_N];      // their exponents
  __shared__ fx<K> sX[2 * BT_MAX_N];  // x mantissas
  __shared__ int sT[BT_MAX_N];       // x exponents
  __shared__ double sFn;             // ||f||
  __shared__ double sRed[2][8];
  __shared__ int sSys, sBad, sFail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int step = a.counter[1];
  for (;;) {
    if (tid == 0) sSys = atomicAdd(a.counter, 1);
    __syncthreads();
    const int qi = sSys;
    if (qi >= a.S) break;
    const int s = a.order[qi];
    const int n = a.sys_n[s], N = n, ncols = n + 1;
    fx<K> *A = (fx<K> *)(a.A + a.A_off[s] * W);  // column j: A + 2 j N
    fx<K> *Rm = (fx<K> *)(a.Rm + a.R_off[s] * W);  // entry (k, j): Rm + 2 (j ncols + k)
    double *Zs = a.Zs + a.C_off[s] * (K + 1);
    double *x = a.x + a.x_off[s] * W;
    if (tid == 0) {
      sBad = a.status[s] != GN_OK;
      sFail = 0;
    }
    __syncthreads();
    if (sBad) continue;  // a system that failed an earlier step is left as it is
    // original column norms (double), exponents, rank thresholds
    for (int c = warp; c < ncols; c += nw) {
      const double *cp = (const double *)(A + 2 * (size_t)c * N);
      double t = 0.0;
      for (int r = lane; r < N; r += 32) {
        const double re = cp[(size_t)r * W], im = cp[(size_t)r * W + L];
        t = fma(re, re, fma(im, im, t));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) {
        const double n0 = sqrt(t);
        if (!isfinite(n0)) sFail = 1;  // a NaN or an infinity in the column
        const int sj = fx_exponent_of(n0 * 1.0000001 + 1e-300) - S;
        sS[c] = sj;
        sTb[c] = 2 * (fx_exponent_of(n0) - 1 + 8 - 50 * L - sj) + 1;
        if (c == n) sFn = n0;
      }
    }
    __syncthreads();
    // to mantissas in place
    for (int c = warp; c < ncols; c += nw) {
      fx<K> *col = A + 2 * (size_t)c * N;
      const int F = -sS[c];
      for (int r = lane; r < N; r += 32) {
        const double *e = (const double *)(col + 2 * r);
        double d[2 * L];
#pragma unroll
        for (int l = 0; l < 2 * L; l++) d[l] = e[l];
        fx<K> re, im;
        fx_zero<K>(re);
        fx_zero<K>(im);
        bool ok = true;
#pragma unroll
        for (int l = 0; l < L; l++) {
          ok &= fx_add_double<K>(re, d[l], F);
          ok &= fx_add_double<K>(im, d[L + l], F);
        }
        if (!ok) sFail = 1;
        col[2 * r] = re;
        col[2 * r + 1] = im;
      }
    }
    __syncthreads();
    // pivot j by one warp: norm, 1/||a_j||, rank test, normalisation
    auto pivot = [&](int j) {
      fx<K> *aj = A + 2 * (size_t)j * N;
      fx<2 * K + 1> t;
      fx_zero<2 * K + 1>(t);
      for (int r = lane; r < N; r += 32) {
        t = ix_add<2 * K + 1>(t, ix_square<K>(aj[2 * r]));
        t = ix_add<2 * K + 1>(t, ix_square<K>(aj[2 * r + 1]));
      }
      t = warp_sum_fx<2 * K + 1>(t);
      if (j == n) return;  // the residual column is not normalised
      fx<K> Z;
      fx_zero<K>(Z);
      int b = 0, accept = 0;
      if (lane == 0) {
        const int bl = ix_bitlen<2 * K + 1>(t);
        b = (bl + 1) >> 1;
        accept = bl > sTb[j];
        if (!accept && !sFail) sFail = 2;  // a non-finite input is reported as such
        ux<K> tt;
        const int d = 2 * b - 64 * K;
        const fx<2 * K + 1> sh = d >= 0 ? ix_sar<2 * K + 1>(t, d) : ix_shl<2 * K + 1>(t, -d);
#pragma unroll
        for (int w = 0; w < K; w++) tt.w[w] = sh.w[w];
        if (accept) {
          const ux<K> Y = ix_rsqrt_frac<K>(tt);
#pragma unroll
          for (int w = 0; w < K; w++) Z.w[w] = (Y.w[w] >> 1) | ((w + 1 < K) ? (Y.w[w + 1] << 63) : 0);
        }
        sZ[j] = Z;
        sZe[j] = -(b + 64 * K - 3) - sS[j];  // 1/r_jj = Z 2^this
      }
#pragma unroll
      for (int w = 0; w < K; w++) Z.w[w] = __shfl_sync(0xffffffffu, Z.w[w], 0);
      b = __shfl_sync(0xffffffffu, b, 0);
      accept = __shfl_sync(0xffffffffu, accept, 0);
      if (!accept) return;
      uint64_t nz;
      const ux<K> uz = ix_abs<K>(Z, nz);
      for (int e = lane; e < 2 * N; e += 32) {
        uint64_t na;
        const ux<K> ua = ix_abs<K>(aj[e], na);
        const ux<2 * K> p = ix_umul<K>(ua, uz);
        fx<2 * K> pf;
#pragma unroll
        for (int w = 0; w < 2 * K; w++) pf.w[w] = p.w[w];
        pf = ix_sar<2 * K>(pf, b - 1);
        fx<K> q;
#pragma unroll
        for (int w = 0; w < K; w++) q.w[w] = pf.w[w];
        ix_cneg<K>(q, na);
        aj[e] = q;
      }
    };
    if (warp == 0) pivot(0);
    __syncthreads();
    for (int k = 0; k < n; k++) {
      const fx<K> *qk = A + 2 * (size_t)k * N;
      // warp w takes columns k+1+w, k+1+w+nw, ...: warp 0 updates column k+1
      // first and pivots it at once
      for (int j = k + 1 + warp; j < ncols; j += nw) {
        fx<K> *aj = A + 2 * (size_t)j * N;
        fx<K + 1> dr, di;
        bt_dot<K>(qk, aj, N, dr, di);
        const fx<K> rr = ix_narrow<K>(dr), ri = ix_narrow<K>(di);
        bt_axpy<K>(qk, aj, N, rr, ri);
        if (lane == 0) {
          fx<K> *rm = Rm + 2 * ((size_t)j * ncols + k);
          rm[0] = rr;
          rm[1] = ri;
        }
        if (j == k + 1) pivot(k + 1);
      }
      __syncthreads();
    }
    if (tid == 0 && sFail) atomicCAS(a.status + s, GN_OK, sFail == 2 ? GN_ESINGULAR : GN_ENONFINITE);
    if (sFail) continue;  // uniform: read after the barrier above
    // back substitution R x = y, one thread per row (rows i < n), y at the
    // scale of the last column
    const int sig = sS[n];
    fx<KY> Y[2];
    if (tid < n) {
      const fx<K> *e = Rm + 2 * ((size_t)n * ncols + tid);
      Y[0] = ix_widen<K, KY>(e[0]);
      Y[1] = ix_widen<K, KY>(e[1]);
    }
    if (tid == n - 1) {
      fx<K> xr, xi;
      int t;
      bs_solve<K, KY>(Y[0], Y[1], sZ[n - 1], sZe[n - 1], sig, xr, xi, t);
      sX[2 * (n - 1)] = xr;
      sX[2 * (n - 1) + 1] = xi;
      sT[n - 1] = t;
    }
    __syncthreads();
    fx<K> Rr, Ri;
    if (tid < n - 1) {
      const fx<K> *e = Rm + 2 * ((size_t)(n - 1) * ncols + tid);
      Rr = e[0];
      Ri = e[1];
    }
    for (int l = n - 1; l >= 1; l--) {
      fx<K> Nr, Ni;  // next level's r_il, loaded while this level runs
      if (tid < l - 1) {
        const fx<K> *e = Rm + 2 * ((size_t)(l - 1) * ncols + tid);
        Nr = e[0];
        Ni = e[1];
      }
      if (tid < l) {
        const int d = sS[l] + sT[l] - sig;
        bs_update<K, KY>(Y[0], Y[1], Rr, Ri, sX[2 * l], sX[2 * l + 1], d, &sFail);
        if (tid == l - 1) {
          fx<K> xr, xi;
          int t;
          bs_solve<K, KY>(Y[0], Y[1], sZ[l - 1], sZe[l - 1], sig, xr, xi, t);
          sX[2 * (l - 1)] = xr;
          sX[2 * (l - 1) + 1] = xi;
          sT[l - 1] = t;
        }
      }
      Rr = Nr;
      Ri = Ni;
      __syncthreads();
    }
    // x += dx and the norms
    double sd = 0.0;
    for (int i = tid; i < n; i += blockDim.x) {
      cx<L> d;
      fx_to_cascade<K, L>(sX[2 * i], -sT[i], d.re);
      fx_to_cascade<K, L>(sX[2 * i + 1], -sT[i], d.im);
      sd = fma(d.re[0], d.re[0], fma(d.im[0], d.im[0], sd));
      c_store<L>(x + (size_t)i * W, c_add<L>(c_load<L>(x + (size_t)i * W), d));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(0xffffffffu, sd, o);
    if (lane == 0) sRed[0][warp] = sd;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; w++) t += sRed[0][w];
      if (sFail || !isfinite(t)) atomicCAS(a.status + s, GN_OK, GN_ENONFINITE);
      if (a.norms && step >= 0 && step < a.max_steps) {
        a.norms[((size_t)step * a.S + s) * 2] = sFn;
        a.norms[((size_t)step * a.S + s) * 2 + 1] = sqrt(t);
      }
    }
  }
}

__global__ void k_batch_next_step(int32_t *counter) {
  counter[0] = 0;
  counter[1] += 1;
}

static gn_status bws_get(gn_batch *b, int L, BatchWs **out) {
  BatchWs &w = b->ws[L];
  *out = &w;
  if (w.ready) return GN_OK;
  const size_t SW = stage_words(L), W = 2 * (size_t)L;
  gn_status e = GN_OK;
  if (!e) e = bdalloc(&w.pow, SW * b->X * b->pmax);
  if (!e) e = bdalloc(&w.stage_val, SW * b->T);
  if (!e) e = bdalloc(&w.stage_d, SW * b->nnz);
  if (!e) e = bdalloc(&w.A, W * b->A_total);
  if (!e) e = bdalloc(&w.Rm, W * b->R_total);
  if (!e) e = bdalloc(&w.Zs, (size_t)(L + 1) * b->C_total);
  if (!e) e = bdalloc(&w.zero, 1);
  if (!e) e = bdalloc(&w.counter, 2);
  if (!e && cudaMemset(w.zero, 0, sizeof(int32_t)) != cudaSuccess) e = GN_ECUDA;
  if (e) {
    cudaGetLastError();
    bws_free(w);
    return e;
  }
  w.ready = true;
  return GN_OK;
}

static gn_status batch_eval(gn_batch *b, int L, BatchWs *w, const double *d_x, cudaStream_t st) {
  if (cudaMemsetAsync(w->A, 0, sizeof(double) * 2 * L * b->A_total, st) != cudaSuccess) return GN_ECUDA;
  EvalArgs a;
  a.x = d_x;
  a.nvar = b->X;
  a.pmax = b->pmax;
  a.kmax = b->kmax;
  a.pow = w->pow;
  a.stage_val = w->stage_val;
  a.stage_d = w->stage_d;
  a.T = b->T;
  a.mono_off = b->d_mono_off;
  a.occ = b->d_occ;
  a.coef = b->d_coef;
  a.nz = b->nz;
  a.jz_ptr = b->d_jz_ptr;
  a.jz_occ = b->d_jz_occ;
  a.jz_out = b->d_jz_out;
  a.J = w->A;
  a.npoly = b->P;
  a.poly_ptr = b->d_poly_ptr;
  a.f = w->A;
  a.f_out = b->d_f_out;
  a.neg_f = 1;
  a.status = w->zero;
  a.block = w->eval_block;
  a.lanes = w->eval_lanes;
  return launch_eval_int_raw(L, a, st);
}

template <int L>
static gn_status batch_solve_launch(gn_batch *b, BatchWs *w, double *d_x, double *norms, int32_t *status,
                                    int32_t max_steps, int threads, int grid, cudaStream_t st) {
  BsArgs a{w->A, w->Rm, w->Zs, d_x, b->d_A_off, b->d_R_off, b->d_C_off, b->d_x_off, b->d_sys_n,
           w->sorted ? b->d_order : b->d_order_id, b->S, w->counter, status, norms, max_steps};
  k_batch_solve<L><<<grid, threads, 0, st>>>(a);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

static gn_status batch_solve(gn_batch *b, int L, BatchWs *w, double *d_x, double *norms, int32_t *status,
                             int32_t max_steps, int threads, int grid, cudaStream_t st) {
  switch (L) {
    case 1: return batch_solve_launch<1>(b, w, d_x, norms, status, max_steps, threads, grid, st);
    case 2: return batch_solve_launch<2>(b, w, d_x, norms, status, max_steps, threads, grid, st);
    case 4: return batch_solve_launch<4>(b, w, d_x, norms, status, max_steps, threads, grid, st);
  }
  return GN_EINVAL;
}

template <int L>
static int batch_occupancy(int threads) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_solve<L>, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

// The batch's autotuner (outside any capture, on a copy of x): first the CTA
// size of the per-term evaluation kernel (64, 128 or 256 threads, one
// monomial per thread; the kernel is instruction-bound and keeps its forward
// products in local memory, so the CTA size moves occupancy and L1
// residency), timed over every term of the batch; then the solver's launch
// (CTA of 128 or 256 threads, grid = SMs x resident CTAs) and the order of
// its work queue (largest systems first, or as stored), timed over one
// solve of every system.  The fastest of each is kept.
static gn_status batch_tune(gn_batch *b, int L, BatchWs *w, const double *d_x, cudaStream_t st) {
  gn::Range nvtx_range("gn_batch_newton: tune launches");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return GN_ECUDA;
  double *xs = nullptr;
  int32_t *stv = nullptr;
  gn_status e = bdalloc(&xs, 2 * (size_t)L * b->X);
  if (!e) e = bdalloc(&stv, (size_t)b->S);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!e && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) e = GN_ECUDA;
  // x from the caller's copy, every system's status GN_OK, the queue at 0
  auto reset = [&]() -> gn_status {
    if (cudaMemcpyAsync(xs, d_x, sizeof(double) * 2 * L * b->X, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(stv, 0, sizeof(int32_t) * b->S, st) != cudaSuccess ||
        cudaMemsetAsync(w->counter, 0, sizeof(int32_t) * 2, st) != cudaSuccess)
      return GN_ECUDA;
    return GN_OK;
  };
  auto elapsed = [&](float &ms) -> gn_status {
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      return GN_ECUDA;
    return GN_OK;
  };
  // 1. the evaluation kernel's lanes per term and CTA size
  const int ecand[6][2] = {{1, 64}, {1, 128}, {1, 256}, {2, 64}, {2, 128}, {2, 256}};
  float best = 1e30f;
  int eb = 128, el = 1;
  for (int c = 0; c < 6 && !e; c++) {
    w->eval_lanes = ecand[c][0];
    w->eval_block = ecand[c][1];
    e = reset();
    if (!e) e = batch_eval(b, L, w, xs, st);  // warm-up
    if (e) break;
    cudaEventRecord(e0, st);
    e = batch_eval(b, L, w, xs, st);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (!e) e = elapsed(ms);
    if (!e && ms < best) {
      best = ms;
      el = ecand[c][0];
      eb = ecand[c][1];
    }
  }
  w->eval_lanes = el;
  w->eval_block = eb;
  // 2. the solver's CTA size and queue order
  const int cand[2] = {128, 256};
  best = 1e30f;
  w->threads = 0;
  int keep_sorted = 1;
  for (int c = 0; c < 2 && !e; c++) {
    const int th = cand[c];
    if (th < std::min(b->max_n, 256)) continue;  // back substitution needs a thread per row
    int occ = 0;
    switch (L) {
      case 1: occ = batch_occupancy<1>(th); break;
      case 2: occ = batch_occupancy<2>(th); break;
      case 4: occ = batch_occupancy<4>(th); break;
    }
    if (occ <= 0) continue;
    const int grid = sms * occ;
    for (int sorted = 1; sorted >= 0 && !e; sorted--) {
      w->sorted = sorted;
      e = reset();
      if (!e) e = batch_eval(b, L, w, xs, st);
      if (e) break;
      cudaEventRecord(e0, st);
      e = batch_solve(b, L, w, xs, nullptr, stv, 0, th, grid, st);
      cudaEventRecord(e1, st);
      float ms = 0.f;
      if (!e) e = elapsed(ms);
      if (!e && ms < best) {
        best = ms;
        w->threads = th;
        w->grid = grid;
        keep_sorted = sorted;
      }
    }
  }
  w->sorted = keep_sorted;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(xs);
  cudaFree(stv);
  if (!e && !w->threads) e = GN_ECUDA;
  if (e) w->threads = 0;
  return e;
}

static gn_status batch_capture(gn_batch *b, int L, BatchWs *w, double *d_x, double *norms, int32_t *status,
                               int32_t max_steps) {
  gn::Range nvtx_range("gn_batch_newton: capture step graph");
  if (w->exec) {
    cudaGraphExecDestroy(w->exec);
    w->exec = nullptr;
  }
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return GN_ECUDA;
  gn_status e = GN_OK;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) e = GN_ECUDA;
  if (!e) {
    e = batch_eval(b, L, w, d_x, cap);
    if (!e) e = batch_solve(b, L, w, d_x, norms, status, max_steps, w->threads, w->grid, cap);
    if (!e) {
      k_batch_next_step<<<1, 1, 0, cap>>>(w->counter);
      if (cudaPeekAtLastError() != cudaSuccess) e = GN_ECUDA;
    }
    if (cudaStreamEndCapture(cap, &g) != cudaSuccess && !e) e = GN_ECUDA;
  }
  if (!e && cudaGraphInstantiate(&w->exec, g, 0) != cudaSuccess) e = GN_ECUDA;
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (e) {
    cudaGetLastError();
    w->exec = nullptr;
    return e;
  }
  w->gx = d_x;
  w->gnorms = norms;
  w->gstatus = status;
  w->gsteps = max_steps;
  return GN_OK;
}

}  // namespace gn

using namespace gn;

extern "C" {

gn_status gn_batch_create(gn_batch **out, int32_t S, const int64_t *h_sys_n, int64_t T,
                          const int64_t *h_poly_ptr, const int64_t *h_mono_ptr, const int32_t *h_var,
                          const uint8_t *h_exp, const double *h_coef, int32_t coef_limbs) {
  gn::Range nvtx_range("gn_batch_create");
  if (!out) return GN_EINVAL;
  *out = nullptr;
  if (S < 1 || T < 0 || !h_sys_n || !h_poly_ptr || !h_mono_ptr || (T > 0 && !h_coef) ||
      !(coef_limbs == 1 || coef_limbs == 2 || coef_limbs == 4))
    return GN_EINVAL;
  std::vector<int64_t> x_off(S + 1, 0);
  int32_t max_n = 0;
  for (int32_t s = 0; s < S; s++) {
    if (h_sys_n[s] < 1 || h_sys_n[s] > BT_MAX_N) return GN_EINVAL;
    x_off[s + 1] = x_off[s] + h_sys_n[s];
    max_n = std::max(max_n, (int32_t)h_sys_n[s]);
  }
  const int64_t X = x_off[S], P = X;  // square systems: N_s = n_s
  if (h_poly_ptr[0] != 0 || h_poly_ptr[P] != T || h_mono_ptr[0] != 0) return GN_EINVAL;
  for (int64_t i = 0; i < P; i++)
    if (h_poly_ptr[i + 1] < h_poly_ptr[i]) return GN_EINVAL;
  for (int64_t t = 0; t < T; t++)
    if (h_mono_ptr[t + 1] < h_mono_ptr[t]) return GN_EINVAL;
  const int64_t nnz = h_mono_ptr[T];
  if (nnz >= ((int64_t)1 << 31) || T >= ((int64_t)1 << 31) || X >= (1 << 24)) return GN_EINVAL;
  if (nnz > 0 && (!h_var || !h_exp)) return GN_EINVAL;

  gn_batch *b = new (std::nothrow) gn_batch();
  if (!b) return GN_ENOMEM;
  b->S = S;
  b->X = X;
  b->P = P;
  b->T = T;
  b->nnz = nnz;
  b->max_n = max_n;

  // per occurrence: its system, global variable, row; validation
  std::vector<uint32_t> occ(nnz);
  std::vector<int32_t> occ_row(nnz);
  std::vector<int64_t> seen(max_n, -1);
  int32_t kmax = 0, dmax = 1;
  for (int32_t s = 0; s < S; s++) {
    const int32_t n = (int32_t)h_sys_n[s];
    for (int64_t i = x_off[s]; i < x_off[s + 1]; i++) {
      for (int64_t t = h_poly_ptr[i]; t < h_poly_ptr[i + 1]; t++) {
        kmax = std::max(kmax, (int32_t)(h_mono_ptr[t + 1] - h_mono_ptr[t]));
        for (int64_t o = h_mono_ptr[t]; o < h_mono_ptr[t + 1]; o++) {
          const int32_t v = h_var[o];
          if (v < 0 || v >= n || h_exp[o] < 1 || seen[v] == t) {
            delete b;
            return GN_EINVAL;
          }
          seen[v] = t;
          dmax = std::max(dmax, (int32_t)h_exp[o]);
          occ[o] = ((uint32_t)(x_off[s] + v) << 8) | (uint32_t)h_exp[o];
          occ_row[o] = (int32_t)i;
        }
      }
    }
  }
  b->kmax = kmax;
  b->dmax = dmax;
  b->pmax = std::max(dmax - 1, 1);

  // augmented matrices: system s is N x (n+1) at A_off[s], R (n+1)^2 at R_off[s]
  std::vector<int64_t> A_off(S), R_off(S), C_off(S);
  int64_t A = 0, R = 0, C = 0;
  for (int32_t s = 0; s < S; s++) {
    const int64_t n = h_sys_n[s];
    A_off[s] = A;
    R_off[s] = R;
    C_off[s] = C;
    A += n * (n + 1);
    R += (n + 1) * (n + 1);
    C += n + 1;
  }
  b->A_total = A;
  b->R_total = R;
  b->C_total = C;
  std::vector<int32_t> sys_of_var(X);
  for (int32_t s = 0; s < S; s++)
    for (int64_t v = x_off[s]; v < x_off[s + 1]; v++) sys_of_var[v] = s;

  // Jacobian pattern over the global columns: occurrences bucketed by column
  // (stable), runs of equal rows are entries; each entry's place in its
  // system's matrix (column-major, ld n)
  std::vector<int64_t> col_start(X + 1, 0);
  for (int64_t o = 0; o < nnz; o++) col_start[(occ[o] >> 8) + 1]++;
  for (int64_t v = 0; v < X; v++) col_start[v + 1] += col_start[v];
  std::vector<int32_t> by_col(nnz);
  {
    std::vector<int64_t> fill(col_start.begin(), col_start.end() - 1);
    for (int64_t o = 0; o < nnz; o++) by_col[fill[occ[o] >> 8]++] = (int32_t)o;
  }
  std::vector<int32_t> jz_ptr;
  std::vector<int64_t> jz_out;
  for (int64_t v = 0; v < X; v++) {
    const int32_t s = sys_of_var[v];
    const int64_t n = h_sys_n[s];
    for (int64_t p = col_start[v]; p < col_start[v + 1]; p++) {
      const int64_t r = occ_row[by_col[p]];  // global row of the entry
      if (p == col_start[v] || occ_row[by_col[p - 1]] != r) {
        jz_ptr.push_back((int32_t)p);
        jz_out.push_back(A_off[s] + (v - x_off[s]) * n + (r - x_off[s]));
      }
    }
  }
  jz_ptr.push_back((int32_t)nnz);
  b->nz = (int64_t)jz_out.size();
  std::vector<int64_t> f_out(P);
  for (int32_t s = 0; s < S; s++) {
    const int64_t n = h_sys_n[s];
    for (int64_t i = 0; i < n; i++) f_out[x_off[s] + i] = A_off[s] + n * n + i;
  }
  // largest systems first
  std::vector<int32_t> order(S), sys_n(S);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t p, int32_t q) { return h_sys_n[p] > h_sys_n[q]; });
  for (int32_t s = 0; s < S; s++) sys_n[s] = (int32_t)h_sys_n[s];

  std::vector<int32_t> poly_ptr(P + 1), mono_off(T + 1);
  for (int64_t i = 0; i <= P; i++) poly_ptr[i] = (int32_t)h_poly_ptr[i];
  for (int64_t t = 0; t <= T; t++) mono_off[t] = (int32_t)h_mono_ptr[t];
  std::vector<double> coef((size_t)8 * T, 0.0);
  for (int64_t t = 0; t < T; t++)
    for (int part = 0; part < 2; part++)
      for (int l = 0; l < coef_limbs; l++)
        coef[(size_t)(2 * l + part) * T + t] = h_coef[(t * 2 + part) * coef_limbs + l];

  gn_status e = GN_OK;
  if (!e) e = bupload(&b->d_poly_ptr, poly_ptr.data(), poly_ptr.size());
  if (!e) e = bupload(&b->d_mono_off, mono_off.data(), mono_off.size());
  if (!e) e = bupload(&b->d_occ, occ.data(), occ.size());
  if (!e) e = bupload(&b->d_coef, coef.data(), coef.size());
  if (!e) e = bupload(&b->d_jz_ptr, jz_ptr.data(), jz_ptr.size());
  if (!e) e = bupload(&b->d_jz_occ, by_col.data(), by_col.size());
  if (!e) e = bupload(&b->d_jz_out, jz_out.data(), jz_out.size());
  if (!e) e = bupload(&b->d_f_out, f_out.data(), f_out.size());
  if (!e) e = bupload(&b->d_sys_n, sys_n.data(), sys_n.size());
  if (!e) e = bupload(&b->d_order, order.data(), order.size());
  std::iota(order.begin(), order.end(), 0);  // the queue as stored
  if (!e) e = bupload(&b->d_order_id, order.data(), order.size());
  if (!e) e = bupload(&b->d_x_off, x_off.data(), x_off.size());
  if (!e) e = bupload(&b->d_A_off, A_off.data(), A_off.size());
  if (!e) e = bupload(&b->d_R_off, R_off.data(), R_off.size());
  if (!e) e = bupload(&b->d_C_off, C_off.data(), C_off.size());
  if (e) {
    gn_batch_destroy(b);
    return e;
  }
  *out = b;
  return GN_OK;
}

gn_status gn_batch_destroy(gn_batch *b) {
  if (!b) return GN_EINVAL;
  cudaDeviceSynchronize();
  for (BatchWs &w : b->ws) bws_free(w);
  cudaFree(b->d_poly_ptr);
  cudaFree(b->d_mono_off);
  cudaFree(b->d_occ);
  cudaFree(b->d_coef);
  cudaFree(b->d_jz_ptr);
  cudaFree(b->d_jz_occ);
  cudaFree(b->d_jz_out);
  cudaFree(b->d_f_out);
  cudaFree(b->d_sys_n);
  cudaFree(b->d_order);
  cudaFree(b->d_order_id);
  cudaFree(b->d_x_off);
  cudaFree(b->d_A_off);
  cudaFree(b->d_R_off);
  cudaFree(b->d_C_off);
  delete b;
  return GN_OK;
}

gn_status gn_batch_info(const gn_batch *b, int32_t *S, int64_t *X, int64_t *T, int64_t *nnz,
                        int32_t *max_n) {
  if (!b) return GN_EINVAL;
  if (S) *S = b->S;
  if (X) *X = b->X;
  if (T) *T = b->T;
  if (nnz) *nnz = b->nnz;
  if (max_n) *max_n = b->max_n;
  return GN_OK;
}

gn_status gn_batch_tuning(const gn_batch *b, gn_prec prec, int32_t *eval_block, int32_t *eval_lanes,
                          int32_t *solve_threads, int32_t *solve_grid, int32_t *largest_first) {
  if (!b || !(prec == 1 || prec == 2 || prec == 4)) return GN_EINVAL;
  const BatchWs &w = b->ws[prec];
  if (!w.threads) return GN_EINVAL;  // not tuned yet
  if (eval_block) *eval_block = w.eval_block;
  if (eval_lanes) *eval_lanes = w.eval_lanes;
  if (solve_threads) *solve_threads = w.threads;
  if (solve_grid) *solve_grid = w.grid;
  if (largest_first) *largest_first = w.sorted;
  return GN_OK;
}

gn_status gn_batch_newton(gn_batch *b, gn_prec prec, double *d_x, int32_t steps, double *d_norms,
                          int32_t *d_status, void *cuda_stream) {
  gn::Range nvtx_range("gn_batch_newton");
  if (!b || !(prec == 1 || prec == 2 || prec == 4) || !d_x || !d_status || steps < 1 || b->kmax > 64)
    return GN_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  BatchWs *w;
  gn_status e = bws_get(b, prec, &w);
  if (e) return e;
  if (!w->threads) {
    e = batch_tune(b, prec, w, d_x, st);
    if (e) return e;
  }
  if (!w->exec || w->gx != d_x || w->gnorms != d_norms || w->gstatus != d_status ||
      (d_norms && steps > w->gsteps)) {
    e = batch_capture(b, prec, w, d_x, d_norms, d_status, steps);
    if (e) return e;
  }
  // the step index (for the norms) restarts at 0; the queue is reset by each step
  if (cudaMemsetAsync(w->counter, 0, sizeof(int32_t) * 2, st) != cudaSuccess) return GN_ECUDA;
  for (int32_t k = 0; k < steps; k++)
    if (cudaGraphLaunch(w->exec, st) != cudaSuccess) return GN_ECUDA;
  return GN_OK;
}

}  // extern "C"
