// mgs.cu — modified Gram-Schmidt on [A b] (Section 3 of Verschelde & Yu) as
// one persistent launch of thread-block clusters.
//
// The arithmetic per column is that of the figure "The modified
// Gram-Schmidt orthogonalization algorithm": column j receives, in order
// k = 0, 1, ..., j-1, r_kj = q_k^H a_j and a_j <- a_j - r_kj q_k, then
// r_jj = ||a_j||, q_j = a_j / r_jj.  Any schedule that keeps that order per
// column computes the same thing, so the work is laid out for GB300:
//
//   * G clusters of C = 8 CTAs, one CTA per SM.  Cluster g owns the columns
//     j = g (mod G); CTA rank r of every cluster owns rows [r ms, (r+1) ms).
//     The owner of column j publishes q_j row slice by row slice through a
//     flag per (j, r) in global memory (release/acquire); a CTA waits only for
//     the slice of q_k that its own rows need.  The owner of column k+1 treats
//     it first (lookahead), so the chain of pivots runs ahead of the bulk.
//   * Inner products and norms are summed exactly on the integer pipe
//     (fx.cuh): each CTA reduces its rows, the cluster adds the C partials
//     through distributed shared memory.  FP64 is spent only on the TwoProd
//     pieces of the products (mwfx.cuh).  The GPU's FP64 rate per SM is about
//     1/64 of its FP32 rate, and a CTA-wide tree of double-double additions
//     would put ~100 dependent FP64 instructions (64 cycles each) on the
//     critical path of every pivot.
//   * The K20C version launched one kernel per pivot and delayed each
//     normalisation by a step so blocks would not read a half-normalised
//     column; here the flags give that ordering inside one launch.
//
// Every wait is bounded (about one second); a wait that gives up records
// GN_ETIMEOUT and every CTA of the cluster leaves together, so no CTA is
// left at a cluster barrier.
#include <cooperative_groups.h>

#include <mutex>

#include "ifx.cuh"
#include "internal.h"
#include "mwfx.cuh"

namespace cg = cooperative_groups;

namespace gn {

constexpr int MF_THREADS = 256;
constexpr int MF_WARPS = MF_THREADS / 32;
constexpr int MF_C = 8;                         // CTAs per cluster
constexpr long long MF_WAIT_CYCLES = 2000000000LL;  // bound of one wait (~1 s)
constexpr size_t MF_SMEM_FLOOR = 120 * 1024;    // keeps one CTA per SM

struct MfArgs {
  double *A;
  int32_t m;
  int64_t lda;
  int32_t ncols;
  double *R;
  int64_t ldr;
  double *rinv;
  double *nrm0;     // [ncols] original column norms (double), written for the report
  uint32_t *flags;  // [ncols][MF_C], zero at launch
  int32_t *status;
  double *Rm;       // r_kj mantissas (K limbs re, im) at column scale, layout of R; may be null
  double *Zs;       // per pivot: K limbs of 1/r_jj's mantissa, then its exponent (as double)
  int32_t G;
  int32_t maxown;
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int L>
__device__ __forceinline__ cx<L> ld_cg(const double *p) {
  cx<L> z;
#pragma unroll
  for (int l = 0; l < L; l++) {
    z.re[l] = __ldcg(p + l);
    z.im[l] = __ldcg(p + L + l);
  }
  return z;
}

// shared-memory layout, identical on host and device
template <int L>
struct MfLayout {
  static constexpr int NL = FxCfg<L>::NL;
  size_t oF, oN0, oN0p, oPart, oCrit, oWarp, oRb, oQ, oMisc, bytes;
  __host__ __device__ MfLayout(int maxown, int ms) {
    size_t o = 0;
    auto take = [&](size_t b) {
      size_t at = o;
      o += (b + 15) & ~(size_t)15;
      return at;
    };
    oF = take(sizeof(int) * maxown);
    oN0 = take(sizeof(double) * maxown);
    oN0p = take(sizeof(double) * maxown);
    oPart = take(sizeof(fx<NL>) * 4 * maxown);  // [2 buffers][maxown][re, im]
    oCrit = take(sizeof(fx<NL>) * 4);           // dot re, dot im, norm, pad
    oWarp = take(sizeof(fx<NL>) * 2 * MF_WARPS);
    oRb = take(sizeof(cx<L>) * (maxown + 1));
    oQ = take(sizeof(cx<L>) * (ms > 0 ? ms : 1));
    oMisc = take(64 + sizeof(double) * 2 * L);
    bytes = o;
  }
};

// Exact CTA-wide sum of two accumulators; the result is valid in thread 0.
template <int NL>
__device__ void cta_sum2(fx<NL> &a, fx<NL> &b, fx<NL> *sWarp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  a = fx_warp_sum<NL>(a);
  b = fx_warp_sum<NL>(b);
  __syncthreads();
  if (lane == 0) {
    sWarp[2 * warp] = a;
    sWarp[2 * warp + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < MF_WARPS; w++) {
      fx_add_to<NL>(a, sWarp[2 * w]);
      fx_add_to<NL>(b, sWarp[2 * w + 1]);
    }
  }
}

template <int L>
__global__ void __launch_bounds__(MF_THREADS, 1) k_mgs_flow(MfArgs a) {
  constexpr int NL = FxCfg<L>::NL;
  constexpr int BITS = FxCfg<L>::BITS;
  constexpr int W = 2 * L;
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int g = blockIdx.x / MF_C;
  const int G = a.G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = a.m, ncols = a.ncols;
  const int ms = (m + MF_C - 1) / MF_C;
  const int i0 = min(m, rank * ms), i1 = min(m, i0 + ms);
  const int no = (g < ncols) ? (ncols - g + G - 1) / G : 0;  // owned columns g + G c, c < no

  MfLayout<L> lay(a.maxown, ms);
  int *sF = (int *)(smem + lay.oF);
  double *sN0 = (double *)(smem + lay.oN0);
  double *sN0p = (double *)(smem + lay.oN0p);
  fx<NL> *sPart = (fx<NL> *)(smem + lay.oPart);
  fx<NL> *sCrit = (fx<NL> *)(smem + lay.oCrit);
  fx<NL> *sWarp = (fx<NL> *)(smem + lay.oWarp);
  cx<L> *sRb = (cx<L> *)(smem + lay.oRb);
  cx<L> *sQ = (cx<L> *)(smem + lay.oQ);
  int *sOk = (int *)(smem + lay.oMisc);            // this CTA's wait result, read by the cluster
  int *sCritOk = sOk + 1;                          // pivot accepted (identical in every CTA)
  double *sRinv = (double *)(smem + lay.oMisc + 16);
  bool ok = true;  // fx range checks of this thread

  // original column norms (double), for the rank test and the fixed-point scales
  for (int c = warp; c < no; c += MF_WARPS) {
    const double *col = a.A + (int64_t)(g + G * c) * a.lda * W;
    double s = 0.0;
    for (int i = i0 + lane; i < i1; i += 32) {
      double re = col[(int64_t)i * W], im = col[(int64_t)i * W + L];
      s = fma(re, re, fma(im, im, s));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sN0p[c] = s;
  }
  cl.sync();
  for (int c = tid; c < no; c += MF_THREADS) {
    double t = 0.0;
    for (int r = 0; r < MF_C; r++) t += cl.map_shared_rank(sN0p, r)[c];
    double n0 = sqrt(t);
    sN0[c] = n0;
    if (rank == 0) a.nrm0[g + G * c] = n0;
    sF[c] = BITS - fx_exponent_of(n0 * 1.0000001 + 1e-300);
  }
  __syncthreads();

  // pivot j: norm of column j (already updated by q_0..q_{j-1}), rank test,
  // normalisation and publication of q_j; for the last column only z = r_jj
  auto pivot = [&](int j, int c) {
    double *aj = a.A + (int64_t)j * a.lda * W;
    const int E = fx_exponent_of(sN0[c] * 1.0000001 + 1e-300);
    const int Fn = BITS - 2 * E;
    fx<NL> nr, dummy;
    fx_zero<NL>(nr);
    fx_zero<NL>(dummy);
    for (int i = i0 + tid; i < i1; i += MF_THREADS) {
      cx<L> x = c_load<L>(aj + (int64_t)i * W);
      ok &= fx_add_prod<L, NL>(nr, x.re, x.re, false, Fn);
      ok &= fx_add_prod<L, NL>(nr, x.im, x.im, false, Fn);
    }
    cta_sum2<NL>(nr, dummy, sWarp);
    if (tid == 0) sCrit[2] = nr;
    cl.sync();
    if (tid == 0) {
      fx<NL> t;
      fx_zero<NL>(t);
      for (int r = 0; r < MF_C; r++) fx_add_to<NL>(t, cl.map_shared_rank(sCrit, r)[2]);
      rl<L> s2;
      fx_to_cascade<NL, L>(t, Fn, s2.v);
      rl<L> rjj = r_sqrt<L>(s2);
      int accept = 1;
      if (!isfinite(rjj.v[0])) {
        accept = 0;
        atomicCAS(a.status, GN_OK, GN_ENONFINITE);
      } else if (j < ncols - 1) {
        if (!(rjj.v[0] > ldexp(sN0[c], 8 - 50 * L))) {
          accept = 0;
          atomicCAS(a.status, GN_OK, GN_ESINGULAR);
        } else {
          rl<L> inv = r_recip<L>(rjj);
#pragma unroll
          for (int l = 0; l < L; l++) sRinv[l] = inv.v[l];
          if (rank == 0)
            for (int l = 0; l < L; l++) a.rinv[(int64_t)j * L + l] = inv.v[l];
        }
      }
      if (rank == 0) {
        cx<L> rc = c_zero<L>();
#pragma unroll
        for (int l = 0; l < L; l++) rc.re[l] = rjj.v[l];
        c_store<L>(a.R + ((int64_t)j * a.ldr + j) * W, rc);
      }
      *sCritOk = accept;
    }
    __syncthreads();
    if (j < ncols - 1) {
      if (*sCritOk) {
        double inv[L];
#pragma unroll
        for (int l = 0; l < L; l++) inv[l] = sRinv[l];
        for (int i = i0 + tid; i < i1; i += MF_THREADS) {
          cx<L> x = c_load<L>(aj + (int64_t)i * W);
          c_store<L>(aj + (int64_t)i * W, fx_scale_real<L>(x, inv, BITS - 2, ok));
        }
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) st_release(a.flags + (size_t)j * MF_C + rank, *sCritOk ? 1u : 2u);
    }
  };

  if (g == 0 && no > 0) pivot(0, 0);

  for (int k = 0; k < ncols - 1; k++) {
    const int cstart = (k + 1 > g) ? (k + 1 - g + G - 1) / G : 0;
    if (cstart >= no) break;  // nothing left for this cluster (uniform)
    // wait for the rows of q_k that this CTA needs
    if (tid == 0) {
      const uint32_t *f = a.flags + (size_t)k * MF_C + rank;
      const long long t0 = clock64();
      uint32_t v;
      for (;;) {
        v = ld_acquire(f);
        if (v) break;
        if (*(volatile int32_t *)a.status != GN_OK) {
          v = 2;
          break;
        }
        if (clock64() - t0 > MF_WAIT_CYCLES) {
          atomicCAS(a.status, GN_OK, GN_ETIMEOUT);
          v = 2;
          break;
        }
        __nanosleep(32);
      }
      *sOk = (v == 1);
    }
    cl.sync();
    int allok = 1;
    for (int r = 0; r < MF_C; r++) allok &= *cl.map_shared_rank(sOk, r);
    if (!allok) break;  // uniform across the cluster
    const double *qk = a.A + (int64_t)k * a.lda * W;
    for (int i = i0 + tid; i < i1; i += MF_THREADS) sQ[i - i0] = ld_cg<L>(qk + (int64_t)i * W);
    __syncthreads();

    int cb = cstart;
    const int j1 = k + 1;
    if (j1 % G == g) {
      // lookahead: the next pivot column first
      const int c = (j1 - g) / G;
      double *aj = a.A + (int64_t)j1 * a.lda * W;
      const int F = sF[c];
      fx<NL> re, im;
      fx_zero<NL>(re);
      fx_zero<NL>(im);
      for (int i = i0 + tid; i < i1; i += MF_THREADS)
        ok &= fx_add_conj_prod<L, NL>(re, im, sQ[i - i0], c_load<L>(aj + (int64_t)i * W), F);
      cta_sum2<NL>(re, im, sWarp);
      if (tid == 0) {
        sCrit[0] = re;
        sCrit[1] = im;
      }
      cl.sync();
      if (tid == 0) {
        fx<NL> tr, ti;
        fx_zero<NL>(tr);
        fx_zero<NL>(ti);
        for (int r = 0; r < MF_C; r++) {
          fx<NL> *rc = cl.map_shared_rank(sCrit, r);
          fx_add_to<NL>(tr, rc[0]);
          fx_add_to<NL>(ti, rc[1]);
        }
        cx<L> rk;
        fx_to_cascade<NL, L>(tr, F, rk.re);
        fx_to_cascade<NL, L>(ti, F, rk.im);
        sRb[a.maxown] = rk;
        if (rank == 0) c_store<L>(a.R + ((int64_t)j1 * a.ldr + k) * W, rk);
      }
      __syncthreads();
      const cx<L> rk = sRb[a.maxown];
      for (int i = i0 + tid; i < i1; i += MF_THREADS) {
        cx<L> x = c_load<L>(aj + (int64_t)i * W);
        c_store<L>(aj + (int64_t)i * W, fx_axpy<L>(x, rk, sQ[i - i0], F, ok));
      }
      __syncthreads();
      pivot(j1, c);
      cb = c + 1;
    }
    // the rest of this cluster's columns
    const int nb = no - cb;
    if (nb > 0) {
      const int buf = k & 1;
      for (int cc = warp; cc < nb; cc += MF_WARPS) {
        const int c = cb + cc;
        const double *aj = a.A + (int64_t)(g + G * c) * a.lda * W;
        const int F = sF[c];
        fx<NL> re, im;
        fx_zero<NL>(re);
        fx_zero<NL>(im);
        for (int i = i0 + lane; i < i1; i += 32)
          ok &= fx_add_conj_prod<L, NL>(re, im, sQ[i - i0], c_load<L>(aj + (int64_t)i * W), F);
        re = fx_warp_sum<NL>(re);
        im = fx_warp_sum<NL>(im);
        if (lane == 0) {
          sPart[(buf * a.maxown + c) * 2] = re;
          sPart[(buf * a.maxown + c) * 2 + 1] = im;
        }
      }
      cl.sync();
      for (int cc = tid; cc < nb; cc += MF_THREADS) {
        const int c = cb + cc;
        fx<NL> tr, ti;
        fx_zero<NL>(tr);
        fx_zero<NL>(ti);
        for (int r = 0; r < MF_C; r++) {
          const fx<NL> *p = cl.map_shared_rank(sPart, r) + (buf * a.maxown + c) * 2;
          fx_add_to<NL>(tr, p[0]);
          fx_add_to<NL>(ti, p[1]);
        }
        cx<L> rk;
        fx_to_cascade<NL, L>(tr, sF[c], rk.re);
        fx_to_cascade<NL, L>(ti, sF[c], rk.im);
        sRb[c] = rk;
        if (rank == 0) c_store<L>(a.R + ((int64_t)(g + G * c) * a.ldr + k) * W, rk);
      }
      __syncthreads();
      for (int cc = warp; cc < nb; cc += MF_WARPS) {
        const int c = cb + cc;
        double *aj = a.A + (int64_t)(g + G * c) * a.lda * W;
        const cx<L> rk = sRb[c];
        const int F = sF[c];
        for (int i = i0 + lane; i < i1; i += 32) {
          cx<L> x = c_load<L>(aj + (int64_t)i * W);
          c_store<L>(aj + (int64_t)i * W, fx_axpy<L>(x, rk, sQ[i - i0], F, ok));
        }
      }
    }
  }
  if (!ok) atomicCAS(a.status, GN_OK, GN_ENONFINITE);
  cl.sync();  // no CTA leaves while a sibling may still read its shared memory
}

}  // namespace gn

#include "mgs_int.cuh"

namespace gn {

// Largest number of co-resident clusters for each precision, per device.
static std::mutex g_mf_mutex;
static int g_mf_clusters[64][5];

template <int L>
static int mf_max_clusters(int maxown, int ms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(g_mf_mutex);
  int &slot = g_mf_clusters[dev][L];
  if (slot == 0) {
    slot = -1;
    const size_t bytes = MF_SMEM_FLOOR;
    if (cudaFuncSetAttribute(k_mgs_int<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(MF_C * 64);
      cfg.blockDim = dim3(MF_THREADS);
      cfg.dynamicSmemBytes = bytes;
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = MF_C;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_mgs_int<L>, &cfg) == cudaSuccess && n > 0) slot = n;
    }
    cudaGetLastError();
  }
  (void)maxown;
  (void)ms;
  return slot;
}

template <int L>
static gn_status mf_launch(double *A, int32_t m, int64_t lda, int32_t ncols, double *R, int64_t ldr,
                           double *rinv, uint32_t *flags, int32_t *status, double *Rm, double *Zs,
                           cudaStream_t st) {
  const int ms = (m + MF_C - 1) / MF_C;
  int maxc = mf_max_clusters<L>(0, ms);
  if (maxc <= 0) return GN_ECUDA;
  const int G = maxc < ncols ? maxc : ncols;
  const int maxown = (ncols + G - 1) / G;
  MiLayout<L> lay(maxown, ms);
  size_t bytes = lay.bytes > MF_SMEM_FLOOR ? lay.bytes : MF_SMEM_FLOOR;
  if (bytes > 227 * 1024) return GN_EINVAL;
  if (bytes > MF_SMEM_FLOOR &&
      cudaFuncSetAttribute(k_mgs_int<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
          cudaSuccess)
    return GN_ECUDA;
  if (cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (size_t)ncols * MF_C, st) != cudaSuccess)
    return GN_ECUDA;
  MfArgs args{A, m, lda, ncols, R, ldr, rinv, rinv + (size_t)ncols * L, flags, status, Rm, Zs,
              G, maxown};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(MF_C * G);
  cfg.blockDim = dim3(MF_THREADS);
  cfg.dynamicSmemBytes = bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = MF_C;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_mgs_int<L>, args) != cudaSuccess) return GN_ECUDA;
  return GN_OK;
}

template <int L>
static gn_status mi_to_cascade(double *A, int32_t m, int64_t lda, int32_t ncols, const double *rinv,
                               const int32_t *status, cudaStream_t st) {
  const double *sexp = rinv + (size_t)ncols * L + ncols;
  dim3 grid((m + 255) / 256, ncols);
  k_mgs_int_to_cascade<L><<<grid, 256, 0, st>>>(A, m, lda, ncols, sexp, status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

template <int L>
static bool mf_fits(int32_t m, int32_t ncols) {
  const int maxc = mf_max_clusters<L>(0, 0);
  if (maxc <= 0) return false;
  const int G = maxc < ncols ? maxc : ncols;
  return MiLayout<L>((ncols + G - 1) / G, (m + MF_C - 1) / MF_C).bytes <= 227 * 1024;
}

bool mgs_flow_fits(int L, int32_t m, int32_t ncols) {
  switch (L) {
    case 1: return mf_fits<1>(m, ncols);
    case 2: return mf_fits<2>(m, ncols);
    case 4: return mf_fits<4>(m, ncols);
  }
  return false;
}

int mgs_flow_clusters(int L) {
  switch (L) {
    case 1: return mf_max_clusters<1>(0, 0);
    case 2: return mf_max_clusters<2>(0, 0);
    case 4: return mf_max_clusters<4>(0, 0);
  }
  return 0;
}

template <int L>
static gn_status bs_launch(const double *Rm, int64_t ldr, int32_t n, const double *Zs,
                           const double *rinv, double *dx, int32_t *status, cudaStream_t st) {
  const double *sexp = rinv + (size_t)(n + 1) * L + (n + 1);
  const size_t bytes = bs_smem_bytes<L>(n);
  // one row per thread up to 512 unknowns, two up to 1024; whole warps
  const int rows = n <= BS_MAX_THREADS ? 1 : 2;
  const int per = (n + rows - 1) / rows;
  const int threads = 32 * ((per + 31) / 32);
  if (rows == 1) {
    if (bytes > 48 * 1024 && cudaFuncSetAttribute(k_backsub_int<L, 1>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)bytes) != cudaSuccess)
      return GN_ECUDA;
    k_backsub_int<L, 1><<<1, threads, bytes, st>>>(Rm, ldr, n, Zs, sexp, dx, status);
  } else {
    if (bytes > 48 * 1024 && cudaFuncSetAttribute(k_backsub_int<L, 2>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  (int)bytes) != cudaSuccess)
      return GN_ECUDA;
    k_backsub_int<L, 2><<<1, threads, bytes, st>>>(Rm, ldr, n, Zs, sexp, dx, status);
  }
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

gn_status launch_backsub_int(int L, const double *Rm, int64_t ldr, int32_t n, const double *Zs,
                             const double *rinv, double *dx, int32_t *status, cudaStream_t st) {
  if (n < 1 || n > 2 * BS_MAX_THREADS) return GN_EINVAL;
  switch (L) {
    case 1: return bs_launch<1>(Rm, ldr, n, Zs, rinv, dx, status, st);
    case 2: return bs_launch<2>(Rm, ldr, n, Zs, rinv, dx, status, st);
    case 4: return bs_launch<4>(Rm, ldr, n, Zs, rinv, dx, status, st);
  }
  return GN_EINVAL;
}

gn_status launch_mgs_to_cascade(int L, double *A, int32_t m, int64_t lda, int32_t ncols,
                                const double *rinv, const int32_t *status, cudaStream_t st) {
  switch (L) {
    case 1: return mi_to_cascade<1>(A, m, lda, ncols, rinv, status, st);
    case 2: return mi_to_cascade<2>(A, m, lda, ncols, rinv, status, st);
    case 4: return mi_to_cascade<4>(A, m, lda, ncols, rinv, status, st);
  }
  return GN_EINVAL;
}

gn_status launch_mgs_flow(int L, double *A, int32_t m, int64_t lda, int32_t ncols, double *R,
                          int64_t ldr, double *rinv, uint32_t *flags, int32_t *status, double *Rm,
                          double *Zs, cudaStream_t st) {
  switch (L) {
    case 1: return mf_launch<1>(A, m, lda, ncols, R, ldr, rinv, flags, status, Rm, Zs, st);
    case 2: return mf_launch<2>(A, m, lda, ncols, R, ldr, rinv, flags, status, Rm, Zs, st);
    case 4: return mf_launch<4>(A, m, lda, ncols, R, ldr, rinv, flags, status, Rm, Zs, st);
  }
  return GN_EINVAL;
}

}  // namespace gn
