// mgs.cu — modified Gram-Schmidt on [A b] (Section 3 of Verschelde & Yu) as
// one persistent launch of thread-block clusters, in block floating point on
// the integer pipe (kernels in mgs_int.cuh).
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
//   * Columns are K-limb integer mantissas with one exponent each; inner
//     products and norms are exact integer sums.  Each warp's partial goes
//     to every CTA of the cluster by asynchronous distributed-shared-memory
//     stores that complete on the receiver's mbarrier, so a reduction costs
//     one message latency and no cluster-wide barrier.
//   * The K20C version launched one kernel per pivot and delayed each
//     normalisation by a step so blocks would not read a half-normalised
//     column; here the flags give that ordering inside one launch.
//
// Every wait is bounded (about one second by default, gn_set_wait_limit); a
// wait that gives up records GN_ETIMEOUT, later waits see the bad status and
// give up at once, and every CTA of the cluster leaves together, so no CTA
// is left at a cluster barrier.
#include <cooperative_groups.h>

#include <mutex>

#include "bs.cuh"
#include "bsb.cuh"
#include "ifx.cuh"
#include "internal.h"
#include "mw.cuh"

namespace cg = cooperative_groups;

namespace gn {

constexpr int MF_THREADS = 256;
constexpr int MF_WARPS = MF_THREADS / 32;
constexpr int MF_C = 8;                         // CTAs per cluster
constexpr long long MF_WAIT_CYCLES = 2000000000LL;  // default bound of one wait (~1 s)

// Bound of one device-side wait in SM clock cycles, read by every launch of
// k_mgs_int at its start (so captured graphs see a changed value on their
// next replay).  gn_set_wait_limit changes it on the current device.
__device__ long long g_mf_wait_cycles = MF_WAIT_CYCLES;
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
  int32_t maxown;     // columns per cluster, a multiple of the block width
  int32_t smem_cols;  // columns live in shared memory (else in place in A)
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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

// clusters, columns per cluster and shared-memory layout of one launch
template <int L>
struct MfPlan {
  int G = 0, maxown = 0, ms = 0;
  bool cols = false;
  size_t bytes = 0;
};

template <int L>
static bool mf_plan(int32_t m, int32_t ncols, MfPlan<L> &p) {
  if (ncols >= (1 << 18)) return false;  // the kernel's block indices stay below 2^16
  const int maxc = mf_max_clusters<L>(0, 0);
  if (maxc <= 0) return false;
  const int nblk = (ncols + MF_B - 1) / MF_B;
  p.G = maxc < nblk ? maxc : nblk;
  p.maxown = ((nblk + p.G - 1) / p.G) * MF_B;
  p.ms = (m + MF_C - 1) / MF_C;
  const size_t with = MiLayout<L>(p.maxown, p.ms, true).bytes;
  p.cols = with <= 227 * 1024;
  p.bytes = p.cols ? with : MiLayout<L>(p.maxown, p.ms, false).bytes;
  if (p.bytes < MF_SMEM_FLOOR) p.bytes = MF_SMEM_FLOOR;
  return p.bytes <= 227 * 1024;
}

template <int L>
static gn_status mf_launch(double *A, int32_t m, int64_t lda, int32_t ncols, double *R, int64_t ldr,
                           double *rinv, uint32_t *flags, int32_t *status, double *Rm, double *Zs,
                           cudaStream_t st) {
  MfPlan<L> p;
  if (mf_max_clusters<L>(0, 0) <= 0) return GN_ECUDA;
  if (!mf_plan<L>(m, ncols, p)) return GN_EINVAL;
  if (p.bytes > MF_SMEM_FLOOR &&
      cudaFuncSetAttribute(k_mgs_int<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.bytes) !=
          cudaSuccess)
    return GN_ECUDA;
  if (cudaMemsetAsync(flags, 0, sizeof(uint32_t) * (size_t)ncols * MF_C, st) != cudaSuccess)
    return GN_ECUDA;
  MfArgs args{A, m, lda, ncols, R, ldr, rinv, rinv + (size_t)ncols * L, flags, status, Rm, Zs,
              p.G, p.maxown, p.cols ? 1 : 0};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(MF_C * p.G);
  cfg.blockDim = dim3(MF_THREADS);
  cfg.dynamicSmemBytes = p.bytes;
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
  MfPlan<L> p;
  return mf_plan<L>(m, ncols, p);
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

// whether a cluster of BSC solve CTAs can be placed (queried once per precision)
template <int L>
static bool bsc_available() {
  static int ok = -1;
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  if (ok < 0) {
    const size_t bytes = bsc_smem_bytes<L>(2 * BS_MAX_THREADS);
    ok = 0;
    if (cudaFuncSetAttribute(k_backsub_cl<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
            cudaSuccess &&
        cudaFuncSetAttribute(k_backsub_cl<L>, cudaFuncAttributeNonPortableClusterSizeAllowed, 0) ==
            cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(BSC);
      cfg.blockDim = dim3(BSB_THREADS);
      cfg.dynamicSmemBytes = bytes;
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = BSC;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, k_backsub_cl<L>, &cfg) == cudaSuccess && nc > 0) ok = 1;
    }
    cudaGetLastError();
  }
  return ok == 1;
}

template <int L>
static gn_status bsb_launch(const double *Rm, int64_t ldr, int32_t n, const double *Zs,
                            const double *rinv, double *Xinv, double *dx, int32_t *status,
                            cudaStream_t st) {
  const double *sexp = rinv + (size_t)(n + 1) * L + (n + 1);
  const int nb = (n + BSB - 1) / BSB;
  if (bsc_available<L>()) {
    k_bs_inv<L><<<(unsigned)nb, BSB * BSB, 0, st>>>(Rm, ldr, n, Zs, sexp, Xinv, status);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(BSC);
    cfg.blockDim = dim3(BSB_THREADS);
    cfg.dynamicSmemBytes = bsc_smem_bytes<L>(n);
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = BSC;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_backsub_cl<L>, (const double *)Rm, ldr, n, sexp,
                           (const double *)Xinv, dx, status) != cudaSuccess)
      return GN_ECUDA;
    return GN_OK;
  }
  return bs_launch<L>(Rm, ldr, n, Zs, rinv, dx, status, st);  // no cluster: one level at a time
}

// the same for the forward substitution of the adjoint
template <int L>
static bool fsc_available() {
  static int ok = -1;
  static std::mutex mu;
  std::lock_guard<std::mutex> g(mu);
  if (ok < 0) {
    const size_t bytes = bsc_smem_bytes<L>(2 * BS_MAX_THREADS);
    ok = 0;
    if (cudaFuncSetAttribute(k_fwdsub_cl<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) ==
        cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(BSC);
      cfg.blockDim = dim3(BSB_THREADS);
      cfg.dynamicSmemBytes = bytes;
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = BSC;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      int nc = 0;
      if (cudaOccupancyMaxActiveClusters(&nc, k_fwdsub_cl<L>, &cfg) == cudaSuccess && nc > 0) ok = 1;
    }
    cudaGetLastError();
  }
  return ok == 1;
}

template <int L>
static gn_status fsc_launch(const double *Rm, int64_t ldr, int32_t n, const double *Zs,
                            const double *rinv, double *Xinv, const double *g, double *w,
                            int32_t *status, cudaStream_t st) {
  if (!fsc_available<L>()) return GN_EINVAL;
  const double *sexp = rinv + (size_t)(n + 1) * L + (n + 1);
  const int nb = (n + BSB - 1) / BSB;
  k_bs_inv<L><<<(unsigned)nb, BSB * BSB, 0, st>>>(Rm, ldr, n, Zs, sexp, Xinv, status);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(BSC);
  cfg.blockDim = dim3(BSB_THREADS);
  cfg.dynamicSmemBytes = bsc_smem_bytes<L>(n);
  cfg.stream = st;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = BSC;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_fwdsub_cl<L>, (const double *)Rm, ldr, n, sexp, (const double *)Xinv, g,
                         w, status) != cudaSuccess)
    return GN_ECUDA;
  return GN_OK;
}

bool fwdsub_int_available(int L, int32_t n) {
  if (n < 2 * BSB || n > 2 * BS_MAX_THREADS) return false;
  switch (L) {
    case 1: return fsc_available<1>();
    case 2: return fsc_available<2>();
    case 4: return fsc_available<4>();
  }
  return false;
}

gn_status launch_fwdsub_int(int L, const double *Rm, int64_t ldr, int32_t n, const double *Zs,
                            const double *rinv, double *Xinv, const double *g, double *w,
                            int32_t *status, cudaStream_t st) {
  switch (L) {
    case 1: return fsc_launch<1>(Rm, ldr, n, Zs, rinv, Xinv, g, w, status, st);
    case 2: return fsc_launch<2>(Rm, ldr, n, Zs, rinv, Xinv, g, w, status, st);
    case 4: return fsc_launch<4>(Rm, ldr, n, Zs, rinv, Xinv, g, w, status, st);
  }
  return GN_EINVAL;
}

void backsub_prepare(int L) {
  switch (L) {
    case 1: bsc_available<1>(); fsc_available<1>(); break;
    case 2: bsc_available<2>(); fsc_available<2>(); break;
    case 4: bsc_available<4>(); fsc_available<4>(); break;
  }
}

gn_status launch_backsub_int(int L, const double *Rm, int64_t ldr, int32_t n, const double *Zs,
                             const double *rinv, double *Xinv, double *dx, int32_t *status,
                             cudaStream_t st) {
  if (n < 1 || n > 2 * BS_MAX_THREADS) return GN_EINVAL;
  // blocked with inverse diagonal blocks from two blocks up (one level at a
  // time below that, or without the scratch)
  if (Xinv && n >= 2 * BSB) {
    switch (L) {
      case 1: return bsb_launch<1>(Rm, ldr, n, Zs, rinv, Xinv, dx, status, st);
      case 2: return bsb_launch<2>(Rm, ldr, n, Zs, rinv, Xinv, dx, status, st);
      case 4: return bsb_launch<4>(Rm, ldr, n, Zs, rinv, Xinv, dx, status, st);
    }
    return GN_EINVAL;
  }
  switch (L) {
    case 1: return bs_launch<1>(Rm, ldr, n, Zs, rinv, dx, status, st);
    case 2: return bs_launch<2>(Rm, ldr, n, Zs, rinv, dx, status, st);
    case 4: return bs_launch<4>(Rm, ldr, n, Zs, rinv, dx, status, st);
  }
  return GN_EINVAL;
}

template <int L>
static gn_status mi_r_out(double *R, const double *Rm, int64_t ldr, int32_t ncols, double *rinv,
                          const int32_t *status, cudaStream_t st) {
  const double *sexp = rinv + (size_t)ncols * L + ncols;
  k_mgs_r_out<L><<<ncols, 128, 0, st>>>(R, Rm, ldr, ncols, sexp, rinv, status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

gn_status launch_mgs_r_out(int L, double *R, const double *Rm, int64_t ldr, int32_t ncols,
                           double *rinv, const int32_t *status, cudaStream_t st) {
  switch (L) {
    case 1: return mi_r_out<1>(R, Rm, ldr, ncols, rinv, status, st);
    case 2: return mi_r_out<2>(R, Rm, ldr, ncols, rinv, status, st);
    case 4: return mi_r_out<4>(R, Rm, ldr, ncols, rinv, status, st);
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

extern "C" gn_status gn_set_wait_limit(int64_t cycles, int64_t *previous) {
  if (cycles < 0) return GN_EINVAL;
  long long old = 0;
  if (previous) {
    if (cudaMemcpyFromSymbol(&old, gn::g_mf_wait_cycles, sizeof(old)) != cudaSuccess) {
      cudaGetLastError();
      return GN_ECUDA;
    }
    *previous = old;
  }
  const long long v = cycles == 0 ? gn::MF_WAIT_CYCLES : (long long)cycles;
  if (cudaMemcpyToSymbol(gn::g_mf_wait_cycles, &v, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return GN_ECUDA;
  }
  return GN_OK;
}
