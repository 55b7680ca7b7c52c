// gram_tc.cu — the Gram matrix of CholeskyQR (cholqr.cu) on the tensor cores,
// exactly, with tcgen05 MMAs accumulating in tensor memory.
//
// G_ij = sum_r conj(a_ri) a_rj for the columns of [A b] (N x nc, double
// complex).  Entry a = M 2^s_j of column j has a 62-bit mantissa M at the
// column's scale (|M| < 2^62, sum_r |M_r|^2 < 2^124).  M is cut into eight
// balanced 7-bit digits,
//   M = sum_{s < 8} D_s 2^(55 - 7s) + e,   |D_0| <= 128, |D_s| <= 64, |e| <= 2^5,
// each exact in bf16.  For a digit pair (s, t) one BF16 product on the tensor
// cores forms, per 128 x 128 tile of G's upper triangle,
//   Re P_st = sum_r D_s(ar_i) D_t(ar_j) + D_s(ai_i) D_t(ai_j)
//   Im P_st = sum_r D_s(ar_i) D_t(ai_j) - D_s(ai_i) D_t(ar_j)
// in FP32 in tensor memory, and every partial sum is an integer below 2^24,
// so FP32 holds it exactly:
//   * s, t >= 1: at most 2N terms of magnitude <= 64^2, and N <= 2048;
//   * s = 0 or t = 0: by Cauchy-Schwarz, the column norm bounds
//     sum_r D_0^2 by 2^14 + 2^8 sqrt(2N) + N/2, so the sums stay below 2^20.
// k_gram_combine then forms S = sum_{s,t} P_st 2^(7 (14 - s - t)) exactly in
// 128-bit integers (|S| < 2^115) and rounds 2^(s_i + s_j + 12) S to a double
// once.  So G is the exact Gram matrix of the columns rounded to 56 bits at
// their scales (the IMAD form in cholqr.cu keeps 62), then one rounding.
//
// The tensor-core kernel takes one (tile, digit pair) per CTA.  One thread
// copies 64-row chunks of the four operand tiles (D_s of ar and ai for the
// tile's i columns, D_t of ar and ai for its j columns) into a ring of three
// shared-memory buffers with tensor-memory-access bulk copies (one 4-d box
// per tile, landing in the no-swizzle K-major layout of the MMA: 8-row x
// 16-byte core matrices); another issues the 16 MMAs of a chunk (M = N =
// 128, K = 16; the imaginary part's second product with the B-negate bit of
// the instruction descriptor) and commits them to the buffer's mbarrier,
// which lets the copier refill it.  The epilogue reads the two 128 x 128
// FP32 accumulators from tensor memory (32x32b loads: warp w owns lanes
// 32w .. 32w + 31, the tile's rows) and stores them for the combining
// kernel.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "fx.cuh"
#include "ifx.cuh"
#include "internal.h"

namespace gn {

constexpr int GT_TILE = 128;     // tile of G: M = N of the MMA
constexpr int GT_KC = 64;        // rows of A per staged chunk
constexpr int GT_DIG = 8;        // digits per mantissa
constexpr int GT_PAIRS = GT_DIG * GT_DIG;
constexpr int GT_THREADS = 128;
constexpr int GT_STAGES = 3;
constexpr int GT_OPERAND = GT_TILE * GT_KC * 2;         // bytes of one staged operand tile
constexpr int GT_STAGE = 4 * GT_OPERAND;                // Ar, Ai, Br, Bi
constexpr int GT_SMEM = GT_STAGES * GT_STAGE + 1024;    // + alignment slack (one CTA per SM)
constexpr int GT_TMEM_COLS = 2 * GT_TILE;               // Re and Im accumulators
constexpr long long GT_WAIT_CYCLES = 2000000000LL;      // bound of one wait (~1 s)
constexpr int GT_MAX_N = 2048;                          // exactness bound of the digit sums

// geometry shared by the launcher and the kernels
struct GtGeom {
  int N, nc, Np, ncp, nb, ntiles;
  __host__ __device__ GtGeom(int N_, int nc_) : N(N_), nc(nc_) {
    Np = (N + GT_KC - 1) / GT_KC * GT_KC;
    nb = (nc + GT_TILE - 1) / GT_TILE;
    ncp = nb * GT_TILE;
    ntiles = nb * (nb + 1) / 2;
  }
  __host__ __device__ size_t plane_elems() const { return (size_t)ncp * Np; }
  // digit planes: [digit][part] of [row / 8][column][row % 8] bf16 (k_gram_digits)
  __host__ __device__ size_t digit_bytes() const { return (size_t)GT_DIG * 2 * plane_elems() * 2; }
  // products: [pair][tile][part][column][row] f32 within a tile
  __host__ __device__ size_t prod_bytes() const {
    return (size_t)GT_PAIRS * ntiles * 2 * GT_TILE * GT_TILE * 4;
  }
};

size_t gram_tc_scratch_bytes(int32_t N, int32_t nc) {
  const GtGeom g(N, nc);
  return ((g.digit_bytes() + 255) & ~(size_t)255) + g.prod_bytes();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
typedef CUresult (*GtEncode)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static GtEncode gt_encode() {
  static GtEncode fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (GtEncode)p;
    else
      cudaGetLastError();
  });
  return fn;
}

bool gram_tc_available(int32_t N, int32_t nc) {
  return N >= 1 && N <= GT_MAX_N && nc >= 1 && gt_encode() != nullptr;
}

// ---- tcgen05 helpers ----

__device__ __forceinline__ uint32_t gt_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading (K-direction core) and
// stride (M/N-direction core) byte offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t gt_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D f32 (bits 4-5 = 1), A and B bf16
// (bits 7-9, 10-12 = 1), B negated (bit 14), both K-major, N >> 3 at bit 17,
// M >> 4 at bit 24
__host__ __device__ constexpr uint32_t gt_idesc(int M, int N, int bneg) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)bneg << 14) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void gt_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void gt_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(gt_smem(bar))
               : "memory");
}

__device__ __forceinline__ bool gt_wait(uint64_t *bar, uint32_t par) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(gt_smem(bar)), "r"(par)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > GT_WAIT_CYCLES) return false;
  }
}

// 32 consecutive columns of this warp's 32 lanes of tensor memory
__device__ __forceinline__ void gt_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// the tile (ib, jb), ib <= jb, of linear index t (column-by-column order)
__device__ __forceinline__ void gt_tile(int t, int &ib, int &jb) {
  int j = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((j + 1) * (j + 2) / 2 <= t) j++;
  while (j * (j + 1) / 2 > t) j--;
  jb = j;
  ib = t - j * (j + 1) / 2;
}

// Digit planes of the columns, blocked for the tensor-memory-access copies:
// element (row r, column j) of plane p = 2 digit + part at
//   p Np ncp + (r / 8) 8 ncp + 8 j + r % 8,
// so 8 consecutive rows of a column are one 16-byte piece and a row block's
// pieces run over the columns.  Thread per (r % 8, j, r / 8) in that order
// (stores contiguous); zeros outside N x nc.  M from the double at the
// column's scale 2^s_j (fx_add_double, as the IMAD Gram takes it); D_s =
// M's balanced base-128 digits from the top (round half up at each step),
// as bf16 (exact: |D| <= 128).
__global__ void k_gram_digits(const double *__restrict__ A, int32_t N, int32_t nc, int32_t Np, int32_t ncp,
                              const double *__restrict__ sexp, __nv_bfloat16 *__restrict__ D,
                              const int32_t *__restrict__ status) {
  if (*status != GN_OK) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)Np * ncp) return;
  const int r8 = (int)(t & 7), j = (int)((t >> 3) % ncp), rb = (int)((t >> 3) / ncp);
  const int r = rb * 8 + r8;
  const size_t plane = (size_t)ncp * Np;
  const size_t at = (size_t)rb * 8 * ncp + (size_t)j * 8 + r8;
#pragma unroll
  for (int part = 0; part < 2; part++) {
    int64_t x = 0;
    if (r < N && j < nc) {
      fx<1> m;
      fx_zero<1>(m);
      fx_add_double<1>(m, A[((int64_t)j * N + r) * 2 + part], -(int)sexp[j]);
      x = (int64_t)m.w[0];
    }
#pragma unroll
    for (int s = 0; s < GT_DIG; s++) {
      const int w = 55 - 7 * s;
      const int64_t d = (x + ((int64_t)1 << (w - 1))) >> w;  // arithmetic shift: floor
      x -= d << w;
      D[(size_t)(s * 2 + part) * plane + at] = __float2bfloat16_rn((float)d);
    }
  }
}

__device__ __forceinline__ void gt_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(gt_smem(bar)), "r"(bytes)
               : "memory");
}

// one operand tile of a chunk: box {64, 16 column groups, 8 row blocks, 1
// plane} of the 4-d view (8 (j % 8) + r % 8, j / 8, r / 8, plane) of the
// digit planes (innermost 128 contiguous bytes: whole sectors), which lands
// in shared memory as [row block][column][8 rows]: core matrix (column group
// g, row block k) at (16 k + g) 128 bytes, so 8-column groups are 128 B
// apart (SBO) and the two row blocks of one K = 16 step 2048 B apart (LBO)
__device__ __forceinline__ void gt_tma(void *dst, const CUtensorMap *map, int cg0, int rb0, int plane,
                                       uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(gt_smem(dst)),
      "l"((uint64_t)map), "r"(0), "r"(cg0), "r"(rb0), "r"(plane), "r"(gt_smem(bar))
      : "memory");
}

// One (tile, digit pair) per CTA: the two FP32 products of the pair for the
// tile into P (layout of GtGeom::prod_bytes).  Thread 0 copies the chunks
// into a ring of GT_STAGES buffers (each the four operand tiles, full[]
// completes when they have landed); thread 32 issues each chunk's 16 MMAs
// and commits them to empty[] (the buffer may be refilled) and, after the
// last, to fin.  Every wait is bounded; one that gives up records
// GN_ETIMEOUT and the tile's products are not written.
__global__ void __launch_bounds__(GT_THREADS, 1)
    k_gram_tc(const __grid_constant__ CUtensorMap dmap, GtGeom g, float *__restrict__ P,
              int32_t *__restrict__ status) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  __shared__ __align__(8) uint64_t full[GT_STAGES], empty[GT_STAGES], fin;
  __shared__ uint32_t tbase;
  __shared__ int sFail;
  if (*(volatile int32_t *)status != GN_OK) return;  // uniform: before any allocation
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x % g.ntiles, pair = blockIdx.x / g.ntiles;
  const int ds = pair / GT_DIG, dt = pair % GT_DIG;
  int ib, jb;
  gt_tile(tile, ib, jb);
  unsigned char *base = (unsigned char *)(((uintptr_t)gsm + 1023) & ~(uintptr_t)1023);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gt_smem(&tbase)),
                 "n"(GT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int q = 0; q < GT_STAGES; q++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(gt_smem(&full[q])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(gt_smem(&empty[q])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(gt_smem(&fin)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sFail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tRe = tbase, tIm = tbase + GT_TILE;
  const int nch = g.Np / GT_KC;

  if (tid == 0) {
    // producer
    for (int c = 0; c < nch; c++) {
      const int st = c % GT_STAGES, u = c / GT_STAGES;
      if (c >= GT_STAGES && !gt_wait(&empty[st], (uint32_t)((u - 1) & 1))) {
        sFail = 1;
        break;
      }
      unsigned char *sb = base + (size_t)st * GT_STAGE;
      gt_expect(&full[st], GT_STAGE);
      const int rb0 = c * (GT_KC / 8);
      gt_tma(sb, &dmap, ib * (GT_TILE / 8), rb0, ds * 2 + 0, &full[st]);
      gt_tma(sb + GT_OPERAND, &dmap, ib * (GT_TILE / 8), rb0, ds * 2 + 1, &full[st]);
      gt_tma(sb + 2 * GT_OPERAND, &dmap, jb * (GT_TILE / 8), rb0, dt * 2 + 0, &full[st]);
      gt_tma(sb + 3 * GT_OPERAND, &dmap, jb * (GT_TILE / 8), rb0, dt * 2 + 1, &full[st]);
    }
  } else if (tid == 32) {
    // MMA issuer
    const uint32_t idp = gt_idesc(GT_TILE, GT_TILE, 0), idn = gt_idesc(GT_TILE, GT_TILE, 1);
    for (int c = 0; c < nch; c++) {
      const int st = c % GT_STAGES, u = c / GT_STAGES;
      if (!gt_wait(&full[st], (uint32_t)(u & 1))) {
        sFail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sb = gt_smem(base + (size_t)st * GT_STAGE);
      const uint32_t aR = sb, aI = sb + GT_OPERAND, bR = sb + 2 * GT_OPERAND, bI = sb + 3 * GT_OPERAND;
#pragma unroll
      for (int ks = 0; ks < GT_KC / 16; ks++) {
        const uint32_t ko = ks * 4096;  // 16 rows: two row blocks
        const int acc = (c > 0 || ks > 0) ? 1 : 0;
        gt_mma(tRe, gt_desc(aR + ko, 2048, 128), gt_desc(bR + ko, 2048, 128), idp, acc);
        gt_mma(tRe, gt_desc(aI + ko, 2048, 128), gt_desc(bI + ko, 2048, 128), idp, 1);
        gt_mma(tIm, gt_desc(aR + ko, 2048, 128), gt_desc(bI + ko, 2048, 128), idp, acc);
        gt_mma(tIm, gt_desc(aI + ko, 2048, 128), gt_desc(bR + ko, 2048, 128), idn, 1);
      }
      gt_commit(&empty[st]);
    }
    gt_commit(&fin);  // every MMA issued above
  }
  // the last MMAs (fin completes once, phase 0)
  int ok = gt_wait(&fin, 0);
  __syncthreads();
  ok = ok && !sFail;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int row = 32 * warp + lane;
    float *out = P + ((size_t)pair * g.ntiles + tile) * 2 * GT_TILE * GT_TILE;
#pragma unroll 1
    for (int part = 0; part < 2; part++) {
#pragma unroll 1
      for (int cb = 0; cb < GT_TILE; cb += 32) {
        uint32_t v[32];
        gt_ld32((part ? tIm : tRe) + ((uint32_t)(32 * warp) << 16) + (uint32_t)cb, v);
        float *o = out + (size_t)part * GT_TILE * GT_TILE;
#pragma unroll
        for (int q = 0; q < 32; q++) o[(size_t)(cb + q) * GT_TILE + row] = __uint_as_float(v[q]);
      }
    }
  } else if (tid == 0) {
    atomicCAS(status, GN_OK, GN_ETIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tRe), "n"(GT_TMEM_COLS)
                 : "memory");
}

// G's upper triangle from the products: thread per entry of a tile (rows
// fastest, as P is laid out); per part, the pairs of equal weight added in
// 64-bit integers (Q_d, d = s + t, at most 8 terms below 2^24), then
// S = sum_d Q_d 2^(7 (14 - d)) in 128 bits, rounded once to the double
// 2^(s_i + s_j + 12) S.
__global__ void k_gram_combine(const float *__restrict__ P, GtGeom g, const double *__restrict__ sexp,
                               double *__restrict__ G, const int32_t *__restrict__ status) {
  if (*status != GN_OK) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)g.ntiles * GT_TILE * GT_TILE) return;
  const int tile = (int)(t / (GT_TILE * GT_TILE)), e = (int)(t % (GT_TILE * GT_TILE));
  int ib, jb;
  gt_tile(tile, ib, jb);
  const int i = ib * GT_TILE + (e % GT_TILE), j = jb * GT_TILE + (e / GT_TILE);
  if (i > j || j >= g.nc) return;
  const int F = -((int)sexp[i] + (int)sexp[j] + 12);
  const size_t tstride = (size_t)g.ntiles * 2 * GT_TILE * GT_TILE;  // one pair
#pragma unroll 1
  for (int part = 0; part < 2; part++) {
    const float *p = P + ((size_t)tile * 2 + part) * GT_TILE * GT_TILE + e;
    int64_t Q[2 * GT_DIG - 1];
#pragma unroll
    for (int d = 0; d < 2 * GT_DIG - 1; d++) Q[d] = 0;
#pragma unroll
    for (int ds = 0; ds < GT_DIG; ds++)
#pragma unroll
      for (int dt = 0; dt < GT_DIG; dt++) Q[ds + dt] += (int64_t)(int32_t)p[(size_t)(ds * GT_DIG + dt) * tstride];
    u128_t S = 0;
#pragma unroll
    for (int d = 0; d < 2 * GT_DIG - 1; d++) S += (u128_t)(__int128)Q[d] << (7 * (2 * GT_DIG - 2 - d));
    fx<2> v;
    v.w[0] = (uint64_t)S;
    v.w[1] = (uint64_t)(S >> 64);
    double out[1];
    fx_to_cascade<2, 1>(v, F, out);
    G[((int64_t)j * g.nc + i) * 2 + part] = out[0];
  }
}

gn_status launch_gram_tc(int32_t N, int32_t nc, const double *A, const double *sexp, double *G, void *scratch,
                         int32_t *status, cudaStream_t st) {
  if (!gram_tc_available(N, nc) || !scratch) return GN_EINVAL;
  const GtGeom g(N, nc);
  __nv_bfloat16 *D = (__nv_bfloat16 *)scratch;
  float *P = (float *)((char *)scratch + ((g.digit_bytes() + 255) & ~(size_t)255));
  const int64_t nd = (int64_t)g.Np * g.ncp;
  // the 4-d view (8 (j % 8) + r % 8, j / 8, r / 8, plane) of the digit
  // planes; box {64, 16, 8, 1}
  CUtensorMap map;
  const cuuint64_t dims[4] = {64, (cuuint64_t)(g.ncp / 8), (cuuint64_t)(g.Np / 8), 2 * GT_DIG};
  const cuuint64_t strides[3] = {128, (cuuint64_t)16 * g.ncp, (cuuint64_t)2 * g.plane_elems()};
  const cuuint32_t box[4] = {64, GT_TILE / 8, GT_KC / 8, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  if (gt_encode()(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, D, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return GN_ECUDA;
  k_gram_digits<<<(unsigned)((nd + 255) / 256), 256, 0, st>>>(A, N, nc, g.Np, g.ncp, sexp, D, status);
  if (cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM) != cudaSuccess)
    return GN_ECUDA;
  k_gram_tc<<<(unsigned)(g.ntiles * GT_PAIRS), GT_THREADS, GT_SMEM, st>>>(map, g, P, status);
  const int64_t ne = (int64_t)g.ntiles * GT_TILE * GT_TILE;
  k_gram_combine<<<(unsigned)((ne + 255) / 256), 256, 0, st>>>(P, g, sexp, G, status);
  return cudaPeekAtLastError() == cudaSuccess ? GN_OK : GN_ECUDA;
}

}  // namespace gn
