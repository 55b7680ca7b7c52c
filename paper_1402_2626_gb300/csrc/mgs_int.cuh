// mgs_int.cuh — the MGS kernel of mgs.cu in block floating point on the
// integer pipe (included by mgs.cu).
//
// Column j is held in place as K-limb integer mantissas with one exponent
// s_j (a_ij = A_ij 2^s_j, |A_ij| < 2^(64K-2), s_j from the column's original
// norm), pivots as Q_ij = q_ij 2^(64K-2).  With K = L limbs the integer form
// has the byte size of the L-limb floating-point form, so the conversion is
// in place.  Per pivot k and column j:
//   D_kj = sum_i conj(Q_ik) A_ij / 2^(64K-2)      (r_kj = D_kj 2^s_j)
//   A_ij <- A_ij - D_kj Q_ik / 2^(64K-2)
//   T_j  = sum_i |A_ij|^2 (exact)                 (r_jj = sqrt(T_j) 2^s_j)
//   Q_ij = A_ij Z_j / 2^(b_j - 1),  Z_j ~ 2^(b_j + 64K - 3) / sqrt(T_j)
// The reciprocal square root comes from an FP32 seed and integer Newton
// steps (ifx.cuh).
#pragma once

namespace gn {

// ---- messages between the CTAs of a cluster ----

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// the cluster address of this CTA's shared location a in the CTA of rank r
__device__ __forceinline__ uint32_t cl_mapa(uint32_t a, uint32_t r) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(r));
  return d;
}

__device__ __forceinline__ void mb_init(uint64_t *bar, uint32_t count = 1) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// this CTA's arrival for the current phase, announcing `bytes` to come
__device__ __forceinline__ void mb_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// 8 bytes to the cluster address ra; completes 8 bytes of the transaction
// count of the mbarrier at cluster address rb
__device__ __forceinline__ void st_async8(uint32_t ra, uint64_t v, uint32_t rb) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.u64 [%0], %1, [%2];" ::"r"(ra),
               "l"(v), "r"(rb)
               : "memory");
}

// Wait until the phase of parity par of a local mbarrier has completed
// (acquire at cluster scope: the stores that completed it are visible).
// Gives up after g_mf_wait_cycles (recording GN_ETIMEOUT), or soon after the
// status word turns bad; returns whether the phase completed.
__device__ __forceinline__ bool mb_wait(uint64_t *bar, uint32_t par, int32_t *status) {
  const uint32_t a = smem_u32(bar);
  const long long lim = g_mf_wait_cycles;  // consumed only once the wait spins
  const long long t0 = clock64();
  for (uint32_t it = 0;; it++) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(par)
        : "memory");
    if (done) return true;
    if ((it & 15) == 15 && *(volatile int32_t *)status != GN_OK) return false;
    if (clock64() - t0 > lim) {
      atomicCAS(status, GN_OK, GN_ETIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ bool status_ok(const int32_t *status) {
  return *(volatile const int32_t *)status == GN_OK;
}

// arrival (release at CTA scope) on a local mbarrier
__device__ __forceinline__ void mb_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Warps 0 .. MF_CW-1 run the factorisation; warp MF_CW releases the pivot
// flags (a release at GPU scope waits for the pivot's global stores, about
// a microsecond, which must not sit on the pivot chain).  The compute warps
// synchronise among themselves on named barrier 1.
constexpr int MF_CW = MF_WARPS - 1;
constexpr int MF_CT = MF_CW * 32;
constexpr int MF_NPUB = 4;  // pivots handed to the publisher warp in flight
// The pivot chain (the column after the current pivot: its dot with q_k,
// axpy, norm, reciprocal square root and normalisation) runs on MF_QW warps
// of each CTA; in each, lane 4 d + p takes rows 8 w + d (+32 i) and one of
// the four real products of each complex one, so a lane's dependent chain
// is a quarter of a whole complex product.  Integer sums are exact, so the
// results are those of one warp doing all four products.
constexpr int MF_QW = 4;
constexpr int MF_QS = MF_QW * 8;  // reduction slots of one chain sum: a warp per CTA, 8 CTAs
static_assert(MF_QS <= 32, "a chain sum is read by one lane per slot");

__device__ __forceinline__ void cw_sync() { asm volatile("bar.sync 1, %0;" ::"n"(MF_CT) : "memory"); }

__device__ __forceinline__ int cw_sync_or(int pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, %2, q;\n\tselp.s32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"(pred), "n"(MF_CT)
      : "memory");
  return r;
}

// One reduction site: two slot buffers and two mbarriers, used alternately.
// Use u writes buffer u & 1 and completes phase (u >> 1) & 1 of its
// mbarrier.  A CTA sends its part of use u + 2 only after use u + 1 is
// complete, which needs every CTA's part of use u + 1, which every warp
// sends after reading its buffer for use u: so a buffer is never written
// while it is read, and an mbarrier never holds two uses at once.  Every CTA
// of a cluster makes the same uses in the same order.
struct MbSite {
  uint64_t *bar;   // [2]
  uint64_t *slot;  // [2][slots][words]
  uint32_t use;
};

// Exact cluster-wide sum of NV values of N limbs held by the lanes of ONE
// warp in every CTA (use u of the site): the warp adds its lanes and sends
// the total to every CTA (slot [rank]); the same warp of every CTA adds the 8
// slots.  On return all lanes of the calling warps hold the totals.  A wait
// that gives up leaves them undefined and the status word bad.
template <int N, int NV>
__device__ void warp_cluster_sum(fx<N> (&v)[NV], const MbSite &site, uint32_t u, int rank,
                                 int32_t *status) {
  constexpr int SW = N * NV;  // words per slot
  const int lane = threadIdx.x & 31;
  const uint32_t b = u & 1, par = (u >> 1) & 1;
  uint64_t *bar = site.bar + b;
  uint64_t *sl = site.slot + (size_t)b * MF_C * SW;
  if (lane == 0) mb_expect(bar, MF_C * SW * 8);
#pragma unroll
  for (int q = 0; q < NV; q++) v[q] = warp_sum_fx<N>(v[q]);
  if (lane < MF_C) {
    const uint32_t ra = cl_mapa(smem_u32(sl + (size_t)rank * SW), lane);
    const uint32_t rb = cl_mapa(smem_u32(bar), lane);
#pragma unroll
    for (int q = 0; q < NV; q++)
#pragma unroll
      for (int w = 0; w < N; w++) st_async8(ra + 8 * (q * N + w), v[q].w[w], rb);
  }
  mb_wait(bar, par, status);
#pragma unroll
  for (int q = 0; q < NV; q++) {
#pragma unroll
    for (int w = 0; w < N; w++) v[q].w[w] = (lane < MF_C) ? sl[(size_t)lane * SW + q * N + w] : 0;
    v[q] = warp_sum_fx<N>(v[q]);
  }
}

// Exact cluster-wide sum as warp_cluster_sum, sent by MF_QW warps of every
// CTA (the chain warps; cs is the caller's index among them): each sends its
// warp total to slot [cs][rank] of every CTA, and every calling warp adds
// all MF_QS slots, one lane per slot.  Chain warp 0 announces the bytes.
template <int N>
__device__ void chain_cluster_sum(fx<N> &v, const MbSite &site, uint32_t u, int rank, int cs,
                                  int32_t *status) {
  const int lane = threadIdx.x & 31;
  const uint32_t b = u & 1, par = (u >> 1) & 1;
  uint64_t *bar = site.bar + b;
  uint64_t *sl = site.slot + (size_t)b * MF_QS * N;
  if (cs == 0 && lane == 0) mb_expect(bar, MF_QS * N * 8);
  v = warp_sum_fx<N>(v);
  if (lane < MF_C) {
    const uint32_t ra = cl_mapa(smem_u32(sl + (size_t)(cs * MF_C + rank) * N), lane);
    const uint32_t rb = cl_mapa(smem_u32(bar), lane);
#pragma unroll
    for (int w = 0; w < N; w++) st_async8(ra + 8 * w, v.w[w], rb);
  }
  mb_wait(bar, par, status);
#pragma unroll
  for (int w = 0; w < N; w++) v.w[w] = (lane < MF_QS) ? sl[(size_t)lane * N + w] : 0;
  v = warp_sum_fx<N>(v);
}

// Columns per ownership block: column j belongs to cluster (j / MF_B) mod G,
// so the pivot chain stays inside one cluster for MF_B - 1 of every MF_B
// columns.
constexpr int MF_B = 4;
static_assert(MF_B + MF_QW - 1 <= MF_CW, "chain warps: the pivot's own warp and warps MF_B ..");

// shared-memory layout of k_mgs_int, identical on host and device
template <int L>
struct MiLayout {
  static constexpr int K = L;
  static constexpr int SW_PIV = 2 * K + 1;  // norm: 2K+1 limbs
  static constexpr int SW_DOT = 2 * (K + 1);  // a dot: re, im of K+1 limbs
  static constexpr int NBAR = 8 + 2 * MF_NPUB;  // 4 sites x 2, publication full/empty
  size_t oS, oTb, oN0, oN0p, oR, oQ, oBar, oPub, oPiv, oCh, oLa, oBulk, oA, bytes;
  __host__ __device__ MiLayout(int maxown, int ms, bool cols) {
    size_t o = 0;
    auto take = [&](size_t b) {
      size_t at = o;
      o += (b + 15) & ~(size_t)15;
      return at;
    };
    const size_t msr = ms > 0 ? ms : 1;
    oS = take(sizeof(int) * maxown);                   // column exponents s_j
    oTb = take(sizeof(int) * maxown);                  // rank-test bit lengths
    oN0 = take(sizeof(double) * maxown);               // original norms
    oN0p = take(sizeof(double) * maxown);              // this CTA's part of them
    oR = take(sizeof(fx<K>) * 2 * maxown);             // r_kj mantissas of a bulk step
    oQ = take(sizeof(fx<K>) * 2 * msr);                // a pivot slice read from global memory
    oBar = take(sizeof(uint64_t) * NBAR);              // mbarriers
    oPub = take(sizeof(int) * 2 * MF_NPUB);            // handed-off pivots: column, accepted
    oPiv = take(sizeof(uint64_t) * 2 * MF_QS * SW_PIV);
    oCh = take(sizeof(uint64_t) * 2 * MF_QS * SW_DOT);
    oLa = take(sizeof(uint64_t) * 2 * (MF_B - 1) * MF_C * SW_DOT);
    oBulk = take(sizeof(uint64_t) * 2 * (size_t)maxown * MF_C * SW_DOT);
    oA = take(cols ? sizeof(fx<K>) * 2 * msr * maxown : 0);  // the CTA's rows of its columns
    bytes = (o + 255) & ~(size_t)255;
  }
};

template <int L>
__global__ void __launch_bounds__(MF_THREADS, 1) k_mgs_int(MfArgs a) {
  constexpr int K = L;          // limbs per real mantissa
  constexpr int W = 2 * L;      // doubles (= 64-bit words) per complex entry
  constexpr int S = 64 * K - 2; // scale of the pivot columns Q
  constexpr int B = MF_B;
  constexpr int SWD = MiLayout<L>::SW_DOT;
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int g = blockIdx.x / MF_C;
  const int G = a.G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = a.m, ncols = a.ncols;
  const int ms = (m + MF_C - 1) / MF_C;
  const int i0 = min(m, rank * ms), i1 = min(m, i0 + ms), nr = i1 - i0;

  // block-cyclic ownership: global column j <-> (owner, local index).  The
  // quotient by G (<= 152) of a block index (< 2^16) is an exact high
  // multiply by ceil(2^32 / G): these run on the pivot chain every column.
  static_assert(MF_B == 4, "the block index is j >> 2");
  const uint32_t Gm = (uint32_t)((0x100000000ull + (uint64_t)G - 1) / (uint64_t)G);
  auto owner = [&](int j) {
    const uint32_t bj = (uint32_t)j >> 2;
    return (int)(bj - __umulhi(bj, Gm) * (uint32_t)G);
  };
  auto lcol = [&](int j) { return (int)(__umulhi((uint32_t)j >> 2, Gm) * B + (j & 3)); };
  auto gcol = [&](int c) { return ((c / B) * G + g) * B + (c % B); };
  const int nblk = (ncols + B - 1) / B;
  int no = (g < nblk) ? ((nblk - g + G - 1) / G) * B : 0;  // my columns
  if (no > 0 && owner(ncols - 1) == g) no -= nblk * B - ncols;
  const int jlast = no > 0 ? gcol(no - 1) : -1;

  const MiLayout<L> lay(a.maxown, ms, a.smem_cols != 0);
  int *sS = (int *)(smem + lay.oS);
  int *sTb = (int *)(smem + lay.oTb);
  double *sN0 = (double *)(smem + lay.oN0);
  double *sN0p = (double *)(smem + lay.oN0p);
  fx<K> *sR = (fx<K> *)(smem + lay.oR);  // [maxown][2], by local column
  fx<K> *sQ = (fx<K> *)(smem + lay.oQ);  // [ms][2]
  fx<K> *sA = (fx<K> *)(smem + lay.oA);  // [maxown][ms][2]
  uint64_t *bars = (uint64_t *)(smem + lay.oBar);
  uint64_t *pubFull = bars + 8, *pubEmpty = bars + 8 + MF_NPUB;
  int *sPubJ = (int *)(smem + lay.oPub), *sPubAcc = sPubJ + MF_NPUB;
  MbSite piv{bars + 0, (uint64_t *)(smem + lay.oPiv), 0};
  MbSite la{bars + 2, (uint64_t *)(smem + lay.oLa), 0};  // the block's later columns
  MbSite bulk{bars + 4, (uint64_t *)(smem + lay.oBulk), 0};
  MbSite ch{bars + 6, (uint64_t *)(smem + lay.oCh), 0};  // the chain column's dot
  bool ok = true;

  if (tid == 0) {
    for (int q = 0; q < MiLayout<L>::NBAR; q++)
      mb_init(bars + q, (q >= 8 && q < 8 + MF_NPUB) ? MF_QW : 1);  // pubFull: every chain warp
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // this CTA's rows of global column j (the publication slot of pivots)
  auto pubp = [&](int j) { return (fx<K> *)(a.A + ((int64_t)j * a.lda + i0) * W); };
  // this CTA's rows of local column c: entry (i0 + r, part) at [2 r + part]
  auto colp = [&](int c) {
    return a.smem_cols ? sA + (size_t)c * ms * 2 : pubp(gcol(c));
  };

  // original column norms (double), exponents, conversion to mantissas
  for (int c = warp; c < no; c += MF_WARPS) {
    const double *cp = a.A + ((int64_t)gcol(c) * a.lda + i0) * W;
    double s = 0.0;
    for (int r = lane; r < nr; r += 32) {
      double re = cp[(int64_t)r * W], im = cp[(int64_t)r * W + L];
      s = fma(re, re, fma(im, im, s));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sN0p[c] = s;
  }
  cl.sync();  // also publishes the mbarrier initialisation to the cluster
  for (int c = tid; c < no; c += MF_THREADS) {
    double t = 0.0;
    for (int r = 0; r < MF_C; r++) t += cl.map_shared_rank(sN0p, r)[c];
    const double n0 = sqrt(t);
    // a NaN or an infinity anywhere in the column: every CTA of the owner
    // cluster sees it here, before any pivot could record a rank deficiency
    if (!isfinite(n0)) atomicCAS(a.status, GN_OK, GN_ENONFINITE);
    sN0[c] = n0;
    const int sj = fx_exponent_of(n0 * 1.0000001 + 1e-300) - S;
    sS[c] = sj;
    // rank test: ||a_j||^2 = T 2^(2 s_j) must exceed (||a_j^0|| 2^(8-50L))^2, taken
    // on bit lengths: reject when bitlen(T) <= 2 (floor(log2 ||a_j^0||) + 8 - 50L - s_j) + 1
    sTb[c] = 2 * (fx_exponent_of(n0) - 1 + 8 - 50 * L - sj) + 1;
    if (rank == 0) {
      a.nrm0[gcol(c)] = n0;
      a.nrm0[ncols + gcol(c)] = (double)sj;
    }
  }
  __syncthreads();
  for (int c = warp; c < no; c += MF_WARPS) {
    const double *cp = a.A + ((int64_t)gcol(c) * a.lda + i0) * W;
    fx<K> *d = colp(c);
    const int F = -sS[c];
    for (int r = lane; r < nr; r += 32) {
      const double *e = cp + (int64_t)r * W;
      fx<K> re, im;
      fx_zero<K>(re);
      fx_zero<K>(im);
#pragma unroll
      for (int l = 0; l < L; l++) {
        ok &= fx_add_double<K>(re, e[l], F);
        ok &= fx_add_double<K>(im, e[L + l], F);
      }
      d[2 * r] = re;
      d[2 * r + 1] = im;
    }
  }
  __syncthreads();

  // the chain warps: lane 4 d + p of chain warp cs takes rows 8 cs + d
  // (+32 i) and the part p of each (rows of a warp-uniform block rb)
  const int qp = lane & 3, qd = lane >> 2;

  // Pivot j by the MF_QW chain warps of each CTA (cs = index among them):
  // exact norm (squares of the real parts in lanes p = 0, of the imaginary
  // parts in p = 1), cluster sum, 1/||a_j|| by integer Newton in lane 0 of
  // every chain warp (the same value in each), rank test, normalisation of
  // the warp's rows (into the CTA's column and the publication slot), hand-
  // off to the publisher; the R diagonal and 1/r_jj afterwards.
  auto pivot = [&](int j, uint32_t u, int cs) {
    const int c = lcol(j);
    fx<K> *aj = colp(c);
    const int sj = sS[c];
    fx<2 * K + 1> t;
    fx_zero<2 * K + 1>(t);
    for (int r = 8 * cs + qd; r < nr; r += 32)
      if (qp < 2) t = ix_add<2 * K + 1>(t, ix_square<K>(aj[2 * r + qp]));
    chain_cluster_sum<2 * K + 1>(t, piv, u, rank, cs, a.status);
    ux<K> Y;
    fx<K> Z;
    ux<K> tt;
    int bl = 0, b = 0, accept = 0;
    fx_zero<K>(Z);
    if (lane == 0) {
      const fx<2 * K + 1> T = t;
      bl = ix_bitlen<2 * K + 1>(T);
      b = (bl + 1) >> 1;  // sqrt(T) < 2^b
      accept = (bl > 0) && (j == ncols - 1 || bl > sTb[c]);
      if (!accept && j < ncols - 1 && cs == 0) atomicCAS(a.status, GN_OK, GN_ESINGULAR);
      // t = T / 2^(2b) in [1/4, 1) as K limbs of fraction
      {
        fx<2 * K + 1> sh;
        const int d = 2 * b - 64 * K;
        if (d >= 0) {
          sh = ix_sar<2 * K + 1>(T, d);
        } else {
          // left shift by -d (T < 2^(2b) < 2^(64K))
          sh = ix_shl<2 * K + 1>(T, -d);
        }
#pragma unroll
        for (int w = 0; w < K; w++) tt.w[w] = sh.w[w];
      }
      if (accept) {
        Y = ix_rsqrt_frac<K>(tt);  // 2^S / sqrt(t)
#pragma unroll
        for (int w = 0; w < K; w++) Z.w[w] = (Y.w[w] >> 1) | ((w + 1 < K) ? (Y.w[w + 1] << 63) : 0);
      }
    }
    if (j < ncols - 1) {
#pragma unroll
      for (int w = 0; w < K; w++) Z.w[w] = __shfl_sync(0xffffffffu, Z.w[w], 0);
      b = __shfl_sync(0xffffffffu, b, 0);
      accept = __shfl_sync(0xffffffffu, accept, 0);
      if (accept) {
        const int sh = b - 1;
        uint64_t nz;
        const ux<K> uz = ix_abs<K>(Z, nz);
        fx<K> *pj = pubp(j);
        for (int r = 8 * cs + qd; r < nr; r += 32) {
          if (qp >= 2) continue;
          const int e = 2 * r + qp;
          uint64_t na;
          ux<K> ua = ix_abs<K>(aj[e], na);
          ux<2 * K> p = ix_umul<K>(ua, uz);
          fx<2 * K> pf;
#pragma unroll
          for (int w = 0; w < 2 * K; w++) pf.w[w] = p.w[w];
          pf = ix_sar<2 * K>(pf, sh);
          fx<K> q;
#pragma unroll
          for (int w = 0; w < K; w++) q.w[w] = pf.w[w];
          ix_cneg<K>(q, na);
          aj[e] = q;
          if (a.smem_cols) pj[e] = q;
        }
      }
      // hand q_j to the publisher warp once every chain warp's rows are in:
      // each warp's stores are ordered before its lane 0's arrival (release),
      // the publisher's flag release after the last of them
      __syncwarp();
      if (lane == 0) {
        const int pp = lcol(j), ps = pp % MF_NPUB;
        if (mb_wait(pubEmpty + ps, ((pp / MF_NPUB) & 1) ^ 1, a.status)) {
          if (cs == 0) {
            sPubJ[ps] = j;
            sPubAcc[ps] = accept;
          }
          mb_arrive(pubFull + ps);
        }
      }
    }
    // for back substitution and the R output: 1/r_jj = Z 2^e, and t and b in
    // the diagonal slot of R (k_mgs_r_out forms r_jj and 1/r_jj from them)
    if (lane == 0 && rank == 0 && cs == 0) {
      if (accept && j < ncols - 1) {
        double *zs = a.Zs + (size_t)j * (K + 1);
#pragma unroll
        for (int w = 0; w < K; w++) ((uint64_t *)zs)[w] = Z.w[w];
        zs[K] = (double)(-(b + 64 * K - 3) - sj);  // 1/r_jj = Z 2^this
      }
      uint64_t *rd = (uint64_t *)(a.R + ((int64_t)j * a.ldr + j) * W);
#pragma unroll
      for (int w = 0; w < K; w++) rd[w] = (bl > 0) ? tt.w[w] : 0;
      rd[K] = (uint64_t)b;
    }
  };

  // the chain warps' share of conj(q)^T a over this CTA's rows for one
  // column: lanes p = 0, 1 add qr ar, qi ai (real part), p = 2, 3 add
  // qr ai, -qi ar (imaginary part); each part summed over the warp
  auto chain_dot = [&](const fx<K> *q, const fx<K> *aj, int cs, fx<K + 1> &dr, fx<K + 1> &di) {
    const int qo = (qp == 1 || qp == 3) ? 1 : 0, ao = (qp == 1 || qp == 2) ? 1 : 0;
    fx<K + 1> acc;
    fx_zero<K + 1>(acc);
    for (int r = 8 * cs + qd; r < nr; r += 32)
      acc = ix_add_cneg<K + 1>(acc, ix_mul_shift<K>(q[2 * r + qo], aj[2 * r + ao]), qp == 3);
    fx<K + 1> pr, pi;
#pragma unroll
    for (int w = 0; w <= K; w++) {
      pr.w[w] = qp < 2 ? acc.w[w] : 0;
      pi.w[w] = qp < 2 ? 0 : acc.w[w];
    }
    dr = warp_sum_fx<K + 1>(pr);
    di = warp_sum_fx<K + 1>(pi);
  };

  // the chain warps' rows of a_j <- a_j - r q: lane p forms rr qr, ri qi,
  // rr qi, ri qr (p = 0 .. 3); lane 0 of a quad takes the real part
  // rr qr - ri qi, lane 2 the imaginary part rr qi + ri qr, from its
  // partner's product (the same integer results as one lane forming all four)
  auto chain_axpy = [&](const fx<K> *q, fx<K> *aj, int cs, const fx<K> &rr, const fx<K> &ri) {
    const int qo = (qp == 1 || qp == 2) ? 1 : 0;
    const fx<K> rv = (qp & 1) ? ri : rr;
    for (int rb = 8 * cs; rb < nr; rb += 32) {  // warp-uniform: every lane shuffles
      const int r = rb + qd;
      fx<K + 1> pr;
      if (r < nr) {
        pr = ix_mul_shift<K>(rv, q[2 * r + qo]);
      } else {
        fx_zero<K + 1>(pr);
      }
      fx<K + 1> po;
#pragma unroll
      for (int w = 0; w <= K; w++) po.w[w] = __shfl_xor_sync(0xffffffffu, pr.w[w], 1);
      if (r < nr && (qp & 1) == 0) {
        const fx<K + 1> d = ix_add_cneg<K + 1>(pr, po, qp == 0);
        fx<K> *x = aj + 2 * r + (qp >> 1);
        *x = ix_narrow<K>(ix_sub<K + 1>(ix_widen<K, K + 1>(*x), d));
      }
    }
  };

  // r_kj = q_k^H a_j as K-limb mantissas at the scale of column j
  // (|r_kj| <= ||a_j^0||, so they fit; k_mgs_r_out converts them)
  auto out_r = [&](int k, int c, const fx<K + 1> &tr, const fx<K + 1> &ti) {
    fx<K> *rm = (fx<K> *)(a.Rm + ((int64_t)gcol(c) * a.ldr + k) * W);
    rm[0] = ix_narrow<K>(tr);
    rm[1] = ix_narrow<K>(ti);
  };

  // conj(q)^T a over this CTA's rows for one column, by one warp; lanes over rows
  auto warp_dot = [&](const fx<K> *q, const fx<K> *aj, fx<K + 1> &dr, fx<K + 1> &di) {
    fx_zero<K + 1>(dr);
    fx_zero<K + 1>(di);
    for (int r = lane; r < nr; r += 32) {
      const fx<K> qr = q[2 * r], qi = q[2 * r + 1];
      const fx<K> ar = aj[2 * r], ai = aj[2 * r + 1];
      dr = ix_add<K + 1>(dr, ix_mul_shift<K>(qr, ar));
      dr = ix_add<K + 1>(dr, ix_mul_shift<K>(qi, ai));
      di = ix_add<K + 1>(di, ix_mul_shift<K>(qr, ai));
      di = ix_sub<K + 1>(di, ix_mul_shift<K>(qi, ar));
    }
    dr = warp_sum_fx<K + 1>(dr);
    di = warp_sum_fx<K + 1>(di);
  };

  // a_j <- a_j - r q over this CTA's rows, by one warp
  auto warp_axpy = [&](const fx<K> *q, fx<K> *aj, const fx<K> &rr, const fx<K> &ri) {
    for (int r = lane; r < nr; r += 32) {
      const fx<K> qr = q[2 * r], qi = q[2 * r + 1];
      fx<K + 1> xr = ix_widen<K, K + 1>(aj[2 * r]);
      fx<K + 1> xi = ix_widen<K, K + 1>(aj[2 * r + 1]);
      xr = ix_sub<K + 1>(xr, ix_mul_shift<K>(rr, qr));
      xr = ix_add<K + 1>(xr, ix_mul_shift<K>(ri, qi));
      xi = ix_sub<K + 1>(xi, ix_mul_shift<K>(rr, qi));
      xi = ix_sub<K + 1>(xi, ix_mul_shift<K>(ri, qr));
      aj[2 * r] = ix_narrow<K>(xr);
      aj[2 * r + 1] = ix_narrow<K>(xi);
    }
  };

  // send this warp's dot to slot [base + rank] of every CTA of the cluster
  auto send_dot = [&](uint64_t *sl, uint64_t *bar, int base, const fx<K + 1> &dr, const fx<K + 1> &di) {
    if (lane < MF_C) {
      const uint32_t ra = cl_mapa(smem_u32(sl + ((size_t)base + rank) * SWD), lane);
      const uint32_t rb = cl_mapa(smem_u32(bar), lane);
#pragma unroll
      for (int w = 0; w < K + 1; w++) {
        st_async8(ra + 8 * w, dr.w[w], rb);
        st_async8(ra + 8 * (K + 1 + w), di.w[w], rb);
      }
    }
  };

  // conj(q)^T a for two columns at once, by one warp (two independent
  // product chains per lane; q's rows are loaded once)
  auto warp_dot2 = [&](const fx<K> *q, const fx<K> *a1, const fx<K> *a2, fx<K + 1> (&d)[4]) {
#pragma unroll
    for (int v = 0; v < 4; v++) fx_zero<K + 1>(d[v]);
    for (int r = lane; r < nr; r += 32) {
      const fx<K> qr = q[2 * r], qi = q[2 * r + 1];
      const fx<K> ar = a1[2 * r], ai = a1[2 * r + 1], br = a2[2 * r], bi = a2[2 * r + 1];
      d[0] = ix_add<K + 1>(d[0], ix_mul_shift<K>(qr, ar));
      d[2] = ix_add<K + 1>(d[2], ix_mul_shift<K>(qr, br));
      d[0] = ix_add<K + 1>(d[0], ix_mul_shift<K>(qi, ai));
      d[2] = ix_add<K + 1>(d[2], ix_mul_shift<K>(qi, bi));
      d[1] = ix_add<K + 1>(d[1], ix_mul_shift<K>(qr, ai));
      d[3] = ix_add<K + 1>(d[3], ix_mul_shift<K>(qr, bi));
      d[1] = ix_sub<K + 1>(d[1], ix_mul_shift<K>(qi, ar));
      d[3] = ix_sub<K + 1>(d[3], ix_mul_shift<K>(qi, br));
    }
#pragma unroll
    for (int v = 0; v < 4; v++) d[v] = warp_sum_fx<K + 1>(d[v]);
  };

  // a1 <- a1 - r1 q and a2 <- a2 - r2 q over this CTA's rows, by one warp
  auto warp_axpy2 = [&](const fx<K> *q, fx<K> *a1, fx<K> *a2, const fx<K> &r1r, const fx<K> &r1i,
                        const fx<K> &r2r, const fx<K> &r2i) {
    for (int r = lane; r < nr; r += 32) {
      const fx<K> qr = q[2 * r], qi = q[2 * r + 1];
      fx<K + 1> xr = ix_widen<K, K + 1>(a1[2 * r]), xi = ix_widen<K, K + 1>(a1[2 * r + 1]);
      fx<K + 1> yr = ix_widen<K, K + 1>(a2[2 * r]), yi = ix_widen<K, K + 1>(a2[2 * r + 1]);
      xr = ix_sub<K + 1>(xr, ix_mul_shift<K>(r1r, qr));
      yr = ix_sub<K + 1>(yr, ix_mul_shift<K>(r2r, qr));
      xr = ix_add<K + 1>(xr, ix_mul_shift<K>(r1i, qi));
      yr = ix_add<K + 1>(yr, ix_mul_shift<K>(r2i, qi));
      xi = ix_sub<K + 1>(xi, ix_mul_shift<K>(r1r, qi));
      yi = ix_sub<K + 1>(yi, ix_mul_shift<K>(r2r, qi));
      xi = ix_sub<K + 1>(xi, ix_mul_shift<K>(r1i, qr));
      yi = ix_sub<K + 1>(yi, ix_mul_shift<K>(r2i, qr));
      a1[2 * r] = ix_narrow<K>(xr);
      a1[2 * r + 1] = ix_narrow<K>(xi);
      a2[2 * r] = ix_narrow<K>(yr);
      a2[2 * r + 1] = ix_narrow<K>(yi);
    }
  };

  // Apply q_k (this CTA's rows at q) to the local columns [c0, c1): dots by
  // warps (column c0 + cc on warp cc mod MF_CW, two of a warp's columns at a
  // time), totals through the bulk site, axpys.  Every thread calls it.
  auto bulk_apply = [&](int k, const fx<K> *q, int c0, int c1) {
    const int nb = c1 - c0;
    if (nb <= 0) return;
    const uint32_t u = bulk.use++;
    const uint32_t bb = u & 1, par = (u >> 1) & 1;
    uint64_t *bar = bulk.bar + bb;
    uint64_t *sl = bulk.slot + (size_t)bb * a.maxown * MF_C * SWD;
    if (tid == 0) mb_expect(bar, (uint32_t)(nb * MF_C * SWD * 8));
    for (int cc = warp; cc < nb; cc += 2 * MF_CW) {
      const int c2 = cc + MF_CW;
      if (c2 < nb) {
        fx<K + 1> d[4];
        warp_dot2(q, colp(c0 + cc), colp(c0 + c2), d);
        send_dot(sl, bar, cc * MF_C, d[0], d[1]);
        send_dot(sl, bar, c2 * MF_C, d[2], d[3]);
      } else {
        fx<K + 1> dr, di;
        warp_dot(q, colp(c0 + cc), dr, di);
        send_dot(sl, bar, cc * MF_C, dr, di);
      }
    }
    mb_wait(bar, par, a.status);
    for (int cc = tid; cc < nb; cc += MF_CT) {
      fx<K + 1> tr, ti;
      fx_zero<K + 1>(tr);
      fx_zero<K + 1>(ti);
      for (int r = 0; r < MF_C; r++) {
        const uint64_t *p = sl + ((size_t)cc * MF_C + r) * SWD;
        fx<K + 1> x, y;
#pragma unroll
        for (int w = 0; w < K + 1; w++) {
          x.w[w] = p[w];
          y.w[w] = p[K + 1 + w];
        }
        tr = ix_add<K + 1>(tr, x);
        ti = ix_add<K + 1>(ti, y);
      }
      sR[2 * cc] = ix_narrow<K>(tr);
      sR[2 * cc + 1] = ix_narrow<K>(ti);
      if (rank == 0) out_r(k, c0 + cc, tr, ti);
    }
    cw_sync();
    for (int cc = warp; cc < nb; cc += 2 * MF_CW) {
      const int c2 = cc + MF_CW;
      if (c2 < nb) {
        warp_axpy2(q, colp(c0 + cc), colp(c0 + c2), sR[2 * cc], sR[2 * cc + 1], sR[2 * c2],
                   sR[2 * c2 + 1]);
      } else {
        warp_axpy(q, colp(c0 + cc), sR[2 * cc], sR[2 * cc + 1]);
      }
    }
    cw_sync();  // sR, sQ and the slots are free for the next use
  };

  // this CTA's rows of q_k from the publication slot into sQ (after its flag)
  auto load_q = [&](int k) {
    const fx<K> *qk = pubp(k);
    for (int e = tid; e < 2 * nr; e += MF_CT) {
      fx<K> v;
#pragma unroll
      for (int w = 0; w < K; w++) v.w[w] = __ldcg(&qk[e].w[w]);
      sQ[e] = v;
    }
    cw_sync();
  };

  if (warp == MF_CW) {
    // the publisher: releases the flags of this CTA's pivots in order
    const int npub = no - ((no > 0 && owner(ncols - 1) == g) ? 1 : 0);
    for (int pp = 0; pp < npub; pp++) {
      const int ps = pp % MF_NPUB;
      const bool got = mb_wait(pubFull + ps, (pp / MF_NPUB) & 1, a.status);
      if (!__all_sync(0xffffffffu, got)) break;  // the warp leaves together
      if (lane == 0) {
        st_release(a.flags + (size_t)sPubJ[ps] * MF_C + rank, sPubAcc[ps] ? 1u : 2u);
        mb_arrive(pubEmpty + ps);
      }
      __syncwarp();
    }
  } else {
  // the chain warps for pivot column j: warp (j mod B) and warps B ..
  // B + MF_QW - 2, which the block's other columns leave free
  auto chain_slot = [&](int j) {
    return warp == (j & (B - 1)) ? 0 : ((warp >= B && warp < B + MF_QW - 1) ? warp - B + 1 : -1);
  };

  if (owner(0) == g && no > 0) {
    const uint32_t u = piv.use++;
    const int cs = chain_slot(0);
    if (cs >= 0) pivot(0, u, cs);
    cw_sync();
  }

  // Progress of the bulk updates, in MGS order per column: the columns of
  // the cluster's next block (local [cf, cf + B), which lead the chain when
  // it reaches the cluster) have received the q's before kn, the cluster's
  // later columns those before kp.  While the chain is within one step of the
  // next block, only that block is updated (the later columns wait until the
  // chain has left the cluster); otherwise every later column is.
  int kp = 0, kn = 0;
  int cfb = -1;  // the block kn refers to (its first local column)
  int cf = 0;    // first local column with global index > k
  for (int k = 0; k < ncols - 1; k++) {
    if (k >= jlast) break;
    while (cf < no && gcol(cf) <= k) cf++;
    if (cf != cfb) {  // a new next block: its columns are where the later ones are
      kn = kp;
      cfb = cf;
    }
    const bool lak = owner(k + 1) == g;  // this cluster takes the pivot chain
    const int cb = min(cf + B, no);
    // the chain reaches this cluster's next block right after q_{k+1}
    const bool near = !lak && k + 2 < ncols && owner(k + 2) == g;
    // this iteration's bulk updates: column ranges [rc0, rc1) with the first
    // q each still lacks (rk); one range when the next block and the later
    // columns are level, else the block first
    int rk[2], rc0[2], rc1[2], nrg = 0;
    if (!lak) {
      if (kn == kp && !near) {
        rk[0] = kp, rc0[0] = cf, rc1[0] = no, nrg = 1;
      } else {
        rk[0] = kn, rc0[0] = cf, rc1[0] = cb, nrg = 1;
        if (!near) rk[1] = kp, rc0[1] = cb, rc1[1] = no, nrg = 2;
      }
    } else if ((k + 1) % B == 0) {  // a new block of this cluster takes the chain at k+1
      rk[0] = kn, rc0[0] = cf, rc1[0] = cb, nrg = 1;
    }
    // the q's before q_k that the ranges lack
    for (int r = 0; r < nrg; r++) {
      for (int kk = rk[r]; kk < k; kk++) {
        const fx<K> *qq = sQ;
        if (owner(kk) == g) {
          qq = colp(lcol(kk));
        } else {
          load_q(kk);
        }
        bulk_apply(kk, qq, rc0[r], rc1[r]);
      }
    }
    // q_k: this cluster's own, or published by its owner
    const fx<K> *q;
    if (owner(k) == g) {
      q = colp(lcol(k));
    } else {
      int okv = 1;
      if (tid == 0) {
        const uint32_t *f = a.flags + (size_t)k * MF_C + rank;
        const long long lim = g_mf_wait_cycles;
        const long long t0 = clock64();
        uint32_t v;
        for (;;) {
          v = ld_acquire(f);
          if (v) break;
          if (!status_ok(a.status)) {
            v = 2;
            break;
          }
          if (clock64() - t0 > lim) {
            atomicCAS(a.status, GN_OK, GN_ETIMEOUT);
            v = 2;
            break;
          }
          __nanosleep(32);
        }
        okv = (v == 1);
      }
      // the one place a CTA leaves the loop early: uniform over the CTA; the
      // other CTAs of the cluster then find the status bad in their next wait
      if (cw_sync_or(tid == 0 && !okv)) break;
      load_q(k);
      q = sQ;
    }
    if (lak) {
      // the block's columns after k: column k+1 (the chain) on the MF_QW chain
      // warps, each later one on warp (j mod B): dot, cluster sum, axpy; then
      // the pivot k+1 on the chain warps, which publishes q_{k+1}.  Slots of
      // column j1 + t start at t MF_QS; the chain's fill MF_QS of them, the
      // others MF_C.
      const int j1 = k + 1, jend = min(((k + 1) / B + 1) * B, ncols), nla = jend - j1;
      // the chain column's dot on its own site (the chain does not wait for
      // the later columns' dots); the later columns on the window site
      const uint32_t uc = ch.use++;
      const uint32_t uw = nla > 1 ? la.use++ : 0u;
      const int cs = chain_slot(j1);
      const int t = cs >= 0 ? 0 : warp - (j1 % B);  // this warp's column j1 + t
      if (cs >= 0 || (warp < B && t > 0 && t < nla)) {
        const uint32_t u = cs >= 0 ? uc : uw;
        const uint32_t bb = u & 1, par = (u >> 1) & 1;
        uint64_t *bar = (cs >= 0 ? ch.bar : la.bar) + bb;
        uint64_t *sl = cs >= 0 ? ch.slot + (size_t)bb * MF_QS * SWD
                               : la.slot + (size_t)bb * (B - 1) * MF_C * SWD;
        const int base = cs >= 0 ? 0 : (t - 1) * MF_C;  // first slot of this column
        if (lane == 0 && cs == 0) mb_expect(bar, (uint32_t)(MF_QS * SWD * 8));
        if (lane == 0 && t == 1) mb_expect(bar, (uint32_t)((nla - 1) * MF_C * SWD * 8));
        const int c = lcol(j1 + t);
        fx<K> *aj = colp(c);
        fx<K + 1> dr, di;
        if (cs >= 0) {
          chain_dot(q, aj, cs, dr, di);
        } else {
          warp_dot(q, aj, dr, di);
        }
        send_dot(sl, bar, base + (cs > 0 ? cs : 0) * MF_C, dr, di);
        mb_wait(bar, par, a.status);
        const int ns = cs >= 0 ? MF_QS : MF_C;
        fx<K + 1> v[2];
#pragma unroll
        for (int w = 0; w < K + 1; w++) {
          v[0].w[w] = (lane < ns) ? sl[((size_t)base + lane) * SWD + w] : 0;
          v[1].w[w] = (lane < ns) ? sl[((size_t)base + lane) * SWD + K + 1 + w] : 0;
        }
        v[0] = warp_sum_fx<K + 1>(v[0]);
        v[1] = warp_sum_fx<K + 1>(v[1]);
        if (cs >= 0) {
          chain_axpy(q, aj, cs, ix_narrow<K>(v[0]), ix_narrow<K>(v[1]));
          const uint32_t pu = piv.use;
          pivot(j1, pu, cs);
          if (cs == 0 && lane == 0 && rank == 0) out_r(k, c, v[0], v[1]);
        } else {
          warp_axpy(q, aj, ix_narrow<K>(v[0]), ix_narrow<K>(v[1]));
          if (lane == 0 && rank == 0) out_r(k, c, v[0], v[1]);
        }
      }
      piv.use++;
      cw_sync();  // q_{k+1} and the block's columns are visible to every compute warp
    } else {
      // q_k to the ranges, which now lack nothing before it
      for (int r = 0; r < nrg; r++) bulk_apply(k, q, rc0[r], rc1[r]);
      kn = k + 1;
      if (!near) kp = k + 1;
    }
    if (lak && (k + 1) % B == 0) kn = k;
  }
  }  // compute warps
  __syncthreads();
  if (!ok) atomicCAS(a.status, GN_OK, GN_ENONFINITE);
  // the residual column b - Q y back to global memory
  if (a.smem_cols && no > 0 && owner(ncols - 1) == g && status_ok(a.status)) {
    const fx<K> *src = colp(lcol(ncols - 1));
    fx<K> *dst = pubp(ncols - 1);
    for (int e = tid; e < 2 * nr; e += MF_THREADS) dst[e] = src[e];
  }
  // after a failure, asynchronous stores sent before it may still be in
  // flight towards CTAs that no longer wait for them: let them land
  if (!status_ok(a.status)) __nanosleep(20000);
  cl.sync();
}

// R from the mantissas k_mgs_int left: r_kj = Rm_kj 2^(s_j) above the
// diagonal; on it, t and b of the pivot give r_jj = sqrt(t) 2^(b + s_j) and
// 1/r_jj = (1/sqrt(t)) 2^-(b + s_j); zeros below.  One CTA per column.
template <int L>
__global__ void k_mgs_r_out(double *R, const double *Rm, int64_t ldr, int32_t ncols,
                            const double *sexp, double *rinv, const int32_t *status) {
  constexpr int K = L, W = 2 * L, S = 64 * K - 2;
  if (*status != GN_OK) return;
  const int j = blockIdx.x;
  const int sj = (int)sexp[j];
  double *col = R + (int64_t)j * ldr * W;
  for (int k = threadIdx.x; k < ncols; k += blockDim.x) {
    cx<L> z = c_zero<L>();
    if (k < j) {
      const fx<K> *rm = (const fx<K> *)(Rm + ((int64_t)j * ldr + k) * W);
      fx_to_cascade<K, L>(rm[0], -sj, z.re);
      fx_to_cascade<K, L>(rm[1], -sj, z.im);
    } else if (k == j) {
      const uint64_t *rd = (const uint64_t *)(col + (int64_t)j * W);
      ux<K> tt;
#pragma unroll
      for (int w = 0; w < K; w++) tt.w[w] = rd[w];
      const int b = (int)rd[K];
      if (b > 0) {
        const ux<K> Y = ix_rsqrt_frac<K>(tt);  // 2^S / sqrt(t)
        // sqrt(t) = t y: (tt Y) / 2^(64K), scale 2^S
        const ux<2 * K> ty = ix_umul<K>(tt, Y);
        fx<K> M, Yf;
#pragma unroll
        for (int w = 0; w < K; w++) {
          M.w[w] = ty.w[K + w];
          Yf.w[w] = Y.w[w];
        }
        fx_to_cascade<K, L>(M, S - b - sj, z.re);  // r_jj = sqrt(t) 2^(b + s_j)
        if (j < ncols - 1) {
          double ri[L];
          fx_to_cascade<K, L>(Yf, S + b + sj, ri);  // 1/r_jj = y 2^-(b + s_j)
#pragma unroll
          for (int l = 0; l < L; l++) rinv[(int64_t)j * L + l] = ri[l];
        }
      }
    }
    c_store<L>(col + (int64_t)k * W, z);
  }
}

// Q (and the residual b - Q y) back from mantissas to L-limb cascades:
// column j < n at scale 2^-(64K-2), the last column at 2^s_n.
template <int L>
__global__ void k_mgs_int_to_cascade(double *A, int32_t m, int64_t lda, int32_t ncols,
                                     const double *sexp, const int32_t *status) {
  constexpr int K = L, W = 2 * L;
  if (*status != GN_OK) return;
  const int j = blockIdx.y;
  const int F = (j < ncols - 1) ? (64 * K - 2) : -(int)sexp[j];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    double *e = A + ((int64_t)j * lda + i) * W;
    fx<K> *v = (fx<K> *)e;
    fx<K> re = v[0], im = v[1];
    double cr[L], ci[L];
    fx_to_cascade<K, L>(re, F, cr);
    fx_to_cascade<K, L>(im, F, ci);
#pragma unroll
    for (int l = 0; l < L; l++) {
      e[l] = cr[l];
      e[L + l] = ci[l];
    }
  }
}

// Back substitution R[0:n,0:n] x = y on the mantissas the MGS kernel left
// (Section 3, eq. 5 read as x_l = (y_l - sum_{j>l} r_lj x_j) / r_ll), column
// oriented: at level l every row i < l subtracts r_il x_l.  y is held in
// fixed point at the scale of the last column (K+2 limbs: two limbs of
// headroom for intermediate growth), each x_l in block floating point (K-limb
// mantissa per part, one exponent).  One CTA; row i belongs to thread
// i mod T.  The owner of row l-1 forms x_{l-1} as soon as its own update with
// x_l is done, so a level costs one barrier; the r_il of a later level are
// loaded while the current one runs, and the reciprocals 1/r_ll and the
// column exponents sit in shared memory.  All integer.
constexpr int BS_MAX_THREADS = 512;

// shared memory of k_backsub_int for n unknowns
template <int L>
__host__ __device__ constexpr size_t bs_smem_bytes(int n) {
  return sizeof(fx<L>) * 3 * (size_t)(n > 0 ? n : 1) + sizeof(int) * (3 * (size_t)n + 2);
}

template <int L, int ROWS>
__global__ void __launch_bounds__(BS_MAX_THREADS) k_backsub_int(
    const double *__restrict__ Rm, int64_t ldr, int32_t n, const double *__restrict__ Zs,
    const double *__restrict__ sexp, double *__restrict__ dx, int32_t *__restrict__ status) {
  constexpr int K = L, W = 2 * L, KY = K + 2;
  constexpr int D = (ROWS == 1 && L < 4) ? 3 : 2;  // levels of r_il held in registers
  extern __shared__ __align__(16) unsigned char bsm[];
  fx<K> *sX = (fx<K> *)bsm;          // [n][2] mantissas of x
  fx<K> *sZ = sX + 2 * n;            // [n] mantissas of 1/r_ll
  int *sT = (int *)(sZ + n);         // [n] exponents of x
  int *sZe = sT + n;                 // [n] exponents of 1/r_ll
  int *sS = sZe + n;                 // [n+1] column exponents
  int *sFail = sS + n + 1;
  if (*status != GN_OK) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n; i += nt) {
    const uint64_t *z = (const uint64_t *)(Zs + (size_t)i * (K + 1));
#pragma unroll
    for (int w = 0; w < K; w++) sZ[i].w[w] = z[w];
    sZe[i] = (int)Zs[(size_t)i * (K + 1) + K];
    sS[i] = (int)sexp[i];
  }
  const int sig = (int)sexp[n];  // scale of y (the last column)
  if (tid == 0) {
    sS[n] = sig;
    *sFail = 0;
  }
  fx<KY> Y[ROWS][2];
#pragma unroll
  for (int p = 0; p < ROWS; p++) {
    const int i = tid + nt * p;
    if (i < n) {
      const fx<K> *e = (const fx<K> *)(Rm + ((int64_t)n * ldr + i) * W);
      Y[p][0] = ix_widen<K, KY>(e[0]);
      Y[p][1] = ix_widen<K, KY>(e[1]);
    } else {
      fx_zero<KY>(Y[p][0]);
      fx_zero<KY>(Y[p][1]);
    }
  }
  // r_il of the next D levels in registers.  The level loop is unrolled by
  // D so that every slot keeps its own registers: a load is consumed D - 1
  // levels after it is issued and no register copy waits on it.
  auto load_level = [&](int lv, fx<K>(&rr)[ROWS], fx<K>(&ri)[ROWS]) {
#pragma unroll
    for (int p = 0; p < ROWS; p++) {
      const int i = tid + nt * p;
      if (i < lv) {
        const fx<K> *e = (const fx<K> *)(Rm + ((int64_t)lv * ldr + i) * W);
#pragma unroll
        for (int w = 0; w < K; w++) {
          rr[p].w[w] = __ldg((const unsigned long long *)&e[0].w[w]);
          ri[p].w[w] = __ldg((const unsigned long long *)&e[1].w[w]);
        }
      }
    }
  };
  // level l: load level l - (D-1) into (nr, ni), subtract r_il x_l from the
  // rows i < l with (rr, ri), the owner of row l-1 solves x_{l-1}; one barrier
  auto level = [&](int l, const fx<K>(&rr)[ROWS], const fx<K>(&ri)[ROWS], fx<K>(&nr)[ROWS],
                   fx<K>(&ni)[ROWS]) {
    load_level(l - (D - 1), nr, ni);
    const fx<K> xr = sX[2 * l], xi = sX[2 * l + 1];
    const int d = sS[l] + sT[l] - sig;
    // highest row first: for the owner of row l-1 that is row l-1 itself
#pragma unroll
    for (int p = ROWS - 1; p >= 0; p--) {
      const int i = tid + nt * p;
      if (i < l) {
        bs_update<K, KY>(Y[p][0], Y[p][1], rr[p], ri[p], xr, xi, d, sFail);
        if (i == l - 1) {
          fx<K> Xr, Xi;
          int t;
          bs_solve<K, KY>(Y[p][0], Y[p][1], sZ[l - 1], sZe[l - 1], sig, Xr, Xi, t);
          sX[2 * (l - 1)] = Xr;
          sX[2 * (l - 1) + 1] = Xi;
          sT[l - 1] = t;
        }
      }
    }
    __syncthreads();
  };
  fx<K> Ar[ROWS], Ai[ROWS], Br[ROWS], Bi[ROWS], Cr[ROWS], Ci[ROWS];
  load_level(n - 1, Ar, Ai);
  if (D == 3) load_level(n - 2, Br, Bi);
  __syncthreads();
  // x_{n-1}
  if (tid == (n - 1) % nt) {
    const int po = (n - 1) / nt;
#pragma unroll
    for (int p = 0; p < ROWS; p++)
      if (p == po) {
        fx<K> xr, xi;
        int t;
        bs_solve<K, KY>(Y[p][0], Y[p][1], sZ[n - 1], sZe[n - 1], sig, xr, xi, t);
        sX[2 * (n - 1)] = xr;
        sX[2 * (n - 1) + 1] = xi;
        sT[n - 1] = t;
      }
  }
  __syncthreads();
  if constexpr (D == 3) {
    for (int l = n - 1; l >= 1; l -= 3) {
      level(l, Ar, Ai, Cr, Ci);
      if (l - 1 >= 1) level(l - 1, Br, Bi, Ar, Ai);
      if (l - 2 >= 1) level(l - 2, Cr, Ci, Br, Bi);
    }
  } else {
    for (int l = n - 1; l >= 1; l -= 2) {
      level(l, Ar, Ai, Br, Bi);
      if (l - 1 >= 1) level(l - 1, Br, Bi, Ar, Ai);
    }
  }
  if (*sFail && tid == 0) atomicCAS(status, GN_OK, GN_ENONFINITE);
  // outputs: x_l = X 2^t as L-limb cascades
  for (int l = tid; l < n; l += nt) {
    double cr[L], ci[L];
    fx_to_cascade<K, L>(sX[2 * l], -sT[l], cr);
    fx_to_cascade<K, L>(sX[2 * l + 1], -sT[l], ci);
#pragma unroll
    for (int q = 0; q < L; q++) {
      dx[(int64_t)l * W + q] = cr[q];
      dx[(int64_t)l * W + L + q] = ci[q];
    }
  }
}

}  // namespace gn
