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
// The reciprocal square root comes from the double rsqrt and one or two
// Newton steps (FP64 TwoProd pieces, exact integer sums).
#pragma once

namespace gn {

// 1 / sqrt(s) for a positive cascade s of L limbs, to about 2^(-52 L)
// relative: rsqrt seed, then Newton y <- y - y (s y^2 - 1) / 2 with the
// residual s y^2 - 1 summed exactly (its leading bits cancel).
template <int L>
__device__ void rsqrt_cascade(const double (&s)[L], double (&y)[L]) {
#pragma unroll
  for (int l = 0; l < L; l++) y[l] = 0.0;
  double y0 = rsqrt(s[0]);
  if constexpr (L == 1) {
    // one Newton step in double: y (3 - s y^2) / 2
    double h = __fma_rn(-s[0] * y0, y0, 1.0);
    y[0] = __fma_rn(0.5 * y0, h, y0);
    return;
  } else {
    // step 1 (to ~104 bits): y1 = y0 - y0 d / 2, d = s y0^2 - 1
    double p, e;
    two_prod(y0, y0, p, e);
    double d = __fma_rn(s[0], p, -1.0);
    d = __fma_rn(s[0], e, d);
    d = __fma_rn(s[1], p, d);
    double c = -0.5 * y0 * d;
    double y1h, y1l;
    fast_two_sum(y0, c, y1h, y1l);
    if constexpr (L == 2) {
      y[0] = y1h;
      y[1] = y1l;
      return;
    } else {
      // step 2 (to ~208 bits) with exact sums: d = s y1^2 - 1, y2 = y1 - y1 d / 2
      constexpr int NL = 5;
      const int F = 290;  // values near 1
      double q[4] = {y1h, y1l, 0.0, 0.0};
      fx<NL> acc;
      fx_zero<NL>(acc);
      fx_add_prod<4, NL>(acc, q, q, false, F);
      double y2c[4];
      fx_to_cascade<NL, 4>(acc, F, y2c);  // y1^2
      fx_zero<NL>(acc);
      fx_add_prod<4, NL>(acc, s, y2c, false, F);
      fx_add_bits<NL>(acc, fx_dbits(1.0) ^ 0x8000000000000000ull, F);
      double dd[4];
      fx_to_cascade<NL, 4>(acc, F, dd);  // d ~ 2^-104, about 186 bits above the resolution
      // y2 = y1 - y1 d / 2
      fx_zero<NL>(acc);
      fx_add_limbs<4, NL>(acc, q, false, F);
      double hd[4] = {0.5 * dd[0], 0.5 * dd[1], 0.5 * dd[2], 0.5 * dd[3]};
      fx_add_prod<4, NL>(acc, q, hd, true, F);
      fx_to_cascade<NL, 4>(acc, F, y);
    }
  }
}

// Exact sum over the cluster of NV values of N limbs held by every thread:
// each warp adds its lanes, writes the warp total to its slot in this CTA's
// sSlot ([MF_WARPS][NV]), one cluster barrier, then warp 0 of every CTA adds
// the MF_C x MF_WARPS slots.  On return all lanes of warp 0 hold the totals
// in v.  *sOk = okv is this CTA's flag; the return value (valid in warp 0) is
// the AND over the cluster.  Every thread of every CTA must call it, and two
// calls with the same sSlot must be separated by another cluster barrier.
template <int N, int NV>
__device__ int cluster_sum(fx<N> (&v)[NV], fx<N> *sSlot, int *sOk, int okv, cg::cluster_group &cl) {
  static_assert(MF_C * MF_WARPS == 64, "two slots per lane");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int q = 0; q < NV; q++) {
      fx<N> u;
#pragma unroll
      for (int w = 0; w < N; w++) u.w[w] = __shfl_xor_sync(0xffffffffu, v[q].w[w], o);
      v[q] = ix_add<N>(v[q], u);
    }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < NV; q++) sSlot[warp * NV + q] = v[q];
  if (threadIdx.x == 0) *sOk = okv;
  cl.sync();
  int all = 1;
  if (warp == 0) {
    const int e0 = lane, e1 = lane + 32;
    const fx<N> *p0 = cl.map_shared_rank(sSlot, e0 / MF_WARPS) + (e0 % MF_WARPS) * NV;
    const fx<N> *p1 = cl.map_shared_rank(sSlot, e1 / MF_WARPS) + (e1 % MF_WARPS) * NV;
#pragma unroll
    for (int q = 0; q < NV; q++) v[q] = ix_add<N>(p0[q], p1[q]);
    int okr = (lane < MF_C) ? *cl.map_shared_rank(sOk, lane) : 1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int q = 0; q < NV; q++) {
        fx<N> u;
#pragma unroll
        for (int w = 0; w < N; w++) u.w[w] = __shfl_xor_sync(0xffffffffu, v[q].w[w], o);
        v[q] = ix_add<N>(v[q], u);
      }
    all = __all_sync(0xffffffffu, okr);
  }
  return all;
}

template <int L>
__global__ void __launch_bounds__(MF_THREADS, 1) k_mgs_int(MfArgs a) {
  constexpr int K = L;          // limbs per real mantissa
  constexpr int W = 2 * L;      // doubles (= 64-bit words) per complex entry
  constexpr int S = 64 * K - 2; // scale of the pivot columns Q
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int g = blockIdx.x / MF_C;
  const int G = a.G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m = a.m, ncols = a.ncols;
  const int ms = (m + MF_C - 1) / MF_C;
  const int i0 = min(m, rank * ms), i1 = min(m, i0 + ms);
  const int no = (g < ncols) ? (ncols - g + G - 1) / G : 0;

  // shared memory
  int *sS = (int *)smem;                                   // [maxown] column exponents s_j
  int *sTb = sS + a.maxown;                                // [maxown] rank-test bit lengths
  double *sN0 = (double *)(smem + 16 * ((a.maxown * 8 + 15) / 16));  // [maxown]
  double *sN0p = sN0 + a.maxown;                           // [maxown]
  fx<K + 1> *sDot = (fx<K + 1> *)(sN0p + a.maxown);        // [2][maxown][2] bulk partials
  fx<K + 1> *sCritD = sDot + 4 * a.maxown;                 // [MF_WARPS][2] lookahead dot slots
  fx<2 * K + 1> *sCritT = (fx<2 * K + 1> *)(sCritD + 2 * MF_WARPS);  // [MF_WARPS] norm slots
  fx<K> *sR = (fx<K> *)(sCritT + MF_WARPS);                // [maxown + 1][2] r_kj mantissas
  fx<K> *sQ = sR + 2 * (a.maxown + 1);                     // [ms][2] pivot slice
  // wait results read by the cluster: [0,1] bulk step by parity, [2,3]
  // lookahead step by parity, [4] the pivot's (always 1)
  int *sOk = (int *)(sQ + 2 * (ms > 0 ? ms : 1));
  int *sAll = sOk + 5;                                     // cluster decision broadcast
  int *sB = sOk + 6;                                       // b_j of the pivot
  int *sAccept = sOk + 7;
  fx<K> *sZ = (fx<K> *)(sOk + 8);                          // normalisation multiplier
  fx<K> *sTT = sZ + 1;                                     // t of the pivot (fraction)
  bool ok = true;

  auto col = [&](int j) { return (fx<K> *)(a.A + (int64_t)j * a.lda * W); };

  // original column norms (double), exponents, conversion to mantissas in place
  for (int c = warp; c < no; c += MF_WARPS) {
    const double *cp = a.A + (int64_t)(g + G * c) * a.lda * W;
    double s = 0.0;
    for (int i = i0 + lane; i < i1; i += 32) {
      double re = cp[(int64_t)i * W], im = cp[(int64_t)i * W + L];
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
    const double n0 = sqrt(t);
    sN0[c] = n0;
    const int sj = fx_exponent_of(n0 * 1.0000001 + 1e-300) - S;
    sS[c] = sj;
    // rank test: ||a_j||^2 = T 2^(2 s_j) must exceed (||a_j^0|| 2^(8-50L))^2, taken
    // on bit lengths: reject when bitlen(T) <= 2 (floor(log2 ||a_j^0||) + 8 - 50L - s_j) + 1
    sTb[c] = 2 * (fx_exponent_of(n0) - 1 + 8 - 50 * L - sj) + 1;
    if (rank == 0) {
      a.nrm0[g + G * c] = n0;
      a.nrm0[ncols + g + G * c] = (double)sj;
    }
  }
  __syncthreads();
  for (int c = warp; c < no; c += MF_WARPS) {
    double *cp = a.A + (int64_t)(g + G * c) * a.lda * W;
    const int F = -sS[c];
    for (int i = i0 + lane; i < i1; i += 32) {
      double *e = cp + (int64_t)i * W;
      fx<K> re, im;
      fx_zero<K>(re);
      fx_zero<K>(im);
#pragma unroll
      for (int l = 0; l < L; l++) {
        ok &= fx_add_double<K>(re, e[l], F);
        ok &= fx_add_double<K>(im, e[L + l], F);
      }
      fx<K> *d = (fx<K> *)e;
      d[0] = re;
      d[1] = im;
    }
  }
  __syncthreads();

  // pivot j: norm (exact), 1/||a_j|| by integer Newton, rank test,
  // normalisation, publication; the R diagonal and 1/r_jj limbs afterwards
  auto pivot = [&](int j, int c) {
    fx<K> *aj = col(j);
    const int sj = sS[c];
    fx<2 * K + 1> t[1];
    fx_zero<2 * K + 1>(t[0]);
    for (int e = tid; e < 2 * (i1 - i0); e += MF_THREADS) {
      const int i = i0 + (e >> 1), part = e & 1;
      t[0] = ix_add<2 * K + 1>(t[0], ix_square<K>(aj[2 * i + part]));
    }
    cluster_sum<2 * K + 1, 1>(t, sCritT, sOk + 4, 1, cl);
    ux<K> Y;
    int bl = 0, b = 0;
    if (tid == 0) {
      const fx<2 * K + 1> T = t[0];
      bl = ix_bitlen<2 * K + 1>(T);
      b = (bl + 1) >> 1;  // sqrt(T) < 2^b
      int accept = (bl > 0) && (j == ncols - 1 || bl > sTb[c]);
      if (!accept && j < ncols - 1) atomicCAS(a.status, GN_OK, GN_ESINGULAR);
      // t = T / 2^(2b) in [1/4, 1) as K limbs of fraction
      ux<K> tt;
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
      fx<K> Z;
      fx_zero<K>(Z);
      if (accept) {
        Y = ix_rsqrt_frac<K>(tt);  // 2^S / sqrt(t)
#pragma unroll
        for (int w = 0; w < K; w++) Z.w[w] = (Y.w[w] >> 1) | ((w + 1 < K) ? (Y.w[w + 1] << 63) : 0);
      }
      *sZ = Z;
      *sB = b;
      *sAccept = accept;
#pragma unroll
      for (int w = 0; w < K; w++) sTT->w[w] = tt.w[w];
    }
    __syncthreads();
    if (j < ncols - 1) {
      if (*sAccept) {
        const fx<K> Z = *sZ;
        const int sh = *sB - 1;
        uint64_t nz;
        const ux<K> uz = ix_abs<K>(Z, nz);
        for (int e = tid; e < 2 * (i1 - i0); e += MF_THREADS) {
          const int i = i0 + (e >> 1), part = e & 1;
          uint64_t na;
          ux<K> ua = ix_abs<K>(aj[2 * i + part], na);
          ux<2 * K> p = ix_umul<K>(ua, uz);
          fx<2 * K> pf;
#pragma unroll
          for (int w = 0; w < 2 * K; w++) pf.w[w] = p.w[w];
          pf = ix_sar<2 * K>(pf, sh);
          fx<K> q;
#pragma unroll
          for (int w = 0; w < K; w++) q.w[w] = pf.w[w];
          ix_cneg<K>(q, na);
          aj[2 * i + part] = q;
        }
      }
      __syncthreads();
      if (tid == 0) st_release(a.flags + (size_t)j * MF_C + rank, *sAccept ? 1u : 2u);
    }
    // off the critical path: r_jj, 1/r_jj as limbs, and the pivot's mantissa for back substitution
    if (tid == 0 && rank == 0) {
      cx<L> rc = c_zero<L>();
      if (bl > 0) {
        ux<K> tt;
#pragma unroll
        for (int w = 0; w < K; w++) tt.w[w] = sTT->w[w];
        if (!*sAccept) Y = ix_rsqrt_frac<K>(tt);
        // sqrt(t) = t y: (tt Y) / 2^(64K), scale 2^S
        ux<2 * K> ty = ix_umul<K>(tt, Y);
        fx<K> M;
#pragma unroll
        for (int w = 0; w < K; w++) M.w[w] = ty.w[K + w];
        fx_to_cascade<K, L>(M, S - b - sj, rc.re);  // r_jj = sqrt(t) 2^(b + s_j)
        if (*sAccept && j < ncols - 1) {
          fx<K> Yf;
#pragma unroll
          for (int w = 0; w < K; w++) Yf.w[w] = Y.w[w];
          double ri[L];
          fx_to_cascade<K, L>(Yf, S + b + sj, ri);  // 1/r_jj = y 2^-(b + s_j)
#pragma unroll
          for (int l = 0; l < L; l++) a.rinv[(int64_t)j * L + l] = ri[l];
          if (a.Zs) {
            double *zs = a.Zs + (size_t)j * (K + 1);
            const fx<K> Z = *sZ;
#pragma unroll
            for (int w = 0; w < K; w++) ((uint64_t *)zs)[w] = Z.w[w];
            zs[K] = (double)(-(b + 64 * K - 3) - sj);  // 1/r_jj = Z 2^this
          }
        }
      }
      c_store<L>(a.R + ((int64_t)j * a.ldr + j) * W, rc);
    }
  };

  if (g == 0 && no > 0) pivot(0, 0);

  for (int k = 0; k < ncols - 1; k++) {
    const int cstart = (k + 1 > g) ? (k + 1 - g + G - 1) / G : 0;
    if (cstart >= no) break;
    // wait for the rows of q_k that this CTA needs; the cluster compares
    // notes at the step's first barrier
    int okv = 1;
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
      okv = (v == 1);
    }
    __syncthreads();
    const fx<K> *qk = col(k);
    for (int e = tid; e < 2 * (i1 - i0); e += MF_THREADS) {
      const int i = i0 + (e >> 1), part = e & 1;
      fx<K> v;
#pragma unroll
      for (int w = 0; w < K; w++) v.w[w] = __ldcg(&qk[2 * i + part].w[w]);
      sQ[2 * (i - i0) + part] = v;
    }
    __syncthreads();

    int cb = cstart;
    const int j1 = k + 1;
    int allok = 1;
    if (j1 % G == g) {
      // lookahead column: 2 threads per row (real part, imaginary part)
      const int c = (j1 - g) / G;
      fx<K> *aj = col(j1);
      const int sj = sS[c];
      fx<K + 1> d2[2];
      fx_zero<K + 1>(d2[0]);
      fx_zero<K + 1>(d2[1]);
      for (int e = tid; e < 2 * (i1 - i0); e += MF_THREADS) {
        const int i = i0 + (e >> 1), part = e & 1;
        const fx<K> qr = sQ[2 * (i - i0)], qi = sQ[2 * (i - i0) + 1];
        const fx<K> ar = aj[2 * i], ai = aj[2 * i + 1];
        if (part == 0) {  // Re conj(q) a = qr ar + qi ai
          d2[0] = ix_add<K + 1>(d2[0], ix_mul_shift<K>(qr, ar));
          d2[0] = ix_add<K + 1>(d2[0], ix_mul_shift<K>(qi, ai));
        } else {  // Im conj(q) a = qr ai - qi ar
          d2[1] = ix_add<K + 1>(d2[1], ix_mul_shift<K>(qr, ai));
          d2[1] = ix_sub<K + 1>(d2[1], ix_mul_shift<K>(qi, ar));
        }
      }
      allok = cluster_sum<K + 1, 2>(d2, sCritD, sOk + 2 + (k & 1), okv, cl);
      if (tid == 0) {
        *sAll = allok;
        sR[2 * a.maxown] = ix_narrow<K>(d2[0]);
        sR[2 * a.maxown + 1] = ix_narrow<K>(d2[1]);
      }
      __syncthreads();
      allok = *sAll;
      if (!allok) break;
      {
        const fx<K> rr = sR[2 * a.maxown], ri = sR[2 * a.maxown + 1];
        for (int e = tid; e < 2 * (i1 - i0); e += MF_THREADS) {
          const int i = i0 + (e >> 1), part = e & 1;
          const fx<K> qr = sQ[2 * (i - i0)], qi = sQ[2 * (i - i0) + 1];
          fx<K + 1> x = ix_widen<K, K + 1>(aj[2 * i + part]);
          if (part == 0) {  // Re(a - r q) = ar - rr qr + ri qi
            x = ix_sub<K + 1>(x, ix_mul_shift<K>(rr, qr));
            x = ix_add<K + 1>(x, ix_mul_shift<K>(ri, qi));
          } else {  // Im(a - r q) = ai - rr qi - ri qr
            x = ix_sub<K + 1>(x, ix_mul_shift<K>(rr, qi));
            x = ix_sub<K + 1>(x, ix_mul_shift<K>(ri, qr));
          }
          aj[2 * i + part] = ix_narrow<K>(x);
        }
      }
      __syncthreads();
      pivot(j1, c);
      if (tid == 0 && rank == 0) {  // r_kj of the lookahead column, after the publication
        const fx<K> rr = sR[2 * a.maxown], ri = sR[2 * a.maxown + 1];
        if (a.Rm) {
          fx<K> *rm = (fx<K> *)(a.Rm + ((int64_t)j1 * a.ldr + k) * W);
          rm[0] = rr;
          rm[1] = ri;
        }
        cx<L> rk;
        fx_to_cascade<K, L>(rr, -sj, rk.re);
        fx_to_cascade<K, L>(ri, -sj, rk.im);
        c_store<L>(a.R + ((int64_t)j1 * a.ldr + k) * W, rk);
      }
      cb = c + 1;
    }
    const int nb = no - cb;
    if (nb > 0) {
      const int buf = k & 1;
      for (int cc = warp; cc < nb; cc += MF_WARPS) {
        const int c = cb + cc;
        const fx<K> *aj = col(g + G * c);
        fx<K + 1> dr, di;
        fx_zero<K + 1>(dr);
        fx_zero<K + 1>(di);
        for (int i = i0 + lane; i < i1; i += 32) {
          const fx<K> qr = sQ[2 * (i - i0)], qi = sQ[2 * (i - i0) + 1];
          const fx<K> ar = aj[2 * i], ai = aj[2 * i + 1];
          dr = ix_add<K + 1>(dr, ix_mul_shift<K>(qr, ar));
          dr = ix_add<K + 1>(dr, ix_mul_shift<K>(qi, ai));
          di = ix_add<K + 1>(di, ix_mul_shift<K>(qr, ai));
          di = ix_sub<K + 1>(di, ix_mul_shift<K>(qi, ar));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          fx<K + 1> u, v;
#pragma unroll
          for (int w = 0; w < K + 1; w++) {
            u.w[w] = __shfl_xor_sync(0xffffffffu, dr.w[w], o);
            v.w[w] = __shfl_xor_sync(0xffffffffu, di.w[w], o);
          }
          dr = ix_add<K + 1>(dr, u);
          di = ix_add<K + 1>(di, v);
        }
        if (lane == 0) {
          sDot[(buf * a.maxown + c) * 2] = dr;
          sDot[(buf * a.maxown + c) * 2 + 1] = di;
        }
      }
      if (tid == 0) sOk[buf] = (j1 % G == g) ? 1 : okv;  // lookahead already checked the wait
      cl.sync();
      if (warp == 0) {
        int okr = (lane < MF_C) ? cl.map_shared_rank(sOk, lane)[buf] : 1;
        okr = __all_sync(0xffffffffu, okr);
        if (lane == 0) *sAll = okr;
      }
      for (int cc = tid; cc < nb; cc += MF_THREADS) {
        const int c = cb + cc;
        fx<K + 1> tr, ti;
        fx_zero<K + 1>(tr);
        fx_zero<K + 1>(ti);
        for (int r = 0; r < MF_C; r++) {
          const fx<K + 1> *p = cl.map_shared_rank(sDot, r) + (buf * a.maxown + c) * 2;
          tr = ix_add<K + 1>(tr, p[0]);
          ti = ix_add<K + 1>(ti, p[1]);
        }
        sR[2 * c] = ix_narrow<K>(tr);
        sR[2 * c + 1] = ix_narrow<K>(ti);
        if (rank == 0) {
          if (a.Rm) {
            fx<K> *rm = (fx<K> *)(a.Rm + ((int64_t)(g + G * c) * a.ldr + k) * W);
            rm[0] = sR[2 * c];
            rm[1] = sR[2 * c + 1];
          }
          cx<L> rk;
          fx_to_cascade<K + 1, L>(tr, -sS[c], rk.re);
          fx_to_cascade<K + 1, L>(ti, -sS[c], rk.im);
          c_store<L>(a.R + ((int64_t)(g + G * c) * a.ldr + k) * W, rk);
        }
      }
      __syncthreads();
      if (!*sAll) break;
      for (int cc = warp; cc < nb; cc += MF_WARPS) {
        const int c = cb + cc;
        fx<K> *aj = col(g + G * c);
        const fx<K> rr = sR[2 * c], ri = sR[2 * c + 1];
        for (int i = i0 + lane; i < i1; i += 32) {
          const fx<K> qr = sQ[2 * (i - i0)], qi = sQ[2 * (i - i0) + 1];
          fx<K + 1> xr = ix_widen<K, K + 1>(aj[2 * i]);
          fx<K + 1> xi = ix_widen<K, K + 1>(aj[2 * i + 1]);
          xr = ix_sub<K + 1>(xr, ix_mul_shift<K>(rr, qr));
          xr = ix_add<K + 1>(xr, ix_mul_shift<K>(ri, qi));
          xi = ix_sub<K + 1>(xi, ix_mul_shift<K>(rr, qi));
          xi = ix_sub<K + 1>(xi, ix_mul_shift<K>(ri, qr));
          aj[2 * i] = ix_narrow<K>(xr);
          aj[2 * i + 1] = ix_narrow<K>(xi);
        }
      }
    }
  }
  if (!ok) atomicCAS(a.status, GN_OK, GN_ENONFINITE);
  cl.sync();
}

template <int L>
struct MiLayout {
  size_t bytes;
  __host__ __device__ MiLayout(int maxown, int ms) {
    constexpr int K = L;
    size_t b = 16 * ((maxown * 8 + 15) / 16);
    b += 16 * maxown;                                  // sN0, sN0p
    b += sizeof(fx<K + 1>) * (4 * maxown + 2 * MF_WARPS);  // sDot, sCritD
    b += sizeof(fx<2 * K + 1>) * MF_WARPS;             // sCritT
    b += sizeof(fx<K>) * 2 * (maxown + 1);             // sR
    b += sizeof(fx<K>) * 2 * (ms > 0 ? ms : 1);        // sQ
    b += 32 + 2 * sizeof(fx<K>) + 64;                  // flags, Z, t, slack
    bytes = (b + 255) & ~(size_t)255;
  }
};

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

// x = y 2^sig * Z 2^e as a K-limb mantissa per part and the exponent t
template <int K, int KY>
__device__ __forceinline__ void bs_solve(const fx<KY> &yr, const fx<KY> &yi, const fx<K> &Z, int e,
                                         int sig, fx<K> &Xr, fx<K> &Xi, int &t) {
  uint64_t nz;
  const ux<K> uz = ix_abs<K>(Z, nz);
  fx<KY + K> P[2];
  int B = 0;
#pragma unroll
  for (int part = 0; part < 2; part++) {
    uint64_t ny;
    const ux<KY> uy = ix_abs<KY>(part ? yi : yr, ny);
    // |y| |Z| as KY + K limbs
#pragma unroll
    for (int w = 0; w < KY + K; w++) P[part].w[w] = 0;
#pragma unroll
    for (int a = 0; a < KY; a++) {
      u128_t carry = 0;
#pragma unroll
      for (int b = 0; b < K; b++) {
        u128_t tt = (u128_t)uy.w[a] * uz.w[b] + P[part].w[a + b] + carry;
        P[part].w[a + b] = (uint64_t)tt;
        carry = tt >> 64;
      }
      P[part].w[a + K] = (uint64_t)carry;
    }
    const int bl = ix_bitlen<KY + K>(P[part]);
    B = bl > B ? bl : B;
    ix_cneg<KY + K>(P[part], ny ^ nz);
  }
  const int sh = B > 64 * K - 2 ? B - (64 * K - 2) : 0;
  const fx<KY + K> qr = ix_sar<KY + K>(P[0], sh), qi = ix_sar<KY + K>(P[1], sh);
#pragma unroll
  for (int w = 0; w < K; w++) {
    Xr.w[w] = qr.w[w];
    Xi.w[w] = qi.w[w];
  }
  t = sig + e + sh;
}

// (yr, yi) -= r x, with r x at scale 2^d relative to the units of y
template <int K, int KY>
__device__ __forceinline__ void bs_update(fx<KY> &yr, fx<KY> &yi, const fx<K> &rr, const fx<K> &ri,
                                          const fx<K> &xr, const fx<K> &xi, int d, int *sFail) {
  // re = rr xr - ri xi, im = rr xi + ri xr as 2K+1 limbs
  fx<2 * K + 1> pr, pi;
  {
    uint64_t n1, n2, n3, n4;
    ux<K> a1 = ix_abs<K>(rr, n1), b1 = ix_abs<K>(xr, n2);
    ux<K> a2 = ix_abs<K>(ri, n3), b2 = ix_abs<K>(xi, n4);
    ux<2 * K> p1 = ix_umul<K>(a1, b1), p2 = ix_umul<K>(a2, b2);
    ux<2 * K> p3 = ix_umul<K>(a1, b2), p4 = ix_umul<K>(a2, b1);
    fx<2 * K + 1> f1, f2, f3, f4;
#pragma unroll
    for (int w = 0; w < 2 * K; w++) {
      f1.w[w] = p1.w[w];
      f2.w[w] = p2.w[w];
      f3.w[w] = p3.w[w];
      f4.w[w] = p4.w[w];
    }
    f1.w[2 * K] = f2.w[2 * K] = f3.w[2 * K] = f4.w[2 * K] = 0;
    ix_cneg<2 * K + 1>(f1, n1 ^ n2);
    ix_cneg<2 * K + 1>(f2, n3 ^ n4);
    ix_cneg<2 * K + 1>(f3, n1 ^ n4);
    ix_cneg<2 * K + 1>(f4, n3 ^ n2);
    pr = ix_sub<2 * K + 1>(f1, f2);
    pi = ix_add<2 * K + 1>(f3, f4);
  }
  fx<KY> ur, ui;
  if (d <= 0) {
    const int s = -d;
    if (s >= 64 * (2 * K + 1)) {
      fx_zero<KY>(ur);
      fx_zero<KY>(ui);
    } else {
      const fx<2 * K + 1> qr = ix_sar<2 * K + 1>(pr, s), qi = ix_sar<2 * K + 1>(pi, s);
#pragma unroll
      for (int w = 0; w < KY; w++) {
        ur.w[w] = w < 2 * K + 1 ? qr.w[w] : (0 - (qr.w[2 * K] >> 63));
        ui.w[w] = w < 2 * K + 1 ? qi.w[w] : (0 - (qi.w[2 * K] >> 63));
      }
    }
  } else {
    // a product larger than the units of y by 2^d: only harmless when tiny
    if (ix_bitlen<2 * K + 1>(pr) + d > 64 * KY - 2 || ix_bitlen<2 * K + 1>(pi) + d > 64 * KY - 2)
      *sFail = 1;
#pragma unroll
    for (int w = 0; w < KY; w++) {
      ur.w[w] = w < 2 * K + 1 ? pr.w[w] : (0 - (pr.w[2 * K] >> 63));
      ui.w[w] = w < 2 * K + 1 ? pi.w[w] : (0 - (pi.w[2 * K] >> 63));
    }
    // shift left by d (d < 64 KY guaranteed by the check above when it succeeds)
    const int dd = d < 64 * KY ? d : 64 * KY - 1;
    ur = ix_shl<KY>(ur, dd);
    ui = ix_shl<KY>(ui, dd);
  }
  yr = ix_sub<KY>(yr, ur);
  yi = ix_sub<KY>(yi, ui);
}

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
