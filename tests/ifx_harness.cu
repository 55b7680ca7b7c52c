// Host harness for csrc/ifx.cuh (test support).  Reads lines
// "op K a_0..a_{K-1} b_0..b_{K-1} [s]" (hex limbs, little-endian) and prints
// the result limbs in hex.  ops: mul (ix_mul_shift), sq (ix_square),
// add, sub, sar (by s), bitlen, rsqrt, rsqrtseed (with a given seed); and "xsar N a_0..a_{N-1} s" / "xshl N ..."
// (ix_sar / ix_shl on N-limb values, N = 1..5 or 9).
#include <cstdio>
#include <cstring>
#include <cstdint>
#include "../paper_1402_2626_gb300/csrc/ifx.cuh"

template <int K>
static void run(const char *op) {
  gn::fx<K> a, b;
  for (int i = 0; i < K; i++) scanf("%llx", (unsigned long long *)&a.w[i]);
  for (int i = 0; i < K; i++) scanf("%llx", (unsigned long long *)&b.w[i]);
  int s = 0;
  if (!strcmp(op, "sar")) scanf("%d", &s);
  if (!strcmp(op, "mul")) {
    gn::fx<K + 1> r = gn::ix_mul_shift<K>(a, b);
    for (int i = 0; i < K + 1; i++) printf("%llx ", (unsigned long long)r.w[i]);
  } else if (!strcmp(op, "sq")) {
    gn::fx<2 * K + 1> r = gn::ix_square<K>(a);
    for (int i = 0; i < 2 * K + 1; i++) printf("%llx ", (unsigned long long)r.w[i]);
  } else if (!strcmp(op, "add")) {
    gn::fx<K> r = gn::ix_add<K>(a, b);
    for (int i = 0; i < K; i++) printf("%llx ", (unsigned long long)r.w[i]);
  } else if (!strcmp(op, "sub")) {
    gn::fx<K> r = gn::ix_sub<K>(a, b);
    for (int i = 0; i < K; i++) printf("%llx ", (unsigned long long)r.w[i]);
  } else if (!strcmp(op, "sar")) {
    gn::fx<K> r = gn::ix_sar<K>(a, s);
    for (int i = 0; i < K; i++) printf("%llx ", (unsigned long long)r.w[i]);
  } else if (!strcmp(op, "rsqrt")) {
    gn::ux<K> t;
    for (int i = 0; i < K; i++) t.w[i] = a.w[i];
    gn::ux<K> y = gn::ix_rsqrt_frac<K>(t);
    for (int i = 0; i < K; i++) printf("%llx ", (unsigned long long)y.w[i]);
  } else if (!strcmp(op, "rsqrtseed")) {
    // t in a, then the one-limb seed Y1 (scale 2^62)
    gn::ux<K> t;
    for (int i = 0; i < K; i++) t.w[i] = a.w[i];
    unsigned long long y1;
    scanf("%llx", &y1);
    gn::ux<1> Y1;
    Y1.w[0] = y1;
    gn::ux<K> y = gn::ix_rsqrt_from_seed<K>(t, Y1);
    for (int i = 0; i < K; i++) printf("%llx ", (unsigned long long)y.w[i]);
  } else if (!strcmp(op, "mulf")) {
    // a (K+1 limbs: a_0..a_{K-1} then one more) times b (K limbs)
    gn::fx<K + 1> a1;
    for (int i = 0; i < K; i++) a1.w[i] = a.w[i];
    unsigned long long top;
    scanf("%llx", &top);
    a1.w[K] = top;
    gn::fx<2 * K + 1> r = gn::ix_mul_full<K + 1, K>(a1, b);
    for (int i = 0; i < 2 * K + 1; i++) printf("%llx ", (unsigned long long)r.w[i]);
  } else if (!strcmp(op, "bitlen")) {
    printf("%x ", gn::ix_bitlen<K>(a));
  }
  printf("\n");
}

template <int N>
static void run_shift(const char *op) {
  gn::fx<N> a;
  for (int i = 0; i < N; i++) scanf("%llx", (unsigned long long *)&a.w[i]);
  int s = 0;
  scanf("%d", &s);
  gn::fx<N> r = !strcmp(op, "xsar") ? gn::ix_sar<N>(a, s) : gn::ix_shl<N>(a, s);
  for (int i = 0; i < N; i++) printf("%llx ", (unsigned long long)r.w[i]);
  printf("\n");
}

int main() {
  char op[16];
  int K;
  while (scanf("%15s %d", op, &K) == 2) {
    if (op[0] == 'x') {
      switch (K) {
        case 1: run_shift<1>(op); break;
        case 2: run_shift<2>(op); break;
        case 3: run_shift<3>(op); break;
        case 4: run_shift<4>(op); break;
        case 5: run_shift<5>(op); break;
        case 9: run_shift<9>(op); break;
        default: return 2;
      }
      fflush(stdout);
      continue;
    }
    if (K == 1) run<1>(op);
    else if (K == 2) run<2>(op);
    else if (K == 4) run<4>(op);
    else return 2;
    fflush(stdout);
  }
  return 0;
}
