// Host harness for csrc/cf.cuh (test support).  Lines:
//   "mul K L  ar[L] ai[L] br[L] bi[L]"   (doubles as hex bits) -> product cascade
//   "scale K L ar[L] ai[L] d"                                  -> d * a cascade
//   "rt K L ar[L] ai[L]"                                       -> round trip
#include <cstdio>
#include <cstring>
#include <cstdint>
#include "../paper_1402_2626_gb300/csrc/cf.cuh"

static double rd() {
  unsigned long long b;
  scanf("%llx", &b);
  double d;
  memcpy(&d, &b, 8);
  return d;
}
static void pr(double d) {
  unsigned long long b;
  memcpy(&b, &d, 8);
  printf("%llx ", b);
}

template <int K, int L>
static void run(const char *op) {
  double ar[L], ai[L], br[L], bi[L];
  for (int l = 0; l < L; l++) ar[l] = rd();
  for (int l = 0; l < L; l++) ai[l] = rd();
  gn::cf<K> a = gn::cf_from_cascade<K, L>(ar, ai), r;
  if (!strcmp(op, "mul")) {
    for (int l = 0; l < L; l++) br[l] = rd();
    for (int l = 0; l < L; l++) bi[l] = rd();
    gn::cf<K> b = gn::cf_from_cascade<K, L>(br, bi);
    r = gn::cf_mul<K>(a, b);
  } else if (!strcmp(op, "scale")) {
    unsigned d;
    scanf("%u", &d);
    r = gn::cf_scale_int<K>(a, d);
  } else {
    r = a;
  }
  double orr[L], oi[L];
  gn::cf_to_cascade<K, L>(r, orr, oi);
  for (int l = 0; l < L; l++) pr(orr[l]);
  for (int l = 0; l < L; l++) pr(oi[l]);
  printf("\n");
}

int main() {
  char op[16];
  int K, L;
  while (scanf("%15s %d %d", op, &K, &L) == 3) {
    if (K == 1 && L == 1) run<1, 1>(op);
    else if (K == 2 && L == 2) run<2, 2>(op);
    else if (K == 4 && L == 4) run<4, 4>(op);
    else return 2;
    fflush(stdout);
  }
  return 0;
}
