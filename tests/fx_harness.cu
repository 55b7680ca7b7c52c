// Host harness for csrc/fx.cuh (test support): reads "F L count" then count
// doubles (as hex bit patterns) from stdin, accumulates them exactly in a
// 3- or 5-limb fixed-point accumulator and prints the L-limb cascade.
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "../paper_1402_2626_gb300/csrc/fx.cuh"

template <int NL, int L>
static int run(int F, int count) {
  gn::fx<NL> a;
  gn::fx_zero<NL>(a);
  int ok = 1;
  for (int i = 0; i < count; i++) {
    unsigned long long b;
    if (scanf("%llx", &b) != 1) return 2;
    double d;
    memcpy(&d, &b, 8);
    ok &= gn::fx_add_double<NL>(a, d, F) ? 1 : 0;
  }
  double out[L];
  gn::fx_to_cascade<NL, L>(a, F, out);
  printf("%d", ok);
  for (int l = 0; l < L; l++) {
    unsigned long long b;
    memcpy(&b, &out[l], 8);
    printf(" %llx", b);
  }
  printf("\n");
  return 0;
}

int main() {
  int NL, F, L, count;
  while (scanf("%d %d %d %d", &NL, &F, &L, &count) == 4) {
    int r = 0;
    if (NL == 3 && L == 2) r = run<3, 2>(F, count);
    else if (NL == 5 && L == 4) r = run<5, 4>(F, count);
    else if (NL == 2 && L == 1) r = run<2, 1>(F, count);
    else return 3;
    if (r) return r;
    fflush(stdout);
  }
  return 0;
}
