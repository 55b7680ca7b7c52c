// Host harness for csrc/cf.cuh (test support).  Lines:
//   "mul K L  ar[L] ai[L] br[L] bi[L]"   (doubles as hex bits) -> product cascade
//   "scale K L ar[L] ai[L] d"                                  -> d * a cascade
//   "rt K L ar[L] ai[L]"                                       -> round trip
//   "same K N seed"   N random cases: cf_normalize and cf_mul against the
//                     forms written out below (two shift branches; four signed
//                     products then a subtraction and an addition), bit for
//                     bit -> "ok N" or "bad i"
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

// SplitMix64 (the published constants of that generator)
static uint64_t sm_state;
static uint64_t sm_next() {
  uint64_t z = (sm_state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// a signed N-limb value below 2^bits in magnitude; now and then a power of two
template <int N>
static gn::fx<N> rnd_bits(int bits) {
  gn::fx<N> v;
  for (int i = 0; i < N; i++) v.w[i] = 0;
  if (sm_next() % 10 == 0) {
    if (bits > 0) v.w[(bits - 1) / 64] = 1ull << ((bits - 1) % 64);
  } else {
    for (int i = 0; i < N && 64 * i < bits; i++) {
      const int keep = bits - 64 * i;
      v.w[i] = keep >= 64 ? sm_next() : (sm_next() & ((1ull << keep) - 1));
    }
  }
  if (sm_next() & 1) gn::ix_cneg<N>(v, 1);
  return v;
}

// renormalisation with the shift's two directions as separate barrel shifts
template <int K>
static int ref_normalize(gn::fx<K + 1> re, gn::fx<K + 1> im, gn::fx<K> &ore, gn::fx<K> &oim) {
  uint64_t n1, n2;
  const gn::ux<K + 1> ur = gn::ix_abs<K + 1>(re, n1), ui = gn::ix_abs<K + 1>(im, n2);
  gn::fx<K + 1> ar, ai;
  for (int w = 0; w <= K; w++) {
    ar.w[w] = ur.w[w];
    ai.w[w] = ui.w[w];
  }
  const int b1 = gn::ix_bitlen<K + 1>(ar), b2 = gn::ix_bitlen<K + 1>(ai);
  const int B = b1 > b2 ? b1 : b2;
  if (B == 0) {
    gn::fx_zero<K>(ore);
    gn::fx_zero<K>(oim);
    return gn::CF_EZERO;
  }
  const int sh = B - (64 * K - 2);
  if (sh >= 0) {
    re = gn::ix_sar<K + 1>(re, sh);
    im = gn::ix_sar<K + 1>(im, sh);
  } else {
    re = gn::ix_shl<K + 1>(re, -sh);
    im = gn::ix_shl<K + 1>(im, -sh);
  }
  ore = gn::ix_narrow<K>(re);
  oim = gn::ix_narrow<K>(im);
  return sh;
}

// the product as four signed truncated products, a subtraction and an addition
template <int K>
static gn::cf<K> ref_mul(const gn::cf<K> &a, const gn::cf<K> &b) {
  gn::fx<K + 1> re = gn::ix_sub<K + 1>(gn::ix_mul_shift<K>(a.re, b.re), gn::ix_mul_shift<K>(a.im, b.im));
  gn::fx<K + 1> im = gn::ix_add<K + 1>(gn::ix_mul_shift<K>(a.re, b.im), gn::ix_mul_shift<K>(a.im, b.re));
  gn::cf<K> r;
  const int sh = ref_normalize<K>(re, im, r.re, r.im);
  r.e = (sh == gn::CF_EZERO || a.e == gn::CF_EZERO || b.e == gn::CF_EZERO) ? gn::CF_EZERO
                                                                           : a.e + b.e + (64 * K - 2) + sh;
  return r;
}

template <int K>
static void same(long n) {
  for (long t = 0; t < n; t++) {
    // renormalisation of (K+1)-limb values of any size up to 2^(64K + 53)
    const int b1 = (int)(sm_next() % (64 * K + 54)), b2 = (int)(sm_next() % (64 * K + 54));
    gn::fx<K + 1> re = rnd_bits<K + 1>(b1), im = rnd_bits<K + 1>(sm_next() % 4 ? b2 : b1);
    gn::fx<K> o1r, o1i, o2r, o2i;
    gn::fx<K + 1> r2 = re, i2 = im;
    const int s1 = ref_normalize<K>(re, im, o1r, o1i);
    const int s2 = gn::cf_normalize<K>(r2, i2, o2r, o2i);
    bool ok = s1 == s2;
    for (int i = 0; i < K; i++) ok &= o1r.w[i] == o2r.w[i] && o1i.w[i] == o2i.w[i];
    // products of normalised values (and, now and then, of arbitrary ones)
    gn::cf<K> a, b;
    const bool any = sm_next() % 5 == 0;
    const int ba = any ? 1 + (int)(sm_next() % (64 * K - 1)) : 64 * K - 2 - (int)(sm_next() % 2);
    const int bb = any ? 1 + (int)(sm_next() % (64 * K - 1)) : 64 * K - 2 - (int)(sm_next() % 2);
    a.re = rnd_bits<K>(ba);
    a.im = rnd_bits<K>(ba - (int)(sm_next() % 4));
    b.re = rnd_bits<K>(bb);
    b.im = rnd_bits<K>(bb - (int)(sm_next() % 4));
    a.e = (int)(sm_next() % 200) - 100;
    b.e = (int)(sm_next() % 200) - 100;
    if (sm_next() % 50 == 0) a = gn::cf_zero<K>();
    const gn::cf<K> x = ref_mul<K>(a, b), y = gn::cf_mul<K>(a, b);
    ok &= x.e == y.e;
    for (int i = 0; i < K; i++) ok &= x.re.w[i] == y.re.w[i] && x.im.w[i] == y.im.w[i];
    if (!ok) {
      printf("bad %ld\n", t);
      return;
    }
  }
  printf("ok %ld\n", n);
}

int main() {
  char op[16];
  int K, L;
  while (scanf("%15s %d %d", op, &K, &L) == 3) {
    if (!strcmp(op, "same")) {
      unsigned long long seed;
      if (scanf("%llu", &seed) != 1) return 2;
      sm_state = seed;
      if (K == 1) same<1>(L);
      else if (K == 2) same<2>(L);
      else if (K == 4) same<4>(L);
      else return 2;
    } else if (K == 1 && L == 1) run<1, 1>(op);
    else if (K == 2 && L == 2) run<2, 2>(op);
    else if (K == 4 && L == 4) run<4, 4>(op);
    else return 2;
    fflush(stdout);
  }
  return 0;
}
