/*
 * CPU oracle for the Gauss-Newton hot path of Verschelde & Yu, "GPU
 * acceleration of Newton's method for large systems of polynomial equations
 * in double double and quad double arithmetic" (2014).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark load this library; the product path never does.
 * It shares no code with the CUDA library.
 *
 * It is slow on purpose and meant to be checked by eye against the paper:
 *
 *   Arithmetic.  A real number at precision L (L = 1, 2, 4 doubles: double,
 *   double double, quad double, Section 1) is a cascade of L doubles.  Every
 *   operation on such numbers first forms the EXACT result as a floating-point
 *   expansion (Shewchuk 1997, "Adaptive precision floating-point arithmetic":
 *   Knuth's TwoSum, the FMA form of TwoProduct, Grow-Expansion with zero
 *   elimination), then rounds that expansion to L limbs: limb 0 is the
 *   expansion's value to within an ulp, limb 1 the same for what is left,
 *   and so on.  Complex operations round the real and the imaginary part once
 *   each.  Division is long division with exact remainders; square root is
 *   Newton's iteration on s -> (s + a/s)/2.
 *
 *   Evaluation and differentiation (Section 2).  Two modes:
 *     definition: every term and every partial derivative is formed on its
 *       own by repeated multiplication, no sharing (the "straightforward"
 *       count n-1 + n(n-2) of Section 2.2);
 *     reverse: table of pure powers and common factor (Section 2.1, eq. 1),
 *       Speelpenning product and gradient with forward products and one
 *       running backward product (Section 2.2, 3k-5 multiplications), then
 *       coefficient x common factor x exponent (Section 2.3) and the sums
 *       into f and J (Section 2.3).
 *
 *   Least squares (Section 3).  Modified Gram-Schmidt on [A b] as in the
 *   figure "The modified Gram-Schmidt orthogonalization algorithm" with
 *   conjugated inner products, eq. 2 for y and z, and back substitution
 *   r_ll x_l = y_l - sum_{j>l} r_lj x_j (the reading of eq. 5).
 *
 *   Coefficient gradient at a root (an extension past the paper: the
 *   implicit function theorem at the Newton fixed point of Section 4):
 *   forward substitution with R^H, lambda = Q w, monomial values by the
 *   definition, grad_t = -lambda_i conj(x^{a_t}).
 *
 * Layout of a complex number at precision L: 2L doubles, the L limbs of the
 * real part then the L limbs of the imaginary part.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no -ffast-math:
 * the error-free transformations need IEEE round-to-nearest arithmetic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define O_OK 0
#define O_EINVAL 1
#define O_ESINGULAR 4
#define O_EOVERFLOW 9

#define XMAX 512

/* ---------------------------------------------------------------------- */
/* Error-free transformations and expansions (Shewchuk 1997)                */
/* ---------------------------------------------------------------------- */

/* s + e == a + b exactly, s = fl(a + b) (Knuth). */
static void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  double br = b - bv;
  double ar = a - av;
  *s = x;
  *e = ar + br;
}

/* p + e == a * b exactly, p = fl(a * b). */
static void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *p = x;
  *e = fma(a, b, -x);
}

/* A nonoverlapping expansion, components in increasing magnitude, no zeros. */
typedef struct {
  int len;
  int overflow;
  double t[XMAX];
} xpn;

static void x_init(xpn *e) {
  e->len = 0;
  e->overflow = 0;
}

/* e := e + b exactly (Grow-Expansion with zero elimination). */
static void x_grow(xpn *e, double b) {
  double q = b;
  int out = 0;
  for (int i = 0; i < e->len; i++) {
    double s, h;
    two_sum(q, e->t[i], &s, &h);
    q = s;
    if (h != 0.0) e->t[out++] = h; /* out <= i: writing in place is safe */
  }
  if (q != 0.0) {
    if (out >= XMAX) {
      e->overflow = 1;
      return;
    }
    e->t[out++] = q;
  }
  e->len = out;
}

/* e := e + a * b exactly. */
static void x_grow_prod(xpn *e, double a, double b) {
  double p, err;
  two_prod(a, b, &p, &err);
  x_grow(e, p);
  x_grow(e, err);
}

/* Round the value of e to a cascade of L doubles; e is consumed. */
static void x_round(xpn *e, int L, double *out) {
  for (int l = 0; l < L; l++) {
    double approx = 0.0;
    for (int i = 0; i < e->len; i++) approx += e->t[i]; /* smallest first */
    out[l] = approx;
    if (approx != 0.0) x_grow(e, -approx);
  }
}

/* Value of e as one double (for comparisons and seeds). */
static double x_approx(const xpn *e) {
  double a = 0.0;
  for (int i = 0; i < e->len; i++) a += e->t[i];
  return a;
}

/* ---------------------------------------------------------------------- */
/* Reals at precision L                                                    */
/* ---------------------------------------------------------------------- */

static void r_add(int L, const double *a, const double *b, double *c) {
  xpn e;
  x_init(&e);
  for (int i = 0; i < L; i++) x_grow(&e, a[i]);
  for (int i = 0; i < L; i++) x_grow(&e, b[i]);
  x_round(&e, L, c);
}

static void r_sub(int L, const double *a, const double *b, double *c) {
  xpn e;
  x_init(&e);
  for (int i = 0; i < L; i++) x_grow(&e, a[i]);
  for (int i = 0; i < L; i++) x_grow(&e, -b[i]);
  x_round(&e, L, c);
}

static void r_mul(int L, const double *a, const double *b, double *c) {
  xpn e;
  x_init(&e);
  for (int i = 0; i < L; i++)
    for (int j = 0; j < L; j++) x_grow_prod(&e, a[i], b[j]);
  x_round(&e, L, c);
}

/* a / b by long division: L+2 quotient digits, each from the exact remainder. */
static int r_div(int L, const double *a, const double *b, double *c) {
  double bh = 0.0;
  for (int i = L - 1; i >= 0; i--) bh += b[i];
  if (bh == 0.0) return O_ESINGULAR;
  xpn rem, quo;
  x_init(&rem);
  x_init(&quo);
  for (int i = 0; i < L; i++) x_grow(&rem, a[i]);
  for (int d = 0; d < L + 2; d++) {
    double q = x_approx(&rem) / bh;
    if (q == 0.0) break;
    x_grow(&quo, q);
    for (int j = 0; j < L; j++) x_grow_prod(&rem, -q, b[j]);
  }
  x_round(&quo, L, c);
  return (rem.overflow || quo.overflow) ? O_EOVERFLOW : O_OK;
}

/* sqrt(a), a >= 0: Newton s <- (s + a/s)/2 from the double square root. */
static int r_sqrt(int L, const double *a, double *c) {
  double ah = 0.0;
  for (int i = L - 1; i >= 0; i--) ah += a[i];
  for (int i = 0; i < L; i++) c[i] = 0.0;
  if (ah <= 0.0) return ah < 0.0 ? O_EINVAL : O_OK;
  double s[4] = {sqrt(ah), 0, 0, 0};
  double q[4], t[4];
  int iters = (L == 1) ? 1 : (L == 2 ? 2 : 3);
  for (int it = 0; it < iters; it++) {
    int st = r_div(L, a, s, q);
    if (st) return st;
    r_add(L, s, q, t);
    for (int i = 0; i < L; i++) s[i] = 0.5 * t[i]; /* exact */
  }
  memcpy(c, s, sizeof(double) * L);
  return O_OK;
}

/* ---------------------------------------------------------------------- */
/* Complex numbers at precision L: [re limbs | im limbs]                   */
/* ---------------------------------------------------------------------- */

static void c_zero(int L, double *c) { memset(c, 0, sizeof(double) * 2 * L); }

static void c_one(int L, double *c) {
  c_zero(L, c);
  c[0] = 1.0;
}

static void c_add(int L, const double *a, const double *b, double *c) {
  r_add(L, a, b, c);
  r_add(L, a + L, b + L, c + L);
}

static void c_sub(int L, const double *a, const double *b, double *c) {
  r_sub(L, a, b, c);
  r_sub(L, a + L, b + L, c + L);
}

/* c = a * b, each part the exact value rounded once. */
static void c_mul(int L, const double *a, const double *b, double *c) {
  xpn e;
  double re[4], im[4];
  x_init(&e);
  for (int i = 0; i < L; i++)
    for (int j = 0; j < L; j++) {
      x_grow_prod(&e, a[i], b[j]);
      x_grow_prod(&e, -a[L + i], b[L + j]);
    }
  x_round(&e, L, re);
  x_init(&e);
  for (int i = 0; i < L; i++)
    for (int j = 0; j < L; j++) {
      x_grow_prod(&e, a[i], b[L + j]);
      x_grow_prod(&e, a[L + i], b[j]);
    }
  x_round(&e, L, im);
  memcpy(c, re, sizeof(double) * L);
  memcpy(c + L, im, sizeof(double) * L);
}

/* c = conj(a) * b */
static void c_conj_mul(int L, const double *a, const double *b, double *c) {
  xpn e;
  double re[4], im[4];
  x_init(&e);
  for (int i = 0; i < L; i++)
    for (int j = 0; j < L; j++) {
      x_grow_prod(&e, a[i], b[j]);
      x_grow_prod(&e, a[L + i], b[L + j]);
    }
  x_round(&e, L, re);
  x_init(&e);
  for (int i = 0; i < L; i++)
    for (int j = 0; j < L; j++) {
      x_grow_prod(&e, a[i], b[L + j]);
      x_grow_prod(&e, -a[L + i], b[j]);
    }
  x_round(&e, L, im);
  memcpy(c, re, sizeof(double) * L);
  memcpy(c + L, im, sizeof(double) * L);
}

/* c = d * a for a small integer d (the exponent factor of Section 2.3). */
static void c_scale_int(int L, const double *a, int d, double *c) {
  double dd = (double)d;
  double re[4], im[4];
  xpn e;
  x_init(&e);
  for (int i = 0; i < L; i++) x_grow_prod(&e, a[i], dd);
  x_round(&e, L, re);
  x_init(&e);
  for (int i = 0; i < L; i++) x_grow_prod(&e, a[L + i], dd);
  x_round(&e, L, im);
  memcpy(c, re, sizeof(double) * L);
  memcpy(c + L, im, sizeof(double) * L);
}

/* |a|^2 = re^2 + im^2 (a real number at precision L). */
static void c_abs2(int L, const double *a, double *r) {
  xpn e;
  x_init(&e);
  for (int i = 0; i < L; i++)
    for (int j = 0; j < L; j++) {
      x_grow_prod(&e, a[i], a[j]);
      x_grow_prod(&e, a[L + i], a[L + j]);
    }
  x_round(&e, L, r);
}

/* c = a / r for a real r. */
static int c_div_real(int L, const double *a, const double *r, double *c) {
  int s1 = r_div(L, a, r, c);
  int s2 = r_div(L, a + L, r, c + L);
  return s1 ? s1 : s2;
}

/* ---------------------------------------------------------------------- */
/* Exported primitives (used by the tests that pin the arithmetic)          */
/* ---------------------------------------------------------------------- */

/* op: 0 add, 1 sub, 2 mul, 3 div, 4 sqrt(a) */
int o_real_op(int L, int op, const double *a, const double *b, double *c) {
  if (L != 1 && L != 2 && L != 4) return O_EINVAL;
  switch (op) {
    case 0: r_add(L, a, b, c); return O_OK;
    case 1: r_sub(L, a, b, c); return O_OK;
    case 2: r_mul(L, a, b, c); return O_OK;
    case 3: return r_div(L, a, b, c);
    case 4: return r_sqrt(L, a, c);
  }
  return O_EINVAL;
}

/* op: 0 add, 1 sub, 2 mul, 3 conj(a)*b, 4 |a|^2 (real part of c), 5 a / re(b) */
int o_cplx_op(int L, int op, const double *a, const double *b, double *c) {
  if (L != 1 && L != 2 && L != 4) return O_EINVAL;
  switch (op) {
    case 0: c_add(L, a, b, c); return O_OK;
    case 1: c_sub(L, a, b, c); return O_OK;
    case 2: c_mul(L, a, b, c); return O_OK;
    case 3: c_conj_mul(L, a, b, c); return O_OK;
    case 4: c_zero(L, c); c_abs2(L, a, c); return O_OK;
    case 5: return c_div_real(L, a, b, c);
  }
  return O_EINVAL;
}

/* ---------------------------------------------------------------------- */
/* Evaluation and differentiation (Section 2)                               */
/* ---------------------------------------------------------------------- */

#define KMAXO 4096

typedef struct {
  int L;
  int cl; /* limbs per part in coef */
  const double *coef;
  const double *x;
} ctx_t;

static void load_coef(const ctx_t *cx, int64_t t, double *c) {
  c_zero(cx->L, c);
  int m = cx->cl < cx->L ? cx->cl : cx->L;
  for (int l = 0; l < m; l++) {
    c[l] = cx->coef[(t * 2 + 0) * cx->cl + l];
    c[cx->L + l] = cx->coef[(t * 2 + 1) * cx->cl + l];
  }
}

static const double *xv(const ctx_t *cx, int v) { return cx->x + (int64_t)v * 2 * cx->L; }

/* x_v^d by d-1 repeated multiplications (d >= 1). */
static void power_naive(const ctx_t *cx, int v, int d, double *out, int64_t *nmul) {
  int L = cx->L;
  memcpy(out, xv(cx, v), sizeof(double) * 2 * L);
  for (int p = 2; p <= d; p++) {
    c_mul(L, out, xv(cx, v), out);
    (*nmul)++;
  }
}

/*
 * Definition mode for one monomial c * prod_s x_{v_s}^{d_s}: the term and the
 * k partials d_s c x_{v_s}^{d_s-1} prod_{r != s} x_{v_r}^{d_r}, each formed on
 * its own (Section 2.2, the straightforward way).  nmul counts the complex
 * multiplications among variable values (not by c, not by d_s).
 */
static void mono_definition(const ctx_t *cx, int k, const int32_t *v, const uint8_t *d,
                            const double *c, double *term, double *part, int64_t *nmul) {
  int L = cx->L;
  double acc[8], pw[8], tmp[8];
  /* value */
  int have = 0;
  for (int s = 0; s < k; s++) {
    power_naive(cx, v[s], d[s], pw, nmul);
    if (!have) {
      memcpy(acc, pw, sizeof(double) * 2 * L);
      have = 1;
    } else {
      c_mul(L, acc, pw, acc);
      (*nmul)++;
    }
  }
  if (!have) c_one(L, acc);
  c_mul(L, c, acc, term);
  /* partials */
  for (int s = 0; s < k; s++) {
    have = 0;
    for (int r = 0; r < k; r++) {
      int e = (r == s) ? d[r] - 1 : d[r];
      if (e == 0) continue;
      power_naive(cx, v[r], e, pw, nmul);
      if (!have) {
        memcpy(acc, pw, sizeof(double) * 2 * L);
        have = 1;
      } else {
        c_mul(L, acc, pw, acc);
        (*nmul)++;
      }
    }
    if (!have) c_one(L, acc);
    c_mul(L, c, acc, tmp);
    c_scale_int(L, tmp, d[s], part + (int64_t)s * 2 * L);
  }
}

/*
 * Reverse mode for one monomial (Sections 2.1-2.3):
 *   common factor CF = prod_{s: d_s >= 2} x_{v_s}^{d_s - 1} from the power table;
 *   Speelpenning: forward products F_s = x_{v_1} ... x_{v_s}, value P = F_k,
 *     gradient G_s = F_{s-1} * (x_{v_{s+1}} ... x_{v_k}) with the backward
 *     product kept in one running location (3k-5 multiplications for k >= 2);
 *   a = c * CF, term = a * P, partial_s = d_s * (a * G_s).
 * pow_tab[(v * pmax + (p-1)) * 2L] holds x_v^p for p = 1..pmax.
 * nmul counts the Speelpenning multiplications only.
 */
static void mono_reverse(const ctx_t *cx, int k, const int32_t *v, const uint8_t *d,
                         const double *c, const double *pow_tab, int pmax, double *term,
                         double *part, double *F, int64_t *nmul) {
  int L = cx->L;
  const int64_t W = 2 * L;
  double cf[8], a[8], B[8], G[8], tmp[8];
  /* common factor, eq. 1 */
  int have = 0;
  for (int s = 0; s < k; s++) {
    if (d[s] < 2) continue;
    const double *tv = pow_tab + ((int64_t)v[s] * pmax + (d[s] - 2)) * W;
    if (!have) {
      memcpy(cf, tv, sizeof(double) * W);
      have = 1;
    } else {
      c_mul(L, cf, tv, cf);
    }
  }
  if (!have) c_one(L, cf);
  c_mul(L, c, cf, a);
  if (k == 0) {
    memcpy(term, a, sizeof(double) * W);
    return;
  }
  /* forward products F[s] = x_{v_0} ... x_{v_s} (0-based) */
  memcpy(F, xv(cx, v[0]), sizeof(double) * W);
  for (int s = 1; s < k; s++) {
    c_mul(L, F + (int64_t)(s - 1) * W, xv(cx, v[s]), F + (int64_t)s * W);
    (*nmul)++;
  }
  c_mul(L, a, F + (int64_t)(k - 1) * W, term);
  if (k == 1) {
    c_one(L, G);
    c_mul(L, a, G, tmp);
    c_scale_int(L, tmp, d[0], part);
    return;
  }
  /* last partial: product of all but the last variable */
  c_mul(L, a, F + (int64_t)(k - 2) * W, tmp);
  c_scale_int(L, tmp, d[k - 1], part + (int64_t)(k - 1) * W);
  /* running backward product B = x_{v_{s+1}} ... x_{v_{k-1}} */
  memcpy(B, xv(cx, v[k - 1]), sizeof(double) * W);
  for (int s = k - 2; s >= 1; s--) {
    c_mul(L, F + (int64_t)(s - 1) * W, B, G);
    (*nmul)++;
    c_mul(L, a, G, tmp);
    c_scale_int(L, tmp, d[s], part + (int64_t)s * W);
    c_mul(L, B, xv(cx, v[s]), B);
    (*nmul)++;
  }
  /* first partial: the full backward product */
  c_mul(L, a, B, tmp);
  c_scale_int(L, tmp, d[0], part);
}

/*
 * Evaluate f and J for polynomials [row0, row1) at x.
 *   f[(i-row0) * 2L], J[((int64)v * ldJ + (i-row0)) * 2L] (column-major).
 *   J and f are overwritten (zero where no term contributes).
 *   mode 0 = definition, 1 = reverse.
 *   nmul_out (optional) receives the number of variable-product multiplications.
 */
int o_eval(int L, int mode, int32_t N, int32_t n, const int64_t *poly_ptr,
           const int64_t *mono_ptr, const int32_t *var, const uint8_t *exp,
           const double *coef, int coef_limbs, const double *x, int32_t row0, int32_t row1,
           double *f, double *J, int64_t ldJ, int nthreads, int64_t *nmul_out) {
  if (L != 1 && L != 2 && L != 4) return O_EINVAL;
  if (row0 < 0 || row1 > N || row0 > row1 || ldJ < row1 - row0) return O_EINVAL;
  const int64_t W = 2 * L;
  ctx_t cx = {L, coef_limbs, coef, x};
  int nr = row1 - row0;
  memset(f, 0, sizeof(double) * W * nr);
  if (J) memset(J, 0, sizeof(double) * W * (size_t)ldJ * n);

  /* power table x_v^p, p = 1..pmax, by repeated multiplication (Section 2.1) */
  int dmax = 1;
  for (int i = row0; i < row1; i++)
    for (int64_t t = poly_ptr[i]; t < poly_ptr[i + 1]; t++)
      for (int64_t o = mono_ptr[t]; o < mono_ptr[t + 1]; o++) {
        if (var[o] < 0 || var[o] >= n || exp[o] < 1) return O_EINVAL;
        if (exp[o] > dmax) dmax = exp[o];
      }
  int pmax = dmax > 1 ? dmax - 1 : 1;
  double *pow_tab = NULL;
  if (mode == 1) {
    pow_tab = (double *)malloc(sizeof(double) * W * (size_t)n * pmax);
    if (!pow_tab) return O_EINVAL;
    for (int v = 0; v < n; v++) {
      memcpy(pow_tab + ((int64_t)v * pmax) * W, xv(&cx, v), sizeof(double) * W);
      for (int p = 2; p <= pmax; p++)
        c_mul(L, pow_tab + ((int64_t)v * pmax + p - 2) * W, xv(&cx, v),
              pow_tab + ((int64_t)v * pmax + p - 1) * W);
    }
  }

  int64_t nmul_total = 0;
  int status = O_OK;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : nmul_total)
#endif
  for (int i = row0; i < row1; i++) {
    double *F = (double *)malloc(sizeof(double) * W * KMAXO);
    double *part = (double *)malloc(sizeof(double) * W * KMAXO);
    double c[8], term[8];
    double *fi = f + (int64_t)(i - row0) * W;
    for (int64_t t = poly_ptr[i]; t < poly_ptr[i + 1]; t++) {
      int k = (int)(mono_ptr[t + 1] - mono_ptr[t]);
      if (k > KMAXO) {
        status = O_EINVAL;
        continue;
      }
      const int32_t *vs = var + mono_ptr[t];
      const uint8_t *ds = exp + mono_ptr[t];
      load_coef(&cx, t, c);
      int64_t nm = 0;
      if (mode == 0)
        mono_definition(&cx, k, vs, ds, c, term, part, &nm);
      else
        mono_reverse(&cx, k, vs, ds, c, pow_tab, pmax, term, part, F, &nm);
      nmul_total += nm;
      /* term summation (Section 2.3), in monomial order */
      c_add(L, fi, term, fi);
      if (J)
        for (int s = 0; s < k; s++) {
          double *Jiv = J + ((int64_t)vs[s] * ldJ + (i - row0)) * W;
          c_add(L, Jiv, part + (int64_t)s * W, Jiv);
        }
    }
    free(F);
    free(part);
  }
  free(pow_tab);
  if (nmul_out) *nmul_out = nmul_total;
  return status;
}

/*
 * Speelpenning product of k values alone (Section 2.2): value and gradient
 * with the forward/backward scheme; returns the multiplication count.
 */
int64_t o_speelpenning(int L, int k, const double *xs, double *value, double *grad) {
  const int64_t W = 2 * L;
  double *F = (double *)malloc(sizeof(double) * W * (k > 0 ? k : 1));
  double B[8];
  int64_t nmul = 0;
  if (k == 0) {
    c_one(L, value);
    free(F);
    return 0;
  }
  memcpy(F, xs, sizeof(double) * W);
  for (int s = 1; s < k; s++) {
    c_mul(L, F + (s - 1) * W, xs + s * W, F + s * W);
    nmul++;
  }
  memcpy(value, F + (k - 1) * W, sizeof(double) * W);
  if (k == 1) {
    c_one(L, grad);
    free(F);
    return nmul;
  }
  memcpy(grad + (k - 1) * W, F + (k - 2) * W, sizeof(double) * W);
  memcpy(B, xs + (k - 1) * W, sizeof(double) * W);
  for (int s = k - 2; s >= 1; s--) {
    c_mul(L, F + (s - 1) * W, B, grad + s * W);
    nmul++;
    c_mul(L, B, xs + s * W, B);
    nmul++;
  }
  memcpy(grad, B, sizeof(double) * W);
  free(F);
  return nmul;
}

/* ---------------------------------------------------------------------- */
/* Modified Gram-Schmidt on [A b] and back substitution (Section 3)         */
/* ---------------------------------------------------------------------- */

/*
 * MGS on the m x ncols column-major matrix A (leading dimension lda), in
 * place, the figure "The modified Gram-Schmidt orthogonalization algorithm":
 *   for k: r_kk = sqrt(a_k^H a_k); q_k = a_k / r_kk;
 *          for j > k: r_kj = q_k^H a_j; a_j = a_j - r_kj q_k.
 * The last column is the right-hand side b of eq. 2: it is orthogonalized
 * against q_1..q_n (giving y = R[0:n, n]) and r_nn = z = ||b - Q y|| is
 * stored, but it is not normalized (q_{n+1} is not needed and z may be 0).
 * R (ncols x ncols, column-major, ldr) receives r_kj; below the diagonal 0.
 * Returns O_ESINGULAR when r_kk <= 2^(8 - 50 L) * ||a_k^(0)|| for k < ncols-1
 * (a rank test a few bits above the unit roundoff of precision L).
 */
int o_mgs(int L, int32_t m, int32_t ncols, double *A, int64_t lda, double *R, int32_t ldr,
          int nthreads) {
  if (L != 1 && L != 2 && L != 4) return O_EINVAL;
  const int64_t W = 2 * L;
  memset(R, 0, sizeof(double) * W * (size_t)ldr * ncols);
  double *nrm0 = (double *)malloc(sizeof(double) * (ncols > 0 ? ncols : 1));
  /* original column norms (double estimate) for the rank test */
  for (int j = 0; j < ncols; j++) {
    double s = 0.0;
    for (int i = 0; i < m; i++) {
      const double *a = A + ((int64_t)j * lda + i) * W;
      s += a[0] * a[0] + a[L] * a[L];
    }
    nrm0[j] = sqrt(s);
  }
  int status = O_OK;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  for (int k = 0; k < ncols; k++) {
    double *ak = A + (int64_t)k * lda * W;
    /* r_kk = sqrt(a_k^H a_k), sum in row order */
    double ss[4] = {0, 0, 0, 0}, t2[8];
    for (int i = 0; i < m; i++) {
      c_abs2(L, ak + i * W, t2);
      r_add(L, ss, t2, ss);
    }
    double rkk[4];
    r_sqrt(L, ss, rkk);
    double *Rkk = R + ((int64_t)k * ldr + k) * W;
    memcpy(Rkk, rkk, sizeof(double) * L);
    if (k == ncols - 1) break; /* z of eq. 2; b is not normalized */
    double thresh = ldexp(nrm0[k], 8 - 50 * L);
    if (!(rkk[0] > thresh)) {
      status = O_ESINGULAR;
      break;
    }
    /* q_k = a_k / r_kk */
    for (int i = 0; i < m; i++) c_div_real(L, ak + i * W, rkk, ak + i * W);
    /* right-looking update of the trailing columns */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int j = k + 1; j < ncols; j++) {
      double *aj = A + (int64_t)j * lda * W;
      double r[8], p[8];
      c_zero(L, r);
      for (int i = 0; i < m; i++) {
        c_conj_mul(L, ak + i * W, aj + i * W, p);
        c_add(L, r, p, r);
      }
      memcpy(R + ((int64_t)j * ldr + k) * W, r, sizeof(double) * W);
      for (int i = 0; i < m; i++) {
        c_mul(L, r, ak + i * W, p);
        c_sub(L, aj + i * W, p, aj + i * W);
      }
    }
  }
  free(nrm0);
  return status;
}

/*
 * Back substitution R[0:n,0:n] x = y with y = R[0:n, n] (Section 3, eq. 5 read
 * as the standard upper-triangular recurrence):
 *   x_l = (y_l - sum_{j=l+1}^{n-1} r_lj x_j) / r_ll, l = n-1 down to 0.
 */
int o_backsub(int L, int32_t n, const double *R, int32_t ldr, double *x) {
  if (L != 1 && L != 2 && L != 4) return O_EINVAL;
  const int64_t W = 2 * L;
  for (int l = n - 1; l >= 0; l--) {
    double acc[8], p[8];
    memcpy(acc, R + ((int64_t)n * ldr + l) * W, sizeof(double) * W);
    for (int j = l + 1; j < n; j++) {
      c_mul(L, R + ((int64_t)j * ldr + l) * W, x + (int64_t)j * W, p);
      c_sub(L, acc, p, acc);
    }
    const double *rll = R + ((int64_t)l * ldr + l) * W;
    int st = c_div_real(L, acc, rll, x + (int64_t)l * W);
    if (st) return st;
  }
  return O_OK;
}

/* x := x + dx componentwise (the Newton update of Section 4). */
int o_axpy_update(int L, int32_t n, double *x, const double *dx) {
  const int64_t W = 2 * L;
  for (int i = 0; i < n; i++) c_add(L, x + i * W, dx + i * W, x + i * W);
  return O_OK;
}

/*
 * Adjoint of a converged Gauss-Newton solve (the gradient of a real loss
 * with respect to the coefficients, by the implicit function theorem applied
 * to the Newton fixed point of Section 4; the paper stops at the forward
 * solve, so this is an extension).
 *
 * At a root x of f(x; c) = 0 with J of full column rank, a change dc of the
 * coefficients moves the root by dx = -J^+ (df/dc) dc, J^+ = R^-1 Q^H for
 * the factors J = QR of Section 3.  For a real loss with gradient
 * g = dL/dRe x + i dL/dIm x, the gradient with respect to c is
 * sum_j g_j conj(dx_j/dc) = -((J^+)^H g)_i conj(df_i/dc) for a coefficient c
 * of polynomial i, and df_i/dc_t = x^{a_t}.  Hence three steps:
 *   o_adjoint:    R^H w = g by forward substitution,
 *                 w_l = (g_l - sum_{j<l} conj(r_jl) w_j) / r_ll (r_ll real),
 *                 then lambda = Q w, lambda_i = sum_l q_il w_l (l ascending);
 *   o_monomials:  m_t = x^{a_t}, each power by repeated multiplication in
 *                 support order (the definition of eq. 1);
 *   o_coef_grad:  grad_t = -lambda_{i(t)} conj(m_t).
 * Q (m x n) and R (n x n, upper part read) are column-major as o_mgs leaves
 * them: the first n columns of the overwritten [J b] and of its R.
 */
int o_adjoint(int L, int32_t m, int32_t n, const double *Q, int64_t ldq, const double *R,
              int32_t ldr, const double *g, double *w, double *lam) {
  if (L != 1 && L != 2 && L != 4) return O_EINVAL;
  const int64_t W = 2 * L;
  for (int l = 0; l < n; l++) {
    double acc[8], p[8];
    memcpy(acc, g + (int64_t)l * W, sizeof(double) * W);
    for (int j = 0; j < l; j++) {
      c_conj_mul(L, R + ((int64_t)l * ldr + j) * W, w + (int64_t)j * W, p);
      c_sub(L, acc, p, acc);
    }
    int st = c_div_real(L, acc, R + ((int64_t)l * ldr + l) * W, w + (int64_t)l * W);
    if (st) return st;
  }
  for (int i = 0; i < m; i++) {
    double acc[8], p[8];
    c_zero(L, acc);
    for (int l = 0; l < n; l++) {
      c_mul(L, Q + ((int64_t)l * ldq + i) * W, w + (int64_t)l * W, p);
      c_add(L, acc, p, acc);
    }
    memcpy(lam + (int64_t)i * W, acc, sizeof(double) * W);
  }
  return O_OK;
}

int o_monomials(int L, int64_t T, const int64_t *mono_ptr, const int32_t *var,
                const uint8_t *exp, const double *x, double *out) {
  if (L != 1 && L != 2 && L != 4) return O_EINVAL;
  const int64_t W = 2 * L;
  for (int64_t t = 0; t < T; t++) {
    double acc[8];
    c_one(L, acc);
    for (int64_t o = mono_ptr[t]; o < mono_ptr[t + 1]; o++)
      for (int r = 0; r < exp[o]; r++) c_mul(L, acc, x + (int64_t)var[o] * W, acc);
    memcpy(out + t * W, acc, sizeof(double) * W);
  }
  return O_OK;
}

int o_coef_grad(int L, int32_t N, const int64_t *poly_ptr, const double *lam,
                const double *mono, double *grad) {
  if (L != 1 && L != 2 && L != 4) return O_EINVAL;
  const int64_t W = 2 * L;
  for (int i = 0; i < N; i++)
    for (int64_t t = poly_ptr[i]; t < poly_ptr[i + 1]; t++) {
      c_conj_mul(L, mono + t * W, lam + (int64_t)i * W, grad + t * W);
      for (int l = 0; l < W; l++) grad[t * W + l] = -grad[t * W + l];
    }
  return O_OK;
}

int o_version(void) { return 1; }
