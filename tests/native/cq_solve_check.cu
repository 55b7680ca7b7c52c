// Test driver for the triangular solves of the mixed solver's CholeskyQR
// (cholqr.cu): the diagonal-block inverses (k_cq_binv) and the blocked solves
// on one cluster (launch_cq_solve), against substitution in double on the CPU.
//
// Built by tests/test_gpu_cq_solve.py from this file and the library's object
// files; prints one JSON line per case and exits non-zero if a check fails.
//   * The factor R^ (upper triangular, complex, real positive diagonal) is
//     stored as float-float values h + l, which are exact doubles; the CPU
//     solves with exactly those values.
//   * Step solve: R dx = y, R = R^ diag(2^(s_j + 62)), y = R^[0:n, n]
//     2^(s_n + 62): dx_j = z_j 2^(s_n - s_j) with R^ z = R^[0:n, n].
//   * Refinement solves: R^H w = c, then R dx = w: with c^_j = c_j
//     2^-(s_j + 62), (R^)^H w = c^, R^ z = w, dx_j = z_j 2^-(s_j + 62).
//   * The factors have kappa below 10 and float-float operations carry about
//     2^-47 each, so z must agree to 2^-40 normwise; the scales are undone
//     before comparing, since the s_j spread dx over many binades.  A
//     right-hand side near 1e-60 checks that the solves rescale it into the
//     float range.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "../../include/gn.h"

namespace gn {
__global__ void k_cq_binv(double *R, int32_t nc, int32_t n, const int32_t *status);
gn_status launch_cq_solve(bool refine, int32_t n, const double *R, const double *sexp, const double *c,
                          double *dx, int32_t *status, cudaStream_t st);
}  // namespace gn

using cd = std::complex<double>;

// a double as float-float, and the exact double that the pair represents
static double ff_round(double v, float &h, float &l) {
  h = (float)v;
  l = (float)(v - (double)h);
  return (double)h + (double)l;
}

static int run_case(const char *name, int n, bool refine, double cscale, unsigned seed) {
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> ud(-1.0, 1.0), dg(0.6, 1.0);
  std::uniform_int_distribution<int> se(-90, -40);
  const int nc = n + 1;
  std::vector<float> Rf((size_t)nc * nc * 4, 0.f);  // float4 per entry, column-major
  std::vector<cd> Rx((size_t)nc * nc, 0.0);         // the exact values, column-major
  const double off = 0.3 / std::sqrt((double)n);
  for (int j = 0; j <= n; j++)
    for (int i = 0; i <= std::min(j, n - 1); i++) {
      double re = i == j ? dg(rng) : off * ud(rng), im = i == j ? 0.0 : off * ud(rng);
      if (j == n) {  // the right-hand side column y^
        re = ud(rng);
        im = ud(rng);
      }
      float *f = &Rf[((size_t)j * nc + i) * 4];
      re = ff_round(re, f[0], f[1]);
      im = ff_round(im, f[2], f[3]);
      Rx[(size_t)j * nc + i] = cd(re, im);
    }
  std::vector<double> sexp(nc);
  for (int j = 0; j <= n; j++) sexp[j] = (double)se(rng);
  std::vector<cd> c(n);
  for (int j = 0; j < n; j++) c[j] = cd(ud(rng), ud(rng)) * cscale;
  // CPU reference in the z domain
  auto r = [&](int i, int j) { return Rx[(size_t)j * nc + i]; };
  std::vector<cd> b(n), z(n);
  if (refine) {
    std::vector<cd> w(n);
    for (int j = 0; j < n; j++) b[j] = std::ldexp(1.0, -((int)sexp[j] + 62)) * c[j];
    for (int i = 0; i < n; i++) {  // (R^)^H w = b, forward
      cd s = b[i];
      for (int l = 0; l < i; l++) s -= std::conj(r(l, i)) * w[l];
      w[i] = s / r(i, i).real();
    }
    b = w;
  } else {
    for (int i = 0; i < n; i++) b[i] = r(i, n);
  }
  for (int i = n - 1; i >= 0; i--) {  // R^ z = b, backward
    cd s = b[i];
    for (int l = i + 1; l < n; l++) s -= r(i, l) * z[l];
    z[i] = s / r(i, i).real();
  }
  double *dR = nullptr, *dS = nullptr, *dC = nullptr, *dX = nullptr;
  int32_t *dst = nullptr;
  cudaMalloc(&dR, Rf.size() * sizeof(float));
  cudaMalloc(&dS, nc * sizeof(double));
  cudaMalloc(&dC, 2 * (size_t)n * sizeof(double));
  cudaMalloc(&dX, 2 * (size_t)n * sizeof(double));
  cudaMalloc(&dst, 2 * sizeof(int32_t));
  cudaMemcpy(dR, Rf.data(), Rf.size() * sizeof(float), cudaMemcpyHostToDevice);
  cudaMemcpy(dS, sexp.data(), nc * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemcpy(dC, c.data(), 2 * (size_t)n * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(dX, 0, 2 * (size_t)n * sizeof(double));
  cudaMemset(dst, 0, 2 * sizeof(int32_t));
  gn::k_cq_binv<<<(unsigned)((n + 31) / 32), 1024>>>(dR, nc, n, dst);
  const gn_status le = gn::launch_cq_solve(refine, n, dR, dS, refine ? dC : nullptr, dX, dst, 0);
  const cudaError_t err = cudaDeviceSynchronize();
  int32_t hst = -1;
  cudaMemcpy(&hst, dst, sizeof(int32_t), cudaMemcpyDeviceToHost);
  std::vector<cd> dx(n);
  cudaMemcpy(dx.data(), dX, 2 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost);
  double num = 0.0, den = 0.0;
  for (int j = 0; j < n; j++) {
    // back to the z domain
    const int sh = refine ? (int)sexp[j] + 62 : (int)sexp[j] - (int)sexp[n];
    const cd zg = std::ldexp(1.0, sh) * dx[j];
    num = std::fmax(num, std::abs(zg - z[j]));
    den = std::fmax(den, std::abs(z[j]));
  }
  const double rel = den > 0.0 ? num / den : num;
  const bool ok = err == cudaSuccess && le == GN_OK && hst == GN_OK && rel <= std::ldexp(1.0, -40);
  printf("{\"case\": \"%s\", \"n\": %d, \"refine\": %d, \"cuda\": %d, \"launch\": %d, \"status\": %d, "
         "\"rel_err\": %.3e, \"ok\": %d}\n",
         name, n, refine ? 1 : 0, (int)err, (int)le, hst, rel, ok ? 1 : 0);
  fflush(stdout);
  cudaFree(dR);
  cudaFree(dS);
  cudaFree(dC);
  cudaFree(dX);
  cudaFree(dst);
  return ok ? 0 : 1;
}

int main() {
  int bad = 0;
  bad |= run_case("step_32", 32, false, 1.0, 11);           // one block
  bad |= run_case("step_77", 77, false, 1.0, 12);           // three blocks, the last ragged
  bad |= run_case("step_300", 300, false, 1.0, 13);         // ten blocks: two CTAs own two
  bad |= run_case("step_1024", 1024, false, 1.0, 14);       // the largest: four blocks per CTA
  bad |= run_case("refine_77", 77, true, 1.0, 15);
  bad |= run_case("refine_1024", 1024, true, 1.0, 16);
  bad |= run_case("refine_1024_tiny", 1024, true, 1e-60, 17);  // far below the float range
  bad |= run_case("refine_545", 545, true, 1e-30, 18);         // 18 blocks, the last one row
  return bad;
}
