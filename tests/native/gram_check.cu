// Test driver for the Gram matrix of CholeskyQR: the tensor-core form
// (launch_gram_tc) and the integer-pipe form (k_cq_gram) against an exact
// reference computed here on the CPU, and against each other.
//
// Built by tests/test_gpu_gram_tc.py from this file and the library's object
// files; prints one JSON line per case and exits non-zero if a check fails.
//   * integer entries (|v| <= 2^20) times power-of-two column scales: the
//     Gram entries are integers below 2^53 times powers of two, so the exact
//     value (128-bit integer sums on the CPU) is a double, and both GPU forms
//     must reproduce it bit for bit;
//   * Gaussian entries: the two GPU forms are each exact for the columns
//     rounded to 56 (tensor) or 62 (integer) bits at their scales, then
//     rounded once, so they agree to 2^-51 of ||a_i|| ||a_j||.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <random>
#include <vector>

#include "../../include/gn.h"

namespace gn {
__global__ void k_cq_gram(const double *A, int32_t N, int32_t nc, const double *sexp, double *G,
                          const int32_t *status);
bool gram_tc_available(int32_t N, int32_t nc);
size_t gram_tc_scratch_bytes(int32_t N, int32_t nc);
gn_status launch_gram_tc(int32_t N, int32_t nc, const double *A, const double *sexp, double *G, void *scratch,
                         int32_t *status, cudaStream_t st);
}  // namespace gn

// the column scales of both kernels: ||a_j|| < 2^(62 + s_j)
static double col_scale(const std::vector<double> &A, int N, int j) {
  double s = 0;
  for (int r = 0; r < N; r++)
    for (int p = 0; p < 2; p++) s += A[((size_t)j * N + r) * 2 + p] * A[((size_t)j * N + r) * 2 + p];
  int e;
  frexp(std::sqrt(s) * 1.0000001 + 1e-300, &e);
  return (double)(e - 62);
}

static int run_case(const char *name, int N, int nc, bool integer, unsigned seed) {
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  std::uniform_int_distribution<long long> ui(-(1LL << 20), 1LL << 20);
  std::vector<double> A((size_t)N * nc * 2);
  std::vector<int> cexp(nc);
  std::vector<long long> Ai(integer ? A.size() : 0);
  for (int j = 0; j < nc; j++) {
    cexp[j] = (j % 7) * 9 - 20;  // columns of different magnitudes
    for (int r = 0; r < N; r++)
      for (int p = 0; p < 2; p++) {
        const size_t at = ((size_t)j * N + r) * 2 + p;
        if (integer) {
          Ai[at] = ui(rng);
          A[at] = std::ldexp((double)Ai[at], cexp[j]);
        } else {
          A[at] = std::ldexp(nd(rng), cexp[j]);
        }
      }
  }
  std::vector<double> sexp(nc);
  for (int j = 0; j < nc; j++) sexp[j] = col_scale(A, N, j);
  const size_t gb = (size_t)nc * nc * 2 * sizeof(double);
  double *dA = nullptr, *dS = nullptr, *G1 = nullptr, *G2 = nullptr;
  int32_t *st = nullptr;
  void *scr = nullptr;
  cudaMalloc(&dA, A.size() * 8);
  cudaMalloc(&dS, nc * 8);
  cudaMalloc(&G1, gb);
  cudaMalloc(&G2, gb);
  cudaMalloc(&st, 8);
  cudaMalloc(&scr, gn::gram_tc_scratch_bytes(N, nc));
  cudaMemcpy(dA, A.data(), A.size() * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dS, sexp.data(), nc * 8, cudaMemcpyHostToDevice);
  cudaMemset(G1, 0, gb);
  cudaMemset(G2, 0, gb);
  cudaMemset(st, 0, 8);
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&e2);
  const int nb = (nc + 31) / 32;
  float t_int = 0, t_tc = 0;
  int launch_err = 0;
  for (int rep = 0; rep < 3; rep++) {
    cudaEventRecord(e0);
    gn::k_cq_gram<<<nb * (nb + 1) / 2, 256>>>(dA, N, nc, dS, G1, st);
    cudaEventRecord(e1);
    launch_err |= (int)gn::launch_gram_tc(N, nc, dA, dS, G2, scr, st, 0);
    cudaEventRecord(e2);
    cudaEventSynchronize(e2);
    cudaEventElapsedTime(&t_int, e0, e1);
    cudaEventElapsedTime(&t_tc, e1, e2);
  }
  const cudaError_t err = cudaDeviceSynchronize();
  int32_t hst = -1;
  cudaMemcpy(&hst, st, 4, cudaMemcpyDeviceToHost);
  std::vector<double> g1(gb / 8), g2(gb / 8);
  cudaMemcpy(g1.data(), G1, gb, cudaMemcpyDeviceToHost);
  cudaMemcpy(g2.data(), G2, gb, cudaMemcpyDeviceToHost);
  std::vector<double> nrm(nc);
  for (int j = 0; j < nc; j++) {
    double s = 0;
    for (int r = 0; r < N; r++)
      for (int p = 0; p < 2; p++) s += A[((size_t)j * N + r) * 2 + p] * A[((size_t)j * N + r) * 2 + p];
    nrm[j] = std::sqrt(s);
  }
  // the exact reference on every entry of small cases, on a sample of large ones
  const int every = (long long)nc * nc * N > 200000000LL ? 97 : 1;
  long long n_exact_tc = 0, n_exact_int = 0, checked = 0, entries = 0, differ = 0;
  double maxnorm = 0;
  for (int j = 0; j < nc; j++)
    for (int i = 0; i <= j; i++) {
      double ex[2] = {0, 0};
      const bool check = integer && ((long long)i * 7 + j) % every == 0;
      if (check) {
        __int128 re = 0, im = 0;
        for (int r = 0; r < N; r++) {
          const long long ar = Ai[((size_t)i * N + r) * 2], ai = Ai[((size_t)i * N + r) * 2 + 1];
          const long long br = Ai[((size_t)j * N + r) * 2], bi = Ai[((size_t)j * N + r) * 2 + 1];
          re += (__int128)ar * br + (__int128)ai * bi;
          im += (__int128)ar * bi - (__int128)ai * br;
        }
        // below 2^53 (N <= 4096, |v| <= 2^20): exact as doubles
        ex[0] = std::ldexp((double)(long long)re, cexp[i] + cexp[j]);
        ex[1] = std::ldexp((double)(long long)im, cexp[i] + cexp[j]);
      }
      for (int p = 0; p < 2; p++) {
        const double a = g1[((size_t)j * nc + i) * 2 + p], b = g2[((size_t)j * nc + i) * 2 + p];
        entries++;
        if (a != b) differ++;
        if (check) {
          checked++;
          n_exact_int += (a == ex[p]);
          n_exact_tc += (b == ex[p]);
        }
        maxnorm = std::fmax(maxnorm, std::fabs(a - b) / (nrm[i] * nrm[j]));
      }
    }
  const bool ok = err == cudaSuccess && hst == 0 && launch_err == 0 &&
                  (integer ? (checked > 0 && n_exact_tc == checked && n_exact_int == checked && differ == 0)
                           : maxnorm <= std::ldexp(1.0, -51));
  printf(
      "{\"case\": \"%s\", \"N\": %d, \"nc\": %d, \"integer\": %d, \"cuda\": %d, \"status\": %d, "
      "\"ms_int\": %.4f, \"ms_tc\": %.4f, \"entries\": %lld, \"checked\": %lld, \"exact_tc\": %lld, \"exact_int\": %lld, "
      "\"differ\": %lld, \"max_normwise\": %.3e, \"ok\": %d}\n",
      name, N, nc, integer ? 1 : 0, (int)err, hst, t_int, t_tc, entries, checked, n_exact_tc, n_exact_int, differ, maxnorm,
      ok ? 1 : 0);
  fflush(stdout);
  cudaFree(dA);
  cudaFree(dS);
  cudaFree(G1);
  cudaFree(G2);
  cudaFree(st);
  cudaFree(scr);
  return ok ? 0 : 1;
}

int main() {
  if (!gn::gram_tc_available(1536, 1025)) {
    printf("{\"case\": \"available\", \"ok\": 0}\n");
    return 1;
  }
  int bad = 0;
  bad |= run_case("int_200x70", 200, 70, true, 1);
  bad |= run_case("int_1536x1025", 1536, 1025, true, 2);   // the mixed-precision workload's shape
  bad |= run_case("gauss_1536x1025", 1536, 1025, false, 3);
  bad |= run_case("gauss_2048x300", 2048, 300, false, 4);  // the tensor form's row limit
  bad |= run_case("gauss_37x5", 37, 5, false, 5);          // one ragged tile
  bad |= run_case("int_1000x129", 1000, 129, true, 6);     // two tile columns, one nearly empty
  return bad;
}
