// rates.cu — issue-rate probes of the GB300 pipes the library's design rests
// on: FP64 fused multiply-add (the pipe of the paper's double double and quad
// double arithmetic), FP64 tensor products (DMMA, mma.sync m8n8k4), 32-bit
// integer multiply-add (IMAD, the pipe of the integer-mantissa arithmetic)
// and FP32 fused multiply-add for scale.  A measurement tool for bench.py,
// not part of the Gauss-Newton path.
//
// Every kernel runs a fixed number of iterations of several independent
// dependency chains per thread (enough to cover each pipe's latency) on a
// grid of `blocks_per_sm` x SMs CTAs, and writes one value per thread so that
// nothing is optimised away.  Rates are lane-operations per second (one FMA
// or IMAD per lane; for DMMA, 512 floating-point operations per warp-wide
// m8n8k4 product), timed with CUDA events after one warm-up launch.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;

__global__ void __launch_bounds__(THREADS) k_fp64_fma(double *out, double b, double c, int iters) {
  double a[CHAINS];
#pragma unroll
  for (int q = 0; q < CHAINS; q++) a[q] = threadIdx.x + q;
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int q = 0; q < CHAINS; q++) a[q] = fma(a[q], b, c);
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < CHAINS; q++) s += a[q];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(THREADS) k_fp32_fma(double *out, float b, float c, int iters) {
  float a[CHAINS];
#pragma unroll
  for (int q = 0; q < CHAINS; q++) a[q] = threadIdx.x + q;
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int q = 0; q < CHAINS; q++) a[q] = fmaf(a[q], b, c);
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < CHAINS; q++) s += a[q];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(THREADS) k_imad(double *out, uint32_t b, uint32_t c, int iters) {
  uint32_t a[CHAINS];
#pragma unroll
  for (int q = 0; q < CHAINS; q++) a[q] = threadIdx.x + q;
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int q = 0; q < CHAINS; q++) a[q] = a[q] * b + c;
  uint32_t s = 0;
#pragma unroll
  for (int q = 0; q < CHAINS; q++) s ^= a[q];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

// one warp-wide 8x8x4 FP64 product per mma.sync, CHAINS / 2 independent
// accumulators per warp
__global__ void __launch_bounds__(THREADS) k_dmma(double *out, double av, double bv, int iters) {
  constexpr int ACC = CHAINS / 2;
  double d[ACC][2];
#pragma unroll
  for (int q = 0; q < ACC; q++) d[q][0] = d[q][1] = 0.0;
  const double a = av + threadIdx.x, b = bv - threadIdx.x;
  for (int i = 0; i < iters; i++)
#pragma unroll
    for (int q = 0; q < ACC; q++)
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
          : "+d"(d[q][0]), "+d"(d[q][1])
          : "d"(a), "d"(b));
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < ACC; q++) s += d[q][0] + d[q][1];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// which: 0 FP64 FMA, 1 DMMA, 2 IMAD, 3 FP32 FMA.  Writes the rate in
// G lane-operations/s (DMMA: GFLOP/s) and the kernel time in ms.  Returns 0,
// or a CUDA error code.
extern "C" int gn_probe_rate(int which, int blocks_per_sm, int iters, double *rate, double *ms) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  if (which < 0 || which > 3 || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1) return -1;
  const int blocks = sms * blocks_per_sm;
  double *out = nullptr;
  e = cudaMalloc((void **)&out, sizeof(double) * (size_t)blocks * THREADS);
  if (e != cudaSuccess) return (int)e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto launch = [&]() {
    switch (which) {
      case 0: k_fp64_fma<<<blocks, THREADS>>>(out, 0.999999, 1e-7, iters); break;
      case 1: k_dmma<<<blocks, THREADS>>>(out, 0.5, 0.25, iters); break;
      case 2: k_imad<<<blocks, THREADS>>>(out, 1664525u, 1013904223u, iters); break;
      case 3: k_fp32_fma<<<blocks, THREADS>>>(out, 0.999999f, 1e-7f, iters); break;
    }
  };
  launch();  // warm-up
  cudaEventRecord(a);
  launch();
  cudaEventRecord(b);
  e = cudaEventSynchronize(b);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return (int)e;
  const double threads = (double)blocks * THREADS;
  double ops;
  if (which == 1)
    ops = threads / 32.0 * (CHAINS / 2) * (double)iters * 512.0;  // warp-wide products x flops
  else
    ops = threads * CHAINS * (double)iters;
  *ms = t;
  *rate = ops / (t * 1e-3) / 1e9;
  return 0;
}
