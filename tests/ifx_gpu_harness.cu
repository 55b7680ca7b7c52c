// GPU harness for csrc/ifx.cuh (test support): the device forms of the
// multi-limb integer operations, one thread per case.  Reads lines
// "op K a_0..a_{K-1} b_0..b_{K-1}" (hex limbs, little-endian) and prints the
// result limbs in hex, in input order.  ops: umul (ix_umul, 2K limbs), mul
// (ix_mul_shift, K+1), sq (ix_square of a, 2K+1), rsqrt (ix_rsqrt_frac of a
// with the device's FP32 seed, K).
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../paper_1402_2626_gb300/csrc/ifx.cuh"

static int nout(int op, int K) {
  return op == 0 ? 2 * K : op == 1 ? K + 1 : op == 2 ? 2 * K + 1 : K;
}

template <int K>
__global__ void k_ops(int n, const int *op, const uint64_t *in, uint64_t *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const uint64_t *a = in + (size_t)c * 2 * K, *b = a + K;
  uint64_t *o = out + (size_t)c * (2 * K + 1);
  gn::fx<K> fa, fb;
  gn::ux<K> ua, ub;
  for (int i = 0; i < K; i++) {
    fa.w[i] = ua.w[i] = a[i];
    fb.w[i] = ub.w[i] = b[i];
  }
  if (op[c] == 0) {
    const gn::ux<2 * K> p = gn::ix_umul<K>(ua, ub);
    for (int i = 0; i < 2 * K; i++) o[i] = p.w[i];
  } else if (op[c] == 1) {
    const gn::fx<K + 1> p = gn::ix_mul_shift<K>(fa, fb);
    for (int i = 0; i < K + 1; i++) o[i] = p.w[i];
  } else if (op[c] == 2) {
    const gn::fx<2 * K + 1> p = gn::ix_square<K>(fa);
    for (int i = 0; i < 2 * K + 1; i++) o[i] = p.w[i];
  } else {
    const gn::ux<K> y = gn::ix_rsqrt_frac<K>(ua);
    for (int i = 0; i < K; i++) o[i] = y.w[i];
  }
}

template <int K>
static bool run(const std::vector<int> &op, const std::vector<uint64_t> &in, std::vector<uint64_t> &out) {
  const int n = (int)op.size();
  out.assign((size_t)n * (2 * K + 1), 0);
  if (n == 0) return true;
  int *d_op;
  uint64_t *d_in, *d_out;
  if (cudaMalloc(&d_op, sizeof(int) * n) || cudaMalloc(&d_in, sizeof(uint64_t) * in.size()) ||
      cudaMalloc(&d_out, sizeof(uint64_t) * out.size()))
    return false;
  cudaMemcpy(d_op, op.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
  cudaMemcpy(d_in, in.data(), sizeof(uint64_t) * in.size(), cudaMemcpyHostToDevice);
  k_ops<K><<<(n + 127) / 128, 128>>>(n, d_op, d_in, d_out);
  const bool ok = cudaMemcpy(out.data(), d_out, sizeof(uint64_t) * out.size(), cudaMemcpyDeviceToHost) ==
                  cudaSuccess;
  cudaFree(d_op);
  cudaFree(d_in);
  cudaFree(d_out);
  return ok;
}

int main() {
  const char *names[] = {"umul", "mul", "sq", "rsqrt"};
  std::vector<int> ops[5], order_k, order_i;
  std::vector<uint64_t> ins[5];
  char name[16];
  int K;
  while (scanf("%15s %d", name, &K) == 2) {
    if (K != 1 && K != 2 && K != 4) return 2;
    int op = -1;
    for (int q = 0; q < 4; q++)
      if (!strcmp(name, names[q])) op = q;
    if (op < 0) return 2;
    for (int i = 0; i < 2 * K; i++) {
      unsigned long long v;
      if (scanf("%llx", &v) != 1) return 2;
      ins[K].push_back(v);
    }
    order_k.push_back(K);
    order_i.push_back((int)ops[K].size());
    ops[K].push_back(op);
  }
  std::vector<uint64_t> outs[5];
  if (!run<1>(ops[1], ins[1], outs[1]) || !run<2>(ops[2], ins[2], outs[2]) ||
      !run<4>(ops[4], ins[4], outs[4])) {
    fprintf(stderr, "CUDA error\n");
    return 1;
  }
  for (size_t c = 0; c < order_k.size(); c++) {
    const int k = order_k[c], i = order_i[c];
    const uint64_t *o = outs[k].data() + (size_t)i * (2 * k + 1);
    for (int w = 0; w < nout(ops[k][i], k); w++) printf("%llx ", (unsigned long long)o[w]);
    printf("\n");
  }
  return 0;
}
