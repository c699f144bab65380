// Test helper: evaluates cuRAND's public Philox4x32-10 block function on
// counters and keys read from stdin and prints the outputs, so that a test
// can compare the CPU oracle's Philox with the library's.
#include <cstdio>
#include <vector>

#include <curand_kernel.h>

__global__ void philox_blocks(const uint4 *ctr, const uint2 *key, uint4 *out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

int main() {
  int n = 0;
  if (scanf("%d", &n) != 1 || n <= 0 || n > (1 << 20)) return 2;
  std::vector<uint4> c(n), o(n);
  std::vector<uint2> k(n);
  for (int i = 0; i < n; ++i)
    if (scanf("%u %u %u %u %u %u", &c[i].x, &c[i].y, &c[i].z, &c[i].w, &k[i].x, &k[i].y) != 6)
      return 2;
  uint4 *dc = nullptr, *dout = nullptr;
  uint2 *dk = nullptr;
  if (cudaMalloc(&dc, sizeof(uint4) * n) != cudaSuccess) return 3;
  if (cudaMalloc(&dout, sizeof(uint4) * n) != cudaSuccess) return 3;
  if (cudaMalloc(&dk, sizeof(uint2) * n) != cudaSuccess) return 3;
  cudaMemcpy(dc, c.data(), sizeof(uint4) * n, cudaMemcpyHostToDevice);
  cudaMemcpy(dk, k.data(), sizeof(uint2) * n, cudaMemcpyHostToDevice);
  philox_blocks<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
  if (cudaMemcpy(o.data(), dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost) != cudaSuccess) return 4;
  for (int i = 0; i < n; ++i) printf("%u %u %u %u\n", o[i].x, o[i].y, o[i].z, o[i].w);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return 0;
}
