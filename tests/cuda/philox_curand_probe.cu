// Test-only probe: raw Philox4x32-10 blocks from cuRAND's device API
// (curand_init + curand4 on curandStatePhilox4_32_10_t).  Used to pin the
// oracle's own Philox implementation against an independent library.
// Input on stdin: lines "seed subsequence offset"; output: 4 hex words per line.
#include <cstdio>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void probe(const unsigned long long *seed, const unsigned long long *sub,
                      const unsigned long long *off, uint4 *out, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed[i], sub[i], off[i], &st);
  out[i] = curand4(&st);
}

int main() {
  std::vector<unsigned long long> s, q, o;
  unsigned long long a, b, c;
  while (scanf("%llu %llu %llu", &a, &b, &c) == 3) { s.push_back(a); q.push_back(b); o.push_back(c); }
  int n = (int)s.size();
  if (n == 0) return 1;
  unsigned long long *ds, *dq, *dof;
  uint4 *dout;
  cudaMalloc(&ds, n * 8); cudaMalloc(&dq, n * 8); cudaMalloc(&dof, n * 8); cudaMalloc(&dout, n * 16);
  cudaMemcpy(ds, s.data(), n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dq, q.data(), n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(dof, o.data(), n * 8, cudaMemcpyHostToDevice);
  probe<<<(n + 127) / 128, 128>>>(ds, dq, dof, dout, n);
  std::vector<uint4> out(n);
  if (cudaMemcpy(out.data(), dout, n * 16, cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
  for (int i = 0; i < n; ++i) printf("%08x %08x %08x %08x\n", out[i].x, out[i].y, out[i].z, out[i].w);
  return 0;
}
