// Device harness: the warp-cooperative capsule minimizer against the
// sequential one, both compiled for the GPU, on the same inputs.  Built by
// tests/test_gpu_capsule_warp.py with nvcc.
#include <cuda_runtime.h>

#include "twa_math.cuh"

using namespace twa;

namespace {

// One warp per item; inputs are 11 floats: a, b, c0, c1, wl, wh, r.
__global__ void compare_kernel(const float* in, int n, float* seq, float* war) {
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (item >= n) return;  // warp-uniform
  const float* q = in + (size_t)item * 11;
  const float2 a = mk(q[0], q[1]), b = mk(q[2], q[3]), c0 = mk(q[4], q[5]), c1 = mk(q[6], q[7]);
  float2 wl, wh;
  capsule_prox_free_warp(a, b, q[8], q[9], c0, c1, q[10], wl, wh);
  if ((threadIdx.x & 31) == 0) {
    float2 vl, vh;
    capsule_prox_free(a, b, q[8], q[9], c0, c1, q[10], vl, vh);
    float* s = seq + (size_t)item * 4;
    float* w = war + (size_t)item * 4;
    s[0] = vl.x; s[1] = vl.y; s[2] = vh.x; s[3] = vh.y;
    w[0] = wl.x; w[1] = wl.y; w[2] = wh.x; w[3] = wh.y;
  }
}

}  // namespace

extern "C" int capsule_compare(const float* h_in, int n, float* h_seq, float* h_war) {
  float *in = nullptr, *seq = nullptr, *war = nullptr;
  cudaError_t e = cudaMalloc(&in, (size_t)n * 11 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&seq, (size_t)n * 4 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&war, (size_t)n * 4 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(in, h_in, (size_t)n * 11 * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    compare_kernel<<<(n + 3) / 4, 128>>>(in, n, seq, war);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h_seq, seq, (size_t)n * 4 * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h_war, war, (size_t)n * 4 * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(in);
  cudaFree(seq);
  cudaFree(war);
  return (int)e;
}
