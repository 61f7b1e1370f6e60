// Device helpers shared by the libsrp kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace srp {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// a * conj(b)
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// 64-bit key whose unsigned order is (value, then lower index) -- the largest key is
// the maximum value with the lowest index among equals.  Key 0 means "no cell".
__device__ __forceinline__ unsigned long long argmax_key(float v, int i) {
  unsigned u = __float_as_uint(v);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return (static_cast<unsigned long long>(u) << 32) |
         static_cast<unsigned long long>(0xFFFFFFFFu - static_cast<unsigned>(i));
}

// Lets `kern` launch with up to the device's opt-in maximum of dynamic shared memory.  The
// value set is the same for every launch, so that host threads launching the kernel with
// different sizes at the same time (plans used concurrently) cannot undo each other's
// setting between the call and the launch.
template <typename Kernel>
inline cudaError_t allow_max_dynamic_smem(Kernel kern) {
  int dev = 0, most = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&most, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kern);  // the kernel's static shared memory counts too
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              most - static_cast<int>(fa.sharedSizeBytes));
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, k, o);
    k = other > k ? other : k;
  }
  return k;
}

}  // namespace srp
