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

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, k, o);
    k = other > k ? other : k;
  }
  return k;
}

// Radix-2 Stockham FFT of length H in shared memory, natural order in and out,
// unnormalised.  Called by H/2 threads of one group (j = 0..H/2-1); every thread of
// the block must call it (it synchronises the block after each stage).  tw holds
// exp(-2 pi i t / Nt) for t < Nt/2 and H divides Nt; twshift = log2(Nt / H).
// INV selects exp(+...).  Returns the buffer that holds the result.
template <bool INV>
__device__ __forceinline__ float2* stockham_fft(float2* a, float2* b, int H, int j,
                                                const float2* tw, int twshift) {
  const int half = H >> 1;
  for (int Ns = 1; Ns < H; Ns <<= 1) {
    const int k = j & (Ns - 1);
    float2 v0 = a[j];
    float2 v1 = a[j + half];
    float2 w = tw[(k * (H / (2 * Ns))) << twshift];
    if (INV) w.y = -w.y;
    v1 = cmul(v1, w);
    const int d = ((j - k) << 1) + k;
    b[d] = make_float2(v0.x + v1.x, v0.y + v1.y);
    b[d + Ns] = make_float2(v0.x - v1.x, v0.y - v1.y);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace srp
