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

// Table lookup of exp(-+2 pi i u / Nt) for 0 <= u < 3 Nt / 4 (the table tw holds t < Nt/2 =
// S entries; beyond, exp(-2 pi i (u - S)/Nt) changes sign).
__device__ __forceinline__ float2 tw_lookup(const float2* tw, int u, int S) {
  if (u < S) return tw[u];
  const float2 w = tw[u - S];
  return make_float2(-w.x, -w.y);
}

// Radix-4 Stockham FFT of length H (a power of two >= 4) in shared memory, natural order in
// and out, unnormalised; one radix-2 stage first when log2 H is odd.  Called by H/4
// threads of one group (j = 0..H/4-1); every thread of the block must call it (it
// synchronises the block after each stage).  tw holds exp(-2 pi i t / Nt) for t < Nt/2,
// Nt = H << twshift.  Stage with sub-transform length Ns: inputs a[j + m H/4] (m = 0..3),
// twiddles w^m with w = exp(-2 pi i k / 4Ns), k = j mod Ns, outputs at (j - k) 4 + k + m Ns.
template <bool INV>
__device__ __forceinline__ float2* stockham_fft_r4(float2* a, float2* b, int H, int j,
                                                   const float2* tw, int twshift) {
  const int q = H >> 2;
  const int S = (H << twshift) >> 1;  // table entries
  int Ns = 1;
  if ((__ffs(H) - 1) & 1) {  // log2 H odd: radix-2 stage with Ns = 1 (all twiddles 1)
    for (int jj = j; jj < 2 * q; jj += q) {
      const float2 v0 = a[jj], v1 = a[jj + 2 * q];
      b[2 * jj] = make_float2(v0.x + v1.x, v0.y + v1.y);
      b[2 * jj + 1] = make_float2(v0.x - v1.x, v0.y - v1.y);
    }
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    Ns = 2;
  }
  for (; Ns < H; Ns <<= 2) {
    const int k = j & (Ns - 1);
    const float2 a0 = a[j];
    float2 a1 = a[j + q], a2 = a[j + 2 * q], a3 = a[j + 3 * q];
    const int t1 = (k * (H / (4 * Ns))) << twshift;
    float2 w1 = tw_lookup(tw, t1, S), w2 = tw_lookup(tw, 2 * t1, S), w3 = tw_lookup(tw, 3 * t1, S);
    if (INV) {
      w1.y = -w1.y;
      w2.y = -w2.y;
      w3.y = -w3.y;
    }
    a1 = cmul(a1, w1);
    a2 = cmul(a2, w2);
    a3 = cmul(a3, w3);
    const float2 s02 = make_float2(a0.x + a2.x, a0.y + a2.y), d02 = make_float2(a0.x - a2.x, a0.y - a2.y);
    const float2 s13 = make_float2(a1.x + a3.x, a1.y + a3.y), d13 = make_float2(a1.x - a3.x, a1.y - a3.y);
    // -i d13 (forward) or +i d13 (inverse)
    const float2 r13 = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
    const int d = ((j - k) << 2) + k;
    b[d] = make_float2(s02.x + s13.x, s02.y + s13.y);
    b[d + Ns] = make_float2(d02.x + r13.x, d02.y + r13.y);
    b[d + 2 * Ns] = make_float2(s02.x - s13.x, s02.y - s13.y);
    b[d + 3 * Ns] = make_float2(d02.x - r13.x, d02.y - r13.y);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace srp
