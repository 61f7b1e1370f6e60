// Interpolation stage of SLRI-SRP and SSPI-SRP, with the argmax (Eq. imax) fused.
//
//   SLRI (boxed Eq. z_circlr_computed):  u = Lambda_fat xi      (R x L, per frame)
//                                        z = Lambda_tall u      (J x R, per frame)
//   SSPI (boxed Eq. z_circsp_computed):  z_i = sum_{(c, v) in row i} v * xi[c]
#include "srp_internal.h"
#include "srp_device.cuh"

#include <cuda.h>

#include <cstdint>
#include <mutex>

namespace srp {

// ---------------------------------------------------------------------------------
// u[f][r] = sum_l fat[r][l] xi[f][l].  FB frames per block staged in shared memory;
// one warp per r, lanes stride over l, FB dot products share each fat load.
// ---------------------------------------------------------------------------------
template <int FB>
__global__ __launch_bounds__(256) void slri_fat_kernel(const float* __restrict__ xi,
                                                       const float* __restrict__ fat,
                                                       float* __restrict__ U, int F, int L,
                                                       int R) {
  extern __shared__ float xs[];  // [FB][L]
  const int f0 = blockIdx.x * FB;
  const int nf = min(FB, F - f0);
  for (int e = threadIdx.x; e < FB * L; e += blockDim.x) {
    const int fb = e / L;
    xs[e] = fb < nf ? xi[static_cast<size_t>(f0) * L + e] : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int r = warp; r < R; r += (blockDim.x >> 5)) {
    float acc[FB];
#pragma unroll
    for (int fb = 0; fb < FB; ++fb) acc[fb] = 0.f;
    const float* fr = fat + static_cast<size_t>(r) * L;
    for (int l = lane; l < L; l += 32) {
      const float a = __ldg(fr + l);
#pragma unroll
      for (int fb = 0; fb < FB; ++fb) acc[fb] = fmaf(a, xs[fb * L + l], acc[fb]);
    }
#pragma unroll
    for (int fb = 0; fb < FB; ++fb) {
      float v = acc[fb];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
      if (lane == 0 && fb < nf) U[static_cast<size_t>(f0 + fb) * R + r] = v;
    }
  }
}

cudaError_t launch_slri_fat(const float* xi, const float* fat, float* U, int F, int L, int R,
                            cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  const size_t budget = 160 * 1024;
  int fb = 8;
  while (fb > 1 && static_cast<size_t>(fb) * L * sizeof(float) > budget) fb >>= 1;
  const size_t smem = static_cast<size_t>(fb) * L * sizeof(float);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  const int grid = (F + fb - 1) / fb;
#define SRP_FAT(FBV)                                                                         \
  case FBV: {                                                                                \
    cudaError_t e = allow_max_dynamic_smem(slri_fat_kernel<FBV>);                            \
    if (e != cudaSuccess) return e;                                                          \
    slri_fat_kernel<FBV><<<grid, 256, smem, s>>>(xi, fat, U, F, L, R);                       \
    break;                                                                                   \
  }
  switch (fb) {
    SRP_FAT(8)
    SRP_FAT(4)
    SRP_FAT(2)
    SRP_FAT(1)
    default:
      return cudaErrorInvalidValue;
  }
#undef SRP_FAT
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// z[f][i] = sum_r tall[i][r] u[f][r].  Each thread keeps the R coefficients of CPT
// cells (cell = base + c*256 + tid, so stores are coalesced) in registers and walks
// FB frames whose u rows sit in shared memory (broadcast reads).  The argmax of each
// frame is reduced per warp, then per block, then merged with one atomicMax.
// ---------------------------------------------------------------------------------
template <int R, int CPT>
__device__ __forceinline__ void slri_tall_body(const float* __restrict__ U,
                                               const float* __restrict__ tall,
                                               float* __restrict__ Z,
                                               unsigned long long* __restrict__ keys, int F,
                                               int J, int FB, int bx, int by) {
  extern __shared__ float4 sm4[];
  float* Us = reinterpret_cast<float*>(sm4);                                  // [FB][R]
  unsigned long long* red = reinterpret_cast<unsigned long long*>(Us + FB * R);  // [8][FB]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ibase = bx * (256 * CPT);
  const int f0 = by * FB;
  const int nf = min(FB, F - f0);
  for (int e = tid; e < nf * R; e += 256) Us[e] = U[static_cast<size_t>(f0) * R + e];
  float t[CPT][R];
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int i = ibase + c * 256 + tid;
    if (i < J) {
      const float4* src = reinterpret_cast<const float4*>(tall + static_cast<size_t>(i) * R);
#pragma unroll
      for (int r4 = 0; r4 < R / 4; ++r4) {
        const float4 v = __ldg(src + r4);
        t[c][4 * r4] = v.x; t[c][4 * r4 + 1] = v.y; t[c][4 * r4 + 2] = v.z; t[c][4 * r4 + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) t[c][r] = 0.f;
    }
  }
  __syncthreads();
  for (int fb = 0; fb < nf; ++fb) {
    const float4* u4 = reinterpret_cast<const float4*>(Us + fb * R);
    float z[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) z[c] = 0.f;
#pragma unroll
    for (int r4 = 0; r4 < R / 4; ++r4) {
      const float4 u = u4[r4];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        z[c] = fmaf(t[c][4 * r4], u.x, z[c]);
        z[c] = fmaf(t[c][4 * r4 + 1], u.y, z[c]);
        z[c] = fmaf(t[c][4 * r4 + 2], u.z, z[c]);
        z[c] = fmaf(t[c][4 * r4 + 3], u.w, z[c]);
      }
    }
    float* zr = Z + static_cast<size_t>(f0 + fb) * J;
    float bv = -INFINITY;
    int bi = -1;
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
      const int i = ibase + c * 256 + tid;
      if (i < J) {
        zr[i] = z[c];
        if (bi < 0 || z[c] > bv) { bv = z[c]; bi = i; }
      }
    }
    unsigned long long best = bi >= 0 ? argmax_key(bv, bi) : 0ull;
    best = warp_max_u64(best);
    if (lane == 0) red[warp * FB + fb] = best;
  }
  __syncthreads();
  for (int fb = tid; fb < nf; fb += 256) {
    unsigned long long b = 0ull;
#pragma unroll
    for (int w = 0; w < 8; ++w) b = red[w * FB + fb] > b ? red[w * FB + fb] : b;
    if (b) atomicMax(keys + f0 + fb, b);
  }
}

template <int R, int CPT>
__global__ __launch_bounds__(256) void slri_tall_kernel(const float* __restrict__ U,
                                                        const float* __restrict__ tall,
                                                        float* __restrict__ Z,
                                                        unsigned long long* __restrict__ keys,
                                                        int F, int J, int FB) {
  slri_tall_body<R, CPT>(U, tall, Z, keys, F, J, FB, blockIdx.x, blockIdx.y);
}

// Grouped (serving): items (session, cell block, frame block of 64), walked by the CTAs.
template <int R, int CPT>
__global__ __launch_bounds__(256) void slri_tall_group_kernel(const GroupInterp* __restrict__ g,
                                                              const int4* __restrict__ items,
                                                              const int* __restrict__ count) {
  const int n = *count;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int4 it = items[i];
    const GroupInterp e = g[it.x];
    slri_tall_body<R, CPT>(e.in, e.tall, e.Z, e.keys, e.F, e.J, 64, it.y, it.z);
    __syncthreads();  // the next item reuses the shared memory
  }
}

template <int R, int CPT>
static cudaError_t run_tall_group(const GroupInterp* g, const int4* items, const int* count,
                                  int grid, cudaStream_t s) {
  const size_t smem = sizeof(float) * 64 * R + sizeof(unsigned long long) * 8 * 64;
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_dynamic_smem(slri_tall_group_kernel<R, CPT>);
    if (e != cudaSuccess) return e;
  }
  slri_tall_group_kernel<R, CPT><<<grid, 256, smem, s>>>(g, items, count);
  return cudaGetLastError();
}

int slri_tall_cells_per_block(int Rp) { return 256 * (Rp <= 16 ? 4 : Rp <= 32 ? 2 : 1); }

cudaError_t launch_slri_tall_group(const GroupInterp* g, const int4* items, const int* count,
                                   int grid, int Rp, cudaStream_t s) {
  if (grid < 1) return cudaErrorInvalidValue;
  switch (Rp) {  // the cells per thread of launch_slri_tall
    case 8: return run_tall_group<8, 4>(g, items, count, grid, s);
    case 16: return run_tall_group<16, 4>(g, items, count, grid, s);
    case 24: return run_tall_group<24, 2>(g, items, count, grid, s);
    case 32: return run_tall_group<32, 2>(g, items, count, grid, s);
    case 40: return run_tall_group<40, 1>(g, items, count, grid, s);
    case 48: return run_tall_group<48, 1>(g, items, count, grid, s);
    case 56: return run_tall_group<56, 1>(g, items, count, grid, s);
    case 64: return run_tall_group<64, 1>(g, items, count, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int R, int CPT>
static cudaError_t run_tall(const float* U, const float* tall, float* Z, unsigned long long* keys,
                            int F, int J, cudaStream_t s) {
  const int FB = 64;
  const size_t smem = sizeof(float) * FB * R + sizeof(unsigned long long) * 8 * FB;
  dim3 grid((J + 256 * CPT - 1) / (256 * CPT), (F + FB - 1) / FB);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_max_dynamic_smem(slri_tall_kernel<R, CPT>);
    if (e != cudaSuccess) return e;
  }
  slri_tall_kernel<R, CPT><<<grid, 256, smem, s>>>(U, tall, Z, keys, F, J, FB);
  return cudaGetLastError();
}

cudaError_t launch_slri_tall(const float* U, const float* tall, float* Z,
                             unsigned long long* keys, int F, int J, int R, cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  switch (R) {  // R is the padded rank (a multiple of 8, <= 64)
    case 8: return run_tall<8, 4>(U, tall, Z, keys, F, J, s);
    case 16: return run_tall<16, 4>(U, tall, Z, keys, F, J, s);
    case 24: return run_tall<24, 2>(U, tall, Z, keys, F, J, s);
    case 32: return run_tall<32, 2>(U, tall, Z, keys, F, J, s);
    case 40: return run_tall<40, 1>(U, tall, Z, keys, F, J, s);
    case 48: return run_tall<48, 1>(U, tall, Z, keys, F, J, s);
    case 56: return run_tall<56, 1>(U, tall, Z, keys, F, J, s);
    case 64: return run_tall<64, 1>(U, tall, Z, keys, F, J, s);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------------
// SSPI gather.  A block stages xi of FB = 32*FPL frames transposed in shared memory
// ([L][FB+1], lanes read consecutive frames), then walks row blocks of 64 cells: one
// warp per row, taps read 32 at a time (coalesced) and broadcast by shuffle, FPL
// frames per lane.  Row results go through a shared-memory tile so the map rows are
// written coalesced and the argmax is reduced per frame.
// ---------------------------------------------------------------------------------
template <int FPL>
__device__ __forceinline__ void sspi_body(const float* __restrict__ xi,
                                          const long long* __restrict__ row_ptr,
                                          const int2* __restrict__ taps, float* __restrict__ Z,
                                          unsigned long long* __restrict__ keys, int F, int J,
                                          int L, int fx, int rb_begin, int rb_end, int rb_step) {
  constexpr int FB = 32 * FPL, RB = 64, XS = FB + 1, OS = RB + 1;
  extern __shared__ float sm[];
  float* xs = sm;            // [L][XS]
  float* os = sm + L * XS;   // [FB][OS]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int f0 = fx * FB;
  const int nf = min(FB, F - f0);
  for (int e = tid; e < FB * L; e += 256) {
    const int fb = e / L, l = e - fb * L;
    xs[l * XS + fb] = fb < nf ? xi[static_cast<size_t>(f0 + fb) * L + l] : 0.f;
  }
  __syncthreads();
  for (int rb = rb_begin; rb < rb_end; rb += rb_step) {
    const int i0 = rb * RB;
    for (int rr = warp; rr < RB; rr += 8) {
      const int i = i0 + rr;
      float acc[FPL];
#pragma unroll
      for (int q = 0; q < FPL; ++q) acc[q] = 0.f;
      if (i < J) {
        const long long s = row_ptr[i], e = row_ptr[i + 1];
        for (long long b = s; b < e; b += 32) {
          const int2 tp = (b + lane < e) ? __ldg(taps + b + lane) : make_int2(0, 0);
          const int cnt = static_cast<int>(min(32ll, e - b));
          for (int t = 0; t < cnt; ++t) {
            const int c = __shfl_sync(0xFFFFFFFFu, tp.x, t);
            const float v = __int_as_float(__shfl_sync(0xFFFFFFFFu, tp.y, t));
            const float* xr = xs + c * XS + lane;
#pragma unroll
            for (int q = 0; q < FPL; ++q) acc[q] = fmaf(v, xr[32 * q], acc[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < FPL; ++q) os[(lane + 32 * q) * OS + rr] = acc[q];
    }
    __syncthreads();
    for (int fb = warp; fb < nf; fb += 8) {
      unsigned long long best = 0ull;
      float* zr = Z + static_cast<size_t>(f0 + fb) * J;
      for (int rr = lane; rr < RB; rr += 32) {
        const int i = i0 + rr;
        if (i < J) {
          const float v = os[fb * OS + rr];
          zr[i] = v;
          const unsigned long long k = argmax_key(v, i);
          best = k > best ? k : best;
        }
      }
      best = warp_max_u64(best);
      if (lane == 0 && best) atomicMax(keys + f0 + fb, best);
    }
    __syncthreads();
  }
}

template <int FPL>
__global__ __launch_bounds__(256) void sspi_kernel(const float* __restrict__ xi,
                                                   const long long* __restrict__ row_ptr,
                                                   const int2* __restrict__ taps,
                                                   float* __restrict__ Z,
                                                   unsigned long long* __restrict__ keys, int F,
                                                   int J, int L, int nrb) {
  sspi_body<FPL>(xi, row_ptr, taps, Z, keys, F, J, L, blockIdx.x, blockIdx.y, nrb, gridDim.y);
}

// Grouped (serving): items (session, frame group, first row block, end row block).
template <int FPL>
__global__ __launch_bounds__(256) void sspi_group_kernel(const GroupInterp* __restrict__ g,
                                                         const int4* __restrict__ items,
                                                         const int* __restrict__ count) {
  const int n = *count;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int4 it = items[i];
    const GroupInterp e = g[it.x];
    sspi_body<FPL>(e.in, e.row_ptr, e.taps, e.Z, e.keys, e.F, e.J, e.L, it.y, it.z, it.w, 1);
    __syncthreads();  // the next item restages the shared memory
  }
}

template <int FPL>
static size_t sspi_smem(int L) {
  return sizeof(float) * (static_cast<size_t>(L) * (32 * FPL + 1) + 32 * FPL * 65);
}

cudaError_t launch_sspi(const float* xi, const long long* row_ptr, const int2* taps, float* Z,
                        unsigned long long* keys, int F, int J, int L, int num_sms,
                        cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  const int nrb = (J + 63) / 64;
  const size_t lim2 = 110 * 1024, lim1 = 220 * 1024;
  if (sspi_smem<2>(L) <= lim2) {
    const size_t smem = sspi_smem<2>(L);
    const int fx = (F + 63) / 64;
    int gy = (2 * num_sms * 4 + fx - 1) / fx;
    gy = max(1, min(gy, nrb));
    cudaError_t e = allow_max_dynamic_smem(sspi_kernel<2>);
    if (e != cudaSuccess) return e;
    sspi_kernel<2><<<dim3(fx, gy), 256, smem, s>>>(xi, row_ptr, taps, Z, keys, F, J, L, nrb);
  } else if (sspi_smem<1>(L) <= lim1) {
    const size_t smem = sspi_smem<1>(L);
    const int fx = (F + 31) / 32;
    int gy = (num_sms * 4 + fx - 1) / fx;
    gy = max(1, min(gy, nrb));
    cudaError_t e = allow_max_dynamic_smem(sspi_kernel<1>);
    if (e != cudaSuccess) return e;
    sspi_kernel<1><<<dim3(fx, gy), 256, smem, s>>>(xi, row_ptr, taps, Z, keys, F, J, L, nrb);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// SSPI gather for long sample vectors.  Row block b (64 consecutive cells) stages only
// the columns its taps use (blk_cols[blk_ptr[b]..blk_ptr[b+1]), sorted; taps carry the
// column's position in that list) for FB frames, transposed in shared memory
// ([U][FB+1]).  One warp per row: lanes take the row's taps 32 at a time with FB
// accumulators each, then a halving reduction leaves lane l with the row's value for
// frame l >> (5 - log2 FB).  Results go through a shared-memory tile as in sspi_kernel.
// ---------------------------------------------------------------------------------
template <int FB>
__device__ __forceinline__ void halving_reduce(float (&acc)[FB], int lane) {
  int n = FB;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    if (n > 1) {
      n >>= 1;
      const bool upper = (lane & off) != 0;
#pragma unroll
      for (int j = 0; j < FB / 2; ++j) {
        if (j < n) {
          const float send = upper ? acc[j] : acc[j + n];
          const float keep = upper ? acc[j + n] : acc[j];
          acc[j] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, off);
        }
      }
    } else {
      acc[0] += __shfl_xor_sync(0xFFFFFFFFu, acc[0], off);
    }
  }
}

template <>
__device__ __forceinline__ void halving_reduce<1>(float (&acc)[1], int) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) acc[0] += __shfl_xor_sync(0xFFFFFFFFu, acc[0], off);
}

template <int FB>
__global__ __launch_bounds__(256) void sspi_band_kernel(
    const float* __restrict__ xi, const long long* __restrict__ row_ptr,
    const int2* __restrict__ taps, const long long* __restrict__ blk_ptr,
    const int* __restrict__ blk_cols, float* __restrict__ Z, unsigned long long* __restrict__ keys,
    int F, int J, int L) {
  constexpr int RB = 64, XS = FB + 1, OS = RB + 1;
  constexpr int LOG = FB == 32 ? 5 : FB == 16 ? 4 : FB == 8 ? 3 : FB == 4 ? 2 : FB == 2 ? 1 : 0;
  extern __shared__ float sm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b = blockIdx.y;
  const long long c0 = blk_ptr[b];
  const int U = static_cast<int>(blk_ptr[b + 1] - c0);
  float* xs = sm;                                 // [U][XS]
  float* os = sm + static_cast<size_t>(U) * XS;   // [FB][OS]
  const int f0 = blockIdx.x * FB;
  const int nf = min(FB, F - f0);
  for (int e = tid; e < U * FB; e += 256) {
    const int fb = e / U, u = e - fb * U;
    xs[u * XS + fb] = fb < nf ? xi[static_cast<size_t>(f0 + fb) * L + blk_cols[c0 + u]] : 0.f;
  }
  __syncthreads();
  const int i0 = b * RB;
  for (int rr = warp; rr < RB; rr += 8) {
    const int i = i0 + rr;
    float acc[FB];
#pragma unroll
    for (int q = 0; q < FB; ++q) acc[q] = 0.f;
    if (i < J) {
      const long long e = row_ptr[i + 1];
      for (long long t = row_ptr[i] + lane; t < e; t += 32) {
        const int2 tp = __ldg(taps + t);
        const float v = __int_as_float(tp.y);
        const float* xr = xs + tp.x * XS;
#pragma unroll
        for (int q = 0; q < FB; ++q) acc[q] = fmaf(v, xr[q], acc[q]);
      }
    }
    halving_reduce<FB>(acc, lane);
    if ((lane & ((32 >> LOG) - 1)) == 0) os[(lane >> (5 - LOG)) * OS + rr] = acc[0];
  }
  __syncthreads();
  for (int fb = warp; fb < nf; fb += 8) {
    unsigned long long best = 0ull;
    float* zr = Z + static_cast<size_t>(f0 + fb) * J;
    for (int rr = lane; rr < RB; rr += 32) {
      const int i = i0 + rr;
      if (i < J) {
        const float v = os[fb * OS + rr];
        zr[i] = v;
        const unsigned long long k = argmax_key(v, i);
        best = k > best ? k : best;
      }
    }
    best = warp_max_u64(best);
    if (lane == 0 && best) atomicMax(keys + f0 + fb, best);
  }
}

size_t sspi_band_smem(int U, int FB) {
  return sizeof(float) * (static_cast<size_t>(U) * (FB + 1) + static_cast<size_t>(FB) * 65);
}

bool sspi_full_fits(int L) { return sspi_smem<1>(L) <= 220 * 1024; }

int sspi_group_frames(int Lmax) { return sspi_smem<2>(Lmax) <= 110 * 1024 ? 64 : 32; }

cudaError_t launch_sspi_group(const GroupInterp* g, const int4* items, const int* count, int grid,
                              int Lmax, cudaStream_t s) {
  if (grid < 1 || !sspi_full_fits(Lmax)) return cudaErrorInvalidValue;
  if (sspi_group_frames(Lmax) == 64) {
    const size_t smem = sspi_smem<2>(Lmax);
    cudaError_t e = allow_max_dynamic_smem(sspi_group_kernel<2>);
    if (e != cudaSuccess) return e;
    sspi_group_kernel<2><<<grid, 256, smem, s>>>(g, items, count);
  } else {
    const size_t smem = sspi_smem<1>(Lmax);
    cudaError_t e = allow_max_dynamic_smem(sspi_group_kernel<1>);
    if (e != cudaSuccess) return e;
    sspi_group_kernel<1><<<grid, 256, smem, s>>>(g, items, count);
  }
  return cudaGetLastError();
}

cudaError_t launch_sspi_band(const float* xi, const long long* row_ptr, const int2* taps,
                             const long long* blk_ptr, const int* blk_cols, int umax, int FB,
                             float* Z, unsigned long long* keys, int F, int J, int L,
                             cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  const int nrb = (J + 63) / 64;
  if (nrb > 65535) return cudaErrorInvalidValue;
  const size_t smem = sspi_band_smem(umax, FB);
  if (smem > 220 * 1024) return cudaErrorInvalidValue;
  const dim3 grid((F + FB - 1) / FB, nrb);
#define SRP_BAND(FBV)                                                                        \
  case FBV: {                                                                                \
    cudaError_t e = allow_max_dynamic_smem(sspi_band_kernel<FBV>);                           \
    if (e != cudaSuccess) return e;                                                          \
    sspi_band_kernel<FBV><<<grid, 256, smem, s>>>(xi, row_ptr, taps, blk_ptr, blk_cols, Z,   \
                                                  keys, F, J, L);                            \
    break;                                                                                   \
  }
  switch (FB) {
    SRP_BAND(32)
    SRP_BAND(16)
    SRP_BAND(8)
    SRP_BAND(4)
    SRP_BAND(2)
    SRP_BAND(1)
    default:
      return cudaErrorInvalidValue;
  }
#undef SRP_BAND
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
__global__ void argmax_finalize_kernel(const unsigned long long* __restrict__ keys,
                                       int* __restrict__ out, int F) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const unsigned long long k = keys[f];
  out[f] = k ? static_cast<int>(0xFFFFFFFFu - static_cast<unsigned>(k & 0xFFFFFFFFull)) : -1;
}

cudaError_t launch_argmax_finalize(const unsigned long long* keys, int* argmax, int F,
                                   cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  argmax_finalize_kernel<<<(F + 255) / 256, 256, 0, s>>>(keys, argmax, F);
  return cudaGetLastError();
}

}  // namespace srp

// ---------------------------------------------------------------------------------
// Allocation-free SLRI interpolation (srp_slri_apply_static in include/libsrp.h).
// The intermediate u = Lambda_fat xi and the argmax keys live in one file-scope device
// array instead of plan scratch: u at offset 0 (kStaticUFloats floats), keys after it.
// Host code must not pass the array's name to a kernel (on the host it is only a
// stand-in): the device address is looked up with cudaGetSymbolAddress, with the device
// current, once per CUDA context, and cached under the context's process-unique ID
// (cuCtxGetId), so that a device reset or a new primary context gets a fresh lookup
// instead of an address that belonged to a context that no longer exists.
// ---------------------------------------------------------------------------------
namespace srp {
namespace {
constexpr size_t kStaticUFloats = size_t(1) << 20;  // F * R <= 1,048,576 (4 MiB)
constexpr int kStaticMaxFrames = 65536;             // argmax keys (512 KiB)
constexpr size_t kStaticBytes =
    kStaticUFloats * sizeof(float) + kStaticMaxFrames * sizeof(unsigned long long);
constexpr int kStaticCache = 64;  // contexts remembered (oldest replaced)
struct StaticAddr {
  unsigned long long ctx_id;  // 0: empty
  void* addr;
};
std::mutex g_static_mu;
StaticAddr g_static_addr[kStaticCache] = {};
int g_static_next = 0;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
}  // namespace

static __device__ __align__(256) unsigned char g_slri_static_scratch[kStaticBytes];

// The process-unique ID of the context current on this thread, 0 if none is bound yet.
static srp_status current_context_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || !f1 ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f2) {
      set_error("srp_slri_apply_static: the driver has no cuCtxGetCurrent / cuCtxGetId");
      return SRP_ECUDA;
    }
    g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext c = nullptr;
  if (g_ctx_current(&c) != CUDA_SUCCESS) {
    set_error("srp_slri_apply_static: cuCtxGetCurrent failed");
    return SRP_ECUDA;
  }
  *id = 0;
  if (c && g_ctx_id(c, id) != CUDA_SUCCESS) {
    set_error("srp_slri_apply_static: cuCtxGetId failed");
    return SRP_ECUDA;
  }
  return SRP_OK;
}

static srp_status static_scratch(void** out) {
  int dev = 0;
  SRP_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_static_mu);
  unsigned long long id = 0;
  srp_status st = current_context_id(&id);
  if (st != SRP_OK) return st;
  if (id != 0) {
    for (const StaticAddr& e : g_static_addr)
      if (e.ctx_id == id) {
        *out = e.addr;
        return SRP_OK;
      }
  }
  // first call in this context: the lookup binds the device's primary context if this
  // thread has none yet
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_slri_static_scratch);
  if (e != cudaSuccess || !p) {
    set_error(std::string("srp_slri_apply_static: cudaGetSymbolAddress failed: ") +
              cudaGetErrorString(e));
    return SRP_ECUDA;
  }
  st = current_context_id(&id);
  if (st != SRP_OK) return st;
  if (id != 0) {
    g_static_addr[g_static_next] = {id, p};
    g_static_next = (g_static_next + 1) % kStaticCache;
  }
  *out = p;
  return SRP_OK;
}

}  // namespace srp

extern "C" srp_status srp_slri_apply_static(const float* xi, const float* fat, const float* tall,
                                            int F, int L, int R, int J, float* maps, int* argmax,
                                            void* stream) {
  using namespace srp;
  clear_error();
  if (F < 0) {
    set_error("srp_slri_apply_static: F < 0");
    return SRP_EINVAL;
  }
  if (F == 0) return SRP_OK;
  if (!xi || !fat || !tall || !maps) {
    set_error("srp_slri_apply_static: xi, fat, tall or maps is NULL");
    return SRP_EINVAL;
  }
  if (L < 1 || L > 50000 || J < 1) {
    set_error("srp_slri_apply_static: need 1 <= L <= 50000 and J >= 1");
    return SRP_EINVAL;
  }
  if (R < 8 || R > 64 || R % 8 != 0) {
    set_error("srp_slri_apply_static: R must be one of 8, 16, ..., 64 (pad factors with zeros)");
    return SRP_EINVAL;
  }
  if (F > kStaticMaxFrames || static_cast<size_t>(F) * R > kStaticUFloats) {
    set_error("srp_slri_apply_static: F = " + std::to_string(F) + ", R = " + std::to_string(R) +
              " exceeds the static scratch (F <= 65536 and F * R <= 1048576)");
    return SRP_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(tall) % 16 != 0) {
    set_error("srp_slri_apply_static: tall must be 16-byte aligned");
    return SRP_EINVAL;
  }
  void* base = nullptr;
  srp_status st = static_scratch(&base);
  if (st != SRP_OK) return st;
  float* U = static_cast<float*>(base);
  unsigned long long* keys =
      reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(base) +
                                            kStaticUFloats * sizeof(float));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SRP_CUDA_TRY(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * F, s));
  SRP_CUDA_TRY(launch_slri_fat(xi, fat, U, F, L, R, s));
  SRP_CUDA_TRY(launch_slri_tall(U, tall, maps, keys, F, J, R, s));
  if (argmax) SRP_CUDA_TRY(launch_argmax_finalize(keys, argmax, F, s));
  return SRP_OK;
}
