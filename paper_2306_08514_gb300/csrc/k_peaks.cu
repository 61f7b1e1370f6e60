// Several source estimates per frame: the peak picking behind Eq. (qshat)-(imax),
// extended to several sources.  Eq. (imax) is taken K times per frame, each time over the
// candidate locations not yet excluded; a pick excludes itself and every location closer
// than d_min to it.  The lowest index wins a tie (the order of argmax_key).
//
// Pick 0 is the contraction's argmax (its keys are already merged per frame).  Every later
// pick is one pass over the frames' map rows: blocks of 2048 cells and 8 frames test each
// cell against the frame's earlier picks, reduce the largest key per frame and merge it into
// keys[f] with atomicMax; a per-frame take kernel decodes the key, writes the pick and
// clears the key for the next pass.  The exclusion test is made in FP32 with a fixed operation order (no contraction
// into FMA), so that the decision is reproducible on the host:
//   d^2 = ((dx*dx + dy*dy) + dz*dz), d = q_i - q_pick, every operation rounded to FP32,
//   excluded when d^2 < t, t = d_min^2 rounded to FP32.
#include "srp_internal.h"
#include "srp_device.cuh"

namespace srp {

namespace {
constexpr int kPeakCellsPerThread = 8;
constexpr int kPeakThreads = 256;
constexpr int kPeakMaxBlocksY = 65535;  // frame blocks index grid y
}  // namespace

__device__ __forceinline__ float peak_dist2(float4 a, float4 b) {
  const float dx = __fsub_rn(a.x, b.x);
  const float dy = __fsub_rn(a.y, b.y);
  const float dz = __fsub_rn(a.z, b.z);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Pass for pick k >= 1 of the frames f0 + blockIdx.y * FPB .. + FPB - 1: each thread keeps
// the coordinates of its cells in registers and tests them for every frame of the block.
constexpr int kPeakFramesPerBlock = 8;

__global__ __launch_bounds__(kPeakThreads) void peaks_pass_kernel(
    const float* __restrict__ Z, int F, int J, const float4* __restrict__ grid,
    const int* __restrict__ picks, int K, int k, float t, unsigned long long* __restrict__ keys,
    int f0) {
  constexpr int FPB = kPeakFramesPerBlock;
  __shared__ float4 pc[FPB][kPeaksMax];
  __shared__ int pi[FPB][kPeaksMax];
  __shared__ int ended[FPB];
  __shared__ unsigned long long red[kPeakThreads / 32][FPB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int fb0 = f0 + blockIdx.y * FPB;
  const int nf = min(FPB, F - fb0);
  if (tid < FPB) ended[tid] = tid < nf ? 0 : 1;
  __syncthreads();
  for (int e = tid; e < nf * k; e += kPeakThreads) {
    const int fl = e / k, j = e - fl * k;
    const int i = picks[static_cast<size_t>(fb0 + fl) * K + j];
    pi[fl][j] = i;
    if (i < 0) {
      ended[fl] = 1;
    } else {
      pc[fl][j] = __ldg(grid + i);
    }
  }
  __syncthreads();
  const int base = blockIdx.x * (kPeakThreads * kPeakCellsPerThread);
  float4 q[kPeakCellsPerThread];
#pragma unroll
  for (int c = 0; c < kPeakCellsPerThread; ++c) {
    const int i = base + c * kPeakThreads + tid;
    q[c] = i < J ? __ldg(grid + i) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // every map value of the block's frames and cells is loaded before any is tested, so the
  // loads are in flight together
  float v[FPB][kPeakCellsPerThread];
#pragma unroll
  for (int fl = 0; fl < FPB; ++fl) {
    const float* zr = Z + static_cast<size_t>(fb0 + (fl < nf ? fl : 0)) * J;
#pragma unroll
    for (int c = 0; c < kPeakCellsPerThread; ++c) {
      const int i = base + c * kPeakThreads + tid;
      v[fl][c] = (fl < nf && i < J) ? zr[i] : 0.f;
    }
  }
#pragma unroll
  for (int fl = 0; fl < FPB; ++fl) {
    if (fl >= nf) break;  // uniform over the block
    unsigned long long best = 0ull;
    if (!ended[fl]) {  // uniform over the block
#pragma unroll
      for (int c = 0; c < kPeakCellsPerThread; ++c) {
        const int i = base + c * kPeakThreads + tid;
        if (i < J) {
          bool ok = true;
          for (int j = 0; j < k; ++j) ok = ok && i != pi[fl][j] && !(peak_dist2(q[c], pc[fl][j]) < t);
          if (ok) {
            const unsigned long long key = argmax_key(v[fl][c], i);
            best = key > best ? key : best;
          }
        }
      }
    }
    best = warp_max_u64(best);
    if (lane == 0) red[warp][fl] = best;
  }
  __syncthreads();
  if (tid < nf) {
    unsigned long long b = 0ull;
#pragma unroll
    for (int w = 0; w < kPeakThreads / 32; ++w) b = red[w][tid] > b ? red[w][tid] : b;
    if (b) atomicMax(keys + fb0 + tid, b);
  }
}

// keys[f] -> pick k of frame f (or -1: no location left, or an earlier pick was -1);
// the key is cleared for the next pass.
__global__ void peaks_take_kernel(const float* __restrict__ Z, int F, int J,
                                  unsigned long long* __restrict__ keys, int* __restrict__ picks,
                                  float* __restrict__ values, int K, int k) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  int* pr = picks + static_cast<size_t>(f) * K;
  const unsigned long long key = keys[f];
  keys[f] = 0ull;
  const bool ended = k > 0 && pr[k - 1] < 0;
  const int i = (!ended && key) ? static_cast<int>(0xFFFFFFFFu - static_cast<unsigned>(key & 0xFFFFFFFFull))
                                : -1;
  pr[k] = i;
  if (values)
    values[static_cast<size_t>(f) * K + k] =
        i >= 0 ? Z[static_cast<size_t>(f) * J + i] : __int_as_float(0x7fc00000);
}

cudaError_t launch_peaks(const float* Z, int F, int J, const float4* grid,
                         unsigned long long* keys, int K, float t, int* picks, float* values,
                         cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  if (K < 1 || K > kPeaksMax) return cudaErrorInvalidValue;
  const int tb = 256, tg = (F + tb - 1) / tb;
  peaks_take_kernel<<<tg, tb, 0, s>>>(Z, F, J, keys, picks, values, K, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int gx = (J + kPeakThreads * kPeakCellsPerThread - 1) / (kPeakThreads * kPeakCellsPerThread);
  constexpr int span = kPeakMaxBlocksY * kPeakFramesPerBlock;  // frames per launch
  for (int k = 1; k < K; ++k) {
    for (int f0 = 0; f0 < F; f0 += span) {
      const int nf = F - f0 < span ? F - f0 : span;
      const int gy = (nf + kPeakFramesPerBlock - 1) / kPeakFramesPerBlock;
      peaks_pass_kernel<<<dim3(gx, gy), kPeakThreads, 0, s>>>(Z, f0 + nf, J, grid, picks, K, k, t,
                                                               keys, f0);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    peaks_take_kernel<<<tg, tb, 0, s>>>(Z, F, J, keys, picks, values, K, k);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int peaks_launches(int F, int K) {
  const int span = kPeakMaxBlocksY * kPeakFramesPerBlock;
  const int slices = (F + span - 1) / span;
  return 1 + (K - 1) * (slices + 1);
}

}  // namespace srp
