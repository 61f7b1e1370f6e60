// conv. FD-SRP in FP32 on the CUDA cores: Z = A B^T (boxed Eq. z_computed written as a
// real product over the stacked [Re psi | Im psi] and [2cos | -2sin] rows), with the
// per-frame argmax (Eq. imax) fused into the epilogue.
//
// A [F][Kd], B [J][Kd], Z [F][J], all row-major with the reduction dimension Kd = P*N
// contiguous.  Block tile 128 frames x 128 cells, k-step 8, 256 threads each owning an
// 8x8 sub-tile split into two 4-row and two 4-column strips (conflict-free float4
// shared-memory reads), double-buffered shared memory with register prefetch.
#include "srp_internal.h"
#include "srp_device.cuh"

namespace srp {

namespace {
constexpr int BM = 128, BN = 128, BK = 8, PADS = 4;
}

// With kslice < Kd the reduction is split: block z covers k-tiles
// [z*kslice, (z+1)*kslice) and writes its partial map to Z + z*F*J without the argmax
// (the partials are summed by split_reduce_argmax_kernel).
// Frame tiles run fastest (blockIdx.x) so the CTAs in flight share the B (SRP matrix)
// tiles through L2.
//
// GEN: B is the SRP matrix generated on the fly instead of read (for grids whose stored
// matrix would not fit): column c = p N + r holds 2cos(theta_k) (r = k < K) or
// -2sin(theta_k) (r = K + k), theta_k = 2 pi frac(k tau_p(i) / N), k = 0 giving 0.  tau is
// split as tau_hi + tau_lo with tau_hi carrying 13 significant bits, so k tau_hi (k < 2^11)
// and its fraction of N are exact in FP32 and the phase is accurate to ~1e-7.
struct GenB {
  const float* tau_hi;  // [J][P]
  const float* tau_lo;  // [J][P]
  int P, N;
};

__device__ __forceinline__ float gen_b(const GenB& g, int i, int c) {
  const int q = c / g.N, r = c - q * g.N;
  const int K = g.N >> 1;
  const int k = r < K ? r : r - K;
  if (k == 0) return 0.f;
  const float th = __ldg(g.tau_hi + static_cast<size_t>(i) * g.P + q);
  const float tl = __ldg(g.tau_lo + static_cast<size_t>(i) * g.P + q);
  const float invN = 1.f / static_cast<float>(g.N);
  const float x = static_cast<float>(k) * th * invN;  // exact
  const float rr = (x - floorf(x)) + static_cast<float>(k) * tl * invN;
  float sn, cs;
  sincospif(2.f * rr, &sn, &cs);
  return r < K ? 2.f * cs : -2.f * sn;
}

template <bool SPLIT, bool GEN>
__global__ __launch_bounds__(256, 2) void sgemm_nt_argmax_kernel(
    const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ Z,
    unsigned long long* __restrict__ keys, int F, int J, int Kd, int kslice, const GenB gb) {
  __shared__ __align__(16) float As[2][BK][BM + PADS];
  __shared__ __align__(16) float Bs[2][BK][BN + PADS];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int lr = tid >> 1, lk = (tid & 1) * 4;
  const bool aok = (m0 + lr) < F;
  const bool bok = (n0 + lr) < J;
  const int kbeg = SPLIT ? blockIdx.z * kslice : 0;
  const int kend = SPLIT ? min(Kd, kbeg + kslice) : Kd;
  if (SPLIT) Z += static_cast<size_t>(blockIdx.z) * F * J;
  const float4* Ap = reinterpret_cast<const float4*>(A + static_cast<size_t>(aok ? m0 + lr : 0) * Kd + kbeg + lk);
  const float4* Bp = GEN ? nullptr
                        : reinterpret_cast<const float4*>(B + static_cast<size_t>(bok ? n0 + lr : 0) * Kd + kbeg + lk);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  auto load_b = [&](int kt) -> float4 {
    if (!bok) return z4;
    if (!GEN) return __ldg(Bp + kt * (BK / 4));
    const int c = kbeg + kt * BK + lk;
    return make_float4(gen_b(gb, n0 + lr, c), gen_b(gb, n0 + lr, c + 1), gen_b(gb, n0 + lr, c + 2),
                       gen_b(gb, n0 + lr, c + 3));
  };
  float4 ra = aok ? __ldg(Ap) : z4;
  float4 rb = load_b(0);
  As[0][lk + 0][lr] = ra.x; As[0][lk + 1][lr] = ra.y; As[0][lk + 2][lr] = ra.z; As[0][lk + 3][lr] = ra.w;
  Bs[0][lk + 0][lr] = rb.x; Bs[0][lk + 1][lr] = rb.y; Bs[0][lk + 2][lr] = rb.z; Bs[0][lk + 3][lr] = rb.w;
  __syncthreads();

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  const int nk = (kend - kbeg) / BK;
  for (int kt = 0; kt < nk; ++kt) {
    const int cur = kt & 1;
    if (kt + 1 < nk) {
      ra = aok ? __ldg(Ap + (kt + 1) * (BK / 4)) : z4;
      rb = load_b(kt + 1);
    }
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[cur][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[cur][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (kt + 1 < nk) {
      const int nx = cur ^ 1;
      As[nx][lk + 0][lr] = ra.x; As[nx][lk + 1][lr] = ra.y; As[nx][lk + 2][lr] = ra.z; As[nx][lk + 3][lr] = ra.w;
      Bs[nx][lk + 0][lr] = rb.x; Bs[nx][lk + 1][lr] = rb.y; Bs[nx][lk + 2][lr] = rb.z; Bs[nx][lk + 3][lr] = rb.w;
    }
    __syncthreads();
  }

  // epilogue: store, then per-row (frame) argmax over this block's 128 cells
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    unsigned long long best = 0ull;
    if (m < F) {
      float* zr = Z + static_cast<size_t>(m) * J;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        if (n < J) {
          zr[n] = acc[i][j];
          if (!SPLIT) {
            const unsigned long long kk = argmax_key(acc[i][j], n);
            best = kk > best ? kk : best;
          }
        }
      }
    }
    if (!SPLIT) {  // reduce over the 16 threads sharing this row (one half-warp)
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, best, o);
        best = other > best ? other : best;
      }
      if (tx == 0 && m < F && best) atomicMax(keys + m, best);
    }
  }
}

// Z[f][i] = sum over the nsplit partial maps [nsplit][F][J] (summed in FP64), plus the
// argmax keys.  Z's rows are ldz floats apart and its column 0 is cell col0 of the map (a
// column block of a wider map); the keys carry col0 + i.
__global__ __launch_bounds__(256) void split_reduce_argmax_kernel(const float* __restrict__ part,
                                                                  int nsplit, float* __restrict__ Z,
                                                                  unsigned long long* __restrict__ keys,
                                                                  int F, int J, int ldz, int col0) {
  __shared__ unsigned long long red[8];
  const int f = blockIdx.x;
  const size_t FJ = static_cast<size_t>(F) * J;
  unsigned long long best = 0ull;
  for (int i = blockIdx.y * 1024 + threadIdx.x; i < min(J, (blockIdx.y + 1) * 1024); i += 256) {
    const size_t idx = static_cast<size_t>(f) * J + i;
    double acc = 0.0;
    for (int z = 0; z < nsplit; ++z) acc += static_cast<double>(part[z * FJ + idx]);
    const float v = static_cast<float>(acc);
    if (Z) Z[static_cast<size_t>(f) * ldz + i] = v;  // Z == NULL: estimates only
    const unsigned long long k = argmax_key(v, col0 + i);
    best = k > best ? k : best;
  }
  best = warp_max_u64(best);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0ull;
    for (int w = 0; w < 8; ++w) b = red[w] > b ? red[w] : b;
    if (b) atomicMax(keys + f, b);
  }
}

int sgemm_split_count(int Kd) {
  const int per = 16384;  // reduction terms accumulated sequentially in FP32 per slice
  return Kd <= per ? 1 : (Kd + per - 1) / per;
}

cudaError_t launch_sgemm_nt_argmax(const float* A, const float* B, float* Z,
                                   unsigned long long* keys, int F, int J, int Kd,
                                   float* split_ws, cudaStream_t s, const float* tau_hi,
                                   const float* tau_lo, int P, int N) {
  if (F <= 0) return cudaSuccess;
  if (Kd % BK != 0) return cudaErrorInvalidValue;
  const bool gen = tau_hi != nullptr;
  const GenB gb{tau_hi, tau_lo, P, N};
  const int nsplit = sgemm_split_count(Kd);
  if (nsplit == 1) {
    dim3 grid((F + BM - 1) / BM, (J + BN - 1) / BN, 1);
    if (gen)
      sgemm_nt_argmax_kernel<false, true><<<grid, 256, 0, s>>>(A, B, Z, keys, F, J, Kd, Kd, gb);
    else
      sgemm_nt_argmax_kernel<false, false><<<grid, 256, 0, s>>>(A, B, Z, keys, F, J, Kd, Kd, gb);
    return cudaGetLastError();
  }
  if (!split_ws) return cudaErrorInvalidValue;
  int kslice = (Kd / BK + nsplit - 1) / nsplit * BK;
  const int nz = (Kd + kslice - 1) / kslice;
  dim3 grid((F + BM - 1) / BM, (J + BN - 1) / BN, nz);
  if (gen)
    sgemm_nt_argmax_kernel<true, true><<<grid, 256, 0, s>>>(A, B, split_ws, keys, F, J, Kd, kslice, gb);
  else
    sgemm_nt_argmax_kernel<true, false><<<grid, 256, 0, s>>>(A, B, split_ws, keys, F, J, Kd, kslice, gb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_split_reduce(split_ws, nz, Z, keys, F, J, s);
}

cudaError_t launch_split_reduce(const float* ws, int nz, float* Z, unsigned long long* keys,
                                int F, int J, cudaStream_t s, int ldz, int col0) {
  dim3 g2(F, (J + 1023) / 1024);
  split_reduce_argmax_kernel<<<g2, 256, 0, s>>>(ws, nz, Z, keys, F, J, ldz > 0 ? ldz : J, col0);
  return cudaGetLastError();
}

}  // namespace srp
