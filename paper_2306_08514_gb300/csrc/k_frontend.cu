// Front end of the SRP path: STFT + PHAT, cross-spectra, sampling of the TD GCCs, and the
// operands of the conventional SRP-matrix product.
//
//   y-hat_m(omega_k) = y_m / |y_m|                   PHAT, Eq. corrmatrix
//   psi_p(omega_k)  = y-hat_m y-hat_m'^*            k = 1..K-1 (Eq. psi_p_single)
//   xi_p(nT)        = iFFT_2K[psi-bar_p](n)          Eq. xi_p_ifft, n_prime (or its matrix
//                                                    form S-bar_p psi-bar_p, Eq. xi_computed)
//   H_p[i,k]        = exp(j omega_k Delta t_p(i))    Eq. H_p_single
#include "srp_internal.h"

#include <algorithm>
#include <cmath>
#include "srp_device.cuh"
#include "srp_ops.cuh"

namespace srp {

// ---------------------------------------------------------------------------------
// STFT + PHAT.  One group of N/16 threads per (frame, microphone), 256 threads per
// block.  The N real samples are packed as H = N/2 complex numbers z[j] = x[2j] + i x[2j+1],
// transformed by the H-point mixed-radix FFT (p8fft), and the N-point spectrum is recovered
// for k = 1..K-1 as X[k] = E[k] + W^k O[k] with E = (Z[k] + Z[H-k]^*)/2,
// O = (Z[k] - Z[H-k]^*)/(2i).  An all-zero channel gives exactly X = 0, hence y-hat = 0
// (|y|^2 < 1e-30 -> 0).
// ---------------------------------------------------------------------------------
// out[idx] = v in the operand type ot (an OpType value) chosen at run time
__device__ __forceinline__ void put_op_rt(int ot, void* hi, void* lo, size_t idx, float v) {
  switch (static_cast<OpType>(ot)) {
    case OpType::F32: op_store<float, false>(hi, lo, idx, v); break;
    case OpType::F16: op_store<__half, false>(hi, lo, idx, v); break;
    case OpType::BF16: op_store<__nv_bfloat16, false>(hi, lo, idx, v); break;
    case OpType::F16X2: op_store<__half, true>(hi, lo, idx, v); break;
    case OpType::BF16X2: op_store<__nv_bfloat16, true>(hi, lo, idx, v); break;
    case OpType::TF32: op_store<tf32_t, false>(hi, lo, idx, v); break;
    case OpType::TF32X2: op_store<tf32_t, true>(hi, lo, idx, v); break;
  }
}

// Padded FFT buffers hold element i at i + i/16: the strided stores of the early stages
// then spread over the banks.
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int fpad_len(int H) { return H + H / 16; }

// Mixed-radix Stockham FFT of compile-time length H (natural order in and out,
// unnormalised) on padded buffers: a first stage of radix R0 = 2, 4 or 8 with Ns = 1 (no
// twiddles), then radix-8 stages.  Stage with sub-transform length Ns and radix R:
// butterfly b (< H/R) takes a[b + m H/R], m < R, multiplies input m by w^(m k) (w =
// exp(-2 pi i / (R Ns)), exp(+...) when INV; k = b mod Ns), transforms, and writes output r
// to ((b - k) R + k) + r Ns.  Called by H/8 threads per transform (t = 0..H/8-1), each
// owning one radix-8 butterfly per stage; the thread's twiddles w^k, w^2k, w^4k of each
// radix-8 stage are in registers (p8_twiddles).  Every thread of the block takes part in
// the barriers.
template <int H>
struct P8 {
  static constexpr int LOG = __builtin_ctz(H);
  static constexpr int R0 = LOG % 3 == 0 ? 8 : (LOG % 3 == 1 ? 2 : 4);
  static constexpr int LOG0 = R0 == 8 ? 3 : (R0 == 4 ? 2 : 1);
  static constexpr int NTW = (LOG - LOG0) / 3;  // radix-8 stages after the first
};

template <int H, int TWS, bool INV>
__device__ __forceinline__ void p8_twiddles(const float2* __restrict__ twg, int t,
                                            float2 (&tw3)[P8<H>::NTW > 0 ? P8<H>::NTW : 1][3]) {
  int Ns = P8<H>::R0;
#pragma unroll
  for (int st = 0; st < P8<H>::NTW; ++st, Ns <<= 3) {
    const int k = t & (Ns - 1);
    const int u = (k * (H / (8 * Ns))) << TWS;  // w^k = table[u]; 4u < table size
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const float2 w = __ldg(twg + (u << m));
      tw3[st][m] = INV ? make_float2(w.x, -w.y) : w;
    }
  }
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// 4-point DFT in place (forward: exp(-...), inverse: exp(+...))
template <bool INV>
__device__ __forceinline__ void dft4(float2& c0, float2& c1, float2& c2, float2& c3) {
  const float2 s02 = cadd(c0, c2), d02 = csub(c0, c2), s13 = cadd(c1, c3), d13 = csub(c1, c3);
  const float2 r13 = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);  // +-i d13
  c0 = cadd(s02, s13);
  c1 = cadd(d02, r13);
  c2 = csub(s02, s13);
  c3 = csub(d02, r13);
}

// 8-point DFT in place: a_m = x_m + x_{m+4} give the even outputs (4-point DFT), b_m =
// (x_m - x_{m+4}) W8^m the odd ones
template <bool INV>
__device__ __forceinline__ void dft8(float2 (&x)[8]) {
  constexpr float h = 0.70710678118654752440f;
  float2 a0 = cadd(x[0], x[4]), a1 = cadd(x[1], x[5]), a2 = cadd(x[2], x[6]), a3 = cadd(x[3], x[7]);
  float2 b0 = csub(x[0], x[4]), b1 = csub(x[1], x[5]), b2 = csub(x[2], x[6]), b3 = csub(x[3], x[7]);
  if (INV) {  // W8 = (1 + i)/sqrt2, W8^2 = i, W8^3 = (-1 + i)/sqrt2
    b1 = make_float2(h * (b1.x - b1.y), h * (b1.x + b1.y));
    b2 = make_float2(-b2.y, b2.x);
    b3 = make_float2(-h * (b3.x + b3.y), h * (b3.x - b3.y));
  } else {    // W8 = (1 - i)/sqrt2, W8^2 = -i, W8^3 = (-1 - i)/sqrt2
    b1 = make_float2(h * (b1.x + b1.y), h * (b1.y - b1.x));
    b2 = make_float2(b2.y, -b2.x);
    b3 = make_float2(h * (b3.y - b3.x), -h * (b3.x + b3.y));
  }
  dft4<INV>(a0, a1, a2, a3);
  dft4<INV>(b0, b1, b2, b3);
  x[0] = a0; x[2] = a1; x[4] = a2; x[6] = a3;
  x[1] = b0; x[3] = b1; x[5] = b2; x[7] = b3;
}

template <int H, bool INV>
__device__ __forceinline__ float2* p8fft(float2* a, float2* b, int t,
                                         const float2 (&tw3)[P8<H>::NTW > 0 ? P8<H>::NTW : 1][3]) {
  constexpr int R0 = P8<H>::R0;
  constexpr int T = H / 8;
  // first stage, Ns = 1: 8 / R0 butterflies of radix R0 per thread
  {
    constexpr int S = H / R0;
#pragma unroll
    for (int i = 0; i < 8 / R0; ++i) {
      const int bi = t + i * T;
      if constexpr (R0 == 8) {
        float2 x[8];
#pragma unroll
        for (int m = 0; m < 8; ++m) x[m] = a[fpad(bi + m * S)];
        dft8<INV>(x);
#pragma unroll
        for (int r = 0; r < 8; ++r) b[fpad(bi * 8 + r)] = x[r];
      } else if constexpr (R0 == 4) {
        float2 c0 = a[fpad(bi)], c1 = a[fpad(bi + S)], c2 = a[fpad(bi + 2 * S)], c3 = a[fpad(bi + 3 * S)];
        dft4<INV>(c0, c1, c2, c3);
        b[fpad(bi * 4)] = c0;
        b[fpad(bi * 4 + 1)] = c1;
        b[fpad(bi * 4 + 2)] = c2;
        b[fpad(bi * 4 + 3)] = c3;
      } else {
        const float2 v0 = a[fpad(bi)], v1 = a[fpad(bi + S)];
        b[fpad(bi * 2)] = cadd(v0, v1);
        b[fpad(bi * 2 + 1)] = csub(v0, v1);
      }
    }
    __syncthreads();
    float2* tmp = a;
    a = b;
    b = tmp;
  }
  // radix-8 stages, one butterfly per thread
  int Ns = R0;
#pragma unroll
  for (int st = 0; st < P8<H>::NTW; ++st, Ns <<= 3) {
    const int k = t & (Ns - 1);
    float2 x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) x[m] = a[fpad(t + m * T)];
    const float2 w1 = tw3[st][0], w2 = tw3[st][1], w4 = tw3[st][2];
    const float2 w3 = cmul(w2, w1), w5 = cmul(w4, w1), w6 = cmul(w4, w2), w7 = cmul(w6, w1);
    x[1] = cmul(x[1], w1);
    x[2] = cmul(x[2], w2);
    x[3] = cmul(x[3], w3);
    x[4] = cmul(x[4], w4);
    x[5] = cmul(x[5], w5);
    x[6] = cmul(x[6], w6);
    x[7] = cmul(x[7], w7);
    dft8<INV>(x);
    const int d = ((t - k) << 3) + k;
#pragma unroll
    for (int r = 0; r < 8; ++r) b[fpad(d + r * Ns)] = x[r];
    __syncthreads();
    float2* tmp = a;
    a = b;
    b = tmp;
  }
  return a;
}

template <int H>
__global__ __launch_bounds__(256) void stft_phat_kernel(const float* __restrict__ frames, int M,
                                                        const float* __restrict__ window,
                                                        const float2* __restrict__ twiddle,
                                                        float2* __restrict__ yhat) {
  extern __shared__ float2 smem[];
  constexpr int N = 2 * H, K = H;
  constexpr int Tg = H / 8;  // threads per channel group
  float2* tw = smem;         // H entries
  float2* bufA = smem + H + threadIdx.y * 2 * fpad_len(H);
  float2* bufB = bufA + fpad_len(H);
  const int tid = threadIdx.y * Tg + threadIdx.x;
  for (int t = tid; t < H; t += Tg * blockDim.y) tw[t] = twiddle[t];
  float2 tw3[P8<H>::NTW > 0 ? P8<H>::NTW : 1][3];
  p8_twiddles<H, 1, false>(twiddle, threadIdx.x, tw3);
  const int f = blockIdx.y;
  const int m = blockIdx.x * blockDim.y + threadIdx.y;
  const bool live = m < M;
  const float2* x2 =
      reinterpret_cast<const float2*>(frames + (static_cast<size_t>(f) * M + (live ? m : 0)) * N);
  const float2* w2 = reinterpret_cast<const float2*>(window);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int j = threadIdx.x + i * Tg;
    const float2 v = live ? __ldg(x2 + j) : make_float2(0.f, 0.f);
    const float2 w = __ldg(w2 + j);
    bufA[fpad(j)] = make_float2(v.x * w.x, v.y * w.y);
  }
  __syncthreads();
  const float2* Z = p8fft<H, false>(bufA, bufB, threadIdx.x, tw3);
  if (!live) return;  // no barrier follows
  float2* out = yhat + (static_cast<size_t>(f) * M + m) * K;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = threadIdx.x + i * Tg;
    const float2 zk = Z[fpad(k)];
    const float2 zr = Z[fpad((H - k) & (H - 1))];
    const float2 zc = make_float2(zr.x, -zr.y);
    const float2 E = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
    const float2 O = make_float2(0.5f * (zk.y - zc.y), -0.5f * (zk.x - zc.x));
    const float2 WO = cmul(tw[k], O);
    const float2 Y = make_float2(E.x + WO.x, E.y + WO.y);
    const float p = Y.x * Y.x + Y.y * Y.y;
    float2 r = make_float2(0.f, 0.f);
    if (k > 0 && p >= 1e-30f) {  // DC is not used (Sec. II-D)
      const float sc = __frsqrt_rn(p);
      r = make_float2(Y.x * sc, Y.y * sc);
    }
    out[k] = r;
  }
}

// Launches that index frames by blockIdx.y take at most kMaxGridY frames each; longer
// batches are issued as consecutive launches on offset base pointers.
constexpr int kMaxGridY = 65535;

cudaError_t launch_stft_phat(const float* frames, int F, int M, int N, const float* window,
                             const float2* twiddle, float2* yhat, cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  if (F > kMaxGridY) {
    const cudaError_t e = launch_stft_phat(frames, kMaxGridY, M, N, window, twiddle, yhat, s);
    if (e != cudaSuccess) return e;
    const size_t f0 = kMaxGridY;
    return launch_stft_phat(frames + f0 * M * N, F - kMaxGridY, M, N, window, twiddle,
                            yhat + f0 * M * (N / 2), s);
  }
  const int H = N / 2, Tg = H / 8;
  const int cpb = 256 / Tg;  // channels per block
  dim3 block(Tg, cpb);
  dim3 grid((M + cpb - 1) / cpb, F);
  const size_t smem = sizeof(float2) * (H + static_cast<size_t>(cpb) * 2 * fpad_len(H));
  switch (H) {
    case 128: stft_phat_kernel<128><<<grid, block, smem, s>>>(frames, M, window, twiddle, yhat); break;
    case 256: stft_phat_kernel<256><<<grid, block, smem, s>>>(frames, M, window, twiddle, yhat); break;
    case 512: stft_phat_kernel<512><<<grid, block, smem, s>>>(frames, M, window, twiddle, yhat); break;
    case 1024: stft_phat_kernel<1024><<<grid, block, smem, s>>>(frames, M, window, twiddle, yhat); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Sampling.  Two pairs share one N-point complex iFFT: the input is
// psi-bar_a + i psi-bar_b, both two-sided (Appendix, Eq. psi_p_two) and Hermitian, so
// the (unnormalised) inverse transform is xi-bar_a + i xi-bar_b.  The lags
// n = -N_p..N_p are read at index mod(n, N) (Eq. n_prime) and stored ascending.
// ---------------------------------------------------------------------------------
template <int N>
__global__ __launch_bounds__(N / 8) void gcc_samples_kernel(
    const float2* __restrict__ yhat, int M, int P, const int2* __restrict__ pairs,
    const int* __restrict__ Np, const int* __restrict__ off, int L,
    const float2* __restrict__ twiddle, int ot, void* out, void* out_lo, int out_cols) {
  __shared__ float2 buf[2 * fpad_len(N)];
  constexpr int K = N >> 1;
  constexpr int T = N >> 3;  // threads: one radix-8 butterfly each per stage
  float2* bufA = buf;
  float2* bufB = buf + fpad_len(N);
  const int j = threadIdx.x;
  float2 tw3[P8<N>::NTW > 0 ? P8<N>::NTW : 1][3];
  p8_twiddles<N, 0, true>(twiddle, j, tw3);
  const int f = blockIdx.y;
  const int pa = 2 * blockIdx.x;
  const int pb = pa + 1;
  const bool hasb = pb < P;
  const int2 qa = __ldg(pairs + pa);
  const int2 qb = hasb ? __ldg(pairs + pb) : make_int2(0, 0);
  const float2* yf = yhat + static_cast<size_t>(f) * M * K;
#pragma unroll
  for (int i = 0; i < K / T; ++i) {
    const int k = j + i * T;
    if (k == 0) {
      bufA[fpad(0)] = make_float2(0.f, 0.f);
      bufA[fpad(K)] = make_float2(0.f, 0.f);
      continue;
    }
    const float2 a = cmul_conj(__ldg(yf + qa.x * K + k), __ldg(yf + qa.y * K + k));
    const float2 b = hasb ? cmul_conj(__ldg(yf + qb.x * K + k), __ldg(yf + qb.y * K + k))
                          : make_float2(0.f, 0.f);
    bufA[fpad(k)] = make_float2(a.x - b.y, a.y + b.x);      // psi_a + i psi_b
    bufA[fpad(N - k)] = make_float2(a.x + b.y, b.x - a.y);  // psi_a^* + i psi_b^*
  }
  __syncthreads();
  const float2* x = p8fft<N, true>(bufA, bufB, j, tw3);
  const size_t row = static_cast<size_t>(f) * out_cols;
  const int na = __ldg(Np + pa);
  const size_t oa = row + __ldg(off + pa);
  for (int t = j; t < 2 * na + 1; t += T) put_op_rt(ot, out, out_lo, oa + t, x[fpad((t - na + N) & (N - 1))].x);
  if (hasb) {
    const int nb = __ldg(Np + pb);
    const size_t ob = row + __ldg(off + pb);
    for (int t = j; t < 2 * nb + 1; t += T) put_op_rt(ot, out, out_lo, ob + t, x[fpad((t - nb + N) & (N - 1))].y);
  }
  if (blockIdx.x == 0)  // the operand's zero padding beyond L
    for (int c = L + j; c < out_cols; c += T) put_op_rt(ot, out, out_lo, row + c, 0.f);
}

cudaError_t launch_gcc_samples(const float2* yhat, int F, int M, int P, int N, const int2* pairs,
                               const int* Np, const int* off, int L, const float2* twiddle,
                               OpType t, void* out, void* out_lo, int out_cols, cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  if (out_cols < L) return cudaErrorInvalidValue;
  if (F > kMaxGridY) {
    cudaError_t e = launch_gcc_samples(yhat, kMaxGridY, M, P, N, pairs, Np, off, L, twiddle, t,
                                       out, out_lo, out_cols, s);
    if (e != cudaSuccess) return e;
    const size_t f0 = kMaxGridY, rows = f0 * out_cols * op_bytes(t);
    char* hi = static_cast<char*>(out) + rows;
    char* lo = out_lo ? static_cast<char*>(out_lo) + rows : nullptr;
    return launch_gcc_samples(yhat + f0 * M * (N / 2), F - kMaxGridY, M, P, N, pairs, Np, off,
                              L, twiddle, t, hi, lo, out_cols, s);
  }
  dim3 grid((P + 1) / 2, F);
  const int ot = static_cast<int>(t);
  switch (N) {
    case 256:
      gcc_samples_kernel<256><<<grid, 32, 0, s>>>(yhat, M, P, pairs, Np, off, L, twiddle, ot, out, out_lo, out_cols);
      break;
    case 512:
      gcc_samples_kernel<512><<<grid, 64, 0, s>>>(yhat, M, P, pairs, Np, off, L, twiddle, ot, out, out_lo, out_cols);
      break;
    case 1024:
      gcc_samples_kernel<1024><<<grid, 128, 0, s>>>(yhat, M, P, pairs, Np, off, L, twiddle, ot, out, out_lo, out_cols);
      break;
    case 2048:
      gcc_samples_kernel<2048><<<grid, 256, 0, s>>>(yhat, M, P, pairs, Np, off, L, twiddle, ot, out, out_lo, out_cols);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Lag windows up to this N_p are sampled in the matrix form of Eq. xi_computed (the sampling
// GEMM of the fused front end or of gcc_mma_kernel); wider ones by the iFFT.
int gcc_direct_max_lag() { return 32; }


// ---------------------------------------------------------------------------------
// Fused front end: one CTA per frame runs the STFT + PHAT of every channel (the
// half-length transform of stft_phat_kernel on the mixed-radix FFT, channel groups of
// N/16 threads) into shared memory, then either samples every pair (the matrix form of
// Eq. xi_p_ifft as a per-frame GEMM on the warp-level tensor cores) and writes the operand
// the interpolation contraction needs -- xi in FP32 [F][L] (FP32 SSPI gather), xi in the
// operand type [F][Lpad] (tensor-core SI / TD / SSPI), or u = Lambda_fat xi (SLRI, a second
// small GEMM) as [F][Rp] or [F][64] scaled by `scale` -- or writes the packed cross-spectra
// of the conv. FD-SRP / LR-SRP operand.  Saves the y-hat round trip through global memory
// and the separate sampling, packing and Lambda_fat launches.
// ---------------------------------------------------------------------------------
// FrontParams (srp_internal.h): the per-batch arguments of the fused front kernel.

// D += A B for one m16n8k16 tile on the warp-level tensor cores (FP16 in, FP32 accumulate).
// Fragments: a[0] = (row g, K cols 2t, 2t+1), a[1] = (row g+8, same), a[2] / a[3] = the
// same rows at K cols + 8; b0 = (K rows 2t, 2t+1, col g), b1 = K rows + 8; d = (row g,
// cols 2t, 2t+1), (row g+8, same); g = lane / 4, t = lane % 4.  The lower half of each
// 32-bit register holds the element of the smaller K index.
__device__ __forceinline__ void mma_16816(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                          unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// v = hi + lo in FP16 pairs (x in the lower half)
__device__ __forceinline__ void split_h2(float2 v, unsigned& hi, unsigned& lo) {
  const __half2 h = __floats2half2_rn(v.x, v.y);
  const float2 back = __half22float2(h);
  const __half2 l = __floats2half2_rn(v.x - back.x, v.y - back.y);
  hi = *reinterpret_cast<const unsigned*>(&h);
  lo = *reinterpret_cast<const unsigned*>(&l);
}

// Rows of y-hat in shared memory are padded by 4 entries, so that the 8 rows a
// fragment gathers at once fall into distinct bank groups.
__host__ __device__ constexpr int front_row(int K) { return K + 4; }

// ---------------------------------------------------------------------------------
// Sampling for short lag windows (N_p <= 32) from y-hat in global memory, as the per-frame
// GEMM of the fused front end's sampling (Eq. xi_p_ifft at the lags n = -N_p..N_p in the
// matrix form of Eq. xi_computed: rows = pairs, K = bins with Re psi and Im psi
// interleaved, columns = lags; B = front_sampling_table; FP16 hi + lo, three products on
// the warp-level tensor cores, or the hi product alone for operands of 8 to 11 bits).  It
// serves the frames the fused kernel cannot hold (N =
// 2048, or many channels): one CTA per frame stages the spectra of all M channels and the
// sampling table's fragments through shared memory 64 bins at a time, copied
// asynchronously one chunk ahead (two buffers); in each round every warp owns MTW m-tiles
// of 16 pairs and keeps their sums in registers across the chunks -- each k-step's three
// products go into a fresh accumulator, which is then added in FP32 (round to nearest), so
// that the tensor cores' truncating accumulation stays small -- and the samples are
// written in the operand type, zero padded beyond L.
// ---------------------------------------------------------------------------------
constexpr int kMmaChunk = 64;                 // bins per staged chunk (8 k-steps)
constexpr int kMmaRow = kMmaChunk + 4;        // padded row: 8 rows x 4 bins hit distinct banks

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<unsigned>(__cvta_generic_to_shared(smem))),
               "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int NTM, bool X3>
__global__ __launch_bounds__(256, NTM <= 4 ? 2 : 1) void gcc_mma_kernel(
    const float2* __restrict__ yhat, int M, int P, int K, const int2* __restrict__ pairs,
    const int* __restrict__ Np, const int* __restrict__ off, int L,
    const uint4* __restrict__ stab, int NT, int nq0, int ot, void* out, void* out_lo,
    int out_cols) {
  constexpr int MTW = NTM <= 4 ? 4 : 2;  // m-tiles per warp and round (registers)
  constexpr int KS = kMmaChunk / 8;      // k-steps per chunk
  // two buffers, each [M][kMmaRow] spectra then [KS][NT][32] fragments of the table
  extern __shared__ float2 ys[];
  const int buf_f2 = M * kMmaRow + KS * NT * 32 * 2;  // one buffer in float2 units
  const int f = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  const int MT = (P + 15) >> 4;
  const int nch = K / kMmaChunk, nrounds = (MT + 8 * MTW - 1) / (8 * MTW);
  const float2* yf = yhat + static_cast<size_t>(f) * M * K;
  const size_t orow = static_cast<size_t>(f) * out_cols;
  // stage i = (round, chunk): the chunk's spectra of every channel and its table fragments,
  // copied asynchronously one stage ahead of the computation
  auto stage = [&](int i) {
    const int c0 = (i % nch) * kMmaChunk;
    float2* yb = ys + (i & 1) * buf_f2;
    uint4* bb = reinterpret_cast<uint4*>(yb + M * kMmaRow);
    for (int e = tid; e < M * (kMmaChunk / 2); e += 256) {
      const int m = e / (kMmaChunk / 2), j = e - m * (kMmaChunk / 2);
      cp_async16(yb + m * kMmaRow + 2 * j, yf + static_cast<size_t>(m) * K + c0 + 2 * j);
    }
    const uint4* bsrc = stab + static_cast<size_t>(c0 >> 3) * NT * 32;
    for (int e = tid; e < KS * NT * 32; e += 256) cp_async16(bb + e, bsrc + e);
    cp_async_commit();
  };
  float sum[MTW][NTM][4];
  int ch_a0[MTW], ch_b0[MTW], ch_a1[MTW], ch_b1[MTW];
  const int total = nrounds * nch;
  stage(0);
  for (int i = 0; i < total; ++i) {
    const int r0 = (i / nch) * 8 * MTW, c = i % nch;
    if (c == 0) {
#pragma unroll
      for (int g = 0; g < MTW; ++g) {
#pragma unroll
        for (int t = 0; t < NTM; ++t)
#pragma unroll
          for (int e = 0; e < 4; ++e) sum[g][t][e] = 0.f;
        // the channels of this thread's two rows (pairs past P read pair 0; their samples
        // are never written) as row offsets into a staged chunk
        const int ra = (r0 + g * 8 + warp) * 16 + gq, rb = ra + 8;
        const int2 pa = __ldg(pairs + (ra < P ? ra : 0)), pb = __ldg(pairs + (rb < P ? rb : 0));
        ch_a0[g] = pa.x * kMmaRow;
        ch_b0[g] = pa.y * kMmaRow;
        ch_a1[g] = pb.x * kMmaRow;
        ch_b1[g] = pb.y * kMmaRow;
      }
    }
    if (i + 1 < total) {
      stage(i + 1);        // its buffer was released by the barrier ending stage i - 1
      cp_async_wait<1>();  // this thread's copies of stage i have landed
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();       // ... and every thread's
    const float2* yb = ys + (i & 1) * buf_f2;
    const uint4* bs = reinterpret_cast<const uint4*>(yb + M * kMmaRow);
    // each k-step: the table fragments once, then for every m-tile of the warp its psi
    // fragments and a fresh three-product chain, added into the FP32 sums (short dependent
    // chains, the m-tiles independent of one another)
#pragma unroll(NTM <= 4 ? 2 : 1)
    for (int s = 0; s < KS; ++s) {
      uint4 b[NTM];
#pragma unroll
      for (int t = 0; t < NTM; ++t)
        if (t < NT) b[t] = bs[(s * NT + t) * 32 + lane];
#pragma unroll
      for (int g = 0; g < MTW; ++g) {
        if (r0 + g * 8 + warp >= MT) continue;  // warp-uniform
        const float2* q = yb + 8 * s + tq;
        const float2 v[4] = {cmul_conj(q[ch_a0[g]], q[ch_b0[g]]), cmul_conj(q[ch_a1[g]], q[ch_b1[g]]),
                             cmul_conj(q[ch_a0[g] + 4], q[ch_b0[g] + 4]),
                             cmul_conj(q[ch_a1[g] + 4], q[ch_b1[g] + 4])};
        unsigned ah[4], al[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (X3) {
            split_h2(v[e], ah[e], al[e]);
          } else {
            const __half2 h = __floats2half2_rn(v[e].x, v[e].y);
            ah[e] = *reinterpret_cast<const unsigned*>(&h);
          }
        }
#pragma unroll
        for (int t = 0; t < NTM; ++t) {
          if (t < NT) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            if (X3) {
              mma_16816(c, al, b[t].x, b[t].y);
              mma_16816(c, ah, b[t].z, b[t].w);
            }
            mma_16816(c, ah, b[t].x, b[t].y);
#pragma unroll
            for (int e = 0; e < 4; ++e) sum[g][t][e] += c[e];
          }
        }
      }
    }
    __syncthreads();  // stage i's buffer may be refilled (by stage i + 2)
    if (c + 1 < nch) continue;
    // the round is complete.  d fragments: (row gq, cols 2tq, 2tq+1) and (row gq + 8,
    // same); column c is lag c - nq0
#pragma unroll
    for (int g = 0; g < MTW; ++g) {
      if (r0 + g * 8 + warp >= MT) continue;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = (r0 + g * 8 + warp) * 16 + gq + 8 * h;
        if (r >= P) continue;
        const int nq = __ldg(Np + r);
        const size_t o = orow + __ldg(off + r) + nq;  // lag 0 of pair r
#pragma unroll
        for (int t = 0; t < NTM; ++t) {
          if (t >= NT) continue;
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int n = t * 8 + 2 * tq + cc - nq0;
            if (n >= -nq && n <= nq) put_op_rt(ot, out, out_lo, o + n, sum[g][t][2 * h + cc]);
          }
        }
      }
    }
  }
  for (int c = L + tid; c < out_cols; c += 256) put_op_rt(ot, out, out_lo, orow + c, 0.f);
}

size_t gcc_mma_smem_bytes(int M, int max_Np) {  // two stage buffers
  return 2 * (sizeof(float2) * static_cast<size_t>(M) * kMmaRow +
              sizeof(uint4) * (kMmaChunk / 8) * front_ntiles(max_Np) * 32);
}

bool gcc_mma_supported(int M, int N, int max_Np) {
  return N >= 2 * kMmaChunk && (N / 2) % kMmaChunk == 0 && max_Np <= gcc_direct_max_lag() &&
         gcc_mma_smem_bytes(M, max_Np) <= 200 * 1024;
}

cudaError_t launch_gcc_mma(const float2* yhat, int F, int M, int P, int N, const int2* pairs,
                           const int* Np, const int* off, int L, const uint4* stab, int max_Np,
                           OpType t, void* out, void* out_lo, int out_cols, cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  if (!gcc_mma_supported(M, N, max_Np) || out_cols < L) return cudaErrorInvalidValue;
  const int NT = front_ntiles(max_Np), NTM = front_ntm(max_Np);
  const size_t smem = gcc_mma_smem_bytes(M, max_Np);
  // FP32-class operands (FP32 and the hi + lo types) sample with the three products of
  // the hi + lo split (22 significant bits); single 16-bit and TF32 operands, which keep 8
  // to 11 bits of each sample, with the one product of FP16 psi and table
  const bool x3 = t == OpType::F32 || op_split(t);
  void (*kern)(const float2*, int, int, int, const int2*, const int*, const int*, int,
               const uint4*, int, int, int, void*, void*, int) =
      x3 ? (NTM == 2 ? gcc_mma_kernel<2, true> : NTM == 4 ? gcc_mma_kernel<4, true> : gcc_mma_kernel<9, true>)
         : (NTM == 2 ? gcc_mma_kernel<2, false> : NTM == 4 ? gcc_mma_kernel<4, false> : gcc_mma_kernel<9, false>);
  cudaError_t e = allow_max_dynamic_smem(kern);
  if (e != cudaSuccess) return e;
  kern<<<F, 256, smem, s>>>(yhat, M, P, N / 2, pairs, Np, off, L, stab, NT, max_Np,
                            static_cast<int>(t), out, out_lo, out_cols);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Sampling by iFFT for 2K = 1024 on the warp-level tensor cores, for operands that keep 8
// to 11 bits (BF16, FP16, TF32 plans).  Each warp takes one complex transform of length
// 1024 (two pairs, as gcc_samples_kernel: psi-bar_a + i psi-bar_b, two-sided and Hermitian,
// so the inverse transform is xi-bar_a + i xi-bar_b) and splits it as 32 x 32
// (Cooley-Tukey: input index 32 n1 + n2, output index k1 + 32 k2):
//   Y[k1][n2] = sum_n1 e^{+2 pi i k1 n1 / 32} x[32 n1 + n2]        (real-form GEMM 64x64x32)
//   Y[k1][n2] *= e^{+2 pi i k1 n2 / 1024}                           (twiddles)
//   x-bar[k1 + 32 k2] = sum_n2 Y[k1][n2] e^{+2 pi i n2 k2 / 32}    (real-form GEMM 32x64x64)
// on mma.sync m16n8k16 with FP16 operands and FP32 accumulation; the first product's
// accumulators become the second's A fragments in registers.  One CTA of 256 threads per
// frame stages the frame's spectra (rows padded 4 entries per 64 bins: the fragments'
// gathers hit distinct banks) and the DFT tables (dft_tables) in shared memory.  Samples
// are written in the operand type, zero padded beyond L.
// ---------------------------------------------------------------------------------
constexpr int kDftRow = 512 + 32;  // padded spectrum row (float2)
constexpr int kTwRow = 36;         // twiddle row (float2): the 8 rows of a gather hit distinct banks
constexpr int kDftTables = 512 + 512 + 32 * kTwRow / 2;  // uint4: A of step 1, B of step 2, twiddles
__device__ __forceinline__ int dft_bin(int k) { return k + 4 * (k >> 6); }

// f16 pair (x in the lower half)
__device__ __forceinline__ unsigned pack_h2(float x, float y) {
  const __half2 h = __floats2half2_rn(x, y);
  return *reinterpret_cast<const unsigned*>(&h);
}

template <typename T>
__global__ __launch_bounds__(256, 2) void gcc_dft1024_kernel(
    const float2* __restrict__ yhat, int M, int P, const int2* __restrict__ pairs,
    const int* __restrict__ Np, const int* __restrict__ off, int L,
    const uint4* __restrict__ tables, void* out, int out_cols) {
  constexpr int K = 512, NFFT = 1024;
  extern __shared__ float2 dsm[];
  float2* ys = dsm;                                          // [M][kDftRow]
  uint4* ta = reinterpret_cast<uint4*>(ys + M * kDftRow);     // A of step 1: [4 i][4 s][32] uint4
  uint2* tb = reinterpret_cast<uint2*>(ta + 512);             // B of step 2: [4 q][8 j][32] uint2
  float2* tw = reinterpret_cast<float2*>(tb + 1024);          // [32 k1][kTwRow: 32 n2 + pad]
  const int f = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  {
    const float4* src = reinterpret_cast<const float4*>(yhat + static_cast<size_t>(f) * M * K);
    for (int e = tid; e < M * (K / 2); e += 256) {  // two bins per float4
      const int m = e / (K / 2), j = e - m * (K / 2);
      *reinterpret_cast<float4*>(ys + m * kDftRow + dft_bin(2 * j)) = __ldg(src + e);
    }
    for (int e = tid; e < kDftTables; e += 256) ta[e] = __ldg(tables + e);
  }
  __syncthreads();
  const size_t orow = static_cast<size_t>(f) * out_cols;
  const int ntr = (P + 1) >> 1;
  for (int tr = warp; tr < ntr; tr += 8) {
    const int pa = 2 * tr, pb = pa + 1;
    const bool hasb = pb < P;
    const int2 qa = __ldg(pairs + pa);
    const int2 qb = hasb ? __ldg(pairs + pb) : qa;
    const int ya0 = qa.x * kDftRow, ya1 = qa.y * kDftRow;  // spectrum rows in ys
    const int yb0 = qb.x * kDftRow, yb1 = qb.y * kDftRow;
    // B fragments of step 1: rows 0..31 Re x[32 n1 + n2], rows 32..63 Im (n1 = row mod 32),
    // columns n2; this thread holds n1 = 16 s + 2 t + {0, 1, 8, 9}, n2 = 8 j + g
    unsigned b1[4][4][2];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float re[4], im[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int n1 = 16 * s + 2 * t + (e & 1) + 8 * (e >> 1);
          const int k = 32 * n1 + 8 * j + g;  // bin of the two-sided spectrum
          const int kk = k <= K ? k : NFFT - k;
          float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
          if (kk != 0 && kk != K) {
            const int o = dft_bin(kk);
            a = cmul_conj(ys[ya0 + o], ys[ya1 + o]);
            if (hasb) b = cmul_conj(ys[yb0 + o], ys[yb1 + o]);
          }
          // psi_a + i psi_b below the Nyquist bin, psi_a^* + i psi_b^* above it
          re[e] = k <= K ? a.x - b.y : a.x + b.y;
          im[e] = k <= K ? a.y + b.x : b.x - a.y;
        }
        b1[s][j][0] = pack_h2(re[0], re[1]);
        b1[s][j][1] = pack_h2(re[2], re[3]);
        b1[s + 2][j][0] = pack_h2(im[0], im[1]);
        b1[s + 2][j][1] = pack_h2(im[2], im[3]);
      }
    // step 1: C1 [64 rows: Re Y (k1), Im Y (k1)][32 cols: n2], for k1 = 16 r .. 16 r + 15 at
    // a time (m-tiles r and r + 2: the real and imaginary parts of the same rows); then the
    // twiddles and the A fragments of step 2: rows k1, columns [Re Y (n2) | Im Y (n2)]
    unsigned a2[2][4][4];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      float c1[2][4][4];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
          for (int e = 0; e < 4; ++e) c1[u][j][e] = 0.f;
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint4 av = ta[((r + 2 * u) * 4 + s) * 32 + lane];
          const unsigned a[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) mma_16816(c1[u][j], a, b1[s][j][0], b1[s][j][1]);
        }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float yr[4], yi[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k1 = 16 * r + g + 8 * (e >> 1), n2 = 8 * j + 2 * t + (e & 1);
          const float2 w = tw[k1 * kTwRow + n2];
          const float xr = c1[0][j][e], xi = c1[1][j][e];
          yr[e] = xr * w.x - xi * w.y;
          yi[e] = xr * w.y + xi * w.x;
        }
        // n-tile j (columns 8 j ..) is half of k-step j / 2 (Re) or 2 + j / 2 (Im)
        const int q = j >> 1, h = (j & 1) * 2;
        a2[r][q][h] = pack_h2(yr[0], yr[1]);
        a2[r][q][h + 1] = pack_h2(yr[2], yr[3]);
        a2[r][q + 2][h] = pack_h2(yi[0], yi[1]);
        a2[r][q + 2][h + 1] = pack_h2(yi[2], yi[3]);
      }
    }
    // step 2: C2 [32 rows k1][64 cols: Re Z (k2), Im Z (k2)]; x-bar[k1 + 32 k2] = Z[k1][k2]
    const int na = __ldg(Np + pa), nb = hasb ? __ldg(Np + pb) : -1;
    const size_t oa = orow + __ldg(off + pa) + na;          // lag 0 of pair a
    const size_t ob = hasb ? orow + __ldg(off + pb) + nb : 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      // n-tile j holds output indices 256 (j mod 4) .. + 255 of pair a (j < 4) or b: lags
      // 0..255, 256..511, -512..-257, -256..-1; windows narrower than 256 skip the middle two
      const int nq = j < 4 ? na : nb, jj = j & 3;
      if (nq < 0 || (jj == 1 && nq < 256) || (jj == 2 && nq < 257)) continue;  // warp-uniform
      float c2[2][4];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int e = 0; e < 4; ++e) c2[r][e] = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint2 bv = tb[(q * 8 + j) * 32 + lane];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          // A fragment order: (row g, k 2t..), (row g+8, k 2t..), (row g, k 2t+8..), (row g+8, k 2t+8..)
          const unsigned a[4] = {a2[r][q][0], a2[r][q][1], a2[r][q][2], a2[r][q][3]};
          mma_16816(c2[r], a, bv.x, bv.y);
        }
      }
      // columns 8 j + 2 t (+1): Re Z for j < 4 (pair a), Im Z for j >= 4 (pair b)
      const size_t o = j < 4 ? oa : ob;
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k1 = 16 * r + g + 8 * (e >> 1);
          const int k2 = 8 * (j & 3) + 2 * t + (e & 1);
          const int idx = k1 + 32 * k2;
          const int n = idx < K ? idx : idx - NFFT;  // lag (Eq. n_prime)
          if (n >= -nq && n <= nq) op_store<T, false>(out, nullptr, o + n, c2[r][e]);
        }
    }
  }
  for (int c = L + tid; c < out_cols; c += 256) op_store<T, false>(out, nullptr, orow + c, 0.f);
}

size_t gcc_dft_smem_bytes(int M) {
  return sizeof(float2) * static_cast<size_t>(M) * kDftRow + sizeof(uint4) * kDftTables;
}

bool gcc_dft_supported(int M, int N, OpType t) {
  const bool narrow = t == OpType::BF16 || t == OpType::F16 || t == OpType::TF32;
  return narrow && N == 1024 && gcc_dft_smem_bytes(M) <= 110 * 1024;
}

// Host tables of gcc_dft1024_kernel: A of step 1 (the real form [[C, -S], [S, C]] of
// e^{+2 pi i k1 n1 / 32}) in m16n8k16 A-fragment order [4][4][32] uint4, B of step 2 ([[C, S],
// [-S, C]] of e^{+2 pi i n2 k2 / 32}) in B-fragment order [4][8][32] uint2, and the twiddles
// e^{+2 pi i k1 n2 / 1024} [32][kTwRow] float2: kDftTables uint4 in all.
void dft_tables(std::vector<uint4>& tab) {
  tab.assign(kDftTables, make_uint4(0, 0, 0, 0));
  auto h = [](double v) {
    const __half_raw r(__float2half_rn(static_cast<float>(v)));
    return static_cast<unsigned>(r.x);
  };
  auto pk = [&](double lo, double hi) { return h(lo) | (h(hi) << 16); };
  auto cs = [](int a, int b, int n, double& c, double& sn) {
    const long long u = (static_cast<long long>(a) * b) % n;  // exact angle reduction
    const double th = 2.0 * M_PI * static_cast<double>(u) / n;
    c = std::cos(th);
    sn = std::sin(th);
  };
  auto A1 = [&](int row, int col) {  // rows: Re out (k1), Im out; cols: Re in (n1), Im in
    double c, sn;
    cs(row & 31, col & 31, 32, c, sn);
    const int rb = row >> 5, cb = col >> 5;
    return rb == cb ? c : (rb == 0 ? -sn : sn);
  };
  auto B2 = [&](int row, int col) {  // rows: Re Y (n2), Im Y; cols: Re Z (k2), Im Z
    double c, sn;
    cs(row & 31, col & 31, 32, c, sn);
    const int rb = row >> 5, cb = col >> 5;
    return rb == cb ? c : (rb == 0 ? sn : -sn);
  };
  for (int i = 0; i < 4; ++i)
    for (int s = 0; s < 4; ++s)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, t = lane & 3, r0 = 16 * i + g, c0 = 16 * s + 2 * t;
        uint4& e = tab[(i * 4 + s) * 32 + lane];
        e.x = pk(A1(r0, c0), A1(r0, c0 + 1));
        e.y = pk(A1(r0 + 8, c0), A1(r0 + 8, c0 + 1));
        e.z = pk(A1(r0, c0 + 8), A1(r0, c0 + 9));
        e.w = pk(A1(r0 + 8, c0 + 8), A1(r0 + 8, c0 + 9));
      }
  uint2* tb = reinterpret_cast<uint2*>(tab.data() + 512);
  for (int q = 0; q < 4; ++q)
    for (int j = 0; j < 8; ++j)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, t = lane & 3, k0 = 16 * q + 2 * t, n = 8 * j + g;
        uint2& e = tb[(q * 8 + j) * 32 + lane];
        e.x = pk(B2(k0, n), B2(k0 + 1, n));
        e.y = pk(B2(k0 + 8, n), B2(k0 + 9, n));
      }
  float2* tw = reinterpret_cast<float2*>(tab.data() + 1024);
  for (int k1 = 0; k1 < 32; ++k1)
    for (int n2 = 0; n2 < 32; ++n2) {
      double c, sn;
      cs(k1, n2, 1024, c, sn);
      tw[k1 * kTwRow + n2] = make_float2(static_cast<float>(c), static_cast<float>(sn));
    }
}

cudaError_t launch_gcc_dft(const float2* yhat, int F, int M, int P, int N, const int2* pairs,
                           const int* Np, const int* off, int L, const uint4* tables, OpType t,
                           void* out, void* out_lo, int out_cols, cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  if (!gcc_dft_supported(M, N, t) || out_cols < L) return cudaErrorInvalidValue;
  (void)out_lo;  // single-plane operand types only
  const size_t smem = gcc_dft_smem_bytes(M);
  void (*kern)(const float2*, int, int, const int2*, const int*, const int*, int, const uint4*,
               void*, int) = t == OpType::BF16 ? gcc_dft1024_kernel<__nv_bfloat16>
                            : t == OpType::F16 ? gcc_dft1024_kernel<__half>
                                               : gcc_dft1024_kernel<tf32_t>;
  cudaError_t e = allow_max_dynamic_smem(kern);
  if (e != cudaSuccess) return e;
  kern<<<F, 256, smem, s>>>(yhat, M, P, pairs, Np, off, L, tables, out, out_cols);
  return cudaGetLastError();
}

// One CTA of 256 threads per frame; H = N/2 is the complex FFT length (= K), NTM bounds
// the n-tiles of the sampling GEMM.
template <int H, int NTM>
__device__ __forceinline__ void front_body(const FrontParams& a, const int f) {
  extern __shared__ float2 sm[];
  constexpr int N = 2 * H, K = H, KS = front_row(K);
  constexpr int Tg = H / 8;              // threads per channel group (radix-8 FFT)
  constexpr int groups = 256 / Tg;       // channels transformed at once
  constexpr int NW = 8;                  // warps
  const int M = a.M;
  float2* tw = sm;                                   // H
  float2* yh = tw + H;                               // M*KS
  float2* fbuf = yh + static_cast<size_t>(M) * KS;   // FFT buffers / GEMM partials
  float* xis = reinterpret_cast<float*>(fbuf) + a.fbuf_floats;  // L
  const int tid = threadIdx.x;
  for (int t = tid; t < H; t += 256) tw[t] = a.twiddle[t];
  // each thread owns the complex samples j + i Tg (i = 0..7) of its group's channel
  const int grp = tid / Tg, j = tid - grp * Tg;
  float2* bufA = fbuf + grp * 2 * fpad_len(H);
  float2* bufB = bufA + fpad_len(H);
  float2 tw3[P8<H>::NTW > 0 ? P8<H>::NTW : 1][3];
  p8_twiddles<H, 1, false>(a.twiddle, j, tw3);
  const float2* w2 = reinterpret_cast<const float2*>(a.window);
  for (int m0 = 0; m0 < M; m0 += groups) {
    const int m = m0 + grp;
    const float2* x2 = reinterpret_cast<const float2*>(a.frames + (static_cast<size_t>(f) * M + (m < M ? m : 0)) * N);
    float2 xv[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) xv[i] = m < M ? __ldg(x2 + j + i * Tg) : make_float2(0.f, 0.f);
    __syncthreads();  // twiddles ready / previous round's buffers consumed
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float2 ww = __ldg(w2 + j + i * Tg);
      bufA[fpad(j + i * Tg)] = make_float2(xv[i].x * ww.x, xv[i].y * ww.y);
    }
    __syncthreads();
    // every thread of the block takes part in the FFT's barriers
    const float2* Z = p8fft<H, false>(bufA, bufB, j, tw3);
    if (m < M) {
      // real spectrum from the packed transform, then PHAT
      float2* out = yh + static_cast<size_t>(m) * KS;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = j + i * Tg;
        const float2 zk = Z[fpad(k)];
        const float2 zr = Z[fpad((H - k) & (H - 1))];
        const float2 zc = make_float2(zr.x, -zr.y);
        const float2 E = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
        const float2 O = make_float2(0.5f * (zk.y - zc.y), -0.5f * (zk.x - zc.x));
        const float2 WO = cmul(tw[k], O);
        const float2 Y = make_float2(E.x + WO.x, E.y + WO.y);
        const float p = Y.x * Y.x + Y.y * Y.y;
        float2 r = make_float2(0.f, 0.f);
        if (k > 0 && p >= 1e-30f) {
          const float sc = __frsqrt_rn(p);
          r = make_float2(Y.x * sc, Y.y * sc);
        }
        out[k] = r;
      }
    }
  }
  __syncthreads();
  if (a.conv_out) {
    // conv. FD-SRP operand (layout of conv_pack_kernel): per pair, Re psi_p(k) at p N + k and
    // Im psi_p(k) at p N + K + k, k = 0..K-1 (psi(0) = 0: y-hat(0) is zero)
    const size_t row = static_cast<size_t>(f) * a.P * N;
    for (int e = tid; e < a.P * K; e += 256) {
      const int p = e / K, k = e - p * K;
      const int2 pr = __ldg(a.pairs + p);
      const float2 v = cmul_conj(yh[pr.x * KS + k], yh[pr.y * KS + k]);
      put_op_rt(a.ot, a.out, a.out_lo, row + static_cast<size_t>(p) * N + k, v.x);
      put_op_rt(a.ot, a.out, a.out_lo, row + static_cast<size_t>(p) * N + K + k, v.y);
    }
    return;
  }
  // Sampling (Eq. xi_p_ifft at the lags n = -N_p..N_p) as a GEMM per frame: rows = pairs,
  // K = bins 0..K-1 with Re psi and Im psi interleaved, columns j = lags n = j - nq0, and
  // B[2k][j] = 2 cos(pi k n / K), B[2k+1][j] = -2 sin(pi k n / K), so that
  // xi_p(n) = 2 Re sum_k psi_p(k) exp(j pi k n / K).  psi and B in FP16 hi + lo, three
  // products per fragment pair (hi hi, lo hi, hi lo): the dropped lo lo term is below
  // 2^-22 of each product.  Per tile of 16 pairs, warp w sums the k-steps of its eighth of
  // the bins into part[w]; the eight partials are then added in warp order (deterministic).
  const int lane = tid & 31, warp = tid >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  {
    constexpr int NCM = NTM * 8;        // partial row stride
    constexpr int kst = (K / 8) / NW;   // k-steps per warp
    const int MT = (a.P + 15) >> 4;
    const int NT = a.NT;
    float* part = reinterpret_cast<float*>(fbuf);  // [NW][16][NCM]
    for (int mt = 0; mt < MT; ++mt) {
      const int r0 = mt * 16 + gq, r1 = r0 + 8;
      const bool v0 = r0 < a.P, v1 = r1 < a.P;
      const int2 p0 = v0 ? __ldg(a.pairs + r0) : make_int2(0, 0);
      const int2 p1 = v1 ? __ldg(a.pairs + r1) : make_int2(0, 0);
      const int sb = warp * kst;
      const float2* yA0 = yh + p0.x * KS + sb * 8 + tq;
      const float2* yB0 = yh + p0.y * KS + sb * 8 + tq;
      const float2* yA1 = yh + p1.x * KS + sb * 8 + tq;
      const float2* yB1 = yh + p1.y * KS + sb * 8 + tq;
      const uint4* bt = a.stab + static_cast<size_t>(sb) * NT * 32 + lane;
      // hi x hi and the two lo products in separate accumulators (independent chains),
      // except for many n-tiles (register budget)
      constexpr bool SA = NTM <= 4;
      float acc[NTM][4], accl[SA ? NTM : 1][4];
#pragma unroll
      for (int t = 0; t < NTM; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[t][e] = accl[SA ? t : 0][e] = 0.f;
      // small n-tile counts: the B fragments of the next k-step are loaded one step ahead
      constexpr bool PF = false;
      uint4 bn[PF ? NTM : 1];
      if constexpr (PF) {
#pragma unroll
        for (int t = 0; t < NTM; ++t)
          if (t < NT) bn[t] = __ldg(bt + t * 32);
      }
#pragma unroll(kst <= 4 ? kst : 1)
      for (int s = 0; s < kst; ++s) {
        const float2 zero = make_float2(0.f, 0.f);
        unsigned ah[4], al[4];
        split_h2(v0 ? cmul_conj(yA0[8 * s], yB0[8 * s]) : zero, ah[0], al[0]);
        split_h2(v1 ? cmul_conj(yA1[8 * s], yB1[8 * s]) : zero, ah[1], al[1]);
        split_h2(v0 ? cmul_conj(yA0[8 * s + 4], yB0[8 * s + 4]) : zero, ah[2], al[2]);
        split_h2(v1 ? cmul_conj(yA1[8 * s + 4], yB1[8 * s + 4]) : zero, ah[3], al[3]);
        uint4 bc[PF ? NTM : 1];
        if constexpr (PF) {
#pragma unroll
          for (int t = 0; t < NTM; ++t) {
            bc[t] = bn[t];
            if (t < NT && s + 1 < kst) bn[t] = __ldg(bt + (s + 1) * NT * 32 + t * 32);
          }
        }
#pragma unroll
        for (int t = 0; t < NTM; ++t) {
          if (t < NT) {
            const uint4 b = PF ? bc[PF ? t : 0] : __ldg(bt + s * NT * 32 + t * 32);
            float(&dl)[4] = SA ? accl[SA ? t : 0] : acc[t];
            mma_16816(dl, al, b.x, b.y);
            mma_16816(dl, ah, b.z, b.w);
            mma_16816(acc[t], ah, b.x, b.y);
          }
        }
      }
      if constexpr (SA) {
#pragma unroll
        for (int t = 0; t < NTM; ++t)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[t][e] += accl[SA ? t : 0][e];
      }
      float* pw = part + warp * 16 * NCM;
#pragma unroll
      for (int t = 0; t < NTM; ++t) {
        if (t < NT) {
          const int c = t * 8 + 2 * tq;
          *reinterpret_cast<float2*>(pw + gq * NCM + c) = make_float2(acc[t][0], acc[t][1]);
          *reinterpret_cast<float2*>(pw + (gq + 8) * NCM + c) = make_float2(acc[t][2], acc[t][3]);
        }
      }
      __syncthreads();
      for (int e = tid; e < 16 * NCM; e += 256) {
        const int rr = e / NCM, c = e - rr * NCM;
        const int r = mt * 16 + rr, n = c - a.nq0;
        if (r >= a.P || c >= NT * 8) continue;
        const int nq = __ldg(a.Np + r);
        if (abs(n) > nq) continue;
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) v += part[w * 16 * NCM + e];
        xis[__ldg(a.off + r) + nq + n] = v;
      }
      __syncthreads();
    }
  }
  const size_t row = static_cast<size_t>(f) * a.out_cols;
  if (!a.ftab) {
    for (int l = tid; l < a.out_cols; l += 256)
      put_op_rt(a.ot, a.out, a.out_lo, row + l, l < a.L ? xis[l] : 0.f);
    return;
  }
  // u = Lambda_fat xi on the warp-level tensor cores: A = Lambda_fat tiles of 16 rows x 16
  // samples (fragment table, FP16 hi + lo), B = xi as column 0 (FP16 hi + lo, columns 1..7
  // zero); warp w takes the k-steps w, w + 8, ...; partials added in warp order.
  {
    const int MTf = (a.Rp + 15) >> 4, KSf = (a.L + 15) >> 4;
    float* part = reinterpret_cast<float*>(fbuf);  // [NW][MTf * 16]
    for (int mt = 0; mt < MTf; ++mt) {
      float d[4] = {0.f, 0.f, 0.f, 0.f}, dl[4] = {0.f, 0.f, 0.f, 0.f};
      for (int s = warp; s < KSf; s += NW) {
        const uint4* fa = a.ftab + ((static_cast<size_t>(mt) * KSf + s) * 32 + lane) * 2;
        const uint4 h = __ldg(fa), l = __ldg(fa + 1);
        unsigned bh0 = 0u, bl0 = 0u, bh1 = 0u, bl1 = 0u;
        if (gq == 0) {
          const int l0 = s * 16 + 2 * tq;
          split_h2(make_float2(l0 < a.L ? xis[l0] : 0.f, l0 + 1 < a.L ? xis[l0 + 1] : 0.f), bh0, bl0);
          split_h2(make_float2(l0 + 8 < a.L ? xis[l0 + 8] : 0.f, l0 + 9 < a.L ? xis[l0 + 9] : 0.f), bh1, bl1);
        }
        const unsigned ah[4] = {h.x, h.y, h.z, h.w}, al[4] = {l.x, l.y, l.z, l.w};
        mma_16816(dl, al, bh0, bh1);
        mma_16816(dl, ah, bl0, bl1);
        mma_16816(d, ah, bh0, bh1);
      }
      if (tq == 0) {
        part[warp * MTf * 16 + mt * 16 + gq] = d[0] + dl[0];
        part[warp * MTf * 16 + mt * 16 + gq + 8] = d[2] + dl[2];
      }
    }
    __syncthreads();
    for (int r = tid; r < a.out_cols; r += 256) {
      float u = 0.f;
      if (r < a.Rp) {
#pragma unroll
        for (int w = 0; w < NW; ++w) u += part[w * MTf * 16 + r];
      }
      put_op_rt(a.ot, a.out, a.out_lo, row + r, u * a.scale);
    }
  }
}

template <int H, int NTM>
__global__ __launch_bounds__(256, NTM <= 2 ? 4 : NTM <= 4 ? 3 : 2) void front_kernel(const FrontParams a) {
  front_body<H, NTM>(a, blockIdx.x);
}

// Grouped front end (serving): items[i] = (index into params, frame within that list
// entry's batch); blocks walk the items the host counted (*count), so one launch serves the
// frames of many sessions.  Every session in a launch shares H and NTM; the dynamic shared
// memory covers the largest of them.
template <int H, int NTM>
__global__ __launch_bounds__(256, NTM <= 2 ? 4 : NTM <= 4 ? 3 : 2) void front_group_kernel(
    const FrontParams* __restrict__ params, const int2* __restrict__ items,
    const int* __restrict__ count) {
  const int n = *count;
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int2 it = items[i];
    const FrontParams a = params[it.x];
    front_body<H, NTM>(a, it.y);
    __syncthreads();  // the next item reuses the shared memory
  }
}

cudaError_t launch_front_group(const FrontParams* params, const int2* items, const int* count,
                               int grid, int N, int NTM, size_t smem, cudaStream_t s) {
  const int H = N / 2;
  void (*kern)(const FrontParams*, const int2*, const int*) = nullptr;
#define SRP_FRONT_G(HV, NTV) if (H == HV && NTM == NTV) kern = front_group_kernel<HV, NTV>;
  SRP_FRONT_G(128, 2) SRP_FRONT_G(128, 4) SRP_FRONT_G(128, 9)
  SRP_FRONT_G(256, 2) SRP_FRONT_G(256, 4) SRP_FRONT_G(256, 9)
  SRP_FRONT_G(512, 2) SRP_FRONT_G(512, 4) SRP_FRONT_G(512, 9)
#undef SRP_FRONT_G
  if (!kern || grid < 1) return cudaErrorInvalidValue;
  cudaError_t e = allow_max_dynamic_smem(kern);
  if (e != cudaSuccess) return e;
  kern<<<grid, 256, smem, s>>>(params, items, count);
  return cudaGetLastError();
}

// The parameters launch_front would pass (the caller fills frames and out per batch).
FrontParams front_params(int M, int N, const float* window, const float2* twiddle, int P,
                         const int2* pairs, const int* Np, const int* off, const uint4* stab,
                         int L, int max_Np, const uint4* ftab, int Rp, int out_cols, float scale,
                         OpType t, int NTM) {
  const int H = N / 2, groups = 256 / (H / 8);
  if (NTM < front_ntm(max_Np)) NTM = front_ntm(max_Np);
  const int fbuf_floats = std::max(4 * groups * fpad_len(H), 8 * 16 * 8 * NTM);
  return FrontParams{nullptr, M, P, L, window, twiddle, pairs, Np, off, stab, max_Np,
                     front_ntiles(max_Np), fbuf_floats, ftab, Rp, out_cols, scale,
                     static_cast<int>(t), nullptr, nullptr, 0};
}

int front_max_N() { return 1024; }

int front_ntiles(int max_Np) { return (2 * max_Np + 1 + 7) / 8; }

// n-tile bucket of the kernel instantiation (its partial rows hold 8 NTM floats)
int front_ntm(int max_Np) {
  const int NT = front_ntiles(max_Np);
  return NT <= 2 ? 2 : NT <= 4 ? 4 : 9;
}

void front_sampling_table(int N, int max_Np, std::vector<uint4>& tab) {
  const int K = N / 2, KST = K / 8, NT = front_ntiles(max_Np);
  tab.assign(static_cast<size_t>(KST) * NT * 32, make_uint4(0, 0, 0, 0));
  // (2 cos(pi k n / K), -2 sin(pi k n / K)) as FP16 hi and lo pairs, angle reduced exactly
  auto entry = [&](int k, int n, unsigned& hi, unsigned& lo) {
    double c = 0.0, sn = 0.0;
    if (k > 0) {
      const long long u = ((static_cast<long long>(k) * n) % (2 * K) + 2 * K) % (2 * K);
      const double th = M_PI * static_cast<double>(u) / K;
      c = 2.0 * std::cos(th);
      sn = -2.0 * std::sin(th);
    }
    const __half hc = __float2half_rn(static_cast<float>(c));
    const __half hs = __float2half_rn(static_cast<float>(sn));
    const __half lc = __float2half_rn(static_cast<float>(c - static_cast<double>(__half2float(hc))));
    const __half ls = __float2half_rn(static_cast<float>(sn - static_cast<double>(__half2float(hs))));
    const __half_raw rhc(hc), rhs(hs), rlc(lc), rls(ls);
    hi = static_cast<unsigned>(rhc.x) | (static_cast<unsigned>(rhs.x) << 16);
    lo = static_cast<unsigned>(rlc.x) | (static_cast<unsigned>(rls.x) << 16);
  };
  for (int s = 0; s < KST; ++s)
    for (int t = 0; t < NT; ++t)
      for (int lane = 0; lane < 32; ++lane) {
        const int col = t * 8 + (lane >> 2), tq = lane & 3;
        if (col >= 2 * max_Np + 1) continue;
        const int n = col - max_Np;
        uint4& e = tab[(static_cast<size_t>(s) * NT + t) * 32 + lane];
        entry(s * 8 + tq, n, e.x, e.z);
        entry(s * 8 + tq + 4, n, e.y, e.w);
      }
}

// twiddles, y-hat rows, FFT buffers (reused for the sampling partials of 8 warps), xi
void front_fat_table(const float* fat, int Rp, int L, std::vector<uint4>& tab) {
  const int MTf = (Rp + 15) / 16, KSf = (L + 15) / 16;
  tab.assign(static_cast<size_t>(MTf) * KSf * 32 * 2, make_uint4(0, 0, 0, 0));
  auto val = [&](int r, int l) { return r < Rp && l < L ? fat[static_cast<size_t>(r) * L + l] : 0.f; };
  auto pack = [](float x, float y, unsigned& hi, unsigned& lo) {
    const __half hx = __float2half_rn(x), hy = __float2half_rn(y);
    const __half lx = __float2half_rn(x - __half2float(hx)), ly = __float2half_rn(y - __half2float(hy));
    const __half_raw rhx(hx), rhy(hy), rlx(lx), rly(ly);
    hi = static_cast<unsigned>(rhx.x) | (static_cast<unsigned>(rhy.x) << 16);
    lo = static_cast<unsigned>(rlx.x) | (static_cast<unsigned>(rly.x) << 16);
  };
  for (int mt = 0; mt < MTf; ++mt)
    for (int s = 0; s < KSf; ++s)
      for (int lane = 0; lane < 32; ++lane) {
        const int r0 = mt * 16 + (lane >> 2), r1 = r0 + 8;
        const int c0 = s * 16 + 2 * (lane & 3), c1 = c0 + 8;
        uint4* e = &tab[((static_cast<size_t>(mt) * KSf + s) * 32 + lane) * 2];
        pack(val(r0, c0), val(r0, c0 + 1), e[0].x, e[1].x);
        pack(val(r1, c0), val(r1, c0 + 1), e[0].y, e[1].y);
        pack(val(r0, c1), val(r0, c1 + 1), e[0].z, e[1].z);
        pack(val(r1, c1), val(r1, c1 + 1), e[0].w, e[1].w);
      }
}

size_t front_smem_bytes_ntm(int M, int N, int L, int NTM) {
  const int H = N / 2, Tg = H / 8;
  const int groups = 256 / Tg;
  const size_t fbuf = std::max(sizeof(float2) * groups * 2 * fpad_len(H),
                               sizeof(float) * 8 * 16 * 8 * NTM);
  return sizeof(float2) * (H + static_cast<size_t>(M) * front_row(H)) + fbuf + sizeof(float) * L;
}

size_t front_smem_bytes(int M, int N, int L, int max_Np) {
  return front_smem_bytes_ntm(M, N, L, front_ntm(max_Np));
}

bool front_supported(int M, int N, int L, int max_Np) {
  return N >= 256 && N <= front_max_N() && max_Np <= gcc_direct_max_lag() &&
         front_smem_bytes(M, N, L, max_Np) <= 200 * 1024;
}

static cudaError_t front_launch(const FrontParams& a, int F, int N, int NTM, size_t smem,
                                cudaStream_t s);

cudaError_t launch_front(const float* frames, int F, int M, int N, const float* window,
                         const float2* twiddle, int P, const int2* pairs, const int* Np,
                         const int* off, const uint4* stab, int L, int max_Np, const uint4* ftab,
                         int Rp, int out_cols, float scale, OpType t, void* out, void* out_lo,
                         cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  if (!front_supported(M, N, L, max_Np)) return cudaErrorNotSupported;
  const int NT = front_ntiles(max_Np);
  const int H = N / 2, groups = 256 / (H / 8);
  const int NTM = front_ntm(max_Np);
  const int fbuf_floats = std::max(4 * groups * fpad_len(H), 8 * 16 * 8 * NTM);
  const int ot = static_cast<int>(t);
  FrontParams a{frames, M, P, L, window, twiddle, pairs, Np, off, stab, max_Np, NT,
                fbuf_floats, ftab, Rp, out_cols, scale, ot, out, out_lo, 0};
  return front_launch(a, F, N, front_ntm(max_Np), front_smem_bytes(M, N, L, max_Np), s);
}

bool front_conv_supported(int M, int N) { return front_supported(M, N, 0, 0); }

cudaError_t launch_front_conv(const float* frames, int F, int M, int N, const float* window,
                              const float2* twiddle, int P, const int2* pairs, OpType t, void* A,
                              void* A_lo, cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  if (!front_conv_supported(M, N)) return cudaErrorNotSupported;
  const int H = N / 2, groups = 256 / (H / 8);
  FrontParams a{frames, M, P, 0, window, twiddle, pairs, nullptr, nullptr, nullptr, 0, 1,
                std::max(4 * groups * fpad_len(H), 8 * 16 * 8 * 2), nullptr, 0, 0, 1.f,
                static_cast<int>(t), A, A_lo, 1};
  return front_launch(a, F, N, 2, front_smem_bytes(M, N, 0, 0), s);
}

static cudaError_t front_launch(const FrontParams& a, int F, int N, int NTM, size_t smem,
                                cudaStream_t s) {
  const int H = N / 2;
  // one dispatch table entry per (FFT length, n-tile bucket)
  void (*kern)(const FrontParams) = nullptr;
#define SRP_FRONT(HV, NTV) if (H == HV && NTM == NTV) kern = front_kernel<HV, NTV>;
  SRP_FRONT(128, 2) SRP_FRONT(128, 4) SRP_FRONT(128, 9)
  SRP_FRONT(256, 2) SRP_FRONT(256, 4) SRP_FRONT(256, 9)
  SRP_FRONT(512, 2) SRP_FRONT(512, 4) SRP_FRONT(512, 9)
#undef SRP_FRONT
  if (!kern) return cudaErrorInvalidValue;
  cudaError_t e = allow_max_dynamic_smem(kern);
  if (e != cudaSuccess) return e;
  kern<<<F, 256, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Streaming front: frames from consecutive hops with overlap state.  The concatenation
// [hist (N - hop samples per channel) | hop 0 | hop 1 | ... | hop B-1] is cut into B frames
// of N samples with stride hop; the last N - hop samples become the next history.
// hops: [B][M][hop]; hist_in / hist_out: [M][N - hop]; frames: [B][M][N].
// ---------------------------------------------------------------------------------
__global__ void stream_frames_kernel(const float* __restrict__ hops, int B, int M, int hop, int N,
                                     const float* __restrict__ hist_in, float* __restrict__ frames,
                                     float* __restrict__ hist_out) {
  const int Hn = N - hop;
  const size_t total = static_cast<size_t>(B) * M * N;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int n = static_cast<int>(e % N);
    const size_t bm = e / N;
    const int m = static_cast<int>(bm % M);
    const int b = static_cast<int>(bm / M);
    const long long c = static_cast<long long>(b) * hop + n;  // index in the concatenation
    float v;
    if (c < Hn) {
      v = hist_in[static_cast<size_t>(m) * Hn + c];
    } else {
      const long long h = c - Hn;
      v = hops[(static_cast<size_t>(h / hop) * M + m) * hop + (h % hop)];
    }
    frames[e] = v;
  }
  // new history: concatenation positions [B hop, B hop + Hn)
  const size_t th = static_cast<size_t>(M) * Hn;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < th;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int m = static_cast<int>(e / Hn);
    const long long c = static_cast<long long>(B) * hop + static_cast<long long>(e % Hn);
    float v;
    if (c < Hn) {
      v = hist_in[static_cast<size_t>(m) * Hn + c];
    } else {
      const long long h = c - Hn;
      v = hops[(static_cast<size_t>(h / hop) * M + m) * hop + (h % hop)];
    }
    hist_out[e] = v;
  }
}

cudaError_t launch_stream_frames(const float* hops, int B, int M, int hop, int N,
                                 const float* hist_in, float* frames, float* hist_out,
                                 cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  size_t total = static_cast<size_t>(B) * M * N;
  int g = static_cast<int>(std::min<size_t>((total + 255) / 256, 152 * 16));
  stream_frames_kernel<<<g, 256, 0, s>>>(hops, B, M, hop, N, hist_in, frames, hist_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// conv. FD-SRP operand A [F][P*N]: row f holds, per pair, Re psi_p(k) at p*N + k and
// Im psi_p(k) at p*N + K + k (k = 0..K-1, psi(0) = 0).  With B[i] = [2cos, -2sin]
// (launch_conv_matrix) the dot product is 2 Re[H_p psi_p] summed over pairs.
// ---------------------------------------------------------------------------------
template <typename T, bool SPLIT>
__global__ void conv_pack_kernel(const float2* __restrict__ yhat, int F, int M, int P, int N,
                                 const int2* __restrict__ pairs, void* __restrict__ A,
                                 void* __restrict__ A_lo) {
  const int K = N >> 1;
  const size_t total = static_cast<size_t>(F) * P * K;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(e % K);
    const size_t fp = e / K;
    const int p = static_cast<int>(fp % P);
    const int f = static_cast<int>(fp / P);
    const int2 q = pairs[p];
    const float2* yf = yhat + static_cast<size_t>(f) * M * K;
    const float2 v = cmul_conj(yf[q.x * K + k], yf[q.y * K + k]);
    const size_t base = (static_cast<size_t>(f) * P + p) * N + k;
    op_store<T, SPLIT>(A, A_lo, base, v.x);
    op_store<T, SPLIT>(A, A_lo, base + K, v.y);
  }
}

static int grid_for(size_t total, int block) {
  size_t g = (total + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

cudaError_t launch_conv_pack(const float2* yhat, int F, int M, int P, int N, const int2* pairs,
                             OpType t, void* A, void* A_lo, cudaStream_t s) {
  if (F <= 0) return cudaSuccess;
  const size_t total = static_cast<size_t>(F) * P * (N / 2);
  const int g = grid_for(total, 256);
  op_dispatch(t, [&](auto tag) {
    using Tag = decltype(tag);
    conv_pack_kernel<typename Tag::type, Tag::split><<<g, 256, 0, s>>>(yhat, F, M, P, N, pairs, A, A_lo);
  });
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// The SRP matrix in GEMM layout, generated once per plan from the FP64 TDOA table:
// theta = 2 pi k tau_p(i) / N with tau in samples (omega_k Delta t = pi k tau / K,
// Eq. w_k), reduced exactly in FP64 to 2 * frac(k tau / N) before sincospi.
// ---------------------------------------------------------------------------------
template <typename T, bool SPLIT>
__global__ void conv_matrix_kernel(const double* __restrict__ tau, int J, int P, int N,
                                   void* __restrict__ B, void* __restrict__ B_lo) {
  const int K = N >> 1;
  const size_t total = static_cast<size_t>(J) * P * K;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int k = static_cast<int>(e % K);
    const size_t ip = e / K;  // i * P + p
    double c = 0.0, sn = 0.0;
    if (k != 0) {
      const double t = static_cast<double>(k) * tau[ip];
      const double r = t - static_cast<double>(N) * floor(t / static_cast<double>(N));
      sincospi(2.0 * r / static_cast<double>(N), &sn, &c);
      c *= 2.0;
      sn *= -2.0;
    }
    const size_t base = ip * N + k;
    op_store_d<T, SPLIT>(B, B_lo, base, c);
    op_store_d<T, SPLIT>(B, B_lo, base + K, sn);
  }
}

// The same rows from the TDOAs split as tau_hi + tau_lo (tau_hi with 13 significant bits,
// so k tau_hi / N and its fraction are exact in FP32 for k < 2^11), with FP32 sincospif:
// phases within ~4e-7 rad, the accuracy of the FP16 / TF32 hi + lo planes, at FP32 rates
// (the FP64 reduction and sincospi above run at the FP64 rate, 1/64 of FP32 on GB300).
// Used per call where the matrix is generated in chunks of cells.  One block per row
// (cell, pair), threads over the bins.
template <typename T, bool SPLIT>
__global__ __launch_bounds__(128) void conv_matrix_split_kernel(const float* __restrict__ tau_hi,
                                                                const float* __restrict__ tau_lo,
                                                                size_t rows, int N,
                                                                void* __restrict__ B,
                                                                void* __restrict__ B_lo) {
  const int K = N >> 1;
  const float invN = 1.f / static_cast<float>(N);
  for (size_t ip = blockIdx.x; ip < rows; ip += gridDim.x) {
    const float th = __ldg(tau_hi + ip), tl = __ldg(tau_lo + ip);
    const size_t base = ip * N;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
      float c = 0.f, sn = 0.f;
      if (k != 0) {
        const float x = static_cast<float>(k) * th * invN;  // exact
        const float rr = (x - floorf(x)) + static_cast<float>(k) * tl * invN;
        sincospif(2.f * rr, &sn, &c);
        c *= 2.f;
        sn *= -2.f;
      }
      op_store<T, SPLIT>(B, B_lo, base + k, c);
      op_store<T, SPLIT>(B, B_lo, base + K + k, sn);
    }
  }
}

cudaError_t launch_conv_matrix_split(const float* tau_hi, const float* tau_lo, int J, int P, int N,
                                     OpType t, void* B, void* B_lo, cudaStream_t s) {
  const size_t rows = static_cast<size_t>(J) * P;
  if (rows == 0) return cudaSuccess;
  const int g = static_cast<int>(std::min<size_t>(rows, 152 * 64));
  op_dispatch(t, [&](auto tag) {
    using Tag = decltype(tag);
    conv_matrix_split_kernel<typename Tag::type, Tag::split><<<g, 128, 0, s>>>(tau_hi, tau_lo, rows, N, B, B_lo);
  });
  return cudaGetLastError();
}

cudaError_t launch_conv_matrix(const double* tau_dev, int J, int P, int N, OpType t, void* B,
                               void* B_lo, cudaStream_t s) {
  const size_t total = static_cast<size_t>(J) * P * (N / 2);
  const int g = grid_for(total, 256);
  op_dispatch(t, [&](auto tag) {
    using Tag = decltype(tag);
    conv_matrix_kernel<typename Tag::type, Tag::split><<<g, 256, 0, s>>>(tau_dev, J, P, N, B, B_lo);
  });
  return cudaGetLastError();
}

}  // namespace srp
