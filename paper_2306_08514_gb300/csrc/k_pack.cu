// Operand preparation for the tensor-core contractions (k_tc_gemm.cu):
//   * pack16:       FP32 rows -> operand rows (FP16, BF16 or TF32) padded to a multiple of
//                   64 columns, optionally split into hi + lo planes (srp_ops.cuh);
//   * csr_to_dense: the kept entries of Lambda_sp (Eq. min_Lambda_sp) scattered into a
//                   zeroed dense [J][Lpad] operand;
//   * interp_dense: Lambda of SI-SRP, [Lambda_p]_{i,n} = sinc(Delta t_p(i)/T - n)
//                   (Eq. Lambda_p), or its conv. TD-SRP counterpart, 1 where
//                   n = round(Delta t_p(i)/T) (Eq. TD_SRP), evaluated in FP64 per entry.
#include "srp_internal.h"
#include "srp_ops.cuh"

namespace srp {

namespace {

int grid_for(size_t total, int block) {
  size_t g = (total + block - 1) / block;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return static_cast<int>(g);
}

template <typename T, bool SPLIT>
__global__ void pack16_kernel(const float* __restrict__ X, int rows, int C, int Cpad, float scale,
                              void* hi, void* lo) {
  const size_t total = static_cast<size_t>(rows) * Cpad;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int c = static_cast<int>(e % Cpad);
    const size_t r = e / Cpad;
    const float v = c < C ? X[r * C + c] * scale : 0.f;
    op_store<T, SPLIT>(hi, lo, e, v);
  }
}

// One warp per row: scatter the row's taps {col, value bits} into the zeroed operand.
template <typename T, bool SPLIT>
__global__ void csr_to_dense_kernel(const long long* __restrict__ row_ptr,
                                    const int2* __restrict__ taps, int J, int Cpad, void* hi,
                                    void* lo) {
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int lane = threadIdx.x & 31;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < J; i += warps) {
    for (long long t = row_ptr[i] + lane; t < row_ptr[i + 1]; t += 32) {
      const int2 tp = taps[t];
      op_store<T, SPLIT>(hi, lo, static_cast<size_t>(i) * Cpad + tp.x, __int_as_float(tp.y));
    }
  }
}

// Column l < L belongs to pair col_pair[l] at lag col_lag[l]; columns L..Cpad-1 are zero.
template <typename T, bool SPLIT>
__global__ void interp_dense_kernel(const double* __restrict__ tau, int J, int P,
                                    const int* __restrict__ col_pair,
                                    const int* __restrict__ col_lag, int L, int Cpad, int td,
                                    void* hi, void* lo) {
  const size_t total = static_cast<size_t>(J) * Cpad;
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < total;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const int l = static_cast<int>(e % Cpad);
    const size_t i = e / Cpad;
    double v = 0.0;
    if (l < L) {
      const double t = tau[i * P + col_pair[l]];
      const double n = static_cast<double>(col_lag[l]);
      if (td) {
        const double r = t < 0.0 ? -floor(-t + 0.5) : floor(t + 0.5);  // halves away from 0
        v = r == n ? 1.0 : 0.0;
      } else {
        const double x = t - n;
        v = x == 0.0 ? 1.0 : sinpi(x) / (M_PI * x);
      }
    }
    op_store_d<T, SPLIT>(hi, lo, e, v);
  }
}

}  // namespace

#define SRP_DISPATCH_OP(t, KERNEL, ...)                                            \
  op_dispatch(t, [&](auto tag) {                                                   \
    using Tag = decltype(tag);                                                     \
    KERNEL<typename Tag::type, Tag::split><<<g, 256, 0, s>>>(__VA_ARGS__);         \
  });

cudaError_t launch_pack16(const float* X, int rows, int C, int Cpad, float scale, OpType t,
                          void* hi, void* lo, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (C > Cpad) return cudaErrorInvalidValue;
  const int g = grid_for(static_cast<size_t>(rows) * Cpad, 256);
  SRP_DISPATCH_OP(t, pack16_kernel, X, rows, C, Cpad, scale, hi, lo)
  return cudaGetLastError();
}

cudaError_t launch_csr_to_dense(const long long* row_ptr, const int2* taps, int J, int Cpad,
                                OpType t, void* hi, void* lo, cudaStream_t s) {
  const size_t eb = op_bytes(t);
  cudaError_t e = cudaMemsetAsync(hi, 0, static_cast<size_t>(J) * Cpad * eb, s);
  if (e == cudaSuccess && op_split(t))
    e = cudaMemsetAsync(lo, 0, static_cast<size_t>(J) * Cpad * eb, s);
  if (e != cudaSuccess) return e;
  const int g = grid_for(static_cast<size_t>(J) * 32, 256);
  SRP_DISPATCH_OP(t, csr_to_dense_kernel, row_ptr, taps, J, Cpad, hi, lo)
  return cudaGetLastError();
}

cudaError_t launch_interp_dense(const double* tau, int J, int P, const int* col_pair,
                                const int* col_lag, int L, int Cpad, bool td, OpType t, void* hi,
                                void* lo, cudaStream_t s) {
  const int g = grid_for(static_cast<size_t>(J) * Cpad, 256);
  SRP_DISPATCH_OP(t, interp_dense_kernel, tau, J, P, col_pair, col_lag, L, Cpad, td ? 1 : 0, hi, lo)
  return cudaGetLastError();
}

#undef SRP_DISPATCH_OP

}  // namespace srp
