// Low-rank fit of Lambda for long sample vectors (Eq. min_Lambda_lr, Sec. IV-A) when the
// L x L Gram matrix is too large for the host eigensolver.
//
// Subspace iteration with Rayleigh-Ritz on G = Lambda^T Lambda, never forming G:
//   Q (L x k, orthonormal)  ->  Y = Lambda Q  ->  Z = Lambda^T Y = G Q
//   T = Q^T Z (k x k), T = W diag(theta) W^T  ->  Q <- orth(Z W)
// until the leading R Ritz values are stationary; then V_R = Q W_R, sigma = sqrt(theta),
// Lambda_tall = Lambda V_R, Lambda_fat = V_R^T (Eckart-Young: the best rank-R fit).
// The two products run on the device in FP64 with the entries of Lambda generated on
// the fly: sinc(tau - n) = (-1)^n sin(pi tau) / (pi (tau - n)), one division per entry
// with sin(pi tau_p(i)) precomputed per (i, p).  Orthonormalisation and the k x k
// eigenproblem run on the host in FP64.
#include "srp_internal.h"

#include <mutex>

#include <algorithm>
#include <cmath>
#include <complex>
#include <random>

namespace srp {

namespace {

constexpr int ROWS = 64;    // rows of Lambda per block chunk (Lambda X)
constexpr int ROWS_T = 32;  // rows of Lambda per block chunk (Lambda^T Y)
constexpr int COLS = 32;    // columns of Lambda per block chunk

__device__ __forceinline__ double lam_entry(double tau, double s, int n) {
  const double x = tau - static_cast<double>(n);
  if (x == 0.0) return 1.0;
  return ((n & 1) ? -s : s) / (M_PI * x);
}

// The entry in the product's type: FP64 as above, or FP32 from the FP64 difference tau - n
// (the early iterations of the subspace iteration run in FP32, see run_fit).
template <typename T>
__device__ __forceinline__ T lam_entry_t(double tau, double s, int n);
template <>
__device__ __forceinline__ double lam_entry_t<double>(double tau, double s, int n) {
  return lam_entry(tau, s, n);
}
template <>
__device__ __forceinline__ float lam_entry_t<float>(double tau, double s, int n) {
  const double x = tau - static_cast<double>(n);
  if (x == 0.0) return 1.f;
  return static_cast<float>((n & 1) ? -s : s) / (3.14159265358979323846f * static_cast<float>(x));
}

// Y[i][c] = sum_l Lambda[i][l] X[l][c], rows i of this block, c < KT.
template <typename T, int KT>
__global__ __launch_bounds__(256) void lam_apply_kernel(const double* __restrict__ tau,
                                                        const double* __restrict__ stau, int J,
                                                        int P, const int* __restrict__ col_pair,
                                                        const int* __restrict__ col_lag, int L,
                                                        const T* __restrict__ X,
                                                        T* __restrict__ Y) {
  __shared__ T lam[ROWS][COLS + 1];
  __shared__ T xs[COLS][KT];
  const int t = threadIdx.x;
  const int i0 = blockIdx.x * ROWS;
  const int r = t >> 2, cq = t & 3;
  T acc[KT / 4];
#pragma unroll
  for (int j = 0; j < KT / 4; ++j) acc[j] = T(0);
  for (int l0 = 0; l0 < L; l0 += COLS) {
    for (int e = t; e < ROWS * COLS; e += 256) {
      const int rr = e / COLS, ll = e % COLS;
      const int i = i0 + rr, l = l0 + ll;
      T v = T(0);
      if (i < J && l < L) {
        const size_t ip = static_cast<size_t>(i) * P + col_pair[l];
        v = lam_entry_t<T>(tau[ip], stau[ip], col_lag[l]);
      }
      lam[rr][ll] = v;
    }
    for (int e = t; e < COLS * KT; e += 256) {
      const int ll = e / KT, c = e % KT;
      xs[ll][c] = (l0 + ll < L) ? X[static_cast<size_t>(l0 + ll) * KT + c] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int ll = 0; ll < COLS; ++ll) {
      const T a = lam[r][ll];
#pragma unroll
      for (int j = 0; j < KT / 4; ++j) acc[j] = fma(a, xs[ll][cq + 4 * j], acc[j]);
    }
    __syncthreads();
  }
  const int i = i0 + r;
  if (i < J)
#pragma unroll
    for (int j = 0; j < KT / 4; ++j) Y[static_cast<size_t>(i) * KT + cq + 4 * j] = acc[j];
}

// Zpart[s][l][c] = sum_{i in split s} Lambda[i][l] Y[i][c], columns l of this block.
template <typename T, int KT>
__global__ __launch_bounds__(256) void lam_t_apply_kernel(const double* __restrict__ tau,
                                                          const double* __restrict__ stau, int J,
                                                          int P, const int* __restrict__ col_pair,
                                                          const int* __restrict__ col_lag, int L,
                                                          const T* __restrict__ Y,
                                                          int rows_per_split,
                                                          T* __restrict__ Zpart) {
  __shared__ T lam[ROWS_T][COLS + 1];
  __shared__ T ys[ROWS_T][KT];
  const int t = threadIdx.x;
  const int l0 = blockIdx.x * COLS;
  const int ib = blockIdx.y * rows_per_split;
  const int ie = min(J, ib + rows_per_split);
  const int lc = t >> 3, cq = t & 7;
  T acc[KT / 8];
#pragma unroll
  for (int j = 0; j < KT / 8; ++j) acc[j] = T(0);
  for (int i0 = ib; i0 < ie; i0 += ROWS_T) {
    for (int e = t; e < ROWS_T * COLS; e += 256) {
      const int rr = e / COLS, ll = e % COLS;
      const int i = i0 + rr, l = l0 + ll;
      T v = T(0);
      if (i < ie && l < L) {
        const size_t ip = static_cast<size_t>(i) * P + col_pair[l];
        v = lam_entry_t<T>(tau[ip], stau[ip], col_lag[l]);
      }
      lam[rr][ll] = v;
    }
    for (int e = t; e < ROWS_T * KT; e += 256) {
      const int rr = e / KT, c = e % KT;
      ys[rr][c] = (i0 + rr < ie) ? Y[static_cast<size_t>(i0 + rr) * KT + c] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < ROWS_T; ++rr) {
      const T a = lam[rr][lc];
#pragma unroll
      for (int j = 0; j < KT / 8; ++j) acc[j] = fma(a, ys[rr][cq + 8 * j], acc[j]);
    }
    __syncthreads();
  }
  const int l = l0 + lc;
  if (l < L)
#pragma unroll
    for (int j = 0; j < KT / 8; ++j)
      Zpart[(static_cast<size_t>(blockIdx.y) * L + l) * KT + cq + 8 * j] = acc[j];
}

__global__ void sin_pi_kernel(const double* __restrict__ tau, size_t n, double* __restrict__ s) {
  for (size_t e = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x)
    s[e] = sinpi(tau[e]);
}

// Modified Gram-Schmidt, twice, on the columns of A (rows x cols, row-major).
void orthonormalise(std::vector<double>& A, int rows, int cols) {
  // on the transpose, so that every dot product and update runs over contiguous memory
  std::vector<double> T(A.size());
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) T[static_cast<size_t>(c) * rows + r] = A[static_cast<size_t>(r) * cols + c];
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < cols; ++c) {
      double* tc = T.data() + static_cast<size_t>(c) * rows;
      for (int b = 0; b < c; ++b) {
        const double* tb = T.data() + static_cast<size_t>(b) * rows;
        double d = 0.0;
        for (int r = 0; r < rows; ++r) d += tb[r] * tc[r];
        for (int r = 0; r < rows; ++r) tc[r] -= d * tb[r];
      }
      double nn = 0.0;
      for (int r = 0; r < rows; ++r) nn += tc[r] * tc[r];
      nn = std::sqrt(nn);
      const double inv = nn > 0 ? 1.0 / nn : 0.0;
      for (int r = 0; r < rows; ++r) tc[r] *= inv;
    }
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) A[static_cast<size_t>(r) * cols + c] = T[static_cast<size_t>(c) * rows + r];
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// Fit scratch comes from device_alloc like every plan buffer (so the allocation-failure
// hook reaches it); a failed allocation is SRP_ENOMEM.
#define SRP_FIT_ALLOC(buf, bytes)                                                 \
  do {                                                                            \
    if (device_alloc(&(buf).p, (bytes)) != cudaSuccess) {                         \
      cudaGetLastError();                                                         \
      ::srp::set_error("fit scratch allocation of " + std::to_string(bytes) + " bytes failed"); \
      return SRP_ENOMEM;                                                          \
    }                                                                             \
  } while (0)

template <int KT>
srp_status run_fit(const Geometry& g, int R, int k, std::vector<float>& tall,
                   std::vector<float>& fat, std::vector<double>& sigma, cudaStream_t s) {
  const int J = g.J, L = g.L, P = g.P;
  std::vector<int> col_pair(L), col_lag(L);
  for (int q = 0; q < P; ++q)
    for (int n = -g.Np[q]; n <= g.Np[q]; ++n) {
      col_pair[g.off[q] + n + g.Np[q]] = q;
      col_lag[g.off[q] + n + g.Np[q]] = n;
    }
  const int splits = std::max(1, std::min(64, 4 * 152 / std::max(1, (L + COLS - 1) / COLS)));
  const int rows_per_split = ((J + splits - 1) / splits + ROWS_T - 1) / ROWS_T * ROWS_T;
  const int nsplit = (J + rows_per_split - 1) / rows_per_split;
  DevBuf d_tau, d_s, d_cols, d_X, d_Y, d_Z;
  const size_t JP = static_cast<size_t>(J) * P;
  SRP_FIT_ALLOC(d_tau, JP * 8);
  SRP_FIT_ALLOC(d_s, JP * 8);
  SRP_FIT_ALLOC(d_cols, sizeof(int) * 2 * L);
  SRP_FIT_ALLOC(d_X, sizeof(double) * L * KT);
  SRP_FIT_ALLOC(d_Y, sizeof(double) * static_cast<size_t>(J) * KT);
  SRP_FIT_ALLOC(d_Z, sizeof(double) * static_cast<size_t>(nsplit) * L * KT);
  auto* tau = static_cast<double*>(d_tau.p);
  auto* stau = static_cast<double*>(d_s.p);
  auto* cols = static_cast<int*>(d_cols.p);
  SRP_CUDA_TRY(cudaMemcpyAsync(tau, g.tau.data(), JP * 8, cudaMemcpyHostToDevice, s));
  SRP_CUDA_TRY(cudaMemcpyAsync(cols, col_pair.data(), sizeof(int) * L, cudaMemcpyHostToDevice, s));
  SRP_CUDA_TRY(cudaMemcpyAsync(cols + L, col_lag.data(), sizeof(int) * L, cudaMemcpyHostToDevice, s));
  sin_pi_kernel<<<1024, 256, 0, s>>>(tau, JP, stau);
  SRP_CUDA_TRY(cudaGetLastError());

  // Z = Lambda^T Lambda Q on the device: Y = Lambda X, then Z = Lambda^T Y in row splits
  // summed on the host in FP64.  fp32: the products in FP32 (entries, operands and sums).
  std::vector<double> Zp(static_cast<size_t>(nsplit) * L * KT);
  std::vector<float> Zpf;
  auto apply_G = [&](const std::vector<double>& Q, std::vector<double>& Zout, bool fp32) -> srp_status {
    const size_t n = static_cast<size_t>(L) * KT;
    if (fp32) {
      std::vector<float> Xf(n, 0.f);
      for (int l = 0; l < L; ++l)
        for (int c = 0; c < k; ++c) Xf[static_cast<size_t>(l) * KT + c] = static_cast<float>(Q[static_cast<size_t>(l) * k + c]);
      SRP_CUDA_TRY(cudaMemcpyAsync(d_X.p, Xf.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s));
      lam_apply_kernel<float, KT><<<(J + ROWS - 1) / ROWS, 256, 0, s>>>(
          tau, stau, J, P, cols, cols + L, L, static_cast<float*>(d_X.p), static_cast<float*>(d_Y.p));
      SRP_CUDA_TRY(cudaGetLastError());
      dim3 grid((L + COLS - 1) / COLS, nsplit);
      lam_t_apply_kernel<float, KT><<<grid, 256, 0, s>>>(tau, stau, J, P, cols, cols + L, L,
                                                         static_cast<float*>(d_Y.p), rows_per_split,
                                                         static_cast<float*>(d_Z.p));
      SRP_CUDA_TRY(cudaGetLastError());
      Zpf.resize(Zp.size());
      SRP_CUDA_TRY(cudaMemcpyAsync(Zpf.data(), d_Z.p, sizeof(float) * Zpf.size(), cudaMemcpyDeviceToHost, s));
      SRP_CUDA_TRY(cudaStreamSynchronize(s));
      for (size_t e = 0; e < Zp.size(); ++e) Zp[e] = Zpf[e];
    } else {
      std::vector<double> Xh(n, 0.0);
      for (int l = 0; l < L; ++l)
        for (int c = 0; c < k; ++c) Xh[static_cast<size_t>(l) * KT + c] = Q[static_cast<size_t>(l) * k + c];
      SRP_CUDA_TRY(cudaMemcpyAsync(d_X.p, Xh.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
      lam_apply_kernel<double, KT><<<(J + ROWS - 1) / ROWS, 256, 0, s>>>(
          tau, stau, J, P, cols, cols + L, L, static_cast<double*>(d_X.p), static_cast<double*>(d_Y.p));
      SRP_CUDA_TRY(cudaGetLastError());
      dim3 grid((L + COLS - 1) / COLS, nsplit);
      lam_t_apply_kernel<double, KT><<<grid, 256, 0, s>>>(tau, stau, J, P, cols, cols + L, L,
                                                          static_cast<double*>(d_Y.p), rows_per_split,
                                                          static_cast<double*>(d_Z.p));
      SRP_CUDA_TRY(cudaGetLastError());
      SRP_CUDA_TRY(cudaMemcpyAsync(Zp.data(), d_Z.p, sizeof(double) * Zp.size(), cudaMemcpyDeviceToHost, s));
      SRP_CUDA_TRY(cudaStreamSynchronize(s));
    }
    Zout.assign(static_cast<size_t>(L) * k, 0.0);
    parallel_for(L, [&](long long b, long long e) {
      for (int sp = 0; sp < nsplit; ++sp)
        for (long long l = b; l < e; ++l)
          for (int c = 0; c < k; ++c)
            Zout[static_cast<size_t>(l) * k + c] += Zp[(static_cast<size_t>(sp) * L + l) * KT + c];
    });
    return SRP_OK;
  };

  std::mt19937_64 rng(12345);
  std::normal_distribution<double> nd;
  std::vector<double> Q(static_cast<size_t>(L) * k), Z, W, theta, Tm;
  for (auto& v : Q) v = nd(rng);
  orthonormalise(Q, L, k);
  std::vector<double> prev(R, 0.0);
  std::vector<int> order(k);
  bool converged = false;
  // Two phases: FP32 products until the Ritz values settle at FP32 accuracy (their relative
  // change below 1e-6, or no longer shrinking), then FP64 products until they change by
  // less than 1e-13.  The iteration corrects the earlier phase's rounding itself, so the
  // result is that of the FP64 iteration; the FP32 products run ~60x faster on GB300.
  bool fp32 = true;
  int fp64_its = 0;
  double best32 = 1e300;
  int stale32 = 0;
  for (int it = 0; it < 400; ++it) {
    srp_status st = apply_G(Q, Z, fp32);
    if (st != SRP_OK) return st;
    // T = Q^T Z, summed row by row in fixed chunks (deterministic), then symmetrised
    Tm.assign(static_cast<size_t>(k) * k, 0.0);
    {
      std::mutex mu;
      std::vector<std::pair<long long, std::vector<double>>> parts;
      parallel_for(L, [&](long long b, long long e) {
        std::vector<double> t(static_cast<size_t>(k) * k, 0.0);
        for (long long l = b; l < e; ++l) {
          const double* ql = Q.data() + static_cast<size_t>(l) * k;
          const double* zl = Z.data() + static_cast<size_t>(l) * k;
          for (int a = 0; a < k; ++a) {
            const double qa = ql[a];
            double* ta = t.data() + static_cast<size_t>(a) * k;
            for (int c = 0; c < k; ++c) ta[c] += qa * zl[c];
          }
        }
        std::lock_guard<std::mutex> lock(mu);
        parts.emplace_back(b, std::move(t));
      });
      std::sort(parts.begin(), parts.end(),
                [](const auto& x, const auto& y) { return x.first < y.first; });
      for (const auto& pt : parts)
        for (size_t e = 0; e < Tm.size(); ++e) Tm[e] += pt.second[e];
    }
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b) {
        const double m = 0.5 * (Tm[static_cast<size_t>(a) * k + b] + Tm[static_cast<size_t>(b) * k + a]);
        Tm[static_cast<size_t>(a) * k + b] = Tm[static_cast<size_t>(b) * k + a] = m;
      }
    jacobi_eigen(k, Tm, W, theta);
    for (int i = 0; i < k; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return theta[a] > theta[b]; });
    double change = 0.0;
    for (int r = 0; r < R; ++r) {
      const double th = theta[order[r]];
      change = std::max(change, std::fabs(th - prev[r]) / std::max(th, 1e-300));
      prev[r] = th;
    }
    // Ritz vectors of this Q and the next basis orth(Z W) (W sorted)
    std::vector<double> QW(static_cast<size_t>(L) * k, 0.0), ZW(static_cast<size_t>(L) * k, 0.0);
    parallel_for(L, [&](long long b, long long e) {
      for (long long l = b; l < e; ++l)
        for (int c = 0; c < k; ++c) {
          double qa = 0.0, za = 0.0;
          const int wc = order[c];
          for (int a = 0; a < k; ++a) {
            const double w = W[static_cast<size_t>(a) * k + wc];
            qa += Q[static_cast<size_t>(l) * k + a] * w;
            za += Z[static_cast<size_t>(l) * k + a] * w;
          }
          QW[static_cast<size_t>(l) * k + c] = qa;
          ZW[static_cast<size_t>(l) * k + c] = za;
        }
    });
    if (fp32) {
      if (change < best32 * 0.5) {
        best32 = change;
        stale32 = 0;
      } else {
        ++stale32;
      }
      if (it > 2 && (change < 1e-6 || stale32 >= 4)) fp32 = false;
    } else if (++fp64_its > 2 && change < 1e-13) {
      Q.swap(QW);
      converged = true;
      break;
    }
    orthonormalise(ZW, L, k);
    Q.swap(ZW);
  }
  if (!converged) {
    set_error("low-rank fit: subspace iteration did not converge");
    return SRP_EUNSUPPORTED;
  }
  sigma.resize(k);  // all k Ritz values of the last Rayleigh-Ritz step
  for (int c = 0; c < k; ++c) sigma[c] = std::sqrt(std::max(0.0, theta[order[c]]));
  // tall = Lambda V_R (one more device product), fat = V_R^T
  const int Rp = (R + 7) / 8 * 8;
  fat.assign(static_cast<size_t>(Rp) * L, 0.f);
  for (int r = 0; r < R; ++r)
    for (int l = 0; l < L; ++l) fat[static_cast<size_t>(r) * L + l] = static_cast<float>(Q[static_cast<size_t>(l) * k + r]);
  std::vector<double> Xh(static_cast<size_t>(L) * KT, 0.0);
  for (int l = 0; l < L; ++l)
    for (int c = 0; c < R; ++c) Xh[static_cast<size_t>(l) * KT + c] = Q[static_cast<size_t>(l) * k + c];
  SRP_CUDA_TRY(cudaMemcpyAsync(d_X.p, Xh.data(), sizeof(double) * L * KT, cudaMemcpyHostToDevice, s));
  lam_apply_kernel<double, KT><<<(J + ROWS - 1) / ROWS, 256, 0, s>>>(tau, stau, J, P, cols, cols + L, L,
                                                                     static_cast<double*>(d_X.p),
                                                                     static_cast<double*>(d_Y.p));
  SRP_CUDA_TRY(cudaGetLastError());
  std::vector<double> Yh(static_cast<size_t>(J) * KT);
  SRP_CUDA_TRY(cudaMemcpyAsync(Yh.data(), d_Y.p, sizeof(double) * Yh.size(), cudaMemcpyDeviceToHost, s));
  SRP_CUDA_TRY(cudaStreamSynchronize(s));
  tall.assign(static_cast<size_t>(J) * Rp, 0.f);
  for (int i = 0; i < J; ++i)
    for (int r = 0; r < R; ++r) tall[static_cast<size_t>(i) * Rp + r] = static_cast<float>(Yh[static_cast<size_t>(i) * KT + r]);
  return SRP_OK;
}

// ------------------------------------------------------------------------------------
// LR-SRP (Sec. III-A): the best rank-R approximation of the complex SRP matrix H
// (J x D, D = P (K-1), [H]_{i,(p,k)} = e^{j omega_k Delta t_p(i)}, Eq. H_p_single), from the
// same subspace iteration on H^H H with complex FP64 products; H entries are generated on
// the fly from the FP64 TDOA table as e^{j 2 pi frac(k tau / N)}.
// ------------------------------------------------------------------------------------
constexpr int LR_ROWS = 32;   // rows of H per chunk (H X)
constexpr int LR_COLS = 16;   // columns of H per chunk
constexpr int LR_ROWS_T = 16; // rows of H per chunk (H^H Y)

__device__ __forceinline__ double2 h_entry(const double* __restrict__ tau, int P, int K, int i, int d) {
  const int q = d / (K - 1);
  const int k = d - q * (K - 1) + 1;
  const double t = static_cast<double>(k) * tau[static_cast<size_t>(i) * P + q];
  const double N = 2.0 * K;
  const double r = t - N * floor(t / N);  // k tau mod N, exact reduction in FP64
  double sn, cs;
  sincospi(2.0 * r / N, &sn, &cs);
  return make_double2(cs, sn);
}

// Y[i][c] = sum_d H[i][d] X[d][c] (complex), rows of this block.
template <int KT>
__global__ __launch_bounds__(256) void lr_apply_kernel(const double* __restrict__ tau, int J, int P,
                                                       int K, int D, const double2* __restrict__ X,
                                                       double2* __restrict__ Y) {
  __shared__ double2 hs[LR_ROWS][LR_COLS + 1];
  __shared__ double2 xs[LR_COLS][KT];
  const int t = threadIdx.x;
  const int i0 = blockIdx.x * LR_ROWS;
  const int r = t >> 3, cq = t & 7;
  double2 acc[KT / 8];
#pragma unroll
  for (int j = 0; j < KT / 8; ++j) acc[j] = make_double2(0.0, 0.0);
  for (int d0 = 0; d0 < D; d0 += LR_COLS) {
    for (int e = t; e < LR_ROWS * LR_COLS; e += 256) {
      const int rr = e / LR_COLS, dd = e % LR_COLS;
      hs[rr][dd] = (i0 + rr < J && d0 + dd < D) ? h_entry(tau, P, K, i0 + rr, d0 + dd)
                                                 : make_double2(0.0, 0.0);
    }
    for (int e = t; e < LR_COLS * KT; e += 256) {
      const int dd = e / KT, c = e % KT;
      xs[dd][c] = (d0 + dd < D) ? X[static_cast<size_t>(d0 + dd) * KT + c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int dd = 0; dd < LR_COLS; ++dd) {
      const double2 h = hs[r][dd];
#pragma unroll
      for (int j = 0; j < KT / 8; ++j) {
        const double2 x = xs[dd][cq + 8 * j];
        acc[j].x = fma(h.x, x.x, fma(-h.y, x.y, acc[j].x));
        acc[j].y = fma(h.x, x.y, fma(h.y, x.x, acc[j].y));
      }
    }
    __syncthreads();
  }
  const int i = i0 + r;
  if (i < J)
#pragma unroll
    for (int j = 0; j < KT / 8; ++j) Y[static_cast<size_t>(i) * KT + cq + 8 * j] = acc[j];
}

// Zpart[s][d][c] = sum_{i in split s} conj(H[i][d]) Y[i][c].
template <int KT>
__global__ __launch_bounds__(256) void lr_t_apply_kernel(const double* __restrict__ tau, int J,
                                                         int P, int K, int D,
                                                         const double2* __restrict__ Y,
                                                         int rows_per_split,
                                                         double2* __restrict__ Zpart) {
  __shared__ double2 hs[LR_ROWS_T][LR_COLS + 1];
  __shared__ double2 ys[LR_ROWS_T][KT];
  const int t = threadIdx.x;
  const int d0 = blockIdx.x * LR_COLS;
  const int ib = blockIdx.y * rows_per_split;
  const int ie = min(J, ib + rows_per_split);
  const int dc = t >> 4, cq = t & 15;
  double2 acc[KT / 16];
#pragma unroll
  for (int j = 0; j < KT / 16; ++j) acc[j] = make_double2(0.0, 0.0);
  for (int i0 = ib; i0 < ie; i0 += LR_ROWS_T) {
    for (int e = t; e < LR_ROWS_T * LR_COLS; e += 256) {
      const int rr = e / LR_COLS, dd = e % LR_COLS;
      hs[rr][dd] = (i0 + rr < ie && d0 + dd < D) ? h_entry(tau, P, K, i0 + rr, d0 + dd)
                                                  : make_double2(0.0, 0.0);
    }
    for (int e = t; e < LR_ROWS_T * KT; e += 256) {
      const int rr = e / KT, c = e % KT;
      ys[rr][c] = (i0 + rr < ie) ? Y[static_cast<size_t>(i0 + rr) * KT + c] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < LR_ROWS_T; ++rr) {
      const double2 h = hs[rr][dc];  // conj(h) * y
#pragma unroll
      for (int j = 0; j < KT / 16; ++j) {
        const double2 y = ys[rr][cq + 16 * j];
        acc[j].x = fma(h.x, y.x, fma(h.y, y.y, acc[j].x));
        acc[j].y = fma(h.x, y.y, fma(-h.y, y.x, acc[j].y));
      }
    }
    __syncthreads();
  }
  const int d = d0 + dc;
  if (d < D)
#pragma unroll
    for (int j = 0; j < KT / 16; ++j)
      Zpart[(static_cast<size_t>(blockIdx.y) * D + d) * KT + cq + 16 * j] = acc[j];
}

using cplx = std::complex<double>;

// Modified Gram-Schmidt, twice, on the columns of a complex rows x cols matrix.
void orthonormalise_c(std::vector<cplx>& A, int rows, int cols) {
  std::vector<cplx> T(A.size());  // on the transpose (contiguous columns)
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) T[static_cast<size_t>(c) * rows + r] = A[static_cast<size_t>(r) * cols + c];
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < cols; ++c) {
      cplx* tc = T.data() + static_cast<size_t>(c) * rows;
      for (int b = 0; b < c; ++b) {
        const cplx* tb = T.data() + static_cast<size_t>(b) * rows;
        cplx d = 0.0;
        for (int r = 0; r < rows; ++r) d += std::conj(tb[r]) * tc[r];
        for (int r = 0; r < rows; ++r) tc[r] -= d * tb[r];
      }
      double nn = 0.0;
      for (int r = 0; r < rows; ++r) nn += std::norm(tc[r]);
      nn = std::sqrt(nn);
      const double inv = nn > 0 ? 1.0 / nn : 0.0;
      for (int r = 0; r < rows; ++r) tc[r] *= inv;
    }
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) A[static_cast<size_t>(r) * cols + c] = T[static_cast<size_t>(c) * rows + r];
}

// Eigen-decomposition of a k x k Hermitian T through the real symmetric 2k x 2k matrix
// [[Re T, -Im T], [Im T, Re T]], whose eigenvalues are those of T, each twice; from each
// pair one complex eigenvector x + jy is kept (the other is j times it).
void hermitian_eigen(int k, const std::vector<cplx>& T, std::vector<cplx>& W, std::vector<double>& th) {
  const int n = 2 * k;
  std::vector<double> A(static_cast<size_t>(n) * n), V, ev;
  for (int a = 0; a < k; ++a)
    for (int b = 0; b < k; ++b) {
      const cplx t = T[static_cast<size_t>(a) * k + b];
      A[static_cast<size_t>(a) * n + b] = t.real();
      A[static_cast<size_t>(a) * n + k + b] = -t.imag();
      A[static_cast<size_t>(k + a) * n + b] = t.imag();
      A[static_cast<size_t>(k + a) * n + k + b] = t.real();
    }
  jacobi_eigen(n, A, V, ev);
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] > ev[b]; });
  W.assign(static_cast<size_t>(k) * k, 0.0);  // columns: eigenvectors
  th.clear();
  int got = 0;
  for (int oi = 0; oi < n && got < k; ++oi) {
    const int c = order[oi];
    std::vector<cplx> v(k);
    for (int a = 0; a < k; ++a) v[a] = cplx(V[static_cast<size_t>(a) * n + c], V[static_cast<size_t>(k + a) * n + c]);
    for (int b = 0; b < got; ++b) {  // remove the directions already kept
      cplx d = 0.0;
      for (int a = 0; a < k; ++a) d += std::conj(W[static_cast<size_t>(a) * k + b]) * v[a];
      for (int a = 0; a < k; ++a) v[a] -= d * W[static_cast<size_t>(a) * k + b];
    }
    double nn = 0.0;
    for (int a = 0; a < k; ++a) nn += std::norm(v[a]);
    nn = std::sqrt(nn);
    if (nn < 0.5) continue;  // the partner of an eigenvector already kept
    for (int a = 0; a < k; ++a) W[static_cast<size_t>(a) * k + got] = v[a] / nn;
    th.push_back(ev[c]);
    ++got;
  }
  while (static_cast<int>(th.size()) < k) th.push_back(0.0);
}

template <int KT>
srp_status run_lr_fit(const Geometry& g, int R, int k, std::vector<cplx>& tall,
                      std::vector<cplx>& fat, std::vector<double>& sigma, cudaStream_t s) {
  const int J = g.J, P = g.P, K = g.K;
  const int D = P * (K - 1);
  const int splits = std::max(1, std::min(64, 4 * 152 / std::max(1, (D + LR_COLS - 1) / LR_COLS)));
  const int rows_per_split = ((J + splits - 1) / splits + LR_ROWS_T - 1) / LR_ROWS_T * LR_ROWS_T;
  const int nsplit = (J + rows_per_split - 1) / rows_per_split;
  DevBuf d_tau, d_X, d_Y, d_Z;
  const size_t JP = static_cast<size_t>(J) * P;
  SRP_FIT_ALLOC(d_tau, JP * 8);
  SRP_FIT_ALLOC(d_X, sizeof(double2) * static_cast<size_t>(D) * KT);
  SRP_FIT_ALLOC(d_Y, sizeof(double2) * static_cast<size_t>(J) * KT);
  SRP_FIT_ALLOC(d_Z, sizeof(double2) * static_cast<size_t>(nsplit) * D * KT);
  auto* tau = static_cast<double*>(d_tau.p);
  SRP_CUDA_TRY(cudaMemcpyAsync(tau, g.tau.data(), JP * 8, cudaMemcpyHostToDevice, s));
  std::vector<cplx> Xh(static_cast<size_t>(D) * KT), Zp(static_cast<size_t>(nsplit) * D * KT);
  auto apply_Y = [&](const std::vector<cplx>& Q, int cols) -> srp_status {  // d_Y = H Q
    for (int d = 0; d < D; ++d)
      for (int c = 0; c < KT; ++c) Xh[static_cast<size_t>(d) * KT + c] = c < cols ? Q[static_cast<size_t>(d) * k + c] : 0.0;
    SRP_CUDA_TRY(cudaMemcpyAsync(d_X.p, Xh.data(), sizeof(double2) * D * KT, cudaMemcpyHostToDevice, s));
    lr_apply_kernel<KT><<<(J + LR_ROWS - 1) / LR_ROWS, 256, 0, s>>>(tau, J, P, K, D,
                                                                    static_cast<double2*>(d_X.p),
                                                                    static_cast<double2*>(d_Y.p));
    SRP_CUDA_TRY(cudaGetLastError());
    return SRP_OK;
  };
  auto apply_G = [&](const std::vector<cplx>& Q, std::vector<cplx>& Zout) -> srp_status {
    srp_status st = apply_Y(Q, k);
    if (st != SRP_OK) return st;
    dim3 grid((D + LR_COLS - 1) / LR_COLS, nsplit);
    lr_t_apply_kernel<KT><<<grid, 256, 0, s>>>(tau, J, P, K, D, static_cast<double2*>(d_Y.p),
                                               rows_per_split, static_cast<double2*>(d_Z.p));
    SRP_CUDA_TRY(cudaGetLastError());
    SRP_CUDA_TRY(cudaMemcpyAsync(Zp.data(), d_Z.p, sizeof(double2) * Zp.size(), cudaMemcpyDeviceToHost, s));
    SRP_CUDA_TRY(cudaStreamSynchronize(s));
    Zout.assign(static_cast<size_t>(D) * k, 0.0);
    for (int sp = 0; sp < nsplit; ++sp)
      for (int d = 0; d < D; ++d)
        for (int c = 0; c < k; ++c) Zout[static_cast<size_t>(d) * k + c] += Zp[(static_cast<size_t>(sp) * D + d) * KT + c];
    return SRP_OK;
  };
  std::mt19937_64 rng(54321);
  std::normal_distribution<double> nd;
  std::vector<cplx> Q(static_cast<size_t>(D) * k), Z, W, T;
  for (auto& v : Q) v = cplx(nd(rng), nd(rng));
  orthonormalise_c(Q, D, k);
  std::vector<double> prev(R, 0.0), theta;
  bool converged = false;
  for (int it = 0; it < 300; ++it) {
    srp_status st = apply_G(Q, Z);
    if (st != SRP_OK) return st;
    T.assign(static_cast<size_t>(k) * k, 0.0);  // Q^H Z (summed row by row), Hermitian part
    for (int l = 0; l < D; ++l) {
      const cplx* ql = Q.data() + static_cast<size_t>(l) * k;
      const cplx* zl = Z.data() + static_cast<size_t>(l) * k;
      for (int a = 0; a < k; ++a) {
        const cplx qa = std::conj(ql[a]);
        cplx* ta = T.data() + static_cast<size_t>(a) * k;
        for (int b = 0; b < k; ++b) ta[b] += qa * zl[b];
      }
    }
    for (int a = 0; a < k; ++a)
      for (int b = a; b < k; ++b) {
        const cplx m = 0.5 * (T[static_cast<size_t>(a) * k + b] + std::conj(T[static_cast<size_t>(b) * k + a]));
        T[static_cast<size_t>(a) * k + b] = m;
        T[static_cast<size_t>(b) * k + a] = std::conj(m);
      }
    hermitian_eigen(k, T, W, theta);  // descending
    double change = 0.0;
    for (int r = 0; r < R; ++r) {
      change = std::max(change, std::fabs(theta[r] - prev[r]) / std::max(theta[r], 1e-300));
      prev[r] = theta[r];
    }
    std::vector<cplx> QW(static_cast<size_t>(D) * k, 0.0), ZW(static_cast<size_t>(D) * k, 0.0);
    for (int l = 0; l < D; ++l)
      for (int c = 0; c < k; ++c) {
        cplx qa = 0.0, za = 0.0;
        for (int a = 0; a < k; ++a) {
          const cplx w = W[static_cast<size_t>(a) * k + c];
          qa += Q[static_cast<size_t>(l) * k + a] * w;
          za += Z[static_cast<size_t>(l) * k + a] * w;
        }
        QW[static_cast<size_t>(l) * k + c] = qa;
        ZW[static_cast<size_t>(l) * k + c] = za;
      }
    if (it > 2 && change < 1e-13) {
      Q.swap(QW);
      converged = true;
      break;
    }
    orthonormalise_c(ZW, D, k);
    Q.swap(ZW);
  }
  if (!converged) {
    set_error("LR fit: subspace iteration did not converge");
    return SRP_EUNSUPPORTED;
  }
  sigma.resize(k);
  for (int c = 0; c < k; ++c) sigma[c] = std::sqrt(std::max(0.0, theta[c]));
  // H_fat = V_R^H (R x D), H_tall = H V_R (J x R)
  fat.assign(static_cast<size_t>(R) * D, 0.0);
  for (int r = 0; r < R; ++r)
    for (int d = 0; d < D; ++d) fat[static_cast<size_t>(r) * D + d] = std::conj(Q[static_cast<size_t>(d) * k + r]);
  srp_status st = apply_Y(Q, R);
  if (st != SRP_OK) return st;
  std::vector<cplx> Yh(static_cast<size_t>(J) * KT);
  SRP_CUDA_TRY(cudaMemcpyAsync(Yh.data(), d_Y.p, sizeof(double2) * Yh.size(), cudaMemcpyDeviceToHost, s));
  SRP_CUDA_TRY(cudaStreamSynchronize(s));
  tall.assign(static_cast<size_t>(J) * R, 0.0);
  for (int i = 0; i < J; ++i)
    for (int r = 0; r < R; ++r) tall[static_cast<size_t>(i) * R + r] = Yh[static_cast<size_t>(i) * KT + r];
  return SRP_OK;
}

}  // namespace

srp_status fit_lr_device(const Geometry& g, int R, std::vector<std::complex<double>>& tall,
                         std::vector<std::complex<double>>& fat, std::vector<double>& sigma,
                         cudaStream_t s) {
  const int D = g.P * (g.K - 1);
  const int want = R + 32;  // as fit_low_rank_device: the whole column bucket is used
  if (want <= 32) return run_lr_fit<32>(g, R, std::min(D, 32), tall, fat, sigma, s);
  if (want <= 64) return run_lr_fit<64>(g, R, std::min(D, 64), tall, fat, sigma, s);
  return run_lr_fit<96>(g, R, std::min(D, 96), tall, fat, sigma, s);
}

srp_status fit_low_rank_device(const Geometry& g, int R, std::vector<float>& tall,
                               std::vector<float>& fat, std::vector<double>& sigma,
                               cudaStream_t s) {
  // at least 32 guard columns, and every column of the kernel's bucket used (the padding
  // would cost the same and the extra columns speed the convergence up)
  const int want = R + 32;
  if (want <= 32) return run_fit<32>(g, R, std::min(g.L, 32), tall, fat, sigma, s);
  if (want <= 64) return run_fit<64>(g, R, std::min(g.L, 64), tall, fat, sigma, s);
  return run_fit<96>(g, R, std::min(g.L, 96), tall, fat, sigma, s);
}

}  // namespace srp
