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

#include <algorithm>
#include <cmath>
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

// Y[i][c] = sum_l Lambda[i][l] X[l][c], rows i of this block, c < KT.
template <int KT>
__global__ __launch_bounds__(256) void lam_apply_kernel(const double* __restrict__ tau,
                                                        const double* __restrict__ stau, int J,
                                                        int P, const int* __restrict__ col_pair,
                                                        const int* __restrict__ col_lag, int L,
                                                        const double* __restrict__ X,
                                                        double* __restrict__ Y) {
  __shared__ double lam[ROWS][COLS + 1];
  __shared__ double xs[COLS][KT];
  const int t = threadIdx.x;
  const int i0 = blockIdx.x * ROWS;
  const int r = t >> 2, cq = t & 3;
  double acc[KT / 4];
#pragma unroll
  for (int j = 0; j < KT / 4; ++j) acc[j] = 0.0;
  for (int l0 = 0; l0 < L; l0 += COLS) {
    for (int e = t; e < ROWS * COLS; e += 256) {
      const int rr = e / COLS, ll = e % COLS;
      const int i = i0 + rr, l = l0 + ll;
      double v = 0.0;
      if (i < J && l < L) {
        const size_t ip = static_cast<size_t>(i) * P + col_pair[l];
        v = lam_entry(tau[ip], stau[ip], col_lag[l]);
      }
      lam[rr][ll] = v;
    }
    for (int e = t; e < COLS * KT; e += 256) {
      const int ll = e / KT, c = e % KT;
      xs[ll][c] = (l0 + ll < L) ? X[static_cast<size_t>(l0 + ll) * KT + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int ll = 0; ll < COLS; ++ll) {
      const double a = lam[r][ll];
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
template <int KT>
__global__ __launch_bounds__(256) void lam_t_apply_kernel(const double* __restrict__ tau,
                                                          const double* __restrict__ stau, int J,
                                                          int P, const int* __restrict__ col_pair,
                                                          const int* __restrict__ col_lag, int L,
                                                          const double* __restrict__ Y,
                                                          int rows_per_split,
                                                          double* __restrict__ Zpart) {
  __shared__ double lam[ROWS_T][COLS + 1];
  __shared__ double ys[ROWS_T][KT];
  const int t = threadIdx.x;
  const int l0 = blockIdx.x * COLS;
  const int ib = blockIdx.y * rows_per_split;
  const int ie = min(J, ib + rows_per_split);
  const int lc = t >> 3, cq = t & 7;
  double acc[KT / 8];
#pragma unroll
  for (int j = 0; j < KT / 8; ++j) acc[j] = 0.0;
  for (int i0 = ib; i0 < ie; i0 += ROWS_T) {
    for (int e = t; e < ROWS_T * COLS; e += 256) {
      const int rr = e / COLS, ll = e % COLS;
      const int i = i0 + rr, l = l0 + ll;
      double v = 0.0;
      if (i < ie && l < L) {
        const size_t ip = static_cast<size_t>(i) * P + col_pair[l];
        v = lam_entry(tau[ip], stau[ip], col_lag[l]);
      }
      lam[rr][ll] = v;
    }
    for (int e = t; e < ROWS_T * KT; e += 256) {
      const int rr = e / KT, c = e % KT;
      ys[rr][c] = (i0 + rr < ie) ? Y[static_cast<size_t>(i0 + rr) * KT + c] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < ROWS_T; ++rr) {
      const double a = lam[rr][lc];
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
  for (int pass = 0; pass < 2; ++pass)
    for (int c = 0; c < cols; ++c) {
      for (int b = 0; b < c; ++b) {
        double d = 0.0;
        for (int r = 0; r < rows; ++r) d += A[static_cast<size_t>(r) * cols + b] * A[static_cast<size_t>(r) * cols + c];
        for (int r = 0; r < rows; ++r) A[static_cast<size_t>(r) * cols + c] -= d * A[static_cast<size_t>(r) * cols + b];
      }
      double nn = 0.0;
      for (int r = 0; r < rows; ++r) nn += A[static_cast<size_t>(r) * cols + c] * A[static_cast<size_t>(r) * cols + c];
      nn = std::sqrt(nn);
      const double inv = nn > 0 ? 1.0 / nn : 0.0;
      for (int r = 0; r < rows; ++r) A[static_cast<size_t>(r) * cols + c] *= inv;
    }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

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
  SRP_CUDA_TRY(cudaMalloc(&d_tau.p, JP * 8));
  SRP_CUDA_TRY(cudaMalloc(&d_s.p, JP * 8));
  SRP_CUDA_TRY(cudaMalloc(&d_cols.p, sizeof(int) * 2 * L));
  SRP_CUDA_TRY(cudaMalloc(&d_X.p, sizeof(double) * L * KT));
  SRP_CUDA_TRY(cudaMalloc(&d_Y.p, sizeof(double) * static_cast<size_t>(J) * KT));
  SRP_CUDA_TRY(cudaMalloc(&d_Z.p, sizeof(double) * static_cast<size_t>(nsplit) * L * KT));
  auto* tau = static_cast<double*>(d_tau.p);
  auto* stau = static_cast<double*>(d_s.p);
  auto* cols = static_cast<int*>(d_cols.p);
  SRP_CUDA_TRY(cudaMemcpyAsync(tau, g.tau.data(), JP * 8, cudaMemcpyHostToDevice, s));
  SRP_CUDA_TRY(cudaMemcpyAsync(cols, col_pair.data(), sizeof(int) * L, cudaMemcpyHostToDevice, s));
  SRP_CUDA_TRY(cudaMemcpyAsync(cols + L, col_lag.data(), sizeof(int) * L, cudaMemcpyHostToDevice, s));
  sin_pi_kernel<<<1024, 256, 0, s>>>(tau, JP, stau);
  SRP_CUDA_TRY(cudaGetLastError());

  // Y = Lambda X (host X [L][k] -> host Y [J][KT]) and Z = Lambda^T Y
  std::vector<double> Xh(static_cast<size_t>(L) * KT), Zh(static_cast<size_t>(L) * KT);
  std::vector<double> Zp(static_cast<size_t>(nsplit) * L * KT);
  auto apply_G = [&](const std::vector<double>& Q, std::vector<double>& Zout) -> srp_status {
    for (int l = 0; l < L; ++l)
      for (int c = 0; c < KT; ++c) Xh[static_cast<size_t>(l) * KT + c] = c < k ? Q[static_cast<size_t>(l) * k + c] : 0.0;
    SRP_CUDA_TRY(cudaMemcpyAsync(d_X.p, Xh.data(), sizeof(double) * L * KT, cudaMemcpyHostToDevice, s));
    lam_apply_kernel<KT><<<(J + ROWS - 1) / ROWS, 256, 0, s>>>(tau, stau, J, P, cols, cols + L, L,
                                                               static_cast<double*>(d_X.p),
                                                               static_cast<double*>(d_Y.p));
    SRP_CUDA_TRY(cudaGetLastError());
    dim3 grid((L + COLS - 1) / COLS, nsplit);
    lam_t_apply_kernel<KT><<<grid, 256, 0, s>>>(tau, stau, J, P, cols, cols + L, L,
                                                static_cast<double*>(d_Y.p), rows_per_split,
                                                static_cast<double*>(d_Z.p));
    SRP_CUDA_TRY(cudaGetLastError());
    SRP_CUDA_TRY(cudaMemcpyAsync(Zp.data(), d_Z.p, sizeof(double) * Zp.size(), cudaMemcpyDeviceToHost, s));
    SRP_CUDA_TRY(cudaStreamSynchronize(s));
    Zout.assign(static_cast<size_t>(L) * k, 0.0);
    for (int sp = 0; sp < nsplit; ++sp)
      for (int l = 0; l < L; ++l)
        for (int c = 0; c < k; ++c)
          Zout[static_cast<size_t>(l) * k + c] += Zp[(static_cast<size_t>(sp) * L + l) * KT + c];
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
  for (int it = 0; it < 300; ++it) {
    srp_status st = apply_G(Q, Z);
    if (st != SRP_OK) return st;
    Tm.assign(static_cast<size_t>(k) * k, 0.0);  // T = Q^T Z, symmetrised
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        double d = 0.0;
        for (int l = 0; l < L; ++l) d += Q[static_cast<size_t>(l) * k + a] * Z[static_cast<size_t>(l) * k + b];
        Tm[static_cast<size_t>(a) * k + b] = d;
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
    for (int l = 0; l < L; ++l)
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
    if (it > 2 && change < 1e-13) {
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
  for (int l = 0; l < L; ++l)
    for (int c = 0; c < KT; ++c) Xh[static_cast<size_t>(l) * KT + c] = c < R ? Q[static_cast<size_t>(l) * k + c] : 0.0;
  SRP_CUDA_TRY(cudaMemcpyAsync(d_X.p, Xh.data(), sizeof(double) * L * KT, cudaMemcpyHostToDevice, s));
  lam_apply_kernel<KT><<<(J + ROWS - 1) / ROWS, 256, 0, s>>>(tau, stau, J, P, cols, cols + L, L,
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

}  // namespace

srp_status fit_low_rank_device(const Geometry& g, int R, std::vector<float>& tall,
                               std::vector<float>& fat, std::vector<double>& sigma,
                               cudaStream_t s) {
  const int k = std::min(g.L, R + 32);
  if (k <= 32) return run_fit<32>(g, R, k, tall, fat, sigma, s);
  if (k <= 64) return run_fit<64>(g, R, k, tall, fat, sigma, s);
  return run_fit<96>(g, R, k, tall, fat, sigma, s);
}

}  // namespace srp
