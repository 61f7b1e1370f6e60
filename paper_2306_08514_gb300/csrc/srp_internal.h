// Internal declarations shared by the libsrp translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include <complex>
#include <functional>
#include <cstdint>
#include <string>
#include <vector>

#include "libsrp.h"

namespace srp {

constexpr int kHostPipe = 16;  // events of the srp_map_host copy pipeline

// Runs fn(begin, end) over [0, n) in contiguous chunks on the host's threads (the chunks
// depend only on n and the thread count).
void parallel_for(long long n, const std::function<void(long long, long long)>& fn);

// A method's fit as a saved plan holds it (srp_plan_save / srp_plan_create_from_file).
struct FitData {
  std::vector<double> sigma;                             // SLRI, LR-SRP
  std::vector<float> tall, fat;                          // SLRI: [J][Rp], [Rp][L]
  long long nnz = 0, tied = 0;                           // SSPI
  std::vector<long long> row_ptr;
  std::vector<int> col;
  std::vector<float> val;
  std::vector<std::complex<double>> ht, hf;              // LR-SRP: [J][R], [R][P(K-1)]
};

// ------------------------------------------------------------------ device memory
// cudaMalloc, except that the next n calls fail as if the device were out of memory after
// srp_debug_fail_allocations(n) (failure-detection tests).
cudaError_t device_alloc(void** ptr, size_t bytes);

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
void clear_error();

#define SRP_CUDA_TRY(expr)                                                          \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      ::srp::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));         \
      return SRP_ECUDA;                                                             \
    }                                                                               \
  } while (0)

// ------------------------------------------------------------------ host fitting
struct Geometry {
  int M = 0, P = 0, J = 0, N = 0, K = 0, L = 0;
  double fs = 0, c = 0;
  std::vector<int> pm, pmp;      // pair p -> (m, m'), m > m'
  std::vector<int> Np, off;      // N_p and the offset of pair p in the stacked xi
  std::vector<double> tau;       // [J][P] TDOA in samples, Delta t_p(i) * fs
};

// Builds pairs, N_p, offsets and the FP64 TDOA table (Eq. Deltat_i, Eq. N_p).
srp_status build_geometry(const srp_plan_desc& d, Geometry& g);

// Row i of Lambda (Eq. Lambda_p): sinc(tau_p(i) - n) for every pair and lag
// n = -N_p..N_p (ascending), written to row[0..L).
void lambda_row(const Geometry& g, int i, double* row);

// Top-R eigenpairs of Lambda^T Lambda -> tall [J][R] (= Lambda V_R), fat [R][L]
// (= V_R^T), sigma [L] (descending singular values).
srp_status fit_low_rank(const Geometry& g, int R, std::vector<float>& tall,
                        std::vector<float>& fat, std::vector<double>& sigma);

// Large L: the same factors from a subspace iteration on Lambda^T Lambda whose products
// Lambda X and Lambda^T Y run on the device in FP64 (k_fit.cu); sigma holds the leading
// singular values that the iteration resolves (at least R).
srp_status fit_low_rank_device(const Geometry& g, int R, std::vector<float>& tall,
                               std::vector<float>& fat, std::vector<double>& sigma,
                               cudaStream_t s);

// LR-SRP: the best rank-R approximation of the complex SRP matrix H (J x P(K-1)),
// H_tall = H V_R (J x R, row-major), H_fat = V_R^H (R x P(K-1)), by a device subspace
// iteration on H^H H (k_fit.cu).
srp_status fit_lr_device(const Geometry& g, int R, std::vector<std::complex<double>>& tall,
                         std::vector<std::complex<double>>& fat, std::vector<double>& sigma,
                         cudaStream_t s);

// Symmetric eigen-decomposition (cyclic Jacobi).  A: n x n row-major, destroyed;
// V: eigenvectors as columns; d: eigenvalues (unsorted).
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V, std::vector<double>& d);

// The Q_Lambda largest-magnitude entries of Lambda as CSR rows.
srp_status fit_sparse(const Geometry& g, long long nnz, std::vector<long long>& row_ptr,
                      std::vector<int>& col, std::vector<float>& val, long long& tied);

unsigned host_threads();

// ------------------------------------------------------------------ kernels
// Operand type of a contraction: FP32 (CUDA cores), or one or two (hi + lo) planes of
// FP16, BF16 or TF32 for the tensor cores.  The values double as the front kernel's output
// codes.
enum class OpType { F32 = 0, F16 = 1, BF16 = 2, F16X2 = 3, BF16X2 = 4, TF32 = 5, TF32X2 = 6 };
inline bool op_split(OpType t) {
  return t == OpType::F16X2 || t == OpType::BF16X2 || t == OpType::TF32X2;
}
inline bool op_tf32(OpType t) { return t == OpType::TF32 || t == OpType::TF32X2; }
inline size_t op_bytes(OpType t) { return t == OpType::F32 || op_tf32(t) ? 4 : 2; }
// tensor-core k-blocks (128-byte rows) per 64 operand columns
inline int op_kb_per64(OpType t) { return op_tf32(t) ? 2 : 1; }
// Front end: window + real DFT of length N + PHAT, y-hat [F][M][K] (bin 0 zeroed).
cudaError_t launch_stft_phat(const float* frames, int F, int M, int N, const float* window,
                             const float2* twiddle, float2* yhat, cudaStream_t s);
// Cross-spectra, two-sided iFFT of length N, lag selection -> out [F][out_cols] in operand
// type t (xi in columns 0..L-1, zeros beyond; FP32 xi: t = F32, out_cols = L).
cudaError_t launch_gcc_samples(const float2* yhat, int F, int M, int P, int N,
                               const int2* pairs, const int* Np, const int* off, int L,
                               const float2* twiddle, OpType t, void* out, void* out_lo,
                               int out_cols, cudaStream_t s);
// Lag windows up to this N_p are sampled in the matrix form of Eq. xi_computed.
int gcc_direct_max_lag();
// The same samples (N_p <= gcc_direct_max_lag()) as a per-frame GEMM on the warp-level
// tensor cores from y-hat [F][M][N/2] in global memory, written in operand type t into
// out [F][out_cols] (zero padded beyond L); stab = front_sampling_table(N, max_Np).
bool gcc_mma_supported(int M, int N, int max_Np);
// The iFFT sampling for 2K = 1024 and operands of 8 to 11 bits (BF16, FP16, TF32) as 32 x 32
// DFTs on the warp-level tensor cores; tables = dft_tables.
bool gcc_dft_supported(int M, int N, OpType t);
void dft_tables(std::vector<uint4>& tab);
cudaError_t launch_gcc_dft(const float2* yhat, int F, int M, int P, int N, const int2* pairs,
                           const int* Np, const int* off, int L, const uint4* tables, OpType t,
                           void* out, void* out_lo, int out_cols, cudaStream_t s);
cudaError_t launch_gcc_mma(const float2* yhat, int F, int M, int P, int N, const int2* pairs,
                           const int* Np, const int* off, int L, const uint4* stab, int max_Np,
                           OpType t, void* out, void* out_lo, int out_cols, cudaStream_t s);
// Frames from consecutive hops [B][M][hop] and the history [M][N - hop] (streaming front).
cudaError_t launch_stream_frames(const float* hops, int B, int M, int hop, int N,
                                 const float* hist_in, float* frames, float* hist_out,
                                 cudaStream_t s);
// Cross-spectra packed as the conv GEMM operand A [F][P*N]:
// A[f][p*N + k] = Re psi_p(k), A[f][p*N + K + k] = Im psi_p(k), k = 0..K-1, psi(0) = 0.
// Fused STFT + PHAT + sampling (+ Lambda_fat) per frame: writes xi (ftab == NULL)
// or u = Lambda_fat xi * scale, rows of out_cols entries (zero padded) in operand type t.
// The sampling and the Lambda_fat product are per-frame GEMMs on the warp-level tensor
// cores against two tables in fragment order, FP16 hi + lo: stab from
// front_sampling_table(N, max_Np) (exp(j pi k n / K) for n = -max_Np..max_Np) and ftab
// from front_fat_table(fat [Rp][L], Rp, L).
// Returns cudaErrorNotSupported where front_supported() is false (the caller then runs
// the separate kernels).
bool front_supported(int M, int N, int L, int max_Np);
void front_sampling_table(int N, int max_Np, std::vector<uint4>& tab);
void front_fat_table(const float* fat, int Rp, int L, std::vector<uint4>& tab);
cudaError_t launch_front(const float* frames, int F, int M, int N, const float* window,
                         const float2* twiddle, int P, const int2* pairs, const int* Np,
                         const int* off, const uint4* stab, int L, int max_Np, const uint4* ftab,
                         int Rp, int out_cols, float scale, OpType t, void* out, void* out_lo,
                         cudaStream_t s);

cudaError_t launch_conv_pack(const float2* yhat, int F, int M, int P, int N, const int2* pairs,
                             OpType t, void* A, void* A_lo, cudaStream_t s);
// The same operand straight from the frames: the front kernel's STFT + PHAT in shared
// memory, then the cross-spectra packed (no y-hat round trip through memory).
bool front_conv_supported(int M, int N);
cudaError_t launch_front_conv(const float* frames, int F, int M, int N, const float* window,
                              const float2* twiddle, int P, const int2* pairs, OpType t, void* A,
                              void* A_lo, cudaStream_t s);
// SRP matrix in GEMM layout B [J][P*N]: 2cos(theta), -2sin(theta), theta = 2 pi k tau / N.
cudaError_t launch_conv_matrix(const double* tau_dev, int J, int P, int N, OpType t, void* B,
                               void* B_lo, cudaStream_t s);
// The same rows from the TDOAs split as tau_hi + tau_lo (FP32 phases, ~4e-7 rad): per-call
// generation of chunks of cells.
cudaError_t launch_conv_matrix_split(const float* tau_hi, const float* tau_lo, int J, int P, int N,
                                     OpType t, void* B, void* B_lo, cudaStream_t s);
// Z[F][J] = A B^T in FP32 FFMA, fused per-frame argmax keys.  For long reductions
// (sgemm_split_count(Kd) > 1) the k range is split into slices of <= 16384 terms whose
// partial maps go to split_ws [nsplit][F][J] and are summed in FP64.
int sgemm_split_count(int Kd);
// With tau_hi != NULL, B is not read: the SRP matrix of P pairs and frame length N is
// generated on the fly from the split TDOA table tau_hi + tau_lo [J][P] (FP32 pairs).
cudaError_t launch_sgemm_nt_argmax(const float* A, const float* B, float* Z,
                                   unsigned long long* keys, int F, int J, int Kd,
                                   float* split_ws, cudaStream_t s, const float* tau_hi = nullptr,
                                   const float* tau_lo = nullptr, int P = 0, int N = 0);
// Sums nz partial maps [nz][F][J] in FP64 into Z (rows ldz floats apart, 0: J) and merges
// the argmax keys (cell indices offset by col0).
cudaError_t launch_split_reduce(const float* ws, int nz, float* Z, unsigned long long* keys,
                                int F, int J, cudaStream_t s, int ldz = 0, int col0 = 0);
// Tensor-core contraction (tcgen05, k_tc_gemm.cu): Z[F][J] = A B^T with K-major operands
// A [F][Kd], B [J][Kd] of type t (FP16, BF16 or TF32; Kd a multiple of tc_gemm_k_block()),
// FP32 accumulation, fused argmax keys.  The split types (op_split) run three products over
// hi and lo planes.  With kb_ptr
// (device, [ceil(J / tc_gemm_cell_tile()) + 1]) and kb_idx, the cells of list tile n only
// visit the 64-column windows starting at the columns kb_idx[kb_ptr[n] .. kb_ptr[n+1])
// (block-sparse B; multiples of 8, windows disjoint, columns past Kd read as zero).  Dense reductions whose
// output tiles do not fill the GPU are split into tc_gemm_slices(...) slices written to
// split_ws (tc_gemm_workspace_floats(...) floats suffice for any F <= F_max) and summed
// in FP64.  A bounded wait that runs out stores a non-zero code in *err.
struct TcGemm {
  const void* A = nullptr;
  const void* A_lo = nullptr;
  const void* B = nullptr;
  const void* B_lo = nullptr;
  OpType t = OpType::F16;
  int F = 0, J = 0, Kd = 0;
  const int* kb_ptr = nullptr;
  const int* kb_idx = nullptr;
  float* Z = nullptr;
  int ldz = 0;        // row stride of Z in floats (0: J); with col0 a column block of a wider map
  int col0 = 0;       // index of Z's first column in the map (argmax keys carry col0 + column)
  bool no_split = false;  // never split the reduction into slices
  int force_slices = 0;   // > 0: split the (dense) reduction into this many slices
  unsigned long long* keys = nullptr;
  float* split_ws = nullptr;
  int* err = nullptr;
  int variant = -1;   // TC_* kernel variant, -1: the heuristic's choice
  int max_ctas = 0;   // cap on the persistent grid (0: one CTA per SM)
  bool stall = false; // failure-detection test: no operand load is issued, the bounded
                      // waits (0.2 s) run out and *err records the timeout
};
// Kernel variants (tile width and shared-memory split) the autotuner chooses from.
enum { TC_LONG_256 = 0,   // 128x256 tiles, 4 operand stages, 1 output box per epilogue warp
       TC_SHORT_256 = 1,  // 128x256 tiles, 2 stages, 4 boxes (short reductions)
       TC_LONG_128 = 2,   // 128x128 tiles, 4 stages, 2 boxes (small grids: twice the tiles)
       TC_FUSED3_256 = 3, // hi + lo precisions: 128x256 tiles, 2 stages each holding the hi and
                          // lo planes of A and B for one k-block (the three products in turn)
       TC_NBASE = 4,      // variant v + 4: variant v in clusters of 2 CTAs (two frame tiles)
                          // that share each B tile by TMA multicast; v + 8: clusters of
                          // 2 x 2 that also share each A tile (dense reductions)
       TC_NVARIANTS = 12 };
// CTAs per cluster of a variant (1, 2 or 4).
int tc_gemm_cluster_size(int variant);
bool tc_gemm_variant_valid(int variant, OpType t);
int tc_gemm_default_variant(int Kd, OpType t, int F);
cudaError_t launch_tc_gemm(const TcGemm& g, int num_sms, cudaStream_t s);
int tc_gemm_slices(int F, int J, int Kd, OpType t, int num_sms);
size_t tc_gemm_workspace_floats(int F_max, int J, int Kd, OpType t, int num_sms);
int tc_gemm_cell_tile();
// Resolves the tensor-map encoder and sets the kernel's shared-memory attribute on the
// current device (done at plan creation, so that later launches can be graph-captured).
cudaError_t tc_gemm_prepare();
int tc_gemm_k_block();

// Operand preparation (k_pack.cu).  pack16: X [rows][C] FP32 -> [rows][Cpad] (zero
// padded) in type t after multiplying by scale; csr_to_dense: CSR taps -> zeroed dense
// [J][Cpad]; interp_dense: SI sinc (td = false) or TD one-hot (td = true) entries from the
// FP64 TDOA table tau [J][P], column l < L being pair col_pair[l] at lag col_lag[l].
cudaError_t launch_pack16(const float* X, int rows, int C, int Cpad, float scale, OpType t,
                          void* hi, void* lo, cudaStream_t s);
cudaError_t launch_csr_to_dense(const long long* row_ptr, const int2* taps, int J, int Cpad,
                                OpType t, void* hi, void* lo, cudaStream_t s);
cudaError_t launch_interp_dense(const double* tau, int J, int P, const int* col_pair,
                                const int* col_lag, int L, int Cpad, bool td, OpType t, void* hi,
                                void* lo, cudaStream_t s);

// SLRI: U[F][R] = xi Lambda_fat^T ; Z = U Lambda_tall^T (fused argmax keys).
cudaError_t launch_slri_fat(const float* xi, const float* fat, float* U, int F, int L, int R,
                            cudaStream_t s);
cudaError_t launch_slri_tall(const float* U, const float* tall, float* Z,
                             unsigned long long* keys, int F, int J, int R, cudaStream_t s);
// SSPI: Z[f][i] = sum over row i's taps of val * xi[f][col] (fused argmax keys).
cudaError_t launch_sspi(const float* xi, const long long* row_ptr, const int2* taps, float* Z,
                        unsigned long long* keys, int F, int J, int L, int num_sms,
                        cudaStream_t s);
// Fused front end (k_frontend.cu): STFT + PHAT + sampling (+ Lambda_fat xi), one CTA per
// frame.  These are its per-batch arguments.
struct FrontParams {
  const float* frames;
  int M, P, L;
  const float* window;
  const float2* twiddle;
  const int2* pairs;
  const int* Np;
  const int* off;
  const uint4* stab;  // sampling operand in fragment order (front_sampling_table)
  int nq0, NT;        // lag offset of its columns (max N_p) and its n-tiles
  int fbuf_floats;    // FFT buffers / sampling partials (floats)
  const uint4* ftab;  // SLRI: Lambda_fat in fragment order (front_fat_table); NULL: write xi
  int Rp;
  int out_cols;       // row length of the output (L, Lpad, Rp or 64)
  float scale;        // applied to u before packing
  int ot;             // operand type of the output
  void* out;
  void* out_lo;
  int conv_out;       // 1: write the conv operand row [P*N] of psi instead of sampling
};
// front_params: the arguments launch_front would build (frames and out left NULL), for a
// kernel instantiated with NTM n-tiles (at least front_ntm(max_Np): a wider instantiation
// serves narrower plans, whose partial buffers are then sized for it).
FrontParams front_params(int M, int N, const float* window, const float2* twiddle, int P,
                         const int2* pairs, const int* Np, const int* off, const uint4* stab,
                         int L, int max_Np, const uint4* ftab, int Rp, int out_cols, float scale,
                         OpType t, int NTM);
size_t front_smem_bytes(int M, int N, int L, int max_Np);
size_t front_smem_bytes_ntm(int M, int N, int L, int NTM);
int front_ntm(int max_Np);
int front_ntiles(int max_Np);
// Grouped front end: items [(params index, frame)], *count of them, on `grid` CTAs that
// walk the list; every entry shares N and front_ntm(max_Np); smem = the largest
// front_smem_bytes of the entries.
cudaError_t launch_front_group(const FrontParams* params, const int2* items, const int* count,
                               int grid, int N, int NTM, size_t smem, cudaStream_t s);
// Grouped interpolation (serving, FP32): one entry per session in a launch.
struct GroupInterp {
  const float* in;            // SLRI: u [F][Rp];  SSPI: xi [F][L]
  const float* tall;          // SLRI: Lambda_tall [J][Rp]
  const long long* row_ptr;   // SSPI: taps as CSR rows
  const int2* taps;
  float* Z;                   // maps [F][J]
  unsigned long long* keys;   // argmax keys [F]
  int F, J, L;
};
// SLRI: items (entry, cell block of slri_tall_cells_per_block(Rp) cells, frame block of 64);
// every entry has the padded rank Rp.
int slri_tall_cells_per_block(int Rp);
cudaError_t launch_slri_tall_group(const GroupInterp* g, const int4* items, const int* count,
                                   int grid, int Rp, cudaStream_t s);
// SSPI (whole-vector gather, sspi_full_fits(L) for every entry): items (entry, frame group of
// sspi_group_frames(Lmax) frames, first and end 64-cell row block).
int sspi_group_frames(int Lmax);
cudaError_t launch_sspi_group(const GroupInterp* g, const int4* items, const int* count, int grid,
                              int Lmax, cudaStream_t s);
// SSPI for long sample vectors: per 64-cell row block only the columns its taps use are
// staged (blk_ptr [J/64 + 1], blk_cols; taps carry positions in the block's list), FB
// frames per block (32, 16, .., 1) chosen so that sspi_band_smem(umax, FB) fits.
bool sspi_full_fits(int L);
size_t sspi_band_smem(int U, int FB);
cudaError_t launch_sspi_band(const float* xi, const long long* row_ptr, const int2* taps,
                             const long long* blk_ptr, const int* blk_cols, int umax, int FB,
                             float* Z, unsigned long long* keys, int F, int J, int L,
                             cudaStream_t s);
// keys -> argmax (lowest index among equal maxima).
cudaError_t launch_argmax_finalize(const unsigned long long* keys, int* argmax, int F,
                                   cudaStream_t s);
// Several estimates per frame (k_peaks.cu): pick 0 from the argmax keys of the maps Z
// [F][J], then K - 1 exclusion passes; picks [F][K] (-1: none left), values [F][K] or NULL.
// keys are left cleared.  grid: the cells' FP32 coordinates (x, y, z, 0).
constexpr int kPeaksMax = 16;
cudaError_t launch_peaks(const float* Z, int F, int J, const float4* grid,
                         unsigned long long* keys, int K, float t, int* picks, float* values,
                         cudaStream_t s);
int peaks_launches(int F, int K);

}  // namespace srp

// ------------------------------------------------------------------ the plan
struct srp_plan_s {
  int device = 0;
  srp_plan_desc desc{};
  srp::Geometry g;
  int R = 0;
  long long nnz = 0, tied = 0;
  int Fmax = 0;
  int num_sms = 0;
  srp::OpType op = srp::OpType::F32;
  int Lpad = 0;       // L rounded up to a multiple of 64 (dense interpolation operands)
  int slri_exp = 0;   // tensor-core SLRI: u scaled by 2^-slri_exp, Lambda_tall by 2^slri_exp;
                      // LR: u scaled by 2^slri_exp, the tall factor by 2^-slri_exp
  int lr_kd = 0;      // LR: contraction depth of the tall product (2R padded to 64)
  int max_Np = 0;     // largest N_p over the pairs
  int tc_variant = -1;     // tensor-core kernel variant chosen by srp_plan_autotune (-1: heuristic)
  bool use_front = false;  // interpolation methods: one fused front-end launch per chunk
  bool use_mma_sampling = false;  // otherwise, short lag windows: sampling by gcc_mma
  bool use_dft_sampling = false;  // otherwise, 2K = 1024, 8-11-bit operands: gcc_dft1024
  bool fat_gemm = false;   // SLRI with long sample vectors: u = Lambda_fat xi as a GEMM
  bool h_generated = false;  // conv FP32: SRP matrix generated inside the GEMM, not stored
  int h_slices = 0;          //   slices of each chunk's reduction (d_split holds the partials)
  int h_chunk = 0;           // conv on the tensor cores, SRP matrix too large to store: cells
                             // per chunk whose rows are generated into d_H before each GEMM
                             // (from d_tau_hi / d_tau_lo)
  std::vector<double> sigma;
  std::vector<std::complex<double>> lr_tall, lr_fat;  // LR-SRP factors kept for srp_plan_save
  std::vector<long long> h_row_ptr;  // SSPI taps kept on the host for export
  std::vector<int> h_col;
  std::vector<float> h_val;
  // device tables
  int2* d_pairs = nullptr;
  int* d_Np = nullptr;
  int* d_off = nullptr;
  float2* d_twiddle = nullptr;
  float* d_window = nullptr;
  void* d_H = nullptr;
  float* d_tau_hi = nullptr;  // conv with the SRP matrix generated on the fly: split TDOAs
  float* d_tau_lo = nullptr;
  void* d_H_lo = nullptr;
  float* d_tall = nullptr;
  float* d_fat = nullptr;
  long long* d_row_ptr = nullptr;
  int2* d_taps = nullptr;
  long long* d_blk_ptr = nullptr;  // FP32 SSPI, long sample vectors: per-block column lists
  int* d_blk_cols = nullptr;
  int sspi_umax = 0;               //   (0: the whole-L gather), the longest list
  int sspi_fb = 0;                 //   frames per thread block
  void* d_B = nullptr;     // dense interpolation operand [J][Lpad] (SI, TD, tensor-core SSPI)
  void* d_B_lo = nullptr;  //   or Lambda_tall as [J][64] (tensor-core SLRI); lo plane for FP16X2
  int* d_kb_ptr = nullptr;  // block-sparse window lists per cell tile of d_B (first columns)
  int* d_kb_idx = nullptr;
  // scratch
  float2* d_yhat = nullptr;
  void* d_A = nullptr;
  void* d_A_lo = nullptr;
  float* d_split = nullptr;  // conv FP32 split-reduction partial maps
  float* d_xi = nullptr;
  float* d_U = nullptr;
  unsigned long long* d_keys = nullptr;
  unsigned long long* d_keys2 = nullptr;  // LR: keys of the fat product (not an argmax)
  void* d_A2 = nullptr;     // LR: u as the operand of the tall product [Fmax][lr_kd]
  void* d_A2_lo = nullptr;
  int* d_err = nullptr;  // non-zero after a bounded wait inside a kernel ran out
  bool use_front_conv = false;  // conv / LR operand from the fused front kernel
  bool stall_next = false;  // srp_debug_stall_next_contraction
  uint4* d_stab = nullptr;  // fused front end or gcc_mma: the sampling operand (front_sampling_table);
                            // gcc_dft1024: its DFT tables (dft_tables)
  uint4* d_ftab = nullptr;  // fused front end, SLRI: Lambda_fat (front_fat_table)
  // staging for srp_map_host, and its copy pipeline (two D2H streams and one H2D stream;
  // events recycled round-robin to order them against the compute stream)
  cudaStream_t copy_streams[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t pipe_events[srp::kHostPipe] = {};
  float* d_stage_frames = nullptr;
  // streaming (srp_stream_push): hop size, two history buffers [M][N - hop], frame staging
  int stream_hop = 0;
  int stream_cur = 0;
  float* d_hist[2] = {nullptr, nullptr};
  float* d_stream_frames = nullptr;
  float* d_est_maps = nullptr;  // estimates-only calls of FP32 plans: map scratch [Fmax][J]
  std::vector<float> h_grid4;    // the cells' coordinates rounded to FP32, (x, y, z, 0)
  float4* d_grid4 = nullptr;     // the same on the device (srp_map_peaks, made on first use)
  float* d_peak_maps = nullptr;  // srp_map_peaks without maps: L2-sized map scratch
  int peak_chunk = 0;            //   frames per chunk of that scratch
  float* d_stage_maps = nullptr;
  int* d_stage_arg = nullptr;
  size_t device_bytes = 0;
  double fit_seconds = 0;
  long long launches = 0;  // kernels launched by srp_map / srp_map_host / srp_gcc_samples
  // per-stage timing: 5 events per internal chunk of the last call
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  int chunks_recorded = 0;
};
