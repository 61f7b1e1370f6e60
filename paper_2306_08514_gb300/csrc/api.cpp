// The C-ABI of libsrp (include/libsrp.h): argument checks, plan construction, and the
// per-call launch sequence of the SRP path.
#include "srp_internal.h"

#include <mutex>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <functional>

namespace srp {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

namespace {

srp_status fail(srp_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Everything that can be checked without a GPU.
srp_status validate(const srp_plan_desc* d) {
  if (!d) return fail(SRP_EINVAL, "desc is NULL");
  if (d->M < 2 || d->M > 64) return fail(SRP_EINVAL, "M must be in 2..64");
  if (!d->mic_xyz) return fail(SRP_EINVAL, "mic_xyz is NULL");
  // the split-K reduction covers 1024 cells per block row and the FP32 FFMA GEMM 128, with
  // at most 65535 block rows (checked before grid_xyz is read)
  if (d->J < 1 || d->J > 65535 * 1024) return fail(SRP_EINVAL, "J must be in 1..67107840");
  if (d->precision == SRP_FP32 && d->J > 65535 * 128)
    return fail(SRP_EINVAL, "SRP_FP32 plans take J <= 8388480 (use a tensor-core precision)");
  if (!d->grid_xyz) return fail(SRP_EINVAL, "grid_xyz is NULL");
  if (!(d->fs > 0) || !std::isfinite(d->fs)) return fail(SRP_EINVAL, "fs must be > 0");
  if (!is_pow2(d->N) || d->N < 256 || d->N > 2048)
    return fail(SRP_EINVAL, "N must be a power of two in 256..2048");
  if (d->window < 0 || d->window > 2) return fail(SRP_EINVAL, "window must be 0, 1 or 2");
  if (!(d->c > 0) || !std::isfinite(d->c)) return fail(SRP_EINVAL, "c must be > 0");
  if (d->n_aux < 0 || d->n_aux > 64) return fail(SRP_EINVAL, "n_aux must be in 0..64");
  if (d->max_frames < 1 || d->max_frames > 65536)
    return fail(SRP_EINVAL, "max_frames must be in 1..65536");
  if (d->far_field != 0 && d->far_field != 1) return fail(SRP_EINVAL, "far_field must be 0 or 1");
  if (d->h_on_the_fly < -1 || d->h_on_the_fly > 1) return fail(SRP_EINVAL, "h_on_the_fly must be -1, 0 or 1");
  for (int i = 0; i < 3 * d->M; ++i)
    if (!std::isfinite(d->mic_xyz[i])) return fail(SRP_EINVAL, "mic_xyz has a non-finite value");
  for (long long i = 0; i < 3ll * d->J; ++i)
    if (!std::isfinite(d->grid_xyz[i])) return fail(SRP_EINVAL, "grid_xyz has a non-finite value");
  if (d->far_field)
    for (long long i = 0; i < d->J; ++i) {
      const double* q = d->grid_xyz + 3 * i;
      if (std::fabs(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] - 1.0) > 1e-9)
        return fail(SRP_EINVAL, "far-field grid rows must be unit vectors");
    }
  if (d->method < SRP_CONV || d->method > SRP_LR) return fail(SRP_EINVAL, "unknown method");
  if (d->precision < SRP_FP32 || d->precision > SRP_TF32)
    return fail(SRP_EINVAL, "unknown precision");
  if (d->method == SRP_TD && d->n_aux < 1)
    return fail(SRP_EINVAL, "conv. TD-SRP needs n_aux >= 1 (the rounded lag must be sampled)");
  return SRP_OK;
}

void window_table(int N, int kind, std::vector<float>& w) {
  w.resize(N);
  for (int n = 0; n < N; ++n) {
    const double h = 0.5 - 0.5 * std::cos(2.0 * M_PI * n / N);
    w[n] = static_cast<float>(kind == SRP_WIN_HANN ? h : kind == SRP_WIN_SQRT_HANN ? std::sqrt(h) : 1.0);
  }
}

template <typename T>
cudaError_t dalloc(srp_plan_s* p, T** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = device_alloc(reinterpret_cast<void**>(ptr), bytes);
  if (e == cudaSuccess) p->device_bytes += bytes;
  return e;
}

void free_plan(srp_plan_s* p) {
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  for (cudaEvent_t e : p->pipe_events)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t cs : p->copy_streams)
    if (cs) cudaStreamDestroy(cs);
  void* ptrs[] = {p->d_pairs, p->d_Np, p->d_off, p->d_twiddle, p->d_window, p->d_H, p->d_H_lo,
                  p->d_tall, p->d_fat, p->d_row_ptr, p->d_taps, p->d_yhat, p->d_A, p->d_A_lo,
                  p->d_split, p->d_xi, p->d_U, p->d_keys, p->d_err, p->d_stage_frames, p->d_stage_maps, p->d_stab, p->d_ftab,
                  p->d_stage_arg, p->d_B, p->d_B_lo, p->d_kb_ptr, p->d_kb_idx, p->d_hist[0],
                  p->d_hist[1], p->d_stream_frames, p->d_est_maps, p->d_A2, p->d_A2_lo,
                  p->d_keys2, p->d_tau_hi, p->d_tau_lo, p->d_grid4, p->d_peak_maps,
                  p->d_blk_ptr, p->d_blk_cols};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete p;
}

#define SRP_ALLOC(plan, ptr, bytes)                                                        \
  do {                                                                                     \
    cudaError_t _e = dalloc(plan, &(ptr), (bytes));                                        \
    if (_e != cudaSuccess) {                                                               \
      cudaGetLastError();                                                                  \
      set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(_e)); \
      free_plan(plan);                                                                     \
      return _e == cudaErrorMemoryAllocation ? SRP_ENOMEM : SRP_ECUDA;                     \
    }                                                                                      \
  } while (0)

#define SRP_PLAN_CUDA(plan, expr)                                                          \
  do {                                                                                     \
    cudaError_t _e = (expr);                                                               \
    if (_e != cudaSuccess) {                                                               \
      set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                       \
      free_plan(plan);                                                                     \
      return SRP_ECUDA;                                                                    \
    }                                                                                      \
  } while (0)

OpType op_of(int precision) {
  switch (precision) {
    case SRP_BF16: return OpType::BF16;
    case SRP_FP16: return OpType::F16;
    case SRP_BF16X3: return OpType::BF16X2;
    case SRP_FP16X3: return OpType::F16X2;
    case SRP_TF32: return OpType::TF32;
    case SRP_TF32X3: return OpType::TF32X2;
    default: return OpType::F32;
  }
}

// Contraction depth of the tensor-core SLRI product (R <= 64 padded to one k-block); also
// the multiple that pads L for the dense interpolation operands.
constexpr int kSlriKd = 64;

// Largest L for which the low-rank fit eigen-decomposes the L x L Gram matrix on the host.
constexpr int kGramMaxL = 768;

// Beyond this L (without the fused front end) SLRI forms u = Lambda_fat xi as a GEMM.
constexpr int kFatGemmMinL = 1024;

// A stored SRP matrix above this size is generated on the fly instead (FP32 conv) or in
// chunks of cells before each chunk's GEMM (tensor cores, chunks of at most kMaxChunkH).
constexpr double kMaxStoredH = 64e9;
constexpr double kMaxChunkH = 48e9;
constexpr int kChunkSliceSteps = 512;  // k-steps per reduction slice of a chunk's GEMM
constexpr int kChunkMaxSlices = 64;

// One chunk of at most Fmax frames through the whole path.
constexpr int kMaxChunkEvents = 4096;

srp_status mark(srp_plan_s* p, int stage, cudaStream_t s) {
  if (!p->profiling || p->chunks_recorded >= kMaxChunkEvents) return SRP_OK;
  const size_t idx = static_cast<size_t>(p->chunks_recorded) * 5 + stage;
  while (p->events.size() <= idx) {
    cudaEvent_t e;
    SRP_CUDA_TRY(cudaEventCreate(&e));
    p->events.push_back(e);
  }
  SRP_CUDA_TRY(cudaEventRecord(p->events[idx], s));
  return SRP_OK;
}

#define SRP_MARK(p, stage, s)                      \
  do {                                             \
    srp_status _st = mark((p), (stage), (s));      \
    if (_st != SRP_OK) return _st;                 \
  } while (0)

// Z = A B^T with the plan's operand type: FP32 FFMA (SIMT) or the tensor cores.
cudaError_t contract_to(srp_plan_s* p, const void* A, const void* A_lo, const void* B,
                        const void* B_lo, int Kd, const int* kb_ptr, const int* kb_idx, int F,
                        float* out, int Jout, unsigned long long* keys, cudaStream_t s) {
  if (p->op == OpType::F32) {
    p->launches += sgemm_split_count(Kd) > 1 ? 2 : 1;
    return launch_sgemm_nt_argmax(static_cast<const float*>(A), static_cast<const float*>(B), out,
                                  keys, F, Jout, Kd, p->d_split, s);
  }
  p->launches += (!kb_ptr && tc_gemm_slices(F, Jout, Kd, p->op, p->num_sms) > 1) ? 2 : 1;
  TcGemm tg;
  tg.A = A;
  tg.A_lo = A_lo;
  tg.B = B;
  tg.B_lo = B_lo;
  tg.t = p->op;
  tg.F = F;
  tg.J = Jout;
  tg.Kd = Kd;
  tg.kb_ptr = kb_ptr;
  tg.kb_idx = kb_idx;
  tg.Z = out;
  tg.keys = keys;
  tg.split_ws = p->d_split;
  tg.err = p->d_err;
  tg.variant = p->tc_variant;
  tg.stall = p->stall_next;
  p->stall_next = false;
  return launch_tc_gemm(tg, p->num_sms, s);
}

// A block of jn map columns starting at column c0 (rows J apart): Z[:, c0 + j] = A B_j^T
// for the jn rows of B, argmax keys over the whole map; the reduction in the plan's
// h_slices slices (summed in FP64).
cudaError_t contract_cols(srp_plan_s* p, const void* A, const void* A_lo, const void* B,
                          const void* B_lo, int Kd, int F, float* out, int c0, int jn,
                          cudaStream_t s) {
  p->launches += p->h_slices > 1 ? 2 : 1;
  TcGemm tg;
  tg.A = A;
  tg.A_lo = A_lo;
  tg.B = B;
  tg.B_lo = B_lo;
  tg.t = p->op;
  tg.F = F;
  tg.J = jn;
  tg.Kd = Kd;
  tg.Z = out;
  tg.ldz = p->g.J;
  tg.col0 = c0;
  tg.force_slices = p->h_slices;
  tg.no_split = p->h_slices <= 1;
  tg.split_ws = p->d_split;
  tg.keys = p->d_keys;
  tg.err = p->d_err;
  tg.variant = p->tc_variant;
  tg.stall = p->stall_next;
  p->stall_next = false;
  return launch_tc_gemm(tg, p->num_sms, s);
}

// Z = A B^T into the maps, argmax keys of the plan.
cudaError_t contract(srp_plan_s* p, const void* A, const void* A_lo, const void* B, const void* B_lo,
                     int Kd, const int* kb_ptr, const int* kb_idx, int F, float* maps, cudaStream_t s) {
  return contract_to(p, A, A_lo, B, B_lo, Kd, kb_ptr, kb_idx, F, maps, p->g.J, p->d_keys, s);
}

// Samples of the TD GCCs (Eq. xi_p_ifft / xi_computed) into out [F][cols] in operand type t
// (zero padded beyond L): for short lag windows by the per-frame sampling GEMM on the
// warp-level tensor cores, otherwise (or where its staged spectra would not fit in shared
// memory) by the two-pairs-per-iFFT kernel -- for 2K = 1024 and 8-11-bit operands its
// 32 x 32 form on the warp-level tensor cores; all write the operand directly.
cudaError_t sample_to(srp_plan_s* p, const float2* yhat, int F, void* out, void* out_lo, int cols,
                      OpType t, cudaStream_t s) {
  const Geometry& g = p->g;
  ++p->launches;
  if (p->use_mma_sampling)
    return launch_gcc_mma(yhat, F, g.M, g.P, g.N, p->d_pairs, p->d_Np, p->d_off, g.L, p->d_stab,
                          p->max_Np, t, out, out_lo, cols, s);
  if (p->use_dft_sampling && gcc_dft_supported(g.M, g.N, t))
    return launch_gcc_dft(yhat, F, g.M, g.P, g.N, p->d_pairs, p->d_Np, p->d_off, g.L, p->d_stab,
                          t, out, out_lo, cols, s);
  return launch_gcc_samples(yhat, F, g.M, g.P, g.N, p->d_pairs, p->d_Np, p->d_off, g.L,
                            p->d_twiddle, t, out, out_lo, cols, s);
}

// FP32 SSPI gather of p->d_xi into maps: the whole-L kernel, or the per-block column lists
// for long sample vectors.
cudaError_t sspi_gather(srp_plan_s* p, float* maps, int F, cudaStream_t s) {
  const Geometry& g = p->g;
  if (p->sspi_umax > 0)
    return launch_sspi_band(p->d_xi, p->d_row_ptr, p->d_taps, p->d_blk_ptr, p->d_blk_cols,
                            p->sspi_umax, p->sspi_fb, maps, p->d_keys, F, g.J, g.L, s);
  return launch_sspi(p->d_xi, p->d_row_ptr, p->d_taps, maps, p->d_keys, F, g.J, g.L,
                     p->num_sms, s);
}

// A counted kernel launch of the per-call path.
#define SRP_LAUNCH(expr)  \
  do {                    \
    ++p->launches;        \
    SRP_CUDA_TRY(expr);   \
  } while (0)

srp_status run_chunk(srp_plan_s* p, const float* frames, int F, float* maps, int* argmax,
                     cudaStream_t s) {
  const Geometry& g = p->g;
  SRP_CUDA_TRY(cudaMemsetAsync(p->d_keys, 0, sizeof(unsigned long long) * F, s));
  SRP_MARK(p, 0, s);
  const int method = p->desc.method;
  const int Rp = (p->R + 7) / 8 * 8;
  if (p->use_front) {
    // one fused launch: STFT + PHAT + sampling (+ Lambda_fat for SLRI) -> the operand
    const bool tc = p->op != OpType::F32;
    const bool slri = method == SRP_SLRI;
    void* out = slri ? (tc ? p->d_A : p->d_U)
                     : ((method == SRP_SSPI && !tc) ? static_cast<void*>(p->d_xi) : p->d_A);
    const int cols = slri ? (tc ? kSlriKd : Rp) : ((method == SRP_SSPI && !tc) ? g.L : p->Lpad);
    const float scale = slri && tc ? std::ldexp(1.f, -p->slri_exp) : 1.f;
    SRP_LAUNCH(launch_front(frames, F, g.M, g.N, p->d_window, p->d_twiddle, g.P, p->d_pairs,
                            p->d_Np, p->d_off, p->d_stab, g.L, p->max_Np, slri ? p->d_ftab : nullptr, Rp,
                            cols, scale, p->op, out, p->d_A_lo, s));
    SRP_MARK(p, 1, s);
    SRP_MARK(p, 2, s);
    if (slri && !tc) {
      SRP_LAUNCH(launch_slri_tall(p->d_U, p->d_tall, maps, p->d_keys, F, g.J, Rp, s));
    } else if (slri) {
      SRP_CUDA_TRY(contract(p, p->d_A, p->d_A_lo, p->d_B, p->d_B_lo, kSlriKd, nullptr, nullptr,
                            F, maps, s));
    } else if (method == SRP_SSPI && !tc) {
      SRP_LAUNCH(sspi_gather(p, maps, F, s));
    } else {
      SRP_CUDA_TRY(contract(p, p->d_A, p->d_A_lo, p->d_B, p->d_B_lo, p->Lpad, p->d_kb_ptr,
                            p->d_kb_idx, F, maps, s));
    }
    SRP_MARK(p, 3, s);
    if (argmax) SRP_LAUNCH(launch_argmax_finalize(p->d_keys, argmax, F, s));
    SRP_MARK(p, 4, s);
    if (p->profiling && p->chunks_recorded < kMaxChunkEvents) ++p->chunks_recorded;
    return SRP_OK;
  }
  if (p->use_front_conv) {
    // conv / LR operand straight from the frames (one fused launch)
    SRP_LAUNCH(launch_front_conv(frames, F, g.M, g.N, p->d_window, p->d_twiddle, g.P, p->d_pairs,
                                 p->op, p->d_A, p->d_A_lo, s));
    SRP_MARK(p, 1, s);
  } else {
    SRP_LAUNCH(launch_stft_phat(frames, F, g.M, g.N, p->d_window, p->d_twiddle, p->d_yhat, s));
    SRP_MARK(p, 1, s);
    if (method == SRP_CONV || method == SRP_LR)
      SRP_LAUNCH(launch_conv_pack(p->d_yhat, F, g.M, g.P, g.N, p->d_pairs, p->op, p->d_A,
                                  p->d_A_lo, s));
  }
  switch (method) {
    case SRP_CONV: {
      SRP_MARK(p, 2, s);
      if (p->h_chunk > 0) {
        // chunks of cells: generate their SRP-matrix rows, then their block of map columns
        for (int c0 = 0; c0 < g.J; c0 += p->h_chunk) {
          const int jn = std::min(p->h_chunk, g.J - c0);
          const size_t o = static_cast<size_t>(c0) * g.P;
          SRP_LAUNCH(launch_conv_matrix_split(p->d_tau_hi + o, p->d_tau_lo + o, jn, g.P, g.N,
                                              p->op, p->d_H, p->d_H_lo, s));
          SRP_CUDA_TRY(contract_cols(p, p->d_A, p->d_A_lo, p->d_H, p->d_H_lo, g.P * g.N, F,
                                     maps ? maps + c0 : nullptr, c0, jn, s));
        }
      } else if (p->h_generated) {
        p->launches += sgemm_split_count(g.P * g.N) > 1 ? 2 : 1;
        SRP_CUDA_TRY(launch_sgemm_nt_argmax(static_cast<const float*>(p->d_A), nullptr, maps,
                                            p->d_keys, F, g.J, g.P * g.N, p->d_split, s,
                                            p->d_tau_hi, p->d_tau_lo, g.P, g.N));
      } else {
        SRP_CUDA_TRY(contract(p, p->d_A, p->d_A_lo, p->d_H, p->d_H_lo, g.P * g.N, nullptr, nullptr,
                              F, maps, s));
      }
      break;
    }
    case SRP_LR: {
      // u = H_fat psi as a real product over the conv operand (rows u_re, u_im), then
      // z = 2 Re[H_tall u] = [2 Re H_tall | -2 Im H_tall] [u_re; u_im] (boxed Eq. z_lr)
      SRP_MARK(p, 2, s);
      SRP_CUDA_TRY(contract_to(p, p->d_A, p->d_A_lo, p->d_H, p->d_H_lo, g.P * g.N, nullptr, nullptr,
                               F, p->d_U, 2 * p->R, p->d_keys2, s));
      SRP_LAUNCH(launch_pack16(p->d_U, F, 2 * p->R, p->lr_kd, std::ldexp(1.f, p->slri_exp), p->op,
                               p->d_A2, p->d_A2_lo, s));
      SRP_CUDA_TRY(contract(p, p->d_A2, p->d_A2_lo, p->d_B, p->d_B_lo, p->lr_kd, nullptr, nullptr,
                            F, maps, s));
      break;
    }
    case SRP_SLRI: {
      if (p->fat_gemm) {
        SRP_CUDA_TRY(sample_to(p, p->d_yhat, F, p->d_A2, p->d_A2_lo, p->Lpad, p->op, s));
        SRP_MARK(p, 2, s);
        SRP_CUDA_TRY(contract_to(p, p->d_A2, p->d_A2_lo, p->d_H, p->d_H_lo, p->Lpad, nullptr,
                                 nullptr, F, p->d_U, Rp, p->d_keys2, s));
      } else {
        SRP_CUDA_TRY(sample_to(p, p->d_yhat, F, p->d_xi, nullptr, g.L, OpType::F32, s));
        SRP_MARK(p, 2, s);
        SRP_LAUNCH(launch_slri_fat(p->d_xi, p->d_fat, p->d_U, F, g.L, Rp, s));
      }
      if (p->op == OpType::F32) {
        SRP_LAUNCH(launch_slri_tall(p->d_U, p->d_tall, maps, p->d_keys, F, g.J, Rp, s));
      } else {
        SRP_LAUNCH(launch_pack16(p->d_U, F, Rp, kSlriKd, std::ldexp(1.f, -p->slri_exp), p->op,
                                   p->d_A, p->d_A_lo, s));
        SRP_CUDA_TRY(contract(p, p->d_A, p->d_A_lo, p->d_B, p->d_B_lo, kSlriKd, nullptr, nullptr,
                              F, maps, s));
      }
      break;
    }
    case SRP_SSPI:
    case SRP_SI:
    case SRP_TD: {
      if (method == SRP_SSPI && p->op == OpType::F32) {
        SRP_CUDA_TRY(sample_to(p, p->d_yhat, F, p->d_xi, nullptr, g.L, OpType::F32, s));
        SRP_MARK(p, 2, s);
        SRP_LAUNCH(sspi_gather(p, maps, F, s));
      } else {
        SRP_CUDA_TRY(sample_to(p, p->d_yhat, F, p->d_A, p->d_A_lo, p->Lpad, p->op, s));
        SRP_MARK(p, 2, s);
        SRP_CUDA_TRY(contract(p, p->d_A, p->d_A_lo, p->d_B, p->d_B_lo, p->Lpad, p->d_kb_ptr,
                              p->d_kb_idx, F, maps, s));
      }
      break;
    }
    default:
      return fail(SRP_EINVAL, "unknown method");
  }
  SRP_MARK(p, 3, s);
  if (argmax) SRP_LAUNCH(launch_argmax_finalize(p->d_keys, argmax, F, s));
  SRP_MARK(p, 4, s);
  if (p->profiling && p->chunks_recorded < kMaxChunkEvents) ++p->chunks_recorded;
  return SRP_OK;
}

}  // namespace
}  // namespace srp

using namespace srp;

// Plan creation; `fit` (from a saved plan) replaces the method's FP64 fit when given.
static srp_status create_plan(const srp_plan_desc* desc, void* stream, srp_plan_t* out,
                              const FitData* fit) {
  clear_error();
  if (!out) return fail(SRP_EINVAL, "out is NULL");
  *out = nullptr;
  srp_status st = validate(desc);
  if (st != SRP_OK) return st;
  const auto t0 = std::chrono::steady_clock::now();
  srp_plan_s* p = new srp_plan_s();
  p->desc = *desc;
  p->Fmax = desc->max_frames;
  st = build_geometry(*desc, p->g);
  if (st != SRP_OK) {
    delete p;
    return st;
  }
  const Geometry& g = p->g;
  p->h_grid4.resize(4 * static_cast<size_t>(g.J));
  for (int i = 0; i < g.J; ++i) {
    for (int a = 0; a < 3; ++a)
      p->h_grid4[4 * static_cast<size_t>(i) + a] = static_cast<float>(desc->grid_xyz[3 * static_cast<size_t>(i) + a]);
    p->h_grid4[4 * static_cast<size_t>(i) + 3] = 0.f;
  }
  // method-specific host-side checks (still no GPU needed)
  if (desc->method == SRP_SLRI) {
    if (desc->rank < 1 || desc->rank > 64 || desc->rank > std::min(g.J, g.L)) {
      delete p;
      return fail(SRP_EINVAL, "rank must be in 1..min(64, J, L) (L = " + std::to_string(g.L) + ")");
    }
    p->R = desc->rank;
  }
  if (desc->method == SRP_LR) {
    const int D = g.P * (g.K - 1);
    if (desc->rank < 1 || desc->rank > 64 || desc->rank > std::min(g.J, D)) {
      delete p;
      return fail(SRP_EINVAL, "rank must be in 1..min(64, J, P(K-1))");
    }
    p->R = desc->rank;
  }
  if (desc->method == SRP_SSPI) {
    const double t = desc->taps_per_loc_pair;
    const double nz = std::llround(t * static_cast<double>(g.J) * g.P);
    if (!(t > 0) || !(nz >= 1) || nz > static_cast<double>(g.J) * g.L) {
      delete p;
      return fail(SRP_EINVAL, "taps_per_loc_pair gives Q_Lambda outside 1..J*L");
    }
    p->nnz = static_cast<long long>(nz);
  }
  p->op = op_of(desc->precision);
  p->Lpad = (g.L + kSlriKd - 1) / kSlriKd * kSlriKd;
  p->max_Np = *std::max_element(g.Np.begin(), g.Np.end());
  p->use_front = desc->method != SRP_CONV && desc->method != SRP_LR &&
                 front_supported(g.M, g.N, g.L, p->max_Np);
  p->use_front_conv = (desc->method == SRP_CONV || desc->method == SRP_LR) &&
                      front_conv_supported(g.M, g.N);
  p->use_mma_sampling = desc->method != SRP_CONV && desc->method != SRP_LR && !p->use_front &&
                        gcc_mma_supported(g.M, g.N, p->max_Np);
  p->use_dft_sampling = desc->method != SRP_CONV && desc->method != SRP_LR && !p->use_front &&
                        !p->use_mma_sampling && gcc_dft_supported(g.M, g.N, p->op);
  if (desc->method == SRP_SI || desc->method == SRP_TD ||
      (desc->method == SRP_SSPI && p->op != OpType::F32)) {
    const double bbytes = static_cast<double>(g.J) * p->Lpad * op_bytes(p->op) *
                          (op_split(p->op) ? 2 : 1);
    if (bbytes > 200e9) {
      delete p;
      return fail(SRP_EUNSUPPORTED, "dense interpolation operand would need more than 200 GB");
    }
  }
  if (desc->method == SRP_CONV) {
    const double hbytes = static_cast<double>(g.J) * g.P * g.N * op_bytes(p->op) *
                          (op_split(p->op) ? 2 : 1);
    p->h_generated = desc->h_on_the_fly == 1 || (desc->h_on_the_fly == 0 && hbytes > kMaxStoredH);
    if (p->h_generated && p->op != OpType::F32) {
      // tensor cores: the rows of a chunk of cells are generated before each GEMM of the
      // chunk; the chunk gives about two waves of tiles with the largest batch (whole
      // 256-cell tiles, at most kMaxChunkH bytes)
      p->h_generated = false;
      const double per_cell = hbytes / g.J;
      int ncell_tiles = 1;
      {
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
          cudaGetLastError();
          sms = 152;
        }
        const int frame_tiles = (p->Fmax + 127) / 128;
        ncell_tiles = std::max(1, (2 * sms + frame_tiles - 1) / frame_tiles);
      }
      const int by_budget = std::max(1, static_cast<int>(kMaxChunkH / (per_cell * 256)));
      p->h_chunk = std::min(g.J, 256 * std::min(ncell_tiles, by_budget));
    }
  }

  // ---- device part
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SRP_PLAN_CUDA(p, cudaGetDevice(&p->device));
  if (p->op != OpType::F32) SRP_PLAN_CUDA(p, tc_gemm_prepare());
  SRP_PLAN_CUDA(p, cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
  std::vector<int2> pairs(g.P);
  for (int q = 0; q < g.P; ++q) pairs[q] = make_int2(g.pm[q], g.pmp[q]);
  std::vector<float2> tw(g.N / 2);
  for (int t = 0; t < g.N / 2; ++t)
    tw[t] = make_float2(static_cast<float>(std::cos(2.0 * M_PI * t / g.N)),
                        static_cast<float>(-std::sin(2.0 * M_PI * t / g.N)));
  std::vector<float> win;
  window_table(g.N, desc->window, win);
  SRP_ALLOC(p, p->d_pairs, sizeof(int2) * g.P);
  SRP_ALLOC(p, p->d_Np, sizeof(int) * g.P);
  SRP_ALLOC(p, p->d_off, sizeof(int) * g.P);
  SRP_ALLOC(p, p->d_twiddle, sizeof(float2) * g.N / 2);
  SRP_ALLOC(p, p->d_window, sizeof(float) * g.N);
  SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_pairs, pairs.data(), sizeof(int2) * g.P, cudaMemcpyHostToDevice, s));
  SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_Np, g.Np.data(), sizeof(int) * g.P, cudaMemcpyHostToDevice, s));
  SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_off, g.off.data(), sizeof(int) * g.P, cudaMemcpyHostToDevice, s));
  SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_twiddle, tw.data(), sizeof(float2) * g.N / 2, cudaMemcpyHostToDevice, s));
  SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_window, win.data(), sizeof(float) * g.N, cudaMemcpyHostToDevice, s));
  std::vector<uint4> stab;
  if (p->use_front || p->use_mma_sampling || p->use_dft_sampling) {
    if (p->use_dft_sampling)
      dft_tables(stab);
    else
      front_sampling_table(g.N, p->max_Np, stab);
    SRP_ALLOC(p, p->d_stab, sizeof(uint4) * stab.size());
    SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_stab, stab.data(), sizeof(uint4) * stab.size(),
                                     cudaMemcpyHostToDevice, s));
  }
  const size_t F = static_cast<size_t>(p->Fmax);
  SRP_ALLOC(p, p->d_yhat, sizeof(float2) * F * g.M * (g.N / 2));
  SRP_ALLOC(p, p->d_keys, sizeof(unsigned long long) * F);
  SRP_ALLOC(p, p->d_err, sizeof(int));
  SRP_PLAN_CUDA(p, cudaMemsetAsync(p->d_err, 0, sizeof(int), s));

  if (desc->method == SRP_CONV && p->h_generated) {
    // the SRP matrix is generated inside the GEMM from the TDOAs split as tau_hi + tau_lo,
    // tau_hi with 13 significant bits (so k tau_hi is exact in FP32 for k < 2^11)
    const size_t Kd = static_cast<size_t>(g.P) * g.N;
    std::vector<float> th(g.tau.size()), tl(g.tau.size());
    for (size_t e = 0; e < g.tau.size(); ++e) {
      const double t = g.tau[e];
      int ex = 0;
      const double m = std::frexp(t, &ex);                     // t = m 2^ex, 0.5 <= |m| < 1
      const double hi = std::ldexp(std::trunc(std::ldexp(m, 13)), ex - 13);
      th[e] = static_cast<float>(hi);
      tl[e] = static_cast<float>(t - hi);
    }
    SRP_ALLOC(p, p->d_tau_hi, sizeof(float) * th.size());
    SRP_ALLOC(p, p->d_tau_lo, sizeof(float) * tl.size());
    SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_tau_hi, th.data(), sizeof(float) * th.size(), cudaMemcpyHostToDevice, s));
    SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_tau_lo, tl.data(), sizeof(float) * tl.size(), cudaMemcpyHostToDevice, s));
    SRP_ALLOC(p, p->d_A, F * Kd * sizeof(float));
    const int nsplit = sgemm_split_count(static_cast<int>(Kd));
    if (nsplit > 1) SRP_ALLOC(p, p->d_split, sizeof(float) * nsplit * F * g.J);
    SRP_PLAN_CUDA(p, cudaStreamSynchronize(s));
  } else if (desc->method == SRP_CONV && p->h_chunk > 0) {
    // tensor cores, SRP matrix generated per chunk of cells before each chunk's GEMM: the
    // FP64 TDOA table stays on the device, d_H holds one chunk's rows
    const size_t Kd = static_cast<size_t>(g.P) * g.N;
    const size_t eb = op_bytes(p->op);
    const bool split = op_split(p->op);
    SRP_ALLOC(p, p->d_H, static_cast<size_t>(p->h_chunk) * Kd * eb);
    if (split) SRP_ALLOC(p, p->d_H_lo, static_cast<size_t>(p->h_chunk) * Kd * eb);
    SRP_ALLOC(p, p->d_A, F * Kd * eb);
    if (split) SRP_ALLOC(p, p->d_A_lo, F * Kd * eb);
    // the TDOAs split as tau_hi (13 significant bits) + tau_lo for the FP32 generation
    std::vector<float> th(g.tau.size()), tl(g.tau.size());
    for (size_t e = 0; e < g.tau.size(); ++e) {
      const double t = g.tau[e];
      int ex = 0;
      const double m = std::frexp(t, &ex);
      const double hi = std::ldexp(std::trunc(std::ldexp(m, 13)), ex - 13);
      th[e] = static_cast<float>(hi);
      tl[e] = static_cast<float>(t - hi);
    }
    SRP_ALLOC(p, p->d_tau_hi, sizeof(float) * th.size());
    SRP_ALLOC(p, p->d_tau_lo, sizeof(float) * tl.size());
    SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_tau_hi, th.data(), sizeof(float) * th.size(), cudaMemcpyHostToDevice, s));
    SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_tau_lo, tl.data(), sizeof(float) * tl.size(), cudaMemcpyHostToDevice, s));
    // a chunk's reduction (P N columns: about 1e6 on the 32-microphone grid) in slices of
    // about kChunkSliceSteps k-steps: the CTAs sharing a cell tile's rows of H then walk
    // short, equal reductions and stay together, so those rows come from L2 once instead of
    // from DRAM for every frame tile; the partial maps are summed in FP64
    const int ksteps = static_cast<int>(Kd / 64) * op_kb_per64(p->op);
    p->h_slices = std::max(1, std::min(kChunkMaxSlices, ksteps / kChunkSliceSteps));
    if (p->h_slices > 1)
      SRP_ALLOC(p, p->d_split, sizeof(float) * static_cast<size_t>(p->h_slices) * F * p->h_chunk);
    SRP_PLAN_CUDA(p, cudaStreamSynchronize(s));
  } else if (desc->method == SRP_CONV) {
    const size_t Kd = static_cast<size_t>(g.P) * g.N;
    const size_t eb = op_bytes(p->op);
    const bool split = op_split(p->op);
    SRP_ALLOC(p, p->d_H, static_cast<size_t>(g.J) * Kd * eb);
    if (split) SRP_ALLOC(p, p->d_H_lo, static_cast<size_t>(g.J) * Kd * eb);
    SRP_ALLOC(p, p->d_A, F * Kd * eb);
    if (split) SRP_ALLOC(p, p->d_A_lo, F * Kd * eb);
    size_t ws_floats = 0;
    if (p->op == OpType::F32) {
      const int nsplit = sgemm_split_count(static_cast<int>(Kd));
      if (nsplit > 1) ws_floats = static_cast<size_t>(nsplit) * F * g.J;
    } else {
      ws_floats = tc_gemm_workspace_floats(p->Fmax, g.J, static_cast<int>(Kd), p->op, p->num_sms);
    }
    if (ws_floats > 0) SRP_ALLOC(p, p->d_split, sizeof(float) * ws_floats);
    double* d_tau = nullptr;
    if (device_alloc(reinterpret_cast<void**>(&d_tau), sizeof(double) * g.tau.size()) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc for the TDOA table failed");
      free_plan(p);
      return SRP_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(d_tau, g.tau.data(), sizeof(double) * g.tau.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_conv_matrix(d_tau, g.J, g.P, g.N, p->op, p->d_H, p->d_H_lo, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_tau);
    if (e != cudaSuccess) {
      set_error(std::string("SRP matrix generation: ") + cudaGetErrorString(e));
      free_plan(p);
      return SRP_ECUDA;
    }
  } else if (desc->method == SRP_LR) {
    // LR-SRP (Sec. III-A): rank-R fit of H, then the real-ified factors
    //   fat  B1 [2R][P N]: row r     = [Re Hf_r at k, -Im Hf_r at K + k] per pair (u_re)
    //                      row R + r = [Im Hf_r at k,  Re Hf_r at K + k] per pair (u_im)
    //   tall B2 [J][lr_kd]: [2 Re Ht | -2 Im Ht] * 2^-e, zero padded to lr_kd columns
    const int R = p->R, D = g.P * (g.K - 1);
    const size_t Kd = static_cast<size_t>(g.P) * g.N;
    const size_t eb = op_bytes(p->op);
    const bool split = op_split(p->op);
    std::vector<std::complex<double>> ht, hf;
    srp_status fst = SRP_OK;
    if (fit) {
      ht = fit->ht;
      hf = fit->hf;
      p->sigma = fit->sigma;
    } else {
      fst = fit_lr_device(g, R, ht, hf, p->sigma, s);
    }
    if (fst != SRP_OK) {
      free_plan(p);
      return fst;
    }
    p->lr_kd = (2 * R + kSlriKd - 1) / kSlriKd * kSlriKd;
    if (p->op != OpType::F32) {
      // |u| <= ||psi||_2 <= sqrt(D) (rows of H_fat are orthonormal, |psi| <= 1); the tall
      // entries are at most 2 sigma_1: scale them by 2^-e into the FP16 range
      p->slri_exp = std::max(0, static_cast<int>(std::ceil(std::log2(2.0 * p->sigma[0] / 16384.0))));
      const bool fp16 = p->op == OpType::F16 || p->op == OpType::F16X2;
      if (fp16 && std::sqrt(static_cast<double>(D)) * std::ldexp(1.0, p->slri_exp) > 16384.0) {
        free_plan(p);
        return fail(SRP_EUNSUPPORTED, "LR-SRP operands exceed the FP16 range (use SRP_FP32)");
      }
    }
    std::vector<float> b1(static_cast<size_t>(2 * R) * Kd, 0.f), b2(static_cast<size_t>(g.J) * 2 * R);
    for (int r = 0; r < R; ++r)
      for (int q = 0; q < g.P; ++q)
        for (int k = 1; k < g.K; ++k) {
          const std::complex<double> v = hf[static_cast<size_t>(r) * D + q * (g.K - 1) + (k - 1)];
          const size_t c = static_cast<size_t>(q) * g.N + k;
          b1[r * Kd + c] = static_cast<float>(v.real());
          b1[r * Kd + c + g.K] = static_cast<float>(-v.imag());
          b1[(R + r) * Kd + c] = static_cast<float>(v.imag());
          b1[(R + r) * Kd + c + g.K] = static_cast<float>(v.real());
        }
    const double sc = std::ldexp(1.0, -p->slri_exp);
    for (int i = 0; i < g.J; ++i)
      for (int r = 0; r < R; ++r) {
        const std::complex<double> v = ht[static_cast<size_t>(i) * R + r];
        b2[static_cast<size_t>(i) * 2 * R + r] = static_cast<float>(2.0 * v.real() * sc);
        b2[static_cast<size_t>(i) * 2 * R + R + r] = static_cast<float>(-2.0 * v.imag() * sc);
      }
    float* d_tmp = nullptr;
    const size_t tmp_n = std::max(b1.size(), b2.size());
    if (device_alloc(reinterpret_cast<void**>(&d_tmp), sizeof(float) * tmp_n) != cudaSuccess) {
      cudaGetLastError();
      free_plan(p);
      return fail(SRP_ENOMEM, "LR factor staging");
    }
    SRP_ALLOC(p, p->d_H, static_cast<size_t>(2 * R) * Kd * eb);
    if (split) SRP_ALLOC(p, p->d_H_lo, static_cast<size_t>(2 * R) * Kd * eb);
    SRP_ALLOC(p, p->d_B, static_cast<size_t>(g.J) * p->lr_kd * eb);
    if (split) SRP_ALLOC(p, p->d_B_lo, static_cast<size_t>(g.J) * p->lr_kd * eb);
    cudaError_t e = cudaMemcpyAsync(d_tmp, b1.data(), sizeof(float) * b1.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = launch_pack16(d_tmp, 2 * R, static_cast<int>(Kd), static_cast<int>(Kd), 1.f, p->op, p->d_H, p->d_H_lo, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_tmp, b2.data(), sizeof(float) * b2.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = launch_pack16(d_tmp, g.J, 2 * R, p->lr_kd, 1.f, p->op, p->d_B, p->d_B_lo, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_tmp);
    if (e != cudaSuccess) {
      set_error(std::string("LR factors: ") + cudaGetErrorString(e));
      free_plan(p);
      return SRP_ECUDA;
    }
    p->lr_tall = std::move(ht);  // kept for srp_plan_save
    p->lr_fat = std::move(hf);
    SRP_ALLOC(p, p->d_A, F * Kd * eb);
    if (split) SRP_ALLOC(p, p->d_A_lo, F * Kd * eb);
    SRP_ALLOC(p, p->d_U, sizeof(float) * F * 2 * R);
    SRP_ALLOC(p, p->d_A2, F * p->lr_kd * eb);
    if (split) SRP_ALLOC(p, p->d_A2_lo, F * p->lr_kd * eb);
    SRP_ALLOC(p, p->d_keys2, sizeof(unsigned long long) * F);
    size_t ws = 0;
    if (p->op == OpType::F32) {
      const int nsplit = sgemm_split_count(static_cast<int>(Kd));
      if (nsplit > 1) ws = static_cast<size_t>(nsplit) * F * 2 * R;
    } else {
      ws = std::max(tc_gemm_workspace_floats(p->Fmax, 2 * R, static_cast<int>(Kd), p->op, p->num_sms),
                    tc_gemm_workspace_floats(p->Fmax, g.J, p->lr_kd, p->op, p->num_sms));
    }
    if (ws > 0) SRP_ALLOC(p, p->d_split, sizeof(float) * ws);
  } else {
    SRP_ALLOC(p, p->d_xi, sizeof(float) * F * g.L);
    const size_t eb = op_bytes(p->op);
    const bool split = op_split(p->op);
    if (desc->method == SRP_SLRI) {
      std::vector<float> tall, fat;
      // exact Gram eigen-decomposition for short sample vectors, device subspace
      // iteration beyond (the L x L Jacobi solve grows as L^3)
      srp_status fst = SRP_OK;
      if (fit) {
        tall = fit->tall;
        fat = fit->fat;
        p->sigma = fit->sigma;
      } else {
        fst = g.L <= kGramMaxL ? fit_low_rank(g, p->R, tall, fat, p->sigma)
                               : fit_low_rank_device(g, p->R, tall, fat, p->sigma, s);
      }
      if (fst != SRP_OK) {
        free_plan(p);
        return fst;
      }
      const int Rp = (p->R + 7) / 8 * 8;
      SRP_ALLOC(p, p->d_tall, sizeof(float) * tall.size());
      SRP_ALLOC(p, p->d_fat, sizeof(float) * fat.size());
      SRP_ALLOC(p, p->d_U, sizeof(float) * F * Rp);
      SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_tall, tall.data(), sizeof(float) * tall.size(), cudaMemcpyHostToDevice, s));
      SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_fat, fat.data(), sizeof(float) * fat.size(), cudaMemcpyHostToDevice, s));
      std::vector<uint4> ftab;
      if (p->use_front) {
        front_fat_table(fat.data(), Rp, g.L, ftab);
        SRP_ALLOC(p, p->d_ftab, sizeof(uint4) * ftab.size());
        SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_ftab, ftab.data(), sizeof(uint4) * ftab.size(),
                                         cudaMemcpyHostToDevice, s));
      }
      if (p->op != OpType::F32) {
        // u = Lambda_fat xi has |u_r| <= ||xi||_2 <= 2K sqrt(P) (Parseval over the 2K lags of
        // each pair, |psi| <= 1): scale u by 2^-e into the FP16 range and Lambda_tall by 2^e.
        const double ubound = 2.0 * g.K * std::sqrt(static_cast<double>(g.P));
        p->slri_exp = std::max(0, static_cast<int>(std::ceil(std::log2(ubound / 16384.0))));
        SRP_ALLOC(p, p->d_B, static_cast<size_t>(g.J) * kSlriKd * eb);
        if (split) SRP_ALLOC(p, p->d_B_lo, static_cast<size_t>(g.J) * kSlriKd * eb);
        SRP_ALLOC(p, p->d_A, F * kSlriKd * eb);
        if (split) SRP_ALLOC(p, p->d_A_lo, F * kSlriKd * eb);
        SRP_PLAN_CUDA(p, launch_pack16(p->d_tall, g.J, Rp, kSlriKd, std::ldexp(1.f, p->slri_exp),
                                       p->op, p->d_B, p->d_B_lo, s));
      }
      size_t ws = p->op == OpType::F32
                      ? 0
                      : tc_gemm_workspace_floats(p->Fmax, g.J, kSlriKd, p->op, p->num_sms);
      if (!p->use_front && g.L > kFatGemmMinL) {
        // long sample vectors: u = Lambda_fat xi as a GEMM (xi operand [F][Lpad], factor
        // [Rp][Lpad]) instead of the per-frame dot products
        p->fat_gemm = true;
        SRP_ALLOC(p, p->d_H, static_cast<size_t>(Rp) * p->Lpad * eb);
        if (split) SRP_ALLOC(p, p->d_H_lo, static_cast<size_t>(Rp) * p->Lpad * eb);
        SRP_ALLOC(p, p->d_A2, F * p->Lpad * eb);
        if (split) SRP_ALLOC(p, p->d_A2_lo, F * p->Lpad * eb);
        SRP_ALLOC(p, p->d_keys2, sizeof(unsigned long long) * F);
        SRP_PLAN_CUDA(p, launch_pack16(p->d_fat, Rp, g.L, p->Lpad, 1.f, p->op, p->d_H, p->d_H_lo, s));
        if (p->op == OpType::F32) {
          const int nsplit = sgemm_split_count(p->Lpad);
          if (nsplit > 1) ws = std::max(ws, static_cast<size_t>(nsplit) * F * Rp);
        } else {
          ws = std::max(ws, tc_gemm_workspace_floats(p->Fmax, Rp, p->Lpad, p->op, p->num_sms));
        }
      }
      if (ws > 0) SRP_ALLOC(p, p->d_split, sizeof(float) * ws);
      SRP_PLAN_CUDA(p, cudaStreamSynchronize(s));
    } else {
      const int Lpad = p->Lpad;
      const int tile = tc_gemm_cell_tile();
      const int ntiles = (g.J + tile - 1) / tile;
      // block-sparse B: per cell tile, the first columns of disjoint 64-column windows that
      // cover every column a cell of the tile uses.  Windows start at multiples of 8 (the
      // TMA x-coordinate rule for 16-bit operands) and are laid greedily: each starts at the
      // first uncovered used column rounded down to 8, which never reaches back into the
      // previous window since that ends on a multiple of 8.  Columns beyond Lpad read zeros.
      std::vector<int> kb_ptr, kb_idx;
      auto add_lists = [&](const std::function<void(int, std::vector<char>&)>& mark_cells) {
        kb_ptr.assign(1, 0);
        std::vector<char> used(Lpad);
        for (int n = 0; n < ntiles; ++n) {
          std::fill(used.begin(), used.end(), 0);
          for (int i = n * tile; i < std::min(g.J, (n + 1) * tile); ++i) mark_cells(i, used);
          for (int c = 0; c < Lpad;) {
            if (!used[c]) {
              ++c;
              continue;
            }
            const int start = c & ~7;
            kb_idx.push_back(start);
            c = start + kSlriKd;
          }
          kb_ptr.push_back(static_cast<int>(kb_idx.size()));
        }
      };
      if (desc->method == SRP_SSPI) {
        srp_status fst = SRP_OK;
        if (fit) {
          p->nnz = fit->nnz;
          p->tied = fit->tied;
          p->h_row_ptr = fit->row_ptr;
          p->h_col = fit->col;
          p->h_val = fit->val;
        } else {
          fst = fit_sparse(g, p->nnz, p->h_row_ptr, p->h_col, p->h_val, p->tied);
        }
        if (fst != SRP_OK) {
          free_plan(p);
          return fst;
        }
        std::vector<int2> taps(static_cast<size_t>(p->nnz));
        for (long long t = 0; t < p->nnz; ++t) {
          int vb;
          std::memcpy(&vb, &p->h_val[t], 4);
          taps[t] = make_int2(p->h_col[t], vb);
        }
        if (p->op == OpType::F32 && !sspi_full_fits(g.L)) {
          // long sample vectors: per 64-cell block, the sorted columns its taps use; the
          // taps then index that list (the host keeps the global columns for export)
          const int nrb = (g.J + 63) / 64;
          std::vector<long long> bptr(nrb + 1, 0);
          std::vector<int> bcols, mark(g.L, -1), loc(g.L, 0);
          int umax = 0;
          for (int b = 0; b < nrb; ++b) {
            const int i0 = b * 64, i1 = std::min(g.J, i0 + 64);
            std::vector<int> cols;
            for (long long t = p->h_row_ptr[i0]; t < p->h_row_ptr[i1]; ++t) {
              const int c = p->h_col[t];
              if (mark[c] != b) {
                mark[c] = b;
                cols.push_back(c);
              }
            }
            std::sort(cols.begin(), cols.end());
            for (size_t u = 0; u < cols.size(); ++u) loc[cols[u]] = static_cast<int>(u);
            for (long long t = p->h_row_ptr[i0]; t < p->h_row_ptr[i1]; ++t) taps[t].x = loc[p->h_col[t]];
            bcols.insert(bcols.end(), cols.begin(), cols.end());
            bptr[b + 1] = static_cast<long long>(bcols.size());
            umax = std::max(umax, static_cast<int>(cols.size()));
          }
          int fb = 32;
          while (fb > 1 && sspi_band_smem(umax, fb) > 220 * 1024) fb >>= 1;
          if (sspi_band_smem(umax, fb) > 220 * 1024) {
            free_plan(p);
            return fail(SRP_EUNSUPPORTED, "the FP32 SSPI gather needs the taps of 64 cells to span at most " +
                                              std::to_string((220 * 1024 / 4 - 65) / 2) +
                                              " columns (" + std::to_string(umax) +
                                              " here; use a tensor-core precision)");
          }
          p->sspi_umax = umax;
          p->sspi_fb = fb;
          SRP_ALLOC(p, p->d_blk_ptr, sizeof(long long) * bptr.size());
          SRP_ALLOC(p, p->d_blk_cols, sizeof(int) * std::max<size_t>(1, bcols.size()));
          SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_blk_ptr, bptr.data(), sizeof(long long) * bptr.size(), cudaMemcpyHostToDevice, s));
          if (!bcols.empty())
            SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_blk_cols, bcols.data(), sizeof(int) * bcols.size(), cudaMemcpyHostToDevice, s));
          SRP_PLAN_CUDA(p, cudaStreamSynchronize(s));  // the host vectors go out of scope
        }
        SRP_ALLOC(p, p->d_row_ptr, sizeof(long long) * (g.J + 1));
        SRP_ALLOC(p, p->d_taps, sizeof(int2) * taps.size());
        SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_row_ptr, p->h_row_ptr.data(), sizeof(long long) * (g.J + 1), cudaMemcpyHostToDevice, s));
        SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_taps, taps.data(), sizeof(int2) * taps.size(), cudaMemcpyHostToDevice, s));
        if (p->op != OpType::F32) {
          SRP_ALLOC(p, p->d_B, static_cast<size_t>(g.J) * Lpad * eb);
          if (split) SRP_ALLOC(p, p->d_B_lo, static_cast<size_t>(g.J) * Lpad * eb);
          SRP_PLAN_CUDA(p, launch_csr_to_dense(p->d_row_ptr, p->d_taps, g.J, Lpad, p->op, p->d_B,
                                               p->d_B_lo, s));
          add_lists([&](int i, std::vector<char>& used) {
            for (long long t = p->h_row_ptr[i]; t < p->h_row_ptr[i + 1]; ++t)
              used[p->h_col[t]] = 1;
          });
          SRP_PLAN_CUDA(p, cudaStreamSynchronize(s));
          cudaFree(p->d_row_ptr);  // the dense operand replaces the tap list on the device
          cudaFree(p->d_taps);
          p->device_bytes -= sizeof(long long) * (g.J + 1) + sizeof(int2) * taps.size();
          p->d_row_ptr = nullptr;
          p->d_taps = nullptr;
        }
      } else {
        // SI-SRP (Eq. Lambda) or conv. TD-SRP (Eq. TD_SRP): dense operand from the TDOAs.
        std::vector<int> col_pair(g.L), col_lag(g.L);
        for (int q = 0; q < g.P; ++q)
          for (int n = -g.Np[q]; n <= g.Np[q]; ++n) {
            col_pair[g.off[q] + n + g.Np[q]] = q;
            col_lag[g.off[q] + n + g.Np[q]] = n;
          }
        SRP_ALLOC(p, p->d_B, static_cast<size_t>(g.J) * Lpad * eb);
        if (split) SRP_ALLOC(p, p->d_B_lo, static_cast<size_t>(g.J) * Lpad * eb);
        double* d_tau = nullptr;
        int* d_cols = nullptr;
        cudaError_t e = device_alloc(reinterpret_cast<void**>(&d_tau), sizeof(double) * g.tau.size());
        if (e == cudaSuccess) e = device_alloc(reinterpret_cast<void**>(&d_cols), sizeof(int) * 2 * g.L);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d_tau, g.tau.data(), sizeof(double) * g.tau.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d_cols, col_pair.data(), sizeof(int) * g.L, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(d_cols + g.L, col_lag.data(), sizeof(int) * g.L, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
          e = launch_interp_dense(d_tau, g.J, g.P, d_cols, d_cols + g.L, g.L, Lpad,
                                  desc->method == SRP_TD, p->op, p->d_B, p->d_B_lo, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (d_tau) cudaFree(d_tau);
        if (d_cols) cudaFree(d_cols);
        if (e != cudaSuccess) {
          cudaGetLastError();
          set_error(std::string("interpolation operand: ") + cudaGetErrorString(e));
          free_plan(p);
          return e == cudaErrorMemoryAllocation ? SRP_ENOMEM : SRP_ECUDA;
        }
        if (desc->method == SRP_TD && p->op != OpType::F32) {
          add_lists([&](int i, std::vector<char>& used) {
            for (int q = 0; q < g.P; ++q) {
              const double t = g.tau[static_cast<size_t>(i) * g.P + q];
              const double r = t < 0.0 ? -std::floor(-t + 0.5) : std::floor(t + 0.5);
              used[g.off[q] + static_cast<int>(r) + g.Np[q]] = 1;
            }
          });
        }
      }
      if (!kb_ptr.empty()) {
        SRP_ALLOC(p, p->d_kb_ptr, sizeof(int) * kb_ptr.size());
        SRP_ALLOC(p, p->d_kb_idx, sizeof(int) * std::max<size_t>(1, kb_idx.size()));
        SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_kb_ptr, kb_ptr.data(), sizeof(int) * kb_ptr.size(), cudaMemcpyHostToDevice, s));
        if (!kb_idx.empty())
          SRP_PLAN_CUDA(p, cudaMemcpyAsync(p->d_kb_idx, kb_idx.data(), sizeof(int) * kb_idx.size(), cudaMemcpyHostToDevice, s));
      }
      if (desc->method != SRP_SSPI || p->op != OpType::F32) {
        SRP_ALLOC(p, p->d_A, F * Lpad * eb);
        if (split) SRP_ALLOC(p, p->d_A_lo, F * Lpad * eb);
        size_t ws = 0;
        if (p->op == OpType::F32) {
          const int nsplit = sgemm_split_count(Lpad);
          if (nsplit > 1) ws = static_cast<size_t>(nsplit) * F * g.J;
        } else if (kb_ptr.empty()) {
          ws = tc_gemm_workspace_floats(p->Fmax, g.J, Lpad, p->op, p->num_sms);
        }
        if (ws > 0) SRP_ALLOC(p, p->d_split, sizeof(float) * ws);
      }
      SRP_PLAN_CUDA(p, cudaStreamSynchronize(s));
    }
  }
  SRP_PLAN_CUDA(p, cudaStreamSynchronize(s));
  p->g.tau.clear();
  p->g.tau.shrink_to_fit();
  p->fit_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = p;
  return SRP_OK;
}

extern "C" srp_status srp_plan_create(const srp_plan_desc* desc, void* stream, srp_plan_t* out) {
  return create_plan(desc, stream, out, nullptr);
}

// ------------------------------------------------------------------ plan files
// Little-endian binary: magic, version, method, the hash of the inputs the fit depends on,
// sizes, the fit (SLRI: sigma, Lambda_tall [J][Rp], Lambda_fat [Rp][L] in FP32; SSPI: the
// CSR taps; LR-SRP: sigma and the complex FP64 factors), and an FNV-1a checksum of the
// preceding bytes.
namespace {
constexpr char kPlanMagic[8] = {'S', 'R', 'P', 'P', 'L', 'A', 'N', '\0'};
constexpr uint32_t kPlanVersion = 1;

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* d, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(d);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
  template <typename T>
  void val(const T& v) { add(&v, sizeof(T)); }
};

// hash of everything the method's fit depends on (not the precision, window or batch size)
uint64_t fit_inputs_hash(const srp_plan_desc& d) {
  Fnv f;
  f.val(d.M);
  f.add(d.mic_xyz, sizeof(double) * 3 * d.M);
  f.val(d.J);
  f.add(d.grid_xyz, sizeof(double) * 3 * static_cast<size_t>(d.J));
  f.val(d.fs);
  f.val(d.N);
  f.val(d.c);
  f.val(d.n_aux);
  f.val(static_cast<int>(d.method));
  f.val(d.method == SRP_SLRI || d.method == SRP_LR ? d.rank : 0);
  f.val(d.method == SRP_SSPI ? d.taps_per_loc_pair : 0.0);
  f.val(d.far_field);
  return f.h;
}

struct Writer {
  std::FILE* fp;
  Fnv sum;
  bool ok = true;
  void add(const void* d, size_t n) {
    if (n == 0) return;
    ok = ok && std::fwrite(d, 1, n, fp) == n;
    sum.add(d, n);
  }
  template <typename T>
  void val(const T& v) { add(&v, sizeof(T)); }
  template <typename T>
  void vec(const std::vector<T>& v) {
    const uint64_t n = v.size();
    val(n);
    add(v.data(), sizeof(T) * v.size());
  }
};

struct Reader {
  std::vector<unsigned char> buf;
  size_t pos = 0;
  bool ok = true;
  void get(void* d, size_t n) {
    if (!ok || buf.size() - pos < n) {
      ok = false;
      return;
    }
    std::memcpy(d, buf.data() + pos, n);
    pos += n;
  }
  template <typename T>
  T val() {
    T v{};
    get(&v, sizeof(T));
    return v;
  }
  template <typename T>
  void vec(std::vector<T>& v, uint64_t expect) {
    const uint64_t n = val<uint64_t>();
    if (!ok || n != expect || n > (buf.size() - pos) / sizeof(T)) {
      ok = false;
      return;
    }
    v.resize(n);
    get(v.data(), sizeof(T) * n);
  }
};
}  // namespace

extern "C" srp_status srp_plan_save(srp_plan_t plan, const char* path) {
  clear_error();
  if (!plan || !path) return fail(SRP_EINVAL, "plan or path is NULL");
  const Geometry& g = plan->g;
  const int method = plan->desc.method;
  FitData fit;
  if (method == SRP_SLRI) {
    const int Rp = (plan->R + 7) / 8 * 8;
    fit.tall.resize(static_cast<size_t>(g.J) * Rp);
    fit.fat.resize(static_cast<size_t>(Rp) * g.L);
    SRP_CUDA_TRY(cudaMemcpy(fit.tall.data(), plan->d_tall, sizeof(float) * fit.tall.size(),
                            cudaMemcpyDeviceToHost));
    SRP_CUDA_TRY(cudaMemcpy(fit.fat.data(), plan->d_fat, sizeof(float) * fit.fat.size(),
                            cudaMemcpyDeviceToHost));
  }
  std::FILE* fp = std::fopen(path, "wb");
  if (!fp) return fail(SRP_EINVAL, std::string("cannot open ") + path + " for writing");
  Writer w{fp};
  w.add(kPlanMagic, sizeof(kPlanMagic));
  w.val(kPlanVersion);
  w.val(static_cast<int32_t>(method));
  w.val(fit_inputs_hash(plan->desc));
  w.val(static_cast<int32_t>(g.J));
  w.val(static_cast<int32_t>(g.P));
  w.val(static_cast<int32_t>(g.L));
  w.val(static_cast<int32_t>(plan->R));
  if (method == SRP_SLRI || method == SRP_LR) w.vec(plan->sigma);
  if (method == SRP_SLRI) {
    w.vec(fit.tall);
    w.vec(fit.fat);
  } else if (method == SRP_SSPI) {
    w.val(static_cast<int64_t>(plan->nnz));
    w.val(static_cast<int64_t>(plan->tied));
    w.vec(plan->h_row_ptr);
    w.vec(plan->h_col);
    w.vec(plan->h_val);
  } else if (method == SRP_LR) {
    w.vec(plan->lr_tall);
    w.vec(plan->lr_fat);
  }
  const uint64_t sum = w.sum.h;
  w.val(sum);
  const bool ok = w.ok && std::fclose(fp) == 0;
  if (!ok) return fail(SRP_EINVAL, std::string("writing ") + path + " failed");
  return SRP_OK;
}

extern "C" srp_status srp_plan_create_from_file(const srp_plan_desc* desc, const char* path,
                                                void* stream, srp_plan_t* out) {
  clear_error();
  if (!out) return fail(SRP_EINVAL, "out is NULL");
  *out = nullptr;
  srp_status st = validate(desc);
  if (st != SRP_OK) return st;
  if (!path) return fail(SRP_EINVAL, "path is NULL");
  Reader r;
  {
    std::FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(SRP_EINVAL, std::string("cannot open ") + path);
    unsigned char chunk[1 << 16];
    size_t n;
    while ((n = std::fread(chunk, 1, sizeof(chunk), fp)) > 0) r.buf.insert(r.buf.end(), chunk, chunk + n);
    std::fclose(fp);
  }
  if (r.buf.size() < sizeof(kPlanMagic) + 8 || std::memcmp(r.buf.data(), kPlanMagic, sizeof(kPlanMagic)) != 0)
    return fail(SRP_EINVAL, std::string(path) + " is not a libsrp plan file");
  {
    Fnv f;
    f.add(r.buf.data(), r.buf.size() - 8);
    uint64_t stored;
    std::memcpy(&stored, r.buf.data() + r.buf.size() - 8, 8);
    if (stored != f.h) return fail(SRP_EINVAL, std::string(path) + ": checksum mismatch (damaged file)");
    r.buf.resize(r.buf.size() - 8);
  }
  r.pos = sizeof(kPlanMagic);
  if (r.val<uint32_t>() != kPlanVersion) return fail(SRP_EINVAL, "unsupported plan file version");
  const int method = r.val<int32_t>();
  if (method != desc->method) return fail(SRP_EINVAL, "the plan file holds another method");
  if (r.val<uint64_t>() != fit_inputs_hash(*desc))
    return fail(SRP_EINVAL, "the plan file was made for other inputs (geometry, fs, N, c, "
                            "n_aux, rank, taps or far field differ)");
  Geometry g;
  st = build_geometry(*desc, g);
  if (st != SRP_OK) return st;
  const int J = r.val<int32_t>(), P = r.val<int32_t>(), L = r.val<int32_t>(), R = r.val<int32_t>();
  if (!r.ok || J != g.J || P != g.P || L != g.L) return fail(SRP_EINVAL, "plan file sizes do not match");
  FitData fit;
  const int Rp = (R + 7) / 8 * 8;
  if (method == SRP_SLRI || method == SRP_LR) {
    const uint64_t ns = r.val<uint64_t>();
    r.pos -= sizeof(uint64_t);
    r.vec(fit.sigma, ns);
  }
  if (method == SRP_SLRI) {
    r.vec(fit.tall, static_cast<uint64_t>(J) * Rp);
    r.vec(fit.fat, static_cast<uint64_t>(Rp) * L);
  } else if (method == SRP_SSPI) {
    fit.nnz = r.val<int64_t>();
    fit.tied = r.val<int64_t>();
    r.vec(fit.row_ptr, static_cast<uint64_t>(J) + 1);
    r.vec(fit.col, static_cast<uint64_t>(fit.nnz));
    r.vec(fit.val, static_cast<uint64_t>(fit.nnz));
    // the taps index device buffers: rows must be well formed and columns inside [0, L)
    if (r.ok && (fit.nnz < 0 || fit.row_ptr.front() != 0 || fit.row_ptr.back() != fit.nnz))
      r.ok = false;
    for (size_t i = 1; r.ok && i < fit.row_ptr.size(); ++i)
      if (fit.row_ptr[i] < fit.row_ptr[i - 1]) r.ok = false;
    for (size_t t = 0; r.ok && t < fit.col.size(); ++t)
      if (fit.col[t] < 0 || fit.col[t] >= L) r.ok = false;
  } else if (method == SRP_LR) {
    const int D = P * (g.K - 1);
    r.vec(fit.ht, static_cast<uint64_t>(J) * R);
    r.vec(fit.hf, static_cast<uint64_t>(R) * D);
  }
  if (r.ok && (method == SRP_SLRI || method == SRP_LR) && (R != desc->rank || fit.sigma.empty()))
    r.ok = false;
  if (!r.ok || r.pos != r.buf.size()) return fail(SRP_EINVAL, "plan file contents do not match its header");
  return create_plan(desc, stream, out, &fit);
}

extern "C" srp_status srp_plan_estimate_bytes(const srp_plan_desc* desc, size_t* bytes) {
  clear_error();
  if (!bytes) return fail(SRP_EINVAL, "bytes is NULL");
  srp_status st = validate(desc);
  if (st != SRP_OK) return st;
  const srp_plan_desc& d = *desc;
  // N_p and L from the pair distances (Eq. N_p), without the TDOA table.
  long long L = 0;
  int maxNp = 0;
  for (int mp = 0; mp < d.M - 1; ++mp)
    for (int m = mp + 1; m < d.M; ++m) {
      const double* a = d.mic_xyz + 3 * m;
      const double* b = d.mic_xyz + 3 * mp;
      const double dist = std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) +
                                    (a[2] - b[2]) * (a[2] - b[2]));
      const int np = static_cast<int>(std::floor(dist / d.c * d.fs)) + d.n_aux;
      maxNp = std::max(maxNp, np);
      L += 2 * np + 1;
    }
  if (maxNp >= d.N / 2) return fail(SRP_EINVAL, "N_p >= K: the sample window is wider than the frame");
  const double J = d.J, P = d.M * (d.M - 1) / 2.0, N = d.N, K = d.N / 2.0, F = d.max_frames;
  const double eb = static_cast<double>(op_bytes(op_of(d.precision)));
  const double planes = op_split(op_of(d.precision)) ? 2.0 : 1.0;
  const double Lpad = std::ceil(L / 64.0) * 64.0;
  double b = F * d.M * K * 8.0 + F * 8.0 + 4096.0;  // y-hat, argmax keys, small tables
  switch (d.method) {
    case SRP_CONV: {
      const double hb = J * P * N * eb * planes;
      const bool gen = d.h_on_the_fly == 1 || (d.h_on_the_fly == 0 && hb > 64e9);
      // generated in the FP32 GEMM (the split TDOAs), or per chunk of at most kMaxChunkH
      // bytes for the tensor cores (plus the FP64 TDOA table)
      // the TC chunk path also holds its reduction slices' partial maps (at most 64 x F x the
      // chunk's cells; the chunk bounded here by the whole grid)
      const double hgen = d.precision == SRP_FP32
                              ? J * P * 8.0
                              : std::min(hb, kMaxChunkH) + J * P * 8.0 +
                                    std::min(64.0, std::floor(P * N / 64.0 / kChunkSliceSteps)) * F *
                                        std::min(J, kMaxChunkH / (hb / J)) * 4.0;
      b += (gen ? hgen : hb) + F * P * N * eb * planes;
      if (d.precision == SRP_FP32 && P * N > 16384) b += std::ceil(P * N / 16384.0) * F * J * 4.0;
      break;
    }
    case SRP_SLRI: {
      const double Rp = std::ceil(d.rank / 8.0) * 8.0;
      b += F * L * 4.0 + (J + L + F) * Rp * 4.0;
      if (d.precision != SRP_FP32) b += (J + F) * 64.0 * eb * planes;
      break;
    }
    case SRP_SSPI: {
      const double nnz = std::llround(d.taps_per_loc_pair * J * P);
      b += F * L * 4.0;
      if (d.precision == SRP_FP32)
        b += nnz * 8.0 + (J + 1) * 8.0;
      else
        b += (J + F) * Lpad * eb * planes + (J / 256.0 + 1) * 4.0 + J / 256.0 * Lpad / 64.0 * 4.0;
      break;
    }
    case SRP_LR: {
      const double kd2 = std::ceil(2.0 * d.rank / 64.0) * 64.0;
      b += (2.0 * d.rank + F) * P * N * eb * planes + (J + F) * kd2 * eb * planes +
           F * 2.0 * d.rank * 4.0 + F * 8.0;
      if (d.precision == SRP_FP32 && P * N > 16384)
        b += std::ceil(P * N / 16384.0) * F * 2.0 * d.rank * 4.0;
      else if (d.precision != SRP_FP32)
        b += 152.0 * 128.0 * 2.0 * d.rank * 4.0;  // split-K partial products of the fat GEMM
      break;
    }
    default:  // SI, TD
      b += F * L * 4.0 + (J + F) * Lpad * eb * planes;
      if (d.precision == SRP_FP32 && Lpad > 16384) b += std::ceil(Lpad / 16384.0) * F * J * 4.0;
      break;
  }
  *bytes = static_cast<size_t>(b);
  return SRP_OK;
}

extern "C" srp_status srp_plan_info(srp_plan_t plan, srp_plan_info_t* info) {
  clear_error();
  if (!plan || !info) return fail(SRP_EINVAL, "plan or info is NULL");
  const Geometry& g = plan->g;
  info->M = g.M;
  info->P = g.P;
  info->J = g.J;
  info->N = g.N;
  info->K = g.K;
  info->L = g.L;
  info->rank = plan->R;
  info->nnz = plan->nnz;
  info->tied_at_cut = plan->tied;
  info->device_bytes = plan->device_bytes;
  info->fit_seconds = plan->fit_seconds;
  info->launches = plan->launches;
  return SRP_OK;
}

extern "C" srp_status srp_plan_lags(srp_plan_t plan, int* Np) {
  clear_error();
  if (!plan || !Np) return fail(SRP_EINVAL, "plan or Np is NULL");
  for (int p = 0; p < plan->g.P; ++p) Np[p] = plan->g.Np[p];
  return SRP_OK;
}

extern "C" srp_status srp_map(srp_plan_t plan, const float* frames, int F, float* maps,
                              int* argmax, void* stream) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  if (F < 0) return fail(SRP_EINVAL, "F < 0");
  if (F == 0) return SRP_OK;
  if (!frames || (!maps && !argmax)) return fail(SRP_EINVAL, "frames, or both maps and argmax, NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geometry& g = plan->g;
  float* sink = nullptr;  // estimates only on the FP32 kernels: maps go to plan scratch
  if (!maps && plan->op == OpType::F32) {
    if (!plan->d_est_maps) {
      if (device_alloc(reinterpret_cast<void**>(&plan->d_est_maps),
                       sizeof(float) * plan->Fmax * static_cast<size_t>(g.J)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SRP_ENOMEM, "estimate-only scratch allocation failed");
      }
      plan->device_bytes += sizeof(float) * plan->Fmax * static_cast<size_t>(g.J);
    }
    sink = plan->d_est_maps;
  }
  for (int c0 = 0; c0 < F; c0 += plan->Fmax) {
    const int nf = std::min(plan->Fmax, F - c0);
    float* out = maps ? maps + static_cast<size_t>(c0) * g.J : sink;
    srp_status st = run_chunk(plan, frames + static_cast<size_t>(c0) * g.M * g.N, nf, out,
                              argmax ? argmax + c0 : nullptr, s);
    if (st != SRP_OK) return st;
  }
  return SRP_OK;
}

// Map scratch of srp_map_peaks without maps: chunks of frames whose maps stay within this
// many bytes, a fraction of the 126 MB L2, so that the exclusion passes read them from L2.
constexpr size_t kPeakScratchBytes = size_t(32) << 20;

extern "C" srp_status srp_map_peaks(srp_plan_t plan, const float* frames, int F, float* maps,
                                    int K, double d_min, int* peaks, float* values,
                                    void* stream) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  if (F < 0) return fail(SRP_EINVAL, "F < 0");
  if (K < 1 || K > kPeaksMax) return fail(SRP_EINVAL, "K must be in 1..16");
  if (!(d_min >= 0) || !std::isfinite(d_min)) return fail(SRP_EINVAL, "d_min must be finite and >= 0");
  if (F == 0) return SRP_OK;
  if (!frames || !peaks) return fail(SRP_EINVAL, "frames or peaks is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geometry& g = plan->g;
  if (!plan->d_grid4) {
    const size_t bytes = sizeof(float4) * static_cast<size_t>(g.J);
    if (dalloc(plan, &plan->d_grid4, bytes) != cudaSuccess) {
      cudaGetLastError();
      plan->d_grid4 = nullptr;
      return fail(SRP_ENOMEM, "grid coordinate table allocation failed");
    }
    SRP_CUDA_TRY(cudaMemcpyAsync(plan->d_grid4, plan->h_grid4.data(), bytes, cudaMemcpyHostToDevice, s));
  }
  int chunk = plan->Fmax;
  float* sink = nullptr;
  if (!maps) {
    if (!plan->d_peak_maps) {
      const size_t per = sizeof(float) * static_cast<size_t>(g.J);
      // whole 128-frame tiles of the contraction where the budget allows
      size_t fit = std::max<size_t>(1, kPeakScratchBytes / per);
      if (fit >= 128) fit = fit / 128 * 128;
      int fc = static_cast<int>(std::min<size_t>(plan->Fmax, fit));
      if (dalloc(plan, &plan->d_peak_maps, per * fc) != cudaSuccess) {
        cudaGetLastError();
        plan->d_peak_maps = nullptr;
        return fail(SRP_ENOMEM, "peak map scratch allocation failed");
      }
      plan->peak_chunk = fc;
    }
    sink = plan->d_peak_maps;
    chunk = plan->peak_chunk;
  }
  const float t = static_cast<float>(d_min * d_min);
  for (int c0 = 0; c0 < F; c0 += chunk) {
    const int nf = std::min(chunk, F - c0);
    float* out = maps ? maps + static_cast<size_t>(c0) * g.J : sink;
    srp_status st = run_chunk(plan, frames + static_cast<size_t>(c0) * g.M * g.N, nf, out, nullptr, s);
    if (st != SRP_OK) return st;
    plan->launches += peaks_launches(nf, K);
    SRP_CUDA_TRY(launch_peaks(out, nf, g.J, plan->d_grid4, plan->d_keys, K, t,
                              peaks + static_cast<size_t>(c0) * K,
                              values ? values + static_cast<size_t>(c0) * K : nullptr, s));
  }
  return SRP_OK;
}

extern "C" srp_status srp_map_host(srp_plan_t plan, const float* frames, int F, float* maps,
                                   int* argmax, void* stream) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  if (F < 0) return fail(SRP_EINVAL, "F < 0");
  if (F == 0) return SRP_OK;
  if (!frames || !maps) return fail(SRP_EINVAL, "frames or maps is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geometry& g = plan->g;
  const size_t Fm = static_cast<size_t>(plan->Fmax);
  if (!plan->d_stage_frames) {
    void* a = nullptr;
    void* b = nullptr;
    void* c = nullptr;
    if (device_alloc(&a, sizeof(float) * Fm * g.M * g.N) != cudaSuccess ||
        device_alloc(&b, sizeof(float) * Fm * g.J) != cudaSuccess ||
        device_alloc(&c, sizeof(int) * Fm) != cudaSuccess) {
      cudaGetLastError();
      if (a) cudaFree(a);
      if (b) cudaFree(b);
      return fail(SRP_ENOMEM, "staging allocation failed");
    }
    plan->d_stage_frames = static_cast<float*>(a);
    plan->d_stage_maps = static_cast<float*>(b);
    plan->d_stage_arg = static_cast<int*>(c);
    plan->device_bytes += sizeof(float) * Fm * (g.M * g.N + g.J) + sizeof(int) * Fm;
  }
  // Pipelined over sub-batches of whole 128-frame tiles: the frames of sub-batch b+1 come in
  // on one copy stream and the maps of sub-batch b-1 leave on two others (alternating) while
  // sub-batch b computes on `stream`. The host link (~190 GB/s each way) is the bound, the
  // compute hides behind it.
  if (!plan->copy_streams[0]) {
    for (int k = 0; k < 3; ++k)
      SRP_CUDA_TRY(cudaStreamCreateWithFlags(&plan->copy_streams[k], cudaStreamNonBlocking));
    for (int k = 0; k < kHostPipe; ++k)
      SRP_CUDA_TRY(cudaEventCreateWithFlags(&plan->pipe_events[k], cudaEventDisableTiming));
  }
  cudaStream_t in = plan->copy_streams[2];
  const int parts = 4;
  int sub = std::max(128, (plan->Fmax / parts + 127) / 128 * 128);
  sub = std::min(sub, plan->Fmax);
  int ev = 0, out = 0;
  auto order = [&](cudaStream_t from, cudaStream_t to) -> cudaError_t {
    cudaEvent_t e = plan->pipe_events[ev++ % kHostPipe];
    cudaError_t err = cudaEventRecord(e, from);
    return err != cudaSuccess ? err : cudaStreamWaitEvent(to, e, 0);
  };
  const size_t frame_floats = static_cast<size_t>(g.M) * g.N;
  SRP_CUDA_TRY(order(s, in));  // earlier work of `stream` on the staging buffers
  for (int c0 = 0; c0 < F; c0 += plan->Fmax) {
    const int nf = std::min(plan->Fmax, F - c0);
    for (int b0 = 0; b0 < nf; b0 += sub) {
      const int nb = std::min(sub, nf - b0);
      float* d_frames = plan->d_stage_frames + b0 * frame_floats;
      SRP_CUDA_TRY(cudaMemcpyAsync(d_frames, frames + (c0 + b0) * frame_floats,
                                   sizeof(float) * nb * frame_floats, cudaMemcpyHostToDevice, in));
      SRP_CUDA_TRY(order(in, s));
      srp_status st = run_chunk(plan, d_frames, nb, plan->d_stage_maps + static_cast<size_t>(b0) * g.J,
                                argmax ? plan->d_stage_arg + b0 : nullptr, s);
      if (st != SRP_OK) return st;
      cudaStream_t cs = plan->copy_streams[out++ % 2];
      SRP_CUDA_TRY(order(s, cs));
      SRP_CUDA_TRY(cudaMemcpyAsync(maps + static_cast<size_t>(c0 + b0) * g.J,
                                   plan->d_stage_maps + static_cast<size_t>(b0) * g.J,
                                   sizeof(float) * nb * g.J, cudaMemcpyDeviceToHost, cs));
      if (argmax)
        SRP_CUDA_TRY(cudaMemcpyAsync(argmax + c0 + b0, plan->d_stage_arg + b0, sizeof(int) * nb,
                                     cudaMemcpyDeviceToHost, cs));
    }
    // the next chunk reuses the staging buffers: its frames wait for this chunk's compute,
    // its compute for this chunk's map copies
    SRP_CUDA_TRY(order(s, in));
    for (int k = 0; k < 2; ++k) SRP_CUDA_TRY(order(plan->copy_streams[k], s));
  }
  SRP_CUDA_TRY(cudaStreamSynchronize(s));
  return SRP_OK;
}

extern "C" srp_status srp_stream_push(srp_plan_t plan, const float* hops, int B, int hop,
                                      float* maps, int* argmax, void* stream) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  if (B < 0) return fail(SRP_EINVAL, "B < 0");
  const Geometry& g = plan->g;
  if (hop < 1 || hop > g.N) return fail(SRP_EINVAL, "hop must be in 1..N");
  if (plan->stream_hop != 0 && plan->stream_hop != hop)
    return fail(SRP_EINVAL, "hop differs from the stream's (srp_stream_reset first)");
  if (B == 0) return SRP_OK;
  if (!hops || !maps) return fail(SRP_EINVAL, "hops or maps is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t Hn = static_cast<size_t>(g.N - hop);
  if (plan->stream_hop == 0) {  // first push: silent history, buffers sized for this hop
    for (int k = 0; k < 2; ++k) {
      if (plan->d_hist[k]) cudaFree(plan->d_hist[k]);
      plan->d_hist[k] = nullptr;
      if (device_alloc(reinterpret_cast<void**>(&plan->d_hist[k]),
                       sizeof(float) * std::max<size_t>(1, g.M * Hn)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SRP_ENOMEM, "stream history allocation failed");
      }
    }
    if (!plan->d_stream_frames &&
        device_alloc(reinterpret_cast<void**>(&plan->d_stream_frames),
                     sizeof(float) * plan->Fmax * g.M * g.N) != cudaSuccess) {
      cudaGetLastError();
      return fail(SRP_ENOMEM, "stream frame staging allocation failed");
    }
    SRP_CUDA_TRY(cudaMemsetAsync(plan->d_hist[0], 0, sizeof(float) * g.M * Hn, s));
    plan->stream_cur = 0;
    plan->stream_hop = hop;
  }
  for (int c0 = 0; c0 < B; c0 += plan->Fmax) {
    const int nb = std::min(plan->Fmax, B - c0);
    const int cur = plan->stream_cur;
    ++plan->launches;
    SRP_CUDA_TRY(launch_stream_frames(hops + static_cast<size_t>(c0) * g.M * hop, nb, g.M, hop, g.N,
                                      plan->d_hist[cur], plan->d_stream_frames,
                                      plan->d_hist[1 - cur], s));
    plan->stream_cur = 1 - cur;
    srp_status st = run_chunk(plan, plan->d_stream_frames, nb, maps + static_cast<size_t>(c0) * g.J,
                              argmax ? argmax + c0 : nullptr, s);
    if (st != SRP_OK) return st;
  }
  return SRP_OK;
}

extern "C" srp_status srp_stream_reset(srp_plan_t plan) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  plan->stream_hop = 0;  // the next push starts from a silent history
  return SRP_OK;
}

static_assert(SRP_TUNE_MAX >= TC_NVARIANTS, "the tuning report holds every variant");

extern "C" srp_status srp_plan_autotune(srp_plan_t plan, int F, void* stream,
                                        srp_tune_report_t* report) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  if (F < 1 || F > plan->Fmax) return fail(SRP_EINVAL, "F must be in 1..max_frames");
  srp_tune_report_t rep{};
  rep.variant = -1;
  for (int v = 0; v < SRP_TUNE_MAX; ++v) rep.ms[v] = -1.f;
  if (plan->op == OpType::F32) {  // nothing to choose on the FP32 path
    if (report) *report = rep;
    return SRP_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geometry& g = plan->g;
  float* d_frames = nullptr;
  float* d_maps = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  srp_status st = SRP_OK;
  const bool prof = plan->profiling;
  plan->profiling = false;
  const int saved = plan->tc_variant;
  const long long launches = plan->launches;
  if (device_alloc(reinterpret_cast<void**>(&d_frames), sizeof(float) * F * g.M * g.N) != cudaSuccess ||
      device_alloc(reinterpret_cast<void**>(&d_maps), sizeof(float) * F * static_cast<size_t>(g.J)) != cudaSuccess) {
    cudaGetLastError();
    st = fail(SRP_ENOMEM, "autotune buffers");
  }
  // a deterministic non-silent input: the timing of every stage is data independent
  if (st == SRP_OK && (cudaMemsetAsync(d_frames, 0x3C, sizeof(float) * F * g.M * g.N, s) != cudaSuccess ||
                       cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    st = fail(SRP_ECUDA, "autotune set-up");
  float best = 0.f;
  for (int v = 0; v < TC_NVARIANTS && st == SRP_OK; ++v) {
    if (!tc_gemm_variant_valid(v, plan->op)) continue;
    plan->tc_variant = v;
    for (int it = 0; it < 2 && st == SRP_OK; ++it)  // warm-up
      st = run_chunk(plan, d_frames, F, d_maps, nullptr, s);
    if (st != SRP_OK) break;
    if (cudaEventRecord(e0, s) != cudaSuccess) st = fail(SRP_ECUDA, "event");
    for (int it = 0; it < 5 && st == SRP_OK; ++it) st = run_chunk(plan, d_frames, F, d_maps, nullptr, s);
    if (st != SRP_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = fail(SRP_ECUDA, "autotune timing");
      break;
    }
    rep.ms[v] = ms / 5.f;
    if (rep.variant < 0 || rep.ms[v] < best) {
      best = rep.ms[v];
      rep.variant = v;
    }
  }
  plan->tc_variant = st == SRP_OK ? rep.variant : saved;
  plan->profiling = prof;
  plan->launches = launches;  // the tuning launches are not the caller's
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_frames) cudaFree(d_frames);
  if (d_maps) cudaFree(d_maps);
  if (st == SRP_OK && report) *report = rep;
  return st;
}

extern "C" srp_status srp_plan_set_variant(srp_plan_t plan, int variant) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  if (variant < -1 || variant >= TC_NVARIANTS) return fail(SRP_EINVAL, "variant must be in -1..11");
  if (plan->op == OpType::F32 && variant != -1)
    return fail(SRP_EINVAL, "FP32 plans have no tensor-core variant");
  if (variant >= 0 && !tc_gemm_variant_valid(variant, plan->op))
    return fail(SRP_EINVAL, "variants 3, 7 and 11 (hi and lo planes per stage) need a hi + lo precision");
  plan->tc_variant = variant;
  return SRP_OK;
}

extern "C" srp_status srp_gcc_samples(srp_plan_t plan, const float* frames, int F, float* xi,
                                      void* stream) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  if (plan->desc.method == SRP_CONV || plan->desc.method == SRP_LR)
    return fail(SRP_EUNSUPPORTED, "srp_gcc_samples needs a plan that samples the TD GCC");
  if (F < 0) return fail(SRP_EINVAL, "F < 0");
  if (F == 0) return SRP_OK;
  if (!frames || !xi) return fail(SRP_EINVAL, "frames or xi is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Geometry& g = plan->g;
  for (int c0 = 0; c0 < F; c0 += plan->Fmax) {
    const int nf = std::min(plan->Fmax, F - c0);
    if (plan->use_front) {
      plan->launches += 1;
      SRP_CUDA_TRY(launch_front(frames + static_cast<size_t>(c0) * g.M * g.N, nf, g.M, g.N,
                                plan->d_window, plan->d_twiddle, g.P, plan->d_pairs, plan->d_Np,
                                plan->d_off, plan->d_stab, g.L, plan->max_Np, nullptr, 0, g.L, 1.f, OpType::F32,
                                xi + static_cast<size_t>(c0) * g.L, nullptr, s));
      continue;
    }
    plan->launches += 1;
    SRP_CUDA_TRY(launch_stft_phat(frames + static_cast<size_t>(c0) * g.M * g.N, nf, g.M, g.N,
                                  plan->d_window, plan->d_twiddle, plan->d_yhat, s));
    SRP_CUDA_TRY(sample_to(plan, plan->d_yhat, nf, xi + static_cast<size_t>(c0) * g.L, nullptr, g.L,
                           OpType::F32, s));
  }
  return SRP_OK;
}

extern "C" srp_status srp_plan_sspi_taps(srp_plan_t plan, long long* row_ptr, int* col, float* val) {
  clear_error();
  if (!plan || plan->desc.method != SRP_SSPI) return fail(SRP_EINVAL, "not an SSPI plan");
  if (row_ptr) std::memcpy(row_ptr, plan->h_row_ptr.data(), sizeof(long long) * plan->h_row_ptr.size());
  if (col) std::memcpy(col, plan->h_col.data(), sizeof(int) * plan->h_col.size());
  if (val) std::memcpy(val, plan->h_val.data(), sizeof(float) * plan->h_val.size());
  return SRP_OK;
}

extern "C" srp_status srp_plan_slri_sigma(srp_plan_t plan, double* sigma, int n) {
  clear_error();
  if (!plan || (plan->desc.method != SRP_SLRI && plan->desc.method != SRP_LR))
    return fail(SRP_EINVAL, "not an SLRI or LR plan");
  if (!sigma || n < 0 || n > static_cast<int>(plan->sigma.size()))
    return fail(SRP_EINVAL, "n out of range");
  for (int i = 0; i < n; ++i) sigma[i] = plan->sigma[i];
  return SRP_OK;
}

extern "C" srp_status srp_plan_set_profiling(srp_plan_t plan, int enable) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  plan->profiling = enable != 0;
  plan->chunks_recorded = 0;
  return SRP_OK;
}

extern "C" srp_status srp_plan_stage_ms(srp_plan_t plan, float* ms, int* calls) {
  clear_error();
  if (!plan || !ms) return fail(SRP_EINVAL, "plan or ms is NULL");
  for (int k = 0; k < SRP_NSTAGES; ++k) ms[k] = 0.f;
  for (int c = 0; c < plan->chunks_recorded; ++c) {
    cudaEvent_t* e = plan->events.data() + static_cast<size_t>(c) * 5;
    SRP_CUDA_TRY(cudaEventSynchronize(e[4]));
    for (int k = 0; k < SRP_NSTAGES; ++k) {
      float t = 0.f;
      SRP_CUDA_TRY(cudaEventElapsedTime(&t, e[k], e[k + 1]));
      ms[k] += t;
    }
  }
  if (calls) *calls = plan->chunks_recorded;
  return SRP_OK;
}

extern "C" srp_status srp_plan_status(srp_plan_t plan, void* stream) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int code = 0;
  SRP_CUDA_TRY(cudaMemcpyAsync(&code, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SRP_CUDA_TRY(cudaStreamSynchronize(s));
  if (code != 0) {
    SRP_CUDA_TRY(cudaMemsetAsync(plan->d_err, 0, sizeof(int), s));
    SRP_CUDA_TRY(cudaStreamSynchronize(s));
    return fail(SRP_ETIMEOUT, "a bounded wait inside a kernel ran out (code " + std::to_string(code) +
                                  "); its maps are invalid");
  }
  return SRP_OK;
}

namespace srp {
namespace {
std::mutex g_alloc_mu;
int g_alloc_skip = 0, g_alloc_fail = 0;  // allocations to let through, then to fail
}
cudaError_t device_alloc(void** ptr, size_t bytes) {
  {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    if (g_alloc_skip > 0) {
      --g_alloc_skip;
    } else if (g_alloc_fail > 0) {
      --g_alloc_fail;
      *ptr = nullptr;
      return cudaErrorMemoryAllocation;
    }
  }
  return cudaMalloc(ptr, bytes);
}
}  // namespace srp

extern "C" srp_status srp_debug_fail_allocations(int after, int n) {
  clear_error();
  if (after < 0 || n < 0) return fail(SRP_EINVAL, "after and n must be >= 0");
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc_skip = n > 0 ? after : 0;
  g_alloc_fail = n;
  return SRP_OK;
}

extern "C" srp_status srp_debug_stall_next_contraction(srp_plan_t plan) {
  clear_error();
  if (!plan) return fail(SRP_EINVAL, "plan is NULL");
  if (plan->op == OpType::F32 || plan->h_generated)
    return fail(SRP_EUNSUPPORTED, "the plan runs no tensor-core contraction");
  plan->stall_next = true;
  return SRP_OK;
}

extern "C" void srp_destroy(srp_plan_t plan) {
  if (!plan) return;
  cudaDeviceSynchronize();
  free_plan(plan);
}

extern "C" const char* srp_last_error(void) { return g_last_error.c_str(); }
