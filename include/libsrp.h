/*
 * libsrp -- steered response power (SRP) maps on one GB300 (sm_103a).
 *
 * The hot path of "Scalable-Complexity Steered Response Power Based on Low-Rank
 * and Sparse Interpolation" (Dietzen, De Sena, van Waterschoot):
 *
 *   frames --(window, DFT of length N = 2K, PHAT)--> y-hat_m(omega_k)
 *          --(cross-spectra, Eq. corrmatrix)--> psi_p(omega_k), k = 1..K-1
 *   conv. FD-SRP   z = 2 Re[H psi]                      (boxed Eq. z_computed)
 *   SLRI-SRP       xi = iFFT-sampled TD GCC             (Eq. xi_p_ifft, n_prime)
 *                  z = Lambda_tall (Lambda_fat xi)       (boxed Eq. z_circlr_computed)
 *   SSPI-SRP       z = Lambda_sp xi                      (boxed Eq. z_circsp_computed)
 *   SI-SRP         z = Lambda xi                         (boxed Eq. z_circ_computed)
 *   LR-SRP         z = 2 Re[H_tall (H_fat psi)]          (boxed Eq. z_lr)
 *   conv. TD-SRP   z(i) = sum_p xi_p(round(Delta t_p(i)/T))  (Eq. TD_SRP)
 *   estimate       i_max = argmax_i z(i)                 (Eq. imax)
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - All functions return an srp_status; nothing is thrown across this boundary.
 *   On failure srp_last_error() returns a thread-local, NUL-terminated message
 *   that stays valid until the next libsrp call on the same thread.
 * - "device" pointers are CUDA device (or managed) memory of the current device;
 *   "host" pointers are ordinary (preferably pinned) host memory.  The caller owns
 *   every buffer it passes in.  Device buffers must be 16-byte aligned.
 * - A plan owns its device tables (SRP matrix, interpolation factors, tap lists)
 *   and its scratch buffers; it is bound to the device that was current when it
 *   was created and must be used with that device current.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  srp_map and srp_gcc_samples are asynchronous on `stream`; a plan
 *   may be used by one stream at a time (its scratch is shared by its calls).
 * - Microphone pairs p <-> (m, m') with m > m' are ordered m' outer, m inner
 *   (the double sum of Eq. SRP_omegaT); P = M(M-1)/2 (Sec. II-A).
 * - TD GCC samples of pair p are the lags n = -N_p..N_p in ascending order,
 *   pairs stacked (a relabelling of the paper's n_mod order, Eq. nmod/xi_single).
 */
#ifndef LIBSRP_H
#define LIBSRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srp_plan_s* srp_plan_t;

typedef enum {
  SRP_OK = 0,
  SRP_EINVAL = 1,       /* invalid argument (message says which) */
  SRP_ENOMEM = 2,       /* a device or host allocation failed */
  SRP_ECUDA = 3,        /* a CUDA runtime call failed (message carries its text) */
  SRP_ETIMEOUT = 4,     /* a bounded wait ran out */
  SRP_EUNSUPPORTED = 5, /* valid request that libsrp does not implement */
  SRP_EAGAIN = 6        /* a bounded queue is full: retry after draining results */
} srp_status;

typedef enum {
  SRP_CONV = 0,  /* conv. FD-SRP, Sec. II-D, boxed Eq. z_computed */
  SRP_SLRI = 1,  /* SLRI-SRP, Sec. IV-A, boxed Eq. z_circlr_computed */
  SRP_SSPI = 2,  /* SSPI-SRP, Sec. IV-A, boxed Eq. z_circsp_computed */
  SRP_SI = 3,    /* SI-SRP, Sec. III-B, boxed Eq. z_circ_computed (full sinc Lambda) */
  SRP_TD = 4,    /* conv. TD-SRP, Sec. II-D, Eq. TD_SRP (nearest-sample GCC lookup) */
  SRP_LR = 5     /* LR-SRP, Sec. III-A, boxed Eq. z_lr (rank-R factors of H) */
} srp_method;

/* Arithmetic of the map contraction.  The front end (DFT, PHAT, sampling, Lambda_fat xi) is
 * FP32-class in every case: FP32 FFTs, and the sampling and Lambda_fat products on the
 * warp-level tensor cores with FP16 hi+lo operands.  The tensor-core precisions run every
 * method's contraction on tcgen05 GEMMs: conv over the SRP matrix; SI, TD and SSPI over a
 * dense [J][L] interpolation operand (SSPI and TD skip the all-zero 64-column blocks of
 * each 256-cell tile); SLRI's Lambda_tall product; LR-SRP's two factor products.  "x3":
 * operands split into hi + lo planes (hi = rnd(x), lo = rnd(x - hi)) and three products
 * hi*hi + hi*lo + lo*hi accumulated in FP32. */
typedef enum {
  SRP_FP32 = 0,    /* FP32 operands, FP32 FFMA on CUDA cores */
  SRP_BF16 = 1,    /* BF16 tensor-core GEMM (kind::f16), FP32 accumulate */
  SRP_FP16 = 2,    /* FP16 tensor-core GEMM (kind::f16), FP32 accumulate */
  SRP_BF16X3 = 3,  /* BF16 hi+lo, 3 products: 16 significant bits per operand */
  SRP_FP16X3 = 4,  /* FP16 hi+lo, 3 products: 22 significant bits, FP32-class maps */
  SRP_TF32X3 = 5,  /* TF32 hi+lo, 3 products: 22 significant bits with the FP32 exponent
                      range, FP32-class maps at half the kind::f16 rate */
  SRP_TF32 = 6     /* TF32 tensor-core GEMM (kind::tf32, FP32 operands rounded to 10
                      mantissa bits), FP32 accumulate */
} srp_precision;

typedef enum {
  SRP_WIN_HANN = 0,       /* periodic Hann */
  SRP_WIN_SQRT_HANN = 1,  /* square-root periodic Hann (the paper's STFT, Sec. V-B) */
  SRP_WIN_RECT = 2        /* no window */
} srp_window;

/* Plan description (all host memory; the arrays are copied by srp_plan_create). */
typedef struct {
  int M;                    /* number of microphones, 2..64 */
  const double* mic_xyz;    /* [M][3] microphone positions r_m in metres */
  int J;                    /* number of candidate locations, 1..67107840 (SRP_FP32:
                               1..8388480) */
  const double* grid_xyz;   /* [J][3] candidate locations q_i in metres (near field,
                               Eq. Deltat_i first case), or unit vectors (far_field) */
  double fs;                /* sampling rate 1/T in Hz, > 0 */
  int N;                    /* frame / DFT length 2K: a power of two in 256..2048 */
  int window;               /* srp_window */
  double c;                 /* speed of sound in m/s (the paper uses 340), > 0 */
  int n_aux;                /* N_aux of Eq. N_p, 0..64 (the paper uses 2) */
  int method;               /* srp_method */
  int rank;                 /* SLRI: R_Lambda of Eq. min_Lambda_lr, 1..64 and <= min(J, L);
                               LR: R_H of Eq. min_lr, 1..64 and <= min(J, P(K-1)) */
  double taps_per_loc_pair; /* SSPI: t, Q_Lambda = round(t * J * P) non-zeros kept by
                               Eq. min_Lambda_sp; 0 < t and Q_Lambda <= J * L */
  int precision;            /* srp_precision */
  int max_frames;           /* frames processed per internal launch (scratch sizing),
                               1..65536; larger calls are processed in chunks */
  int far_field;            /* 0: grid_xyz are locations q_i (near field); 1: grid_xyz are
                               unit incident directions (far field, Eq. Deltat_i second
                               case: Delta t_p(i) = (r_m - r_m')^T q_i / c) */
  int h_on_the_fly;         /* conv: 1 = do not store the whole SRP matrix: SRP_FP32
                               generates it inside the GEMM, the tensor-core precisions
                               generate the rows of one chunk of cells (at most 48 GB, about
                               two waves of output tiles) before each chunk's GEMM; 0 = only
                               when the stored matrix would exceed 64 GB; -1 = never */
} srp_plan_desc;

/* Sizes of a created plan (filled by srp_plan_info). */
typedef struct {
  int M, P, J, N, K;        /* K = N/2; bins used are k = 1..K-1 */
  int L;                    /* number of TD GCC samples, sum_p (2 N_p + 1) */
  int rank;                 /* SLRI rank (0 for other methods) */
  long long nnz;            /* SSPI non-zeros Q_Lambda (0 for other methods) */
  long long tied_at_cut;    /* SSPI: entries whose quantised magnitude equals the
                               smallest kept one (selection ties, broken by (i, p, n)) */
  size_t device_bytes;      /* device memory held by the plan */
  double fit_seconds;       /* host+device time spent in srp_plan_create */
  long long launches;       /* kernels launched by this plan's srp_map / srp_map_host /
                               srp_gcc_samples calls so far (memsets and copies excluded) */
} srp_plan_info_t;

/*
 * srp_plan_create -- build a plan: TDOA table (Eq. Deltat_i, FP64), N_p (Eq. N_p),
 * and per method the device-resident operator:
 *   SRP_CONV: the SRP matrix H of Eq. H_p_single/H_single, stored as the real
 *             matrix [2cos(w_k dt_p(i)) | -2sin(w_k dt_p(i))] in the precision asked, or
 *             (h_on_the_fly, FP32) generated inside the GEMM from the TDOAs split as two
 *             FP32 numbers (phases accurate to ~1e-7) when it would not fit, or on the
 *             tensor cores generated in chunks of cells from the FP64 TDOAs, one chunk's
 *             rows before that chunk's GEMM;
 *   SRP_SLRI: Lambda (Eq. Lambda_p) -> its best rank-R approximation (Eq.
 *             min_Lambda_lr) from the eigen-decomposition of Lambda^T Lambda in FP64
 *             (L <= 768: Jacobi on the Gram matrix; longer: subspace iteration with
 *             Rayleigh-Ritz whose products Lambda X, Lambda^T Y run on the device, in FP32
 *             until the Ritz values settle and then in FP64 to 1e-13 relative),
 *             Lambda_fat = V_R^T, Lambda_tall = Lambda V_R, stored FP32;
 *   SRP_SSPI: the Q_Lambda largest-magnitude entries of Lambda (Eq. min_Lambda_sp),
 *             magnitudes quantised to multiples of 2^-40 and ties broken by ascending
 *             (i, p, n), stored as CSR rows (FP32 values, int32 sample indices) for the
 *             FP32 gather, or densely as [J][L] for the tensor cores;
 *   SRP_SI:   Lambda itself (Eq. Lambda_p, sinc evaluated in FP64), dense [J][L];
 *   SRP_TD:   the one-hot Lambda of conv. TD-SRP, 1 at n = round(Delta t_p(i)/T) with
 *             halves rounded away from zero (needs n_aux >= 1), dense [J][L];
 *   SRP_LR:   the best rank-R approximation (R = rank, 1..64) of the complex SRP matrix H
 *             (Eq. min_lr) from a device subspace iteration on H^H H in FP64,
 *             H_fat = V_R^H and H_tall = H V_R, stored as the real products
 *             [Re | -Im ; Im | Re] H_fat (2R x P N) and [2 Re | -2 Im] H_tall (J x 2R).
 * desc:   host, read only; the arrays are copied.
 * stream: stream for the uploads; the call returns after they complete.
 * out:    receives the plan handle (NULL on failure).
 * Errors: SRP_EINVAL (bad desc, including N_p >= K), SRP_EUNSUPPORTED (sizes libsrp does
 * not handle: the FP32 SSPI gather with L > 1700, a device operand above 200 GB, a
 * low-rank fit that does not converge, 16-bit LR operands out of range), SRP_ENOMEM,
 * SRP_ECUDA.
 */
srp_status srp_plan_create(const srp_plan_desc* desc, void* stream, srp_plan_t* out);

/*
 * srp_plan_estimate_bytes -- device memory a plan for `desc` would hold (tables, operands
 * and scratch for desc->max_frames frames), computed on the host from the pair distances
 * without building anything; used to admit work by HBM footprint.  The estimate covers
 * the allocations of srp_plan_create (within a few KB) but not the staging buffers that
 * srp_map_host adds on its first call.  Errors: SRP_EINVAL (as srp_plan_create).
 */
srp_status srp_plan_estimate_bytes(const srp_plan_desc* desc, size_t* bytes);

/* srp_plan_info -- sizes and memory of a plan.  info: host, written. */
srp_status srp_plan_info(srp_plan_t plan, srp_plan_info_t* info);

/*
 * srp_plan_lags -- N_p of every pair (Eq. N_p).  Np: host int[P], written.
 */
srp_status srp_plan_lags(srp_plan_t plan, int* Np);

/*
 * srp_map -- SRP maps and their argmax for F frames (the whole hot path).
 * frames: device float [F][M][N]: frame f, microphone m, sample n (unwindowed).
 * maps:   device float [F][J], written: z(i) of the plan's method per frame; or NULL for
 *         estimates only (argmax must then be given): on the tensor-core precisions no map
 *         is written at all (the contraction's epilogue keeps only the per-frame maximum),
 *         which removes the F*J*4-byte map write that bounds SLRI / SSPI; FP32 plans write
 *         into plan scratch allocated by the first such call.
 * argmax: device int32 [F] or NULL, written: i_max per frame (Eq. imax), the lowest
 *         index among equal maxima.
 * F = 0 is a no-op.  Asynchronous on `stream`.
 * Errors: SRP_EINVAL (NULL plan/frames, maps and argmax both NULL, F < 0), SRP_ENOMEM,
 * SRP_ECUDA.
 */
srp_status srp_map(srp_plan_t plan, const float* frames, int F, float* maps, int* argmax,
                   void* stream);

/*
 * srp_map_peaks -- several source estimates per frame: the peak picking of Eq. (qshat)-
 * (imax) extended to several sources.  For each frame Eq. (imax) is taken K times, each
 * time over the candidate locations not yet excluded; a pick excludes itself and every
 * location closer than d_min metres to it.  The lowest index wins a tie.  The distance
 * test is made in FP32 on the grid coordinates rounded to FP32: d^2 = ((dx*dx + dy*dy) +
 * dz*dz) with every operation rounded to FP32, excluded when d^2 < d_min^2 (the FP64
 * square rounded to FP32); on a far-field plan the coordinates are the unit directions.
 *   frames: device float [F][M][N].
 *   maps:   device float [F][J], written (as srp_map), or NULL: estimates only.  The maps
 *           then go through plan-owned scratch in chunks of at most 32 MB (whole
 *           128-frame tiles where that allows; allocated on the first such call and kept),
 *           small enough to stay in L2 between the contraction that writes them and the
 *           passes that read them.
 *   K:      picks per frame, 1..16;  d_min: metres, finite, >= 0 (0: the K largest cells).
 *   peaks:  device int32 [F][K], written; -1 where no location is left.
 *   values: device float [F][K] (the map values at the picks, NaN where -1) or NULL.
 * Pick 0 is the argmax srp_map returns.  The first call also copies the grid coordinates
 * to the device (J x 16 bytes, kept by the plan).  Asynchronous on `stream`.
 * Errors: SRP_EINVAL (NULL plan, frames or peaks; F < 0; K or d_min out of range),
 * SRP_ENOMEM, SRP_ECUDA.
 */
srp_status srp_map_peaks(srp_plan_t plan, const float* frames, int F, float* maps, int K,
                         double d_min, int* peaks, float* values, void* stream);

/*
 * srp_map_host -- srp_map on host buffers: copies frames host->device into plan-owned
 * staging, runs the path, copies maps (and argmax) device->host, and synchronises
 * `stream` before returning.  frames: host float [F][M][N]; maps: host float [F][J];
 * argmax: host int32 [F] or NULL (page-locked host memory gives the full link rate).  Each
 * chunk of max_frames frames is processed in sub-batches of whole 128-frame tiles: the
 * frames of one sub-batch come in on a plan-owned copy stream and the maps of the
 * previous ones leave on two others while `stream` computes, ordered with events.  The
 * staging buffers (max_frames frames and maps), the three copy streams and their events
 * are created on the first call and kept by the plan; calls on one plan must not overlap.
 * Errors: as srp_map.
 */
srp_status srp_map_host(srp_plan_t plan, const float* frames, int F, float* maps, int* argmax,
                        void* stream);

/*
 * srp_stream_push -- srp_map on a continuous multichannel stream (Sec. V-B: frames of N
 * samples every hop samples).  hops: device float [B][M][hop], B consecutive blocks of hop
 * new samples per channel.  The plan keeps the last N - hop samples of every channel
 * between calls (in device memory, allocated by the first push), so each block completes
 * one frame: frame b is the N samples ending with block b.  The stream starts from a
 * silent (zero) history.  maps: device float [B][J]; argmax: device int32 [B] or NULL.
 * hop is fixed for the stream: a different hop fails until srp_stream_reset.  B = 0 is a
 * no-op.  Asynchronous on `stream`; pushes must be ordered on one stream.
 * Errors: SRP_EINVAL, SRP_ENOMEM, SRP_ECUDA.
 */
srp_status srp_stream_push(srp_plan_t plan, const float* hops, int B, int hop, float* maps,
                           int* argmax, void* stream);

/* srp_stream_reset -- forget the stream's history; the next push starts a new stream. */
srp_status srp_stream_reset(srp_plan_t plan);

/*
 * srp_gcc_samples -- the sampling stage alone (Eq. xi_p_ifft, n_prime, xi_single):
 * PHAT cross-spectra of every pair, iFFT of the two-sided spectrum (unnormalised,
 * length N), and the 2N_p+1 samples at lags -N_p..N_p.  Valid for every plan but conv.
 * frames: device float [F][M][N]; xi: device float [F][L], written (pair-major,
 * ascending lag).  Valid for every plan but conv.  Asynchronous on `stream`.
 * Errors: SRP_EINVAL, SRP_EUNSUPPORTED (conv plan), SRP_ECUDA.
 */
srp_status srp_gcc_samples(srp_plan_t plan, const float* frames, int F, float* xi, void* stream);

/*
 * srp_plan_autotune -- pick the tensor-core kernel variant of this plan by timing them on
 * the device: 128x256-cell tiles with 4 operand stages (long reductions), 128x256 with 2
 * stages and 4 output boxes per epilogue warp (short reductions, map-write bound),
 * 128x128 tiles (twice the tiles for small grids or batches), and for the hi + lo
 * precisions 128x256 tiles with 2 stages that each hold the hi and lo planes of both
 * operands for one k-block and issue its three products in turn (each operand tile loaded
 * once instead of twice; variant 3); variants 4..7 are variants 0..3 run in clusters of
 * 2 CTAs that take two frame tiles of one cell tile together and share each tile of the
 * SRP / interpolation operand by TMA multicast (each CTA loads half of it), and variants
 * 8..11 in clusters of 2 x 2 that also share each tile of the frame operand between two
 * cell tiles (dense reductions; block-sparse ones run as 4..7); the maps are the same bit
 * for bit.  Each variant runs the whole
 * srp_map path 2 + 5 times on F frames of a synthetic input (plan-owned temporary
 * buffers); the fastest is kept by the plan for later calls.  Until a plan is tuned a
 * heuristic picks by reduction length (and clusters of two from two frame tiles on).
 * FP32 plans have nothing to tune (variant -1).
 * F: 1..max_frames, the batch size the plan will serve.  Synchronises `stream`.
 * report: host, written (or NULL): the chosen variant and the mean milliseconds per
 * srp_map call of every variant (-1 where not run).  Errors: SRP_EINVAL, SRP_ENOMEM,
 * SRP_ECUDA.
 */
enum { SRP_TUNE_MAX = 12 };
typedef struct {
  int variant;
  float ms[SRP_TUNE_MAX];
} srp_tune_report_t;
srp_status srp_plan_autotune(srp_plan_t plan, int F, void* stream, srp_tune_report_t* report);

/* srp_plan_set_variant -- pin the tensor-core variant (0..11 as in srp_plan_autotune) or
 * return to the heuristic (-1).  Errors: SRP_EINVAL (out of range, an FP32 plan, or
 * variant 3, 7 or 11 without a hi + lo precision). */
srp_status srp_plan_set_variant(srp_plan_t plan, int variant);

/*
 * srp_plan_sspi_taps -- copy an SSPI plan's kept entries to the host.
 * row_ptr: host int64 [J+1] or NULL; col: host int32 [nnz] or NULL (sample index into
 * the stacked xi of srp_gcc_samples); val: host float [nnz] or NULL.
 * Errors: SRP_EINVAL (not an SSPI plan).
 */
srp_status srp_plan_sspi_taps(srp_plan_t plan, long long* row_ptr, int* col, float* val);

/*
 * srp_plan_slri_sigma -- the plan's singular values of Lambda (square roots of the
 * eigenvalues of Lambda^T Lambda, descending).  sigma: host double [n]; n <= L when
 * L <= 768, else n <= min(L, R + 32) (the values the subspace iteration resolves).
 * Errors: SRP_EINVAL (not an SLRI plan, n out of range).
 */
srp_status srp_plan_slri_sigma(srp_plan_t plan, double* sigma, int n);

/*
 * Per-stage timing (the tracing hook used by the benchmark).  When enabled, every
 * srp_map / srp_map_host call records CUDA events on its stream around its stages:
 *   SRP_STAGE_FRONTEND   window + DFT + PHAT
 *   SRP_STAGE_SPECTRA    cross-spectra: iFFT sampling (SLRI/SSPI) or operand packing (conv)
 *   SRP_STAGE_CONTRACT   the map contraction (conv GEMM, SLRI fat+tall, SSPI gather)
 *   SRP_STAGE_ARGMAX     argmax finalisation
 * srp_plan_set_profiling(plan, 1) starts a new record (and 0 stops recording); the
 * record holds up to 4096 internal chunks.  srp_plan_stage_ms waits for the recorded
 * events and writes the milliseconds per stage summed over every chunk recorded since
 * profiling was enabled to ms[SRP_NSTAGES]; *calls receives the number of chunks.
 * Errors: SRP_EINVAL (NULL plan/ms), SRP_ECUDA.
 */
enum { SRP_STAGE_FRONTEND = 0, SRP_STAGE_SPECTRA = 1, SRP_STAGE_CONTRACT = 2,
       SRP_STAGE_ARGMAX = 3, SRP_NSTAGES = 4 };
srp_status srp_plan_set_profiling(srp_plan_t plan, int enable);
srp_status srp_plan_stage_ms(srp_plan_t plan, float* ms, int* calls);

/*
 * srp_plan_status -- failure detection for the kernels' bounded waits.  Synchronises
 * `stream`, then returns SRP_ETIMEOUT (and clears the record) if a wait inside one of
 * the plan's kernels ran out since the last query: the kernel then abandoned its tile
 * loop, released its resources and returned, and the maps of that call are invalid.
 * Returns SRP_OK otherwise.  Errors: SRP_EINVAL (NULL plan), SRP_ECUDA.
 */
srp_status srp_plan_status(srp_plan_t plan, void* stream);

/*
 * srp_plan_save / srp_plan_create_from_file -- checkpoint and resume a plan's offline fit
 * (the paper computes the interpolation factors "upfront", Sec. IV; with long sample
 * vectors the FP64 fit dominates plan creation).  srp_plan_save writes the method's fit to
 * `path`: SLRI sigma, Lambda_tall [J][Rp] and Lambda_fat [Rp][L] (FP32, as the plan uses
 * them), the SSPI taps (CSR), or LR-SRP's sigma and complex FP64 factors; other methods
 * have no fit and write the header only.  The file carries a hash of the inputs the fit
 * depends on (microphones, grid, fs, N, c, n_aux, method, rank or taps, far_field) and a
 * checksum.  srp_plan_create_from_file is srp_plan_create with the fit read from `path`
 * instead of computed; the precision, window and max_frames may differ from the saved
 * plan's.  Errors: SRP_EINVAL (NULL arguments, unreadable or damaged file, a file made for
 * other inputs or another method), then as srp_plan_create.  The file format is
 * little-endian and versioned.
 */
srp_status srp_plan_save(srp_plan_t plan, const char* path);
srp_status srp_plan_create_from_file(const srp_plan_desc* desc, const char* path, void* stream,
                                     srp_plan_t* out);

/*
 * Failure-detection test hooks.  They make a failure on the host side of a call, never a
 * device fault, trap or unbounded wait.
 *
 * srp_debug_fail_allocations -- the next `n` device allocations libsrp makes for plans
 * and serving slots fail as if the device were out of memory, after `after` further
 * allocations have succeeded (process-wide; n = 0 clears).  Plan creation then returns
 * SRP_ENOMEM having released what it had allocated; the server refuses the session.
 * Errors: SRP_EINVAL (after or n negative).  Needs no GPU.
 *
 * srp_debug_stall_next_contraction -- the plan's next tensor-core contraction issues no
 * operand loads: its MMA and epilogue warps wait on barriers that nothing completes until
 * their bounded waits (0.2 s for this launch) run out; the kernel releases its tensor
 * memory and returns.  srp_plan_status then reports SRP_ETIMEOUT and the plan stays
 * usable for the next call.  Errors: SRP_EINVAL (NULL plan), SRP_EUNSUPPORTED (the plan
 * has no tensor-core contraction: SRP_FP32).
 */
srp_status srp_debug_fail_allocations(int after, int n);
srp_status srp_debug_stall_next_contraction(srp_plan_t plan);

/*
 * srp_slri_apply_static -- the SLRI interpolation of one batch, u = Lambda_fat xi then
 * z = Lambda_tall u and the argmax per frame, without allocating any memory.  The paper
 * has no counterpart: this entry point exists for callers that cannot allocate device
 * memory when they process frames, e.g. a real-time audio thread with a per-frame
 * deadline (cudaMalloc may block and synchronise the whole device) or a host whose
 * device memory is owned and budgeted by its own pool, which forbids allocations
 * outside it.  Such a caller brings its own factors (e.g. computed offline) and buffers.
 *   xi:     device float [F][L], TD GCC samples (as written by srp_gcc_samples).
 *   fat:    device float [R][L], Lambda_fat.
 *   tall:   device float [J][R], Lambda_tall, 16-byte aligned.
 *   R:      8, 16, 24, ..., 64 (pad a smaller rank with zero rows/columns).
 *   maps:   device float [F][J], written.   argmax: device int32 [F] or NULL, written.
 * Limits: F <= 65536, F * R <= 1048576, 1 <= L <= 50000; larger requests return
 * SRP_EINVAL with a message.  F = 0 is a no-op.  Asynchronous on `stream`.
 * Scratch: the intermediate u and the argmax keys live in one file-scope device array of
 * 4.5 MiB; every GPU that loads libsrp holds it until the process exits.  All calls on
 * a device share it and each call overwrites it (the keys are cleared by the call), so
 * calls whose execution overlaps on the GPU (different streams, or different host
 * threads without ordering) race and give wrong results: serialise them.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it per CUDA context (under
 * the context's process-unique ID), so the first call after a device reset or in a new
 * context repeats the lookup; make the first call on a device before any stream capture.
 * Errors: SRP_EINVAL (sizes, NULL or misaligned pointers), SRP_ECUDA.
 */
srp_status srp_slri_apply_static(const float* xi, const float* fat, const float* tall, int F,
                                 int L, int R, int J, float* maps, int* argmax, void* stream);

/* ==================================================================================
 * Serving: many concurrent sessions on one GPU (the paper has no serving layer; this is
 * the runtime around the per-frame path above).  A session is one microphone array with
 * its own plan description (geometry, grid, method, rank / taps, precision) and hop size.
 *   - Admission by HBM footprint: srp_server_open queues the session; a builder thread
 *     creates its plan once srp_plan_estimate_bytes + its launch buffers fit into
 *     hbm_budget next to the admitted sessions and fewer than max_sessions are active.
 *     Sessions are admitted in arrival order.
 *   - srp_server_push appends samples; frames of N samples are cut every `hop` samples
 *     (the last N - hop samples of each channel carry over) and queue as pending.
 *   - Continuous batching: a scheduler thread moves each session's pending frames (up to
 *     max_batch, a power of two) into a free launch slot as soon as the session's previous
 *     launch has finished (one launch in flight per session); frames arriving meanwhile
 *     join the next launch.  Sessions are spread round-robin over `streams` CUDA streams,
 *     so the launches of different sessions overlap on the device.
 *   - use_graphs: each (slot, power-of-two batch size) launch sequence -- H2D frames, the
 *     SRP path, D2H maps and argmax, a completion callback -- is captured as a CUDA graph by
 *     the builder thread at admission (after srp_plan_autotune picks the session's tile
 *     shape for max_batch) and replayed by the scheduler.
 *   - Grouped launches (group_launches = 1): sessions whose plan is FP32 (CUDA cores),
 *     uses the fused front end (N <= 1024, N_p <= 32) and is SLRI or SSPI with the
 *     whole-vector gather (L <= 1643) are bucketed by (method, N, sampling tiles, padded
 *     rank or gather width).  The scheduler takes the pending frames of every such session
 *     of a bucket that has no launch in flight into one grouped launch: one host-to-device
 *     copy of all their frames and of a work list, one front-end kernel over the list of
 *     (session, frame) items, one interpolation kernel over (session, cell block, frame
 *     block) items, one argmax pass, one device-to-host copy of all their maps.  Each
 *     session still has at most one launch in flight, and its maps equal srp_map's on its
 *     plan bit for bit.  Other sessions launch on their own.
 *   - Latency of a frame = completion of its map's D2H copy - its arrival time (the time
 *     its last sample was pushed, or the caller's t_arrival).
 * All functions are thread-safe.  The server owns its threads, streams and buffers.
 * ================================================================================== */
typedef struct srp_server_s* srp_server_t;

typedef struct {
  size_t hbm_budget;      /* device bytes the sessions may hold together */
  int max_sessions;       /* active sessions at most, 1..4096 */
  int max_batch;          /* frames per launch, a power of two in 1..4096 */
  int streams;            /* CUDA streams the sessions are spread over, 1..64 */
  int slots_per_session;  /* launches a session may have in flight or awaiting poll, 1..16 */
  int pending_frames;     /* pending-frame queue per session (>= max_batch) */
  int use_graphs;         /* 1: replay captured CUDA graphs; 0: issue launches directly */
  int group_launches;     /* 1: sessions that qualify share launches (see below); 0: never */
} srp_server_desc;

typedef struct {
  long long frames_done;      /* frames whose maps were returned by srp_server_poll */
  long long frames_launched;  /* frames submitted to the GPU */
  long long launches;         /* batch launches (each: one srp_map of b frames) */
  long long graph_launches;   /* of which replayed CUDA graphs */
  size_t device_bytes;        /* device memory held (or reserved) by admitted sessions */
  int sessions_active, sessions_queued;
  double latency_p50_s, latency_p99_s, latency_max_s;  /* over frames polled since reset */
  long long group_launches;   /* of `launches`: grouped launches shared by several sessions */
  long long group_frames;     /* frames they carried */
  long long group_sessions;   /* session batches they carried (sum over the launches) */
} srp_server_stats_t;

enum { SRP_SESSION_QUEUED = 0, SRP_SESSION_ACTIVE = 1, SRP_SESSION_CLOSING = 2,
       SRP_SESSION_CLOSED = 3, SRP_SESSION_FAILED = 4 };

/* srp_server_create -- start a server on the current device.  desc: host, read.
 * Errors: SRP_EINVAL (a field out of range), SRP_ECUDA. */
srp_status srp_server_create(const srp_server_desc* desc, srp_server_t* out);

/* srp_server_open -- queue a session.  desc: as for srp_plan_create (copied;
 * desc->max_frames must be >= max_batch); hop: 1..N samples between frames.
 * session: receives the id.  Errors: SRP_EINVAL, SRP_ENOMEM (the session alone exceeds
 * hbm_budget).  A plan that fails to build puts the session in SRP_SESSION_FAILED. */
srp_status srp_server_open(srp_server_t server, const srp_plan_desc* desc, int hop, int* session);

/* srp_server_push -- append n samples per channel.  samples: host float [M][n] (channel
 * major), copied.  t_arrival: arrival time in seconds on the steady clock of
 * srp_server_now, or < 0 for now.  Errors: SRP_EAGAIN (the pending queue would
 * overflow: poll and retry), SRP_EINVAL (unknown or closed session), SRP_ECUDA (failed). */
srp_status srp_server_push(srp_server_t server, int session, const float* samples, int n,
                           double t_arrival);

/* srp_server_poll -- take the session's finished frames, oldest first, whole launches
 * only.  max_frames >= max_batch.  maps: host float [max_frames][J] or NULL; argmax,
 * frame_index (0-based frame number of the session's stream), latency_s: host arrays of
 * max_frames or NULL.  *n_out receives the number of frames written. */
srp_status srp_server_poll(srp_server_t server, int session, int max_frames, float* maps,
                           int* argmax, long long* frame_index, double* latency_s, int* n_out);

/* srp_server_session_info -- state (SRP_SESSION_*), device bytes held, frames pending or in
 * flight.  Returns SRP_ECUDA with the failure message for a failed session. */
srp_status srp_server_session_info(srp_server_t server, int session, int* state,
                                   size_t* device_bytes, int* pending);

/* srp_server_close -- stop a session: pending frames and unpolled results are dropped and
 * its memory is released once its launches in flight finish (queued sessions may then be
 * admitted). */
srp_status srp_server_close(srp_server_t server, int session);

/* srp_server_stats / srp_server_reset_stats -- counters and latency percentiles. */
srp_status srp_server_stats(srp_server_t server, srp_server_stats_t* stats);
srp_status srp_server_reset_stats(srp_server_t server);

/* srp_server_now -- the clock of t_arrival and of the latencies, in seconds. */
double srp_server_now(void);

/* srp_server_destroy -- stop the threads, wait for launches in flight, free everything. */
void srp_server_destroy(srp_server_t server);

/* srp_destroy -- release a plan and its device memory (synchronises the device). */
void srp_destroy(srp_plan_t plan);

/* srp_last_error -- the message of the last failure on this thread ("" if none). */
const char* srp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LIBSRP_H */
