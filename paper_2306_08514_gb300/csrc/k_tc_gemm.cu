// The map contractions on the 5th-generation tensor cores (tcgen05):
//
//   Z[F][J] = A B^T,   A [F][Kd] (one row per frame), B [J][Kd] (one row per cell),
//
// 16-bit operands (F16 or BF16) with FP32 accumulation in TMEM and the per-frame argmax
// (Eq. imax) fused into the epilogue.  It serves every method:
//   conv. FD-SRP  A = [Re psi | Im psi] per pair, B = [2cos | -2sin] (boxed Eq. z_computed);
//   SSPI-SRP      A = xi, B = Lambda_sp stored densely; zero k-blocks of a cell tile are
//                 skipped through a per-tile k-block list (boxed Eq. z_circsp_computed);
//   SLRI-SRP      A = u = Lambda_fat xi, B = Lambda_tall (boxed Eq. z_circlr_computed).
// The FP16 hi+lo mode runs three products (A_hi B_hi, A_hi B_lo, A_lo B_hi) as one longer
// reduction, which carries about 22 significant bits per operand.
//
// Persistent, warp-specialised kernel, one CTA per SM:
//   warp 0      TMA producer: 128x64 tile of A and 256x64 tile of B per k-block into a
//               4-stage (2-stage for <= 3 k-blocks per tile) 128-byte-swizzled
//               shared-memory ring (the FUSED hi + lo kernel: 2 stages, each with the hi
//               and lo planes of both operands);
//   warp 1      TMEM owner and single-thread MMA issuer: 4 x tcgen05.mma (M128 N256 K16)
//               per k-block and product into one of two 128x256 FP32 accumulators (512 TMEM
//               columns);
//   warps 2-9   epilogue: two warps per TMEM lane quarter, each owning 128 of the 256
//               columns of 32 frame rows; results leave through swizzled shared-memory
//               boxes (1 per warp, or 4 with the 2-stage ring) and TMA tensor stores
//               (coalesced, asynchronous).
// The tensor cores round every accumulation step towards zero, which biases long sums
// (about -2e-5 relative after 600 K=16 steps).  So a tile's reduction is cut into
// chunks of KB_PER_CHUNK k-blocks: each chunk starts a fresh TMEM accumulator (the two
// accumulators alternate, so the MMAs of chunk c+1 overlap the drain of chunk c), and the
// epilogue adds every finished chunk into FP32 registers (round to nearest).
// Tiles run m-fastest so the CTAs in flight share the tiles of B.  Cluster variants
// (CS = 2 CTAs per cluster) go further: the two frame tiles of one cell tile run
// together, CTA r of the cluster loads rows [r TN/2, (r+1) TN/2) of each B tile and
// multicasts them into the same stage of both CTAs, and each CTA's MMA issuer frees a
// stage in both (a stage is refilled once both CTAs have consumed it), so each B tile
// crosses L2 once per pair of frame tiles.  Clusters of 2 x 2 (dense reductions) add the
// other direction: the two cell tiles of a cluster share each A tile the same way, so that
// both operands cross L2 once per two tiles (long reductions over operands far larger
// than L2, where the CTAs sharing a tile would otherwise drift apart and re-read it from
// DRAM).  A tile past F or J computes on zero rows and writes nothing; a single frame tile
// runs unclustered.  When the output tiles are too few to
// fill the GPU, or the reduction is long, the (dense) reduction is also split into slices
// written to a workspace and summed in FP64 (split_reduce in k_conv_simt.cu).  Every
// mbarrier wait is bounded (2 s); on a timeout the CTA records an error code, drains its
// own copies and MMAs, frees its TMEM and returns.
#include "srp_internal.h"
#include "srp_device.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

namespace srp {

namespace {
constexpr int TM = 128, TK = 64;
constexpr int LIST_TILE = 256;                // cells per block-sparse k-block list
constexpr int NEPI = 8;                       // epilogue warps
constexpr int NTHREADS = 64 + 32 * NEPI;
constexpr int OUT_BOX = 32 * 32 * 4;          // one 32x32 FP32 output box
constexpr int KB_PER_CHUNK = 8;               // 32 K=16 steps per accumulator chunk
constexpr int BAR_BYTES = 256;
template <int TN, bool FUSED = false>
constexpr int stage_bytes() { return (FUSED ? 2 : 1) * (TM + TN) * TK * 2; }
// Shared-memory splits (variants): STAGES operand stages and BOXES output boxes per
// epilogue warp.  Long reductions keep 4 stages and one box; short ones (bound by the map
// write) keep 2 stages and 4 boxes, so a warp's boxes of a tile leave without waiting for
// one another.  TN is the cell width of a tile (256, or 128 for small grids).
// FUSED (hi + lo precisions): a stage holds A_hi, A_lo, B_hi and B_lo of one k-block and
// feeds all three products, so each operand tile is loaded once instead of twice.  (Half
// k-blocks of 64-byte rows, 64-byte swizzle, in 4 stages measured 4-7 % slower.)
template <int STAGES, int BOXES, int TN, bool FUSED = false>
constexpr int smem_bytes() {
  return STAGES * stage_bytes<TN, FUSED>() + NEPI * BOXES * OUT_BOX + BAR_BYTES + 1024;
}
static_assert(smem_bytes<4, 1, 256>() <= 232448 && smem_bytes<2, 4, 256>() <= 232448 &&
                  smem_bytes<4, 2, 128>() <= 232448 && smem_bytes<2, 1, 256, true>() <= 232448,
              "shared memory budget");
// k-blocks per accumulator chunk of the FUSED kernel: 3 x 12 = 36 K=16 steps
constexpr int KB_PER_CHUNK_FUSED = 3;
// k-steps per tile up to which the heuristic picks 2 stages + 4 boxes (measured on uca8:
// SLRI's one k-block per tile 0.112 -> 0.085 ms; SSPI's five k-blocks run faster with 4)
constexpr int SHORT_MAX_STEPS = 3;
constexpr uint64_t WAIT_NS = 2000000000ull;        // limit of every mbarrier wait
constexpr uint64_t STALL_WAIT_NS = 200000000ull;   // ... in a failure-detection test launch
constexpr int MIN_KB_PER_SLICE = 32;
}  // namespace

struct TcParams {
  int F, J;
  int kb_per_seg, nseg;  // dense k-steps per operand segment, number of segments
  int sub_shift;         // log2 of the k-steps per 64 operand columns (1 for TF32, else 0)
  int tf32;              // kind::tf32 instead of kind::f16
  int stall;             // failure-detection test: the producer issues no loads
  unsigned long long wait_ns;  // limit of every mbarrier wait
  const int* kb_ptr;     // block-sparse: the 64-column windows of cell tile n start at the
  const int* kb_idx;     //   columns kb_idx[kb_ptr[n] .. kb_ptr[n+1]); NULL = dense
  int nM, nN, nslices, kb_per_slice;
  int tma_out;           // 1: results leave by TMA store through tmZ; 0: plain stores
  int tn;                // cell width of a tile
  int ldz, col0;         // row stride of Z; map index of its column 0 (argmax keys)
  float* Z;              // maps [F][ldz] (nslices == 1) or partial maps [nslices][F][J]
  unsigned long long* keys;
  int* err;
};

// The k-step range [s0, s1) of tile t, and the tile's coordinates.
struct TileWork {
  int slice, m, n, s0, s1, m_len, list;
};

// Clusters of CS CTAs: CM frame tiles x CN cell tiles (CS = 1: 1 x 1, 2: 2 x 1, 4: 2 x 2);
// cluster rank r is (rm, rn) = (r mod CM, r / CM).
template <int CS>
struct ClusterShape {
  static constexpr int CM = CS == 1 ? 1 : 2;
  static constexpr int CN = CS == 4 ? 2 : 1;
};

// Tile t of a cluster (t counts groups of CM x CN tiles), as seen by the CTA (rm, rn); CS = 1
// is the plain m-fastest walk.
template <int CS>
__device__ __forceinline__ int tile_groups(const TcParams& p) {
  constexpr int CM = ClusterShape<CS>::CM, CN = ClusterShape<CS>::CN;
  return (p.nM + CM - 1) / CM * ((p.nN + CN - 1) / CN) * p.nslices;
}

template <int CS>
__device__ __forceinline__ TileWork tile_work(const TcParams& p, int t, int rm, int rn) {
  constexpr int CM = ClusterShape<CS>::CM, CN = ClusterShape<CS>::CN;
  TileWork w;
  const int nMg = (p.nM + CM - 1) / CM;
  const int per_slice = nMg * ((p.nN + CN - 1) / CN);
  w.slice = t / per_slice;
  const int rem = t - w.slice * per_slice;
  const int ng = rem / nMg;
  w.n = ng * CN + rn;
  w.m = (rem - ng * nMg) * CM + rm;
  w.list = p.kb_ptr ? (w.n * p.tn) / LIST_TILE : 0;
  w.m_len = p.kb_ptr ? (__ldg(p.kb_ptr + w.list + 1) - __ldg(p.kb_ptr + w.list)) << p.sub_shift
                     : p.kb_per_seg;
  const int nsteps = w.m_len * p.nseg;
  w.s0 = min(nsteps, w.slice * p.kb_per_slice);
  w.s1 = min(nsteps, w.s0 + p.kb_per_slice);
  return w;
}

template <int STAGES, int BOXES, int TN, bool FUSED = false, int CS = 1>
__global__ void __launch_bounds__(NTHREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                   const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1,
                   const __grid_constant__ CUtensorMap tmZ, const TcParams p, const uint32_t idesc) {
  using namespace tc;
  constexpr int A_BYTES = TM * TK * 2;
  constexpr int B_BYTES = TN * TK * 2;
  constexpr int NPL = FUSED ? 2 : 1;         // operand planes per stage (hi, lo)
  constexpr int STAGE_BYTES = NPL * (A_BYTES + B_BYTES);
  constexpr int CHUNK = FUSED ? KB_PER_CHUNK_FUSED : KB_PER_CHUNK;
  constexpr int EPI_COLS = TN / 2;           // columns per epilogue thread
  constexpr uint32_t TMEM_COLS = 2 * TN;     // two accumulators
  // clusters: CTA (rm, rn) loads rows [rm TN/CM, (rm+1) TN/CM) of its B tile for the CM
  // CTAs of its cell tile and rows [rn TM/CN, (rn+1) TM/CN) of its A tile for the CN CTAs
  // of its frame tile, each multicast into the same stage of those CTAs
  constexpr int CM = ClusterShape<CS>::CM, CN = ClusterShape<CS>::CN;
  constexpr int B_SLICE_ROWS = TN / CM;
  constexpr uint32_t B_SLICE_BYTES = B_SLICE_ROWS * TK * 2;
  constexpr int A_SLICE_ROWS = TM / CN;
  constexpr uint32_t A_SLICE_BYTES = A_SLICE_ROWS * TK * 2;
  constexpr uint16_t CMASK = static_cast<uint16_t>((1u << CS) - 1u);
  static_assert(CS == 1 || CS == 2 || CS == 4, "cluster size");
  static_assert(B_SLICE_BYTES % 1024 == 0 && A_SLICE_BYTES % 1024 == 0,
                "slices must keep the 1024-byte swizzle atom");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // stage s: A planes at sA + s * NPL * A_BYTES, B planes at sB + s * NPL * B_BYTES
  const uint32_t sA = smem_u32(smem);
  const uint32_t sB = sA + STAGES * NPL * A_BYTES;
  uint8_t* out_smem = smem + STAGES * STAGE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(out_smem + NEPI * BOXES * OUT_BOX);
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + 2 + a); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), CS);  // freed by the MMA issuer of every CTA of the cluster
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 32 * NEPI);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  // the peers' multicast loads and MMA commits may target this CTA's barriers only once
  // they are initialised
  if constexpr (CS > 1) cluster_sync();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int total = tile_groups<CS>(p);
  const int crank = CS > 1 ? static_cast<int>(cluster_ctarank()) : 0;
  const int rm = crank % CM, rn = crank / CM;
  const int tile0 = CS > 1 ? static_cast<int>(cluster_id_x()) : static_cast<int>(blockIdx.x);
  const int tstep = CS > 1 ? static_cast<int>(cluster_count_x()) : static_cast<int>(gridDim.x);

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      // the CTAs sharing this CTA's B tile (same rn) and A tile (same rm)
      const uint16_t mask_b = static_cast<uint16_t>(((1u << CM) - 1u) << (rn * CM));
      uint16_t mask_a = 0;
#pragma unroll
      for (int j = 0; j < CN; ++j) mask_a |= static_cast<uint16_t>(1u << (rm + CM * j));
      prefetch_tmap(&tmA0);
      prefetch_tmap(&tmB0);
      if (p.nseg > 1) {
        prefetch_tmap(&tmA1);
        prefetch_tmap(&tmB1);
      }
      int stage = 0;
      uint32_t phase = 0;
      uint32_t filled = 0, filled_par = 0;  // per stage: loaded at least once, its parity
      bool ok = true;
      // p.stall (failure-detection test): no load is issued, so the MMA issuer's and the
      // epilogue's bounded waits run out and the CTA records the timeout
      for (int t = tile0; t < total && ok && !p.stall; t += tstep) {
        const TileWork w = tile_work<CS>(p, t, rm, rn);
        const int* list = p.kb_ptr ? p.kb_idx + __ldg(p.kb_ptr + w.list) : nullptr;
        for (int s = w.s0; s < w.s1; ++s) {
          const int seg = s / w.m_len;
          const int loc = s - seg * w.m_len;
          // first column of the k-step's 64-column window (from the list when block-sparse:
          // any multiple of 8, windows disjoint) and, for TF32, which 32-column half; the
          // load overlaps the wait
          const int c64 = list ? __ldg(list + (loc >> p.sub_shift)) : (loc >> p.sub_shift) * TK;
          const int kx = c64 + ((loc & ((1 << p.sub_shift) - 1)) << (6 - p.sub_shift));
          if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, abort_flag, 1, p.wait_ns)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(stage), STAGE_BYTES);
          if constexpr (FUSED) {
            const uint32_t a = sA + stage * 2 * A_BYTES, b = sB + stage * 2 * B_BYTES;
            if constexpr (CN > 1) {
              const uint32_t as = a + rn * A_SLICE_BYTES;
              const int y = w.m * TM + rn * A_SLICE_ROWS;
              tma_load_2d_mc(as, &tmA0, kx, y, full_bar(stage), mask_a);
              tma_load_2d_mc(as + A_BYTES, &tmA1, kx, y, full_bar(stage), mask_a);
            } else {
              tma_load_2d(a, &tmA0, kx, w.m * TM, full_bar(stage));
              tma_load_2d(a + A_BYTES, &tmA1, kx, w.m * TM, full_bar(stage));
            }
            if constexpr (CM > 1) {
              const uint32_t bs = b + rm * B_SLICE_BYTES;
              const int y = w.n * TN + rm * B_SLICE_ROWS;
              tma_load_2d_mc(bs, &tmB0, kx, y, full_bar(stage), mask_b);
              tma_load_2d_mc(bs + B_BYTES, &tmB1, kx, y, full_bar(stage), mask_b);
            } else {
              tma_load_2d(b, &tmB0, kx, w.n * TN, full_bar(stage));
              tma_load_2d(b + B_BYTES, &tmB1, kx, w.n * TN, full_bar(stage));
            }
          } else {
            const CUtensorMap* ta = seg == 2 ? &tmA1 : &tmA0;
            const CUtensorMap* tb = seg == 1 ? &tmB1 : &tmB0;
            if constexpr (CN > 1)
              tma_load_2d_mc(sA + stage * A_BYTES + rn * A_SLICE_BYTES, ta, kx,
                             w.m * TM + rn * A_SLICE_ROWS, full_bar(stage), mask_a);
            else
              tma_load_2d(sA + stage * A_BYTES, ta, kx, w.m * TM, full_bar(stage));
            if constexpr (CM > 1)
              tma_load_2d_mc(sB + stage * B_BYTES + rm * B_SLICE_BYTES, tb, kx,
                             w.n * TN + rm * B_SLICE_ROWS, full_bar(stage), mask_b);
            else
              tma_load_2d(sB + stage * B_BYTES, tb, kx, w.n * TN, full_bar(stage));
          }
          filled |= 1u << stage;
          filled_par = (filled_par & ~(1u << stage)) | (phase << stage);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {  // let this CTA's own loads in flight land before it exits
        volatile int dummy = 0;
        for (int s = 0; s < STAGES; ++s)
          if ((filled >> s) & 1u)
            mbar_wait_bounded(full_bar(s), (filled_par >> s) & 1u, &dummy, 1, p.wait_ns / 10);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int gc = 0;  // chunks issued by this CTA (selects the accumulator and its phase)
      for (int t = tile0; t < total && ok; t += tstep) {
        const TileWork w = tile_work<CS>(p, t, rm, rn);
        for (int c0 = w.s0; c0 < w.s1 && ok; c0 += CHUNK, ++gc) {
          const int acc = gc & 1;
          const uint32_t aph = static_cast<uint32_t>((gc >> 1) & 1);
          if (!mbar_wait_bounded(tempty_bar(acc), aph ^ 1u, abort_flag, 3, p.wait_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + static_cast<uint32_t>(acc * TN);
          const int c1 = min(w.s1, c0 + CHUNK);
          for (int s = c0; s < c1; ++s) {
            if (!mbar_wait_bounded(full_bar(stage), phase, abort_flag, 2, p.wait_ns)) {
              ok = false;
              break;
            }
            tc_fence_after();
            // FUSED: the products A_hi B_hi, A_hi B_lo, A_lo B_hi of this k-block in turn;
            // otherwise the stage's one pair
#pragma unroll
            for (int pr = 0; pr < (FUSED ? 3 : 1); ++pr) {
              const uint32_t a_off = (FUSED && pr == 2) ? A_BYTES : 0u;
              const uint32_t b_off = (FUSED && pr == 1) ? B_BYTES : 0u;
              const uint64_t ad = sdesc_k128(sA + stage * NPL * A_BYTES + a_off);
              const uint64_t bd = sdesc_k128(sB + stage * NPL * B_BYTES + b_off);
              // four MMAs per 128-byte k-step (K = 16 of 16-bit or K = 8 of TF32 each)
              if (p.tf32) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                  mma_tf32(d, ad + static_cast<uint64_t>((k * 32) >> 4),
                           bd + static_cast<uint64_t>((k * 32) >> 4), idesc,
                           (s > c0 || pr > 0 || k > 0) ? 1u : 0u);
              } else {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                  mma_f16(d, ad + static_cast<uint64_t>((k * 32) >> 4),
                          bd + static_cast<uint64_t>((k * 32) >> 4), idesc,
                          (s > c0 || pr > 0 || k > 0) ? 1u : 0u);
              }
            }
            if constexpr (CS > 1)
              mma_commit_mc(empty_bar(stage), CMASK);  // the stage is free in this CTA once
            else                                       // every CTA of the cluster consumed it
              mma_commit(empty_bar(stage));
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
          if (ok) mma_commit(tfull_bar(acc));
        }
      }
      // all MMAs this thread issued must finish before TMEM is released
      mma_commit(drain_bar);
      volatile int dummy = 0;
      mbar_wait_bounded(drain_bar, 0u, &dummy, 1, p.wait_ns);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..9)
    const int q = warp & 3;                 // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;       // which 128 of the 256 columns
    const uint32_t lane_off = static_cast<uint32_t>(q * 32) << 16;
    // BOXES boxes of 32 rows x 128 bytes, 128B-swizzled, owned by this warp
    uint8_t* boxes = out_smem + (warp - 2) * BOXES * OUT_BOX;
    int gc = 0;
    bool ok = true;
    for (int t = tile0; t < total && ok; t += tstep) {
      const TileWork w = tile_work<CS>(p, t, rm, rn);
      float sum[EPI_COLS];
#pragma unroll
      for (int j = 0; j < EPI_COLS; ++j) sum[j] = 0.f;
      for (int c0 = w.s0; c0 < w.s1; c0 += CHUNK, ++gc) {
        const int acc = gc & 1;
        const uint32_t aph = static_cast<uint32_t>((gc >> 1) & 1);
        const bool got = mbar_wait_bounded(tfull_bar(acc), aph, abort_flag, 4, p.wait_ns);
        if (!__all_sync(0xFFFFFFFFu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t col0 = tmem_base + static_cast<uint32_t>(acc * TN + half * EPI_COLS) + lane_off;
#pragma unroll
        for (int c = 0; c < EPI_COLS; c += 16) {
          uint32_t r[16];
          tmem_ld_32x32b_x16(col0 + static_cast<uint32_t>(c), r);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[c + j] += __uint_as_float(r[j]);
        }
        tc_fence_before();
        mbar_arrive(tempty_bar(acc));
      }
      if (!ok) break;
      const int f0 = w.m * TM + q * 32;  // first frame row of this warp
      const int f = f0 + lane;
      const int n0 = w.n * TN + half * EPI_COLS;
      if (p.nslices == 1) {
        float bv = -INFINITY;
        int bi = -1;
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j)
          if (n0 + j < p.J && (bi < 0 || sum[j] > bv)) {
            bv = sum[j];
            bi = n0 + j;
          }
        if (f < p.F && bi >= 0) atomicMax(p.keys + f, argmax_key(bv, p.col0 + bi));
      }
      if (!p.Z) continue;  // estimates only: the argmax is all that leaves
      if (p.tma_out) {
        // 32x32 boxes: row = lane, 16-byte chunk c4 stored at chunk c4 ^ (lane & 7) (the
        // tensor map's 128-byte swizzle), so the eight lanes of each store phase hit
        // distinct banks.  Rows >= F and columns >= J are clipped by the TMA unit.
#pragma unroll
        for (int b = 0; b < EPI_COLS / 32; ++b) {
          if (f0 >= p.F || n0 + b * 32 >= p.J) continue;  // box wholly outside the map
          uint8_t* box = boxes + (b % BOXES) * OUT_BOX;
          // the box's previous store must have read it: before a tile's first box, every
          // store of the previous tile; later, all but the BOXES - 1 newest stores
          if (lane == 0) {
            if (b == 0)
              bulk_wait_read<0>();
            else if (b >= BOXES)
              bulk_wait_read<BOXES - 1>();
          }
          __syncwarp();
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4) {
            float4* dst = reinterpret_cast<float4*>(box + lane * 128 + ((c4 ^ (lane & 7)) << 4));
            *dst = make_float4(sum[b * 32 + 4 * c4], sum[b * 32 + 4 * c4 + 1],
                               sum[b * 32 + 4 * c4 + 2], sum[b * 32 + 4 * c4 + 3]);
          }
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            tma_store_3d(&tmZ, smem_u32(box), n0 + b * 32, f0, w.slice);
            bulk_commit();
          }
        }
      } else if (f < p.F) {
        float* zrow = p.Z + (static_cast<size_t>(w.slice) * p.F + f) * p.ldz + n0;
#pragma unroll
        for (int j = 0; j < EPI_COLS; ++j)
          if (n0 + j < p.J) zrow[j] = sum[j];
      }
    }
    if (lane == 0) bulk_wait_all();
    __syncwarp();
  }
  tc_fence_before();
  __syncthreads();
  // no CTA leaves while a peer may still multicast into its shared memory or arrive on its
  // barriers: every CTA gets here after its MMAs (and with them its commits) completed
  if constexpr (CS > 1) cluster_sync();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem_base, TMEM_COLS);
  }
  if (threadIdx.x == 0 && *abort_flag) atomicExch(p.err, *abort_flag);
}

// ------------------------------------------------------------------------------------
namespace {
std::mutex g_enc_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

cudaError_t get_encode() {
  std::lock_guard<std::mutex> lock(g_enc_mu);
  if (g_encode) return cudaSuccess;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return cudaSuccess;
}

// 2-D K-major operand map over [rows][Kd] elements of ebytes (2 or 4), box of one 128-byte
// k-step (64 or 32 elements) x box_rows, 128-byte swizzle; out-of-range rows read as zero.
cudaError_t make_operand_map(CUtensorMap* m, const void* base, CUtensorMapDataType dt, uint64_t Kd,
                             uint64_t rows, uint32_t box_rows, uint32_t ebytes) {
  cuuint64_t dims[2] = {Kd, rows};
  cuuint64_t strides[1] = {Kd * ebytes};
  cuuint32_t box[2] = {128u / ebytes, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 3-D FP32 output map over [slices][F][J] with rows ld floats apart, box 32 x 32 x 1,
// 128-byte swizzle.
cudaError_t make_output_map(CUtensorMap* m, float* base, uint64_t J, uint64_t F, uint64_t slices,
                            uint64_t ld) {
  cuuint64_t dims[3] = {J, F, slices};
  cuuint64_t strides[2] = {ld * 4, ld * F * 4};
  cuuint32_t box[3] = {32, 32, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}
}  // namespace

// Reduction slices for F frames (dense operands): 1 while the output tiles fill the GPU;
// otherwise enough slices (of at least MIN_KB_PER_SLICE k-blocks) to give every SM a tile.
// k-steps of a dense reduction over Kd columns in operand type t, all segments
static int ksteps_of(int Kd, OpType t) { return Kd / TK * op_kb_per64(t) * (op_split(t) ? 3 : 1); }

static int slices_for(int F, int J, int Kd, OpType t, int num_sms, int tn) {
  if (F <= 0) return 1;
  const long long tiles = static_cast<long long>((F + TM - 1) / TM) * ((J + tn - 1) / tn);
  if (tiles >= num_sms) return 1;
  const int kb_total = ksteps_of(Kd, t);
  const long long want = (num_sms + tiles - 1) / tiles;
  const int cap = kb_total / MIN_KB_PER_SLICE > 1 ? kb_total / MIN_KB_PER_SLICE : 1;
  return static_cast<int>(want < cap ? want : cap);
}

int tc_gemm_slices(int F, int J, int Kd, OpType t, int num_sms) {
  return slices_for(F, J, Kd, t, num_sms, 256);
}

size_t tc_gemm_workspace_floats(int F_max, int J, int Kd, OpType t, int num_sms) {
  size_t need = 0;  // the 256-cell variants need the most slices
  for (int F = 1; F <= F_max; ++F) {
    const int ns = slices_for(F, J, Kd, t, num_sms, 256);
    if (ns > 1) need = std::max(need, static_cast<size_t>(ns) * F * static_cast<size_t>(J));
  }
  return need;
}

namespace {
template <int STAGES, int BOXES, int TN, bool FUSED = false, int CS = 1>
cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(tc_gemm_kernel<STAGES, BOXES, TN, FUSED, CS>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_bytes<STAGES, BOXES, TN, FUSED>());
}

// Clusters of the variant that can be resident at once on the current device (queried at
// plan creation and cached per device, so that a captured launch needs no query).
constexpr int kMaxDevices = 64;
std::mutex g_cl_mu;
int g_max_clusters[kMaxDevices][TC_NVARIANTS] = {};

template <int STAGES, int BOXES, int TN, bool FUSED, int CS>
cudaError_t query_clusters(int variant) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if ((e = set_smem_attr<STAGES, BOXES, TN, FUSED, CS>()) != cudaSuccess) return e;
  if (CS == 1) return cudaSuccess;
  {
    std::lock_guard<std::mutex> lock(g_cl_mu);
    if (g_max_clusters[dev][variant] > 0) return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(CS);
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = smem_bytes<STAGES, BOXES, TN, FUSED>();
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, tc_gemm_kernel<STAGES, BOXES, TN, FUSED, CS>, &cfg);
  if (e != cudaSuccess) return e;
  if (n < 1) return cudaErrorInvalidConfiguration;
  std::lock_guard<std::mutex> lock(g_cl_mu);
  g_max_clusters[dev][variant] = n;
  return cudaSuccess;
}

int max_clusters(int variant) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  std::lock_guard<std::mutex> lock(g_cl_mu);
  return g_max_clusters[dev][variant];
}

// Launches one variant: a plain persistent grid of `ctas` CTAs, or (CS > 1) `ctas` CTAs in
// clusters of CS.
template <int STAGES, int BOXES, int TN, bool FUSED, int CS>
cudaError_t launch_variant(int ctas, const CUtensorMap& mA0, const CUtensorMap& mA1,
                           const CUtensorMap& mB0, const CUtensorMap& mB1, const CUtensorMap& mZ,
                           const TcParams& p, uint32_t idesc, cudaStream_t s) {
  cudaError_t e = set_smem_attr<STAGES, BOXES, TN, FUSED, CS>();
  if (e != cudaSuccess) return e;
  constexpr int smem = smem_bytes<STAGES, BOXES, TN, FUSED>();
  if constexpr (CS == 1) {
    tc_gemm_kernel<STAGES, BOXES, TN, FUSED, 1><<<ctas, NTHREADS, smem, s>>>(mA0, mA1, mB0, mB1, mZ, p, idesc);
    return cudaGetLastError();
  } else {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, tc_gemm_kernel<STAGES, BOXES, TN, FUSED, CS>, mA0, mA1, mB0,
                              mB1, mZ, p, idesc);
  }
}

template <int CS>
cudaError_t prepare_cs() {
  constexpr int c = CS == 1 ? 0 : CS == 2 ? 1 : 2;
  cudaError_t e;
  if ((e = query_clusters<4, 1, 256, false, CS>(TC_LONG_256 + TC_NBASE * c)) != cudaSuccess) return e;
  if ((e = query_clusters<2, 4, 256, false, CS>(TC_SHORT_256 + TC_NBASE * c)) != cudaSuccess) return e;
  if ((e = query_clusters<2, 1, 256, true, CS>(TC_FUSED3_256 + TC_NBASE * c)) != cudaSuccess) return e;
  return query_clusters<4, 2, 128, false, CS>(TC_LONG_128 + TC_NBASE * c);
}

template <int CS>
cudaError_t launch_base(int base, int ctas, const CUtensorMap& mA0, const CUtensorMap& mA1,
                        const CUtensorMap& mB0, const CUtensorMap& mB1, const CUtensorMap& mZ,
                        const TcParams& p, uint32_t idesc, cudaStream_t s) {
  switch (base) {
    case TC_SHORT_256:
      return launch_variant<2, 4, 256, false, CS>(ctas, mA0, mA1, mB0, mB1, mZ, p, idesc, s);
    case TC_LONG_128:
      return launch_variant<4, 2, 128, false, CS>(ctas, mA0, mA1, mB0, mB1, mZ, p, idesc, s);
    case TC_FUSED3_256:
      return launch_variant<2, 1, 256, true, CS>(ctas, mA0, mA1, mB0, mB1, mZ, p, idesc, s);
    default:
      return launch_variant<4, 1, 256, false, CS>(ctas, mA0, mA1, mB0, mB1, mZ, p, idesc, s);
  }
}
}  // namespace

int tc_gemm_cluster_size(int variant) {
  return variant >= 2 * TC_NBASE ? 4 : variant >= TC_NBASE ? 2 : 1;
}

cudaError_t tc_gemm_prepare() {
  cudaError_t e = get_encode();
  if (e != cudaSuccess) return e;
  if ((e = prepare_cs<1>()) != cudaSuccess) return e;
  if ((e = prepare_cs<2>()) != cudaSuccess) return e;
  return prepare_cs<4>();
}

bool tc_gemm_variant_valid(int variant, OpType t) {
  return variant >= 0 && variant < TC_NVARIANTS &&
         (variant % TC_NBASE != TC_FUSED3_256 || op_split(t));
}

int tc_gemm_cell_tile() { return LIST_TILE; }
int tc_gemm_k_block() { return TK; }

int tc_gemm_default_variant(int Kd, OpType t, int F) {
  const int steps = ksteps_of(Kd, t);
  const bool split = op_split(t);
  // short reductions: 2 stages and 4 output boxes; long ones: 4 stages, or for the hi + lo
  // precisions both planes per stage (uca8 conv 6.01 against 6.06 ms, walls16 32.3 / 36.0)
  const int base = steps <= SHORT_MAX_STEPS ? TC_SHORT_256 : split ? TC_FUSED3_256 : TC_LONG_256;
  if (F < 2 * TM) return base;  // one frame tile: nothing to pair
  // frame operands far beyond L2 (nested32 conv: 2 GB) are re-read from DRAM by every cell
  // tile's CTAs unless clusters share them: 2 x 2 (BF16 1131 -> 720 ms, FP16 hi+lo 2989 ->
  // 1397 ms); otherwise clusters of two for the hi + lo and the short reductions (uca8 conv
  // 6.01 -> 5.89 ms, SLRI 0.148 -> 0.147), none for long single-plane ones (walls16 BF16
  // conv 10.48 alone, 10.72 in pairs)
  const double a_bytes = static_cast<double>(F) * Kd * op_bytes(t) * (split ? 2 : 1);
  if (steps > SHORT_MAX_STEPS && a_bytes >= 1e9) return base + 2 * TC_NBASE;
  return (split || steps <= SHORT_MAX_STEPS) ? base + TC_NBASE : base;
}

cudaError_t launch_tc_gemm(const TcGemm& g, int num_sms, cudaStream_t s) {
  if (g.F <= 0) return cudaSuccess;
  if (g.Kd % TK != 0 || g.Kd <= 0) return cudaErrorInvalidValue;
  cudaError_t e = get_encode();
  if (e != cudaSuccess) return e;
  const int variant = g.variant >= 0 ? g.variant : tc_gemm_default_variant(g.Kd, g.t, g.F);
  if (!tc_gemm_variant_valid(variant, g.t)) return cudaErrorInvalidValue;
  const int base = variant % TC_NBASE;
  const bool fused = base == TC_FUSED3_256;
  const int tn = base == TC_LONG_128 ? 128 : 256;
  if (g.t == OpType::F32) return cudaErrorInvalidValue;
  const bool split3 = op_split(g.t);
  const bool tf32 = op_tf32(g.t);
  const bool bf16 = g.t == OpType::BF16 || g.t == OpType::BF16X2;
  const CUtensorMapDataType dt = tf32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                        : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const uint32_t eb = tf32 ? 4u : 2u;
  TcParams p;
  p.F = g.F;
  p.J = g.J;
  p.tn = tn;
  p.sub_shift = tf32 ? 1 : 0;
  p.tf32 = tf32 ? 1 : 0;
  p.stall = g.stall ? 1 : 0;
  p.wait_ns = g.stall ? STALL_WAIT_NS : WAIT_NS;
  p.kb_per_seg = (g.Kd / TK) << p.sub_shift;
  p.nseg = (split3 && !fused) ? 3 : 1;  // FUSED: one pass, the three products per k-block
  p.kb_ptr = g.kb_ptr;
  p.kb_idx = g.kb_idx;
  p.nM = (g.F + TM - 1) / TM;
  p.nN = (g.J + tn - 1) / tn;
  p.nslices = (g.kb_ptr || g.no_split) ? 1
              : g.force_slices > 0 ? g.force_slices
                                   : slices_for(g.F, g.J, g.Kd, g.t, num_sms, tn);
  // clusters share the B tiles of the frame tiles of one cell tile (and, 2 x 2, the A tiles
  // of the cell tiles of one frame tile: dense reductions only, whose k-steps are the same
  // for every cell tile); a single frame tile runs unclustered (its partner would only
  // compute zero rows), a single cell tile or a block-sparse reduction in clusters of 2 x 1
  int cs = p.nM < 2 ? 1 : tc_gemm_cluster_size(variant);
  if (cs == 4 && (g.kb_ptr || p.nN < 2)) cs = 2;
  const int max_cl = cs > 1 ? max_clusters(base + TC_NBASE * (cs == 2 ? 1 : 2)) : 0;
  if (cs > 1 && max_cl < 1) return cudaErrorNotReady;  // tc_gemm_prepare() did not run here
  CUtensorMap mA0, mA1, mB0, mB1, mZ;
  // each CTA loads its slice of B (1/CM of the rows) and of A (1/CN)
  const uint32_t b_rows = static_cast<uint32_t>(tn / (cs == 1 ? 1 : 2));
  const uint32_t a_rows = static_cast<uint32_t>(TM / (cs == 4 ? 2 : 1));
  if ((e = make_operand_map(&mA0, g.A, dt, g.Kd, g.F, a_rows, eb)) != cudaSuccess) return e;
  if ((e = make_operand_map(&mB0, g.B, dt, g.Kd, g.J, b_rows, eb)) != cudaSuccess) return e;
  if (split3) {
    if ((e = make_operand_map(&mA1, g.A_lo, dt, g.Kd, g.F, a_rows, eb)) != cudaSuccess) return e;
    if ((e = make_operand_map(&mB1, g.B_lo, dt, g.Kd, g.J, b_rows, eb)) != cudaSuccess) return e;
  } else {
    mA1 = mA0;
    mB1 = mB0;
  }
  p.col0 = g.col0;
  const int kb_total = p.kb_per_seg * p.nseg;
  if (p.nslices > 1) {
    p.kb_per_slice = (kb_total + p.nslices - 1) / p.nslices;
    p.nslices = (kb_total + p.kb_per_slice - 1) / p.kb_per_slice;
  } else {
    p.kb_per_slice = 1 << 30;
  }
  p.keys = g.keys;
  p.err = g.err;
  if (p.nslices > 1) {  // partial maps [nslices][F][J] in the workspace, summed afterwards
    if (!g.split_ws) return cudaErrorInvalidValue;
    p.Z = g.split_ws;
    p.ldz = g.J;
  } else {
    p.Z = g.Z;
    p.ldz = g.ldz ? g.ldz : g.J;
  }
  // TMA output needs 16-byte row strides and a 16-byte aligned base.
  p.tma_out = p.Z && (p.ldz % 4 == 0) && (reinterpret_cast<uintptr_t>(p.Z) % 16 == 0);
  if (p.tma_out) {
    if ((e = make_output_map(&mZ, p.Z, g.J, g.F, p.nslices, p.ldz)) != cudaSuccess) return e;
  } else {
    mZ = mA0;  // unused
  }
  const uint32_t idesc = tc::idesc_f16(tf32 ? 2u : bf16 ? 1u : 0u, TM, tn);
  if (cs == 1) {
    const int total = p.nM * p.nN * p.nslices;
    int grid = total < num_sms ? total : num_sms;
    if (g.max_ctas > 0 && grid > g.max_ctas) grid = g.max_ctas;
    e = launch_base<1>(base, grid, mA0, mA1, mB0, mB1, mZ, p, idesc, s);
  } else {
    // persistent clusters: no more than can be resident at once, nor than tile groups
    const int cm = 2, cn = cs == 4 ? 2 : 1;
    const int groups = (p.nM + cm - 1) / cm * ((p.nN + cn - 1) / cn) * p.nslices;
    int ncl = groups < max_cl ? groups : max_cl;
    if (g.max_ctas > 0 && ncl > g.max_ctas / cs) ncl = g.max_ctas / cs > 0 ? g.max_ctas / cs : 1;
    e = cs == 2 ? launch_base<2>(base, ncl * cs, mA0, mA1, mB0, mB1, mZ, p, idesc, s)
                : launch_base<4>(base, ncl * cs, mA0, mA1, mB0, mB1, mZ, p, idesc, s);
  }
  if (e != cudaSuccess || p.nslices == 1) return e;
  return launch_split_reduce(g.split_ws, p.nslices, g.Z, g.keys, g.F, g.J, s, g.ldz, g.col0);
}

}  // namespace srp
