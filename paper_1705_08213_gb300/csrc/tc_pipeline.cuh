// Persistent tcgen05 GEMM pipeline shared by the 2-way and 3-way tally kernels.
//
// One CTA per SM, 64 + 32 EW threads:
//   warp 0      TMA producer: a 4-stage ring of 128 x 128-byte A tiles and
//               256 x 128-byte B tiles (K-major, 128-byte swizzle);
//   warp 1      allocates 512 TMEM columns; one thread issues
//               tcgen05.mma.kind::f8f6f4 (M = 128, N = 256, K = 32) into one of
//               two 256-column FP32 accumulators;
//   warps 2..   epilogue, EW = 4 or 8 warps: EW/4 warps per 32-lane quarter of
//               the finished accumulator (warp w may only read lanes
//               32 (w % 4) .. +31), each draining 4 EW... of the 256 columns with
//               tcgen05.ld for Epi.  Eight warps pay off when a tile's K loop is
//               short and the epilogue would otherwise not hide behind the MMAs.
// The scheduler type Sched enumerates the CTA's tiles (b, b + gridDim.x, ...)
// and gives each tile's A and B row offsets; the three roles walk the same
// sequence independently.  Every mbarrier wait is bounded.
#pragma once

#include "ccc_dev.cuh"

namespace ccc {
namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 128;
constexpr int UK = 32;  // K of one kind::f8f6f4 MMA
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK;
constexpr int B_BYTES = BN * BK;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int ACC_COLS = BN;
constexpr int TMEM_COLS = 2 * ACC_COLS;
constexpr int CHUNKS = BN / 32;  // 32-column chunks of an accumulator
constexpr int MAX_THREADS = 64 + 32 * 8;
template <int EW>
struct Epilogue {
  static_assert(EW == 4 || EW == 8, "4 or 8 epilogue warps");
  static constexpr int THREADS = 32 * EW;
  static constexpr int CHUNKS_PER_WARP = CHUNKS / (EW / 4);
};
// Epilogue warps for a tile of nkb K stages: 4 when the K loop is long enough
// to hide the epilogue, else 8.
inline int epilogue_warps(int nkb) { return nkb >= 96 ? 4 : 8; }
constexpr int NUM_BARS = 2 * STAGES + 5;
constexpr uint32_t IDESC = idesc_e4m3_f32(BM, BN);
constexpr size_t SMEM_BYTES = 1024 + static_cast<size_t>(STAGES) * STAGE_BYTES + NUM_BARS * 8 + 64;

static_assert(TMEM_COLS == 512, "two 256-column accumulators fill TMEM");
static_assert(SMEM_BYTES <= 232448, "dynamic shared memory limit");

// Sched requirements:
//   struct Sched { struct Params; __device__ void init(const Params&, int64_t start);
//                  __device__ void advance(int64_t step); bool valid;
//                  __device__ int a_row() const; __device__ int b_row() const;
//                  __device__ int map_index() const;   // which tensor-map pair
//                  __device__ int k_blocks(int nkb) const; };  // K stages of the tile
// Epi requirements:
//   struct Epi { struct Params;
//     template <int NC> __device__ static void tile(const Params&, const Sched&, int quarter,
//                          int lane, uint32_t t_base, uint32_t release_bar, int c0); };
//   Epi::tile<NC> must tcgen05.ld the 32-column chunks c0 .. c0 + NC - 1 of its
//   lane quarter (columns t_base + 32 c) and, after its last load, fence and
//   arrive on release_bar.
template <class Sched, class Epi, int EW>
__device__ __forceinline__ void persistent_gemm(const CUtensorMap *tmA, const CUtensorMap *tmB,
                                                const typename Sched::Params &sp,
                                                const typename Epi::Params &ep, int nkb,
                                                int32_t *status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t *smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * A_BYTES;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + STAGES * B_BYTES);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + NUM_BARS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * STAGES + 2 + a); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), Epilogue<EW>::THREADS);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(tmA);
    tma_prefetch_desc(tmB);
  }
  // tmA / tmB point at arrays of tensor maps; a tile uses entry sc.map_index().
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int stage = 0;
      uint32_t phase = 0;
      int last_parity[STAGES];
      for (int s = 0; s < STAGES; ++s) last_parity[s] = -1;
      bool ok = true;
      Sched sc;
      for (sc.init(sp, blockIdx.x); sc.valid && ok; sc.advance(gridDim.x)) {
        const int ya = sc.a_row();
        const int yb = sc.b_row();
        const CUtensorMap *ma = tmA + sc.map_index();
        const CUtensorMap *mb = tmB + sc.map_index();
        const int kbs = sc.k_blocks(nkb);
        for (int kb = 0; kb < kbs; ++kb) {
          if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, status, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(stage), STAGE_BYTES);
          tma_load_2d(smem_u32(sA + stage * A_BYTES), ma, kb * BK, ya, full_bar(stage));
          tma_load_2d(smem_u32(sB + stage * B_BYTES), mb, kb * BK, yb, full_bar(stage));
          last_parity[stage] = static_cast<int>(phase);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        // Let the copies already issued land before the CTA's memory goes away.
        for (int s = 0; s < STAGES; ++s)
          if (last_parity[s] >= 0)
            mbar_wait_timeout(full_bar(s), static_cast<uint32_t>(last_parity[s]));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int stage = 0;
      uint32_t phase = 0;
      int lt = 0;
      bool ok = true;
      Sched sc;
      for (sc.init(sp, blockIdx.x); sc.valid && ok; sc.advance(gridDim.x), ++lt) {
        const int acc = lt & 1;
        const uint32_t acc_phase = (lt >> 1) & 1;
        if (!mbar_wait_bounded(tempty_bar(acc), acc_phase ^ 1u, status, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * ACC_COLS;
        const int kbs = sc.k_blocks(nkb);
        for (int kb = 0; kb < kbs; ++kb) {
          if (!mbar_wait_bounded(full_bar(stage), phase, status, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + stage * A_BYTES);
          const uint32_t b0 = smem_u32(sB + stage * B_BYTES);
#pragma unroll
          for (int k = 0; k < BK / UK; ++k)
            mma_f8f6f4(d_tmem, smem_desc_sw128(a0 + k * UK), smem_desc_sw128(b0 + k * UK), IDESC,
                       (kb | k) != 0 ? 1u : 0u);
          mma_commit(empty_bar(stage));
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(tfull_bar(acc));
      }
      // All MMAs issued by this thread are complete once the drain barrier fires.
      mma_commit(drain_bar);
      mbar_wait_timeout(drain_bar, 0);
    }
  } else {
    // ---------------- epilogue
    const int quarter = warp & 3;
    constexpr int NC = Epilogue<EW>::CHUNKS_PER_WARP;
    const int c0 = ((warp - 2) >> 2) * NC;
    int lt = 0;
    Sched sc;
    for (sc.init(sp, blockIdx.x); sc.valid; sc.advance(gridDim.x), ++lt) {
      const int acc = lt & 1;
      const uint32_t acc_phase = (lt >> 1) & 1;
      const bool ok = mbar_wait_bounded(tfull_bar(acc), acc_phase, status, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const uint32_t t_base =
          tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + acc * ACC_COLS;
      Epi::template tile<NC>(ep, sc, quarter, lane, t_base, tempty_bar(acc), c0);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

// Row-major 2-D uint8 tensor map over a [rows][kpad] operand matrix with a
// box of 128 bytes x box_rows and 128-byte swizzling (defined in k_tc2.cu).
bool make_operand_map(CUtensorMap *map, const uint8_t *op, int64_t rows, int64_t kpad,
                      uint32_t box_rows);
// The same tiles over an operand stored K-block-major, [kpad / 128][rows][128
// bytes]: a 3-D map (x = byte in the block, y = row, z = K block) whose box of
// 128 bytes x box_rows is one contiguous run (defined in k_tc2.cu).
bool make_blocked_operand_map(CUtensorMap *map, const uint8_t *op, int64_t rows, int64_t kpad,
                              uint32_t box_rows);

}  // namespace tc
}  // namespace ccc
