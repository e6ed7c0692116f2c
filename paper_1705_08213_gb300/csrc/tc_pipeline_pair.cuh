// Persistent tcgen05 GEMM pipeline on SM pairs (cta_group::2), used by the
// 2-way tally kernel.
//
// A cluster of two CTAs computes one 256 x 256 tile: CTA r (r = 0, 1) stages
// A rows [128 r, 128 r + 128) and B rows [128 r, 128 r + 128) of the tile,
// 16 KB each per 128-byte K stage; the leader (r = 0) issues
// tcgen05.mma.cta_group::2 (M = 256, N = 256, K = 32), which reads both CTAs'
// halves and leaves rows [128 r, 128 r + 128) x all 256 columns of the FP32
// accumulator in CTA r's TMEM.  Per SM and per MMA, shared memory holds and
// serves 8 KB of operands instead of 12 KB for a one-CTA 128 x 256 tile.
//
// Synchronisation:
//   full[s]    (leader)  the leader's producer expects both CTAs' bytes; both
//                        CTAs' TMA loads complete on it;
//   empty[s]   (both)    the MMA commit is multicast to both CTAs;
//   tfull[a]   (both)    likewise, when a tile's accumulator is final;
//   tempty[a]  (leader)  both CTAs' epilogue threads arrive (the follower's
//                        remotely) once they have read the accumulator.
// Every mbarrier wait is bounded; clusters synchronise after set-up and
// before the TMEM is released.
#pragma once

#include "ccc_dev.cuh"
#include "tc_pipeline.cuh"

namespace ccc {
namespace tcp {

constexpr int BMH = 128;  // A rows per CTA
constexpr int BNH = 128;  // B rows per CTA
constexpr int BK = 128;
constexpr int UK = 32;
constexpr int STAGES = 6;
constexpr int A_BYTES = BMH * BK;
constexpr int B_BYTES = BNH * BK;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // per CTA
constexpr int ACC_COLS = 256;
constexpr int TMEM_COLS = 512;
constexpr int NUM_BARS = 2 * STAGES + 5;
constexpr uint32_t IDESC = idesc_e4m3_f32(256, 256);
constexpr size_t SMEM_BYTES = 1024 + static_cast<size_t>(STAGES) * STAGE_BYTES + NUM_BARS * 8 + 64;
// Dynamic shared memory of a kernel whose epilogue warps each stage
// `stage_bytes` (Epi::STAGE_BYTES_PER_WARP) after the barriers.
constexpr size_t smem_bytes(int epi_warps, int stage_bytes) {
  return SMEM_BYTES + (stage_bytes > 0 ? 16 + static_cast<size_t>(epi_warps) * stage_bytes : 0);
}

static_assert(SMEM_BYTES <= 232448, "dynamic shared memory limit");

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Address, in the cluster shared window, of the same variable in CTA `rank`.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" :::
                   "memory");
}

// TMA load into this CTA's shared memory, completing on an mbarrier that may
// belong to the peer CTA (cluster address).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const void *tmap, int32_t x, int32_t y,
                                                 uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(bar_cluster)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc_pair(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish_pair() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void mma_f8f6f4_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                                uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive once on the barrier at this CTA-relative address in every CTA of mask
// when all prior tcgen05 operations of this thread complete.
__device__ __forceinline__ void mma_commit_pair(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}

// Sched: as for tc::persistent_gemm, in units of 256-row tiles; a_row/b_row
// give the first row of the tile (the CTA adds 128 r); map_index() selects the
// tile's tensor map in tm[]; the tile's K stages are k_begin() ..
// k_begin() + k_blocks(nkb) - 1.
// Epi: template <int NC> static void tile(const Params&, const Sched&, int rank,
//        int quarter, int lane, uint32_t t_base, uint32_t release_cluster_bar,
//        int c0, float *stage); the release arrives at a cluster address;
//        static constexpr int STAGE_BYTES_PER_WARP: shared memory each epilogue
//        warp may use at `stage` (the kernel is launched with
//        smem_bytes(EW, STAGE_BYTES_PER_WARP)).
template <class Sched, class Epi, int EW>
__device__ __forceinline__ void persistent_gemm_pair(const CUtensorMap *tm,
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
  float *const stage_base = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(tmem_slot) + 64 + 15) & ~static_cast<uintptr_t>(15));

  constexpr int EPI_THREADS = tc::Epilogue<EW>::THREADS;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
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
      mbar_init(tempty_bar(a), 2 * EPI_THREADS);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) tma_prefetch_desc(tm);
  if (warp == 1) {
    tmem_alloc_pair(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // the peer's barriers are initialised before any remote use
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t cstart = blockIdx.x >> 1;
  const int64_t cstep = gridDim.x >> 1;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs)
      int stage = 0;
      uint32_t phase = 0;
      int last_parity[STAGES];
      for (int s = 0; s < STAGES; ++s) last_parity[s] = -1;
      bool ok = true;
      Sched sc;
      for (sc.init(sp, cstart); sc.valid && ok; sc.advance(cstep)) {
        const int ya = sc.a_row() + BMH * static_cast<int>(rank);
        const int yb = sc.b_row() + BNH * static_cast<int>(rank);
        const CUtensorMap *m = tm + sc.map_index();
        const int kbs = sc.k_blocks(nkb);
        const int kb0 = sc.k_begin();
        for (int kb = 0; kb < kbs; ++kb) {
          if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, status, abort_flag)) {
            ok = false;
            break;
          }
          if (leader) mbar_arrive_expect_tx(full_bar(stage), 2 * STAGE_BYTES);
          const uint32_t fb = map_to_rank(full_bar(stage), 0);
          tma_load_2d_pair(smem_u32(sA + stage * A_BYTES), m, (kb0 + kb) * BK, ya, fb);
          tma_load_2d_pair(smem_u32(sB + stage * B_BYTES), m, (kb0 + kb) * BK, yb, fb);
          last_parity[stage] = static_cast<int>(phase);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        // Let the copies already issued land: the leader watches the barriers
        // they complete on; the follower, whose copies complete on the leader's
        // barriers, gives them a bounded grace period.
        if (leader) {
          for (int s = 0; s < STAGES; ++s)
            if (last_parity[s] >= 0)
              mbar_wait_timeout(full_bar(s), static_cast<uint32_t>(last_parity[s]));
        } else {
          const uint64_t t0 = global_timer_ns();
          while (global_timer_ns() - t0 < 1000000ull) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer (leader CTA)
      int stage = 0;
      uint32_t phase = 0;
      int lt = 0;
      bool ok = true;
      Sched sc;
      for (sc.init(sp, cstart); sc.valid && ok; sc.advance(cstep), ++lt) {
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
            mma_f8f6f4_pair(d_tmem, smem_desc_sw128(a0 + k * UK), smem_desc_sw128(b0 + k * UK),
                            IDESC, (kb | k) != 0 ? 1u : 0u);
          mma_commit_pair(empty_bar(stage), 0x3);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit_pair(tfull_bar(acc), 0x3);
      }
      mma_commit_pair(drain_bar, 0x1);
      mbar_wait_timeout(drain_bar, 0);
    }
  } else {
    // ---------------- epilogue (both CTAs)
    const int quarter = warp & 3;
    constexpr int NC = tc::Epilogue<EW>::CHUNKS_PER_WARP;
    const int c0 = ((warp - 2) >> 2) * NC;
    int lt = 0;
    Sched sc;
    for (sc.init(sp, cstart); sc.valid; sc.advance(cstep), ++lt) {
      const int acc = lt & 1;
      const uint32_t acc_phase = (lt >> 1) & 1;
      const bool ok = mbar_wait_bounded(tfull_bar(acc), acc_phase, status, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const uint32_t t_base =
          tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + acc * ACC_COLS;
      Epi::template tile<NC>(ep, sc, static_cast<int>(rank), quarter, lane, t_base,
                             map_to_rank(tempty_bar(acc), 0), c0,
                             stage_base + (warp - 2) * (Epi::STAGE_BYTES_PER_WARP / 4));
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync();  // no remote arrive or load is still aimed at either CTA
  tc_fence_after();
  if (warp == 1) tmem_dealloc_pair(tmem_base, TMEM_COLS);
}

}  // namespace tcp
}  // namespace ccc
