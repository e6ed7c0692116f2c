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
// FP4 (e2m1) operands, kind::mxf4 with UE8M0 scale factors per 32 elements,
// all 1.0: a 128-byte K stage holds 256 entries and one MMA takes K = 64.  The
// block-scaled MMA reads its scale factors from TMEM, and two 256-column
// accumulators already fill the 512 columns, so the FP4 pipeline keeps ONE
// accumulator (columns 0-255) and the scale factors of A and B in columns
// 256-271 and 272-287, written once per launch.  Its epilogue loads the whole
// accumulator into registers before releasing it (8 warps, 128 values each),
// so the next tile's MMAs wait only for that read, not for the stores.
constexpr uint32_t IDESC_FP4 = idesc_e2m1_f32(256, 256, true);
constexpr uint32_t SF_COL = 256;
constexpr uint32_t SF_ONE_UE8M0 = 0x7F7F7F7Fu;
constexpr int FP4_EW = 8;
constexpr size_t SMEM_BYTES = 1024 + static_cast<size_t>(STAGES) * STAGE_BYTES + NUM_BARS * 8 + 64;
// Dynamic shared memory of a kernel whose epilogue warps each stage
// `stage_bytes` (Epi::STAGE_BYTES_PER_WARP) after the barriers.
constexpr size_t smem_bytes(int epi_warps, int stage_bytes) {
  return SMEM_BYTES + (stage_bytes > 0 ? 16 + static_cast<size_t>(epi_warps) * stage_bytes : 0);
}
// The same for tiles of NB < 256 columns (B rows NB / 2 per CTA).
constexpr size_t smem_bytes_nb(int nb, int epi_warps, int stage_bytes) {
  return smem_bytes(epi_warps, stage_bytes) - static_cast<size_t>(STAGES) * (BNH - nb / 2) * BK;
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

// The same for a 3-D tensor map (an operand stored K-block-major).
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const void *tmap, int32_t x, int32_t y,
                                                 int32_t z, uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(bar_cluster)
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

// Block-scaled FP4: D[tmem] (+)= (A * SA) (B * SB)^T with E2M1 operands, K = 64
// per instruction.  kind::mxf4 takes one UE8M0 scale factor per 32 elements
// along K (scale_vec::2X: two per row and instruction), kind::mxf4nvf4 with
// scale_vec::4X one UE4M3 factor per 16 elements; the factors are read from
// TMEM at sfa (rows of A along lanes) and sfb (rows of B).
__device__ __forceinline__ void mma_mxf4_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                              uint32_t idesc, uint32_t sfa, uint32_t sfb,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %6, 0;\n"
      "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], "
      "p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_mxf4nvf4_pair(uint32_t d_tmem, uint64_t a_desc,
                                                  uint64_t b_desc, uint32_t idesc, uint32_t sfa,
                                                  uint32_t sfb, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %6, 0;\n"
      "tcgen05.mma.cta_group::2.kind::mxf4nvf4.block_scale.scale_vec::4X [%0], %1, %2, %3, [%4], "
      "[%5], p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(sfa), "r"(sfb), "r"(accumulate)
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
// KBLK: the operand is stored K-block-major, [nkb][rows][128 bytes], behind a
// 3-D tensor map (x = byte, y = row, z = K block), so that each 128-row box is
// one contiguous 16 KB run.
// FP4: e2m1 operands (kind::mxf4, unit scale factors), one accumulator, the
// epilogue's Epi::tile loading all of its chunks before its release arrive
// (EW must be FP4_EW).
// NB: accumulator columns of a tile (N of the MMA; B rows NB / 2 per CTA).
// Below 256 (FP4 only) two accumulators of NB columns and the scale factors
// fit in the 512 TMEM columns (at 0, NB and 2 NB), so the MMAs of a tile run
// while the epilogue reads the previous one, as for e4m3; B is then loaded
// through tm[1] (box NB / 2 rows) and A through tm[0], and Epi::tile is called
// with PRELOAD false and c0 = (warp's column half) x NC.
template <class Sched, class Epi, int EW, bool KBLK = false, bool FP4 = false, int NB = 256>
__device__ __forceinline__ void persistent_gemm_pair(const CUtensorMap *tm,
                                                     const typename Sched::Params &sp,
                                                     const typename Epi::Params &ep, int nkb,
                                                     int32_t *status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t *smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  constexpr int NBH = NB / 2;             // B rows per CTA
  constexpr int B_BYTES_T = NBH * BK;     // B bytes per CTA and K stage
  constexpr int STAGE_BYTES_T = A_BYTES + B_BYTES_T;
  constexpr int NACC = FP4 && NB == 256 ? 1 : 2;  // accumulator buffers
  constexpr uint32_t SF_T = NACC == 1 ? SF_COL : 2u * NB;  // FP4 scale-factor columns
  static_assert(NB == 256 || (FP4 && !KBLK && NB % 16 == 0 && NB >= 128 &&
                              SF_T + 32 <= static_cast<uint32_t>(TMEM_COLS)),
                "narrow tiles: FP4, two accumulators and the scale factors in TMEM");
  static_assert(B_BYTES_T % 1024 == 0, "B stages on 1024-byte boundaries (128-byte swizzle)");
  constexpr uint32_t IDESC_T = FP4 ? idesc_e2m1_f32(256, NB, true) : IDESC;
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * A_BYTES;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + STAGES * B_BYTES_T);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + NUM_BARS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  float *const stage_base = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(tmem_slot) + 64 + 15) & ~static_cast<uintptr_t>(15));

  constexpr int EPI_THREADS = tc::Epilogue<EW>::THREADS;
  static_assert(!FP4 || EW == FP4_EW, "the FP4 epilogue holds 4 chunks per thread");
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
  if (FP4) {
    // Scale factors 1.0 in both CTAs' columns SF_T .. SF_T + 31 (every
    // byte), written by the first four epilogue warps, one lane quarter each,
    // before the leader's first MMA reads them.
    if (warp >= 2 && warp < 6) {
      uint32_t v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = SF_ONE_UE8M0;
      tmem_st_32x32b_x32(tmem_base + (static_cast<uint32_t>((warp & 3) * 32) << 16) + SF_T, v);
      tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
  }

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
        const int yb = sc.b_row() + NBH * static_cast<int>(rank);
        const CUtensorMap *m = tm + sc.map_index();
        const CUtensorMap *mb = NB == 256 ? m : tm + 1;
        const int kbs = sc.k_blocks(nkb);
        const int kb0 = sc.k_begin();
        for (int kb = 0; kb < kbs; ++kb) {
          if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, status, abort_flag)) {
            ok = false;
            break;
          }
          if (leader) mbar_arrive_expect_tx(full_bar(stage), 2 * STAGE_BYTES_T);
          const uint32_t fb = map_to_rank(full_bar(stage), 0);
          if (KBLK) {
            tma_load_3d_pair(smem_u32(sA + stage * A_BYTES), m, 0, ya, kb0 + kb, fb);
            tma_load_3d_pair(smem_u32(sB + stage * B_BYTES_T), m, 0, yb, kb0 + kb, fb);
          } else {
            tma_load_2d_pair(smem_u32(sA + stage * A_BYTES), m, (kb0 + kb) * BK, ya, fb);
            tma_load_2d_pair(smem_u32(sB + stage * B_BYTES_T), mb, (kb0 + kb) * BK, yb, fb);
          }
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
        const int acc = NACC == 1 ? 0 : (lt & 1);
        const uint32_t acc_phase = NACC == 1 ? (lt & 1) : ((lt >> 1) & 1);
        if (!mbar_wait_bounded(tempty_bar(acc), acc_phase ^ 1u, status, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * NB;
        const int kbs = sc.k_blocks(nkb);
        for (int kb = 0; kb < kbs; ++kb) {
          if (!mbar_wait_bounded(full_bar(stage), phase, status, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + stage * A_BYTES);
          const uint32_t b0 = smem_u32(sB + stage * B_BYTES_T);
#pragma unroll
          for (int k = 0; k < BK / UK; ++k) {
            if (FP4)
              mma_mxf4_pair(d_tmem, smem_desc_sw128(a0 + k * UK), smem_desc_sw128(b0 + k * UK),
                            IDESC_T, tmem_base + SF_T, tmem_base + SF_T + 16,
                            (kb | k) != 0 ? 1u : 0u);
            else
              mma_f8f6f4_pair(d_tmem, smem_desc_sw128(a0 + k * UK), smem_desc_sw128(b0 + k * UK),
                              IDESC, (kb | k) != 0 ? 1u : 0u);
          }
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
      const int acc = NACC == 1 ? 0 : (lt & 1);
      const uint32_t acc_phase = NACC == 1 ? (lt & 1) : ((lt >> 1) & 1);
      const bool ok = mbar_wait_bounded(tfull_bar(acc), acc_phase, status, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const uint32_t t_base = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + acc * NB;
      Epi::template tile<NC, NACC == 1>(ep, sc, static_cast<int>(rank), quarter, lane, t_base,
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

// ---------------------------------------------------------------- packed operands
//
// The same SM-pair GEMM with the operand preparation fused in (the unpack of
// Sec. 3.1 done in shared memory).  TMA brings the 2-bit genotype codes of the
// tile's SNPs, 64 SNPs x 128 entries = 2 KB per operand, CTA and K stage, into
// a ring of packed stages; CW converter warps expand them into the e4m3 count
// rows rho(0), rho(1) in the 128-byte-swizzled K-major layout a TMA load of
// those rows would have written, mask entries past n_f and SNPs past n_v,
// fence the writes for the async proxy and arrive on the leader's conv[]
// barrier.  No operand matrix exists in HBM; the kernel reads 1/8 of its bytes.
// The converter warps form TEAMS teams that take the K stages in turn, so that
// several stages are converted at once.
//   pfull[p]   (both)    the CTA's packed TMA loads complete on it;
//   pempty[p]  (both)    the converting team's warps arrive once they have read it
//                        (one team of WPT warps converts each K stage);
//   lconv[o]   (both)    the converting team's warps arrive (CTA scope) once
//                        operand stage o is written and fenced;
//   rconv[o]   (leader)  the follower's relay thread (its idle MMA warp)
//                        arrives, at cluster scope, once the follower's lconv[o]
//                        completed; the MMA waits on lconv[o] and rconv[o];
//   oempty[o]  (both)    the MMA commit is multicast: operand stage o is free;
//   tfull, tempty, drain as above.
namespace pk {
constexpr int OP_STAGES = 5;
constexpr int P_STAGES = 8;
constexpr int CW = 8;                          // converter warps
constexpr int TEAMS = 4;                       // teams taking the K stages in turn
constexpr int WPT = CW / TEAMS;                // warps per team
constexpr int SNPS = BMH / 2;                  // SNPs per CTA and operand
constexpr int P_SIDE_BYTES = SNPS * (BK / 4);  // 32 bytes of codes per SNP and K stage
constexpr int P_BYTES = 2 * P_SIDE_BYTES;
constexpr int NUM_BARS = 2 * P_STAGES + 3 * OP_STAGES + 5;
constexpr size_t SMEM_BYTES = 1024 + static_cast<size_t>(OP_STAGES) * STAGE_BYTES +
                              static_cast<size_t>(P_STAGES) * P_BYTES + NUM_BARS * 8 + 64;
constexpr size_t smem_bytes(int epi_warps, int stage_bytes) {
  return SMEM_BYTES + (stage_bytes > 0 ? 16 + static_cast<size_t>(epi_warps) * stage_bytes : 0);
}
static_assert(A_BYTES == B_BYTES, "one operand stage size");
static_assert((2 * SNPS * (BK / 16)) % (WPT * 32) == 0, "converter tasks per stage");

// e4m3 rho(0) and rho(1) indexed by code: 00 -> (2, 0), 01 -> (1, 1),
// 10 (missing) -> (0, 0), 11 -> (0, 2); 1.0 = 0x38, 2.0 = 0x40.
constexpr uint32_t kRho0 = 0x00003840u;
constexpr uint32_t kRho1 = 0x40003800u;

__device__ __forceinline__ bool try_wait_acq_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      "selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// mbar_wait_bounded with cluster-scope acquire (arrivals from the peer CTA
// release writes to its shared memory that the MMA then reads).
__device__ __forceinline__ bool wait_bounded_cluster(uint32_t bar, uint32_t parity,
                                                     int32_t *status, volatile int *abort_flag) {
  if (try_wait_acq_cluster(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  uint32_t spins = 0;
  while (true) {
    if (try_wait_acq_cluster(bar, parity)) return true;
    if (((++spins) & 63u) == 0) {
      if (*abort_flag) return false;
      if (global_timer_ns() - t0 > 2000000000ull) {
        record_error(status, CCC_ETIMEOUT);
        *abort_flag = 1;
        return false;
      }
    }
  }
}
}  // namespace pk

// tmP: tensor map over the packed panel (uint64 words [n_v][ld], box 4 words x
// 64 SNPs, no swizzle).  Sched and Epi as for persistent_gemm_pair; the kernel
// runs 64 + 32 EW + 32 CW threads with pk::smem_bytes(EW, Epi::STAGE_BYTES_PER_WARP).
template <class Sched, class Epi, int EW>
__device__ __forceinline__ void persistent_gemm_pair_packed(const CUtensorMap *tmP,
                                                            const typename Sched::Params &sp,
                                                            const typename Epi::Params &ep,
                                                            int nkb, int64_t n_v, int64_t n_f,
                                                            int32_t *status) {
  using pk::OP_STAGES;
  using pk::TEAMS;
  using pk::WPT;
  using pk::P_BYTES;
  using pk::P_SIDE_BYTES;
  using pk::P_STAGES;
  using pk::SNPS;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t *smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t *sA = smem;
  uint8_t *sB = smem + OP_STAGES * A_BYTES;
  uint8_t *sP = sB + OP_STAGES * B_BYTES;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sP + P_STAGES * P_BYTES);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + pk::NUM_BARS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  float *const stage_base = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(tmem_slot) + 64 + 15) & ~static_cast<uintptr_t>(15));

  constexpr int EPI_THREADS = tc::Epilogue<EW>::THREADS;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint32_t bar0 = smem_u32(bars);
  auto pfull_bar = [&](int p) { return bar0 + 8u * p; };
  auto pempty_bar = [&](int p) { return bar0 + 8u * (P_STAGES + p); };
  auto lconv_bar = [&](int o) { return bar0 + 8u * (2 * P_STAGES + o); };
  auto rconv_bar = [&](int o) { return bar0 + 8u * (2 * P_STAGES + OP_STAGES + o); };
  auto oempty_bar = [&](int o) { return bar0 + 8u * (2 * P_STAGES + 2 * OP_STAGES + o); };
  constexpr int TB = 2 * P_STAGES + 3 * OP_STAGES;
  auto tfull_bar = [&](int a) { return bar0 + 8u * (TB + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (TB + 2 + a); };
  const uint32_t drain_bar = bar0 + 8u * (TB + 4);

  if (threadIdx.x == 0) {
    for (int p = 0; p < P_STAGES; ++p) {
      mbar_init(pfull_bar(p), 1);
      mbar_init(pempty_bar(p), WPT);
    }
    for (int o = 0; o < OP_STAGES; ++o) {
      mbar_init(lconv_bar(o), WPT);
      mbar_init(rconv_bar(o), 1);
      mbar_init(oempty_bar(o), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), 2 * EPI_THREADS);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) tma_prefetch_desc(tmP);
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
      // ---------------- TMA producer of packed codes (both CTAs)
      int n = 0;
      int last_parity[P_STAGES];
      for (int p = 0; p < P_STAGES; ++p) last_parity[p] = -1;
      bool ok = true;
      Sched sc;
      for (sc.init(sp, cstart); sc.valid && ok; sc.advance(cstep)) {
        const int ya = sc.a_row() / 2 + SNPS * static_cast<int>(rank);
        const int yb = sc.b_row() / 2 + SNPS * static_cast<int>(rank);
        const int kbs = sc.k_blocks(nkb);
        const int kb0 = sc.k_begin();
        for (int kb = 0; kb < kbs; ++kb, ++n) {
          const int p = n % P_STAGES;
          const uint32_t ph = static_cast<uint32_t>(n / P_STAGES) & 1u;
          if (!mbar_wait_bounded(pempty_bar(p), ph ^ 1u, status, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(pfull_bar(p), P_BYTES);
          const uint32_t dst = smem_u32(sP + p * P_BYTES);
          tma_load_2d(dst, tmP, (kb0 + kb) * (BK / 32), ya, pfull_bar(p));
          tma_load_2d(dst + P_SIDE_BYTES, tmP, (kb0 + kb) * (BK / 32), yb, pfull_bar(p));
          last_parity[p] = static_cast<int>(ph);
        }
      }
      if (!ok) {
        // Let the copies already issued land before the CTA's memory goes away.
        for (int p = 0; p < P_STAGES; ++p)
          if (last_parity[p] >= 0) mbar_wait_timeout(pfull_bar(p), static_cast<uint32_t>(last_parity[p]));
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ---------------- MMA issuer (leader CTA)
      int n = 0;
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
        for (int kb = 0; kb < kbs; ++kb, ++n) {
          const int o = n % OP_STAGES;
          const uint32_t ph = static_cast<uint32_t>(n / OP_STAGES) & 1u;
          if (!mbar_wait_bounded(lconv_bar(o), ph, status, abort_flag) ||
              !pk::wait_bounded_cluster(rconv_bar(o), ph, status, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sA + o * A_BYTES);
          const uint32_t b0 = smem_u32(sB + o * B_BYTES);
#pragma unroll
          for (int k = 0; k < BK / UK; ++k)
            mma_f8f6f4_pair(d_tmem, smem_desc_sw128(a0 + k * UK), smem_desc_sw128(b0 + k * UK),
                            IDESC, (kb | k) != 0 ? 1u : 0u);
          mma_commit_pair(oempty_bar(o), 0x3);
        }
        if (!ok) break;
        mma_commit_pair(tfull_bar(acc), 0x3);
      }
      mma_commit_pair(drain_bar, 0x1);
      mbar_wait_timeout(drain_bar, 0);
    } else if (lane == 0) {
      // ---------------- relay (follower CTA): its operand stages are ready
      int n = 0;
      bool ok = true;
      Sched sc;
      for (sc.init(sp, cstart); sc.valid && ok; sc.advance(cstep)) {
        const int kbs = sc.k_blocks(nkb);
        for (int kb = 0; kb < kbs; ++kb, ++n) {
          const int o = n % OP_STAGES;
          const uint32_t ph = static_cast<uint32_t>(n / OP_STAGES) & 1u;
          if (!mbar_wait_bounded(lconv_bar(o), ph, status, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_cluster(map_to_rank(rconv_bar(o), 0));
        }
      }
    }
  } else if (warp < 2 + EW) {
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
  } else {
    // ---------------- converters (both CTAs)
    // Per K stage, 32 groups of 4 SNPs x 8 chunks of 16 entries: group g is
    // operand g / 16 (A, B), SNPs 4 (g % 16) .. + 3; warp cw takes groups
    // cw, cw + CW, ...  Lane = (SNP 4 (g % 16) + lane / 8, chunk lane % 8): a
    // warp reads 128 contiguous bytes of codes and writes four whole pairs of
    // 128-byte rows.  Rows 2 s and 2 s + 1 of SNP s have (row & 7) = 2 (lane /
    // 8) and 2 (lane / 8) + 1, so each lane's swizzled 16-byte offsets are fixed.
    const int cw = warp - 2 - EW;
    const int team = cw / WPT;
    const int member = cw % WPT;
    const int c = lane & 7;
    const int rr = lane >> 3;
    const uint32_t off0 = static_cast<uint32_t>((c ^ (2 * rr)) << 4);
    const uint32_t off1 = 128u + static_cast<uint32_t>((c ^ (2 * rr + 1)) << 4);
    constexpr int GROUPS = 2 * SNPS / 4;
    static_assert(GROUPS % WPT == 0, "whole groups per converter warp");
    int n = 0;
    Sched sc;
    bool ok = true;
    for (sc.init(sp, cstart); sc.valid && ok; sc.advance(cstep)) {
      // SNPs of the CTA's A and B halves that exist (the rest read as missing).
      const int64_t ra = n_v - (sc.a_row() / 2 + SNPS * static_cast<int64_t>(rank));
      const int64_t rb = n_v - (sc.b_row() / 2 + SNPS * static_cast<int64_t>(rank));
      const int va = ra < 0 ? 0 : (ra > SNPS ? SNPS : static_cast<int>(ra));
      const int vb = rb < 0 ? 0 : (rb > SNPS ? SNPS : static_cast<int>(rb));
      const int kbs = sc.k_blocks(nkb);
      const int kb0 = sc.k_begin();
      for (int kb = 0; kb < kbs; ++kb, ++n) {
        if (n % TEAMS != team) continue;
        const int p = n % P_STAGES;
        const uint32_t pph = static_cast<uint32_t>(n / P_STAGES) & 1u;
        const int o = n % OP_STAGES;
        const uint32_t oph = static_cast<uint32_t>(n / OP_STAGES) & 1u;
        const bool got = mbar_wait_bounded(pfull_bar(p), pph, status, abort_flag) &&
                         mbar_wait_bounded(oempty_bar(o), oph ^ 1u, status, abort_flag);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        // Entries of this lane's chunk inside the panel (2 bits each).
        const int64_t left = n_f - (static_cast<int64_t>(kb0 + kb) * BK + 16 * c);
        const uint32_t mq = left >= 16 ? 0xFFFFFFFFu
                                       : (left <= 0 ? 0u : (1u << (2 * static_cast<int>(left))) - 1u);
        const uint8_t *src = sP + p * P_BYTES + rr * 32 + c * 4;
        uint8_t *dA = sA + o * A_BYTES + rr * 256;
        uint8_t *dB = sB + o * B_BYTES + rr * 256;
#pragma unroll
        for (int it = 0; it < GROUPS / WPT; ++it) {
          const int g = it * WPT + member;
          const int side = g / (GROUPS / 2);
          const int s4 = 4 * (g % (GROUPS / 2));  // first SNP of the group
          const uint32_t m = s4 + rr < (side ? vb : va) ? mq : 0u;
          uint32_t x = *reinterpret_cast<const uint32_t *>(src + side * P_SIDE_BYTES + s4 * 32);
          x = (x & m) | (0xAAAAAAAAu & ~m);  // masked entries read as missing
          // 2-bit codes -> 4-bit byte selectors: lo for entries 0-7, hi for 8-15.
          uint32_t lo = x & 0xFFFFu, hi = x >> 16;
          lo = (lo | (lo << 8)) & 0x00FF00FFu;
          hi = (hi | (hi << 8)) & 0x00FF00FFu;
          lo = (lo | (lo << 4)) & 0x0F0F0F0Fu;
          hi = (hi | (hi << 4)) & 0x0F0F0F0Fu;
          lo = (lo | (lo << 2)) & 0x33333333u;
          hi = (hi | (hi << 2)) & 0x33333333u;
          const uint4 v0 = make_uint4(__byte_perm(pk::kRho0, 0u, lo), __byte_perm(pk::kRho0, 0u, lo >> 16),
                                      __byte_perm(pk::kRho0, 0u, hi), __byte_perm(pk::kRho0, 0u, hi >> 16));
          const uint4 v1 = make_uint4(__byte_perm(pk::kRho1, 0u, lo), __byte_perm(pk::kRho1, 0u, lo >> 16),
                                      __byte_perm(pk::kRho1, 0u, hi), __byte_perm(pk::kRho1, 0u, hi >> 16));
          uint8_t *d = (side ? dB : dA) + s4 * 256;
          if (!CCC_IN_BOUNDS(rr * 256 + s4 * 256 + off1 + 15, A_BYTES, status)) continue;
          *reinterpret_cast<uint4 *>(d + off0) = v0;
          *reinterpret_cast<uint4 *>(d + off1) = v1;
        }
        fence_proxy_async_smem();  // the MMA (async proxy) reads what was written
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(pempty_bar(p));
          mbar_arrive(lconv_bar(o));
        }
      }
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
