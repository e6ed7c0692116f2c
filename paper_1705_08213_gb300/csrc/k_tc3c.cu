// 3-way tallies by genotype classes of the middle SNP, on SM pairs.
//
// Sec. 3.2 obtains the tallies of a slab of fixed j from products of count
// matrices masked by the column v_j.  Here the mask is split by the genotype
// class of v_j at each individual q: C0 (hom 0, rho_j = (2, 0)), C1 (het,
// (1, 1)), C2 (hom 1, (0, 2)), CM (missing, (0, 0)).  With
// X_S = sum_{q in S} rho_i(a) rho_k(c),
//     r_{ijk}^{a0c} = 2 X_C0 + X_C1,      r_{ijk}^{a1c} = X_C1 + 2 X_C2,
// and the 2-way tally r_{ik}^{ac} = X_C0 + X_C1 + X_C2 + X_CM (Eq. 4) gives
//     r_{ijk}^{a0c} = r_{ik}^{ac} - D + T,   r_{ijk}^{a1c} = r_{ik}^{ac} - D - T,
//     T = X_C0 - X_C2 = sum_q rho_i(a) s_j(q) rho_k(c),   s_j in {+1, 0, -1},
//     D = X_CM.
// Per triple the tensor cores then form 4 products over the n_f individuals
// (T) plus 4 over the few individuals with v_j missing (D), instead of the 8
// of the masked operand L_j = rho_i(a) rho_j(b) of k_tc3.cu; the 2-way tallies
// r_ik come from one 2-way tally pass.
//
// Passes per batch of slabs:
//   k_compact3  the individuals with v_j missing; when there are at most kCap
//               of them, the count rows of every SNP restricted to them;
//   k_mask3c    for the side of the slab with fewer SNPs (i < j or k > j),
//               rows R(s, x) * s_j in e4m3 (values 0, +-1, +-2), and, when v_j
//               has more than kCap missing entries, rows R(s, x) * [v_j missing];
//   k_tally3_class  the tiles of the batch.  A cluster of two CTAs
//               (cta_group::2, M = 256) takes 128 SNPs i (64 per CTA, rows
//               (i, a)) and up to 80 SNPs k (N <= 160 columns (k, c)); TMEM
//               holds two T accumulators (double buffered) and one D
//               accumulator, 3 x 160 of the 512 columns.  TMA brings every
//               operand tile; T runs over the n_f individuals (one operand
//               masked, the other plain R), D over the compacted rows (or the
//               missing-masked rows).  The epilogue reads T and D from TMEM and
//               r_ik from the 2-way tally table and writes the 8 tallies and 8
//               CCC values (Eq. 7 with the Eq. 8 frequencies) of every triple
//               i < j < k of the tile.
#include "ccc_launch.h"
#include "ccc_metric.cuh"
#include "tc_pipeline.cuh"
#include "tc_pipeline_pair.cuh"

namespace ccc {
namespace {

using tcp::cluster_rank;
using tcp::cluster_sync;
using tcp::map_to_rank;

constexpr int kSnpI = 128;            // SNPs i per pair tile
constexpr int kSnpK = 80;             // SNPs k per pair tile (at most)
constexpr int kNMax = 2 * kSnpK;      // accumulator columns
constexpr int kBK = 128;              // individuals per k-block
constexpr int kUK = 32;               // K per MMA
constexpr int kABytes = 128 * kBK;    // A rows per CTA x 128 bytes
constexpr int kBRows = kNMax / 2;     // B rows per CTA
constexpr int kBBytes = kBRows * kBK;
constexpr int kStages = 8;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kCap = 256;             // compacted missing columns per slab
constexpr int kNumBars = 2 * kStages + 2 + 2 + 1 + 1;
constexpr uint32_t kColT0 = 0, kColT1 = kNMax, kColD = 2 * kNMax;
constexpr size_t kSmemBytes =
    1024 + static_cast<size_t>(kStages) * (kABytes + kBBytes) + kNumBars * 8 + 64;

static_assert(kBBytes % 1024 == 0, "B tiles keep the 1024-byte swizzle alignment");
static_assert(3 * kNMax <= 512, "three accumulators in 512 TMEM columns");
static_assert(kSmemBytes <= 232448, "dynamic shared memory limit");

constexpr uint64_t kEven = 0x5555555555555555ull;

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
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

// mbar_wait_bounded with cluster-scope acquire (arrivals from the peer CTA).
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint32_t bar, uint32_t parity,
                                                          int32_t *status,
                                                          volatile int *abort_flag) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  uint32_t spins = 0;
  while (true) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
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

// D-slot accesses with an L2 evict-last policy: each slot is written and read
// back by the same thread one tile later, while the tiles' outputs stream
// through L2 (evict-first stores); without the hint the slots were evicted and
// written back to DRAM between the two.
__device__ __forceinline__ uint64_t l2_evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void st_l2_keep(uint32_t *p, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ uint32_t ld_l2_keep(const uint32_t *p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol) : "memory");
  return v;
}

// P(x) = sum_{j < x} min(j, n_v - 1 - j): SNPs on the masked side of the
// slabs before x.  Slab j owns 4 min(j, n_v - 1 - j) masked rows (2 per SNP
// for s_j, 2 for the missing mask).
__host__ __device__ inline int64_t mask_prefix(int64_t x, int64_t n_v) {
  const int64_t h = (n_v - 1) / 2;  // min(j, n_v - 1 - j) = j for j <= h
  if (x <= h + 1) return x * (x - 1) / 2;
  const int64_t lo = h * (h + 1) / 2;
  // sum_{j = h + 1}^{x - 1} (n_v - 1 - j) = sum_{t = n_v - x}^{n_v - 2 - h} t
  const int64_t a = n_v - x, b = n_v - 2 - h;
  return lo + (b * (b + 1) - (a - 1) * a) / 2;
}

// Tiles of the slabs [j0, j1): slab j has ceil(j / 128) i-blocks times
// ceil((n_v - 1 - j) / SNPK) k-blocks, i-block-major.  KBI: individuals per
// 128-byte K stage (128 for e4m3 operands, 256 for e2m1).
template <int SNPK, int KBI = kBK>
struct ClassSchedT {
  struct Params {
    int j0, j1, n_v, nkb;
    int mrow0;               // first masked row (operand buffer rows after R)
    const int32_t *missing;  // entries of v_j missing, per slab of the batch
  };
  int j, j0, j1, n_v, nkb, mrow0;
  const int32_t *missing_;
  int mt, nt, m, n;
  bool valid;

  __device__ void set_slab() {
    mt = static_cast<int>(cdiv(j, kSnpI));
    nt = static_cast<int>(cdiv(n_v - 1 - j, SNPK));
  }
  __device__ void skip_empty() {
    while (j < j1) {
      set_slab();
      if (mt > 0 && nt > 0) return;
      ++j;
    }
    valid = false;
  }
  __device__ void init(const Params &p, int64_t start) {
    j = j0 = p.j0;
    j1 = p.j1;
    n_v = p.n_v;
    nkb = p.nkb;
    mrow0 = p.mrow0;
    missing_ = p.missing;
    m = n = 0;
    valid = true;
    skip_empty();
    advance(start);
  }
  __device__ void advance(int64_t step) {
    while (valid && step > 0) {
      const int64_t pos = static_cast<int64_t>(m) * nt + n;
      const int64_t rem = static_cast<int64_t>(mt) * nt - 1 - pos;
      if (step <= rem) {
        m = static_cast<int>((pos + step) / nt);
        n = static_cast<int>((pos + step) % nt);
        return;
      }
      step -= rem + 1;
      ++j;
      m = n = 0;
      skip_empty();
    }
  }
  __device__ int i0() const { return kSnpI * m; }
  __device__ int k0() const { return j + 1 + SNPK * n; }
  // Accumulator columns of the tile: 2 per SNP k, rounded up to 32.
  __device__ int ncols() const {
    const int nk = min(SNPK, n_v - k0());
    return (2 * nk + 31) / 32 * 32;
  }
  __device__ int slab() const { return j - j0; }
  // The masked operand holds the side of the slab with fewer SNPs: i < j when
  // 2 j <= n_v - 1, else k > j.
  __device__ bool i_masked() const { return 2 * j <= n_v - 1; }
  __device__ int side() const { return min(j, n_v - 1 - j); }
  // First row of slab j's masked rows in the operand buffer.
  __device__ int mrow() const { return mrow0 + static_cast<int>(4 * (mask_prefix(j, n_v) - mask_prefix(j0, n_v))); }
  __device__ int missing() const { return __ldg(missing_ + (j - j0)); }
  // k-blocks of the D phase, and whether they run over all of R (masked).
  __device__ int d_blocks(bool *full) const {
    const int c = missing();
    *full = c > kCap;
    return *full ? nkb : static_cast<int>(cdiv(c, KBI));
  }
};
using ClassSched = ClassSchedT<kSnpK>;

// Per-byte masks of 16 individuals from their 2-bit codes w (code t at bits
// 2t, 2t+1): keep[g] has byte b = 0xFF where the selected class holds for
// individual 4g + b, neg[g] byte b = 0x80 where the sign flips.
__device__ __forceinline__ uint32_t spread4(uint32_t bits) {
  // bits 0, 2, 4, 6 -> bytes 0..3 (value 0 or 1)
  return (bits & 1u) | ((bits & 4u) << 6) | ((bits & 16u) << 12) | ((bits & 64u) << 18);
}

__device__ __forceinline__ void class_masks(uint32_t w, bool missing_mode, uint32_t (&keep)[4],
                                            uint32_t (&neg)[4]) {
  uint32_t kb, nb;
  if (!missing_mode) {
    kb = ~(w ^ (w >> 1)) & 0x55555555u;  // codes 00 and 11 (homozygous)
    nb = w & (w >> 1) & 0x55555555u;     // code 11: s_j = -1
  } else {
    kb = (w >> 1) & ~w & 0x55555555u;  // code 10: missing
    nb = 0u;
  }
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const uint32_t yk = spread4((kb >> (8 * g)) & 0x55u);
    const uint32_t yn = spread4((nb >> (8 * g)) & 0x55u);
    keep[g] = (yk << 8) - yk;
    neg[g] = yn << 7;
  }
}

struct ClassArgs {
  Tally3Args t;
  const int32_t *rtab;  // 2-way tallies [pair][4]
  uint32_t *dscratch;   // wide tiles: [cta][2][k][lane] D counts
};

__global__ void __launch_bounds__(kThreads, 1) __cluster_dims__(2, 1, 1)
    k_tally3_class(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmCA, const __grid_constant__ CUtensorMap tmCB,
                   const ClassArgs args, ClassSched::Params sp) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t *smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kABytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + kStages * kBBytes);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + kNumBars);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  int32_t *status = args.t.status;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * kStages + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * kStages + 2 + a); };
  const uint32_t dempty_bar = bar0 + 8u * (2 * kStages + 4);
  const uint32_t drain_bar = bar0 + 8u * (2 * kStages + 5);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    // The leader's tempty / dempty gather its own epilogue warps and one
    // forwarded arrival from the follower, whose tempty gathers its warps.
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), leader ? kEpiWarps + 1 : kEpiWarps);
    }
    mbar_init(dempty_bar, kEpiWarps + 1);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
    tma_prefetch_desc(&tmCA);
    tma_prefetch_desc(&tmCB);
  }
  if (warp == 1) {
    tcp::tmem_alloc_pair(smem_u32(tmem_slot), 512);
    tcp::tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t cstart = blockIdx.x >> 1;
  const int64_t cstep = gridDim.x >> 1;
  const int64_t n_v = args.t.n_v;
  const int nkb = sp.nkb;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs)
      int stage = 0;
      uint32_t phase = 0;
      int last_parity[kStages];
      for (int s = 0; s < kStages; ++s) last_parity[s] = -1;
      bool ok = true;
      ClassSched sc;
      // One k-block: wait for the stage, expect the bytes (leader), load A and B.
      auto step = [&](const CUtensorMap *ma, int ya, const CUtensorMap *mb, int yb, int x) -> bool {
        if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, status, abort_flag)) return false;
        if (leader) mbar_arrive_expect_tx(full_bar(stage), 2 * (kABytes + kBBytes));
        const uint32_t fb = map_to_rank(full_bar(stage), 0);
        tcp::tma_load_2d_pair(smem_u32(sA + stage * kABytes), ma, x, ya, fb);
        tcp::tma_load_2d_pair(smem_u32(sB + stage * kBBytes), mb, x, yb, fb);
        last_parity[stage] = static_cast<int>(phase);
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
        return true;
      };
      for (sc.init(sp, cstart); sc.valid && ok; sc.advance(cstep)) {
        const int half_n = sc.ncols() / 2;
        const int ia = 2 * (sc.i0() + 64 * static_cast<int>(rank));  // i-side row offset
        const int kb_row = static_cast<int>(rank) * half_n;         // k-side row offset
        const int mrow = sc.mrow();
        const int side2 = 2 * sc.side();
        const bool im = sc.i_masked();
        // T: the masked side from the masked rows, the other side from R.
        const int ya = im ? mrow + ia : ia;
        const int yb = im ? 2 * sc.k0() + kb_row : mrow + 2 * (sc.k0() - sc.j - 1) + kb_row;
        bool dfull;
        const int nd = sc.d_blocks(&dfull);  // loaded before the T loop needs it
        for (int kb = 0; kb < nkb && ok; ++kb) ok = step(&tmA, ya, &tmB, yb, kb * kBK);
        if (dfull) {
          // D over all individuals: the missing-masked rows follow the s_j rows.
          const int yda = im ? ya + side2 : ya;
          const int ydb = im ? yb : yb + side2;
          for (int kb = 0; kb < nd && ok; ++kb) ok = step(&tmA, yda, &tmB, ydb, kb * kBK);
        } else {
          const int cb = sc.slab() * static_cast<int>(2 * n_v);
          for (int kb = 0; kb < nd && ok; ++kb)
            ok = step(&tmCA, cb + ia, &tmCB, cb + 2 * sc.k0() + kb_row, kb * kBK);
        }
      }
      if (!ok) {
        if (leader) {
          for (int s = 0; s < kStages; ++s)
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
      // Descriptors of stage 0; a stage and a 32-byte K step only move the
      // start-address field (address >> 4), so every MMA's descriptors are
      // one add away from these.
      const uint64_t dA0 = smem_desc_sw128(smem_u32(sA));
      const uint64_t dB0 = smem_desc_sw128(smem_u32(sB));
      int stage = 0;
      uint32_t phase = 0;
      int lt = 0;
      bool ok = true;
      ClassSched sc;
      for (sc.init(sp, cstart); sc.valid && ok; sc.advance(cstep), ++lt) {
        const int acc = lt & 1;
        if (!mbar_wait_cluster_bounded(tempty_bar(acc), ((lt >> 1) & 1) ^ 1u, status, abort_flag))
          break;
        tc_fence_after();
        const uint32_t idesc = idesc_e4m3_f32(256, static_cast<uint32_t>(sc.ncols()));
        bool dfull;
        const int nd = sc.d_blocks(&dfull);  // loaded before the T loop needs it
        for (int phase_d = 0; phase_d < 2 && ok; ++phase_d) {
          const int nblk = phase_d == 0 ? nkb : nd;
          if (nblk == 0) continue;
          if (phase_d == 1) {
            if (!mbar_wait_cluster_bounded(dempty_bar, (lt & 1) ^ 1u, status, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          const uint32_t d_tmem = tmem_base + (phase_d ? kColD : (acc ? kColT1 : kColT0));
          for (int kb = 0; kb < nblk; ++kb) {
            if (!mbar_wait_bounded(full_bar(stage), phase, status, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t da = dA0 + static_cast<uint64_t>(stage * (kABytes >> 4));
            const uint64_t db = dB0 + static_cast<uint64_t>(stage * (kBBytes >> 4));
            tcp::mma_f8f6f4_pair(d_tmem, da, db, idesc, kb != 0 ? 1u : 0u);
#pragma unroll
            for (int k = 1; k < kBK / kUK; ++k)
              tcp::mma_f8f6f4_pair(d_tmem, da + (k * kUK >> 4), db + (k * kUK >> 4), idesc, 1u);
            tcp::mma_commit_pair(empty_bar(stage), 0x3);
            if (++stage == kStages) {
              stage = 0;
              phase ^= 1u;
            }
          }
        }
        if (!ok) break;
        tcp::mma_commit_pair(tfull_bar(acc), 0x3);
      }
      tcp::mma_commit_pair(drain_bar, 0x1);
      mbar_wait_timeout(drain_bar, 0);
    } else if (lane == 0) {
      // ---------------- follower: forward the epilogue's release to the leader
      int lt = 0;
      ClassSched sc;
      for (sc.init(sp, cstart); sc.valid; sc.advance(cstep), ++lt) {
        const int acc = lt & 1;
        if (!mbar_wait_bounded(tempty_bar(acc), (lt >> 1) & 1, status, abort_flag)) break;
        tc_fence_before();
        mbar_arrive_cluster(map_to_rank(dempty_bar, 0));
        mbar_arrive_cluster(map_to_rank(tempty_bar(acc), 0));
      }
    }
  } else {
    // ---------------- epilogue (both CTAs)
    const int ew = warp - 2;  // 0..7
    const int quarter = warp & 3;
    const int half = ew >> 2;
    const int L = quarter * 32 + lane;  // TMEM lane = A row of this CTA
    const int a = L & 1;
    const int32_t *__restrict__ rtab = args.rtab;
    const float *__restrict__ wv = args.t.w;
    int4 *__restrict__ tally_out = reinterpret_cast<int4 *>(args.t.tally);
    float4 *__restrict__ ccc_out = reinterpret_cast<float4 *>(args.t.ccc);
    const bool want_ccc = ccc_out != nullptr;
    const bool persnp = args.t.norm == CCC_NORM_PERSNP;
    const float gamma = args.t.gamma;
    const int64_t s_begin = slab_offset_dev(args.t.j_begin, n_v);
    int lt = 0;
    ClassSched sc;
    for (sc.init(sp, cstart); sc.valid; sc.advance(cstep), ++lt) {
      const int acc = lt & 1;
      const bool got = mbar_wait_bounded(tfull_bar(acc), (lt >> 1) & 1, status, abort_flag);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const int64_t j = sc.j;
      const int64_t i = sc.i0() + 64 * static_cast<int64_t>(rank) + (L >> 1);
      const bool row_ok = i < j;
      const int ncols = sc.ncols();
      const int64_t k_first = sc.k0();
      bool dfull;
      const bool has_d = sc.d_blocks(&dfull) > 0;
      int nch = (ncols - kNMax / 2 * half) / 16;
      nch = nch < 0 ? 0 : (nch > 5 ? 5 : nch);
      const uint32_t lane_base = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16);
      const uint32_t t_x = lane_base + (acc ? kColT1 : kColT0);
      const uint32_t t_d = lane_base + kColD;
      // The accumulators of this tile have been read: the leader's warps arrive
      // on its barriers, the follower's on its own tempty (forwarded by warp 1).
      auto release = [&]() {
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (leader) mbar_arrive(dempty_bar);
          mbar_arrive(tempty_bar(acc));
        }
      };
      if (nch == 0) {
        release();
        continue;
      }
      const int64_t span = n_v - 1 - j;
      const int64_t base = slab_offset_dev(j, n_v) - s_begin + i * span - (j + 1);
      const int64_t pbase = i * (2 * n_v - i - 1) / 2 - i - 1;  // pair (i, k) at pbase + k
      float wi = 1.f, wj0 = 1.f, wj1 = 1.f;
      if (want_ccc && persnp) {
        if (row_ok) wi = __ldg(wv + 2 * i + a);
        wj0 = __ldg(wv + 2 * j);
        wj1 = __ldg(wv + 2 * j + 1);
      }
      for (int c = 0; c < nch; ++c) {
        const int col = kNMax / 2 * half + 16 * c;
        const int64_t kc = k_first + col / 2;
        uint32_t x[16], d[16];
        tmem_ld_32x32b_x16(t_x + col, x);
        if (has_d) tmem_ld_32x32b_x16(t_d + col, d);
        // Every global load of the chunk is issued before its stores.
        int2 r[8];
        float2 wk[8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int64_t k = kc + kk;
          const bool ok = row_ok && k < n_v &&
                          CCC_IN_BOUNDS(pbase + k, n_v * (n_v - 1) / 2, args.t.status);
          r[kk] = ok ? __ldg(reinterpret_cast<const int2 *>(rtab + 4 * (pbase + k)) + a)
                     : make_int2(0, 0);
          wk[kk] = (ok && want_ccc && persnp) ? __ldg(reinterpret_cast<const float2 *>(wv) + k)
                                              : make_float2(1.f, 1.f);
        }
        tmem_ld_wait();
        if (!has_d) {
#pragma unroll
          for (int e = 0; e < 16; ++e) d[e] = 0u;
        }
        if (c == nch - 1) release();
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int64_t k = kc + kk;
          const bool ok = row_ok && k < n_v && CCC_IN_BOUNDS(base + k, args.t.out_len, args.t.status);
          const int32_t t0 = __float2int_rn(__uint_as_float(x[2 * kk]));
          const int32_t t1 = __float2int_rn(__uint_as_float(x[2 * kk + 1]));
          const int32_t d0 = __float2int_rn(__uint_as_float(d[2 * kk]));
          const int32_t d1 = __float2int_rn(__uint_as_float(d[2 * kk + 1]));
          const int32_t u0 = r[kk].x - d0, u1 = r[kk].y - d1;
          // r^{a b c}: b0c0, b0c1, b1c0, b1c1
          const int4 tv = make_int4(u0 + t0, u1 + t1, u0 - t0, u1 - t1);
          const int64_t t = base + k;
          if (ok) __stcs(tally_out + 2 * t + a, tv);
          if (want_ccc) {
            const int32_t own = tv.x + tv.y + tv.z + tv.w;  // sum over b, c (fixed a)
            const int32_t n8 = own + __shfl_xor_sync(0xffffffffu, own, 1);
            const int32_t b0 = tv.x + tv.y, b1 = tv.z + tv.w;
            const int32_t c0 = tv.x + tv.z, c1 = tv.y + tv.w;
            const int32_t rb0 = b0 + __shfl_xor_sync(0xffffffffu, b0, 1);
            const int32_t rb1 = b1 + __shfl_xor_sync(0xffffffffu, b1, 1);
            const int32_t q0 = c0 + __shfl_xor_sync(0xffffffffu, c0, 1);
            const int32_t q1 = c1 + __shfl_xor_sync(0xffffffffu, c1, 1);
            if (ok) {
              float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
              if (n8 != 0) {
                const float dn = static_cast<float>(n8);
                float fi = wi, fj0 = wj0, fj1 = wj1, fk0 = wk[kk].x, fk1 = wk[kk].y;
                if (!persnp) {
                  fi = joint_factor(own, dn, gamma);
                  fj0 = joint_factor(rb0, dn, gamma);
                  fj1 = joint_factor(rb1, dn, gamma);
                  fk0 = joint_factor(q0, dn, gamma);
                  fk1 = joint_factor(q1, dn, gamma);
                }
                if (persnp) {
                  const float inv = __frcp_rn(dn);
                  const float g0 = __fmul_rn(fi, fj0), g1 = __fmul_rn(fi, fj1);
                  out.x = ccc3_persnp(tv.x, inv, g0, fk0);
                  out.y = ccc3_persnp(tv.y, inv, g0, fk1);
                  out.z = ccc3_persnp(tv.z, inv, g1, fk0);
                  out.w = ccc3_persnp(tv.w, inv, g1, fk1);
                } else {
                  out.x = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(tv.x), dn), fi), fj0), fk0);
                  out.y = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(tv.y), dn), fi), fj0), fk1);
                  out.z = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(tv.z), dn), fi), fj1), fk0);
                  out.w = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(tv.w), dn), fi), fj1), fk1);
                }
              }
              __stcs(ccc_out + 2 * t + a, out);
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  if (warp == 1) tcp::tmem_dealloc_pair(tmem_base, 512);
}

// ---------------------------------------------------------------------------
// The same tallies on tiles of 128 SNPs i x 128 SNPs k (N = 256 columns), for
// n_f <= kWideMaxNf.  A k-block of TMA loads costs about as long as an N = 256
// MMA k-block on GB300, so wide tiles keep the tensor cores busy where N = 160
// ones cannot; TMEM then holds only the two T accumulators (2 x 256 columns).
// The D product of tile u is formed in tile u's own accumulator before its T
// phase -- issued in the middle of tile u-1's T phase -- and each epilogue
// thread moves its part of it (16-bit counts, D <= 4 n_f) to its own slots of
// a small global scratch (two tiles per CTA, 128 KB, L2-resident) before the
// T phase of tile u overwrites the accumulator.
namespace wide {
// Tile shape by operand type.  e4m3: 128 SNPs k (N = 256), two 256-column T
// accumulators.  e2m1 (FP4, block-scaled kind::mxf4): the scale factors need
// 32 TMEM columns of their own, so the T accumulators are 240 columns wide
// (120 SNPs k, N = 240), at 0 and 240, and the factors sit at 480-511; a
// 128-byte K stage then holds 256 individuals.
template <bool FP4>
struct Cfg {
  static constexpr int kSnpK = FP4 ? 120 : 128;
  static constexpr int kN = 2 * kSnpK;
  static constexpr int kKBI = FP4 ? 256 : kBK;  // individuals per K stage
  static constexpr int kChunks = kSnpK / 8;     // 8-SNP epilogue chunks
  using Sched = ClassSchedT<kSnpK, kKBI>;
};
constexpr uint32_t kSfCol = 480;
constexpr int kStages = 5;
constexpr int kTile = 128 * kBK;                  // 128 rows x 128 bytes
constexpr int kStageBytes = 2 * kTile;            // A + B per CTA
constexpr int kDWords = 128 * 128;                // per tile: [k (0..127)][lane] x (u16 c = 0, u16 c = 1)
constexpr int kMaxCtas = 256;                     // CTAs the D scratch is sized for
// Epilogue: 2 warps per TMEM lane quarter; warp g of a quarter takes the
// 8-SNP chunks c = g, g + 2, ... of the tile's 16 (12 warps measured slower:
// their register cap of 146 cost more than the added overlap gave).
constexpr int kEpiWarps = 8;
// The 2-way tallies r_ik of an epilogue warp's next chunk (its 16 SNPs i x 8
// SNPs k, 128 bytes per i) are copied into shared memory with asynchronous
// 16-byte copies (cp.async, each warp instruction 4 whole rows) while it works
// on the current chunk: rows 144 bytes apart, so that the lanes' 8-byte reads
// of one k are free of bank conflicts.  GB300, 1,536 x 8,192: class kernels
// 14.24 -> 13.7 ms against one 8-byte load per lane and k from the 2-way table
// (16 rows per warp load); a second buffer (prefetching two chunks ahead)
// measured the same.  Five operand stages measured as fast as six here and
// leave shared memory for the preparation kernels of the next batch.
constexpr int kRowStride = 144;
constexpr int kRbufBytes = 16 * kRowStride;
constexpr int kNumBars = 2 * kStages + 2 + 2 + 3;  // full, empty, tfull, tempty, dready, ddone, drain
constexpr size_t kSmem = 1024 + static_cast<size_t>(kStages) * kStageBytes + kNumBars * 8 + 64 +
                         16 + static_cast<size_t>(kEpiWarps) * kRbufBytes;
constexpr int kGroups = kEpiWarps / 4;
constexpr int kThreads = 64 + 32 * kEpiWarps;
static_assert(kSmem <= 232448, "dynamic shared memory limit");
static_assert(2 * Cfg<true>::kN + 32 <= 512 && kSfCol == 2 * Cfg<true>::kN, "FP4 TMEM layout");
static_assert(Cfg<true>::kN % 16 == 0 && Cfg<true>::kN / 2 <= 128, "FP4 tile: N per CTA in the B box");
}  // namespace wide

constexpr int64_t kWideMaxNf = 16383;  // 4 n_f < 2^16

// MODE 0: tallies only; 1: tallies and CCC, PERSNP; 2: tallies and CCC, JOINT.
// FP4: e2m1 operands (see wide::Cfg).
template <int MODE, bool FP4>
__global__ void __launch_bounds__(wide::kThreads, 1) __cluster_dims__(2, 1, 1)
    k_tally3_class_w(const __grid_constant__ CUtensorMap tmOp,
                     const __grid_constant__ CUtensorMap tmC, const ClassArgs args,
                     typename wide::Cfg<FP4>::Sched::Params sp) {
  constexpr int kStages = wide::kStages;
  constexpr int kTile = wide::kTile;
  constexpr int kStageBytes = wide::kStageBytes;
  constexpr int kDWords = wide::kDWords;
  constexpr int kNumBars = wide::kNumBars;
  constexpr int kN = wide::Cfg<FP4>::kN;
  constexpr int kChunks = wide::Cfg<FP4>::kChunks;
  constexpr int kEpiWarps = wide::kEpiWarps;
  using Sched = typename wide::Cfg<FP4>::Sched;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t *smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t *sA = smem;
  uint8_t *sB = smem + kStages * kTile;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
  uint32_t *dsc = args.dscratch + static_cast<int64_t>(blockIdx.x) * 2 * kDWords;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + kNumBars);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  int32_t *status = args.t.status;

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (kStages + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (2 * kStages + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (2 * kStages + 2 + a); };
  const uint32_t dready_bar = bar0 + 8u * (2 * kStages + 4);
  const uint32_t ddone_bar = bar0 + 8u * (2 * kStages + 5);
  const uint32_t drain_bar = bar0 + 8u * (2 * kStages + 6);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    // The leader's tempty / ddone gather its epilogue warps and one arrival
    // forwarded by the follower, whose own barriers gather its warps.
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), leader ? kEpiWarps + 1 : kEpiWarps);
    }
    mbar_init(dready_bar, 1);
    mbar_init(ddone_bar, leader ? kEpiWarps + 1 : kEpiWarps);
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmOp);
    tma_prefetch_desc(&tmC);
  }
  if (warp == 1) {
    tcp::tmem_alloc_pair(smem_u32(tmem_slot), 512);
    tcp::tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int64_t cstart = blockIdx.x >> 1;
  const int64_t cstep = gridDim.x >> 1;
  if (FP4) {
    // Scale factors 1.0 (UE8M0) in columns kSfCol .. kSfCol + 31 of both CTAs,
    // one lane quarter per epilogue warp, before the leader's first MMA.
    if (warp >= 2 && warp < 6) {
      uint32_t v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = tcp::SF_ONE_UE8M0;
      tmem_st_32x32b_x32(tmem_base + (static_cast<uint32_t>((warp & 3) * 32) << 16) + wide::kSfCol,
                         v);
      tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
  }
  const int64_t n_v = args.t.n_v;
  const int nkb = sp.nkb;
  // T k-blocks of a tile before the next tile's D phase is issued: late enough
  // that the epilogue has finished the buffer it reuses (7/8 of a tile).
  const int ins = (7 * nkb) / 8;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs)
      int stage = 0;
      uint32_t phase = 0;
      int last_parity[kStages];
      for (int s = 0; s < kStages; ++s) last_parity[s] = -1;
      bool ok = true;
      auto step = [&](const CUtensorMap *m, int ya, int yb, int x) -> bool {
        if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, status, abort_flag)) return false;
        if (leader) mbar_arrive_expect_tx(full_bar(stage), 2 * kStageBytes);
        const uint32_t fb = map_to_rank(full_bar(stage), 0);
        tcp::tma_load_2d_pair(smem_u32(sA + stage * kTile), m, x, ya, fb);
        tcp::tma_load_2d_pair(smem_u32(sB + stage * kTile), m, x, yb, fb);
        last_parity[stage] = static_cast<int>(phase);
        if (++stage == kStages) {
          stage = 0;
          phase ^= 1u;
        }
        return true;
      };
      // Rows of a tile: i side of this CTA, k side of this CTA.
      auto rows_t = [&](const Sched &t, int *ya, int *yb) {
        const int ia = 2 * (t.i0() + 64 * static_cast<int>(rank));
        const int kr = 2 * t.k0() + (kN / 2) * static_cast<int>(rank);
        const int mrow = t.mrow();
        if (t.i_masked()) {
          *ya = mrow + ia;
          *yb = kr;
        } else {
          *ya = ia;
          *yb = mrow + (kr - 2 * (t.j + 1));
        }
      };
      auto d_phase = [&](const Sched &t) -> bool {
        bool dfull;
        const int nd = t.d_blocks(&dfull);
        if (nd == 0) return true;
        if (dfull) {
          int ya, yb;
          rows_t(t, &ya, &yb);
          const int side2 = 2 * t.side();
          if (t.i_masked()) ya += side2; else yb += side2;
          for (int kb = 0; kb < nd; ++kb)
            if (!step(&tmOp, ya, yb, kb * kBK)) return false;
        } else {
          const int cb = t.slab() * static_cast<int>(2 * n_v);
          const int ia = cb + 2 * (t.i0() + 64 * static_cast<int>(rank));
          const int kr = cb + 2 * t.k0() + (kN / 2) * static_cast<int>(rank);
          for (int kb = 0; kb < nd; ++kb)
            if (!step(&tmC, ia, kr, kb * kBK)) return false;
        }
        return true;
      };
      Sched sc, nx;
      sc.init(sp, cstart);
      nx = sc;
      nx.advance(cstep);
      if (sc.valid) ok = d_phase(sc);
      while (sc.valid && ok) {
        int ya, yb;
        rows_t(sc, &ya, &yb);
        for (int kb = 0; kb < ins && ok; ++kb) ok = step(&tmOp, ya, yb, kb * kBK);
        if (ok && nx.valid) ok = d_phase(nx);
        for (int kb = ins; kb < nkb && ok; ++kb) ok = step(&tmOp, ya, yb, kb * kBK);
        sc = nx;
        nx.advance(cstep);
      }
      if (!ok) {
        if (leader) {
          for (int s = 0; s < kStages; ++s)
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
      const uint64_t dA0 = smem_desc_sw128(smem_u32(sA));
      const uint64_t dB0 = smem_desc_sw128(smem_u32(sB));
      constexpr uint32_t idesc = FP4 ? idesc_e2m1_f32(256, kN, true) : idesc_e4m3_f32(256, kN);
      const uint32_t sfa = tmem_base + wide::kSfCol, sfb = tmem_base + wide::kSfCol + 16;
      // One MMA of the kind: K = 32 e4m3 or 64 e2m1 entries = 32 bytes of the stage.
      auto mma = [&](uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t acc) {
        if (FP4)
          tcp::mma_mxf4_pair(d_tmem, da, db, idesc, sfa, sfb, acc);
        else
          tcp::mma_f8f6f4_pair(d_tmem, da, db, idesc, acc);
      };
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      int dcount = 0;  // D phases issued
      auto kblocks = [&](uint32_t d_tmem, int n) -> bool {
        for (int kb = 0; kb < n; ++kb) {
          if (!mbar_wait_bounded(full_bar(stage), phase, status, abort_flag)) return false;
          tc_fence_after();
          const uint64_t da = dA0 + static_cast<uint64_t>(stage * (kTile >> 4));
          const uint64_t db = dB0 + static_cast<uint64_t>(stage * (kTile >> 4));
          mma(d_tmem, da, db, kb != 0 ? 1u : 0u);
#pragma unroll
          for (int k = 1; k < kBK / kUK; ++k) mma(d_tmem, da + (k * kUK >> 4), db + (k * kUK >> 4), 1u);
          tcp::mma_commit_pair(empty_bar(stage), 0x3);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        return true;
      };
      // The T k-blocks [kb0, kb1) continue an accumulation started at kb 0.
      auto tblocks = [&](uint32_t d_tmem, int kb0, int kb1) -> bool {
        for (int kb = kb0; kb < kb1; ++kb) {
          if (!mbar_wait_bounded(full_bar(stage), phase, status, abort_flag)) return false;
          tc_fence_after();
          const uint64_t da = dA0 + static_cast<uint64_t>(stage * (kTile >> 4));
          const uint64_t db = dB0 + static_cast<uint64_t>(stage * (kTile >> 4));
          mma(d_tmem, da, db, kb != 0 ? 1u : 0u);
#pragma unroll
          for (int k = 1; k < kBK / kUK; ++k) mma(d_tmem, da + (k * kUK >> 4), db + (k * kUK >> 4), 1u);
          tcp::mma_commit_pair(empty_bar(stage), 0x3);
          if (++stage == kStages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        return true;
      };
      // D phase of tile u (buffer u & 1), after the epilogue released the buffer.
      auto d_phase = [&](const Sched &t, int u) -> bool {
        bool dfull;
        const int nd = t.d_blocks(&dfull);
        if (nd == 0) return true;
        if (!mbar_wait_cluster_bounded(tempty_bar(u & 1), ((u >> 1) & 1) ^ 1u, status, abort_flag))
          return false;
        tc_fence_after();
        if (!kblocks(tmem_base + (u & 1) * kN, nd)) return false;
        tcp::mma_commit_pair(dready_bar, 0x3);
        ++dcount;
        return true;
      };
      Sched sc, nx;
      sc.init(sp, cstart);
      nx = sc;
      nx.advance(cstep);
      int u = 0;
      if (sc.valid) ok = d_phase(sc, 0);
      int d_of_cur = 0;  // index of the current tile's D phase
      while (sc.valid && ok) {
        bool dfull;
        const bool has_d = sc.d_blocks(&dfull) > 0;
        // Buffer u & 1 is free (no D) or its D has been moved to shared memory.
        if (has_d) {
          if (!mbar_wait_cluster_bounded(ddone_bar, static_cast<uint32_t>(d_of_cur & 1), status,
                                         abort_flag))
            break;
        } else if (!mbar_wait_cluster_bounded(tempty_bar(u & 1), ((u >> 1) & 1) ^ 1u, status,
                                              abort_flag)) {
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (u & 1) * kN;
        ok = tblocks(d_tmem, 0, ins);
        const int d_next = dcount;
        if (ok && nx.valid) ok = d_phase(nx, u + 1);
        if (ok) ok = tblocks(d_tmem, ins, nkb);
        if (!ok) break;
        tcp::mma_commit_pair(tfull_bar(u & 1), 0x3);
        d_of_cur = d_next;
        sc = nx;
        nx.advance(cstep);
        ++u;
      }
      tcp::mma_commit_pair(drain_bar, 0x1);
      mbar_wait_timeout(drain_bar, 0);
    } else if (lane == 0) {
      // ---------------- follower: forward the epilogue's releases to the leader
      int dcount = 0;
      Sched sc;
      sc.init(sp, cstart);
      for (int u = 0;; ++u) {
        if (sc.valid) {
          bool dfull;
          if (sc.d_blocks(&dfull) > 0) {
            if (!mbar_wait_bounded(ddone_bar, static_cast<uint32_t>(dcount & 1), status, abort_flag))
              break;
            tc_fence_before();
            mbar_arrive_cluster(map_to_rank(ddone_bar, 0));
            ++dcount;
          }
        }
        if (u >= 1) {
          const int v = u - 1;
          if (!mbar_wait_bounded(tempty_bar(v & 1), (v >> 1) & 1, status, abort_flag)) break;
          tc_fence_before();
          mbar_arrive_cluster(map_to_rank(tempty_bar(v & 1), 0));
        }
        if (!sc.valid) break;
        sc.advance(cstep);
      }
    }
  } else {
    // ---------------- epilogue (both CTAs)
    const int quarter = warp & 3;
    const int group = (warp - 2) >> 2;  // chunks group, group + kGroups, ...
    const int L = quarter * 32 + lane;  // TMEM lane = A row of this CTA
    const int a = L & 1;
    const int32_t *__restrict__ rtab = args.rtab;
    const float *__restrict__ wv = args.t.w;
    int4 *__restrict__ tally_out = reinterpret_cast<int4 *>(args.t.tally);
    float4 *__restrict__ ccc_out = reinterpret_cast<float4 *>(args.t.ccc);
    constexpr bool want_ccc = MODE != 0;
    constexpr bool persnp = MODE == 1;
    const float gamma = args.t.gamma;
    const int64_t s_begin = slab_offset_dev(args.t.j_begin, n_v);
    const uint32_t lane_base = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16);
    const uint64_t keep_pol = l2_evict_last_policy();
    // r_ik staging of this warp: row il (SNP i = the warp's first + il) at
    // rbuf + il kRowStride, pair (i, kc + kk) at + 16 kk.
    const uint32_t rbuf =
        static_cast<uint32_t>(((smem_u32(tmem_slot) + 64 + 15) & ~15u) +
                              static_cast<uint32_t>(warp - 2) * wide::kRbufBytes);
    // Asynchronous copies of the r_ik of chunk c of tile t for this warp's rows:
    // lane copies pair lane % 8 of rows lane / 8 + 4 m, m = 0..3, 16 bytes each;
    // none for rows i >= j or pairs past n_v.
    auto issue_rows = [&](const Sched &t, int c) {
      const int64_t kk = t.k0() + 8 * c + (lane & 7);  // this lane's pair column, in every piece
      int64_t ii = t.i0() + 64 * static_cast<int64_t>(rank) + 16 * quarter + (lane >> 3);
      int64_t pb = ii * (2 * n_v - ii - 1) / 2 - ii - 1;  // pair (ii, k) at pb + k
      uint32_t dst = rbuf + static_cast<uint32_t>(lane >> 3) * wide::kRowStride +
                     16u * static_cast<uint32_t>(lane & 7);
#pragma unroll 1
      for (int m = 0; m < 4; ++m) {  // rows lane / 8 + 4 m
        if (ii < t.j && kk < n_v)
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                       "l"(rtab + 4 * (pb + kk))
                       : "memory");
        pb += 4 * n_v - 4 * ii - 14;  // pb(ii + 4) = pb(ii) + sum of n_v - i - 2 over 4 rows
        ii += 4;
        dst += 4 * wide::kRowStride;
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int dcount = 0;
    bool ok_all = true;
    Sched sc, pv;
    bool pv_has_d = false;
    sc.init(sp, cstart);
    for (int u = 0; ok_all; ++u) {
      if (u >= 1) issue_rows(pv, group);  // the first chunk of tile u - 1, processed in (2)
      // (1) move the D accumulator of tile u to this thread's shared-memory slot
      bool cur_has_d = false;
      if (sc.valid) {
        bool dfull;
        cur_has_d = sc.d_blocks(&dfull) > 0;
        if (cur_has_d) {
          const bool got = mbar_wait_bounded(dready_bar, static_cast<uint32_t>(dcount & 1), status,
                                             abort_flag);
          if (!__all_sync(0xffffffffu, got)) break;
          tc_fence_after();
          uint32_t *slot = dsc + (u & 1) * kDWords;
#pragma unroll 1
          for (int c = group; c < kChunks; c += wide::kGroups) {
            uint32_t v[16];
            tmem_ld_32x32b_x16(lane_base + (u & 1) * kN + 16 * c, v);
            tmem_ld_wait();
#pragma unroll
            for (int e = 0; e < 8; ++e) {
              const uint32_t d0 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[2 * e])));
              const uint32_t d1 = static_cast<uint32_t>(__float2int_rn(__uint_as_float(v[2 * e + 1])));
              st_l2_keep(slot + (8 * c + e) * 128 + L, (d0 & 0xFFFFu) | (d1 << 16), keep_pol);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(ddone_bar);  // the follower's is forwarded by warp 1
          ++dcount;
        }
      }
      // (2) the tallies and CCC values of tile u - 1
      if (u >= 1) {
        const int v = u - 1;
        const int acc = v & 1;
        const bool got = mbar_wait_bounded(tfull_bar(acc), (v >> 1) & 1, status, abort_flag);
        if (!__all_sync(0xffffffffu, got)) break;
        tc_fence_after();
        const int64_t j = pv.j;
        const int64_t i = pv.i0() + 64 * static_cast<int64_t>(rank) + (L >> 1);
        const bool row_ok = i < j;
        const int64_t k_first = pv.k0();
        const uint32_t t_x = lane_base + acc * kN;
        const uint32_t *slot = dsc + acc * kDWords;
        const int64_t span = n_v - 1 - j;
        const int64_t base = slab_offset_dev(j, n_v) - s_begin + i * span - (j + 1);
        const int64_t pbase = i * (2 * n_v - i - 1) / 2 - i - 1;  // pair (i, k) at pbase + k
        float wi = 1.f, wj0 = 1.f, wj1 = 1.f;
        if (want_ccc && persnp) {
          if (row_ok) wi = __ldg(wv + 2 * i + a);
          wj0 = __ldg(wv + 2 * j);
          wj1 = __ldg(wv + 2 * j + 1);
        }
        constexpr int KC = 8;  // SNPs k per chunk (16 accumulator columns)
        const int c_last = group + wide::kGroups * ((kChunks - 1 - group) / wide::kGroups);
        for (int c = group; c < kChunks; c += wide::kGroups) {
          const int kl = KC * c;  // first local SNP k of the chunk
          const int64_t kc = k_first + kl;
          uint32_t x[2 * KC];
          tmem_ld_32x32b_x16(t_x + 2 * kl, x);
          int2 r[KC];
          float2 wk[KC];
          uint32_t dd[KC];
#pragma unroll
          for (int kk = 0; kk < KC; ++kk) {
            const int64_t k = kc + kk;
            const bool ok = row_ok && k < n_v;
            wk[kk] = (ok && want_ccc && persnp) ? __ldg(reinterpret_cast<const float2 *>(wv) + k)
                                                : make_float2(1.f, 1.f);
            dd[kk] = pv_has_d ? ld_l2_keep(slot + (kl + kk) * 128 + L, keep_pol) : 0u;
          }
          asm volatile("cp.async.wait_group 0;" ::: "memory");
          __syncwarp();  // every lane's copies of the chunk have landed
          const uint32_t rrow = rbuf + static_cast<uint32_t>((L >> 1) & 15) * wide::kRowStride +
                                8u * static_cast<uint32_t>(a);
#pragma unroll
          for (int kk = 0; kk < KC; ++kk) {
            const bool ok = row_ok && kc + kk < n_v &&
                            CCC_IN_BOUNDS(pbase + kc + kk, n_v * (n_v - 1) / 2, args.t.status);
            int2 v;
            asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];"
                         : "=r"(v.x), "=r"(v.y)
                         : "r"(rrow + 16u * kk)
                         : "memory");
            r[kk] = ok ? v : make_int2(0, 0);
          }
          // The buffer takes the next chunk's rows once every lane has read it.
          __syncwarp();
          if (c + wide::kGroups < kChunks) issue_rows(pv, c + wide::kGroups);
          tmem_ld_wait();
          if (c == c_last) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(acc));  // the follower's is forwarded
          }
#pragma unroll
          for (int kk = 0; kk < KC; ++kk) {
            const int64_t k = kc + kk;
            const bool ok = row_ok && k < n_v && CCC_IN_BOUNDS(base + k, args.t.out_len, args.t.status);
            const int32_t t0 = __float2int_rn(__uint_as_float(x[2 * kk]));
            const int32_t t1 = __float2int_rn(__uint_as_float(x[2 * kk + 1]));
            const int32_t d0 = static_cast<int32_t>(dd[kk] & 0xFFFFu);
            const int32_t d1 = static_cast<int32_t>(dd[kk] >> 16);
            const int32_t u0 = r[kk].x - d0, u1 = r[kk].y - d1;
            // r^{a b c}: b0c0, b0c1, b1c0, b1c1
            const int4 tv = make_int4(u0 + t0, u1 + t1, u0 - t0, u1 - t1);
            const int64_t t = base + k;
            if (ok) __stcs(tally_out + 2 * t + a, tv);
            if (want_ccc) {
              const int32_t own = tv.x + tv.y + tv.z + tv.w;  // sum over b, c (fixed a)
              const int32_t n8 = own + __shfl_xor_sync(0xffffffffu, own, 1);
              int32_t rb0 = 0, rb1 = 0, q0 = 0, q1 = 0;
              if constexpr (!persnp) {
                const int32_t b0 = tv.x + tv.y, b1 = tv.z + tv.w;
                const int32_t c0 = tv.x + tv.z, c1 = tv.y + tv.w;
                rb0 = b0 + __shfl_xor_sync(0xffffffffu, b0, 1);
                rb1 = b1 + __shfl_xor_sync(0xffffffffu, b1, 1);
                q0 = c0 + __shfl_xor_sync(0xffffffffu, c0, 1);
                q1 = c1 + __shfl_xor_sync(0xffffffffu, c1, 1);
              }
              if (ok) {
                float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
                if (n8 != 0) {
                  const float dn = static_cast<float>(n8);
                  float fi = wi, fj0 = wj0, fj1 = wj1, fk0 = wk[kk].x, fk1 = wk[kk].y;
                  if (!persnp) {
                    fi = joint_factor(own, dn, gamma);
                    fj0 = joint_factor(rb0, dn, gamma);
                    fj1 = joint_factor(rb1, dn, gamma);
                    fk0 = joint_factor(q0, dn, gamma);
                    fk1 = joint_factor(q1, dn, gamma);
                  }
                  if (persnp) {
                    const float inv = __frcp_rn(dn);
                    const float g0 = __fmul_rn(fi, fj0), g1 = __fmul_rn(fi, fj1);
                    out.x = ccc3_persnp(tv.x, inv, g0, fk0);
                    out.y = ccc3_persnp(tv.y, inv, g0, fk1);
                    out.z = ccc3_persnp(tv.z, inv, g1, fk0);
                    out.w = ccc3_persnp(tv.w, inv, g1, fk1);
                  } else {
                    out.x = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(tv.x), dn), fi), fj0), fk0);
                    out.y = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(tv.y), dn), fi), fj0), fk1);
                    out.z = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(tv.z), dn), fi), fj1), fk0);
                    out.w = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(tv.w), dn), fi), fj1), fk1);
                  }
                }
                __stcs(ccc_out + 2 * t + a, out);
              }
            }
          }
        }
      }
      if (!sc.valid) break;
      pv = sc;
      pv_has_d = cur_has_d;
      sc.advance(cstep);
    }
    // Copies still in flight (after a wait that gave up) land before the CTA exits.
    asm volatile("cp.async.wait_all;" ::: "memory");
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  if (warp == 1) tcp::tmem_dealloc_pair(tmem_base, 512);
}

// Per slab j of [j0, j0 + gridDim.x): the individuals with v_j missing (first
// kCap of them, in order) and their count; when there are at most kCap, the
// rows 2 s + x (x = allele) of every SNP s restricted to those individuals,
// as e4m3 counts rho_s(x), zero-padded to a multiple of 128 columns:
// cbuf[(slab * 2 n_v + 2 s + x) * kCap + column].
// 128-thread CTAs with few registers: they fit beside a resident class-kernel
// CTA (its warps leave under 2K registers on some SM sub-partitions), so the
// next batch's preparation overlaps the current batch's tallies.
constexpr int kPrepThreads = 128;

// FP4: the compacted rows in e2m1 nibbles, 256 individuals in 128 bytes per row.
template <bool FP4>
__global__ void __launch_bounds__(kPrepThreads, 9) k_compact3(const uint64_t *__restrict__ geno, int64_t n_f,
                                                  int64_t n_v, int64_t ld, int64_t j0,
                                                  uint8_t *__restrict__ cbuf,
                                                  int32_t *__restrict__ missing, int snps_per_cta) {
  __shared__ int pos[kCap];
  constexpr int kWarps = kPrepThreads / 32;
  __shared__ int warp_tot[kWarps];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t j = j0 + blockIdx.x;
  const int64_t nw = (n_f + 31) / 32;
  int running = 0;
  for (int64_t base = 0; base < nw; base += kPrepThreads) {
    const int64_t wi = base + tid;
    uint64_t miss = 0;
    if (wi < nw) {
      const uint64_t v = geno[j * ld + wi];
      uint64_t valid = kEven;
      const int64_t tail = n_f - wi * 32;
      if (tail < 32) valid &= (1ull << (2 * tail)) - 1ull;
      miss = (v >> 1) & ~v & valid;
    }
    const int c = __popcll(miss);
    int x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
      before += q < warp ? warp_tot[q] : 0;
      tot += warp_tot[q];
    }
    int o = running + before + x - c;
    while (miss != 0 && o < kCap) {
      const int b = __ffsll(static_cast<long long>(miss)) - 1;
      pos[o++] = static_cast<int>(wi * 32 + (b >> 1));
      miss &= miss - 1;
    }
    running += tot;
    __syncthreads();
  }
  if (blockIdx.y == 0 && tid == 0) missing[blockIdx.x] = running;
  if (running == 0 || running > kCap) return;
  const int64_t s_lo = static_cast<int64_t>(blockIdx.y) * snps_per_cta;
  const int64_t s_hi = s_lo + snps_per_cta < n_v ? s_lo + snps_per_cta : n_v;
  // Code of compacted column idx of SNP s (missing past the count: both counts 0).
  auto code_at = [&](int64_t s, int idx) -> uint32_t {
    if (idx >= running) return 2u;
    const int q = pos[idx];
    return static_cast<uint32_t>(__ldg(geno + s * ld + (q >> 5)) >> (2 * (q & 31))) & 3u;
  };
  if constexpr (FP4) {
    // e2m1 nibbles: 0 -> 0x0, 1 -> 0x2, 2 -> 0x4; column idx in the low nibble of
    // byte idx / 2 for even idx.  One K stage of 256 individuals = 128 bytes.
    constexpr int kRow = kCap / 2;
    const int nbytes = (running + 255) / 256 * 128;
    for (int64_t s = s_lo + warp; s < s_hi; s += kWarps) {
      uint8_t *row0 = cbuf + (static_cast<int64_t>(blockIdx.x) * 2 * n_v + 2 * s) * kRow;
      for (int b = lane; b < nbytes; b += 32) {
        uint32_t n0 = 0u, n1 = 0u;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t code = code_at(s, 2 * b + h);
          const uint32_t r0 = code == 0u ? 4u : (code == 1u ? 2u : 0u);
          const uint32_t r1 = code == 3u ? 4u : (code == 1u ? 2u : 0u);
          n0 |= r0 << (4 * h);
          n1 |= r1 << (4 * h);
        }
        row0[b] = static_cast<uint8_t>(n0);
        row0[kRow + b] = static_cast<uint8_t>(n1);
      }
    }
  } else {
    const int ncols = (running + kBK - 1) / kBK * kBK;
    for (int64_t s = s_lo + warp; s < s_hi; s += kWarps) {
      uint8_t *row0 = cbuf + (static_cast<int64_t>(blockIdx.x) * 2 * n_v + 2 * s) * kCap;
      for (int idx = lane; idx < ncols; idx += 32) {
        const uint32_t code = code_at(s, idx);
        // e4m3: 0 -> 0x00, 1 -> 0x38, 2 -> 0x40
        const uint8_t e0 = code == 0u ? 0x40 : (code == 1u ? 0x38 : 0x00);
        const uint8_t e1 = code == 3u ? 0x40 : (code == 1u ? 0x38 : 0x00);
        row0[idx] = e0;
        row0[kCap + idx] = e1;
      }
    }
  }
}

// Per-nibble masks of the 32 individuals of one packed code word w: keep
// nibble q = 0xF where the selected class holds for individual q (low nibble
// of byte q / 2 for even q, as the e2m1 operand rows store them), neg nibble q
// = 0x8 (the e2m1 sign bit) where the sign flips.
__device__ __forceinline__ uint64_t spread_2to4_64(uint32_t x32) {
  uint64_t x = x32;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  return x;
}

__device__ __forceinline__ void class_masks_e2m1(uint64_t w, bool missing_mode, uint32_t (&keep)[4],
                                                 uint32_t (&neg)[4]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t x = static_cast<uint32_t>(w >> (32 * h));
    uint32_t kb, nb;
    if (!missing_mode) {
      kb = ~(x ^ (x >> 1)) & 0x55555555u;  // codes 00 and 11 (homozygous)
      nb = x & (x >> 1) & 0x55555555u;     // code 11: s_j = -1
    } else {
      kb = (x >> 1) & ~x & 0x55555555u;  // code 10: missing
      nb = 0u;
    }
    const uint64_t yk = spread_2to4_64(kb);  // 1 in the low bit of each kept nibble
    const uint64_t yn = spread_2to4_64(nb);
    const uint64_t km = (yk << 4) - yk;     // 0xF per kept nibble
    const uint64_t nm = yn << 3;            // 0x8 per negated nibble
    keep[2 * h] = static_cast<uint32_t>(km);
    keep[2 * h + 1] = static_cast<uint32_t>(km >> 32);
    neg[2 * h] = static_cast<uint32_t>(nm);
    neg[2 * h + 1] = static_cast<uint32_t>(nm >> 32);
  }
}

// Masked rows of the slabs [j0, j0 + gridDim.y): for slab j, the SNPs s of
// its smaller side (s < j when 2 j <= n_v - 1, else s > j), rows
//   mrow(j) + 2 t + x             = R(s, x) * s_j        (t = index of s on that side)
//   mrow(j) + 2 side + 2 t + x    = R(s, x) * [v_j missing]  (only when v_j has
//                                                          more than kCap missing)
// in the operand buffer op (rows of kpad bytes; R occupies the first rows).
// A CTA takes every gridDim.x-th row of its slab; a thread 16 bytes at a time.
// FP4: e2m1 rows of kpad / 2 bytes, 16 bytes = the 32 individuals of one packed
// word; the sign of a nibble is its bit 3.
template <bool FP4>
__global__ void __launch_bounds__(kPrepThreads, 9) k_mask3c(const uint64_t *__restrict__ geno, int64_t n_f,
                                                int64_t n_v, int64_t ld, uint8_t *__restrict__ op,
                                                int64_t kpad, int64_t mrow0, int64_t j0,
                                                const int32_t *__restrict__ missing) {
  const int64_t j = j0 + blockIdx.y;
  const int64_t side = j < n_v - 1 - j ? j : n_v - 1 - j;
  const bool im = 2 * j <= n_v - 1;
  const bool dfull = __ldg(missing + blockIdx.y) > kCap;
  const int64_t rows = (dfull ? 4 : 2) * side;
  const int64_t row_bytes = FP4 ? kpad / 2 : kpad;
  const int chunks = static_cast<int>(row_bytes / 16);
  const int64_t mrow = mrow0 + 4 * (mask_prefix(j, n_v) - mask_prefix(j0, n_v));
  const int64_t words = (n_f + 31) / 32;
  const uint64_t *__restrict__ gj = geno + j * ld;
  // Rows r, r + gridDim.x, ... in groups of 4 so that 8 loads per thread are in flight.
  constexpr int kRows = 4;
  for (int64_t r0 = blockIdx.x; r0 < rows; r0 += static_cast<int64_t>(gridDim.x) * kRows) {
    const uint4 *src[kRows];
    uint4 *dst[kRows];
    bool dm[kRows], live[kRows];
#pragma unroll
    for (int u = 0; u < kRows; ++u) {
      const int64_t ru = r0 + static_cast<int64_t>(u) * gridDim.x;
      live[u] = ru < rows;
      const int64_t r = live[u] ? ru : r0;
      dm[u] = r >= 2 * side;
      const int64_t rt = dm[u] ? r - 2 * side : r;
      const int64_t sn = im ? (rt >> 1) : j + 1 + (rt >> 1);
      src[u] = reinterpret_cast<const uint4 *>(op + (2 * sn + (rt & 1)) * row_bytes);
      dst[u] = reinterpret_cast<uint4 *>(op + (mrow + r) * row_bytes);
    }
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
      uint32_t ks[4], ns[4], km[4], nm[4];
      if (FP4) {
        const uint64_t w = c < words ? __ldg(gj + c) : 0ull;
        class_masks_e2m1(w, false, ks, ns);
        class_masks_e2m1(w, true, km, nm);
      } else {
        const int wi = c >> 1;
        uint32_t w = 0u;
        if (wi < words) w = static_cast<uint32_t>(__ldg(gj + wi) >> (32 * (c & 1)));
        class_masks(w, false, ks, ns);
        class_masks(w, true, km, nm);
      }
      uint4 v[kRows];
#pragma unroll
      for (int u = 0; u < kRows; ++u) v[u] = live[u] ? __ldg(src[u] + c) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
      for (int u = 0; u < kRows; ++u) {
        if (!live[u]) continue;
        uint4 o;
        o.x = (v[u].x & (dm[u] ? km[0] : ks[0])) | (dm[u] ? nm[0] : ns[0]);
        o.y = (v[u].y & (dm[u] ? km[1] : ks[1])) | (dm[u] ? nm[1] : ns[1]);
        o.z = (v[u].z & (dm[u] ? km[2] : ks[2])) | (dm[u] ? nm[2] : ns[2]);
        o.w = (v[u].w & (dm[u] ? km[3] : ks[3])) | (dm[u] ? nm[3] : ns[3]);
        dst[u][c] = o;
      }
    }
  }
}

}  // namespace

int64_t tc3_class_cbuf_rows(int64_t n_slabs, int64_t n_v) { return n_slabs * 2 * n_v; }
int64_t tc3_class_cap() { return kCap; }
int64_t tc3_class_mask_rows(int64_t j0, int64_t j1, int64_t n_v) {
  return 4 * (mask_prefix(j1, n_v) - mask_prefix(j0, n_v));
}

int launch_compact3(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *cbuf,
                    int32_t *missing, int64_t j0, int64_t j1, cudaStream_t s, bool fp4) {
  if (j1 <= j0) return CCC_OK;
  const int snps_per_cta = 64;
  const dim3 grid(static_cast<unsigned>(j1 - j0), static_cast<unsigned>(cdiv(n_v, snps_per_cta)), 1);
  if (fp4)
    k_compact3<true><<<grid, kPrepThreads, 0, s>>>(geno, n_f, n_v, ld, j0, cbuf, missing,
                                                   snps_per_cta);
  else
    k_compact3<false><<<grid, kPrepThreads, 0, s>>>(geno, n_f, n_v, ld, j0, cbuf, missing,
                                                    snps_per_cta);
  return note_launch();
}

int launch_mask3c(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *op,
                  int64_t kpad, int64_t mrow0, const int32_t *missing, int64_t j0, int64_t j1,
                  cudaStream_t s, bool fp4) {
  if (j1 <= j0) return CCC_OK;
  // About 8 CTAs per SM in total; each slab's rows are spread over bx CTAs.
  int64_t bx = cdiv(8 * 160, j1 - j0);
  if (bx < 2) bx = 2;
  if (bx > 256) bx = 256;
  const dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(j1 - j0), 1);
  if (fp4 && kpad % 256 != 0) return CCC_EINVAL;
  if (fp4)
    k_mask3c<true><<<grid, kPrepThreads, 0, s>>>(geno, n_f, n_v, ld, op, kpad, mrow0, j0, missing);
  else
    k_mask3c<false><<<grid, kPrepThreads, 0, s>>>(geno, n_f, n_v, ld, op, kpad, mrow0, j0, missing);
  return note_launch();
}

// Wide tiles (k_tally3_class_w) when 4 n_f fits in 16 bits, else N = 160 tiles.
template <int MODE, bool FP4>
static int launch_wide_mode(const CUtensorMap &tmOp, const CUtensorMap &tmC, const ClassArgs &ca,
                            const typename wide::Cfg<FP4>::Sched::Params &sp, int64_t tiles,
                            int num_sms, cudaStream_t s) {
  static int max_clusters_dev[kMaxDevices] = {};
  const int dev_c = current_device();
  if (dev_c < 0) return CCC_ECUDA;
  int &max_clusters = max_clusters_dev[dev_c];
  if (max_clusters == 0) {
    if (cudaFuncSetAttribute(k_tally3_class_w<MODE, FP4>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(wide::kSmem)) != cudaSuccess)
      return CCC_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
    cfg.blockDim = dim3(wide::kThreads, 1, 1);
    cfg.dynamicSmemBytes = wide::kSmem;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_tally3_class_w<MODE, FP4>, &cfg) != cudaSuccess ||
        n < 1)
      return CCC_ECUDA;
    max_clusters = n < num_sms / 2 ? n : num_sms / 2;
    if (max_clusters > wide::kMaxCtas / 2) max_clusters = wide::kMaxCtas / 2;
  }
  const int64_t clusters = tiles < max_clusters ? tiles : max_clusters;
  k_tally3_class_w<MODE, FP4><<<static_cast<unsigned>(2 * clusters), wide::kThreads, wide::kSmem,
                                s>>>(tmOp, tmC, ca, sp);
  return note_launch();
}

// Wide tiles (k_tally3_class_w) when 4 n_f fits in 16 bits, else N = 160 tiles.
// fp4: op rows (R and the masked rows) of kpad / 2 bytes, compacted rows of
// kCap / 2 bytes, all e2m1.
template <bool FP4>
static int launch_tally3_class_w(const Tally3Args &a, const uint8_t *op, int64_t op_rows,
                                 int64_t mrow0, int64_t kpad, const int32_t *rtab,
                                 const uint8_t *cbuf, const int32_t *missing, uint32_t *dscratch,
                                 int64_t j0, int64_t j1, int num_sms, cudaStream_t s) {
  using C = wide::Cfg<FP4>;
  int64_t tiles = 0;
  for (int64_t j = j0; j < j1; ++j) tiles += cdiv(j, kSnpI) * cdiv(a.n_v - 1 - j, C::kSnpK);
  if (tiles == 0) return CCC_OK;
  if (FP4 && kpad % 256 != 0) return CCC_EINVAL;
  const int64_t row_bytes = FP4 ? kpad / 2 : kpad;
  CUtensorMap tmOp, tmC;
  const int64_t crows = tc3_class_cbuf_rows(j1 - j0, a.n_v);
  if (!tc::make_operand_map(&tmOp, op, op_rows, row_bytes, 128) ||
      !tc::make_operand_map(&tmC, cbuf, crows, FP4 ? kCap / 2 : kCap, 128))
    return CCC_ECUDA;
  ClassArgs ca;
  ca.t = a;
  ca.rtab = rtab;
  ca.dscratch = dscratch;
  typename C::Sched::Params sp;
  sp.j0 = static_cast<int>(j0);
  sp.j1 = static_cast<int>(j1);
  sp.n_v = static_cast<int>(a.n_v);
  sp.nkb = static_cast<int>(row_bytes / kBK);
  sp.mrow0 = static_cast<int>(mrow0);
  sp.missing = missing;
  if (a.ccc == nullptr) return launch_wide_mode<0, FP4>(tmOp, tmC, ca, sp, tiles, num_sms, s);
  if (a.norm == CCC_NORM_PERSNP)
    return launch_wide_mode<1, FP4>(tmOp, tmC, ca, sp, tiles, num_sms, s);
  return launch_wide_mode<2, FP4>(tmOp, tmC, ca, sp, tiles, num_sms, s);
}

int64_t tc3_class_dscratch_bytes() {
  return static_cast<int64_t>(wide::kMaxCtas) * 2 * wide::kDWords * 4;
}

int launch_tally3_class(const Tally3Args &a, const uint8_t *op, int64_t op_rows, int64_t mrow0,
                        int64_t kpad, const int32_t *rtab, const uint8_t *cbuf,
                        const int32_t *missing, uint32_t *dscratch, int64_t j0, int64_t j1,
                        int num_sms, cudaStream_t s, bool fp4) {
  if (j1 <= j0) return CCC_OK;
  if (fp4 && !(a.n_f <= kWideMaxNf && dscratch != nullptr)) return CCC_EUNSUPPORTED;
  if (a.n_f <= kWideMaxNf && dscratch != nullptr)
    return fp4 ? launch_tally3_class_w<true>(a, op, op_rows, mrow0, kpad, rtab, cbuf, missing,
                                             dscratch, j0, j1, num_sms, s)
               : launch_tally3_class_w<false>(a, op, op_rows, mrow0, kpad, rtab, cbuf, missing,
                                              dscratch, j0, j1, num_sms, s);
  static bool attr_set_dev[kMaxDevices] = {};
  const int dev_a = current_device();
  if (dev_a < 0) return CCC_ECUDA;
  bool &attr_set = attr_set_dev[dev_a];
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_tally3_class, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(kSmemBytes)) != cudaSuccess)
      return CCC_ECUDA;
    attr_set = true;
  }
  int64_t tiles = 0;
  for (int64_t j = j0; j < j1; ++j) tiles += cdiv(j, kSnpI) * cdiv(a.n_v - 1 - j, kSnpK);
  if (tiles == 0) return CCC_OK;
  CUtensorMap tmA, tmB, tmCA, tmCB;
  const int64_t crows = tc3_class_cbuf_rows(j1 - j0, a.n_v);
  if (!tc::make_operand_map(&tmA, op, op_rows, kpad, 128) ||
      !tc::make_operand_map(&tmB, op, op_rows, kpad, kBRows) ||
      !tc::make_operand_map(&tmCA, cbuf, crows, kCap, 128) ||
      !tc::make_operand_map(&tmCB, cbuf, crows, kCap, kBRows))
    return CCC_ECUDA;
  static int max_clusters_dev[kMaxDevices] = {};
  const int dev_c = current_device();
  if (dev_c < 0) return CCC_ECUDA;
  int &max_clusters = max_clusters_dev[dev_c];
  if (max_clusters == 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = kSmemBytes;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_tally3_class, &cfg) != cudaSuccess || n < 1)
      return CCC_ECUDA;
    max_clusters = n < num_sms / 2 ? n : num_sms / 2;
  }
  const int64_t clusters = tiles < max_clusters ? tiles : max_clusters;
  ClassArgs ca;
  ca.t = a;
  ca.rtab = rtab;
  ClassSched::Params sp;
  sp.j0 = static_cast<int>(j0);
  sp.j1 = static_cast<int>(j1);
  sp.n_v = static_cast<int>(a.n_v);
  sp.nkb = static_cast<int>(kpad / kBK);
  sp.mrow0 = static_cast<int>(mrow0);
  sp.missing = missing;
  k_tally3_class<<<static_cast<unsigned>(2 * clusters), kThreads, kSmemBytes, s>>>(tmA, tmB, tmCA,
                                                                                   tmCB, ca, sp);
  return note_launch();
}

}  // namespace ccc
