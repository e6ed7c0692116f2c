// 2-way tallies on the tcgen05 tensor cores with the CCC value fused into the
// epilogue.
//
// Sec. 3.1 observes that the 2-way tallies have the shape of a GEMM,
// B = V^T o_2 V, with the scalar product replaced by a 2x2 tally.  Writing each
// SNP vector as two count rows, rho_i(0) and rho_i(1) (Sec. 2.1), turns the
// tally into a plain product: r_ij^{ab} = sum_q rho_{i,q}(a) rho_{j,q}(b) is
// entry (2i+a, 2j+b) of the Gram matrix R R^T of the (2 n_v) x n_f count
// matrix R.  Counts 0, 1, 2 are exact in e4m3 and every partial sum stays an
// integer below 2^24, so the FP32 accumulation of kind::f8f6f4 is exact.
//
// Only tiles of the upper triangle are computed (the symmetry of Sec. 2.1);
// pairs i >= j inside diagonal tiles are masked in the epilogue.  A tile is
// 128 operand rows (64 SNPs i) by 256 operand rows (128 SNPs j); the tiles are
// visited in groups of 8 column blocks, rows inside a group in increasing
// order, so that the tiles running at the same time share operand blocks in L2.
#include "ccc_launch.h"
#include "ccc_metric.cuh"
#include "tc_pipeline.cuh"
#include "tc_pipeline_pair.cuh"
#include "tc_sched.cuh"

#include <string.h>

namespace ccc {
namespace {

using namespace tc;

constexpr int SNP_I = BM / 2;
constexpr int SNP_J = BN / 2;

// Row / column block of a tile as the 2-way epilogue sees it: I in 64-SNP
// units (A rows 128 I ..), J in 128-SNP units (B rows 256 J ..).
struct Tile2 {
  int I, J;
};

struct Epi2 {
  using Params = Tally2Args;

  template <int NC>
  __device__ static void tile(const Params &args, const TriSched &sc, int quarter, int lane,
                              uint32_t t_base, uint32_t release_bar, int c0) {
    body<NC, false>(args, Tile2{sc.I, sc.J}, quarter, lane, t_base, release_bar, c0);
  }

  // Accumulator lane = A row (2i + a) of the tile, column = 2j + b.  The
  // release arrive goes to a CTA-local barrier, or (CLUSTER) to a barrier given
  // by its cluster address.  PRELOAD (cluster only): all NC chunks are loaded,
  // and the accumulator released, before the first is processed.
  template <int NC, bool CLUSTER, bool PRELOAD = false>
  __device__ static void body(const Params &args, Tile2 sc, int quarter, int lane,
                              uint32_t t_base, uint32_t release_bar, int c0) {
    const int row = quarter * 32 + lane;
    const int il = row >> 1;
    const int a = row & 1;
    const int64_t n_v = args.n_v;
    const int64_t i = static_cast<int64_t>(sc.I) * SNP_I + il;
    const bool filter = args.hits != nullptr;
    const bool want_ccc = filter || args.ccc != nullptr;
    float wi0 = 1.f, wi1 = 1.f;
    if (want_ccc && args.norm == CCC_NORM_PERSNP && i < n_v) {
      wi0 = __ldg(args.w + 2 * i);
      wi1 = __ldg(args.w + 2 * i + 1);
    }
    const int64_t row_base = i * (2 * n_v - i - 1) / 2 - i - 1;  // pair index = row_base + j
    if constexpr (PRELOAD) {
      static_assert(CLUSTER, "the preloading epilogue releases at cluster scope");
      uint32_t pre[NC][32];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) tmem_ld_32x32b_x32(t_base + (c0 + cc) * 32, pre[cc]);
      tmem_ld_wait();
      tc_fence_before();
      mbar_arrive_cluster(release_bar);
#pragma unroll
      for (int cc = 0; cc < NC; ++cc)
        chunk(args, sc, a, i, row_base, wi0, wi1, filter, want_ccc, c0 + cc, pre[cc]);
    } else {
      for (int c = c0; c < c0 + NC; ++c) {
        uint32_t v[32];
        tmem_ld_32x32b_x32(t_base + c * 32, v);
        tmem_ld_wait();
        if (c == c0 + NC - 1) {
          tc_fence_before();
          if (CLUSTER)
            mbar_arrive_cluster(release_bar);
          else
            mbar_arrive(release_bar);
        }
        chunk(args, sc, a, i, row_base, wi0, wi1, filter, want_ccc, c, v);
      }
    }
  }

  // The 32 columns of chunk c of lane (i, a): 16 SNPs j, tallies and CCC values.
  __device__ __forceinline__ static void chunk(const Params &args, Tile2 sc, int a, int64_t i,
                                               int64_t row_base, float wi0, float wi1, bool filter,
                                               bool want_ccc, int c, const uint32_t (&v)[32]) {
    cols<32>(args, static_cast<int64_t>(sc.J) * SNP_J + c * 16, a, i, row_base, wi0, wi1, filter,
             want_ccc, v);
  }

  // W accumulator columns of lane (i, a) whose first column is (SNP jb, b = 0):
  // W / 2 SNPs j, tallies and CCC values.
  template <int W>
  __device__ __forceinline__ static void cols(const Params &args, int64_t jb, int a, int64_t i,
                                              int64_t row_base, float wi0, float wi1, bool filter,
                                              bool want_ccc, const uint32_t (&v)[W]) {
    const int64_t n_v = args.n_v;
#pragma unroll
    for (int p = 0; p < W / 4; ++p) {
      // columns 4p, 4p+1: j even (b = 0, 1); columns 4p+2, 4p+3: j odd.
      const float e0 = __uint_as_float(v[4 * p + 0]);
      const float e1 = __uint_as_float(v[4 * p + 1]);
      const float o0 = __uint_as_float(v[4 * p + 2]);
      const float o1 = __uint_as_float(v[4 * p + 3]);
      // Allele-0 rows keep the even j and take the partner's (r10, r11);
      // allele-1 rows keep the odd j and take the partner's (r00, r01).
      const float g0 = __shfl_xor_sync(0xffffffffu, a ? e0 : o0, 1);
      const float g1 = __shfl_xor_sync(0xffffffffu, a ? e1 : o1, 1);
      int32_t r00, r01, r10, r11;
      if (a == 0) {
        r00 = __float2int_rn(e0);
        r01 = __float2int_rn(e1);
        r10 = __float2int_rn(g0);
        r11 = __float2int_rn(g1);
      } else {
        r00 = __float2int_rn(g0);
        r01 = __float2int_rn(g1);
        r10 = __float2int_rn(o0);
        r11 = __float2int_rn(o1);
      }
      const int64_t j = jb + 2 * p + a;
      if (i < j && j < n_v && i >= args.i_begin && i < args.i_end) {
        const int64_t pidx = row_base + j - args.pair0;
        if (!filter && !CCC_IN_BOUNDS(pidx, args.out_len, args.status)) continue;
        // Streaming stores: the output passes through L2 once and should not
        // evict the operand blocks that other tiles still read.
        if (!filter) __stcs(reinterpret_cast<int4 *>(args.tally) + pidx, make_int4(r00, r01, r10, r11));
        if (want_ccc) {
          float wj0 = 1.f, wj1 = 1.f;
          if (args.norm == CCC_NORM_PERSNP) {
            const float2 wj = __ldg(reinterpret_cast<const float2 *>(args.w) + j);
            wj0 = wj.x;
            wj1 = wj.y;
          }
          // Thresholded output: most pairs are ruled out without a division.
          const bool skip = filter && args.norm == CCC_NORM_PERSNP &&
                            !may_exceed(r00, r01, r10, r11, wi0, wi1, wj0, wj1, args.threshold);
          if (!skip) {
            const float4 cv =
                ccc2_values(r00, r01, r10, r11, wi0, wi1, wj0, wj1, args.norm, args.gamma);
            if (filter)
              filter_pair(args.hits, args.n_hits, args.cap, args.threshold, i, j, r00, r01, r10,
                          r11, cv);
            else
              __stcs(reinterpret_cast<float4 *>(args.ccc) + pidx, cv);
          }
        }
      }
    }
  }
};

// SM-pair epilogue with the chunk staged in shared memory.  Lane (2i + a)
// holds row (i, a) of a 32 x 32 accumulator chunk (16 SNPs i x 16 SNPs j);
// written row by row to `stage` (stride 33 floats, no bank conflicts), it is
// read back so that in store t lanes 0-15 and 16-31 each take 16 consecutive
// j of one SNP i: every warp store then covers two 256-byte runs of the
// output instead of sixteen 32-byte ones (GB300, 20,000 x 16,384: 6.32 against
// 6.37 ms per launch; thresholded output, which stores few pairs, keeps the
// unstaged body: staging made it 5% slower).
struct Epi2Staged {
  static constexpr int STRIDE = 33;
  static constexpr int STAGE_BYTES_PER_WARP = 32 * STRIDE * 4;

  // PRELOAD: all NC chunks are loaded, and the accumulator released, before
  // the first is processed.
  template <int NC, bool PRELOAD = false>
  __device__ static void body(const Tally2Args &args, Tile2 sc, int quarter, int lane,
                              uint32_t t_base, uint32_t release_cluster_bar, int c0,
                              float *stage) {
    if constexpr (PRELOAD) {
      uint32_t pre[NC][32];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) tmem_ld_32x32b_x32(t_base + (c0 + cc) * 32, pre[cc]);
      tmem_ld_wait();
      tc_fence_before();
      mbar_arrive_cluster(release_cluster_bar);
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) chunk(args, sc, quarter, lane, c0 + cc, pre[cc], stage);
    } else {
      for (int c = c0; c < c0 + NC; ++c) {
        uint32_t v[32];
        tmem_ld_32x32b_x32(t_base + c * 32, v);
        tmem_ld_wait();
        if (c == c0 + NC - 1) {
          tc_fence_before();
          mbar_arrive_cluster(release_cluster_bar);
        }
        chunk(args, sc, quarter, lane, c, v, stage);
      }
    }
  }

  __device__ __forceinline__ static void chunk(const Tally2Args &args, Tile2 sc, int quarter,
                                               int lane, int c, const uint32_t (&v)[32],
                                               float *stage) {
    at(args, static_cast<int64_t>(sc.I) * SNP_I + quarter * 16,
       static_cast<int64_t>(sc.J) * SNP_J + c * 16, lane, v, stage);
  }

  // The 32 x 32 chunk of SNPs i ib .. ib + 15 (lanes) and j jb .. jb + 15 (columns).
  __device__ __forceinline__ static void at(const Tally2Args &args, int64_t ib, int64_t jb,
                                            int lane, const uint32_t (&v)[32], float *stage) {
    const int64_t n_v = args.n_v;
    const bool filter = args.hits != nullptr;
    const bool want_ccc = filter || args.ccc != nullptr;
    const bool persnp = args.norm == CCC_NORM_PERSNP;
    const int jl = lane & 15;
    const int64_t i0 = ib + (lane >> 4);
    __syncwarp();  // the previous chunk's reads are done
#pragma unroll
    for (int k = 0; k < 32; ++k) stage[lane * STRIDE + k] = __uint_as_float(v[k]);
    __syncwarp();
    const int64_t j = jb + jl;
    float wj0 = 1.f, wj1 = 1.f;
    if (want_ccc && persnp && j < n_v) {
      const float2 wj = __ldg(reinterpret_cast<const float2 *>(args.w) + j);
      wj0 = wj.x;
      wj1 = wj.y;
    }
#pragma unroll 2
    for (int t = 0; t < 8; ++t) {
      const int il = 2 * t + (lane >> 4);  // SNP i of this store within the chunk's 16
      const int64_t i = i0 + 2 * t;
      const float *r0 = stage + (2 * il) * STRIDE + 2 * jl;  // row (i, 0)
      const float *r1 = r0 + STRIDE;                          // row (i, 1)
      const int32_t r00 = __float2int_rn(r0[0]);
      const int32_t r01 = __float2int_rn(r0[1]);
      const int32_t r10 = __float2int_rn(r1[0]);
      const int32_t r11 = __float2int_rn(r1[1]);
      if (!(i < j && j < n_v && i >= args.i_begin && i < args.i_end)) continue;
      const int64_t pidx = i * (2 * n_v - i - 1) / 2 - i - 1 + j - args.pair0;
      if (!filter && !CCC_IN_BOUNDS(pidx, args.out_len, args.status)) continue;
      if (!filter) __stcs(reinterpret_cast<int4 *>(args.tally) + pidx, make_int4(r00, r01, r10, r11));
      if (!want_ccc) continue;
      float wi0 = 1.f, wi1 = 1.f;
      if (persnp) {
        const float2 wi = __ldg(reinterpret_cast<const float2 *>(args.w) + i);
        wi0 = wi.x;
        wi1 = wi.y;
      }
      const bool skip = filter && persnp &&
                        !may_exceed(r00, r01, r10, r11, wi0, wi1, wj0, wj1, args.threshold);
      if (skip) continue;
      const float4 cv = ccc2_values(r00, r01, r10, r11, wi0, wi1, wj0, wj1, args.norm, args.gamma);
      if (filter)
        filter_pair(args.hits, args.n_hits, args.cap, args.threshold, i, j, r00, r01, r10, r11, cv);
      else
        __stcs(reinterpret_cast<float4 *>(args.ccc) + pidx, cv);
    }
  }
};

constexpr size_t pair_smem(int ew) { return tcp::smem_bytes(ew, Epi2Staged::STAGE_BYTES_PER_WARP); }
static_assert(pair_smem(8) <= 232448, "dynamic shared memory limit");

template <int EW>
__global__ void __launch_bounds__(64 + 32 * EW, 1)
    k_tally2_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const Tally2Args args, TriSched::Params sp, int nkb) {
  persistent_gemm<TriSched, Epi2, EW>(&tmA, &tmB, sp, args, nkb, args.status);
}

// ---------------------------------------------------------------- SM pairs

struct Epi2Pair {
  using Params = Tally2Args;
  static constexpr int STAGE_BYTES_PER_WARP = Epi2Staged::STAGE_BYTES_PER_WARP;
  template <int NC, bool PRELOAD = false>
  __device__ static void tile(const Params &args, const TriSchedPair &sc, int rank, int quarter,
                              int lane, uint32_t t_base, uint32_t release_cluster_bar, int c0,
                              float *stage) {
    if (args.hits != nullptr)  // thresholded output stores little: no staging
      Epi2::body<NC, true, PRELOAD>(args, Tile2{2 * sc.I + rank, sc.J}, quarter, lane, t_base,
                                    release_cluster_bar, c0);
    else
      Epi2Staged::body<NC, PRELOAD>(args, Tile2{2 * sc.I + rank, sc.J}, quarter, lane, t_base,
                                    release_cluster_bar, c0, stage);
  }
};

template <int EW>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * EW, 1)
    k_tally2_tc_pair(const __grid_constant__ CUtensorMap tm, const Tally2Args args,
                     TriSched::Params sp, int nkb) {
  tcp::persistent_gemm_pair<TriSchedPair, Epi2Pair, EW>(&tm, sp, args, nkb, args.status);
}

// FP4 (e2m1) operands: one accumulator, 8 epilogue warps that load their whole
// quarter-half before releasing it (tcp::persistent_gemm_pair, FP4).  Each
// epilogue thread holds 128 accumulator values.  The 10 warps of a CTA put 3
// warps on two of the SM's four sub-partitions, whose register files hold 16K
// registers each, so a thread may use at most 168 (3 x 32 x 168 <= 16,384):
// that is what __launch_bounds__(320, 1) gives, with a few dozen bytes spilled.
// A higher cap (183 registers, no spills) left no CTA resident.
// Default tile order of the FP4 kernels: groups of 16 column blocks (GB300,
// 20,000 x 16,384: 3.76 ms against 3.80 with 8, 3.82 with 32; 200,000 x 4,096
// thresholded: 121 against 127 ms with 8, 125 with 32).
constexpr int kFp4Group = 16;
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * tcp::FP4_EW, 1)
    k_tally2_tc_pair_fp4(const __grid_constant__ CUtensorMap tm, const Tally2Args args,
                         TriSched::Params sp, int nkb) {
  tcp::persistent_gemm_pair<TriSchedPair, Epi2Pair, tcp::FP4_EW, false, true>(&tm, sp, args, nkb,
                                                                              args.status);
}

// Thresholded FP4 output with two accumulators: tiles of 128 SNPs i by
// kRectJ = 120 SNPs j (N = 240 columns, B rows 120 per CTA), so that two
// accumulators and the scale factors fill the 512 TMEM columns and the MMAs of
// a tile run while the epilogue tests the previous one.  Tiles over
// RectSchedT<128, 120, 240>; A through maps.m[0] (box 128 rows), B through maps.m[1]
// (box 120 rows).  Per column the MMA is 1.4% slower at N = 240 (153.8 cycles
// per instruction against 161.8 at N = 256), and the tiles are 6.6% more per
// triangle, but at short K the single-accumulator kernel above waits for its
// epilogue's read-out on every tile: GB300, 200,000 x 4,096 thresholded,
// 104.2 ms (109.3 with the tile order of the full-output kernel) against 119.9.  Full output stays on the single-accumulator kernel,
// whose epilogue stores interleave with the next tile's MMAs there as well
// (20,000 x 16,384: 3.64 ms against 3.81 with these tiles; x 32,768: 6.67
// against 7.15).
constexpr int kRectJ = 120;
constexpr int kRectNB = 2 * kRectJ;
// Default tile order of the rect kernel: groups of 64 column blocks (GB300,
// 200,000 x 4,096 thresholded: 104.9 ms against 109.4 with 16, 116.8 with 8,
// 104.3 with 128; at 50,000 x 4,096 it read 0.84 GB of DRAM per launch against
// 2.70 GB with 16 and 7.9 GB with 256, whose column group of 123 MB of operand
// rows no longer stays in L2 while the row blocks stream past).
constexpr int kFp4RectGroup = 64;

struct PairMaps {
  CUtensorMap m[2];
};

// Epilogue of a rect tile (thresholded output only): 7 chunks of 32 columns
// (16 SNPs j) and a 16-column tail (8 SNPs j) at column 224; the warps of
// column half 0 take chunks 0-3, those of half 1 chunks 4-6 and the tail, with
// two TMEM loads per wait, releasing the accumulator after their last load.
// The epilogue is what bounds this kernel at short K (about 10,000 cycles of
// MMAs per tile at K = 4,096), so each pair is tested with the accumulator's
// float values and factors staged in shared memory before any integer or
// division work.
struct Epi2Rect {
  using Params = Tally2Args;
  using Sched = RectSchedT<128, kRectJ, kRectNB>;
  static constexpr int STAGE_BYTES_PER_WARP = kRectJ * 8;  // float2 factors of the tile's j
  static constexpr int CHUNKS = kRectJ / 16;  // whole 32-column chunks
  static constexpr int TAIL = kRectNB - 32 * CHUNKS;
  static_assert(TAIL == 16 && CHUNKS == 7, "chunks 0-3, 4-6 and a 16-column tail");
  static_assert(STAGE_BYTES_PER_WARP % 16 == 0, "16-byte staged rows");

  template <int NC, bool PRELOAD>
  __device__ static void tile(const Params &args, const Sched &sc, int rank, int quarter, int lane,
                              uint32_t t_base, uint32_t release_cluster_bar, int c0,
                              float *stage) {
    static_assert(!PRELOAD, "two accumulators: each warp releases after its last load");
    const int half = c0 / NC;
    const int64_t ib = static_cast<int64_t>(2 * sc.I + rank) * SNP_I;  // the CTA's first SNP i
    const int64_t j0 = static_cast<int64_t>(sc.J) * kRectJ;
    if (args.hits == nullptr) {  // launched for thresholded output only
      record_error(args.status, CCC_EINVAL);
      release(release_cluster_bar);
      return;
    }
    filter_tile(args, ib, j0, quarter, lane, t_base, release_cluster_bar, half, stage);
  }

  __device__ __forceinline__ static void release(uint32_t bar) {
    tc_fence_before();
    mbar_arrive_cluster(bar);
  }

  // Thresholded output: lane = row (i, a).  For each pair of the lane's row, its
  // own row's largest weighted entry and sum are exchanged with the partner row
  // (lane ^ 1); only pairs that may exceed the threshold (PERSNP, see
  // may_exceed; every pair for JOINT) go through the integer tallies, the CCC
  // values and filter_pair, so the hit list is what Epi2 produces.
  __device__ static void filter_tile(const Params &args, int64_t ib, int64_t j0, int quarter,
                                     int lane, uint32_t t_base, uint32_t rel, int half,
                                     float *stage) {
    const int64_t n_v = args.n_v;
    const int row = quarter * 32 + lane;
    const int a = row & 1;
    const int64_t i = ib + (row >> 1);
    const bool persnp = args.norm == CCC_NORM_PERSNP;
    float wi0 = 1.f, wi1 = 1.f;
    if (persnp && i < n_v) {
      wi0 = __ldg(args.w + 2 * i);
      wi1 = __ldg(args.w + 2 * i + 1);
    }
    const bool rowok = i < n_v && i >= args.i_begin && i < args.i_end;
    // The factors of the tile's kRectJ SNPs j, in the warp's staging buffer
    // (read by every lane with the same address: broadcasts).
    float2 *wjs = reinterpret_cast<float2 *>(stage);
    const float2 *w2 = reinterpret_cast<const float2 *>(args.w);
    __syncwarp();  // the previous tile's reads are done
    for (int k = lane; k < kRectJ; k += 32) {
      const int64_t j = j0 + k;
      wjs[k] = persnp ? __ldg(w2 + (j < n_v ? j : n_v - 1)) : make_float2(1.f, 1.f);
    }
    __syncwarp();
    // Two TMEM loads per wait: the four pieces of a warp expose two load
    // latencies instead of four.
    const int cb = half ? 4 : 0;
    {
      uint32_t va[32], vb[32];
      tmem_ld_32x32b_x32(t_base + cb * 32, va);
      tmem_ld_32x32b_x32(t_base + (cb + 1) * 32, vb);
      tmem_ld_wait();
      filter_cols<32>(args, j0, 16 * cb, a, i, rowok, persnp, wi0, wi1, va, wjs);
      filter_cols<32>(args, j0, 16 * (cb + 1), a, i, rowok, persnp, wi0, wi1, vb, wjs);
    }
    if (half == 0) {
      uint32_t va[32], vb[32];
      tmem_ld_32x32b_x32(t_base + 2 * 32, va);
      tmem_ld_32x32b_x32(t_base + 3 * 32, vb);
      tmem_ld_wait();
      release(rel);
      filter_cols<32>(args, j0, 32, a, i, rowok, persnp, wi0, wi1, va, wjs);
      filter_cols<32>(args, j0, 48, a, i, rowok, persnp, wi0, wi1, vb, wjs);
    } else {
      uint32_t va[32], vt[TAIL];
      tmem_ld_32x32b_x32(t_base + 6 * 32, va);
      tmem_ld_32x32b_x16(t_base + 32 * CHUNKS, vt);
      tmem_ld_wait();
      release(rel);
      filter_cols<32>(args, j0, 96, a, i, rowok, persnp, wi0, wi1, va, wjs);
      filter_cols<TAIL>(args, j0, 16 * CHUNKS, a, i, rowok, persnp, wi0, wi1, vt, wjs);
    }
  }

  // W columns from SNP jb = j0 + jo on: columns 4p, 4p + 1 are (j = jb + 2p,
  // b = 0, 1), 4p + 2, 4p + 3 are (j = jb + 2p + 1, b = 0, 1); allele-0 rows take
  // the even j, allele-1 rows the odd j.  wjs[k]: factors of SNP j0 + k.
  template <int W>
  __device__ __forceinline__ static void filter_cols(const Params &args, int64_t j0, int jo, int a,
                                                     int64_t i, bool rowok, bool persnp, float wi0,
                                                     float wi1, const uint32_t (&v)[W],
                                                     const float2 *wjs) {
    constexpr int P = W / 4;
    const int64_t n_v = args.n_v;
    const int64_t jb = j0 + jo;
    const float wia = a ? wi1 : wi0;
    const float thr = args.threshold;
    float2 wje[P], wjo[P];  // factors of j = jb + 2p and jb + 2p + 1 (the same in every lane)
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const float4 q = *reinterpret_cast<const float4 *>(wjs + jo + 2 * p);
      wje[p] = make_float2(q.x, q.y);
      wjo[p] = make_float2(q.z, q.w);
    }
    uint32_t cand = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const float e0 = __uint_as_float(v[4 * p + 0]), e1 = __uint_as_float(v[4 * p + 1]);
      const float o0 = __uint_as_float(v[4 * p + 2]), o1 = __uint_as_float(v[4 * p + 3]);
      // this row's part of the pairs (i, j even) and (i, j odd): largest weighted entry, sum
      const float me = fmaxf(e0 * (wia * wje[p].x), e1 * (wia * wje[p].y));
      const float mo = fmaxf(o0 * (wia * wjo[p].x), o1 * (wia * wjo[p].y));
      const float se = e0 + e1, so = o0 + o1;
      const float pm = __shfl_xor_sync(0xffffffffu, a ? me : mo, 1);
      const float ps = __shfl_xor_sync(0xffffffffu, a ? se : so, 1);
      const int64_t j = jb + 2 * p + a;
      const float m = fmaxf(a ? mo : me, pm);
      const float n4 = (a ? so : se) + ps;  // 4 n_ij, an exact integer below 2^24
      const bool may = !persnp || m * (1.f + 0x1p-18f) >= thr * n4;
      cand |= (rowok && i < j && j < n_v && may ? 1u : 0u) << p;
    }
    if (!__any_sync(0xffffffffu, cand != 0)) return;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const float e0 = __uint_as_float(v[4 * p + 0]), e1 = __uint_as_float(v[4 * p + 1]);
      const float o0 = __uint_as_float(v[4 * p + 2]), o1 = __uint_as_float(v[4 * p + 3]);
      const float g0 = __shfl_xor_sync(0xffffffffu, a ? e0 : o0, 1);
      const float g1 = __shfl_xor_sync(0xffffffffu, a ? e1 : o1, 1);
      if (!((cand >> p) & 1u)) continue;
      int32_t r00, r01, r10, r11;
      if (a == 0) {
        r00 = __float2int_rn(e0);
        r01 = __float2int_rn(e1);
        r10 = __float2int_rn(g0);
        r11 = __float2int_rn(g1);
      } else {
        r00 = __float2int_rn(g0);
        r01 = __float2int_rn(g1);
        r10 = __float2int_rn(o0);
        r11 = __float2int_rn(o1);
      }
      const float2 wj = a ? wjo[p] : wje[p];
      if (persnp && !may_exceed(r00, r01, r10, r11, wi0, wi1, wj.x, wj.y, args.threshold)) continue;
      const float4 cv = ccc2_values(r00, r01, r10, r11, wi0, wi1, wj.x, wj.y, args.norm, args.gamma);
      filter_pair(args.hits, args.n_hits, args.cap, args.threshold, i, jb + 2 * p + a, r00, r01,
                  r10, r11, cv);
    }
  }
};

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * tcp::FP4_EW, 1)
    k_tally2_tc_pair_fp4w(const __grid_constant__ PairMaps maps, const Tally2Args args,
                          TriSched::Params sp, int nkb) {
  tcp::persistent_gemm_pair<Epi2Rect::Sched, Epi2Rect, tcp::FP4_EW, false, true, kRectNB>(
      maps.m, sp, args, nkb, args.status);
}

constexpr size_t rect_smem() {
  return tcp::smem_bytes_nb(kRectNB, tcp::FP4_EW, Epi2Rect::STAGE_BYTES_PER_WARP);
}
static_assert(rect_smem() <= 232448, "dynamic shared memory limit");

// ---------------------------------------------------------------- split K

// Partial tallies of one K part, added into the zeroed tally array with
// integer reductions (exact in any order); CCC values follow from the summed
// tallies in a separate pass.
struct Epi2Split {
  using Params = Tally2Args;
  static constexpr int STAGE_BYTES_PER_WARP = 0;
  template <int NC, bool PRELOAD = false>
  __device__ static void tile(const Params &args, const SplitSchedPair &sc, int rank, int quarter,
                              int lane, uint32_t t_base, uint32_t release_cluster_bar, int c0,
                              float *) {
    body<NC, PRELOAD>(args, Tile2{2 * sc.I + rank, sc.J}, quarter, lane, t_base,
                      release_cluster_bar, c0);
  }

  // sc: the CTA's 64-SNP row block I and the tile's 128-SNP column block J.
  template <int NC, bool PRELOAD = false>
  __device__ static void body(const Params &args, Tile2 sc, int quarter, int lane, uint32_t t_base,
                              uint32_t release_cluster_bar, int c0) {
    const int row = quarter * 32 + lane;
    const int a = row & 1;
    const int64_t i = static_cast<int64_t>(sc.I) * SNP_I + (row >> 1);
    const bool row_ok = i < args.n_v && i >= args.i_begin && i < args.i_end;
    const int64_t row_base = i * (2 * args.n_v - i - 1) / 2 - i - 1 - args.pair0;
    if constexpr (PRELOAD) {
      uint32_t pre[NC][32];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) tmem_ld_32x32b_x32(t_base + (c0 + cc) * 32, pre[cc]);
      tmem_ld_wait();
      tc_fence_before();
      mbar_arrive_cluster(release_cluster_bar);
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) chunk(args, sc, a, i, row_ok, row_base, c0 + cc, pre[cc]);
    } else {
      for (int c = c0; c < c0 + NC; ++c) {
        uint32_t v[32];
        tmem_ld_32x32b_x32(t_base + c * 32, v);
        tmem_ld_wait();
        if (c == c0 + NC - 1) {
          tc_fence_before();
          mbar_arrive_cluster(release_cluster_bar);
        }
        chunk(args, sc, a, i, row_ok, row_base, c, v);
      }
    }
  }

  __device__ __forceinline__ static void chunk(const Params &args, Tile2 sc, int a,
                                               int64_t i, bool row_ok, int64_t row_base, int c,
                                               const uint32_t (&v)[32]) {
#pragma unroll
    for (int col = 0; col < 32; ++col) {
      const int64_t j = static_cast<int64_t>(sc.J) * SNP_J + c * 16 + (col >> 1);
      const int32_t r = __float2int_rn(__uint_as_float(v[col]));
      if (row_ok && i < j && j < args.n_v && r != 0 &&
          CCC_IN_BOUNDS(row_base + j, args.out_len, args.status))
        atomicAdd(args.tally + (row_base + j) * 4 + 2 * a + (col & 1), r);
    }
  }
};

template <int EW>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * EW, 1)
    k_tally2_tc_pair_split(const __grid_constant__ CUtensorMap tm, const Tally2Args args,
                           SplitSchedPair::Params sp, int nkb) {
  tcp::persistent_gemm_pair<SplitSchedPair, Epi2Split, EW, true>(&tm, sp, args, nkb, args.status);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * tcp::FP4_EW, 1)
    k_tally2_tc_pair_split_fp4(const __grid_constant__ CUtensorMap tm, const Tally2Args args,
                               SplitSchedPair::Params sp, int nkb) {
  tcp::persistent_gemm_pair<SplitSchedPair, Epi2Split, tcp::FP4_EW, true, true>(&tm, sp, args, nkb,
                                                                                args.status);
}

// ---------------------------------------------------------------- packed operands

// The pair kernels with the 2-bit codes expanded into count rows in shared
// memory (tcp::persistent_gemm_pair_packed): no operand matrix in HBM.
template <int EW>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * EW + 32 * tcp::pk::CW, 1)
    k_tally2_tc_pair_packed(const __grid_constant__ CUtensorMap tmP, const Tally2Args args,
                            TriSched::Params sp, int nkb) {
  tcp::persistent_gemm_pair_packed<TriSchedPair, Epi2Pair, EW>(&tmP, sp, args, nkb, args.n_v,
                                                               args.n_f, args.status);
}

template <int EW>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * EW + 32 * tcp::pk::CW, 1)
    k_tally2_tc_pair_split_packed(const __grid_constant__ CUtensorMap tmP, const Tally2Args args,
                                  SplitSchedPair::Params sp, int nkb) {
  tcp::persistent_gemm_pair_packed<SplitSchedPair, Epi2Split, EW>(&tmP, sp, args, nkb, args.n_v,
                                                                  args.n_f, args.status);
}

constexpr size_t packed_smem(int ew) {
  return tcp::pk::smem_bytes(ew, Epi2Staged::STAGE_BYTES_PER_WARP);
}
static_assert(packed_smem(8) <= 232448, "dynamic shared memory limit");

// ---------------------------------------------------------------- batched panels

struct BatchPanel {
  Tally2Args args;
  TriSched::Params tri;
  int nkb;
  int split;      // K parts per tile (SM-pair launches; 1 = unsplit)
  int64_t tiles;  // tiles of the panel's triangle
};

struct BatchParams {
  int n;
  BatchPanel p[kMaxBatchPanels];
};

struct BatchMaps {
  CUtensorMap a[kMaxBatchPanels];
  CUtensorMap b[kMaxBatchPanels];
};

static_assert(sizeof(BatchParams) + sizeof(BatchMaps) < 32000, "kernel parameter space");

// All units of panel 0, then of panel 1, ...: the CTAs of one persistent
// launch share every panel's triangle, so small panels fill the SMs big ones
// leave idle.  A panel with split > 1 has tiles x split units, part-major as in
// SplitSchedPair (unit u = tile u % tiles, K part u / tiles).
template <class Inner>
struct BatchSchedT {
  using Params = BatchParams;
  const BatchParams *bp;
  int p;
  int64_t pos;  // unit position inside panel p
  Inner t;
  bool valid;

  __device__ int64_t units(int q) const { return bp->p[q].tiles * bp->p[q].split; }
  __device__ void start_panel() {
    while (p < bp->n && units(p) == 0) ++p;
    valid = p < bp->n;
    pos = 0;
    if (valid) t.init(bp->p[p].tri, 0);
  }
  __device__ void init(const Params &params, int64_t start) {
    bp = &params;
    p = 0;
    start_panel();
    advance(start);
  }
  __device__ void advance(int64_t step) {
    while (valid && step > 0) {
      const int64_t rem = units(p) - 1 - pos;
      if (step <= rem) {
        pos += step;
        if (bp->p[p].split == 1)
          t.advance(step);
        else
          t.init(bp->p[p].tri, pos % bp->p[p].tiles);
        return;
      }
      step -= rem + 1;
      ++p;
      start_panel();
    }
  }
  __device__ int part() const { return static_cast<int>(pos / bp->p[p].tiles); }
  __device__ int map_index() const { return p; }
  __device__ int k_begin() const {
    return static_cast<int>(static_cast<int64_t>(part()) * bp->p[p].nkb / bp->p[p].split);
  }
  __device__ int k_blocks(int) const {
    return static_cast<int>(static_cast<int64_t>(part() + 1) * bp->p[p].nkb / bp->p[p].split) -
           k_begin();
  }
  __device__ int a_row() const { return t.a_row(); }
  __device__ int b_row() const { return t.b_row(); }
};
using BatchSched = BatchSchedT<TriSched>;

struct BatchSchedPair : BatchSchedT<TriSchedPair> {};

struct EpiBatchPair {
  using Params = BatchParams;
  static constexpr int STAGE_BYTES_PER_WARP = Epi2Staged::STAGE_BYTES_PER_WARP;
  template <int NC, bool PRELOAD = false>
  __device__ static void tile(const Params &bp, const BatchSchedPair &sc, int rank, int quarter,
                              int lane, uint32_t t_base, uint32_t release_cluster_bar, int c0,
                              float *stage) {
    const BatchPanel &q = bp.p[sc.p];
    if (q.split > 1)  // a K part: partial tallies added into the zeroed output
      Epi2Split::body<NC, PRELOAD>(q.args, Tile2{2 * sc.t.I + rank, sc.t.J}, quarter, lane, t_base,
                                   release_cluster_bar, c0);
    else
      Epi2Staged::body<NC, PRELOAD>(q.args, Tile2{2 * sc.t.I + rank, sc.t.J}, quarter, lane,
                                    t_base, release_cluster_bar, c0, stage);
  }
};

template <int EW>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * EW, 1)
    k_tally2_tc_pair_batched(const __grid_constant__ BatchMaps maps,
                             const __grid_constant__ BatchParams bp) {
  tcp::persistent_gemm_pair<BatchSchedPair, EpiBatchPair, EW>(maps.a, bp, bp, 0,
                                                             bp.p[0].args.status);
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(64 + 32 * tcp::FP4_EW, 1)
    k_tally2_tc_pair_batched_fp4(const __grid_constant__ BatchMaps maps,
                                 const __grid_constant__ BatchParams bp) {
  tcp::persistent_gemm_pair<BatchSchedPair, EpiBatchPair, tcp::FP4_EW, false, true>(
      maps.a, bp, bp, 0, bp.p[0].args.status);
}

struct EpiBatch {
  using Params = BatchParams;
  template <int NC>
  __device__ static void tile(const Params &bp, const BatchSched &sc, int quarter, int lane,
                              uint32_t t_base, uint32_t release_bar, int c0) {
    Epi2::tile<NC>(bp.p[sc.p].args, sc.t, quarter, lane, t_base, release_bar, c0);
  }
};

template <int EW>
__global__ void __launch_bounds__(64 + 32 * EW, 1)
    k_tally2_tc_batched(const __grid_constant__ BatchMaps maps,
                        const __grid_constant__ BatchParams bp) {
  persistent_gemm<BatchSched, EpiBatch, EW>(maps.a, maps.b, bp, bp, 0, bp.p[0].args.status);
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int64_t tc2_num_tiles(int64_t n_v, int64_t I0 = 0, int64_t I1 = int64_t(1) << 40) {
  const int64_t nI = (n_v + SNP_I - 1) / SNP_I;
  const int64_t nJ = (n_v + SNP_J - 1) / SNP_J;
  int64_t t = 0;
  for (int64_t I = I0; I < nI && I < I1; ++I) t += nJ - (I >> 1);
  return t;
}

}  // namespace

namespace tc {

bool make_operand_map(CUtensorMap *map, const uint8_t *op, int64_t rows, int64_t kpad,
                      uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(kpad), static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(kpad)};
  const cuuint32_t box[2] = {128u, box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(op), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_blocked_operand_map(CUtensorMap *map, const uint8_t *op, int64_t rows, int64_t kpad,
                              uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  const cuuint64_t dims[3] = {128u, static_cast<cuuint64_t>(rows),
                              static_cast<cuuint64_t>(kpad / 128)};
  const cuuint64_t strides[2] = {128u, static_cast<cuuint64_t>(rows) * 128u};
  const cuuint32_t box[3] = {128u, box_rows, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t *>(op), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace tc

// Square 128-SNP tiles of the triangle (J >= I) in row blocks [I0, I1).
int64_t tc2_pair_tiles(int64_t n_v, int64_t I0, int64_t I1) {
  const int64_t nB = (n_v + 127) / 128;
  int64_t t = 0;
  for (int64_t I = I0; I < nB && I < I1; ++I) t += nB - I;
  return t;
}

int launch_tally2_tc_pair_batched(const Tally2Args *args, const uint8_t *const *ops,
                                  const int64_t *rows_pad, const int64_t *kpad, const int *split,
                                  int n, int group, int num_sms, cudaStream_t s, bool fp4) {
  static bool attr_set[kMaxDevices] = {};
  if (n < 1 || n > kMaxBatchPanels) return CCC_EINVAL;
  const int dev = current_device();
  if (dev < 0) return CCC_ECUDA;
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_tally2_tc_pair_batched<4>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(pair_smem(4))) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally2_tc_pair_batched<8>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(pair_smem(8))) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally2_tc_pair_batched_fp4,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(pair_smem(tcp::FP4_EW))) != cudaSuccess)
      return CCC_ECUDA;
    attr_set[dev] = true;
  }
  thread_local BatchMaps maps;
  thread_local BatchParams bp;
  memset(&bp, 0, sizeof(bp));
  bp.n = n;
  int64_t units = 0;
  double kw = 0.0;
  for (int k = 0; k < n; ++k) {
    BatchPanel &q = bp.p[k];
    // e2m1 rows hold kpad entries in kpad / 2 bytes; a K stage is 128 bytes.
    if (fp4 && kpad[k] % 256 != 0) return CCC_EINVAL;
    const int64_t row_bytes = fp4 ? kpad[k] / 2 : kpad[k];
    q.args = args[k];
    q.tri.nI = static_cast<int>((args[k].n_v + 127) / 128);
    q.tri.nJ = q.tri.nI;
    q.tri.group = group > 0 ? group : fp4 ? kFp4Group : 8;
    q.tri.shift = 0;
    q.tri.I0 = 0;
    q.tri.I1 = q.tri.nI;
    q.nkb = static_cast<int>(row_bytes / BK);
    q.split = split != nullptr && split[k] > 1 ? (split[k] < q.nkb ? split[k] : q.nkb) : 1;
    q.tiles = args[k].n_v >= 2 ? tc2_pair_tiles(args[k].n_v, 0, q.tri.nI) : 0;
    units += q.tiles * q.split;
    kw += static_cast<double>(q.tiles) * q.nkb;
    if (!make_operand_map(&maps.a[k], ops[k], rows_pad[k], row_bytes, tcp::BMH)) return CCC_ECUDA;
  }
  if (units == 0) return CCC_OK;
  const int ew = fp4 ? tcp::FP4_EW : epilogue_warps(static_cast<int>(kw / static_cast<double>(units)));
  static int max_clusters[kMaxDevices][3] = {};
  int &mc = max_clusters[dev][fp4 ? 2 : ew == 4 ? 0 : 1];
  if (mc == 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
    cfg.blockDim = dim3(static_cast<unsigned>(64 + 32 * ew), 1, 1);
    cfg.dynamicSmemBytes = pair_smem(ew);
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int m = 0;
    const cudaError_t e =
        fp4 ? cudaOccupancyMaxActiveClusters(&m, k_tally2_tc_pair_batched_fp4, &cfg)
        : ew == 4 ? cudaOccupancyMaxActiveClusters(&m, k_tally2_tc_pair_batched<4>, &cfg)
                  : cudaOccupancyMaxActiveClusters(&m, k_tally2_tc_pair_batched<8>, &cfg);
    if (e != cudaSuccess || m < 1) return CCC_ECUDA;
    mc = m < num_sms / 2 ? m : num_sms / 2;
  }
  const int64_t clusters = units < mc ? units : mc;
  const int grid = static_cast<int>(2 * clusters);
  if (fp4)
    k_tally2_tc_pair_batched_fp4<<<grid, 64 + 32 * tcp::FP4_EW, pair_smem(tcp::FP4_EW), s>>>(maps,
                                                                                           bp);
  else if (ew == 4)
    k_tally2_tc_pair_batched<4><<<grid, 64 + 32 * 4, pair_smem(4), s>>>(maps, bp);
  else
    k_tally2_tc_pair_batched<8><<<grid, 64 + 32 * 8, pair_smem(8), s>>>(maps, bp);
  return note_launch();
}

int launch_tally2_tc_batched(const Tally2Args *args, const uint8_t *const *ops,
                             const int64_t *rows_pad, const int64_t *kpad, int n, int group,
                             int num_sms, cudaStream_t s) {
  static bool attr_set[kMaxDevices] = {};
  if (n < 1 || n > kMaxBatchPanels) return CCC_EINVAL;
  const int dev = current_device();
  if (dev < 0) return CCC_ECUDA;
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_tally2_tc_batched<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SMEM_BYTES)) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally2_tc_batched<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SMEM_BYTES)) != cudaSuccess)
      return CCC_ECUDA;
    attr_set[dev] = true;
  }
  thread_local BatchMaps maps;
  thread_local BatchParams bp;
  memset(&bp, 0, sizeof(bp));
  bp.n = n;
  int64_t tiles = 0;
  for (int k = 0; k < n; ++k) {
    BatchPanel &q = bp.p[k];
    q.args = args[k];
    q.tri.nI = static_cast<int>((args[k].n_v + SNP_I - 1) / SNP_I);
    q.tri.nJ = static_cast<int>((args[k].n_v + SNP_J - 1) / SNP_J);
    q.tri.group = group > 0 ? group : 8;
    q.tri.shift = 1;
    q.tri.I0 = 0;
    q.tri.I1 = q.tri.nI;
    q.nkb = static_cast<int>(kpad[k] / BK);
    q.split = 1;
    q.tiles = args[k].n_v >= 2 ? tc2_num_tiles(args[k].n_v) : 0;
    tiles += q.tiles;
    if (!make_operand_map(&maps.a[k], ops[k], rows_pad[k], kpad[k], BM) ||
        !make_operand_map(&maps.b[k], ops[k], rows_pad[k], kpad[k], BN))
      return CCC_ECUDA;
  }
  if (tiles == 0) return CCC_OK;
  // Epilogue warps from the work-weighted K length of the batch.
  double kw = 0.0;
  for (int k = 0; k < n; ++k) kw += static_cast<double>(bp.p[k].tiles) * bp.p[k].nkb;
  const int mean_nkb = static_cast<int>(kw / static_cast<double>(tiles));
  const int grid = static_cast<int>(tiles < num_sms ? tiles : num_sms);
  if (epilogue_warps(mean_nkb) == 4)
    k_tally2_tc_batched<4><<<grid, 64 + 32 * 4, SMEM_BYTES, s>>>(maps, bp);
  else
    k_tally2_tc_batched<8><<<grid, 64 + 32 * 8, SMEM_BYTES, s>>>(maps, bp);
  return note_launch();
}

int launch_tally2_tc_pair(const Tally2Args &a, const uint8_t *op, int64_t rows_pad, int64_t kpad,
                          int num_sms, cudaStream_t s, bool fp4) {
  static bool attr_set[kMaxDevices] = {};
  const int dev = current_device();
  if (dev < 0) return CCC_ECUDA;
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_tally2_tc_pair<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(pair_smem(4))) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally2_tc_pair<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(pair_smem(8))) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally2_tc_pair_fp4, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(pair_smem(tcp::FP4_EW))) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally2_tc_pair_fp4w, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(rect_smem())) != cudaSuccess)
      return CCC_ECUDA;
    attr_set[dev] = true;
  }
  // e2m1 rows hold two entries per byte: kpad entries in kpad / 2 bytes, and
  // each 128-byte K stage covers 256 entries.
  if (fp4 && kpad % 256 != 0) return CCC_EINVAL;
  const int64_t row_bytes = fp4 ? kpad / 2 : kpad;
  static int max_clusters[kMaxDevices][4] = {};
  if (fp4 && a.hits != nullptr) {  // thresholded output: the two-accumulator rect tiles
    PairMaps maps;
    if (!make_operand_map(&maps.m[0], op, rows_pad, row_bytes, tcp::BMH) ||
        !make_operand_map(&maps.m[1], op, rows_pad, row_bytes, kRectJ))
      return CCC_ECUDA;
    TriSched::Params sp;
    sp.nI = static_cast<int>((a.n_v + 127) / 128);
    sp.nJ = static_cast<int>((a.n_v + kRectJ - 1) / kRectJ);
    sp.group = a.group > 0 ? a.group : kFp4RectGroup;
    sp.shift = 0;
    sp.I0 = static_cast<int>((a.i_begin > 0 ? a.i_begin : 0) / 128);
    sp.I1 = static_cast<int>(a.i_end < a.n_v ? (a.i_end + 127) / 128 : sp.nI);
    const int nkb = static_cast<int>(row_bytes / BK);
    const int64_t tiles = rect_tiles<Epi2Rect::Sched>(sp.nI, sp.nJ, sp.I0, sp.I1);
    if (tiles == 0) return CCC_OK;
    int &mc = max_clusters[dev][3];
    if (mc == 0) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr;
      attr.id = cudaLaunchAttributeClusterDimension;
      attr.val.clusterDim.x = 2;
      attr.val.clusterDim.y = 1;
      attr.val.clusterDim.z = 1;
      cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
      cfg.blockDim = dim3(static_cast<unsigned>(64 + 32 * tcp::FP4_EW), 1, 1);
      cfg.dynamicSmemBytes = rect_smem();
      cfg.attrs = &attr;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_tally2_tc_pair_fp4w, &cfg) != cudaSuccess || n < 1)
        return CCC_ECUDA;
      mc = n < num_sms / 2 ? n : num_sms / 2;
    }
    const int64_t clusters = tiles < mc ? tiles : mc;
    k_tally2_tc_pair_fp4w<<<static_cast<int>(2 * clusters), 64 + 32 * tcp::FP4_EW, rect_smem(),
                            s>>>(maps, a, sp, nkb);
    return note_launch();
  }
  CUtensorMap tm;
  if (!make_operand_map(&tm, op, rows_pad, row_bytes, tcp::BMH)) return CCC_ECUDA;
  TriSched::Params sp;
  sp.nI = static_cast<int>((a.n_v + 127) / 128);
  sp.nJ = sp.nI;
  sp.group = a.group > 0 ? a.group : fp4 ? kFp4Group : 8;
  sp.shift = 0;
  sp.I0 = static_cast<int>((a.i_begin > 0 ? a.i_begin : 0) / 128);
  sp.I1 = static_cast<int>(a.i_end < a.n_v ? (a.i_end + 127) / 128 : sp.nI);
  const int nkb = static_cast<int>(row_bytes / BK);
  const int64_t tiles = tc2_pair_tiles(a.n_v, sp.I0, sp.I1);
  if (tiles == 0) return CCC_OK;
  const int ew = fp4 ? tcp::FP4_EW : epilogue_warps(nkb);
  // Persistent grid: as many SM pairs as can be resident at once.
  int &mc = max_clusters[dev][fp4 ? 2 : ew == 4 ? 0 : 1];
  if (mc == 0) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
    cfg.blockDim = dim3(static_cast<unsigned>(64 + 32 * ew), 1, 1);
    cfg.dynamicSmemBytes = pair_smem(ew);
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e =
        fp4 ? cudaOccupancyMaxActiveClusters(&n, k_tally2_tc_pair_fp4, &cfg)
        : ew == 4 ? cudaOccupancyMaxActiveClusters(&n, k_tally2_tc_pair<4>, &cfg)
                  : cudaOccupancyMaxActiveClusters(&n, k_tally2_tc_pair<8>, &cfg);
    if (e != cudaSuccess || n < 1) return CCC_ECUDA;
    mc = n < num_sms / 2 ? n : num_sms / 2;
  }
  const int64_t clusters = tiles < mc ? tiles : mc;
  const int grid = static_cast<int>(2 * clusters);
  if (fp4)
    k_tally2_tc_pair_fp4<<<grid, 64 + 32 * tcp::FP4_EW, pair_smem(tcp::FP4_EW), s>>>(tm, a, sp, nkb);
  else if (ew == 4)
    k_tally2_tc_pair<4><<<grid, 64 + 32 * 4, pair_smem(4), s>>>(tm, a, sp, nkb);
  else
    k_tally2_tc_pair<8><<<grid, 64 + 32 * 8, pair_smem(8), s>>>(tm, a, sp, nkb);
  return note_launch();
}

int launch_tally2_tc_pair_split(const Tally2Args &a, const uint8_t *op, int64_t rows_pad,
                                int64_t kpad, int split, int num_sms, cudaStream_t s, bool fp4) {
  static int max_clusters_dev[kMaxDevices][2] = {};
  const int dev = current_device();
  if (dev < 0) return CCC_ECUDA;
  int &max_clusters = max_clusters_dev[dev][fp4 ? 1 : 0];
  const int threads = 64 + 32 * (fp4 ? tcp::FP4_EW : 4);
  const size_t smem = tcp::SMEM_BYTES;
  if (max_clusters == 0) {
    if (cudaFuncSetAttribute(k_tally2_tc_pair_split<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally2_tc_pair_split_fp4,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return CCC_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
    cfg.blockDim = dim3(static_cast<unsigned>(threads), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = fp4 ? cudaOccupancyMaxActiveClusters(&n, k_tally2_tc_pair_split_fp4, &cfg)
                              : cudaOccupancyMaxActiveClusters(&n, k_tally2_tc_pair_split<4>, &cfg);
    if (e != cudaSuccess || n < 1) return CCC_ECUDA;
    max_clusters = n < num_sms / 2 ? n : num_sms / 2;
  }
  if (fp4 && kpad % 256 != 0) return CCC_EINVAL;
  const int64_t row_bytes = fp4 ? kpad / 2 : kpad;
  const int nkb = static_cast<int>(row_bytes / BK);
  if (split < 1 || split > nkb) return CCC_EINVAL;
  CUtensorMap tm;
  if (!make_blocked_operand_map(&tm, op, rows_pad, row_bytes, tcp::BMH)) return CCC_ECUDA;
  SplitSchedPair::Params sp;
  sp.tri.nI = static_cast<int>((a.n_v + 127) / 128);
  sp.tri.nJ = sp.tri.nI;
  sp.tri.group = a.group > 0 ? a.group : fp4 ? kFp4Group : 8;
  sp.tri.shift = 0;
  sp.tri.I0 = static_cast<int>((a.i_begin > 0 ? a.i_begin : 0) / 128);
  sp.tri.I1 = static_cast<int>(a.i_end < a.n_v ? (a.i_end + 127) / 128 : sp.tri.nI);
  sp.split = split;
  sp.nkb = nkb;
  sp.tiles = tc2_pair_tiles(a.n_v, sp.tri.I0, sp.tri.I1);
  const int64_t units = sp.tiles * split;
  if (units == 0) return CCC_OK;
  const int64_t clusters = units < max_clusters ? units : max_clusters;
  if (fp4)
    k_tally2_tc_pair_split_fp4<<<static_cast<unsigned>(2 * clusters), threads, smem, s>>>(tm, a, sp,
                                                                                         nkb);
  else
    k_tally2_tc_pair_split<4><<<static_cast<unsigned>(2 * clusters), threads, smem, s>>>(tm, a, sp,
                                                                                        nkb);
  return note_launch();
}

// Tensor map over the packed panel for the packed kernels: uint64 words,
// [n_v][ceil(n_f / 32)] with row stride ld, box 4 words (one 128-entry K
// stage) x 64 SNPs, no swizzle; boxes past the panel read zeros, which the
// converters mask.
static bool make_packed_map(CUtensorMap *map, const uint64_t *geno, int64_t n_f, int64_t n_v,
                            int64_t ld) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (enc == nullptr) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>((n_f + 31) / 32),
                              static_cast<cuuint64_t>(n_v)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 8u};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(BK / 32),
                             static_cast<cuuint32_t>(tcp::pk::SNPS)};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t *>(geno), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class K>
static int pair_clusters(K kernel, int threads, size_t smem, int num_sms,
                         int (&cache_dev)[kMaxDevices]) {
  const int dev = current_device();
  if (dev < 0) return -1;
  int *cache = &cache_dev[dev];
  if (*cache == 0) {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
      return -1;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
    cfg.blockDim = dim3(static_cast<unsigned>(threads), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n < 1) return -1;
    *cache = n < num_sms / 2 ? n : num_sms / 2;
  }
  return *cache;
}

static TriSched::Params pair_params(const Tally2Args &a) {
  TriSched::Params sp;
  sp.nI = static_cast<int>((a.n_v + 127) / 128);
  sp.nJ = sp.nI;
  sp.group = a.group > 0 ? a.group : 8;
  sp.shift = 0;
  sp.I0 = static_cast<int>((a.i_begin > 0 ? a.i_begin : 0) / 128);
  sp.I1 = static_cast<int>(a.i_end < a.n_v ? (a.i_end + 127) / 128 : sp.nI);
  return sp;
}

int launch_tally2_tc_pair_packed(const Tally2Args &a, const uint64_t *geno, int64_t ld,
                                 int num_sms, cudaStream_t s) {
  constexpr int CT = 32 * tcp::pk::CW;
  CUtensorMap tm;
  if (!make_packed_map(&tm, geno, a.n_f, a.n_v, ld)) return CCC_ECUDA;
  const TriSched::Params sp = pair_params(a);
  const int nkb = static_cast<int>((a.n_f + BK - 1) / BK);
  const int64_t tiles = tc2_pair_tiles(a.n_v, sp.I0, sp.I1);
  if (tiles == 0) return CCC_OK;
  const int ew = epilogue_warps(nkb);
  static int cache4[kMaxDevices] = {}, cache8[kMaxDevices] = {};
  const int mc = ew == 4 ? pair_clusters(k_tally2_tc_pair_packed<4>, 64 + 32 * 4 + CT,
                                         packed_smem(4), num_sms, cache4)
                         : pair_clusters(k_tally2_tc_pair_packed<8>, 64 + 32 * 8 + CT,
                                         packed_smem(8), num_sms, cache8);
  if (mc < 1) return CCC_ECUDA;
  const int grid = static_cast<int>(2 * (tiles < mc ? tiles : mc));
  if (ew == 4)
    k_tally2_tc_pair_packed<4><<<grid, 64 + 32 * 4 + CT, packed_smem(4), s>>>(tm, a, sp, nkb);
  else
    k_tally2_tc_pair_packed<8><<<grid, 64 + 32 * 8 + CT, packed_smem(8), s>>>(tm, a, sp, nkb);
  return note_launch();
}

int launch_tally2_tc_pair_split_packed(const Tally2Args &a, const uint64_t *geno, int64_t ld,
                                       int split, int num_sms, cudaStream_t s) {
  constexpr int CT = 32 * tcp::pk::CW;
  const int nkb = static_cast<int>((a.n_f + BK - 1) / BK);
  if (split < 1 || split > nkb) return CCC_EINVAL;
  CUtensorMap tm;
  if (!make_packed_map(&tm, geno, a.n_f, a.n_v, ld)) return CCC_ECUDA;
  SplitSchedPair::Params sp;
  sp.tri = pair_params(a);
  sp.split = split;
  sp.nkb = nkb;
  sp.tiles = tc2_pair_tiles(a.n_v, sp.tri.I0, sp.tri.I1);
  const int64_t units = sp.tiles * split;
  if (units == 0) return CCC_OK;
  static int cache[kMaxDevices] = {};
  const int mc = pair_clusters(k_tally2_tc_pair_split_packed<4>, 64 + 32 * 4 + CT,
                               tcp::pk::SMEM_BYTES, num_sms, cache);
  if (mc < 1) return CCC_ECUDA;
  const int64_t clusters = units < mc ? units : mc;
  k_tally2_tc_pair_split_packed<4><<<static_cast<unsigned>(2 * clusters), 64 + 32 * 4 + CT,
                                     tcp::pk::SMEM_BYTES, s>>>(tm, a, sp, nkb);
  return note_launch();
}

int launch_tally2_tc(const Tally2Args &a, const uint8_t *op, int64_t rows_pad, int64_t kpad,
                     int num_sms, cudaStream_t s) {
  static bool attr_set[kMaxDevices] = {};
  const int dev = current_device();
  if (dev < 0) return CCC_ECUDA;
  if (!attr_set[dev]) {
    if (cudaFuncSetAttribute(k_tally2_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SMEM_BYTES)) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally2_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SMEM_BYTES)) != cudaSuccess)
      return CCC_ECUDA;
    attr_set[dev] = true;
  }
  CUtensorMap tmA, tmB;
  if (!make_operand_map(&tmA, op, rows_pad, kpad, BM) ||
      !make_operand_map(&tmB, op, rows_pad, kpad, BN))
    return CCC_ECUDA;
  TriSched::Params sp;
  sp.nI = static_cast<int>((a.n_v + SNP_I - 1) / SNP_I);
  sp.nJ = static_cast<int>((a.n_v + SNP_J - 1) / SNP_J);
  sp.group = a.group > 0 ? a.group : 8;
  sp.shift = 1;
  sp.I0 = static_cast<int>((a.i_begin > 0 ? a.i_begin : 0) / SNP_I);
  sp.I1 = static_cast<int>(a.i_end < a.n_v ? (a.i_end + SNP_I - 1) / SNP_I : sp.nI);
  const int nkb = static_cast<int>(kpad / BK);
  const int64_t tiles = tc2_num_tiles(a.n_v, sp.I0, sp.I1);
  if (tiles == 0) return CCC_OK;
  const int grid = static_cast<int>(tiles < num_sms ? tiles : num_sms);
  if (epilogue_warps(nkb) == 4)
    k_tally2_tc<4><<<grid, 64 + 32 * 4, SMEM_BYTES, s>>>(tmA, tmB, a, sp, nkb);
  else
    k_tally2_tc<8><<<grid, 64 + 32 * 8, SMEM_BYTES, s>>>(tmA, tmB, a, sp, nkb);
  return note_launch();
}

}  // namespace ccc
