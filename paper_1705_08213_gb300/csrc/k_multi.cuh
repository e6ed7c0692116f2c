// The multi-allelic 2-way tally kernel (k_multi.cu describes the method and
// the operand layout), templated on the number of states s.  k_multi.cu
// instantiates s = 2..8 and k_multi_wide.cu s = 9..15.
#pragma once

#include "ccc_launch.h"
#include "ccc_metric.cuh"
#include "tc_pipeline.cuh"
#include "tc_pipeline_pair.cuh"
#include "tc_sched.cuh"

#include <type_traits>

namespace ccc {
namespace {

constexpr int kMultiEpiWarps = 8;
constexpr int kMultiThreads = 64 + 32 * kMultiEpiWarps;

__host__ __device__ constexpr int snps_per_quarter(int s) { return 32 / s; }

struct MultiArgs {
  int64_t n_v;
  const float *w;   // [n_v][s] PERSNP factors, or null
  int32_t *tally;   // [npairs][s*s]
  float *ccc;       // [npairs][s*s], or null
  int32_t *status;
  float gamma;
  int32_t norm;
  // Row range of a phase: only pairs with i_begin <= i < i_end, stored at
  // pair_index(i, j) - pair0.
  int64_t i_begin, i_end, pair0;
  // Pairs the tally / ccc arrays hold (checked builds test every store index).
  int64_t out_len = int64_t(1) << 62;
};

// s consecutive values from registers to global memory (streaming stores).
template <int S>
__device__ __forceinline__ void store_row(int32_t *dst, const int32_t (&v)[S]) {
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int b = 0; b < S; b += 4)
      __stcs(reinterpret_cast<int4 *>(dst + b), make_int4(v[b], v[b + 1], v[b + 2], v[b + 3]));
  } else if constexpr (S % 2 == 0) {
#pragma unroll
    for (int b = 0; b < S; b += 2) __stcs(reinterpret_cast<int2 *>(dst + b), make_int2(v[b], v[b + 1]));
  } else {
#pragma unroll
    for (int b = 0; b < S; ++b) __stcs(dst + b, v[b]);
  }
}

template <int S>
__device__ __forceinline__ void store_row(float *dst, const float (&v)[S]) {
  if constexpr (S % 4 == 0) {
#pragma unroll
    for (int b = 0; b < S; b += 4)
      __stcs(reinterpret_cast<float4 *>(dst + b), make_float4(v[b], v[b + 1], v[b + 2], v[b + 3]));
  } else if constexpr (S % 2 == 0) {
#pragma unroll
    for (int b = 0; b < S; b += 2)
      __stcs(reinterpret_cast<float2 *>(dst + b), make_float2(v[b], v[b + 1]));
  } else {
#pragma unroll
    for (int b = 0; b < S; ++b) __stcs(dst + b, v[b]);
  }
}

// B blocks of NBQ quarters (32 operand rows each): 8 for the 256 x 256 e4m3
// tiles (TriSchedPair), 6 for the 256 x 192 FP4 tiles (RectSchedT; two
// 192-column accumulators and the scale factors fit the 512 TMEM columns).
constexpr int kMultiRectQ = 6;
constexpr int kMultiRectNB = 32 * kMultiRectQ;

template <int S, int NBQ = 8>
struct EpiMultiT {
  using Params = MultiArgs;
  static constexpr int PW = snps_per_quarter(S);
  // The PERSNP factors w_j of the warp's NBQ / 2 quarters of markers.
  static constexpr int STAGE_BYTES_PER_WARP = (NBQ / 2) * 32 * 4;
  using Sched = std::conditional_t<NBQ == 8, TriSchedPair,
                                   RectSchedT<8 * PW, NBQ * PW, 32 * NBQ>>;

  // The warps of column half h (c0 = h NC) take the chunks of 32 columns
  // [h NBQ / 2, (h + 1) NBQ / 2); chunk c is B quarter NBQ J + c.
  template <int NC, bool PRELOAD = false>
  __device__ static void tile(const Params &args, const Sched &sc, int rank, int quarter,
                              int lane, uint32_t t_base, uint32_t release_cluster_bar, int c0,
                              float *stage) {
    static_assert(!PRELOAD, "s-state tiles run on the two-accumulator pipeline");
    static_assert(NBQ % 2 == 0, "two column halves");
    const int cb = (c0 / NC) * (NBQ / 2);
    const int ce = cb + NBQ / 2;
    const int u = lane / S;
    const int a = lane - u * S;
    const int64_t n_v = args.n_v;
    // Accumulator lane = A row (i, a) of CTA `rank`'s 128 rows.
    const int64_t i = ((2 * static_cast<int64_t>(sc.I) + rank) * 4 + quarter) * PW + u;
    const bool row_ok = u < PW && i < n_v;
    const bool want_ccc = args.ccc != nullptr;
    const bool persnp = args.norm == CCC_NORM_PERSNP;
    float wi = 1.f;
    if (want_ccc && persnp && row_ok) wi = __ldg(args.w + i * S + a);
    const int64_t row_base = i * (2 * n_v - i - 1) / 2 - i - 1;  // pair index = row_base + j
    const int src0 = (u < PW ? u : 0) * S;                        // first lane of SNP i
    // w_j of the warp's markers jw0 .. (NBQ / 2 quarters), staged once per tile; every lane
    // then reads the same address (a broadcast) instead of its own global load per pair.
    const int64_t jw0 = (NBQ * static_cast<int64_t>(sc.J) + cb) * PW;
    if (want_ccc && persnp) {
      __syncwarp();  // the previous tile's reads are done
      for (int k = lane; k < (NBQ / 2) * PW * S; k += 32) {
        const int64_t e = jw0 * S + k;
        stage[k] = e < n_v * S ? __ldg(args.w + e) : 1.f;
      }
      __syncwarp();
    }
    for (int c = cb; c < ce; ++c) {
      uint32_t v[32];
      tmem_ld_32x32b_x32(t_base + c * 32, v);
      tmem_ld_wait();
      if (c == ce - 1) {
        tc_fence_before();
        mbar_arrive_cluster(release_cluster_bar);
      }
      // Column chunk c = 32 rows of the B block: its quarter c.
      const int64_t j0 = (NBQ * static_cast<int64_t>(sc.J) + c) * PW;
#pragma unroll
      for (int jl = 0; jl < PW; ++jl) {
        const int64_t j = j0 + jl;
        int32_t r[S];
        int32_t rs = 0;
#pragma unroll
        for (int b = 0; b < S; ++b) {
          r[b] = __float2int_rn(__uint_as_float(v[jl * S + b]));
          rs += r[b];
        }
        // 4 n_ij = sum over the pair's table: the row sums of SNP i's s lanes.
        int32_t n4 = 0;
#pragma unroll
        for (int k = 0; k < S; ++k) n4 += __shfl_sync(0xffffffffu, rs, src0 + k);
        int32_t colsum[S];
        if (want_ccc && !persnp) {
#pragma unroll
          for (int b = 0; b < S; ++b) {
            colsum[b] = 0;
#pragma unroll
            for (int k = 0; k < S; ++k) colsum[b] += __shfl_sync(0xffffffffu, r[b], src0 + k);
          }
        }
        if (!(row_ok && i < j && j < n_v && i >= args.i_begin && i < args.i_end)) continue;
        if (!CCC_IN_BOUNDS(row_base + j - args.pair0, args.out_len, args.status)) continue;
        const int64_t base = (row_base + j - args.pair0) * (S * S) + a * S;
        store_row<S>(args.tally + base, r);
        if (!want_ccc) continue;
        float cv[S];
        if (n4 == 0) {
#pragma unroll
          for (int b = 0; b < S; ++b) cv[b] = 0.f;
        } else if (persnp) {
          const float inv = __frcp_rn(static_cast<float>(n4));
          const float *wjs = stage + ((c - cb) * PW + jl) * S;
#pragma unroll
          for (int b = 0; b < S; ++b)
            cv[b] = __fmul_rn(__fmul_rn(__fmul_rn(static_cast<float>(r[b]), inv), wi), wjs[b]);
        } else {
          const float d = static_cast<float>(n4);
          const float wia = joint_factor(rs, d, args.gamma);
#pragma unroll
          for (int b = 0; b < S; ++b) {
            const float wjb = joint_factor(colsum[b], d, args.gamma);
            cv[b] = __fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(r[b]), d), wia), wjb);
          }
        }
        store_row<S>(args.ccc + base, cv);
      }
    }
  }
};

// Partial tallies of one K part (K split): each accumulator element is added
// into the zeroed tally array with an integer reduction.
template <int S>
struct EpiMultiSplit {
  using Params = MultiArgs;
  static constexpr int PW = snps_per_quarter(S);
  static constexpr int STAGE_BYTES_PER_WARP = 0;

  template <int NC, bool PRELOAD = false>
  __device__ static void tile(const Params &args, const SplitSchedPair &sc, int rank, int quarter,
                              int lane, uint32_t t_base, uint32_t release_cluster_bar, int c0,
                              float *) {
    static_assert(!PRELOAD, "s-state tiles run on the two-accumulator pipeline");
    const int u = lane / S;
    const int a = lane - u * S;
    const int64_t n_v = args.n_v;
    const int64_t i = ((2 * static_cast<int64_t>(sc.I) + rank) * 4 + quarter) * PW + u;
    const bool row_ok = u < PW && i < n_v && i >= args.i_begin && i < args.i_end;
    const int64_t row_base = i * (2 * n_v - i - 1) / 2 - i - 1 - args.pair0;
    for (int c = c0; c < c0 + NC; ++c) {
      uint32_t v[32];
      tmem_ld_32x32b_x32(t_base + c * 32, v);
      tmem_ld_wait();
      if (c == c0 + NC - 1) {
        tc_fence_before();
        mbar_arrive_cluster(release_cluster_bar);
      }
      const int64_t j0 = ((2 * static_cast<int64_t>(sc.J) + (c >> 2)) * 4 + (c & 3)) * PW;
#pragma unroll
      for (int jl = 0; jl < PW; ++jl) {
        const int64_t j = j0 + jl;
        if (!(row_ok && i < j && j < n_v)) continue;
        if (!CCC_IN_BOUNDS(row_base + j, args.out_len, args.status)) continue;
        int32_t *dst = args.tally + (row_base + j) * (S * S) + a * S;
#pragma unroll
        for (int b = 0; b < S; ++b) {
          const int32_t r = __float2int_rn(__uint_as_float(v[jl * S + b]));
          if (r != 0) atomicAdd(dst + b, r);
        }
      }
    }
  }
};

template <int S>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kMultiThreads, 1)
    k_tally2_multi_split(const __grid_constant__ CUtensorMap tm, const MultiArgs args,
                         SplitSchedPair::Params sp, int nkb) {
  tcp::persistent_gemm_pair<SplitSchedPair, EpiMultiSplit<S>, kMultiEpiWarps>(&tm, sp, args, nkb,
                                                                               args.status);
}

template <int S>
using EpiMulti = EpiMultiT<S, 8>;

template <int S>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kMultiThreads, 1)
    k_tally2_multi(const __grid_constant__ CUtensorMap tm, const MultiArgs args,
                   TriSched::Params sp, int nkb) {
  tcp::persistent_gemm_pair<TriSchedPair, EpiMulti<S>, kMultiEpiWarps>(&tm, sp, args, nkb, args.status);
}

// FP4 (e2m1) operands: 256 x 192 tiles on SM pairs, two accumulators
// (tcp::persistent_gemm_pair with NB = 192); A through maps.m[0] (box 128 rows),
// B through maps.m[1] (box 96 rows).
struct MultiMaps {
  CUtensorMap m[2];
};

template <int S>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kMultiThreads, 1)
    k_tally2_multi_fp4(const __grid_constant__ MultiMaps maps, const MultiArgs args,
                       TriSched::Params sp, int nkb) {
  using Epi = EpiMultiT<S, kMultiRectQ>;
  tcp::persistent_gemm_pair<typename Epi::Sched, Epi, kMultiEpiWarps, false, true, kMultiRectNB>(
      maps.m, sp, args, nkb, args.status);
}

constexpr size_t multi_fp4_smem() {
  return tcp::smem_bytes_nb(kMultiRectNB, kMultiEpiWarps, EpiMultiT<2, kMultiRectQ>::STAGE_BYTES_PER_WARP);
}
constexpr size_t multi_smem() {
  return tcp::smem_bytes(kMultiEpiWarps, EpiMultiT<2, 8>::STAGE_BYTES_PER_WARP);
}

// Persistent grid size for a pair kernel of kMultiThreads threads.
template <typename K>
int multi_max_clusters(K kernel, int num_sms) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(tcp::SMEM_BYTES)) != cudaSuccess)
    return 0;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = 2;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
  cfg.blockDim = dim3(kMultiThreads, 1, 1);
  cfg.dynamicSmemBytes = tcp::SMEM_BYTES;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess || n < 1) return 0;
  return n < num_sms / 2 ? n : num_sms / 2;
}

// K-split launch over the whole triangle of nB row blocks (split <= nkb).
template <int S>
int launch_tally2_multi_split_s(const CUtensorMap &tm, const MultiArgs &a, int64_t nB, int group,
                                int nkb, int split, int num_sms, cudaStream_t s) {
  static int max_clusters_dev[kMaxDevices] = {};
  const int dev_c = current_device();
  if (dev_c < 0) return CCC_ECUDA;
  int &max_clusters = max_clusters_dev[dev_c];
  if (max_clusters == 0) max_clusters = multi_max_clusters(k_tally2_multi_split<S>, num_sms);
  if (max_clusters == 0) return CCC_ECUDA;
  if (split < 1 || split > nkb) return CCC_EINVAL;
  SplitSchedPair::Params sp;
  sp.tri.nI = static_cast<int>(nB);
  sp.tri.nJ = sp.tri.nI;
  sp.tri.group = group > 0 ? group : 8;
  sp.tri.shift = 0;
  sp.tri.I0 = 0;
  sp.tri.I1 = sp.tri.nI;
  sp.split = split;
  sp.nkb = nkb;
  sp.tiles = nB * (nB + 1) / 2;
  const int64_t units = sp.tiles * split;
  if (units == 0) return CCC_OK;
  const int64_t clusters = units < max_clusters ? units : max_clusters;
  k_tally2_multi_split<S><<<static_cast<unsigned>(2 * clusters), kMultiThreads, tcp::SMEM_BYTES,
                            s>>>(tm, a, sp, nkb);
  return note_launch();
}

// FP4 launch over the rows [i_begin, i_end) (nI row blocks of 8 PW markers,
// nJ column blocks of 6 PW).
template <int S>
int launch_tally2_multi_fp4_s(const MultiMaps &maps, const MultiArgs &a, int group, int nkb,
                              int num_sms, cudaStream_t s) {
  using Epi = EpiMultiT<S, kMultiRectQ>;
  constexpr int64_t pi = 8 * static_cast<int64_t>(snps_per_quarter(S));
  constexpr int64_t pj = kMultiRectQ * static_cast<int64_t>(snps_per_quarter(S));
  TriSched::Params sp;
  sp.nI = static_cast<int>((a.n_v + pi - 1) / pi);
  sp.nJ = static_cast<int>((a.n_v + pj - 1) / pj);
  // Default tile order: groups of 32 column blocks (GB300, s = 4, 10,000 x
  // 16,384, per call: 4.81 ms against 4.86 with 16, 4.95 with 8, 4.84 with 64).
  sp.group = group > 0 ? group : 32;
  sp.shift = 0;
  sp.I0 = static_cast<int>(a.i_begin / pi);
  const int64_t iend = a.i_end < a.n_v ? a.i_end : a.n_v;
  sp.I1 = static_cast<int>((iend + pi - 1) / pi < sp.nI ? (iend + pi - 1) / pi : sp.nI);
  const int64_t tiles = rect_tiles<typename Epi::Sched>(sp.nI, sp.nJ, sp.I0, sp.I1);
  if (tiles <= 0) return CCC_OK;
  static int max_clusters_dev[kMaxDevices] = {};
  const int dev_c = current_device();
  if (dev_c < 0) return CCC_ECUDA;
  int &max_clusters = max_clusters_dev[dev_c];
  if (max_clusters == 0) {
    if (cudaFuncSetAttribute(k_tally2_multi_fp4<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(multi_fp4_smem())) != cudaSuccess)
      return CCC_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
    cfg.blockDim = dim3(kMultiThreads, 1, 1);
    cfg.dynamicSmemBytes = multi_fp4_smem();
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_tally2_multi_fp4<S>, &cfg) != cudaSuccess || n < 1)
      return CCC_ECUDA;
    max_clusters = n < num_sms / 2 ? n : num_sms / 2;
  }
  const int64_t clusters = tiles < max_clusters ? tiles : max_clusters;
  k_tally2_multi_fp4<S><<<static_cast<unsigned>(2 * clusters), kMultiThreads, multi_fp4_smem(),
                          s>>>(maps, a, sp, nkb);
  return note_launch();
}

template <int S>
int launch_tally2_multi_s(const CUtensorMap &tm, const MultiArgs &a, int64_t nB, int group, int nkb,
                          int num_sms, cudaStream_t s) {
  // Row blocks of 8 PW markers holding rows [i_begin, i_end).
  const int64_t per_block = 8 * static_cast<int64_t>(snps_per_quarter(S));
  const int64_t I0 = a.i_begin / per_block;
  const int64_t I1 = (a.i_end < a.n_v ? a.i_end : a.n_v) + per_block - 1;
  TriSched::Params sp;
  sp.nI = static_cast<int>(nB);
  sp.nJ = sp.nI;
  sp.group = group > 0 ? group : 8;
  sp.shift = 0;
  sp.I0 = static_cast<int>(I0);
  sp.I1 = static_cast<int>(I1 / per_block < nB ? I1 / per_block : nB);
  // Tiles of rows [I0, I1): sum of nB - I.
  const int64_t rows = sp.I1 > sp.I0 ? sp.I1 - sp.I0 : 0;
  const int64_t tiles = rows * nB - (static_cast<int64_t>(sp.I0) + sp.I1 - 1) * rows / 2;
  if (tiles <= 0) return CCC_OK;
  static int max_clusters_dev[kMaxDevices] = {};
  const int dev_c = current_device();
  if (dev_c < 0) return CCC_ECUDA;
  int &max_clusters = max_clusters_dev[dev_c];
  if (max_clusters == 0) {
    if (cudaFuncSetAttribute(k_tally2_multi<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(multi_smem())) != cudaSuccess)
      return CCC_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.gridDim = dim3(static_cast<unsigned>(num_sms), 1, 1);
    cfg.blockDim = dim3(kMultiThreads, 1, 1);
    cfg.dynamicSmemBytes = multi_smem();
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_tally2_multi<S>, &cfg) != cudaSuccess || n < 1)
      return CCC_ECUDA;
    max_clusters = n < num_sms / 2 ? n : num_sms / 2;
  }
  const int64_t clusters = tiles < max_clusters ? tiles : max_clusters;
  k_tally2_multi<S><<<static_cast<unsigned>(2 * clusters), kMultiThreads, multi_smem(), s>>>(tm, a, sp,
                                                                                          nkb);
  return note_launch();
}

}  // namespace
}  // namespace ccc
