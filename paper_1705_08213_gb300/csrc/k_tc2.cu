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
// pairs i >= j inside diagonal tiles are masked in the epilogue.
//
// Tile: A = 128 operand rows (64 SNPs i), B = 256 operand rows (128 SNPs j),
// K stage = 128 bytes.  Warp 0: TMA producer.  Warp 1: TMEM allocation and
// the single MMA-issuing thread.  Warps 2-5: epilogue, one TMEM lane quarter
// each.  Two 256-column FP32 accumulators in TMEM let the epilogue of one
// tile overlap the MMAs of the next.  The kernel is persistent: CTA b takes
// tiles b, b + gridDim.x, ... of a grouped order that keeps a band of 8 column
// blocks hot in L2 while the row blocks stream past.
#include "ccc_dev.cuh"
#include "ccc_launch.h"
#include "ccc_metric.cuh"

namespace ccc {
namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 128;
constexpr int UK = 32;  // K of one kind::f8f6f4 MMA
constexpr int STAGES = 4;
constexpr int SNP_I = BM / 2;
constexpr int SNP_J = BN / 2;
constexpr int A_BYTES = BM * BK;
constexpr int B_BYTES = BN * BK;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int ACC_COLS = BN;
constexpr int TMEM_COLS = 2 * ACC_COLS;
constexpr int GROUP = 8;
constexpr int THREADS = 192;
constexpr int NUM_BARS = 2 * STAGES + 5;
constexpr uint32_t IDESC = idesc_e4m3_f32(BM, BN);
constexpr size_t SMEM_BYTES = 1024 + static_cast<size_t>(STAGES) * STAGE_BYTES + NUM_BARS * 8 + 64;

static_assert(TMEM_COLS == 512, "two 256-column accumulators fill TMEM");
static_assert(SMEM_BYTES <= 232448, "dynamic shared memory limit");

// Walks the upper-triangle tiles (I = 64-SNP row block, J = 128-SNP column
// block, J >= I/2) in groups of GROUP column blocks, rows inside a group in
// increasing order.
struct TileWalker {
  int nI, nJ, nG;
  int g, I, J, col_end, row_end;
  bool valid;

  __device__ void set_group() {
    col_end = min((g + 1) * GROUP, nJ);
    row_end = min(nI, 2 * col_end);
  }
  __device__ void init(int nI_, int nJ_, int64_t start) {
    nI = nI_;
    nJ = nJ_;
    nG = (nJ + GROUP - 1) / GROUP;
    valid = nI > 0 && nJ > 0;
    g = 0;
    I = 0;
    if (valid) set_group();
    J = 0;
    advance(start);
  }
  __device__ void advance(int64_t step) {
    while (valid && step > 0) {
      const int64_t rem = col_end - 1 - J;
      if (step <= rem) {
        J += static_cast<int>(step);
        return;
      }
      step -= rem + 1;
      if (++I >= row_end) {
        if (++g >= nG) {
          valid = false;
          return;
        }
        set_group();
        I = 0;
      }
      J = max(g * GROUP, I >> 1);
    }
  }
};

__global__ void __launch_bounds__(THREADS, 1)
    k_tally2_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const Tally2Args args, int nI, int nJ, int nkb) {
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
      mbar_init(tempty_bar(a), 128);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  int32_t *status = args.status;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int stage = 0;
      uint32_t phase = 0;
      int last_parity[STAGES];
      for (int s = 0; s < STAGES; ++s) last_parity[s] = -1;
      bool ok = true;
      TileWalker tw;
      for (tw.init(nI, nJ, blockIdx.x); tw.valid && ok; tw.advance(gridDim.x)) {
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, status, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(stage), STAGE_BYTES);
          tma_load_2d(smem_u32(sA + stage * A_BYTES), &tmA, kb * BK, tw.I * BM, full_bar(stage));
          tma_load_2d(smem_u32(sB + stage * B_BYTES), &tmB, kb * BK, tw.J * BN, full_bar(stage));
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
          if (last_parity[s] >= 0) mbar_wait_timeout(full_bar(s), static_cast<uint32_t>(last_parity[s]));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int stage = 0;
      uint32_t phase = 0;
      int lt = 0;
      bool ok = true;
      TileWalker tw;
      for (tw.init(nI, nJ, blockIdx.x); tw.valid && ok; tw.advance(gridDim.x), ++lt) {
        const int acc = lt & 1;
        const uint32_t acc_phase = (lt >> 1) & 1;
        if (!mbar_wait_bounded(tempty_bar(acc), acc_phase ^ 1u, status, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * ACC_COLS;
        for (int kb = 0; kb < nkb; ++kb) {
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
    // ---------------- epilogue: TMEM -> tallies (+ CCC) -> HBM
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;  // accumulator lane = A row of the tile
    const int il = row >> 1;
    const int a = row & 1;
    const int64_t n_v = args.n_v;
    int lt = 0;
    TileWalker tw;
    for (tw.init(nI, nJ, blockIdx.x); tw.valid; tw.advance(gridDim.x), ++lt) {
      const int acc = lt & 1;
      const uint32_t acc_phase = (lt >> 1) & 1;
      bool ok = mbar_wait_bounded(tfull_bar(acc), acc_phase, status, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const int64_t i = static_cast<int64_t>(tw.I) * SNP_I + il;
      float wi0 = 1.f, wi1 = 1.f;
      if (args.ccc != nullptr && args.norm == CCC_NORM_PERSNP && i < n_v) {
        wi0 = __ldg(args.w + 2 * i);
        wi1 = __ldg(args.w + 2 * i + 1);
      }
      const int64_t row_base = i * (2 * n_v - i - 1) / 2 - i - 1;  // pair index = row_base + j
      const uint32_t t_base = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + acc * ACC_COLS;
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t v[32];
        tmem_ld_32x32b_x32(t_base + c * 32, v);
        tmem_ld_wait();
        if (c == BN / 32 - 1) {
          tc_fence_before();
          mbar_arrive(tempty_bar(acc));
        }
#pragma unroll
        for (int p = 0; p < 8; ++p) {
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
          const int64_t j = static_cast<int64_t>(tw.J) * SNP_J + c * 16 + 2 * p + a;
          if (i < j && j < n_v) {
            const int64_t pidx = row_base + j;
            reinterpret_cast<int4 *>(args.tally)[pidx] = make_int4(r00, r01, r10, r11);
            if (args.ccc != nullptr) {
              float wj0 = 1.f, wj1 = 1.f;
              if (args.norm == CCC_NORM_PERSNP) {
                const float2 wj = __ldg(reinterpret_cast<const float2 *>(args.w) + j);
                wj0 = wj.x;
                wj1 = wj.y;
              }
              reinterpret_cast<float4 *>(args.ccc)[pidx] =
                  ccc2_values(r00, r01, r10, r11, wi0, wi1, wj0, wj1, args.norm, args.gamma);
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
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

}  // namespace

// Row-major 2-D uint8 tensor map over op[rows][kpad] with a box of
// (128 bytes) x box_rows and 128-byte swizzling.
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

int64_t tc2_num_tiles(int64_t n_v) {
  const int64_t nI = (n_v + SNP_I - 1) / SNP_I;
  const int64_t nJ = (n_v + SNP_J - 1) / SNP_J;
  int64_t t = 0;
  for (int64_t I = 0; I < nI; ++I) t += nJ - (I >> 1);
  return t;
}

int launch_tally2_tc(const Tally2Args &a, const uint8_t *op, int64_t rows_pad, int64_t kpad,
                     int num_sms, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_tally2_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SMEM_BYTES)) != cudaSuccess)
      return CCC_ECUDA;
    attr_set = true;
  }
  CUtensorMap tmA, tmB;
  if (!make_operand_map(&tmA, op, rows_pad, kpad, BM) || !make_operand_map(&tmB, op, rows_pad, kpad, BN))
    return CCC_ECUDA;
  const int nI = static_cast<int>((a.n_v + SNP_I - 1) / SNP_I);
  const int nJ = static_cast<int>((a.n_v + SNP_J - 1) / SNP_J);
  const int nkb = static_cast<int>(kpad / BK);
  const int64_t tiles = tc2_num_tiles(a.n_v);
  const int grid = static_cast<int>(tiles < num_sms ? tiles : num_sms);
  k_tally2_tc<<<grid, THREADS, SMEM_BYTES, s>>>(tmA, tmB, a, nI, nJ, nkb);
  return note_launch();
}

}  // namespace ccc
