// 3-way tallies on the tcgen05 tensor cores with the CCC value fused into the
// epilogue.
//
// Sec. 3.2 computes the 3-way tallies of a slab of fixed j from 2-way
// products of matrices masked by the column v_j.  Here the mask is applied
// to count operands: for fixed j the operand L_j has four rows per SNP i < j,
//     L_j[(i, a, b), q] = rho_{i,q}(a) rho_{j,q}(b)      in {0, 1, 2, 4},
// and the slab is one GEMM with the count matrix R of the SNPs k > j:
//     r_{ijk}^{abc} = sum_q L_j[(i,a,b), q] R[(k,c), q].
// Values 0, 1, 2, 4 are exact in e4m3 and every partial sum is an integer
// below 8 n_f < 2^24, so FP32 accumulation is exact.
//
// k_mask3 writes L_j for a batch of slabs (each slab padded to 32 SNPs i);
// k_tally3_tc runs the persistent pipeline over all (slab, i-block, k-block)
// tiles of the batch: a tile is 128 L rows (32 SNPs i x 4 (a,b)) by 256 R rows
// (128 SNPs k x 2 c), the k-blocks of one i-block being consecutive so the L
// tile is read once from HBM and then from L2.  Only triples i < j < k are
// visited (the tetrahedral subset of Sec. 2.2 / Sec. 4).
#include "ccc_launch.h"
#include "ccc_metric.cuh"
#include "tc_pipeline.cuh"

namespace ccc {
namespace {

using namespace tc;

constexpr int SNP_I = BM / 4;  // 32 SNPs i per tile
constexpr int SNP_K = BN / 2;  // 128 SNPs k per tile

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// sum_{m=0}^{x-1} floor(m / 32)
__host__ __device__ inline int64_t floor32_prefix(int64_t x) {
  const int64_t q = x / 32, r = x % 32;
  return 32 * q * (q - 1) / 2 + r * q;
}

// Number of 32-SNP i-blocks of the slabs j' < j: sum_{j' < j} ceil(j' / 32).
__host__ __device__ inline int64_t iblocks_before(int64_t j) { return floor32_prefix(j + 31); }

// Tiles of a batch of slabs [j0, j1): slab j has ceil(j/32) i-blocks times
// ceil((n_v-1-j)/128) k-blocks; i-block-major inside a slab.
struct SlabSched {
  struct Params {
    int j0, j1, n_v;
  };
  int j, j1, n_v;
  int mt, nt;  // i-blocks, k-blocks of slab j
  int m, n;        // current tile
  int64_t lbase;   // first L row of slab j in the batch (masked-operand buffer)
  bool valid;

  __device__ void set_slab() {
    mt = static_cast<int>(ceil_div(j, SNP_I));
    nt = static_cast<int>(ceil_div(n_v - 1 - j, SNP_K));
  }
  // Move to the first slab >= j that has tiles.
  __device__ void skip_empty() {
    while (j < j1) {
      set_slab();
      if (mt > 0 && nt > 0) return;
      lbase += BM * mt;
      ++j;
    }
    valid = false;
  }
  __device__ void init(const Params &p, int64_t start) {
    j = p.j0;
    j1 = p.j1;
    n_v = p.n_v;
    m = n = 0;
    lbase = 0;
    valid = true;
    skip_empty();
    advance(start);
  }
  __device__ void advance(int64_t step) {
    while (valid && step > 0) {
      const int64_t rem = static_cast<int64_t>(mt) * nt - 1 - (static_cast<int64_t>(m) * nt + n);
      if (step <= rem) {
        const int64_t pos = static_cast<int64_t>(m) * nt + n + step;
        m = static_cast<int>(pos / nt);
        n = static_cast<int>(pos % nt);
        return;
      }
      step -= rem + 1;
      lbase += BM * mt;
      ++j;
      m = n = 0;
      skip_empty();
    }
  }
  __device__ int map_index() const { return 0; }
  __device__ int k_blocks(int nkb) const { return nkb; }
  __device__ int a_row() const { return static_cast<int>(lbase + BM * m); }
  __device__ int b_row() const { return 2 * (j + 1) + BN * n; }
};

struct Epi3 {
  using Params = Tally3Args;

  // Accumulator lane = L row (4 il + 2a + b), column = 2 kl + c.  The four
  // lanes of a quad hold one SNP i; thread ab writes tallies 2ab, 2ab+1 (c = 0, 1)
  // of every triple, so a quad writes each triple's 32 bytes contiguously.
  template <int NC>
  __device__ static void tile(const Params &args, const SlabSched &sc, int quarter, int lane,
                              uint32_t t_base, uint32_t release_bar, int c0) {
    const int row = quarter * 32 + lane;
    const int il = row >> 2;
    const int ab = row & 3;
    const int a = ab >> 1;
    const int b = ab & 1;
    const int64_t n_v = args.n_v;
    const int64_t j = sc.j;
    const int64_t i = static_cast<int64_t>(sc.m) * SNP_I + il;
    const bool row_ok = i < j;
    const bool want_ccc = args.ccc != nullptr;
    const bool persnp = args.norm == CCC_NORM_PERSNP;
    float wi = 1.f, wj = 1.f;
    if (want_ccc && persnp) {
      if (row_ok) wi = __ldg(args.w + 2 * i + a);
      wj = __ldg(args.w + 2 * j + b);
    }
    const int64_t span = n_v - 1 - j;
    const int64_t base = slab_offset_dev(j, n_v) - slab_offset_dev(args.j_begin, n_v) + i * span;
    const int64_t k0 = j + 1 + static_cast<int64_t>(sc.n) * SNP_K;
    for (int c = c0; c < c0 + NC; ++c) {
      uint32_t v[32];
      tmem_ld_32x32b_x32(t_base + c * 32, v);
      tmem_ld_wait();
      if (c == c0 + NC - 1) {
        tc_fence_before();
        mbar_arrive(release_bar);
      }
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const int32_t r0 = __float2int_rn(__uint_as_float(v[2 * kk]));
        const int32_t r1 = __float2int_rn(__uint_as_float(v[2 * kk + 1]));
        // Quad sums: c-marginals (sum over a, b) and 8 n_ijk.
        int32_t q0 = r0 + __shfl_xor_sync(0xffffffffu, r0, 1);
        q0 += __shfl_xor_sync(0xffffffffu, q0, 2);
        int32_t q1 = r1 + __shfl_xor_sync(0xffffffffu, r1, 1);
        q1 += __shfl_xor_sync(0xffffffffu, q1, 2);
        const int32_t own = r0 + r1;
        const int32_t ra = own + __shfl_xor_sync(0xffffffffu, own, 1);  // sum over b, c (fixed a)
        const int32_t rb = own + __shfl_xor_sync(0xffffffffu, own, 2);  // sum over a, c (fixed b)
        const int64_t k = k0 + c * 16 + kk;
        if (row_ok && k < n_v && CCC_IN_BOUNDS(base + (k - j - 1), args.out_len, args.status)) {
          const int64_t t = base + (k - j - 1);
          __stcs(reinterpret_cast<int2 *>(args.tally) + 4 * t + ab, make_int2(r0, r1));
          if (want_ccc) {
            const int32_t n8 = q0 + q1;
            float2 out = make_float2(0.f, 0.f);
            if (n8 != 0) {
              const float d = static_cast<float>(n8);
              float fi = wi, fj = wj, fk0, fk1;
              if (persnp) {
                const float2 wk = __ldg(reinterpret_cast<const float2 *>(args.w) + k);
                fk0 = wk.x;
                fk1 = wk.y;
              } else {
                fi = joint_factor(ra, d, args.gamma);
                fj = joint_factor(rb, d, args.gamma);
                fk0 = joint_factor(q0, d, args.gamma);
                fk1 = joint_factor(q1, d, args.gamma);
              }
              if (persnp) {
                const float inv = __frcp_rn(d);
                const float wij = __fmul_rn(fi, fj);
                out.x = ccc3_persnp(r0, inv, wij, fk0);
                out.y = ccc3_persnp(r1, inv, wij, fk1);
              } else {
                out.x = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(r0), d), fi), fj), fk0);
                out.y = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(r1), d), fi), fj), fk1);
              }
            }
            __stcs(reinterpret_cast<float2 *>(args.ccc) + 4 * t + ab, out);
          }
        }
      }
    }
  }
};

template <int EW>
__global__ void __launch_bounds__(64 + 32 * EW, 1)
    k_tally3_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const Tally3Args args, SlabSched::Params sp, int nkb) {
  persistent_gemm<SlabSched, Epi3, EW>(&tmA, &tmB, sp, args, nkb, args.status);
}

constexpr uint64_t kEven = 0x5555555555555555ull;

__device__ __forceinline__ uint64_t masked_word(const uint64_t *geno, int64_t ld, int64_t s,
                                                int64_t k, int64_t n_f) {
  // Word k of SNP s with every entry past n_f turned into the missing code.
  if (k * 32 >= n_f) return 0xAAAAAAAAAAAAAAAAull;
  uint64_t valid = kEven;
  const int64_t tail = n_f - k * 32;
  if (tail < 32) valid &= (1ull << (2 * tail)) - 1ull;
  const uint64_t vm = valid | (valid << 1);
  return (geno[s * ld + k] & vm) | (0xAAAAAAAAAAAAAAAAull & ~vm);
}

__device__ __forceinline__ uint32_t code_nibbles(uint32_t b) {
  return (b & 0x3u) | ((b << 2) & 0x30u) | ((b << 4) & 0x300u) | ((b << 6) & 0x3000u);
}

// e4m3 products rho_i(a) rho_j(b) for 32 consecutive entries: out[2a + b][g]
// holds the bytes of entries 4g .. 4g + 3.  wi, wj: packed codes of SNP i and
// SNP j for those entries (missing entries must carry the missing code).
// For 4 entries at a time the selector nibble of entry q is code_i(q) + 4 *
// [rho_j(b) = 2], indexing an 8-byte table of e4m3 values rho_i(a) * {1, 2};
// entries with rho_j(b) = 0 are then masked to zero.
__device__ __forceinline__ void mask_products(uint64_t wi, uint64_t wj, uint32_t (&out)[4][8]) {
  // e4m3: 1 = 0x38, 2 = 0x40, 4 = 0x48.  Table bytes 0-3: rho_a(code) x 1,
  // bytes 4-7: rho_a(code) x 2, for codes 00, 01, 10 (missing), 11.
  const uint32_t lo[2] = {0x00003840u, 0x40003800u};
  const uint32_t hi[2] = {0x00004048u, 0x48004000u};
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const uint32_t si = code_nibbles(static_cast<uint32_t>(wi >> (8 * g)) & 0xFFu);
    const uint32_t sj = code_nibbles(static_cast<uint32_t>(wj >> (8 * g)) & 0xFFu);
    // rho_j(0) = 2 <=> code 00; rho_j(1) = 2 <=> code 11 (bit 2 of each nibble).
    const uint32_t two0 = ((~sj & ~(sj >> 1)) & 0x1111u) << 2;
    const uint32_t two1 = ((sj & (sj >> 1)) & 0x1111u) << 2;
    // rho_j(0) != 0 <=> code 00 or 01; rho_j(1) != 0 <=> code 01 or 11.
    const uint32_t nz0 = __byte_perm(0x0000FFFFu, 0u, sj);
    const uint32_t nz1 = __byte_perm(0xFF00FF00u, 0u, sj);
#pragma unroll
    for (int aa = 0; aa < 2; ++aa) {
      out[2 * aa + 0][g] = __byte_perm(lo[aa], hi[aa], si | two0) & nz0;
      out[2 * aa + 1][g] = __byte_perm(lo[aa], hi[aa], si | two1) & nz1;
    }
  }
}

// Codes of 32 entries starting at entry q0 with every entry past n_f turned
// into the missing code.
__device__ __forceinline__ uint64_t mask_tail(uint64_t w, int64_t q0, int64_t n_f) {
  if (q0 >= n_f) return 0xAAAAAAAAAAAAAAAAull;
  if (q0 + 32 <= n_f) return w;
  const uint64_t vm = (1ull << (2 * (n_f - q0))) - 1ull;
  return (w & vm) | (0xAAAAAAAAAAAAAAAAull & ~vm);
}

// L_j rows for the batch of slabs [j0, j0 + gridDim.y).  One thread per
// (i, packed word); i runs over the slab's 32-padded i range.
__global__ void k_mask3(const uint64_t *__restrict__ geno, int64_t n_f, int64_t ld,
                        uint8_t *__restrict__ lop, int64_t kpad, int64_t j0) {
  const int64_t j = j0 + blockIdx.y;
  const int64_t wpr = kpad / 32;
  const int64_t islots = ceil_div(j, SNP_I) * SNP_I;
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= islots * wpr) return;
  const int64_t i = t / wpr;
  const int64_t k = t - i * wpr;
  const int64_t lrow = static_cast<int64_t>(BM) * (iblocks_before(j) - iblocks_before(j0)) + 4 * i;
  uint4 *dst[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) dst[r] = reinterpret_cast<uint4 *>(lop + (lrow + r) * kpad + k * 32);
  if (i >= j) {
#pragma unroll
    for (int r = 0; r < 4; ++r) dst[r][0] = dst[r][1] = make_uint4(0u, 0u, 0u, 0u);
    return;
  }
  const uint64_t wi = masked_word(geno, ld, i, k, n_f);
  const uint64_t wj = masked_word(geno, ld, j, k, n_f);
  uint32_t out[4][8];
  mask_products(wi, wj, out);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    dst[r][0] = make_uint4(out[r][0], out[r][1], out[r][2], out[r][3]);
    dst[r][1] = make_uint4(out[r][4], out[r][5], out[r][6], out[r][7]);
  }
}

// ---------------------------------------------------------------- fused masking
//
// k_tally3_fused forms the masked operand inside the tally kernel: per K stage
// TMA brings the packed codes of the tile's 32 SNPs i (32 x 32 bytes) and of
// v_j (32 bytes) next to the 256 count rows of the k side, and four transform
// warps write the 128 rows x 128 bytes of L_j products straight into the
// stage's 128B-swizzled A buffer (byte c of row r at r * 128 + ((c / 16) ^
// (r % 8)) * 16 + c % 16) before the MMA consumes it.  The masked operand never
// touches HBM.
//
// Warps: 0 TMA producer, 1 TMEM + MMA issuer, 2-5 transform, 6.. epilogue.

constexpr int F_STAGES = STAGES;
constexpr int F_CODE_I = SNP_I * 32;          // 32 SNPs x 32 bytes (128 entries)
constexpr int F_CODE_BYTES = F_CODE_I + 32;   // + v_j
constexpr int F_CODE_STRIDE = 1152;           // 128-byte aligned per stage
constexpr int F_TX = B_BYTES + F_CODE_BYTES;  // TMA bytes per stage
constexpr int F_NUM_BARS = 3 * F_STAGES + 5;
constexpr size_t F_SMEM_BYTES = 1024 + static_cast<size_t>(F_STAGES) * STAGE_BYTES +
                                static_cast<size_t>(F_STAGES) * F_CODE_STRIDE + F_NUM_BARS * 8 + 64;
static_assert(F_SMEM_BYTES <= 232448, "dynamic shared memory limit");

template <int EW>
__global__ void __launch_bounds__(192 + 32 * EW, 1)
    k_tally3_fused(const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmCi,
                   const __grid_constant__ CUtensorMap tmCj, const Tally3Args args,
                   SlabSched::Params sp, int nkb) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t *smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint8_t *sA = smem;
  uint8_t *sB = smem + F_STAGES * A_BYTES;
  uint8_t *sC = sB + F_STAGES * B_BYTES;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sC + F_STAGES * F_CODE_STRIDE);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + F_NUM_BARS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

  constexpr int EPI_THREADS = Epilogue<EW>::THREADS;
  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto afull_bar = [&](int s) { return bar0 + 8u * (F_STAGES + s); };
  auto empty_bar = [&](int s) { return bar0 + 8u * (2 * F_STAGES + s); };
  auto tfull_bar = [&](int a) { return bar0 + 8u * (3 * F_STAGES + a); };
  auto tempty_bar = [&](int a) { return bar0 + 8u * (3 * F_STAGES + 2 + a); };
  const uint32_t drain_bar = bar0 + 8u * (3 * F_STAGES + 4);
  int32_t *status = args.status;

  if (threadIdx.x == 0) {
    for (int s = 0; s < F_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(afull_bar(s), 128);
      mbar_init(empty_bar(s), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(tfull_bar(a), 1);
      mbar_init(tempty_bar(a), EPI_THREADS);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0 && lane == 0) {
    tma_prefetch_desc(&tmB);
    tma_prefetch_desc(&tmCi);
    tma_prefetch_desc(&tmCj);
  }
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
      // ---------------- TMA producer: k-side count rows and packed codes
      int stage = 0;
      uint32_t phase = 0;
      int last_parity[F_STAGES];
      for (int s = 0; s < F_STAGES; ++s) last_parity[s] = -1;
      bool ok = true;
      SlabSched sc;
      for (sc.init(sp, blockIdx.x); sc.valid && ok; sc.advance(gridDim.x)) {
        const int yb = sc.b_row();
        const int yi = SNP_I * sc.m;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait_bounded(empty_bar(stage), phase ^ 1u, status, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(full_bar(stage), F_TX);
          uint8_t *codes = sC + stage * F_CODE_STRIDE;
          tma_load_2d(smem_u32(sB + stage * B_BYTES), &tmB, kb * BK, yb, full_bar(stage));
          tma_load_2d(smem_u32(codes), &tmCi, kb * 32, yi, full_bar(stage));
          tma_load_2d(smem_u32(codes + F_CODE_I), &tmCj, kb * 32, sc.j, full_bar(stage));
          last_parity[stage] = static_cast<int>(phase);
          if (++stage == F_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        for (int s = 0; s < F_STAGES; ++s)
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
      SlabSched sc;
      for (sc.init(sp, blockIdx.x); sc.valid && ok; sc.advance(gridDim.x), ++lt) {
        const int acc = lt & 1;
        const uint32_t acc_phase = (lt >> 1) & 1;
        if (!mbar_wait_bounded(tempty_bar(acc), acc_phase ^ 1u, status, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + acc * ACC_COLS;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait_bounded(full_bar(stage), phase, status, abort_flag) ||
              !mbar_wait_bounded(afull_bar(stage), phase, status, abort_flag)) {
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
          if (++stage == F_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(tfull_bar(acc));
      }
      mma_commit(drain_bar);
      mbar_wait_timeout(drain_bar, 0);
    }
  } else if (warp < 6) {
    // ---------------- transform: packed codes -> L_j products (A stage)
    const int t = threadIdx.x - 64;
    const int il = t >> 2;   // SNP i of the tile
    const int qtr = t & 3;   // entries [32 qtr, 32 qtr + 32) of the stage
    int stage = 0;
    uint32_t phase = 0;
    SlabSched sc;
    bool ok = true;
    for (sc.init(sp, blockIdx.x); sc.valid && ok; sc.advance(gridDim.x)) {
      for (int kb = 0; kb < nkb; ++kb) {
        if (!mbar_wait_bounded(full_bar(stage), phase, status, abort_flag)) {
          ok = false;
          break;
        }
        const uint8_t *codes = sC + stage * F_CODE_STRIDE;
        const int64_t q0 = static_cast<int64_t>(kb) * BK + 32 * qtr;
        const uint64_t wi =
            mask_tail(*reinterpret_cast<const uint64_t *>(codes + il * 32 + qtr * 8), q0, args.n_f);
        const uint64_t wj =
            mask_tail(*reinterpret_cast<const uint64_t *>(codes + F_CODE_I + qtr * 8), q0, args.n_f);
        uint32_t out[4][8];
        mask_products(wi, wj, out);
        uint8_t *a = sA + stage * A_BYTES;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int row = 4 * il + r;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = 2 * qtr + h;
            *reinterpret_cast<uint4 *>(a + row * 128 + ((c ^ (row & 7)) << 4)) =
                make_uint4(out[r][4 * h], out[r][4 * h + 1], out[r][4 * h + 2], out[r][4 * h + 3]);
          }
        }
        fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
        mbar_arrive(afull_bar(stage));
        if (++stage == F_STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
  } else {
    // ---------------- epilogue
    const int quarter = warp & 3;
    constexpr int NC = Epilogue<EW>::CHUNKS_PER_WARP;
    const int c0 = ((warp - 6) >> 2) * NC;
    int lt = 0;
    SlabSched sc;
    for (sc.init(sp, blockIdx.x); sc.valid; sc.advance(gridDim.x), ++lt) {
      const int acc = lt & 1;
      const uint32_t acc_phase = (lt >> 1) & 1;
      const bool ok = mbar_wait_bounded(tfull_bar(acc), acc_phase, status, abort_flag);
      if (!__all_sync(0xffffffffu, ok)) break;
      tc_fence_after();
      const uint32_t t_base =
          tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) + acc * ACC_COLS;
      Epi3::tile<NC>(args, sc, quarter, lane, t_base, tempty_bar(acc), c0);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem_base, TMEM_COLS);
}

}  // namespace

int64_t tc3_lop_rows(int64_t j0, int64_t j1) {
  return static_cast<int64_t>(BM) * (iblocks_before(j1) - iblocks_before(j0));
}

int64_t tc3_num_tiles(int64_t j0, int64_t j1, int64_t n_v) {
  int64_t t = 0;
  for (int64_t j = j0; j < j1; ++j) t += ceil_div(j, SNP_I) * ceil_div(n_v - 1 - j, SNP_K);
  return t;
}

int launch_mask3(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *lop,
                 int64_t kpad, int64_t j0, int64_t j1, cudaStream_t s) {
  (void)n_v;
  if (j1 <= j0) return CCC_OK;
  const int threads = 256;
  const int64_t wpr = kpad / 32;
  const int64_t max_slots = ceil_div(j1 - 1, SNP_I) * SNP_I;  // largest slab in the batch
  const int64_t bx = ceil_div(max_slots * wpr, threads);
  if (bx <= 0) return CCC_OK;
  dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(j1 - j0));
  k_mask3<<<grid, threads, 0, s>>>(geno, n_f, ld, lop, kpad, j0);
  return note_launch();
}

// Tensor map over the packed panel as bytes: rows of ld * 8 bytes, a box of
// 32 bytes (128 entries) x box_rows rows, no swizzle.
static bool make_code_map(CUtensorMap *map, const uint64_t *geno, int64_t n_v, int64_t ld,
                          uint32_t box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (enc == nullptr) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return false;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(ld * 8), static_cast<cuuint64_t>(n_v)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld * 8)};
  const cuuint32_t box[2] = {32u, box_rows};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint64_t *>(geno), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int launch_tally3_fused(const Tally3Args &a, const uint64_t *geno, int64_t ld, const uint8_t *op,
                        int64_t rows_pad, int64_t kpad, int num_sms, cudaStream_t s) {
  static bool attr_set_dev[kMaxDevices] = {};
  const int dev_a = current_device();
  if (dev_a < 0) return CCC_ECUDA;
  bool &attr_set = attr_set_dev[dev_a];
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_tally3_fused<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(F_SMEM_BYTES)) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally3_fused<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(F_SMEM_BYTES)) != cudaSuccess)
      return CCC_ECUDA;
    attr_set = true;
  }
  const int64_t j0 = a.j_begin > 1 ? a.j_begin : 1;
  const int64_t j1 = a.j_end < a.n_v - 1 ? a.j_end : a.n_v - 1;
  if (j1 <= j0) return CCC_OK;
  const int64_t tiles = tc3_num_tiles(j0, j1, a.n_v);
  if (tiles == 0) return CCC_OK;
  CUtensorMap tmB, tmCi, tmCj;
  if (!make_operand_map(&tmB, op, rows_pad, kpad, BN) ||
      !make_code_map(&tmCi, geno, a.n_v, ld, SNP_I) || !make_code_map(&tmCj, geno, a.n_v, ld, 1))
    return CCC_ECUDA;
  SlabSched::Params sp;
  sp.j0 = static_cast<int>(j0);
  sp.j1 = static_cast<int>(j1);
  sp.n_v = static_cast<int>(a.n_v);
  const int nkb = static_cast<int>(kpad / BK);
  const int grid = static_cast<int>(tiles < num_sms ? tiles : num_sms);
  if (epilogue_warps(nkb) == 4)
    k_tally3_fused<4><<<grid, 192 + 32 * 4, F_SMEM_BYTES, s>>>(tmB, tmCi, tmCj, a, sp, nkb);
  else
    k_tally3_fused<8><<<grid, 192 + 32 * 8, F_SMEM_BYTES, s>>>(tmB, tmCi, tmCj, a, sp, nkb);
  return note_launch();
}

int launch_tally3_tc(const Tally3Args &a, const uint8_t *op, int64_t rows_pad, int64_t kpad,
                     uint8_t *lop, int64_t lop_rows, int64_t j0, int64_t j1, int num_sms,
                     cudaStream_t s) {
  static bool attr_set_dev[kMaxDevices] = {};
  const int dev_a = current_device();
  if (dev_a < 0) return CCC_ECUDA;
  bool &attr_set = attr_set_dev[dev_a];
  if (!attr_set) {
    if (cudaFuncSetAttribute(k_tally3_tc<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SMEM_BYTES)) != cudaSuccess ||
        cudaFuncSetAttribute(k_tally3_tc<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(SMEM_BYTES)) != cudaSuccess)
      return CCC_ECUDA;
    attr_set = true;
  }
  const int64_t tiles = tc3_num_tiles(j0, j1, a.n_v);
  if (tiles == 0) return CCC_OK;
  CUtensorMap tmA, tmB;
  if (!make_operand_map(&tmA, lop, lop_rows, kpad, BM) ||
      !make_operand_map(&tmB, op, rows_pad, kpad, BN))
    return CCC_ECUDA;
  SlabSched::Params sp;
  sp.j0 = static_cast<int>(j0);
  sp.j1 = static_cast<int>(j1);
  sp.n_v = static_cast<int>(a.n_v);
  const int nkb = static_cast<int>(kpad / BK);
  const int grid = static_cast<int>(tiles < num_sms ? tiles : num_sms);
  if (epilogue_warps(nkb) == 4)
    k_tally3_tc<4><<<grid, 64 + 32 * 4, SMEM_BYTES, s>>>(tmA, tmB, a, sp, nkb);
  else
    k_tally3_tc<8><<<grid, 64 + 32 * 8, SMEM_BYTES, s>>>(tmA, tmB, a, sp, nkb);
  return note_launch();
}

}  // namespace ccc
