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
  int m, n;    // current tile
  int lbase;   // first L row of slab j in the batch
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
  __device__ int a_row() const { return lbase + BM * m; }
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
        if (row_ok && k < n_v) {
          const int64_t t = base + (k - j - 1);
          reinterpret_cast<int2 *>(args.tally)[4 * t + ab] = make_int2(r0, r1);
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
              out.x = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(r0), d), fi), fj), fk0);
              out.y = __fmul_rn(__fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(r1), d), fi), fj), fk1);
            }
            reinterpret_cast<float2 *>(args.ccc)[4 * t + ab] = out;
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

// L_j rows for the batch of slabs [j0, j0 + gridDim.y).  One thread per
// (i, packed word); i runs over the slab's 32-padded i range.
// For 4 entries at a time: the selector nibble of entry q is code_i(q) + 4 *
// [rho_j(b) = 2], indexing an 8-byte table of e4m3 products rho_i(a) * {1, 2};
// entries with rho_j(b) = 0 are then masked to zero.
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
  // e4m3: 1 = 0x38, 2 = 0x40, 4 = 0x48.  Table bytes 0-3: rho_a(code) x 1,
  // bytes 4-7: rho_a(code) x 2, for codes 00, 01, 10 (missing), 11.
  const uint32_t lo[2] = {0x00003840u, 0x40003800u};
  const uint32_t hi[2] = {0x00004048u, 0x48004000u};
  uint32_t out[4][8];
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
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    dst[r][0] = make_uint4(out[r][0], out[r][1], out[r][2], out[r][3]);
    dst[r][1] = make_uint4(out[r][4], out[r][5], out[r][6], out[r][7]);
  }
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

int launch_tally3_tc(const Tally3Args &a, const uint8_t *op, int64_t rows_pad, int64_t kpad,
                     uint8_t *lop, int64_t lop_rows, int64_t j0, int64_t j1, int num_sms,
                     cudaStream_t s) {
  static bool attr_set = false;
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
