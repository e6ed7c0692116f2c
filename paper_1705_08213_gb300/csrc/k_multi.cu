// 2-way CCC of markers with s allele states on the tcgen05 tensor cores.
//
// Sec. 7 item 2 extends CCC from biallelic SNPs to markers with any number of
// states: a pair of markers gets an s x s table.  Written with the state set
// S = {0..s-1}, Eqs. 1-3 keep their form, and the tally table is again a block
// of a Gram product (Sec. 3.1): with s count rows rho_i(a) per SNP,
// r_ij^{ab} = sum_q rho_{i,q}(a) rho_{j,q}(b) is entry (row(i,a), row(j,b)) of
// R R^T.  Counts 0, 1, 2 are exact in e4m3 and every sum stays an integer
// below 2^24, so the FP32 accumulation of kind::f8f6f4 is exact.
//
// Operand rows.  The rows of a SNP must sit in one 32-lane quarter of the
// accumulator so that the epilogue can sum a pair's table with warp shuffles:
// a quarter (32 rows) holds PW = floor(32 / s) SNPs, SNP i at rows
// 32 (i / PW) + s (i % PW) + a; the 32 - s PW rows left over are zero.  A
// 256-row block then holds 8 PW SNPs, on both sides of the product, and the
// SM-pair pipeline of the biallelic kernel (tc_pipeline_pair.cuh: 256 x 256
// tiles, cta_group::2) walks the upper triangle of those blocks.
//
// Epilogue: the thread of accumulator lane (i, a) holds r_ij^{ab} for every
// column (j, b) of its chunk.  n_ij comes from a shuffle sum over the s lanes
// of SNP i; the CCC values (Eq. 3, PERSNP or JOINT normalisation) use the same
// single-precision operations, in the same order, as the biallelic epilogue,
// so s = 2 reproduces the biallelic results bit for bit.
#include "k_multi.cuh"

namespace ccc {
namespace {

// Bytes of a 4-entry word whose low (high) nibble equals state a: 0x01 per byte.
__device__ __forceinline__ uint32_t nibble_eq(uint32_t nib, uint32_t a) {
  const uint32_t t = nib ^ (a * 0x01010101u);  // bytes 0..15, zero where equal
  return (~((t | 0x80808080u) - 0x01010101u) & 0x80808080u) >> 7;
}

// Bytes whose nibble is >= s (the entry is missing): 0x01 per byte.
__device__ __forceinline__ uint32_t nibble_ge(uint32_t nib, uint32_t s) {
  return (((nib | 0x80808080u) - s * 0x01010101u) & 0x80808080u) >> 7;
}

// Bytes q < n_f of the 4-entry word starting at entry q0: 0x01 per byte.
__device__ __forceinline__ uint32_t valid_bytes(int64_t q0, int64_t n_f) {
  const int64_t k = n_f - q0;
  if (k >= 4) return 0x01010101u;
  if (k <= 0) return 0u;
  return 0x01010101u & ((1u << (8 * k)) - 1u);
}

// ---------------------------------------------------------------- per-SNP counts
//
// One warp per SNP: s_i^a = sum_q rho_{i,q}(a) (Eq. 1 numerators), n_i, and the
// PERSNP factors 1 - gamma s_i^a / (2 n_i) rounded once to fp32 (the formula of
// the biallelic counts kernel).  Templated on the number of states S.
template <int S>
__global__ void __launch_bounds__(256) k_multi_counts(const uint8_t *__restrict__ geno, int64_t n_f,
                                                      int64_t n_v, int64_t ld,
                                                      int32_t *__restrict__ counts,
                                                      float *__restrict__ w, double gamma) {
  constexpr int s = S;
  const int lane = threadIdx.x & 31;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n_v) return;
  const uint8_t *row = geno + i * ld;
  uint32_t c[S];
#pragma unroll
  for (int a = 0; a < S; ++a) c[a] = 0;
  uint32_t n = 0;
  const uint32_t us = static_cast<uint32_t>(s);
  auto count16 = [&](int64_t q0, const uint4 &v) {
    const uint32_t words[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t lo = words[k] & 0x0F0F0F0Fu, hi = (words[k] >> 4) & 0x0F0F0F0Fu;
      const uint32_t present =
          valid_bytes(q0 + 4 * k, n_f) & ~(nibble_ge(lo, us) | nibble_ge(hi, us));
      n += __popc(present);
#pragma unroll
      for (int a = 0; a < S; ++a)
        c[a] += __popc(nibble_eq(lo, a) & present) + __popc(nibble_eq(hi, a) & present);
    }
  };
  // Four 16-byte loads in flight per lane, then the remainder one at a time.
  int64_t q0 = 16 * static_cast<int64_t>(lane);
  for (; q0 + 3 * 16 * 32 < n_f; q0 += 4 * 16 * 32) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const uint4 *>(row + q0 + u * 16 * 32);
#pragma unroll
    for (int u = 0; u < 4; ++u) count16(q0 + u * 16 * 32, v[u]);
  }
  for (; q0 < n_f; q0 += 16 * 32) count16(q0, *reinterpret_cast<const uint4 *>(row + q0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xffffffffu, n, o);
#pragma unroll
    for (int a = 0; a < S; ++a) c[a] += __shfl_xor_sync(0xffffffffu, c[a], o);
  }
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < S; ++a) {
      if (counts) counts[i * (s + 1) + a] = static_cast<int32_t>(c[a]);
      if (w) {
        const double f = n > 0 ? static_cast<double>(c[a]) / (2.0 * static_cast<double>(n)) : 0.0;
        w[i * s + a] = static_cast<float>(1.0 - gamma * f);
      }
    }
    if (counts) counts[i * (s + 1) + s] = static_cast<int32_t>(n);
  }
}

// PERSNP factors from an int32[n_v][s + 1] counts array (same formula).
__global__ void k_multi_factors(const int32_t *__restrict__ counts, int64_t n_v, int s,
                                float *__restrict__ w, double gamma) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_v * s) return;
  const int64_t i = t / s;
  const int a = static_cast<int>(t - i * s);
  const double n = counts[i * (s + 1) + s];
  const double f = n > 0 ? counts[i * (s + 1) + a] / (2.0 * n) : 0.0;
  w[t] = static_cast<float>(1.0 - gamma * f);
}

// ---------------------------------------------------------------- operand rows
//
// One thread per (32-row quarter, 16 individuals): the quarter's PW SNPs each
// give s rows of 16 e4m3 counts (0x00, 0x38 = 1, 0x40 = 2); the rows past
// s PW, SNPs past n_v and individuals past n_f are zero.
__global__ void __launch_bounds__(256) k_multi_unpack(const uint8_t *__restrict__ geno, int64_t n_f,
                                                      int64_t n_v, int64_t ld, int s,
                                                      uint8_t *__restrict__ op, int64_t kpad,
                                                      int64_t n_quarters) {
  const int64_t chunks = kpad / 16;
  const int64_t total = n_quarters * chunks;
  const int pw = snps_per_quarter(s);
  const uint32_t us = static_cast<uint32_t>(s);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t g = t / chunks;
    const int64_t c = t - g * chunks;
    const int64_t q0 = 16 * c;
    uint8_t *dst = op + (32 * g) * kpad + q0;
    int r = 0;
    for (int u = 0; u < pw; ++u) {
      const int64_t i = g * pw + u;
      uint32_t words[4] = {0u, 0u, 0u, 0u};
      if (i < n_v && q0 < n_f) {
        const uint4 v = *reinterpret_cast<const uint4 *>(geno + i * ld + q0);
        words[0] = v.x;
        words[1] = v.y;
        words[2] = v.z;
        words[3] = v.w;
      }
      uint32_t lo[4], hi[4], present[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        lo[k] = words[k] & 0x0F0F0F0Fu;
        hi[k] = (words[k] >> 4) & 0x0F0F0F0Fu;
        present[k] = (i < n_v ? valid_bytes(q0 + 4 * k, n_f) : 0u) &
                     ~(nibble_ge(lo[k], us) | nibble_ge(hi[k], us));
      }
      for (int a = 0; a < s; ++a, ++r) {
        uint32_t e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t fx = nibble_eq(lo[k], a) & present[k];
          const uint32_t fy = nibble_eq(hi[k], a) & present[k];
          e[k] = (fx ^ fy) * 0x38u | (fx & fy) * 0x40u;  // count 1 -> 0x38, 2 -> 0x40
        }
        *reinterpret_cast<uint4 *>(dst + r * kpad) = make_uint4(e[0], e[1], e[2], e[3]);
      }
    }
    for (; r < 32; ++r) *reinterpret_cast<uint4 *>(dst + r * kpad) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// FP4 (e2m1) operand rows: as k_multi_unpack with each count 0, 1, 2 stored
// as the nibble 0x0, 0x2, 0x4, two entries per byte (entry q in the low nibble
// of byte q / 2 for even q), rows of kpad / 2 bytes (kpad a multiple of 256).
// One thread per (32-row quarter, 32 individuals): 16 bytes per row.
__global__ void __launch_bounds__(256) k_multi_unpack_e2m1(const uint8_t *__restrict__ geno,
                                                           int64_t n_f, int64_t n_v, int64_t ld,
                                                           int s, uint8_t *__restrict__ op,
                                                           int64_t kpad, int64_t n_quarters) {
  const int64_t chunks = kpad / 32;
  const int64_t row_bytes = kpad / 2;
  const int64_t total = n_quarters * chunks;
  const int pw = snps_per_quarter(s);
  const uint32_t us = static_cast<uint32_t>(s);
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t g = t / chunks;
    const int64_t c = t - g * chunks;
    const int64_t q0 = 32 * c;
    uint8_t *dst = op + (32 * g) * row_bytes + 16 * c;
    int r = 0;
    for (int u = 0; u < pw; ++u) {
      const int64_t i = g * pw + u;
      uint32_t words[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
      if (i < n_v && q0 < n_f) {
        const uint4 v0 = *reinterpret_cast<const uint4 *>(geno + i * ld + q0);
        words[0] = v0.x;
        words[1] = v0.y;
        words[2] = v0.z;
        words[3] = v0.w;
        if (q0 + 16 < n_f) {  // the row holds ld >= n_f bytes, ld a multiple of 16
          const uint4 v1 = *reinterpret_cast<const uint4 *>(geno + i * ld + q0 + 16);
          words[4] = v1.x;
          words[5] = v1.y;
          words[6] = v1.z;
          words[7] = v1.w;
        }
      }
      uint32_t lo[8], hi[8], present[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        lo[k] = words[k] & 0x0F0F0F0Fu;
        hi[k] = (words[k] >> 4) & 0x0F0F0F0Fu;
        present[k] = (i < n_v ? valid_bytes(q0 + 4 * k, n_f) : 0u) &
                     ~(nibble_ge(lo[k], us) | nibble_ge(hi[k], us));
      }
      for (int a = 0; a < s; ++a, ++r) {
        uint32_t e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          uint32_t x[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int kk = 2 * k + h;
            const uint32_t fx = nibble_eq(lo[kk], a) & present[kk];
            const uint32_t fy = nibble_eq(hi[kk], a) & present[kk];
            // count 1 -> 0x2, 2 -> 0x4 in each byte; then the 4 bytes -> 4 nibbles
            uint32_t b = ((fx ^ fy) << 1) | ((fx & fy) << 2);
            b = (b | (b >> 4)) & 0x00FF00FFu;
            b = (b | (b >> 8)) & 0x0000FFFFu;
            x[h] = b;
          }
          e[k] = x[0] | (x[1] << 16);
        }
        *reinterpret_cast<uint4 *>(dst + r * row_bytes) = make_uint4(e[0], e[1], e[2], e[3]);
      }
    }
    for (; r < 32; ++r)
      *reinterpret_cast<uint4 *>(dst + r * row_bytes) = make_uint4(0u, 0u, 0u, 0u);
  }
}

// ---------------------------------------------------------------- CCC from stored tallies

// One thread per pair: Eq. 3 over the pair's s x s table, the same operations
// as the tally kernel's epilogue.
__global__ void k_metric2_multi(const int32_t *__restrict__ tally, const float *__restrict__ w,
                                int64_t n_v, int s, float gamma, int32_t norm,
                                float *__restrict__ ccc) {
  const int64_t npairs = n_v * (n_v - 1) / 2;
  const int ss = s * s;
  for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < npairs;
       p += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    // Row i of pair p: the largest i with pair_index(i, i + 1) <= p.
    int64_t i = static_cast<int64_t>(
        (2.0 * n_v - 1.0 - sqrt((2.0 * n_v - 1.0) * (2.0 * n_v - 1.0) - 8.0 * static_cast<double>(p))) / 2.0);
    if (i < 0) i = 0;
    while (i > 0 && i * (2 * n_v - i - 1) / 2 > p) --i;
    while ((i + 1) * (2 * n_v - i - 2) / 2 <= p) ++i;
    const int64_t j = p - i * (2 * n_v - i - 1) / 2 + i + 1;
    const int32_t *t = tally + p * ss;
    float *out = ccc + p * ss;
    int32_t n4 = 0;
    for (int x = 0; x < ss; ++x) n4 += t[x];
    if (n4 == 0) {
      for (int x = 0; x < ss; ++x) out[x] = 0.f;
      continue;
    }
    const float d = static_cast<float>(n4);
    const float inv = __frcp_rn(d);
    for (int a = 0; a < s; ++a) {
      float wi;
      if (norm == CCC_NORM_PERSNP) {
        wi = w[i * s + a];
      } else {
        int32_t rs = 0;
        for (int b = 0; b < s; ++b) rs += t[a * s + b];
        wi = joint_factor(rs, d, gamma);
      }
      for (int b = 0; b < s; ++b) {
        const float r = static_cast<float>(t[a * s + b]);
        if (norm == CCC_NORM_PERSNP) {
          out[a * s + b] = __fmul_rn(__fmul_rn(__fmul_rn(r, inv), wi), w[j * s + b]);
        } else {
          int32_t cs = 0;
          for (int x = 0; x < s; ++x) cs += t[x * s + b];
          out[a * s + b] = __fmul_rn(__fmul_rn(__fdiv_rn(r, d), wi), joint_factor(cs, d, gamma));
        }
      }
    }
  }
}

}  // namespace

int64_t multi_rows_pad(int64_t n_v, int s) {
  const int64_t quarters = (n_v + snps_per_quarter(s) - 1) / snps_per_quarter(s);
  return (32 * quarters + 255) / 256 * 256;
}

int launch_multi_counts(const uint8_t *geno, int64_t n_f, int64_t n_v, int64_t ld, int s,
                        int32_t *counts, float *w, double gamma, cudaStream_t st) {
  if (n_v < 1) return CCC_OK;
  const unsigned blocks = static_cast<unsigned>((n_v + 7) / 8);
  switch (s) {
#define CCC_MULTI_COUNTS(S)                                                                   \
  case S:                                                                                    \
    k_multi_counts<S><<<blocks, 256, 0, st>>>(geno, n_f, n_v, ld, counts, w, gamma);       \
    break;
    CCC_MULTI_COUNTS(2) CCC_MULTI_COUNTS(3) CCC_MULTI_COUNTS(4) CCC_MULTI_COUNTS(5)
    CCC_MULTI_COUNTS(6) CCC_MULTI_COUNTS(7) CCC_MULTI_COUNTS(8) CCC_MULTI_COUNTS(9)
    CCC_MULTI_COUNTS(10) CCC_MULTI_COUNTS(11) CCC_MULTI_COUNTS(12) CCC_MULTI_COUNTS(13)
    CCC_MULTI_COUNTS(14) CCC_MULTI_COUNTS(15)
#undef CCC_MULTI_COUNTS
    default:
      return CCC_EINVAL;
  }
  return note_launch();
}

int launch_multi_factors(const int32_t *counts, int64_t n_v, int s, float *w, double gamma,
                         cudaStream_t st) {
  const int64_t n = n_v * s;
  if (n < 1) return CCC_OK;
  k_multi_factors<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(counts, n_v, s, w, gamma);
  return note_launch();
}

int launch_multi_unpack(const uint8_t *geno, int64_t n_f, int64_t n_v, int64_t ld, int s,
                        uint8_t *op, int64_t kpad, int64_t rows_pad, cudaStream_t st, bool fp4) {
  const int64_t quarters = rows_pad / 32;
  if (fp4) {
    if (kpad % 256 != 0) return CCC_EINVAL;
    const int64_t total4 = quarters * (kpad / 32);
    if (total4 < 1) return CCC_OK;
    const int64_t blocks4 = (total4 + 255) / 256 < 152 * 16 ? (total4 + 255) / 256 : 152 * 16;
    k_multi_unpack_e2m1<<<static_cast<unsigned>(blocks4), 256, 0, st>>>(geno, n_f, n_v, ld, s, op,
                                                                         kpad, quarters);
    return note_launch();
  }
  const int64_t total = quarters * (kpad / 16);
  if (total < 1) return CCC_OK;
  const int64_t blocks = (total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16;
  k_multi_unpack<<<static_cast<unsigned>(blocks), 256, 0, st>>>(geno, n_f, n_v, ld, s, op, kpad,
                                                               quarters);
  return note_launch();
}

int launch_tally2_multi(int s, int64_t n_v, const float *w, int32_t *tally, float *out_ccc,
                        int32_t *status, float gamma, int32_t norm, int32_t group, const uint8_t *op,
                        int64_t rows_pad, int64_t kpad, int num_sms, cudaStream_t st,
                        int64_t i_begin, int64_t i_end, int64_t pair0, int split, bool fp4) {
  if (n_v < 2) return CCC_OK;
  if (fp4) {
    // e2m1 rows of kpad / 2 bytes; 256 x 192 tiles, no K split; s <= 8.
    if (split > 1 || s > 8 || kpad % 256 != 0) return CCC_EINVAL;
    MultiMaps maps;
    if (!tc::make_operand_map(&maps.m[0], op, rows_pad, kpad / 2, tcp::BMH) ||
        !tc::make_operand_map(&maps.m[1], op, rows_pad, kpad / 2, kMultiRectNB / 2))
      return CCC_ECUDA;
    MultiArgs a4{n_v, w, tally, out_ccc, status, gamma, norm, i_begin, i_end, pair0};
    a4.out_len = checked_out_len(pairs_in_rows(n_v, i_begin, i_end));
    const int nkb4 = static_cast<int>((kpad / 2) / tcp::BK);
    switch (s) {
      case 2: return launch_tally2_multi_fp4_s<2>(maps, a4, group, nkb4, num_sms, st);
      case 3: return launch_tally2_multi_fp4_s<3>(maps, a4, group, nkb4, num_sms, st);
      case 4: return launch_tally2_multi_fp4_s<4>(maps, a4, group, nkb4, num_sms, st);
      case 5: return launch_tally2_multi_fp4_s<5>(maps, a4, group, nkb4, num_sms, st);
      case 6: return launch_tally2_multi_fp4_s<6>(maps, a4, group, nkb4, num_sms, st);
      case 7: return launch_tally2_multi_fp4_s<7>(maps, a4, group, nkb4, num_sms, st);
      case 8: return launch_tally2_multi_fp4_s<8>(maps, a4, group, nkb4, num_sms, st);
      default: return CCC_EINVAL;
    }
  }
  if (s > 8) return launch_tally2_multi_wide(s, n_v, w, tally, out_ccc, status, gamma, norm, group,
                                             op, rows_pad, kpad, num_sms, st, i_begin, i_end, pair0,
                                             split);
  CUtensorMap tm;
  if (!tc::make_operand_map(&tm, op, rows_pad, kpad, tcp::BMH)) return CCC_ECUDA;
  MultiArgs a{n_v, w, tally, out_ccc, status, gamma, norm, i_begin, i_end, pair0};
  a.out_len = checked_out_len(pairs_in_rows(n_v, i_begin, i_end));
  // 256-row blocks holding a SNP (rows_pad has exactly these).
  const int64_t nB = rows_pad / 256;
  const int nkb = static_cast<int>(kpad / tcp::BK);
  if (split > 1) {
    switch (s) {
      case 2: return launch_tally2_multi_split_s<2>(tm, a, nB, group, nkb, split, num_sms, st);
      case 3: return launch_tally2_multi_split_s<3>(tm, a, nB, group, nkb, split, num_sms, st);
      case 4: return launch_tally2_multi_split_s<4>(tm, a, nB, group, nkb, split, num_sms, st);
      case 5: return launch_tally2_multi_split_s<5>(tm, a, nB, group, nkb, split, num_sms, st);
      case 6: return launch_tally2_multi_split_s<6>(tm, a, nB, group, nkb, split, num_sms, st);
      case 7: return launch_tally2_multi_split_s<7>(tm, a, nB, group, nkb, split, num_sms, st);
      case 8: return launch_tally2_multi_split_s<8>(tm, a, nB, group, nkb, split, num_sms, st);
      default: return CCC_EINVAL;
    }
  }
  switch (s) {
    case 2: return launch_tally2_multi_s<2>(tm, a, nB, group, nkb, num_sms, st);
    case 3: return launch_tally2_multi_s<3>(tm, a, nB, group, nkb, num_sms, st);
    case 4: return launch_tally2_multi_s<4>(tm, a, nB, group, nkb, num_sms, st);
    case 5: return launch_tally2_multi_s<5>(tm, a, nB, group, nkb, num_sms, st);
    case 6: return launch_tally2_multi_s<6>(tm, a, nB, group, nkb, num_sms, st);
    case 7: return launch_tally2_multi_s<7>(tm, a, nB, group, nkb, num_sms, st);
    case 8: return launch_tally2_multi_s<8>(tm, a, nB, group, nkb, num_sms, st);
    default: return CCC_EINVAL;
  }
}

int launch_metric2_multi(const int32_t *tally, const float *w, int64_t n_v, int s, float gamma,
                         int32_t norm, float *out_ccc, cudaStream_t st) {
  const int64_t npairs = n_v * (n_v - 1) / 2;
  if (npairs < 1) return CCC_OK;
  const int64_t blocks = (npairs + 255) / 256 < 152 * 32 ? (npairs + 255) / 256 : 152 * 32;
  k_metric2_multi<<<static_cast<unsigned>(blocks), 256, 0, st>>>(tally, w, n_v, s, gamma, norm,
                                                                 out_ccc);
  return note_launch();
}

}  // namespace ccc
