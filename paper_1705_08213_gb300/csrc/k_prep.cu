// Preparation passes over the packed panel: per-SNP allele counts (Eq. 1),
// the e4m3 count operands for the tensor-core tallies, and the bit planes for
// the popcount tallies.  All are O(n_f n_v) and HBM-bound.
#include "ccc_dev.cuh"
#include "ccc_launch.h"

namespace ccc {

namespace {

constexpr uint64_t kEven = 0x5555555555555555ull;

// Mask of the low bits of every valid 2-bit entry of word w of a row of n_f
// entries (even bit positions only).
__device__ __forceinline__ uint64_t valid_even_mask(int64_t w, int64_t n_f) {
  const int64_t first = w * 32;
  if (first + 32 <= n_f) return kEven;
  if (first >= n_f) return 0;
  const int tail = static_cast<int>(n_f - first);  // 1..31
  return kEven & ((1ull << (2 * tail)) - 1ull);
}

// WPS warps per SNP (256-thread blocks hold 8 / WPS SNPs).  For every word:
// l = (v)_2 bits, h = (v)_1 bits; the missing marker is h & ~l; rho_1 = l + (h & l)
// for present entries.  Several warps per SNP keep enough loads in flight when
// a panel has few SNPs with long vectors.
template <int WPS>
__global__ void __launch_bounds__(256) k_allele_counts(const uint64_t *__restrict__ geno,
                                                       int64_t n_f, int64_t n_v, int64_t ld,
                                                       int32_t *__restrict__ counts,
                                                       float *__restrict__ w, double gamma) {
  constexpr int kSnpsPerBlock = 8 / WPS;
  __shared__ long long part[8][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = warp / WPS, sub = warp % WPS;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * kSnpsPerBlock + slot;
  const int64_t words = (n_f + 31) / 32;
  int64_t n = 0, s1 = 0;
  if (i < n_v) {
    const uint64_t *row = geno + i * ld;
    const int64_t step = 32 * WPS;
    int64_t k = sub * 32 + lane;
    // Four independent loads per iteration.
    for (; k + 3 * step < words; k += 4 * step) {
      uint64_t v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = __ldg(row + k + u * step);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint64_t valid = valid_even_mask(k + u * step, n_f);
        const uint64_t l = v[u] & valid;
        const uint64_t h = (v[u] >> 1) & valid;
        n += __popcll(valid & ~(h & ~l));
        s1 += __popcll(l) + __popcll(h & l);
      }
    }
    for (; k < words; k += step) {
      const uint64_t v = __ldg(row + k);
      const uint64_t valid = valid_even_mask(k, n_f);
      const uint64_t l = v & valid;
      const uint64_t h = (v >> 1) & valid;
      n += __popcll(valid & ~(h & ~l));
      s1 += __popcll(l) + __popcll(h & l);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xffffffffu, n, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (WPS > 1) {
    if (lane == 0) {
      part[warp][0] = n;
      part[warp][1] = s1;
    }
    __syncthreads();
    if (sub != 0) return;
    for (int u = 1; u < WPS; ++u) {
      n += part[warp + u][0];
      s1 += part[warp + u][1];
    }
  }
  if (lane == 0 && i < n_v) {
    const int64_t s0 = 2 * n - s1;
    if (counts) {
      counts[3 * i + 0] = static_cast<int32_t>(s0);
      counts[3 * i + 1] = static_cast<int32_t>(s1);
      counts[3 * i + 2] = static_cast<int32_t>(n);
    }
    if (w) {
      // 1 - gamma f_i(a), f_i(a) = s_i^a / (2 n_i), rounded once to fp32.
      const double f0 = n > 0 ? static_cast<double>(s0) / (2.0 * static_cast<double>(n)) : 0.0;
      const double f1 = n > 0 ? static_cast<double>(s1) / (2.0 * static_cast<double>(n)) : 0.0;
      w[2 * i + 0] = static_cast<float>(1.0 - gamma * f0);
      w[2 * i + 1] = static_cast<float>(1.0 - gamma * f1);
    }
  }
}

// Per-SNP factors 1 - gamma f_i(a) from an int32[n_v][3] counts array.
__global__ void k_factors_from_counts(const int32_t *__restrict__ counts, int64_t n_v,
                                      float *__restrict__ w, double gamma) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_v) return;
  const double n = counts[3 * i + 2];
  const double f0 = n > 0 ? counts[3 * i + 0] / (2.0 * n) : 0.0;
  const double f1 = n > 0 ? counts[3 * i + 1] / (2.0 * n) : 0.0;
  w[2 * i + 0] = static_cast<float>(1.0 - gamma * f0);
  w[2 * i + 1] = static_cast<float>(1.0 - gamma * f1);
}

// Four 2-bit codes (one byte) -> selector nibbles for __byte_perm.
__device__ __forceinline__ uint32_t code_nibbles(uint32_t b) {
  return (b & 0x3u) | ((b << 2) & 0x30u) | ((b << 4) & 0x300u) | ((b << 6) & 0x3000u);
}

// e4m3 bytes of rho(0) and rho(1) indexed by code: 0b00 -> (2,0), 0b01 -> (1,1),
// 0b10 (missing) -> (0,0), 0b11 -> (0,2).  e4m3: 1.0 = 0x38, 2.0 = 0x40.
constexpr uint32_t kRho0E4M3 = 0x00003840u;
constexpr uint32_t kRho1E4M3 = 0x40003800u;

// Operand rows for SNP i: row 2i holds rho_{i,q}(0), row 2i+1 holds rho_{i,q}(1),
// q = 0 .. kpad-1 (zero past n_f).  Rows past 2 n_v are zero.  One thread per
// half of a packed word (16 entries -> 16 bytes in each of the two rows), so
// that each warp store covers 512 contiguous bytes of a row.
__global__ void k_unpack_e4m3(const uint64_t *__restrict__ geno, int64_t n_f, int64_t n_v,
                              int64_t ld, uint8_t *__restrict__ op, int64_t kpad,
                              int64_t snps_pad) {
  const int64_t hpr = kpad / 16;  // 16-entry chunks per operand row
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= hpr * snps_pad) return;
  const int64_t i = t / hpr;
  const int64_t c = t - i * hpr;
  const int64_t k = c >> 1;
  uint64_t v = 0xAAAAAAAAAAAAAAAAull;  // all entries "missing" -> zero operands
  if (i < n_v && k * 32 < n_f) {
    const uint64_t valid = valid_even_mask(k, n_f);
    const uint64_t vm = valid | (valid << 1);
    v = (__ldg(geno + i * ld + k) & vm) | (0xAAAAAAAAAAAAAAAAull & ~vm);
  }
  const uint32_t h = static_cast<uint32_t>(v >> (32 * (c & 1)));
  uint32_t r0[4], r1[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const uint32_t sel = code_nibbles((h >> (8 * b)) & 0xFFu);
    r0[b] = __byte_perm(kRho0E4M3, 0u, sel);
    r1[b] = __byte_perm(kRho1E4M3, 0u, sel);
  }
  uint8_t *d0 = op + (2 * i) * kpad + c * 16;  // row-major [row][kpad]
  uint8_t *d1 = d0 + kpad;
  *reinterpret_cast<uint4 *>(d0) = make_uint4(r0[0], r0[1], r0[2], r0[3]);
  *reinterpret_cast<uint4 *>(d1) = make_uint4(r1[0], r1[1], r1[2], r1[3]);
}

// Spread the sixteen 2-bit fields of x into the low two bits of sixteen 4-bit
// fields (field q of x -> bits 4q, 4q + 1 of the result).
__device__ __forceinline__ uint64_t spread_2to4(uint32_t x32) {
  uint64_t x = x32;
  x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
  x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
  x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  return x;
}

// FP4 (e2m1) operand rows: as k_unpack_e4m3, with each count 0, 1, 2 stored as
// the e2m1 nibble 0x0, 0x2, 0x4 (2^(e-1) (1 + m/2) with e, m = 1, 0 and 2, 0),
// two entries per byte, entry q in the low nibble of byte q / 2 for even q.
// A row holds kpad / 2 bytes (kpad a multiple of 256: one 128-byte K stage is
// 256 entries).  One thread per packed word: 32 entries -> 16 bytes in each of
// the two rows, so that each warp store covers 512 contiguous bytes of a row.
// Per 2-bit field with l = low and h = high code bit: rho(1) = l + (l & h) and,
// for a present entry (not h & ~l), rho(0) = 2 - l; both are 0 when missing.
__global__ void k_unpack_e2m1(const uint64_t *__restrict__ geno, int64_t n_f, int64_t n_v,
                              int64_t ld, uint8_t *__restrict__ op, int64_t kpad,
                              int64_t snps_pad) {
  const int64_t wpr = kpad / 32;  // packed words (32 entries) per operand row
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= wpr * snps_pad) return;
  const int64_t i = t / wpr;
  const int64_t k = t - i * wpr;
  uint64_t v = 0xAAAAAAAAAAAAAAAAull;  // all entries "missing" -> zero operands
  if (i < n_v && k * 32 < n_f) {
    const uint64_t valid = valid_even_mask(k, n_f);
    const uint64_t vm = valid | (valid << 1);
    v = (__ldg(geno + i * ld + k) & vm) | (0xAAAAAAAAAAAAAAAAull & ~vm);
  }
  uint64_t n0[2], n1[2];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const uint32_t x = static_cast<uint32_t>(v >> (32 * half));
    const uint32_t l = x & 0x55555555u;
    const uint32_t h = (x >> 1) & 0x55555555u;
    const uint32_t nh = ~h & 0x55555555u;
    const uint32_t rho1 = l + (l & h);         // 2-bit fields 0, 1, 2
    const uint32_t rho0 = (nh << 1) - (l & nh);  // no borrow between fields
    n0[half] = spread_2to4(rho0) << 1;
    n1[half] = spread_2to4(rho1) << 1;
  }
  uint8_t *d0 = op + (2 * i) * (kpad / 2) + k * 16;  // row-major [row][kpad / 2]
  uint8_t *d1 = d0 + kpad / 2;
  *reinterpret_cast<uint4 *>(d0) =
      make_uint4(static_cast<uint32_t>(n0[0]), static_cast<uint32_t>(n0[0] >> 32),
                 static_cast<uint32_t>(n0[1]), static_cast<uint32_t>(n0[1] >> 32));
  *reinterpret_cast<uint4 *>(d1) =
      make_uint4(static_cast<uint32_t>(n1[0]), static_cast<uint32_t>(n1[0] >> 32),
                 static_cast<uint32_t>(n1[1]), static_cast<uint32_t>(n1[1] >> 32));
}

// k_unpack_e2m1 with the per-SNP factors w = 1 - gamma f_i(a) of
// k_allele_counts formed in the same pass over the codes: one 128-thread block
// per SNP row pair (SNPs >= n_v write zero rows), each thread one packed word
// at a time (a warp stores 512 contiguous bytes of a row), the counts n_i and
// s_i^1 summed over the block.
__global__ void __launch_bounds__(128) k_unpack_e2m1_w(const uint64_t *__restrict__ geno,
                                                      int64_t n_f, int64_t n_v, int64_t ld,
                                                      uint8_t *__restrict__ op, int64_t kpad,
                                                      float *__restrict__ w, double gamma) {
  __shared__ long long part[4][2];
  const int64_t i = blockIdx.x;
  const int64_t wpr = kpad / 32;
  const bool snp = i < n_v;
  int64_t n = 0, s1 = 0;
  for (int64_t k = threadIdx.x; k < wpr; k += 128) {
    uint64_t v = 0xAAAAAAAAAAAAAAAAull;  // all entries "missing" -> zero operands
    if (snp && k * 32 < n_f) {
      const uint64_t raw = __ldg(geno + i * ld + k);
      const uint64_t valid = valid_even_mask(k, n_f);
      const uint64_t l = raw & valid;
      const uint64_t h = (raw >> 1) & valid;
      n += __popcll(valid & ~(h & ~l));
      s1 += __popcll(l) + __popcll(h & l);
      const uint64_t vm = valid | (valid << 1);
      v = (raw & vm) | (0xAAAAAAAAAAAAAAAAull & ~vm);
    }
    uint64_t n0[2], n1[2];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const uint32_t x = static_cast<uint32_t>(v >> (32 * half));
      const uint32_t l = x & 0x55555555u;
      const uint32_t h = (x >> 1) & 0x55555555u;
      const uint32_t nh = ~h & 0x55555555u;
      const uint32_t rho1 = l + (l & h);
      const uint32_t rho0 = (nh << 1) - (l & nh);
      n0[half] = spread_2to4(rho0) << 1;
      n1[half] = spread_2to4(rho1) << 1;
    }
    uint8_t *d0 = op + (2 * i) * (kpad / 2) + k * 16;
    uint8_t *d1 = d0 + kpad / 2;
    *reinterpret_cast<uint4 *>(d0) =
        make_uint4(static_cast<uint32_t>(n0[0]), static_cast<uint32_t>(n0[0] >> 32),
                   static_cast<uint32_t>(n0[1]), static_cast<uint32_t>(n0[1] >> 32));
    *reinterpret_cast<uint4 *>(d1) =
        make_uint4(static_cast<uint32_t>(n1[0]), static_cast<uint32_t>(n1[0] >> 32),
                   static_cast<uint32_t>(n1[1]), static_cast<uint32_t>(n1[1] >> 32));
  }
  if (!snp) return;  // the whole block: i is uniform
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_xor_sync(0xffffffffu, n, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    part[warp][0] = n;
    part[warp][1] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    n = part[0][0] + part[1][0] + part[2][0] + part[3][0];
    s1 = part[0][1] + part[1][1] + part[2][1] + part[3][1];
    const int64_t s0 = 2 * n - s1;
    // 1 - gamma f_i(a), f_i(a) = s_i^a / (2 n_i), rounded once to fp32 (as k_allele_counts).
    const double f0 = n > 0 ? static_cast<double>(s0) / (2.0 * static_cast<double>(n)) : 0.0;
    const double f1 = n > 0 ? static_cast<double>(s1) / (2.0 * static_cast<double>(n)) : 0.0;
    w[2 * i + 0] = static_cast<float>(1.0 - gamma * f0);
    w[2 * i + 1] = static_cast<float>(1.0 - gamma * f1);
  }
}

// K-block-major operand rows, [K block][row][128 bytes], for the K-split
// tally kernel: a 256-thread block takes 32 SNPs (8 threads per SNP, each 16
// bytes of both of its rows per K block) over a range of K blocks, so that a
// warp store covers 1 KB of one K block (4 SNPs x 2 rows x 128 bytes) and a
// block's stores 8 KB; each thread's loads walk along its SNP's packed row.
// FP4: a K block is 256 entries (8 packed words, one per thread); e4m3: 128
// entries (4 words, a half word per thread).  SNPs in [n_v, snps_pad) get zero
// rows, as do entries past n_f.  COUNT: each SNP's n_i and s_i^1 (Eq. 1) over
// the block's entries are added into cnt[2 i], cnt[2 i + 1] (zeroed before).
template <bool FP4, bool COUNT>
__global__ void __launch_bounds__(256) k_unpack_blocked(const uint64_t *__restrict__ geno,
                                                       int64_t n_f, int64_t n_v, int64_t ld,
                                                       uint8_t *__restrict__ op, int64_t snps_pad,
                                                       int64_t nkb, int64_t blocked_rows,
                                                       int64_t kb_per, int32_t *__restrict__ cnt) {
  const int sub = threadIdx.x & 7;
  const int64_t i = static_cast<int64_t>(blockIdx.x) * 32 + (threadIdx.x >> 3);
  if (i >= snps_pad) return;
  const int64_t kb0 = static_cast<int64_t>(blockIdx.y) * kb_per;
  const int64_t kb1 = kb0 + kb_per < nkb ? kb0 + kb_per : nkb;
  const bool snp = i < n_v;
  const uint64_t *row = geno + i * ld;
  uint8_t *base = op + 2 * i * 128 + sub * 16;
  const int64_t kb_stride = blocked_rows * 128;
  int32_t n = 0, s1 = 0;
#pragma unroll 4
  for (int64_t kb = kb0; kb < kb1; ++kb) {
    const int64_t c = kb * 8 + sub;      // 16-byte piece of the row pair
    const int64_t k = FP4 ? c : c >> 1;  // packed word
    uint64_t v = 0xAAAAAAAAAAAAAAAAull;  // all entries "missing" -> zero operands
    if (snp && k * 32 < n_f) {
      const uint64_t valid = valid_even_mask(k, n_f);
      const uint64_t vm = valid | (valid << 1);
      v = (__ldg(row + k) & vm) | (0xAAAAAAAAAAAAAAAAull & ~vm);
    }
    if constexpr (COUNT) {
      // Present entries (not h & ~l) and rho(1) = l + (l & h) of this thread's
      // entries: the whole word (e2m1) or its half (e4m3); padding reads as missing.
      const uint64_t x = FP4 ? v : (v >> (32 * (sub & 1))) & 0xFFFFFFFFull;
      const uint64_t even = FP4 ? kEven : 0x55555555ull;
      const uint64_t l = x & even, h = (x >> 1) & even;
      n += __popcll(even & ~(h & ~l));
      s1 += __popcll(l) + __popcll(h & l);
    }
    uint4 q0, q1;
    if constexpr (FP4) {
      uint64_t n0[2], n1[2];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const uint32_t x = static_cast<uint32_t>(v >> (32 * half));
        const uint32_t l = x & 0x55555555u;
        const uint32_t h = (x >> 1) & 0x55555555u;
        const uint32_t nh = ~h & 0x55555555u;
        n0[half] = spread_2to4((nh << 1) - (l & nh)) << 1;
        n1[half] = spread_2to4(l + (l & h)) << 1;
      }
      q0 = make_uint4(static_cast<uint32_t>(n0[0]), static_cast<uint32_t>(n0[0] >> 32),
                      static_cast<uint32_t>(n0[1]), static_cast<uint32_t>(n0[1] >> 32));
      q1 = make_uint4(static_cast<uint32_t>(n1[0]), static_cast<uint32_t>(n1[0] >> 32),
                      static_cast<uint32_t>(n1[1]), static_cast<uint32_t>(n1[1] >> 32));
    } else {
      const uint32_t h = static_cast<uint32_t>(v >> (32 * (sub & 1)));
      uint32_t r0[4], r1[4];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const uint32_t sel = code_nibbles((h >> (8 * b)) & 0xFFu);
        r0[b] = __byte_perm(kRho0E4M3, 0u, sel);
        r1[b] = __byte_perm(kRho1E4M3, 0u, sel);
      }
      q0 = make_uint4(r0[0], r0[1], r0[2], r0[3]);
      q1 = make_uint4(r1[0], r1[1], r1[2], r1[3]);
    }
    uint8_t *d0 = base + kb * kb_stride;
    *reinterpret_cast<uint4 *>(d0) = q0;
    *reinterpret_cast<uint4 *>(d0 + 128) = q1;
  }
  if constexpr (COUNT) {
    // The 8 threads of a SNP are 8 aligned lanes of one warp.
    const unsigned group = 0xFFu << (threadIdx.x & 24);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      n += __shfl_xor_sync(group, n, o);
      s1 += __shfl_xor_sync(group, s1, o);
    }
    if (sub == 0 && snp && kb0 < kb1) {
      atomicAdd(cnt + 2 * i, n);
      atomicAdd(cnt + 2 * i + 1, s1);
    }
  }
}

// The per-SNP factors 1 - gamma f_i(a) in place of the counts n_i, s_i^1 that
// k_unpack_blocked summed into the same 8 bytes per SNP (the same arithmetic
// as k_allele_counts).
__global__ void k_factors_in_place(float *__restrict__ w, int64_t n_v, double gamma) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n_v) return;
  const int2 c = reinterpret_cast<const int2 *>(w)[i];
  const int64_t n = c.x, s1 = c.y, s0 = 2 * n - s1;
  const double f0 = n > 0 ? static_cast<double>(s0) / (2.0 * static_cast<double>(n)) : 0.0;
  const double f1 = n > 0 ? static_cast<double>(s1) / (2.0 * static_cast<double>(n)) : 0.0;
  reinterpret_cast<float2 *>(w)[i] = make_float2(static_cast<float>(1.0 - gamma * f0),
                                                 static_cast<float>(1.0 - gamma * f1));
}

// Gather the 32 even-position bits of x into the low 32 bits.
__device__ __forceinline__ uint64_t compact_even(uint64_t x) {
  x &= kEven;
  x = (x | (x >> 1)) & 0x3333333333333333ull;
  x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
  x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
  x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
  return x;
}

// Bit planes per 64 entries: P1 = l (one copy of allele 1 for het and hom 1),
// P2 = h & l (the second copy, hom 1 only), M = present; rho_1 = P1 + P2,
// rho_0 = 2M - P1 - P2.  planes[(i * w64 + b) * 4 + {0,1,2}] = {P1, P2, M}.
__global__ void k_planes(const uint64_t *__restrict__ geno, int64_t n_f, int64_t n_v, int64_t ld,
                         uint64_t *__restrict__ planes, int64_t w64) {
  const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n_v * w64) return;
  const int64_t i = t / w64;
  const int64_t b = t - i * w64;
  uint64_t l = 0, h = 0, valid = 0;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int64_t k = 2 * b + half;
    if (k * 32 < n_f) {
      const uint64_t v = geno[i * ld + k];
      const uint64_t vm = valid_even_mask(k, n_f);
      l |= compact_even(v & vm) << (32 * half);
      h |= compact_even((v >> 1) & vm) << (32 * half);
      valid |= compact_even(vm) << (32 * half);
    }
  }
  uint4 *d = reinterpret_cast<uint4 *>(planes + t * 4);
  const uint64_t p1 = l;
  const uint64_t p2 = h & l;
  const uint64_t m = valid & (~h | l);
  d[0] = make_uint4(static_cast<uint32_t>(p1), static_cast<uint32_t>(p1 >> 32),
                    static_cast<uint32_t>(p2), static_cast<uint32_t>(p2 >> 32));
  d[1] = make_uint4(static_cast<uint32_t>(m), static_cast<uint32_t>(m >> 32), 0u, 0u);
}

}  // namespace

int launch_allele_counts(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld,
                         int32_t *counts, float *w, double gamma, cudaStream_t s) {
  if (n_v < 1) return CCC_OK;
  // Warps per SNP: double while the grid holds under 32 warps per SM and every
  // lane still gets at least two words.
  const int64_t words = (n_f + 31) / 32;
  int wps = 1;
  while (wps < 8 && n_v * wps < 152 * 32 && words >= 64 * 2 * wps) wps *= 2;
  const int64_t per_block = 8 / wps;
  const unsigned blocks = static_cast<unsigned>((n_v + per_block - 1) / per_block);
  switch (wps) {
    case 1:
      k_allele_counts<1><<<blocks, 256, 0, s>>>(geno, n_f, n_v, ld, counts, w, gamma);
      break;
    case 2:
      k_allele_counts<2><<<blocks, 256, 0, s>>>(geno, n_f, n_v, ld, counts, w, gamma);
      break;
    case 4:
      k_allele_counts<4><<<blocks, 256, 0, s>>>(geno, n_f, n_v, ld, counts, w, gamma);
      break;
    default:
      k_allele_counts<8><<<blocks, 256, 0, s>>>(geno, n_f, n_v, ld, counts, w, gamma);
      break;
  }
  return note_launch();
}

int launch_factors_from_counts(const int32_t *counts, int64_t n_v, float *w, double gamma,
                               cudaStream_t s) {
  const int threads = 256;
  const int64_t blocks = (n_v + threads - 1) / threads;
  k_factors_from_counts<<<static_cast<unsigned>(blocks), threads, 0, s>>>(counts, n_v, w, gamma);
  return note_launch();
}

int launch_unpack_blocked(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *op,
                          int64_t kpad, int64_t snps_pad, int64_t blocked_rows, bool fp4, float *w,
                          double gamma, cudaStream_t s) {
  const int64_t kblock = fp4 ? 256 : 128;  // entries per 128-byte K block
  if (kpad % kblock != 0 || snps_pad % 32 != 0 || snps_pad < n_v || blocked_rows < 2 * snps_pad)
    return CCC_EINVAL;
  const int64_t nkb = kpad / kblock;
  if (snps_pad < 1 || nkb < 1) return CCC_OK;
  // 32-SNP blocks times K ranges, about 16 blocks per SM in all.
  const int64_t gx = snps_pad / 32;
  if (gx > 0x7FFFFFFF) return CCC_EINVAL;
  int64_t gy = (152 * 16 + gx - 1) / gx;
  if (gy > nkb) gy = nkb;
  if (gy > 65535) gy = 65535;
  const int64_t kb_per = (nkb + gy - 1) / gy;
  gy = (nkb + kb_per - 1) / kb_per;
  const dim3 grid(static_cast<unsigned>(gx), static_cast<unsigned>(gy));
  int32_t *cnt = reinterpret_cast<int32_t *>(w);
  if (w != nullptr && cudaMemsetAsync(w, 0, 8 * static_cast<size_t>(n_v), s) != cudaSuccess)
    return CCC_ECUDA;
  if (fp4 && w != nullptr)
    k_unpack_blocked<true, true><<<grid, 256, 0, s>>>(geno, n_f, n_v, ld, op, snps_pad, nkb,
                                                      blocked_rows, kb_per, cnt);
  else if (fp4)
    k_unpack_blocked<true, false><<<grid, 256, 0, s>>>(geno, n_f, n_v, ld, op, snps_pad, nkb,
                                                       blocked_rows, kb_per, nullptr);
  else if (w != nullptr)
    k_unpack_blocked<false, true><<<grid, 256, 0, s>>>(geno, n_f, n_v, ld, op, snps_pad, nkb,
                                                       blocked_rows, kb_per, cnt);
  else
    k_unpack_blocked<false, false><<<grid, 256, 0, s>>>(geno, n_f, n_v, ld, op, snps_pad, nkb,
                                                        blocked_rows, kb_per, nullptr);
  const int rc = note_launch();
  if (rc != CCC_OK || w == nullptr) return rc;
  const unsigned fb = static_cast<unsigned>((n_v + 255) / 256);
  k_factors_in_place<<<fb, 256, 0, s>>>(w, n_v, gamma);
  return note_launch();
}

int launch_unpack_e4m3(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *op,
                       int64_t kpad, int64_t snps_pad, cudaStream_t s, int64_t blocked_rows) {
  if (blocked_rows != 0)
    return launch_unpack_blocked(geno, n_f, n_v, ld, op, kpad, snps_pad, blocked_rows, false,
                                 nullptr, 0.0, s);
  const int threads = 256;
  const int64_t total = (kpad / 16) * snps_pad;
  const int64_t blocks = (total + threads - 1) / threads;
  k_unpack_e4m3<<<static_cast<unsigned>(blocks), threads, 0, s>>>(geno, n_f, n_v, ld, op, kpad,
                                                                   snps_pad);
  return note_launch();
}

int launch_unpack_e2m1(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *op,
                       int64_t kpad, int64_t snps_pad, cudaStream_t s, int64_t blocked_rows,
                       float *w, double gamma) {
  if (kpad % 256 != 0) return CCC_EINVAL;
  if (blocked_rows != 0)
    return launch_unpack_blocked(geno, n_f, n_v, ld, op, kpad, snps_pad, blocked_rows, true, w,
                                 gamma, s);
  // Fused with the factors while one 128-thread block per SNP still gives the
  // GPU enough loads in flight (152 SMs x 8 blocks); a few long rows take the
  // flat unpack (a thread per word) and the multi-warp count kernel instead.
  if (w != nullptr && snps_pad >= 152 * 8) {
    if (snps_pad < n_v) return CCC_EINVAL;
    k_unpack_e2m1_w<<<static_cast<unsigned>(snps_pad), 128, 0, s>>>(geno, n_f, n_v, ld, op, kpad,
                                                                     w, gamma);
    return note_launch();
  }
  if (w != nullptr) {
    const int rc = launch_allele_counts(geno, n_f, n_v, ld, nullptr, w, gamma, s);
    if (rc != CCC_OK) return rc;
  }
  const int threads = 256;
  const int64_t total = (kpad / 32) * snps_pad;
  const int64_t blocks = (total + threads - 1) / threads;
  k_unpack_e2m1<<<static_cast<unsigned>(blocks), threads, 0, s>>>(geno, n_f, n_v, ld, op, kpad,
                                                                   snps_pad);
  return note_launch();
}

int launch_planes(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint64_t *planes,
                  int64_t w64, cudaStream_t s) {
  const int threads = 256;
  const int64_t blocks = (n_v * w64 + threads - 1) / threads;
  k_planes<<<static_cast<unsigned>(blocks), threads, 0, s>>>(geno, n_f, n_v, ld, planes, w64);
  return note_launch();
}

}  // namespace ccc
