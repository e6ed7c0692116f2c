// 2-way tallies by bitwise AND + population count on the CUDA cores: the plain
// form of Sec. 3.1, where every 2-bit entry is handled by word-wide bitwise
// operations and counted with a hardware population count.
//
// Each SNP is held as three bit planes per 64 entries (built by k_planes):
// P1 = first copy of allele 1 (het or hom 1), P2 = second copy (hom 1),
// M = present.  With rho_1 = P1 + P2 and rho_0 = 2M - rho_1:
//   r11 = sum_q rho_1,i rho_1,j = |P1i&P1j| + |P1i&P2j| + |P2i&P1j| + |P2i&P2j|
//   X   = sum_q rho_1,i m_j     = |P1i&Mj| + |P2i&Mj|
//   Y   = sum_q m_i rho_1,j     = |Mi&P1j| + |Mi&P2j|
//   Z   = sum_q m_i m_j         = |Mi&Mj|
//   r10 = 2X - r11,  r01 = 2Y - r11,  r00 = 4Z - 2X - 2Y + r11.
// P2 is a subset of P1 (hom 1 implies a first copy), so of the four r11 terms
// the last three take two population counts (see the inner loop): eight
// POPC per 64 entries per pair; four accumulators per pair.
//
// Block tile: 64 x 64 SNPs of the upper triangle (J >= I), 256 threads, each
// thread 4 x 4 pairs; the planes of both tiles are staged in shared memory 8
// words (512 entries) at a time.  A K split (gridDim.y parts) gives each block
// a range of words; since the four tallies are linear in the four sums, the
// parts add their partial tallies into the zeroed output with integer
// reductions, and the CCC values follow from the summed tallies (k_metric2).
#include "ccc_dev.cuh"
#include "ccc_launch.h"
#include "ccc_metric.cuh"

namespace ccc {
namespace {

constexpr int TS = 64;       // SNPs per tile side
constexpr int KC = 8;        // 64-entry words per stage
constexpr int THREADS = 256;
constexpr int LDS = TS + 1;  // padded row (u64) against bank conflicts

__device__ __forceinline__ void tile_coords(int64_t t, int64_t nB, int64_t &I, int64_t &J) {
  // Row-major upper triangle with diagonal: row I holds nB - I tiles.
  const double b = 2.0 * nB + 1.0;
  int64_t r = static_cast<int64_t>((b - sqrt(b * b - 8.0 * static_cast<double>(t))) * 0.5);
  if (r < 0) r = 0;
  if (r >= nB) r = nB - 1;
  auto start = [&](int64_t row) { return row * nB - row * (row - 1) / 2; };
  while (r > 0 && start(r) > t) --r;
  while (r + 1 < nB && start(r + 1) <= t) ++r;
  I = r;
  J = r + (t - start(r));
}

__device__ __forceinline__ void load_stage(const uint64_t *__restrict__ planes, int64_t w64,
                                           int64_t kend, int64_t n_v, int64_t snp0, int64_t k0,
                                           uint64_t (*s)[KC][LDS]) {
  // 64 SNPs x KC words x 2 halves of 16 bytes.
  for (int l = threadIdx.x; l < TS * KC * 2; l += THREADS) {
    const int half = l & 1;
    const int word = (l >> 1) % KC;
    const int snp = (l >> 1) / KC;
    const int64_t i = snp0 + snp;
    const int64_t k = k0 + word;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (i < n_v && k < kend) v = __ldg(reinterpret_cast<const uint4 *>(planes + (i * w64 + k) * 4) + half);
    const uint64_t lo = (static_cast<uint64_t>(v.y) << 32) | v.x;
    const uint64_t hi = (static_cast<uint64_t>(v.w) << 32) | v.z;
    if (half == 0) {
      s[0][word][snp] = lo;
      s[1][word][snp] = hi;
    } else {
      s[2][word][snp] = lo;
    }
  }
}

__global__ void __launch_bounds__(THREADS)
    k_tally2_popc(const uint64_t *__restrict__ planes, int64_t w64, const Tally2Args args,
                  int64_t nB, int64_t t0, int64_t part_words) {
  __shared__ uint64_t sI[3][KC][LDS];
  __shared__ uint64_t sJ[3][KC][LDS];
  int64_t I, J;
  tile_coords(t0 + blockIdx.x, nB, I, J);
  const int64_t n_v = args.n_v;
  const int tx = threadIdx.x & 15;
  const int ty = threadIdx.x >> 4;
  uint32_t acc[4][4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[x][y][c] = 0u;

  const int64_t kbeg = static_cast<int64_t>(blockIdx.y) * part_words;
  const int64_t kend = kbeg + part_words < w64 ? kbeg + part_words : w64;
  for (int64_t k0 = kbeg; k0 < kend; k0 += KC) {
    load_stage(planes, w64, kend, n_v, I * TS, k0, sI);
    load_stage(planes, w64, kend, n_v, J * TS, k0, sJ);
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KC; ++k) {
      uint64_t a1[4], a2[4], am[4], b1[4], b2[4], bm[4];
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        a1[x] = sI[0][k][ty + 16 * x];
        a2[x] = sI[1][k][ty + 16 * x];
        am[x] = sI[2][k][ty + 16 * x];
      }
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        b1[y] = sJ[0][k][tx + 16 * y];
        b2[y] = sJ[1][k][tx + 16 * y];
        bm[y] = sJ[2][k][tx + 16 * y];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          // P2 is a subset of P1, so (P1i & P2j) & (P2i & P1j) = P2i & P2j and
          // |P1i&P2j| + |P2i&P1j| + |P2i&P2j| = |p ^ q| + 3 |p & q|.
          const uint64_t p = a1[x] & b2[y], q = a2[x] & b1[y];
          acc[x][y][0] += __popcll(a1[x] & b1[y]) + __popcll(p ^ q) + 3 * __popcll(p & q);
          acc[x][y][1] += __popcll(a1[x] & bm[y]) + __popcll(a2[x] & bm[y]);
          acc[x][y][2] += __popcll(am[x] & b1[y]) + __popcll(am[x] & b2[y]);
          acc[x][y][3] += __popcll(am[x] & bm[y]);
        }
    }
    __syncthreads();
  }

#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int64_t i = I * TS + ty + 16 * x;
    if (i >= n_v || i < args.i_begin || i >= args.i_end) continue;
    const bool filter = args.hits != nullptr;
    const bool partial = gridDim.y > 1;  // K split: partial tallies, no CCC here
    const bool want_ccc = !partial && (filter || args.ccc != nullptr);
    float wi0 = 1.f, wi1 = 1.f;
    if (want_ccc && args.norm == CCC_NORM_PERSNP) {
      wi0 = __ldg(args.w + 2 * i);
      wi1 = __ldg(args.w + 2 * i + 1);
    }
    const int64_t row_base = i * (2 * n_v - i - 1) / 2 - i - 1 - args.pair0;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t j = J * TS + tx + 16 * y;
      if (!(i < j && j < n_v)) continue;
      const int32_t r11 = static_cast<int32_t>(acc[x][y][0]);
      const int32_t X = static_cast<int32_t>(acc[x][y][1]);
      const int32_t Y = static_cast<int32_t>(acc[x][y][2]);
      const int32_t Z = static_cast<int32_t>(acc[x][y][3]);
      const int32_t r10 = 2 * X - r11;
      const int32_t r01 = 2 * Y - r11;
      const int32_t r00 = 4 * Z - 2 * X - 2 * Y + r11;
      const int64_t pidx = row_base + j;
      if (!filter && !CCC_IN_BOUNDS(pidx, args.out_len, args.status)) continue;
      if (partial) {
        int32_t *t = args.tally + 4 * pidx;
        if (r00 != 0) atomicAdd(t + 0, r00);
        if (r01 != 0) atomicAdd(t + 1, r01);
        if (r10 != 0) atomicAdd(t + 2, r10);
        if (r11 != 0) atomicAdd(t + 3, r11);
        continue;
      }
      if (!filter) reinterpret_cast<int4 *>(args.tally)[pidx] = make_int4(r00, r01, r10, r11);
      if (want_ccc) {
        float wj0 = 1.f, wj1 = 1.f;
        if (args.norm == CCC_NORM_PERSNP) {
          const float2 wj = __ldg(reinterpret_cast<const float2 *>(args.w) + j);
          wj0 = wj.x;
          wj1 = wj.y;
        }
        const float4 cv =
            ccc2_values(r00, r01, r10, r11, wi0, wi1, wj0, wj1, args.norm, args.gamma);
        if (filter)
          filter_pair(args.hits, args.n_hits, args.cap, args.threshold, i, j, r00, r01, r10, r11,
                      cv);
        else
          reinterpret_cast<float4 *>(args.ccc)[pidx] = cv;
      }
    }
  }
}

// CCC values from stored tallies: one block per row i, threads over j > i.
__global__ void k_metric2(const int32_t *__restrict__ tally, const float *__restrict__ w,
                          int64_t n_v, float gamma, int32_t norm, float *__restrict__ ccc) {
  for (int64_t i = blockIdx.x; i < n_v; i += gridDim.x) {
    const int64_t row_base = i * (2 * n_v - i - 1) / 2 - i - 1;
    float wi0 = 1.f, wi1 = 1.f;
    if (norm == CCC_NORM_PERSNP) {
      wi0 = __ldg(w + 2 * i);
      wi1 = __ldg(w + 2 * i + 1);
    }
    for (int64_t j = i + 1 + threadIdx.x; j < n_v; j += blockDim.x) {
      const int4 r = __ldg(reinterpret_cast<const int4 *>(tally) + row_base + j);
      float wj0 = 1.f, wj1 = 1.f;
      if (norm == CCC_NORM_PERSNP) {
        const float2 wj = __ldg(reinterpret_cast<const float2 *>(w) + j);
        wj0 = wj.x;
        wj1 = wj.y;
      }
      reinterpret_cast<float4 *>(ccc)[row_base + j] =
          ccc2_values(r.x, r.y, r.z, r.w, wi0, wi1, wj0, wj1, norm, gamma);
    }
  }
}

}  // namespace

int64_t popc2_tiles(int64_t n_v) {
  const int64_t nB = (n_v + TS - 1) / TS;
  return nB * (nB + 1) / 2;
}

int launch_tally2_popc(const Tally2Args &a, const uint64_t *planes, int64_t w64, cudaStream_t s,
                       int split) {
  const int64_t nB = (a.n_v + TS - 1) / TS;
  // Row blocks [B0, B1) of the phase; tiles before row B are B nB - B (B - 1) / 2.
  const int64_t B0 = (a.i_begin > 0 ? a.i_begin : 0) / TS;
  const int64_t B1 = a.i_end < a.n_v ? (a.i_end + TS - 1) / TS : nB;
  auto start = [&](int64_t r) { return r * nB - r * (r - 1) / 2; };
  const int64_t t0 = start(B0);
  const int64_t tiles = start(B1) - t0;
  if (tiles <= 0) return CCC_OK;
  if (tiles > 0x7fffffffLL) return CCC_ERANGE;
  // Parts of whole KC-word stages; split > 1 only with a.tally zeroed, no
  // thresholded output and the CCC values formed afterwards.
  const int64_t stages = (w64 + KC - 1) / KC;
  if (split < 1 || split > 65535 || (split > 1 && a.hits != nullptr)) return CCC_EINVAL;
  if (split > stages) split = static_cast<int>(stages);
  const int64_t part_words = (stages + split - 1) / split * KC;
  const int parts = static_cast<int>((w64 + part_words - 1) / part_words);
  const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(parts > 0 ? parts : 1), 1);
  k_tally2_popc<<<grid, THREADS, 0, s>>>(planes, w64, a, nB, t0, parts > 1 ? part_words : w64);
  return note_launch();
}

int launch_metric2(const int32_t *tally, const float *w, int64_t n_v, float gamma, int32_t norm,
                   float *ccc, cudaStream_t s) {
  const int64_t blocks = n_v < 65536 ? n_v : 65536;
  if (blocks <= 0) return CCC_OK;
  k_metric2<<<static_cast<unsigned>(blocks), 256, 0, s>>>(tally, w, n_v, gamma, norm, ccc);
  return note_launch();
}

}  // namespace ccc
