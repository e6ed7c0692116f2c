// 3-way tallies by bitwise AND + population count (the plain form of Sec. 3.2,
// where each 3-way tally is assembled from bitwise 2-way tallies masked by v_j).
//
// With the bit planes of k_planes (P1, P2 = the two copies of allele 1,
// M = present), rho_1 = P1 + P2 and m = M.  For each triple the eight sums
//     T[x y z] = sum_q X_i Y_j Z_k,  X, Y, Z in {rho_1, m}
// come from AND+POPC of plane triples, and the tallies follow from
// rho_0 = 2m - rho_1:
//     r^{abc} = sum_{x,y,z} C_a(x) C_b(y) C_c(z) T[x y z],
//     C_1(rho_1) = 1, C_1(m) = 0, C_0(rho_1) = -1, C_0(m) = 2.
// The (i, j) plane products are formed once per staged word and shared by all
// k.  P2 is a subset of P1, so of the four (rho_1, rho_1) products the cross
// terms p = P1i & P2j, q = P2i & P1j satisfy p & q = P2i & P2j and enter as
// p ^ q and 3 (p & q): eight (i, j) products, 24 POPC per 64 comparisons
// instead of 27.  Block: one slab j (blockIdx.y), a tile of 32 SNPs i < j by
// 64 SNPs k > j, 256 threads, 2 x 4 triples per thread.
#include "ccc_launch.h"
#include "ccc_dev.cuh"
#include "ccc_metric.cuh"

namespace ccc {
namespace {

constexpr int TI = 32;
constexpr int TK = 64;
constexpr int KC = 8;  // 64-entry words per stage
constexpr int THREADS = 256;

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

__device__ __forceinline__ void planes_of(const uint64_t *__restrict__ planes, int64_t w64,
                                          int64_t s, int64_t k, uint64_t &p1, uint64_t &p2,
                                          uint64_t &m) {
  const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(planes + (s * w64 + k) * 4));
  const uint4 v1 = __ldg(reinterpret_cast<const uint4 *>(planes + (s * w64 + k) * 4) + 1);
  p1 = (static_cast<uint64_t>(v0.y) << 32) | v0.x;
  p2 = (static_cast<uint64_t>(v0.w) << 32) | v0.z;
  m = (static_cast<uint64_t>(v1.y) << 32) | v1.x;
}

__global__ void __launch_bounds__(THREADS)
    k_tally3_popc(const uint64_t *__restrict__ planes, int64_t w64, const Tally3Args args) {
  constexpr int NIJ = 8;
  __shared__ uint64_t sIJ[NIJ][KC][TI + 1];
  __shared__ uint64_t sK[3][KC][TK + 1];
  const int64_t n_v = args.n_v;
  const int64_t j = args.j_begin + blockIdx.y;
  const int64_t mt = cdiv(j, TI);
  const int64_t nt = cdiv(n_v - 1 - j, TK);
  if (static_cast<int64_t>(blockIdx.x) >= mt * nt) return;
  const int64_t i0 = (blockIdx.x / nt) * TI;
  const int64_t k0 = j + 1 + (blockIdx.x % nt) * TK;
  const int tx = threadIdx.x & 15;
  const int ty = threadIdx.x >> 4;
  uint32_t T[2][4][8];
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
      for (int z = 0; z < 8; ++z) T[x][y][z] = 0u;

  for (int64_t kw0 = 0; kw0 < w64; kw0 += KC) {
    // i side: 32 SNPs x KC words -> eight plane products with v_j:
    // (rho_1, rho_1): P1P1, p ^ q, p & q (weight 3); (rho_1, m): P1M, P2M;
    // (m, rho_1): MP1, MP2; (m, m): MM.
    for (int l = threadIdx.x; l < TI * KC; l += THREADS) {
      const int word = l % KC;
      const int si = l / KC;
      const int64_t i = i0 + si;
      const int64_t k = kw0 + word;
      uint64_t a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
      if (i < j && k < w64) {
        planes_of(planes, w64, i, k, a[0], a[1], a[2]);
        planes_of(planes, w64, j, k, b[0], b[1], b[2]);
      }
      const uint64_t p = a[0] & b[1], q = a[1] & b[0];
      sIJ[0][word][si] = a[0] & b[0];
      sIJ[1][word][si] = p ^ q;
      sIJ[2][word][si] = p & q;
      sIJ[3][word][si] = a[0] & b[2];
      sIJ[4][word][si] = a[1] & b[2];
      sIJ[5][word][si] = a[2] & b[0];
      sIJ[6][word][si] = a[2] & b[1];
      sIJ[7][word][si] = a[2] & b[2];
    }
    // k side: 64 SNPs x KC words.
    for (int l = threadIdx.x; l < TK * KC; l += THREADS) {
      const int word = l % KC;
      const int sk = l / KC;
      const int64_t kk = k0 + sk;
      const int64_t k = kw0 + word;
      uint64_t c[3] = {0, 0, 0};
      if (kk < n_v && k < w64) planes_of(planes, w64, kk, k, c[0], c[1], c[2]);
#pragma unroll
      for (int p = 0; p < 3; ++p) sK[p][word][sk] = c[p];
    }
    __syncthreads();
#pragma unroll 2
    for (int w = 0; w < KC; ++w) {
      uint64_t kp[4][3];
#pragma unroll
      for (int y = 0; y < 4; ++y)
#pragma unroll
        for (int p = 0; p < 3; ++p) kp[y][p] = sK[p][w][tx + 16 * y];
#pragma unroll
      for (int x = 0; x < 2; ++x) {
#pragma unroll
        for (int pij = 0; pij < NIJ; ++pij) {
          const uint64_t ij = sIJ[pij][w][ty + 16 * x];
          // plane type of the i and j factors: rho_1 (0) or m (1)
          const int tI = pij >= 5 ? 1 : 0;
          const int tJ = (pij == 3 || pij == 4 || pij == 7) ? 1 : 0;
          const uint32_t wt = pij == 2 ? 3u : 1u;
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            T[x][y][4 * tI + 2 * tJ + 0] += wt * (__popcll(ij & kp[y][0]) + __popcll(ij & kp[y][1]));
            T[x][y][4 * tI + 2 * tJ + 1] += wt * __popcll(ij & kp[y][2]);
          }
        }
      }
    }
    __syncthreads();
  }

  const int64_t span = n_v - 1 - j;
  const int64_t s0 = slab_offset_dev(j, n_v) - slab_offset_dev(args.j_begin, n_v);
  const bool persnp = args.norm == CCC_NORM_PERSNP;
  float wj0 = 1.f, wj1 = 1.f;
  if (args.ccc != nullptr && persnp) {
    wj0 = __ldg(args.w + 2 * j);
    wj1 = __ldg(args.w + 2 * j + 1);
  }
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    const int64_t i = i0 + ty + 16 * x;
    if (i >= j) continue;
    float wi0 = 1.f, wi1 = 1.f;
    if (args.ccc != nullptr && persnp) {
      wi0 = __ldg(args.w + 2 * i);
      wi1 = __ldg(args.w + 2 * i + 1);
    }
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int64_t k = k0 + tx + 16 * y;
      if (k >= n_v) continue;
      int32_t r[8];
#pragma unroll
      for (int abc = 0; abc < 8; ++abc) {
        const int aa = abc >> 2, bb = (abc >> 1) & 1, cc = abc & 1;
        int32_t sum = 0;
#pragma unroll
        for (int xyz = 0; xyz < 8; ++xyz) {
          const int xx = xyz >> 2, yy = (xyz >> 1) & 1, zz = xyz & 1;
          // C_1 = (1, 0), C_0 = (-1, 2) over (rho_1, m)
          const int ca = aa ? (xx ? 0 : 1) : (xx ? 2 : -1);
          const int cb = bb ? (yy ? 0 : 1) : (yy ? 2 : -1);
          const int cz = cc ? (zz ? 0 : 1) : (zz ? 2 : -1);
          sum += ca * cb * cz * static_cast<int32_t>(T[x][y][xyz]);
        }
        r[abc] = sum;
      }
      const int64_t t = s0 + i * span + (k - j - 1);
      if (!CCC_IN_BOUNDS(t, args.out_len, args.status)) continue;
      int4 *td = reinterpret_cast<int4 *>(args.tally) + 2 * t;
      td[0] = make_int4(r[0], r[1], r[2], r[3]);
      td[1] = make_int4(r[4], r[5], r[6], r[7]);
      if (args.ccc != nullptr) {
        float wk0 = 1.f, wk1 = 1.f;
        if (persnp) {
          const float2 wk = __ldg(reinterpret_cast<const float2 *>(args.w) + k);
          wk0 = wk.x;
          wk1 = wk.y;
        }
        float o[8];
        ccc3_values(r, wi0, wi1, wj0, wj1, wk0, wk1, args.norm, args.gamma, o);
        float4 *cd = reinterpret_cast<float4 *>(args.ccc) + 2 * t;
        cd[0] = make_float4(o[0], o[1], o[2], o[3]);
        cd[1] = make_float4(o[4], o[5], o[6], o[7]);
      }
    }
  }
}

// 3-way CCC values from stored tallies: blockIdx.y = slab, threads over (i, k).
__global__ void k_metric3(const int32_t *__restrict__ tally, const float *__restrict__ w,
                          int64_t n_v, int64_t j_begin, float gamma, int32_t norm,
                          float *__restrict__ ccc) {
  const int64_t j = j_begin + blockIdx.y;
  const int64_t span = n_v - 1 - j;
  const int64_t count = j * span;
  const int64_t s0 = slab_offset_dev(j, n_v) - slab_offset_dev(j_begin, n_v);
  const bool persnp = norm == CCC_NORM_PERSNP;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t i = e / span;
    const int64_t k = j + 1 + (e - i * span);
    const int64_t t = s0 + e;
    const int4 a = __ldg(reinterpret_cast<const int4 *>(tally) + 2 * t);
    const int4 b = __ldg(reinterpret_cast<const int4 *>(tally) + 2 * t + 1);
    const int32_t r[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    float wi0 = 1.f, wi1 = 1.f, wj0 = 1.f, wj1 = 1.f, wk0 = 1.f, wk1 = 1.f;
    if (persnp) {
      wi0 = __ldg(w + 2 * i);
      wi1 = __ldg(w + 2 * i + 1);
      wj0 = __ldg(w + 2 * j);
      wj1 = __ldg(w + 2 * j + 1);
      wk0 = __ldg(w + 2 * k);
      wk1 = __ldg(w + 2 * k + 1);
    }
    float o[8];
    ccc3_values(r, wi0, wi1, wj0, wj1, wk0, wk1, norm, gamma, o);
    float4 *cd = reinterpret_cast<float4 *>(ccc) + 2 * t;
    cd[0] = make_float4(o[0], o[1], o[2], o[3]);
    cd[1] = make_float4(o[4], o[5], o[6], o[7]);
  }
}

}  // namespace

int launch_tally3_popc(const Tally3Args &a, const uint64_t *planes, int64_t w64, cudaStream_t s) {
  const int64_t slabs = a.j_end - a.j_begin;
  if (slabs <= 0) return CCC_OK;
  if (slabs > 65535) return CCC_ERANGE;
  int64_t max_tiles = 0;
  for (int64_t j = a.j_begin; j < a.j_end; ++j) {
    const int64_t t = cdiv(j, TI) * cdiv(a.n_v - 1 - j, TK);
    if (t > max_tiles) max_tiles = t;
  }
  if (max_tiles == 0) return CCC_OK;
  if (max_tiles > 0x7fffffffLL) return CCC_ERANGE;
  dim3 grid(static_cast<unsigned>(max_tiles), static_cast<unsigned>(slabs));
  k_tally3_popc<<<grid, THREADS, 0, s>>>(planes, w64, a);
  return note_launch();
}

int launch_metric3(const int32_t *tally, const float *w, int64_t n_v, int64_t j_begin,
                   int64_t j_end, float gamma, int32_t norm, float *ccc, cudaStream_t s) {
  const int64_t slabs = j_end - j_begin;
  if (slabs <= 0) return CCC_OK;
  if (slabs > 65535) return CCC_ERANGE;
  int64_t max_count = 0;
  for (int64_t j = j_begin; j < j_end; ++j) max_count = max_count > j * (n_v - 1 - j) ? max_count : j * (n_v - 1 - j);
  if (max_count == 0) return CCC_OK;
  const int64_t bx = cdiv(max_count, 256) < 1024 ? cdiv(max_count, 256) : 1024;
  dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(slabs));
  k_metric3<<<grid, 256, 0, s>>>(tally, w, n_v, j_begin, gamma, norm, ccc);
  return note_launch();
}

}  // namespace ccc
