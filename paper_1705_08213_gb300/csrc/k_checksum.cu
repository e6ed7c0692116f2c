// Exact checksum of computed results (the extended-precision integer checksum
// the paper's code uses to check results bit for bit, Sec. 5).
//
// C = sum_e h(base + e) * word[e]  (mod 2^128), where word[e] is the e-th
// 32-bit word of an output array (a tally, or the bit pattern of a CCC value),
// taken as unsigned, and h(x) is the SplitMix64 finaliser (Steele, Lea and
// Flood, OOPSLA 2014) of (x + 1) * 0x9E3779B97F4A7C15.  The sum is linear, so
// the checksums of the phases or rank shards of a result, each with its global
// word offset `base`, add up (mod 2^128) to the checksum of the whole.
#include "ccc_dev.cuh"
#include "ccc_launch.h"

namespace ccc {
namespace {

__device__ __forceinline__ uint64_t word_hash(uint64_t x) {
  uint64_t z = (x + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// 128-bit accumulator (lo, hi) += h * w.
__device__ __forceinline__ void mac128(uint64_t &lo, uint64_t &hi, uint64_t h, uint32_t w) {
  const uint64_t plo = h * w;
  const uint64_t phi = __umul64hi(h, w);
  lo += plo;
  hi += phi + (lo < plo ? 1u : 0u);
}

__device__ __forceinline__ void add128(uint64_t &lo, uint64_t &hi, uint64_t blo, uint64_t bhi) {
  lo += blo;
  hi += bhi + (lo < blo ? 1u : 0u);
}

__global__ void __launch_bounds__(256) k_checksum(const uint32_t *__restrict__ words, int64_t count,
                                                  int64_t base, unsigned long long *out) {
  uint64_t lo = 0, hi = 0;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count;
       e += static_cast<int64_t>(gridDim.x) * blockDim.x)
    mac128(lo, hi, word_hash(static_cast<uint64_t>(base + e)), __ldg(words + e));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const uint64_t l2 = __shfl_xor_sync(0xffffffffu, lo, o);
    const uint64_t h2 = __shfl_xor_sync(0xffffffffu, hi, o);
    add128(lo, hi, l2, h2);
  }
  __shared__ uint64_t slo[8], shi[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    slo[warp] = lo;
    shi[warp] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t blo = 0, bhi = 0;
    for (int w = 0; w < (blockDim.x >> 5); ++w) add128(blo, bhi, slo[w], shi[w]);
    // out[0] += blo with the carry into out[1]: the old value tells whether the
    // 64-bit addition wrapped.
    const unsigned long long old = atomicAdd(out, static_cast<unsigned long long>(blo));
    const uint64_t carry = (old + blo < old) ? 1u : 0u;
    atomicAdd(out + 1, static_cast<unsigned long long>(bhi + carry));
  }
}

}  // namespace

int launch_checksum(const uint32_t *words, int64_t count, int64_t base, uint64_t *out,
                    cudaStream_t s) {
  if (cudaMemsetAsync(out, 0, 16, s) != cudaSuccess) return CCC_ECUDA;
  if (count <= 0) return CCC_OK;
  const int64_t blocks = (count + 255) / 256 < 152 * 8 ? (count + 255) / 256 : 152 * 8;
  k_checksum<<<static_cast<unsigned>(blocks), 256, 0, s>>>(
      words, count, base, reinterpret_cast<unsigned long long *>(out));
  return note_launch();
}

}  // namespace ccc
