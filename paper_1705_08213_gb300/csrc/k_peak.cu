// Rate probes for the roofline denominators, measured in SM clock cycles on
// the device so that a kernel's fraction of peak can be taken at the clock it
// ran at: the dense tcgen05 MMA rate of an operand kind on SM pairs, and the
// 64-bit AND + POPC rate of the CUDA cores that the popcount path uses.
//
// MMA probe: one cluster of two CTAs per SM pair, each CTA alone on its SM
// (its shared-memory request exceeds half of an SM's).  Both CTAs fill one
// 128-byte K stage of A (128 rows) and of B (n_cols / 2 <= 128 rows) with the value
// 1.0 of the kind, and for the block-scaled kinds 32 TMEM columns with the
// scale factor 1.0; the leader's thread issues n_mma MMAs (M = 256,
// N = n_cols) back to back into one accumulator, cycling through the four K
// steps of the stage, then commits and waits.  cycles[c] is the clock64
// difference seen by cluster c's issuing thread.  Every accumulator entry must
// equal n_mma * K (K = 32 for e4m3, 64 for e2m1): a check of the operand
// encoding, the instruction descriptor and the unit scale factors, whose
// failures are counted in *bad (a wait that gave up adds 2^20).
#include "ccc_dev.cuh"
#include "ccc_launch.h"
#include "tc_pipeline_pair.cuh"

namespace ccc {
namespace {

constexpr int PR_OP_BYTES = 128 * 128;
constexpr size_t PR_SMEM = 120 * 1024;
constexpr uint32_t PR_TMEM_COLS = 512;
constexpr uint32_t PR_SF_COL = 256;  // scale factors of A at 256, of B at 272
constexpr uint64_t PR_WAIT_NS = 2000000000ull;

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(128, 1)
    k_mma_rate(int kind, int n_cols, int n_mma, int64_t *cycles, int32_t *bad) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t *smem = smem_raw + ((1024u - (raw & 1023u)) & 1023u);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * PR_OP_BYTES);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
  const int warp = threadIdx.x >> 5;
  const uint32_t rank = tcp::cluster_rank();

  // 1.0 as e4m3 (0x38), or two e2m1 nibbles of 1.0 (0x2) per byte.
  const uint32_t one = kind == CCC_MMA_E4M3 ? 0x38383838u : 0x22222222u;
  uint4 *s4 = reinterpret_cast<uint4 *>(smem);
  for (int k = threadIdx.x; k < 2 * PR_OP_BYTES / 16; k += blockDim.x)
    s4[k] = make_uint4(one, one, one, one);
  fence_proxy_async_smem();
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(bar), 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    tcp::tmem_alloc_pair(smem_u32(tmem_slot), PR_TMEM_COLS);
    tcp::tmem_relinquish_pair();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_off = static_cast<uint32_t>(warp * 32) << 16;
  if (kind != CCC_MMA_E4M3) {
    // 1.0 as UE8M0 (0x7F) or UE4M3 (0x38) in every byte of the 32 columns.
    const uint32_t sf = kind == CCC_MMA_E2M1 ? 0x7F7F7F7Fu : 0x38383838u;
    uint32_t v[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = sf;
    tmem_st_32x32b_x32(tmem + lane_off + PR_SF_COL, v);
    tmem_st_wait();
  }
  tc_fence_before();
  __syncthreads();
  tcp::cluster_sync();
  tc_fence_after();

  if (threadIdx.x == 0) {
    if (rank == 0) {
      const uint32_t a0 = smem_u32(smem), b0 = smem_u32(smem + PR_OP_BYTES);
      const uint32_t sfa = tmem + PR_SF_COL, sfb = tmem + PR_SF_COL + 16;
      const uint32_t id = kind == CCC_MMA_E4M3 ? idesc_e4m3_f32(256, n_cols)
                                               : idesc_e2m1_f32(256, n_cols, kind == CCC_MMA_E2M1);
      const long long t0 = clock64();
      for (int n = 0; n < n_mma; ++n) {
        const uint32_t k = static_cast<uint32_t>(n & 3) * 32u;
        const uint64_t ad = smem_desc_sw128(a0 + k), bd = smem_desc_sw128(b0 + k);
        const uint32_t acc = n > 0 ? 1u : 0u;
        if (kind == CCC_MMA_E4M3)
          tcp::mma_f8f6f4_pair(tmem, ad, bd, id, acc);
        else if (kind == CCC_MMA_E2M1)
          tcp::mma_mxf4_pair(tmem, ad, bd, id, sfa, sfb, acc);
        else
          tcp::mma_mxf4nvf4_pair(tmem, ad, bd, id, sfa, sfb, acc);
      }
      tcp::mma_commit_pair(smem_u32(bar), 0x3);
      const bool ok = mbar_wait_timeout(smem_u32(bar), 0, PR_WAIT_NS);
      const long long t1 = clock64();
      cycles[blockIdx.x >> 1] = ok ? static_cast<int64_t>(t1 - t0) : -1;
      if (!ok) atomicAdd(bad, 1 << 20);
    } else if (!mbar_wait_timeout(smem_u32(bar), 0, PR_WAIT_NS)) {
      atomicAdd(bad, 1 << 20);
    }
  }
  __syncthreads();
  tc_fence_after();
  const float expect = static_cast<float>(n_mma) * (kind == CCC_MMA_E4M3 ? 32.f : 64.f);
  int wrong = 0;
  // 32 columns per load (inside the 512 allocated); only the n_cols written count.
  for (int c = 0; c < n_cols; c += 32) {
    uint32_t v[32];
    tmem_ld_32x32b_x32(tmem + lane_off + static_cast<uint32_t>(c), v);
    tmem_ld_wait();
#pragma unroll
    for (int k = 0; k < 32; ++k) wrong += (c + k < n_cols && __uint_as_float(v[k]) != expect) ? 1 : 0;
  }
  if (wrong) atomicAdd(bad, wrong);
  tc_fence_before();
  __syncthreads();
  tcp::cluster_sync();
  tc_fence_after();
  if (warp == 0) tcp::tmem_dealloc_pair(tmem, PR_TMEM_COLS);
}

// POPC probe: every thread keeps eight independent 64-bit AND + POPC chains
// over register operands (one 64-bit add per eight of them changes the second
// operand each iteration, so nothing can be hoisted).  cycles[b] = clock64
// difference of block b between two block-wide barriers.
__global__ void __launch_bounds__(1024, 1) k_popc_rate(int iters, int64_t *cycles, uint64_t *sink) {
  uint64_t a[8];
  uint32_t c[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint64_t z = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) * 8 + k + 1;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    a[k] = z ^ (z >> 31);
    c[k] = 0;
  }
  const uint64_t b = a[0] * 0x9E3779B97F4A7C15ull;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    const uint64_t y = b + static_cast<uint64_t>(it);
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] += static_cast<uint32_t>(__popcll(a[k] & y));
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = static_cast<int64_t>(t1 - t0);
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += c[k];
  if (s == 0x7FFFFFFFu) sink[0] = s;  // keeps the chains live; never true in practice
}

bool g_mma_smem_set[kMaxDevices] = {};

}  // namespace

int launch_mma_rate(int kind, int n_cols, int n_mma, int clusters, int64_t *cycles, int32_t *bad,
                    cudaStream_t s) {
  const int rc = set_smem_once(k_mma_rate, PR_SMEM, g_mma_smem_set);
  if (rc != CCC_OK) return rc;
  k_mma_rate<<<static_cast<unsigned>(2 * clusters), 128, PR_SMEM, s>>>(kind, n_cols, n_mma, cycles,
                                                                       bad);
  return note_launch();
}

int launch_popc_rate(int iters, int blocks, int64_t *cycles, uint64_t *sink, cudaStream_t s) {
  k_popc_rate<<<static_cast<unsigned>(blocks), 1024, 0, s>>>(iters, cycles, sink);
  return note_launch();
}

}  // namespace ccc
