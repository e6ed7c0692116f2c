// CCC values from exact integer tallies, single precision (Eqs. 3-4).
//
// Error budget (u = 2^-24, every operation correctly rounded, no contraction):
//   f = r / n                                   1 rounding
//   PERSNP factor w = 1 - gamma f_i(a)          1 rounding (computed in fp64 once per SNP)
//   JOINT  factor w = (n - gamma R) / n         gamma's own rounding (amplified at most 2x,
//                                               i.e. <= u) + fma + division = 3u
//   products f * w_i * w_j (* w_k)              2 (3) roundings
//   PERSNP evaluates (r * (1/n)) * w_i * w_j (2-way) and
//   ((r * (1/n)) * (w_i w_j)) * w_k (3-way): 1/n and r * (1/n) are 2 roundings.
// Worst case: 2-way 6u (PERSNP) / 9u (JOINT); 3-way 8u / 13u = 7.8e-7 < 1e-6.
// There is no cancellation: every factor is at least 1 - gamma >= 1/3 for gamma <= 2/3.
#pragma once

#include <stdint.h>

namespace ccc {

__device__ __forceinline__ float joint_factor(int32_t marginal, float n, float gamma) {
  return __fdiv_rn(__fmaf_rn(-gamma, static_cast<float>(marginal), n), n);
}

// r = (r00, r01, r10, r11); wi, wj = per-SNP factors (PERSNP) for alleles 0 and 1.
__device__ __forceinline__ float4 ccc2_values(int32_t r00, int32_t r01, int32_t r10, int32_t r11,
                                              float wi0, float wi1, float wj0, float wj1,
                                              int32_t norm, float gamma) {
  const int32_t n4 = r00 + r01 + r10 + r11;  // 4 n_ij
  if (n4 == 0) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float d = static_cast<float>(n4);
  if (norm == CCC_NORM_JOINT) {
    wi0 = joint_factor(r00 + r01, d, gamma);
    wi1 = joint_factor(r10 + r11, d, gamma);
    wj0 = joint_factor(r00 + r10, d, gamma);
    wj1 = joint_factor(r01 + r11, d, gamma);
  }
  float4 c;
  if (norm != CCC_NORM_JOINT) {
    const float inv = __frcp_rn(d);
    c.x = __fmul_rn(__fmul_rn(__fmul_rn(static_cast<float>(r00), inv), wi0), wj0);
    c.y = __fmul_rn(__fmul_rn(__fmul_rn(static_cast<float>(r01), inv), wi0), wj1);
    c.z = __fmul_rn(__fmul_rn(__fmul_rn(static_cast<float>(r10), inv), wi1), wj0);
    c.w = __fmul_rn(__fmul_rn(__fmul_rn(static_cast<float>(r11), inv), wi1), wj1);
    return c;
  }
  c.x = __fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(r00), d), wi0), wj0);
  c.y = __fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(r01), d), wi0), wj1);
  c.z = __fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(r10), d), wi1), wj0);
  c.w = __fmul_rn(__fmul_rn(__fdiv_rn(static_cast<float>(r11), d), wi1), wj1);
  return c;
}

// 3-way PERSNP value from the tally r, 1/n (rounded), w_i w_j (rounded) and w_k.
__device__ __forceinline__ float ccc3_persnp(int32_t r, float inv_n, float wij, float wk) {
  return __fmul_rn(__fmul_rn(__fmul_rn(static_cast<float>(r), inv_n), wij), wk);
}

// r[abc] with a most significant; wi/wj/wk per-SNP factors (PERSNP).
__device__ __forceinline__ void ccc3_values(const int32_t (&r)[8], float wi0, float wi1,
                                            float wj0, float wj1, float wk0, float wk1,
                                            int32_t norm, float gamma, float (&out)[8]) {
  int32_t n8 = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) n8 += r[t];  // 8 n_ijk
  if (n8 == 0) {
#pragma unroll
    for (int t = 0; t < 8; ++t) out[t] = 0.f;
    return;
  }
  const float d = static_cast<float>(n8);
  if (norm == CCC_NORM_JOINT) {
    wi0 = joint_factor(r[0] + r[1] + r[2] + r[3], d, gamma);
    wi1 = joint_factor(r[4] + r[5] + r[6] + r[7], d, gamma);
    wj0 = joint_factor(r[0] + r[1] + r[4] + r[5], d, gamma);
    wj1 = joint_factor(r[2] + r[3] + r[6] + r[7], d, gamma);
    wk0 = joint_factor(r[0] + r[2] + r[4] + r[6], d, gamma);
    wk1 = joint_factor(r[1] + r[3] + r[5] + r[7], d, gamma);
  }
  const float wi[2] = {wi0, wi1}, wj[2] = {wj0, wj1}, wk[2] = {wk0, wk1};
  if (norm != CCC_NORM_JOINT) {
    const float inv = __frcp_rn(d);
#pragma unroll
    for (int t = 0; t < 8; ++t)
      out[t] = ccc3_persnp(r[t], inv, __fmul_rn(wi[t >> 2], wj[(t >> 1) & 1]), wk[t & 1]);
    return;
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const float f = __fdiv_rn(static_cast<float>(r[t]), d);
    out[t] = __fmul_rn(__fmul_rn(__fmul_rn(f, wi[t >> 2]), wj[(t >> 1) & 1]), wk[t & 1]);
  }
}

// PERSNP thresholding without division: false only when every CCC value of the
// pair is certainly at most the threshold, i.e. max_ab r_ab w_i(a) w_j(b) is
// below threshold * n by more than 2^-18 relative (the exact values carry at
// most 6u + 3u of rounding here, u = 2^-24).
__device__ __forceinline__ bool may_exceed(int32_t r00, int32_t r01, int32_t r10, int32_t r11,
                                           float wi0, float wi1, float wj0, float wj1, float threshold) {
  const int32_t n4 = r00 + r01 + r10 + r11;
  if (n4 == 0) return threshold < 0.f;
  const float m = fmaxf(fmaxf(static_cast<float>(r00) * wi0 * wj0, static_cast<float>(r01) * wi0 * wj1),
                        fmaxf(static_cast<float>(r10) * wi1 * wj0, static_cast<float>(r11) * wi1 * wj1));
  return m * (1.f + 0x1p-18f) >= threshold * static_cast<float>(n4);
}

// Append pair (i, j) to the hit list when its largest CCC value exceeds the threshold.
__device__ __forceinline__ void filter_pair(ccc_hit *hits, unsigned long long *n_hits, int64_t cap,
                                            float threshold, int64_t i, int64_t j, int32_t r00,
                                            int32_t r01, int32_t r10, int32_t r11, float4 c) {
  const float mx = fmaxf(fmaxf(c.x, c.y), fmaxf(c.z, c.w));
  if (!(mx > threshold)) return;
  const unsigned long long slot = atomicAdd(n_hits, 1ull);
  if (static_cast<int64_t>(slot) >= cap) return;
  ccc_hit h;
  h.i = static_cast<int32_t>(i);
  h.j = static_cast<int32_t>(j);
  h.tally[0] = r00;
  h.tally[1] = r01;
  h.tally[2] = r10;
  h.tally[3] = r11;
  h.ccc[0] = c.x;
  h.ccc[1] = c.y;
  h.ccc[2] = c.z;
  h.ccc[3] = c.w;
  hits[slot] = h;
}

__device__ __forceinline__ int64_t dev_pair_index(int64_t i, int64_t j, int64_t n_v) {
  return i * (2 * n_v - i - 1) / 2 + (j - i - 1);
}

// Triples in slabs 0 .. j-1: S(j) = sum_{j' < j} j' (n_v - 1 - j').
__host__ __device__ __forceinline__ int64_t slab_offset_dev(int64_t j, int64_t n_v) {
  const int64_t s1 = (j - 1) * j / 2;
  const int64_t s2 = (j - 1) * j * (2 * j - 1) / 6;
  return s1 * (n_v - 1) - s2;
}

}  // namespace ccc
