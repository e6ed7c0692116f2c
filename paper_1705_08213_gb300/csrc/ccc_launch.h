// Internal host-side launch interface between the C ABI (ccc_api.cu) and the
// kernel translation units.  Every launcher returns CCC_OK or CCC_ECUDA.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ccc.h"

namespace ccc {

// Counts one kernel launch and converts a launch failure into CCC_ECUDA.
int note_launch();

// Launch set-up that the CUDA runtime keeps per device context (a kernel's
// dynamic shared-memory limit, its cluster occupancy) is cached per device:
// launchers index their caches with current_device(), which returns the
// current device, or -1 when it cannot be read or is not below kMaxDevices.
constexpr int kMaxDevices = 64;
inline int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
  return d;
}

// Sets the dynamic shared-memory limit of `kernel` on the current device once.
// Returns CCC_OK or CCC_ECUDA.
template <class K>
inline int set_smem_once(K kernel, size_t bytes, bool (&done)[kMaxDevices]) {
  const int d = current_device();
  if (d < 0) return CCC_ECUDA;
  if (done[d]) return CCC_OK;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           static_cast<int>(bytes)) != cudaSuccess)
    return CCC_ECUDA;
  done[d] = true;
  return CCC_OK;
}

// Argument checks of the C ABI (ccc_api.cu): a panel (pointer, sizes, stride,
// alignment, CCC_MAX_NF) and the options of a 2-way call.  CCC_OK or the code
// the entry point returns.
int check_panel(const ccc_panel *p);
int check_opts2(const ccc_opts *o);

// Tensor-core and POPC rate probes (k_peak.cu); see ccc_mma_rate / ccc_popc_rate.
int launch_mma_rate(int kind, int n_cols, int n_mma, int clusters, int64_t *cycles, int32_t *bad,
                    cudaStream_t s);
int launch_popc_rate(int iters, int blocks, int64_t *cycles, uint64_t *sink, cudaStream_t s);

int launch_allele_counts(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld,
                         int32_t *counts, float *w, double gamma, cudaStream_t s);
int launch_factors_from_counts(const int32_t *counts, int64_t n_v, float *w, double gamma,
                               cudaStream_t s);
// K-block-major operand rows, [K block][blocked_rows][128 bytes] (the K-split
// kernel reads them so; blocked_rows >= 2 snps_pad, snps_pad a multiple of 32):
// e4m3 (fp4 false, K blocks of 128 entries) or e2m1 (256 entries).  w != null:
// also the per-SNP factors of launch_allele_counts (w[n_v][2]), counted in the
// same pass over the codes.
int launch_unpack_blocked(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *op,
                          int64_t kpad, int64_t snps_pad, int64_t blocked_rows, bool fp4, float *w,
                          double gamma, cudaStream_t s);
// blocked_rows > 0: launch_unpack_blocked (e4m3); 0: row-major [2 snps_pad][kpad].
int launch_unpack_e4m3(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *op,
                       int64_t kpad, int64_t snps_pad, cudaStream_t s, int64_t blocked_rows = 0);
// The same with e2m1 (FP4) counts, two entries per byte: rows of kpad / 2
// bytes (kpad a multiple of 256); blocked: [kpad / 256][blocked_rows][128].
// w != null: also the per-SNP factors of launch_allele_counts (w[n_v][2],
// 1 - gamma f_i(a)) from the same read of the codes.
int launch_unpack_e2m1(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *op,
                       int64_t kpad, int64_t snps_pad, cudaStream_t s, int64_t blocked_rows = 0,
                       float *w = nullptr, double gamma = 0.0);
int launch_planes(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint64_t *planes,
                  int64_t w64, cudaStream_t s);

// Pairs (i, j), i < j < n_v, with i_begin <= i < i_end: the length of the
// output of a row range (a phase), the whole triangle for [0, n_v).
inline int64_t pairs_in_rows(int64_t n_v, int64_t i_begin, int64_t i_end) {
  if (i_begin < 0) i_begin = 0;
  if (i_end > n_v) i_end = n_v;
  if (i_end <= i_begin) return 0;
  return (i_end - i_begin) * (2 * n_v - i_begin - i_end - 1) / 2;
}

// The output length a launch passes to its kernels: len, or, in the checked
// build after ccc_checked_shrink_outputs(n), len - n (so that the last n
// stores of a call must be caught by the index checks).
int64_t checked_out_len(int64_t len);

// Shared description of a 2-way tally launch.
struct Tally2Args {
  int64_t n_v;
  int64_t n_f;
  const float *w;   // [n_v][2] per-SNP factors 1 - gamma f_i(a) (PERSNP), or null
  int32_t *tally;   // [npairs][4]
  float *ccc;       // [npairs][4] or null (tallies only)
  int32_t *status;  // workspace status word
  float gamma;
  int32_t norm;
  // Thresholded output: when hits is set, nothing is written to tally / ccc;
  // pairs whose largest CCC value exceeds threshold are appended to hits.
  ccc_hit *hits = nullptr;
  unsigned long long *n_hits = nullptr;
  int64_t cap = 0;
  float threshold = 0.f;
  // Column blocks per L2 group of the tensor-core tile order (0 = default 8).
  int32_t group = 0;
  // Row range of a phase: only pairs with i_begin <= i < i_end are computed and
  // pair (i, j) is stored at index pair_index(i, j) - pair0.
  int64_t i_begin = 0;
  int64_t i_end = int64_t(1) << 62;
  int64_t pair0 = 0;
  // Pairs the tally / ccc arrays hold (checked builds test every store index).
  int64_t out_len = int64_t(1) << 62;
};

// Panels per batched tensor-core launch (kernel parameter space).
constexpr int kMaxBatchPanels = 64;

// One persistent tensor-core launch over all tiles of n <= kMaxBatchPanels
// panels, in the given order; ops[k] is panel k's operand matrix.
int launch_tally2_tc_batched(const Tally2Args *args, const uint8_t *const *ops,
                             const int64_t *rows_pad, const int64_t *kpad, int n, int group,
                             int num_sms, cudaStream_t s);
// The same on SM pairs (256 x 256 tiles, cta_group::2).  split[k] > 1 (or
// null: all 1): panel k's tiles run as that many K parts whose partial tallies
// are added into args[k].tally, which must then be zero and gets no CCC values
// (the caller forms them from the summed tallies).  fp4: e2m1 operand rows of
// kpad[k] / 2 bytes (kpad[k] a multiple of 256).
int launch_tally2_tc_pair_batched(const Tally2Args *args, const uint8_t *const *ops,
                                  const int64_t *rows_pad, const int64_t *kpad, const int *split,
                                  int n, int group, int num_sms, cudaStream_t s, bool fp4 = false);

// Square 128-SNP tiles of the triangle (J >= I) in row blocks [I0, I1).
int64_t tc2_pair_tiles(int64_t n_v, int64_t I0, int64_t I1);
// 256 x 256 tiles on SM pairs (cta_group::2); same arguments as launch_tally2_tc.
// fp4: op holds e2m1 rows of kpad / 2 bytes (launch_unpack_e2m1, kpad a
// multiple of 256) and the tiles run on the block-scaled FP4 MMA.
int launch_tally2_tc_pair(const Tally2Args &a, const uint8_t *op, int64_t rows_pad, int64_t kpad,
                          int num_sms, cudaStream_t s, bool fp4 = false);
// The same with the K dimension split into `split` parts (1 <= split <= the
// 128-byte K stages of a row) whose partial tallies are added into a.tally
// with integer reductions (a.tally must be zero; no CCC values, no thresholded
// output).  The operand is K-block-major (launch_unpack_* with blocked_rows).
int launch_tally2_tc_pair_split(const Tally2Args &a, const uint8_t *op, int64_t rows_pad,
                                int64_t kpad, int split, int num_sms, cudaStream_t s,
                                bool fp4 = false);
// The two launches above with the operand preparation fused in: the kernel
// reads the packed panel geno (row stride ld words, even; 16-byte aligned)
// and expands the codes into count rows in shared memory.
int launch_tally2_tc_pair_packed(const Tally2Args &a, const uint64_t *geno, int64_t ld,
                                 int num_sms, cudaStream_t s);
int launch_tally2_tc_pair_split_packed(const Tally2Args &a, const uint64_t *geno, int64_t ld,
                                       int split, int num_sms, cudaStream_t s);
// Tensor-core 2-way tallies over the e4m3 operand matrix op[rows_pad][kpad].
int launch_tally2_tc(const Tally2Args &a, const uint8_t *op, int64_t rows_pad, int64_t kpad,
                     int num_sms, cudaStream_t s);
// Popcount 2-way tallies over planes[n_v][w64][4].
// split > 1: the 64-entry words in that many parts whose partial tallies are
// added into a.tally, which must be zero (no CCC values, no thresholded output).
int launch_tally2_popc(const Tally2Args &a, const uint64_t *planes, int64_t w64, cudaStream_t s,
                       int split = 1);
// 64 x 64-SNP tiles of the popcount kernel over the whole triangle.
int64_t popc2_tiles(int64_t n_v);
// CCC values from stored tallies.
int launch_metric2(const int32_t *tally, const float *w, int64_t n_v, float gamma, int32_t norm,
                   float *ccc, cudaStream_t s);

// Shared description of a 3-way slab launch (slabs j in [j_begin, j_end)).
struct Tally3Args {
  int64_t n_v;
  int64_t n_f;
  int64_t j_begin, j_end;
  const float *w;
  int32_t *tally;  // [S(j_end) - S(j_begin)][8]
  float *ccc;      // same, or null
  int32_t *status;
  float gamma;
  int32_t norm;
  // Triples the tally / ccc arrays hold (checked builds test every store index).
  int64_t out_len = int64_t(1) << 62;
};

// Masked 3-way operands L_j for the slabs [j0, j1) into lop (rows as tc3_lop_rows).
int launch_mask3(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *lop,
                 int64_t kpad, int64_t j0, int64_t j1, cudaStream_t s);
// L rows of the slabs [j0, j1) (each slab padded to 32 SNPs i, 4 rows per SNP).
int64_t tc3_lop_rows(int64_t j0, int64_t j1);
int64_t tc3_num_tiles(int64_t j0, int64_t j1, int64_t n_v);
// Tensor-core 3-way tallies of the slabs [j0, j1) (inside [a.j_begin, a.j_end)).
int launch_tally3_tc(const Tally3Args &a, const uint8_t *op, int64_t rows_pad, int64_t kpad,
                     uint8_t *lop, int64_t lop_rows, int64_t j0, int64_t j1, int num_sms,
                     cudaStream_t s);
// Tensor-core 3-way tallies with the masked operand formed inside the kernel
// from the packed panel (all slabs [a.j_begin, a.j_end) in one launch).
int launch_tally3_fused(const Tally3Args &a, const uint64_t *geno, int64_t ld, const uint8_t *op,
                        int64_t rows_pad, int64_t kpad, int num_sms, cudaStream_t s);
// 3-way tallies by genotype classes of v_j (k_tc3c.cu), per batch of slabs
// [j0, j1):
//   launch_compact3  missing[j - j0] = individuals with v_j missing and, when
//                    at most tc3_class_cap(), the count rows of every SNP
//                    restricted to them (cbuf, tc3_class_cbuf_rows(j1 - j0, n_v)
//                    rows of tc3_class_cap() bytes);
//   launch_mask3c    the masked rows of the batch (tc3_class_mask_rows(j0, j1,
//                    n_v) rows of kpad bytes) into op from row mrow0 on, op's
//                    first rows being the count matrix R;
//   launch_tally3_class  the tallies, with the 2-way tallies rtab ([pair][4],
//                    pairs i < k with i < j1 - 1).
int64_t tc3_class_cap();
int64_t tc3_class_cbuf_rows(int64_t n_slabs, int64_t n_v);
int64_t tc3_class_mask_rows(int64_t j0, int64_t j1, int64_t n_v);
// fp4: e2m1 nibbles; compacted rows of tc3_class_cap() / 2 bytes, masked rows
// (and R) of kpad / 2 bytes.
int launch_compact3(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *cbuf,
                    int32_t *missing, int64_t j0, int64_t j1, cudaStream_t s, bool fp4 = false);
int launch_mask3c(const uint64_t *geno, int64_t n_f, int64_t n_v, int64_t ld, uint8_t *op,
                  int64_t kpad, int64_t mrow0, const int32_t *missing, int64_t j0, int64_t j1,
                  cudaStream_t s, bool fp4 = false);
//                    dscratch (tc3_class_dscratch_bytes()) holds the D counts
//                    of the tiles in flight when n_f <= 16383.
int64_t tc3_class_dscratch_bytes();
//                    fp4: e2m1 operands (the wide tiles only, n_f <= 16383;
//                    else CCC_EUNSUPPORTED).
int launch_tally3_class(const Tally3Args &a, const uint8_t *op, int64_t op_rows, int64_t mrow0,
                        int64_t kpad, const int32_t *rtab, const uint8_t *cbuf,
                        const int32_t *missing, uint32_t *dscratch, int64_t j0, int64_t j1,
                        int num_sms, cudaStream_t s, bool fp4 = false);
int launch_tally3_popc(const Tally3Args &a, const uint64_t *planes, int64_t w64, cudaStream_t s);
int launch_metric3(const int32_t *tally, const float *w, int64_t n_v, int64_t j_begin,
                   int64_t j_end, float gamma, int32_t norm, float *ccc, cudaStream_t s);

// Markers with s allele states (k_multi.cu, k_multi_wide.cu).  Operand rows:
// multi_rows_pad(n_v, s) rows of kpad bytes (32 rows per floor(32 / s) SNPs).
int64_t multi_rows_pad(int64_t n_v, int s);
// counts [n_v][s + 1] (s_i^a, then n_i) and/or PERSNP factors w [n_v][s]; either may be null.
int launch_multi_counts(const uint8_t *geno, int64_t n_f, int64_t n_v, int64_t ld, int s,
                        int32_t *counts, float *w, double gamma, cudaStream_t st);
int launch_multi_factors(const int32_t *counts, int64_t n_v, int s, float *w, double gamma,
                         cudaStream_t st);
// fp4: e2m1 rows of kpad / 2 bytes (kpad a multiple of 256).
int launch_multi_unpack(const uint8_t *geno, int64_t n_f, int64_t n_v, int64_t ld, int s,
                        uint8_t *op, int64_t kpad, int64_t rows_pad, cudaStream_t st,
                        bool fp4 = false);
// Tallies and, when out_ccc is set, CCC values of the pairs with
// i_begin <= i < i_end (s*s each), pair (i, j) at pair_index(i, j) - pair0.
// split > 1 (whole triangle only): the K stages in `split` parts whose partial
// tallies are added into the zeroed tally array, no CCC values.
// fp4 (s <= 8, split 1): op holds e2m1 rows (launch_multi_unpack with fp4) and
// the tiles are 256 x 192 on the block-scaled FP4 MMA.
int launch_tally2_multi(int s, int64_t n_v, const float *w, int32_t *tally, float *out_ccc,
                        int32_t *status, float gamma, int32_t norm, int32_t group, const uint8_t *op,
                        int64_t rows_pad, int64_t kpad, int num_sms, cudaStream_t st,
                        int64_t i_begin, int64_t i_end, int64_t pair0, int split = 1,
                        bool fp4 = false);
int launch_tally2_multi_wide(int s, int64_t n_v, const float *w, int32_t *tally, float *out_ccc,
                             int32_t *status, float gamma, int32_t norm, int32_t group,
                             const uint8_t *op, int64_t rows_pad, int64_t kpad, int num_sms,
                             cudaStream_t st, int64_t i_begin, int64_t i_end, int64_t pair0,
                             int split);
int launch_metric2_multi(const int32_t *tally, const float *w, int64_t n_v, int s, float gamma,
                         int32_t norm, float *out_ccc, cudaStream_t st);

// Exact 128-bit checksum of `count` 32-bit words with global offset `base` into out[2].
int launch_checksum(const uint32_t *words, int64_t count, int64_t base, uint64_t *out,
                    cudaStream_t s);

// Bounded-wait self-test (k_selftest.cu): one CTA whose mbarrier wait cannot complete.
int launch_wait_selftest(int32_t *status, uint64_t limit_ns, cudaStream_t s);

// Host index helpers (also exported through the C ABI).
int64_t pair_index(int64_t i, int64_t j, int64_t n_v);
int64_t slab_offset(int64_t j, int64_t n_v);

}  // namespace ccc
