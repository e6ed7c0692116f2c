/*
 * ccc.h -- C ABI of libccc, the GB300 (sm_103a) hot path for 2-way and 3-way
 * Custom Correlation Coefficient (CCC) calculations.
 *
 * Method: Joubert, Nance, Climer, Weighill, Jacobson, "Parallel Accelerated
 * Custom Correlation Coefficient Calculations for Genomics Applications",
 * Parallel Computing (2018).  Section, equation and table numbers below refer
 * to that paper.
 *
 * ---------------------------------------------------------------------------
 * Input: the packed genotype panel (Sec. 2.1 vector model; Sec. 3.1 packing;
 * Sec. 7 item 1 missing-value marker)
 *
 *   Every entry v_{i,q} of SNP vector i (0 <= i < n_v) for individual q
 *   (0 <= q < n_f) is a pair of allele bits ((v)_1, (v)_2), stored as the
 *   2-bit code 2*(v)_1 + (v)_2:
 *       0b00 = (0,0)  homozygous, genotype 0
 *       0b01 = (0,1)  heterozygous (always stored this way round)
 *       0b11 = (1,1)  homozygous, genotype 2
 *       0b10 = (1,0)  MISSING (the pair the paper reserves as the marker)
 *   SNP i occupies the uint64 words geno[i*ld .. i*ld + ceil(n_f/32) - 1];
 *   entry q sits at bits 2*(q%32)..2*(q%32)+1 of word q/32 (LSB first).
 *   Bits past n_f in the last word and words past ceil(n_f/32) are ignored.
 *   Requirements: n_f >= 1, n_v >= 1, ld >= ceil(n_f/32), ld even (16-byte
 *   rows), geno 16-byte aligned, all device memory.
 *
 * Output indexing
 *   2-way: pairs i < j only, row-major upper triangle without the diagonal,
 *          p = i*(2*n_v - i - 1)/2 + (j - i - 1)      (ccc2_index)
 *          4 values per pair in the order (a,b) = 00, 01, 10, 11, where a is
 *          the allele of SNP i (the lower index) and b that of SNP j.
 *   3-way: triples i < j < k only, slab-major: slab j, then i, then k,
 *          t = S(j) + i*(n_v - 1 - j) + (k - j - 1),
 *          S(j) = sum_{j' < j} j' (n_v - 1 - j')        (ccc3_index)
 *          8 values per triple in the order abc = 000 .. 111 (a for i, b for
 *          j, c for k).  A call over slabs [j_begin, j_end) writes entries
 *          t - S(j_begin).
 *
 * Definitions computed (with rho_{i,q}(a) = number of alleles equal to a in
 * v_{i,q}, 0 for a missing entry):
 *   tally   r_{ij}^{ab}  = sum_q rho_{i,q}(a) rho_{j,q}(b)                 (Eq. 2 numerator)
 *           r_{ijk}^{abc} = sum_q rho_{i,q}(a) rho_{j,q}(b) rho_{k,q}(c)    (Eq. 5 numerator)
 *   counts  s_i^a = sum_q rho_{i,q}(a), n_i = number of non-missing entries (Eq. 1)
 *   CCC     f_ij(a,b) (1 - gamma f_i(a)) (1 - gamma f_j(b))                (Eq. 3)
 *           f_ijk(a,b,c) (1 - gamma f_i(a)) (1 - gamma f_j(b)) (1 - gamma f_k(c))  (Eq. 4)
 *     with f_ij = r/(4 n_ij), f_ijk = r/(8 n_ijk) where n_ij (n_ijk) counts the
 *     jointly non-missing entries, and f_i(a) = s_i^a/(2 n_i) (CCC_NORM_PERSNP)
 *     or the pair's (triple's) own marginal (CCC_NORM_JOINT).  When nothing is
 *     missing both reduce to Eqs. 1-5 as printed.  n_ij = 0 (n_ijk = 0) gives
 *     zero tallies and zero CCC values; n_i = 0 gives f_i = 0.
 *   Tallies are exact 32-bit integers.  CCC values are single precision; the
 *   relative error against exact arithmetic is below 1e-6.
 *
 * Conventions for every entry point
 *   - All buffers are caller-owned device memory unless stated otherwise; the
 *     library allocates nothing.  Scratch space is the caller's workspace,
 *     sized by ccc_workspace_size() and passed in ccc_opts.  Output arrays
 *     (tallies, CCC values, hits) may also be pinned host memory that the
 *     device can address (cudaHostAlloc / cudaHostRegister with unified
 *     addressing): the kernels then store the results over the host link.
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 *     as void*; NULL is the legacy default stream).  They return once the work
 *     is queued.
 *   - Return value: CCC_OK, or a negative CCC_E* code for an argument error
 *     found before anything was queued (nothing is written then), or
 *     CCC_ECUDA when a launch was refused.  Errors found on the device (a
 *     bounded wait that timed out; in the bounds-checking build, an index
 *     outside its buffer) are recorded in the workspace status word, read
 *     with ccc_status().
 * ---------------------------------------------------------------------------
 */
#ifndef CCC_H_
#define CCC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CCC_OK 0
#define CCC_EINVAL (-1)       /* bad pointer, size, stride, alignment or option */
#define CCC_ERANGE (-2)       /* a size beyond what the exact arithmetic allows */
#define CCC_EUNSUPPORTED (-3) /* no usable sm_103a device, or path not available */
#define CCC_ECUDA (-4)        /* a CUDA call failed */
#define CCC_ETIMEOUT (-5)     /* a device-side bounded wait gave up (ccc_status) */
#define CCC_ENOSPACE (-6)     /* workspace smaller than ccc_workspace_size() */
#define CCC_EBOUNDS (-7)      /* a library built with CCC_BOUNDS_CHECK found an index outside its
                                 buffer on the device and skipped the access (ccc_status) */

/* Tally paths. */
#define CCC_PATH_TC 0   /* tcgen05 tensor cores, e4m3 or e2m1 count operands, FP32 accumulate */
#define CCC_PATH_POPC 1 /* bit planes, AND + population count on the CUDA cores */

/* Normalisation of f_i with missing data (see above). */
#define CCC_NORM_PERSNP 0
#define CCC_NORM_JOINT 1

/* Largest n_f accepted: every tally is an integer below 8 n_f and must stay
 * exactly representable in the FP32 accumulators (< 2^24). */
#define CCC_MAX_NF 2097151

typedef struct ccc_panel {
  const uint64_t *geno; /* device pointer to n_v rows of ld uint64 words */
  int64_t n_f;          /* individuals (entries per SNP vector) */
  int64_t n_v;          /* SNP vectors */
  int64_t ld;           /* row stride in uint64 words */
} ccc_panel;

typedef struct ccc_opts {
  int32_t path;           /* CCC_PATH_TC or CCC_PATH_POPC */
  int32_t norm;           /* CCC_NORM_PERSNP or CCC_NORM_JOINT */
  double gamma;           /* the constant of Eqs. 3-4; the paper fixes 2/3 */
  void *workspace;        /* device scratch, 256-byte aligned */
  size_t workspace_bytes; /* its size; must be >= ccc_workspace_size() */
  int32_t group;          /* tensor-core tile order: column blocks per L2 group; 0 = 8 */
  int32_t order;          /* ccc2_batched panel order: 0 = most tile work first, 1 = as given */
  int32_t tile;           /* tensor-core variant.  2-way: 1 = 128 x 256 tiles on one SM,
                             2 = 256 x 256 tiles on a pair of SMs (cta_group::2), 3 = as 2 with
                             the 2-bit codes expanded into count rows in shared memory inside the
                             tally kernel (the unpack of Sec. 3.1 fused; no operand matrix in the
                             workspace, for panels whose 2-bytes-per-entry operands would not fit;
                             slower on GB300); automatic = 2.  ccc2_batched rejects 3.
                             3-way: 1 = masked operands L_j formed in HBM by a separate pass,
                             2 = L_j formed in shared memory inside the tally kernel (repeated
                             for every k-block, slower), 3 = genotype classes of v_j on SM
                             pairs: r^{abc} from the 2-way tallies r_ik, a sign-masked product
                             over all individuals and a product over those with v_j missing
                             (half the tensor work of 1 and 2); automatic = 3.  0 = automatic.
                             The workspace size depends on it. */
  int32_t split;          /* 2-way calls over the whole triangle (tensor cores, biallelic and
                             s-state, and the biallelic popcount path; outputs in device memory):
                             K (individuals) split into this many parts whose partial tallies
                             are summed (the n_pf axis of Sec. 4 on one GPU), for panels with few
                             SNP tiles and long vectors.  0 = automatic (tensor cores: when the
                             triangle has at most half as many tiles as SM pairs and at least 32
                             128-byte K stages, n_f >= 4,096 with e4m3 and 8,192 with e2m1
                             operands; popcount: fewer 64-SNP tiles than four per SM, at least
                             4,096 individuals per part), 1 = off, n >= 2 = n parts (at most one
                             per K stage: n_f / 128 with e4m3, n_f / 256 with e2m1 operands,
                             n_f / 512 on the popcount path).  Same results;
                             the CCC values then come from the summed tallies. */
  int32_t operand;        /* encoding of the tensor-core count operands (CCC_OPERAND_*):
                             E4M3 = one byte per count, kind::f8f6f4 MMAs; E2M1 = FP4, two counts
                             per byte, block-scaled kind::mxf4 MMAs with every scale factor 1.0
                             (half the operand bytes, a higher MMA rate).  Counts 0, 1, 2 are
                             exact in both and the FP32 accumulation is exact below 2^24, so
                             both give the same tallies and CCC values bit for bit.  E2M1 is
                             built for the 2-way SM-pair tiles (opts->tile 0 or 2, with K split,
                             row ranges, ccc2_stream, ccc2_filter and ccc2_batched) and for the
                             3-way genotype-class route (opts->tile 0 or 3, n_f <= 16,383) and
                             for markers with s <= 8 states (ccc2_multi_*, without K split);
                             elsewhere an explicit E2M1 returns CCC_EUNSUPPORTED.  AUTO (0) =
                             E2M1 where it is built, else E4M3.  The workspace size depends on
                             it (for markers it is that of E4M3 rows, which are never smaller). */
  int32_t solo;           /* ccc2_batched on SM pairs: a panel with at least this many 256 x 256
                             tiles runs as its own launch, the others share one persistent
                             launch; 0 = 1024, < 0 = none (every panel in the shared launch). */
} ccc_opts;

/* Operand encodings (ccc_opts.operand). */
#define CCC_OPERAND_AUTO 0
#define CCC_OPERAND_E4M3 1
#define CCC_OPERAND_E2M1 2

/* Operations, for ccc_workspace_size(). */
#define CCC_OP_METRIC 1 /* ccc2_metric / ccc3_metric: status word and per-SNP factors */
#define CCC_OP_2WAY 2
#define CCC_OP_3WAY 3

/* Fill *opts with the defaults: path TC, norm PERSNP, gamma 2/3, no workspace,
 * automatic schedule (group 0, order 0). */
void ccc_opts_default(ccc_opts *opts);

/*
 * Bytes of workspace that the 2-way (op = CCC_OP_2WAY), 3-way
 * (op = CCC_OP_3WAY) or metric-only (op = CCC_OP_METRIC) calls need for this
 * panel and path.  Host only; touches no device memory.  Returns CCC_OK,
 * CCC_EINVAL or CCC_ERANGE.
 */
int ccc_workspace_size(const ccc_panel *panel, const ccc_opts *opts, int op, size_t *bytes);

/*
 * Per-SNP allele sums and non-missing counts (Eq. 1 numerators; Sec. 2.1):
 * counts[3*i + 0] = s_i^0, counts[3*i + 1] = s_i^1, counts[3*i + 2] = n_i.
 * counts: device int32[n_v][3].  Needs no workspace.
 */
int ccc_allele_counts(const ccc_panel *panel, int32_t *counts, void *stream);

/*
 * 2-way tallies of all pairs i < j (Eq. 2 numerators; Sec. 3.1 maps them to a
 * GEMM-shaped product B = V^T o_2 V whose entries are 2x2 tally tables).
 * tally: device int32[n_v (n_v - 1) / 2][4].
 */
int ccc2_tally(const ccc_panel *panel, int32_t *tally, const ccc_opts *opts, void *stream);

/*
 * 2-way CCC values (Eq. 3) from tallies produced by ccc2_tally and counts from
 * ccc_allele_counts.  tally: device int32[npairs][4]; counts: device
 * int32[n_v][3]; ccc: device float[npairs][4].  Uses opts->norm, opts->gamma
 * and a workspace of ccc_workspace_size(.., CCC_OP_METRIC, ..) bytes (the
 * per-SNP factors 1 - gamma f_i(a) are formed there once).
 */
int ccc2_metric(const int32_t *tally, const int32_t *counts, int64_t n_v, const ccc_opts *opts,
                float *ccc, void *stream);

/*
 * Fused 2-way: allele counts, tallies and CCC values in one pass (Eqs. 1-3),
 * the CCC computed in the tally kernel's epilogue.  tally: device
 * int32[npairs][4]; ccc: device float[npairs][4].  Needs the workspace.
 */
int ccc2_tally_metric(const ccc_panel *panel, int32_t *tally, float *ccc, const ccc_opts *opts,
                      void *stream);

/* One pair kept by ccc2_filter. */
typedef struct ccc_hit {
  int32_t i, j;      /* the pair, i < j */
  int32_t tally[4];  /* r^{00}, r^{01}, r^{10}, r^{11} */
  float ccc[4];      /* CCC(0,0), CCC(0,1), CCC(1,0), CCC(1,1) */
} ccc_hit;

/*
 * 2-way with thresholded output (Sec. 7 item 6: in practice only the few
 * values above a threshold are wanted).  Computes the tallies and CCC values
 * of every pair i < j exactly as ccc2_tally_metric does, but stores only the
 * pairs whose largest CCC value exceeds `threshold`: they are appended in no
 * particular order to hits[0 .. min(total, cap)), and *n_hits (a device
 * int64 owned by the caller, cleared by the call) receives the total number
 * of such pairs, which may exceed cap (then only cap of them were stored).
 * Needs the CCC_OP_2WAY workspace.  Either path.  threshold must be finite.
 */
int ccc2_filter(const ccc_panel *panel, float threshold, ccc_hit *hits, int64_t cap,
                int64_t *n_hits, const ccc_opts *opts, void *stream);

/*
 * 2-way over a row range -- one "phase" in the sense of Sec. 7 item 3, where a
 * run computes and stores only part of the results when all of them do not fit
 * in memory at once: the pairs (i, j) with i_begin <= i < i_end and every
 * j > i, with tallies and CCC values as ccc2_tally_metric computes them,
 * stored at index ccc2_index(i, j, n_v) - ccc2_index(i_begin, i_begin + 1, n_v)
 * (these rows are contiguous in the upper-triangle order).  tally, ccc:
 * device [ccc2_rows_count(n_v, i_begin, i_end)][4].  Workspace: CCC_OP_2WAY.
 * 0 <= i_begin <= i_end <= n_v.  Row ranges that start on a multiple of 128
 * (64 with opts->tile = 1) waste no tensor-core work.
 */
int ccc2_tally_metric_rows(const ccc_panel *panel, int64_t i_begin, int64_t i_end,
                           int32_t *tally, float *ccc, const ccc_opts *opts, void *stream);

/* Pairs of the rows [i_begin, i_end): sum of (n_v - 1 - i); -1 if out of range. */
int64_t ccc2_rows_count(int64_t n_v, int64_t i_begin, int64_t i_end);

/*
 * Host helper: split the rows [0, n_v) into n_phases contiguous ranges,
 * bounds[0] = 0 < ... <= bounds[n_phases] = n_v, with inner bounds on
 * multiples of 64 and about equal pair counts.  bounds: host int64[n_phases + 1].
 */
int ccc2_phase_bounds(int64_t n_v, int n_phases, int64_t *bounds);

/*
 * Phased 2-way output to host memory.  Computes all pairs as
 * ccc2_tally_metric does, phase by phase (ccc2_phase_bounds), into two
 * staging buffers in the workspace, and copies each finished phase to the
 * caller's host arrays while the next phase computes, so that device-to-host
 * copies overlap the tensor-core work.  host_tally, host_ccc: host memory
 * [npairs][4] (pinned, or the copies do not overlap; host_ccc may be NULL for
 * tallies only).  Workspace: ccc2_stream_workspace_size().  The copies run on
 * two internal streams created (with four events) by the first call on each
 * device; the caller's stream is made to wait for them, so synchronising the
 * caller's stream means every result is on the host.  n_phases >= 2.
 */
int ccc2_stream_workspace_size(const ccc_panel *panel, int n_phases, const ccc_opts *opts,
                               size_t *bytes);
int ccc2_stream(const ccc_panel *panel, int n_phases, int32_t *host_tally, float *host_ccc,
                const ccc_opts *opts, void *stream);

/*
 * Host helper: split the slabs [0, n_v) into n_phases contiguous ranges,
 * bounds[0] = 0 <= ... <= bounds[n_phases] = n_v, with about equal triple
 * counts (Sec. 7 item 3 emits the result in phases).  bounds: host
 * int64[n_phases + 1].
 */
int ccc3_phase_bounds(int64_t n_v, int n_phases, int64_t *bounds);

/*
 * Phased 3-way output to host memory: all triples as ccc3_tally_metric over
 * [0, n_v) computes them, slab range by slab range (ccc3_phase_bounds), into
 * two staging buffers in the workspace; each finished range is copied to the
 * caller's host arrays while the next one computes.  host_tally, host_ccc:
 * host memory [ntriples][8] (pinned, or the copies do not overlap; host_ccc
 * may be NULL for tallies only).  Workspace: ccc3_stream_workspace_size().
 * The copies run on the two internal streams of ccc2_stream; the caller's
 * stream is made to wait for them.  n_phases >= 2.
 */
int ccc3_stream_workspace_size(const ccc_panel *panel, int n_phases, const ccc_opts *opts,
                               size_t *bytes);
int ccc3_stream(const ccc_panel *panel, int n_phases, int32_t *host_tally, float *host_ccc,
                const ccc_opts *opts, void *stream);

/*
 * Batched 2-way over independent panels (many SNP panels of uneven n_v and n_f,
 * as in a multi-study run): for every panel k, the tallies and CCC values that
 * ccc2_tally_metric would write to tally[k] and ccc[k].  On the tensor-core
 * path with SM-pair tiles a panel with at least opts->solo tiles (default
 * 1024, n_v >= 5,633) runs as its own launch, and all tiles of up to 64
 * smaller panels run in one persistent launch, so small panels fill the SMs
 * that large ones leave idle.  When that shared launch has fewer tiles than
 * two per SM pair and opts->split is 0, its panels' tiles run as K parts
 * (the n_pf axis of Sec. 4 within one launch) whose partial tallies are
 * summed, with the CCC values formed from the sums; opts->split = 1 keeps
 * every tile whole, n >= 2 splits every shared panel into up to n parts.
 * opts->order and opts->group choose the tile order (see ccc2_batched_tune).
 * panels: host array of n_panels panels; tally, ccc: host arrays of n_panels
 * device pointers (ccc may be NULL for tallies only).  Workspace:
 * ccc2_batched_workspace_size(); with opts->tile = 0 it has room for every
 * tile variant that ccc2_batched_tune tries.  The call queues only stream work (memsets
 * and kernels), so it can be captured into a CUDA graph once a first call has
 * run outside capture.
 */
int ccc2_batched_workspace_size(const ccc_panel *panels, int n_panels, const ccc_opts *opts,
                                size_t *bytes);
int ccc2_batched(const ccc_panel *panels, int n_panels, int32_t *const *tally,
                 float *const *ccc, const ccc_opts *opts, void *stream);

/*
 * Schedule autotuner for ccc2_batched: runs the batch once per candidate,
 * timing each with CUDA events on the stream (synchronising it), one choice
 * after another: the tile variant (SM pairs or one SM, when opts->tile is 0),
 * the K-split policy (automatic or off), the solo-launch threshold (1024,
 * none, 512, 2048 tiles), then group 4, 8, 16 x order 0, 1; each choice keeps
 * the fastest candidate.  The choices are stored in opts->tile, split, solo,
 * group and order; the outputs hold a correct result afterwards.
 * The choice is cached under the batch's shape: the multiset of its panels'
 * (n_v, n_f) power-of-two buckets (bucket(x) = bit length of x - 1), with
 * opts->path, opts->tile, opts->operand and the device's SM count.  A later
 * call whose batch has the same key takes the cached choice and runs the
 * batch once, without the timing runs.  The cache lives in the process; when
 * the environment variable CCC_TUNE_CACHE names a file, choices are also
 * appended to it (one text line each) and read back by later processes.
 * CCC_EINVAL for a null opts or panels or n_panels outside 1 .. 1024.
 */
int ccc2_batched_tune(const ccc_panel *panels, int n_panels, int32_t *const *tally,
                      float *const *ccc, ccc_opts *opts, void *stream);

/* Forget the tuning choices the process holds (the CCC_TUNE_CACHE file is left
 * alone and read again by the next ccc2_batched_tune).  Returns CCC_OK. */
int ccc_tune_cache_clear(void);

/*
 * 3-way tallies of all triples i < j < k with j in [j_begin, j_end) (Eq. 5
 * numerators).  For a fixed j the slab is computed as one GEMM-shaped product
 * of an operand masked elementwise by v_j with the panel, the role that the
 * matrices X_{j,xi} play in Sec. 3.2.  tally: device int32[S(j_end) -
 * S(j_begin)][8].  Needs the workspace.  0 <= j_begin <= j_end <= n_v,
 * n_v <= 65535.
 */
int ccc3_tally(const ccc_panel *panel, int64_t j_begin, int64_t j_end, int32_t *tally,
               const ccc_opts *opts, void *stream);

/*
 * 3-way CCC values (Eq. 4) from tallies of ccc3_tally over the same slabs and
 * counts from ccc_allele_counts.  ccc: device float[..][8].  Workspace as for
 * ccc2_metric (CCC_OP_METRIC).
 */
int ccc3_metric(const int32_t *tally, const int32_t *counts, int64_t n_v, int64_t j_begin,
                int64_t j_end, const ccc_opts *opts, float *ccc, void *stream);

/* Fused 3-way: counts, tallies and CCC values (Eqs. 1, 4, 5).  Needs the workspace. */
int ccc3_tally_metric(const ccc_panel *panel, int64_t j_begin, int64_t j_end, int32_t *tally,
                      float *ccc, const ccc_opts *opts, void *stream);

/*
 * Fused 2-way tensor-core call without a workspace, for callers that cannot
 * allocate device memory: code inside a host framework that owns every device
 * allocation through its own pool, plug-ins that are handed only their input
 * and output buffers, or programs that may not allocate once they are running.
 * The paper has no counterpart; it is an interface convenience of this library.
 *
 * Computes what ccc2_tally_metric computes with opts->path == CCC_PATH_TC,
 * bit for bit: the tile variant opts->tile selects (1 = one SM, 0 or 2 = SM
 * pairs) and the tile order opts->group, with e4m3 operands and without the
 * automatic K split (opts->split must be 0 or 1; tile 3 is rejected, an
 * explicit opts->operand = CCC_OPERAND_E2M1 returns CCC_EUNSUPPORTED).  Its scratch (status
 * word, per-SNP factors, e4m3 count operands) lives in a fixed 32 MiB device
 * array built into the library, which every GPU that loads the library holds
 * until the process exits.  The workspace fields of *opts are ignored.
 * Nothing is allocated: no cudaMalloc, no cudaFree.
 *
 *   panel, tally, ccc, opts, stream: as for ccc2_tally_metric (ccc may be NULL:
 *           tallies only); the argument checks are that call's.
 *   status: optional device int32 owned by the caller (NULL allowed); when
 *           given, it is cleared and receives CCC_ETIMEOUT if a device-side
 *           bounded wait gives up.  With NULL that word lives in the built-in
 *           scratch and is not reported.
 * Limit: the panel must fit the built-in scratch,
 *           256 + 8 n_v (rounded up to 1 KiB) + (round_up(2 n_v, 256) + 256)
 *           * round_up(n_f, 128) <= 32 MiB
 *         (for example n_v = 2,048 with n_f <= 7,680); larger panels return
 *         CCC_ERANGE before anything is queued.
 * Set-up: the first call on each device looks up the array's device address
 *         (with that device current); make that first call before capturing
 *         any stream into a CUDA graph.
 * Sharing: every call on a device uses the same array and leaves its contents
 *         behind; calls whose work overlaps on the GPU (different streams
 *         without ordering between them) race on it and must not be issued.
 */
int ccc2_tally_metric_noalloc(const ccc_panel *panel, int32_t *tally, float *ccc,
                              int32_t *status, const ccc_opts *opts, void *stream);

/* ---------------------------------------------------------------------------
 * Markers with s allele states (Sec. 7 item 2: CCC extended from biallelic SNPs to
 * markers with any number of states, a marker with s_1 states against one with
 * s_2 states giving an s_1 x s_2 table of values).
 *
 * Input: one byte per entry, x | (y << 4) for the unordered pair of allele
 * states (x, y) of individual q, 0 <= x, y < s; an entry with x >= s or
 * y >= s is MISSING (0xFF by convention) and contributes nothing.  SNP i
 * occupies bytes geno[i*ld .. i*ld + n_f - 1]; bytes past n_f are ignored.
 * Requirements: 2 <= s <= 15, n_f >= 1, n_v >= 1, ld >= n_f, ld a multiple
 * of 16, geno 16-byte aligned, device memory.  A panel whose markers have
 * different state counts uses s = the largest; the states a marker never
 * takes give zero tallies and zero values.
 *
 * Definitions: Eqs. 1-3 over S = {0..s-1}:
 *   rho_{i,q}(a)  = [x == a] + [y == a]  (0 for a missing entry),
 *   r_{ij}^{ab}   = sum_q rho_{i,q}(a) rho_{j,q}(b),
 *   CCC_{ij}(a,b) = r/(4 n_ij) (1 - gamma f_i(a)) (1 - gamma f_j(b)),
 * with n_ij, f_i and opts->norm as for the biallelic calls.  With s = 2 and
 * 00 -> (0,0), 01 -> (0,1), 11 -> (1,1), 10 -> missing, every result equals
 * the biallelic call's bit for bit.
 *
 * Output: pairs i < j in the order of ccc2_index, s*s values per pair, (a, b)
 * with a (the state of SNP i) major: tally[ccc2_index(i, j, n_v)*s*s + a*s + b].
 * Tensor-core path on SM pairs only: opts->path must be CCC_PATH_TC
 * (CCC_PATH_POPC returns CCC_EUNSUPPORTED), opts->tile 0 or 2.  Tallies are
 * exact; CCC values are within 1e-6 relative of exact arithmetic.
 * --------------------------------------------------------------------------- */
typedef struct ccc_panel_multi {
  const uint8_t *geno; /* device pointer to n_v rows of ld bytes */
  int64_t n_f;         /* individuals */
  int64_t n_v;         /* markers */
  int64_t ld;          /* row stride in bytes */
  int32_t n_states;    /* s */
  int32_t reserved;    /* zero */
} ccc_panel_multi;

/* Bytes of workspace the multi-allelic calls need (host only).  CCC_OK,
 * CCC_EINVAL, CCC_ERANGE or CCC_EUNSUPPORTED (popcount path). */
int ccc_multi_workspace_size(const ccc_panel_multi *panel, const ccc_opts *opts, size_t *bytes);

/* Per-marker state sums and non-missing counts (Eq. 1 numerators):
 * counts[i*(s+1) + a] = s_i^a for a < s, counts[i*(s+1) + s] = n_i.
 * counts: device int32[n_v][s+1].  Needs no workspace. */
int ccc_multi_counts(const ccc_panel_multi *panel, int32_t *counts, void *stream);

/* Tallies of all pairs i < j (Eq. 2 numerators over S x S).  tally: device
 * int32[npairs][s*s], 16-byte aligned.  Needs the workspace. */
int ccc2_multi_tally(const ccc_panel_multi *panel, int32_t *tally, const ccc_opts *opts,
                     void *stream);

/* Fused: tallies and CCC values (Eqs. 1-3 over S x S), the values formed in
 * the tally kernel's epilogue.  tally: device int32[npairs][s*s]; ccc: device
 * float[npairs][s*s]; both 16-byte aligned.  Needs the workspace. */
int ccc2_multi_tally_metric(const ccc_panel_multi *panel, int32_t *tally, float *ccc,
                            const ccc_opts *opts, void *stream);

/* CCC values (Eq. 3 over S x S) from tallies of ccc2_multi_tally and counts of
 * ccc_multi_counts.  tally: device int32[npairs][s*s]; counts: device
 * int32[n_v][s+1]; ccc: device float[npairs][s*s].  Workspace: any that
 * ccc_multi_workspace_size() accepts for a panel with the same n_v and s. */
int ccc2_multi_metric(const int32_t *tally, const int32_t *counts, int64_t n_v, int32_t n_states,
                      const ccc_opts *opts, float *ccc, void *stream);

/* One phase (Sec. 7 item 3) of ccc2_multi_tally_metric: the pairs with
 * i_begin <= i < i_end and every j > i, stored from index
 * ccc2_index(i_begin, i_begin + 1, n_v) on (s*s values per pair).  tally, ccc:
 * device [ccc2_rows_count(n_v, i_begin, i_end)][s*s].  Workspace as for
 * ccc2_multi_tally_metric.  0 <= i_begin <= i_end <= n_v; ranges on multiples
 * of 8*floor(32/s) markers (ccc2_multi_phase_bounds) waste no tensor work. */
int ccc2_multi_tally_metric_rows(const ccc_panel_multi *panel, int64_t i_begin, int64_t i_end,
                                 int32_t *tally, float *ccc, const ccc_opts *opts, void *stream);

/* Host helper: rows [0, n_v) split into n_phases ranges with about equal pair
 * counts, inner bounds on multiples of 8*floor(32/s).  bounds: host
 * int64[n_phases + 1]. */
int ccc2_multi_phase_bounds(int64_t n_v, int32_t n_states, int n_phases, int64_t *bounds);

/* Phased multi-allelic output to host memory, as ccc2_stream does for
 * biallelic panels: every pair computed phase by phase into two staging
 * buffers of the workspace, each finished phase copied to host_tally /
 * host_ccc ([npairs][s*s], pinned host memory; host_ccc may be NULL) while the
 * next one computes, on the two copy streams of ccc2_stream; the caller's
 * stream waits for the copies.  Workspace: ccc2_multi_stream_workspace_size().
 * n_phases >= 2. */
int ccc2_multi_stream_workspace_size(const ccc_panel_multi *panel, int n_phases,
                                     const ccc_opts *opts, size_t *bytes);
int ccc2_multi_stream(const ccc_panel_multi *panel, int n_phases, int32_t *host_tally,
                      float *host_ccc, const ccc_opts *opts, void *stream);

/*
 * Device-side status of the workspace: *status receives CCC_OK or the first
 * CCC_E* code a kernel recorded (CCC_ETIMEOUT when a bounded wait gave up;
 * CCC_EBOUNDS from the bounds-checking build, include/ccc_checked.h).
 * Synchronises the stream.  Every call that takes a workspace clears the word
 * first, so this reports on the calls since the last workspace call began.
 */
int ccc_status(const ccc_opts *opts, int32_t *status, void *stream);

/*
 * Exact checksum of results (the paper's extended-precision integer checksum,
 * Sec. 5, used to check results bit for bit):
 *   C = sum_e h(base + e) * words[e]  (mod 2^128),
 * words[e] = the e-th 32-bit word of an output array taken as unsigned (a
 * tally, or the bit pattern of a CCC value); h(x) = the SplitMix64 finaliser
 * of (x + 1) * 0x9E3779B97F4A7C15.  Linear, so the checksums of the phases or
 * shards of an output, each with base = its first word's global index, add up
 * (mod 2^128) to the whole's.  words: device, 4-byte aligned, count words;
 * out: device uint64[2] = (low, high), 16-byte aligned, cleared and written
 * by the call.  Needs no workspace.
 */
int ccc_checksum(const void *words, int64_t count, int64_t base, uint64_t *out, void *stream);

/*
 * Self-test of the device-side bounded waits (every pipeline of the library
 * waits on mbarriers through the same bounded loop).  Queues one small kernel
 * whose wait cannot complete: after limit_ns nanoseconds of device time
 * (1e6 <= limit_ns <= 2e9) it gives up, writes CCC_ETIMEOUT to *status
 * (device int32 owned by the caller; written only on a timeout) and exits; the
 * CUDA context stays usable.  Returns CCC_OK once queued, CCC_EINVAL for a
 * bad argument.
 */
int ccc_check_bounded_wait(int32_t *status, int64_t limit_ns, void *stream);

/* ---------------------------------------------------------------------------
 * Rate probes.  Measurement only; the paper has no counterpart (its own peak
 * figures, Sec. 6.1, are the vendor's).  They give the roofline denominators
 * of the tensor-core and popcount paths as work per SM clock cycle on this
 * device, so that a kernel's fraction of peak can be taken at the SM clock it
 * ran at (peak = work per SM per cycle x SMs x clock).
 *
 * ccc_mma_rate: `clusters` clusters of two CTAs (one per SM pair, each CTA
 * alone on its SM; 1 <= clusters <= SMs / 2) each issue n_mma
 * (1 <= n_mma <= 65536) dense cta_group::2 MMAs of M = 256, N = n_cols
 * (a multiple of 16 from 64 to 256) back to back from shared-memory operands into one TMEM
 * accumulator, with operands of the given kind:
 *   CCC_MMA_E4M3       kind::f8f6f4, e4m3 operands, K = 32 per MMA;
 *   CCC_MMA_E2M1       kind::mxf4, e2m1 operands with UE8M0 scale factors per
 *                      32 elements (all 1.0), K = 64 per MMA;
 *   CCC_MMA_E2M1_NVF4  kind::mxf4nvf4, e2m1 operands with UE4M3 scale factors
 *                      per 16 elements (all 1.0), K = 64 per MMA.
 * cycles: device int64[clusters], receives the SM clock cycles from the first
 * issue to the completion of the last MMA (-1 if the wait gave up).  bad:
 * device int32, cleared by the call, receives the number of accumulator
 * entries that differ from n_mma * K (operands are all 1.0), plus 2^20 per
 * wait that gave up.  Flops per SM per cycle = 2 * 256 * n_cols * K * n_mma /
 * (2 * cycles).  CCC_EINVAL for an argument outside these ranges.
 *
 * ccc_popc_rate: `blocks` blocks (1 <= blocks <= 65536) of 1024 threads, each
 * thread running iters (1 <= iters <= 1 << 24) iterations of eight independent
 * 64-bit AND + population counts over registers.  cycles: device
 * int64[blocks], SM clock cycles of each block; sink: device uint64 (written
 * only in a case that does not occur; it keeps the work from being removed).
 * 64-bit AND + POPC per SM per cycle = 8 * 1024 * iters * (blocks resident on
 * an SM) / cycles.
 */
#define CCC_MMA_E4M3 0
#define CCC_MMA_E2M1 1
#define CCC_MMA_E2M1_NVF4 2
int ccc_mma_rate(int kind, int n_cols, int n_mma, int clusters, int64_t *cycles, int32_t *bad,
                 void *stream);
int ccc_popc_rate(int iters, int blocks, int64_t *cycles, uint64_t *sink, void *stream);

/* Index helpers (host): positions defined in the header comment; -1 if out of range. */
int64_t ccc2_index(int64_t i, int64_t j, int64_t n_v);
int64_t ccc3_index(int64_t i, int64_t j, int64_t k, int64_t n_v);
int64_t ccc2_count(int64_t n_v);                       /* n_v (n_v - 1) / 2 */
int64_t ccc3_count(int64_t n_v, int64_t j_begin, int64_t j_end); /* S(j_end) - S(j_begin) */

/* Text for a status code. */
const char *ccc_strerror(int status);

/* The CUDA error code (cudaError_t) behind the last CCC_ECUDA of the calling
 * thread: the error a kernel launch reported, else the runtime's pending error
 * (cudaPeekAtLastError); 0 when there is none.  Host only. */
int ccc_last_cuda_error(void);

/* Number of kernels this library has launched in this process (all entry points). */
uint64_t ccc_launch_count(void);

/*
 * Kernel timing, for instrumentation.  While enabled, every launch of a tally
 * kernel (the dominant kernel of each 2-way and 3-way call) is bracketed by
 * two CUDA events recorded on the call's stream, up to 4096 launches.
 * ccc_timing_read() waits for the recorded events, returns the summed device
 * time in milliseconds and the number of bracketed launches, and clears the
 * record.  Host-side state, one record per process; not thread-safe.
 */
int ccc_timing_enable(int enable);
int ccc_timing_read(double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* CCC_H_ */
