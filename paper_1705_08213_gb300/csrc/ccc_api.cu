// C ABI of libccc (declared in include/ccc.h): argument checks, workspace
// layout and the launch sequence of every entry point.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <atomic>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ccc_checked.h"
#include "ccc_launch.h"
#include "tune_cache.h"

namespace ccc {

namespace {

std::atomic<uint64_t> g_launches{0};

// An NVTX range named after the C-ABI call for its lifetime, so that a
// timeline (Nsight Systems, ncu --nvtx) shows each call around its kernels.
// Without a tool attached NVTX calls return at once.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};
// Checked build: output entries hidden from the kernels' index checks.
std::atomic<int64_t> g_checked_shrink{0};

constexpr size_t kAlign = 256;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Largest n_v accepted: operand rows (2 n_v, padded) and tile indices stay in int32.
constexpr int64_t kMaxNV = int64_t(1) << 26;

struct DeviceInfo {
  int device = -1;
  int sms = 0;
  bool sm103 = false;
};

int query_device(DeviceInfo *info) {
  static DeviceInfo cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CCC_ECUDA;
  if (dev < 0 || dev >= 64) return CCC_EUNSUPPORTED;
  DeviceInfo &c = cache[dev];
  if (c.device != dev) {
    int major = 0, minor = 0, sms = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return CCC_ECUDA;
    c.sms = sms;
    c.sm103 = (major == 10 && minor == 3);
    c.device = dev;
  }
  *info = c;
  return c.sm103 ? CCC_OK : CCC_EUNSUPPORTED;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

// Argument checks shared with the allocation-free entry point (ccc_launch.h).
int check_panel(const ccc_panel *p) {
  if (p == nullptr || p->geno == nullptr) return CCC_EINVAL;
  if (p->n_f < 1 || p->n_v < 1) return CCC_EINVAL;
  if (p->ld < (p->n_f + 31) / 32 || (p->ld & 1) != 0) return CCC_EINVAL;
  if (!aligned(p->geno, 16)) return CCC_EINVAL;
  if (p->n_f > CCC_MAX_NF || p->n_v > kMaxNV) return CCC_ERANGE;
  return CCC_OK;
}

#define CCC_TRY_INNER(expr)          \
  do {                               \
    const int rc__ = (expr);         \
    if (rc__ != CCC_OK) return rc__; \
  } while (0)

int check_opts(const ccc_opts *o) {
  if (o == nullptr) return CCC_EINVAL;
  if (o->path != CCC_PATH_TC && o->path != CCC_PATH_POPC) return CCC_EINVAL;
  if (o->norm != CCC_NORM_PERSNP && o->norm != CCC_NORM_JOINT) return CCC_EINVAL;
  if (!(o->gamma >= 0.0 && o->gamma <= 1.0)) return CCC_EINVAL;
  if (o->group < 0 || o->group > 4096 || (o->order != 0 && o->order != 1)) return CCC_EINVAL;
  if (o->tile < 0 || o->tile > 3) return CCC_EINVAL;
  if (o->split < 0 || o->split > 4096) return CCC_EINVAL;
  if (o->operand < CCC_OPERAND_AUTO || o->operand > CCC_OPERAND_E2M1) return CCC_EINVAL;
  return CCC_OK;
}

// FP4 (e2m1) operands for a 2-way tensor-core call: built for the SM-pair
// tiles (tile 0 or 2); automatic = FP4 there.
bool fp4_2way(const ccc_opts *o) {
  if (o->path != CCC_PATH_TC || o->operand == CCC_OPERAND_E4M3) return false;
  return o->tile == 0 || o->tile == 2;
}

// FP4 (e2m1) operands for a 3-way tensor-core call: built for the
// genotype-class route's wide tiles (tile 0 or 3, n_f <= 16,383, where the D
// counts fit 16 bits); automatic = FP4 there.
bool fp4_3way(const ccc_opts *o, int64_t n_f) {
  if (o->path != CCC_PATH_TC || o->operand == CCC_OPERAND_E4M3) return false;
  return (o->tile == 0 || o->tile == 3) && n_f <= 16383;
}

// Options of a 2-way call: tile 3 names a 3-way variant only.
int check_opts2(const ccc_opts *o) {
  CCC_TRY_INNER(check_opts(o));
  if (o->operand == CCC_OPERAND_E2M1 && !fp4_2way(o)) return CCC_EUNSUPPORTED;
  return o->tile > 3 ? CCC_EINVAL : CCC_OK;
}

namespace {

// Workspace layout shared by the 2-way and 3-way calls.
struct Layout {
  size_t status = 0;          // int32 status word
  size_t w = 0;               // float [n_v][2] per-SNP factors
  size_t counts = 0;          // int32 [n_v][3]
  size_t op = 0;              // e4m3 operands [rows_pad][kpad] (TC path)
  size_t planes = 0;          // uint64 [n_v][w64][4] (POPC path)
  size_t lop = 0;             // masked 3-way operands (TC path)
  size_t rtab = 0;            // int32 [pairs][4] 2-way tallies (3-way classes)
  size_t cbuf = 0;            // compacted count rows per slab (3-way classes)
  size_t missing = 0;         // int32 [cbuf_slabs] missing entries of v_j
  size_t dscratch = 0;        // D counts of the wide class tiles in flight
  size_t total = 0;
  int64_t kpad = 0, rows_pad = 0, w64 = 0, lop_rows = 0, cbuf_slabs = 0;
  int64_t mask_rows = 0;      // masked rows per batch buffer after R in op (3-way classes)
  int halves = 1;             // batch buffers (2: the next batch is prepared during this one)
};

int64_t tc_rows_pad(int64_t n_v) { return round_up(2 * n_v, 256) + 256; }

// Panels accepted by one ccc2_batched call.
constexpr int kMaxPanelsPerCall = 1024;

// Bytes of masked 3-way operands staged per batch of slabs.
constexpr size_t kLopBytes = size_t(2) << 30;

// fp4: the 2-way operand matrix holds e2m1 counts, two per byte (K padded to
// 256 entries, rows of kpad / 2 bytes).
Layout make_layout(int64_t n_f, int64_t n_v, int path, int op, int tile = 0, bool fp4 = false) {
  Layout L;
  size_t off = 0;
  L.status = off;
  off += kAlign;
  L.w = off;
  off = align_up(off + sizeof(float) * 2 * static_cast<size_t>(n_v), kAlign);
  L.counts = off;
  off = align_up(off + sizeof(int32_t) * 3 * static_cast<size_t>(n_v), kAlign);
  if (op == CCC_OP_2WAY || op == CCC_OP_3WAY) {
    if (path == CCC_PATH_TC) {
      L.kpad = round_up(n_f, fp4 ? 256 : 128);
      // 2-way tile 3 expands the codes in shared memory: no operand matrix.
      L.rows_pad = (op == CCC_OP_2WAY && tile == 3) ? 0 : tc_rows_pad(n_v);
      off = align_up(off, 1024);
      L.op = off;
      if (op == CCC_OP_3WAY && (tile == 0 || tile == 3)) {
        // Masked rows of as many slabs as fit in kLopBytes (at least the
        // largest slab) right after R, so that one tensor map covers both.
        const int64_t all_rows = tc3_class_mask_rows(0, n_v, n_v);
        const int64_t max_slab = tc3_class_mask_rows((n_v - 1) / 2, (n_v - 1) / 2 + 1, n_v);
        int64_t cap = static_cast<int64_t>(kLopBytes / static_cast<size_t>(fp4 ? L.kpad / 2 : L.kpad));
        if (cap < max_slab) cap = max_slab;
        L.mask_rows = all_rows < cap ? all_rows : cap;
        if (L.mask_rows < 1) L.mask_rows = 1;
        const int64_t per_slab = tc3_class_cbuf_rows(1, n_v) * tc3_class_cap();
        int64_t nb = static_cast<int64_t>(kLopBytes / 2) / per_slab;
        const int64_t nb_rows = (int64_t(1) << 30) / (2 * n_v) - 1;
        if (nb > nb_rows) nb = nb_rows;
        if (nb > n_v) nb = n_v;
        if (nb < 1) nb = 1;
        L.cbuf_slabs = nb;
        L.halves = (all_rows > L.mask_rows || n_v > nb) ? 2 : 1;
      }
      off = align_up(off + static_cast<size_t>(L.rows_pad + L.halves * L.mask_rows) *
                               static_cast<size_t>(fp4 ? L.kpad / 2 : L.kpad),
                     1024);
      if (op == CCC_OP_3WAY && (tile == 0 || tile == 3)) {
        // 2-way tallies of all pairs; compacted rows of cbuf_slabs slabs and
        // their missing counts, per batch buffer.
        L.rtab = off;
        off = align_up(off + 16 * static_cast<size_t>(n_v) * static_cast<size_t>(n_v - 1) / 2 + 16,
                       1024);
        const size_t per_slab = static_cast<size_t>(tc3_class_cbuf_rows(1, n_v) * tc3_class_cap());
        L.cbuf = off;
        off = align_up(off + L.halves * static_cast<size_t>(L.cbuf_slabs) * per_slab, 1024);
        L.missing = off;
        off = align_up(off + L.halves * sizeof(int32_t) * static_cast<size_t>(L.cbuf_slabs), kAlign);
        L.dscratch = off;
        off = align_up(off + static_cast<size_t>(tc3_class_dscratch_bytes()), kAlign);
      } else if (op == CCC_OP_3WAY && tile == 1) {
        // Masked operands of as many slabs as fit in kLopBytes, but at least
        // the largest slab (j = n_v - 2).
        const int64_t all_rows = tc3_lop_rows(0, n_v);
        const int64_t max_slab = tc3_lop_rows(n_v - 1, n_v);
        int64_t cap = static_cast<int64_t>(kLopBytes / static_cast<size_t>(L.kpad));
        cap = cap / 128 * 128;
        if (cap < max_slab) cap = max_slab;
        L.lop_rows = all_rows < cap ? all_rows : cap;
        if (L.lop_rows < 128) L.lop_rows = 128;
        L.lop = off;
        off = align_up(off + static_cast<size_t>(L.lop_rows) * static_cast<size_t>(L.kpad), 1024);
      }
    } else {
      L.w64 = (n_f + 63) / 64;
      L.planes = off;
      off = align_up(off + 32 * static_cast<size_t>(n_v) * static_cast<size_t>(L.w64), kAlign);
    }
  }
  L.total = off;
  return L;
}

int check_workspace(const ccc_opts *o, const Layout &L) {
  if (o->workspace == nullptr || !aligned(o->workspace, kAlign)) return CCC_EINVAL;
  if (o->workspace_bytes < L.total) return CCC_ENOSPACE;
  return CCC_OK;
}

template <typename T>
T *at(const ccc_opts *o, size_t off) {
  return reinterpret_cast<T *>(static_cast<uint8_t *>(o->workspace) + off);
}

int clear_status(const ccc_opts *o, const Layout &L, cudaStream_t s) {
  return cudaMemsetAsync(at<int32_t>(o, L.status), 0, sizeof(int32_t), s) == cudaSuccess
             ? CCC_OK
             : CCC_ECUDA;
}

// Events around tally-kernel launches (ccc_timing_enable / ccc_timing_read).
struct KernelTiming {
  static constexpr int kMax = 4096;
  bool on = false;
  int used = 0;
  cudaEvent_t ev[2 * kMax] = {};
};
KernelTiming g_timing;

// Records the "before" event; returns the slot or -1 when timing is off/full.
int timing_begin(cudaStream_t s) {
  if (!g_timing.on || g_timing.used >= KernelTiming::kMax) return -1;
  const int k = g_timing.used;
  for (int e = 0; e < 2; ++e)
    if (g_timing.ev[2 * k + e] == nullptr && cudaEventCreate(&g_timing.ev[2 * k + e]) != cudaSuccess)
      return -1;
  if (cudaEventRecord(g_timing.ev[2 * k], s) != cudaSuccess) return -1;
  return k;
}

void timing_end(int slot, cudaStream_t s) {
  if (slot < 0) return;
  if (cudaEventRecord(g_timing.ev[2 * slot + 1], s) == cudaSuccess) g_timing.used = slot + 1;
}

#define CCC_TRY(expr)         \
  do {                        \
    const int rc__ = (expr);  \
    if (rc__ != CCC_OK) return rc__; \
  } while (0)

}  // namespace

// The CUDA error behind the last CCC_ECUDA that a launch of this thread saw.
thread_local int g_cuda_error = 0;

int note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return CCC_OK;
  g_cuda_error = static_cast<int>(e);
  return CCC_ECUDA;
}

int64_t pair_index(int64_t i, int64_t j, int64_t n_v) {
  return i * (2 * n_v - i - 1) / 2 + (j - i - 1);
}

int64_t slab_offset(int64_t j, int64_t n_v) {
  // sum_{j' < j} j' (n_v - 1 - j')
  const int64_t s1 = (j - 1) * j / 2;
  const int64_t s2 = (j - 1) * j * (2 * j - 1) / 6;
  return s1 * (n_v - 1) - s2;
}

int64_t checked_out_len(int64_t len) {
#ifdef CCC_BOUNDS_CHECK
  return len - g_checked_shrink.load(std::memory_order_relaxed);
#else
  return len;
#endif
}

int64_t rows_count(int64_t n_v, int64_t i_begin, int64_t i_end) {
  return pair_index(i_end, i_end + 1, n_v) - pair_index(i_begin, i_begin + 1, n_v);
}

// Balanced phase bounds on multiples of `step` rows.
static void phase_bounds(int64_t n_v, int n_phases, int64_t *bounds, int64_t step = 64) {
  const int64_t total = rows_count(n_v, 0, n_v);
  bounds[0] = 0;
  int64_t r = 0;
  for (int p = 1; p < n_phases; ++p) {
    const double target = static_cast<double>(total) * p / n_phases;
    while (r < n_v && static_cast<double>(rows_count(n_v, 0, r)) < target) r += step;
    // The nearer of the two step multiples around the target (the upper one
    // clamped to n_v).
    const int64_t hi = r < n_v ? r : n_v;
    const int64_t lo = r - step;
    int64_t pick = hi;
    if (lo > 0 && lo >= bounds[p - 1] &&
        target - static_cast<double>(rows_count(n_v, 0, lo)) <
            static_cast<double>(rows_count(n_v, 0, hi)) - target) {
      pick = lo;
      r = lo;
    }
    bounds[p] = pick < bounds[p - 1] ? bounds[p - 1] : pick;
  }
  bounds[n_phases] = n_v;
}

// Side stream on which the 3-way class route prepares the next batch of slabs
// (compacted rows, masked rows) while the current batch's tally kernel runs.
struct PrepRes {
  bool ready = false;
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, prepared[2] = {}, consumed[2] = {};
};
PrepRes g_prep_res[64];

int prep_res(int dev, PrepRes **out) {
  PrepRes &r = g_prep_res[dev];
  if (!r.ready) {
    if (cudaStreamCreateWithFlags(&r.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming) != cudaSuccess)
      return CCC_ECUDA;
    for (int k = 0; k < 2; ++k)
      if (cudaEventCreateWithFlags(&r.prepared[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&r.consumed[k], cudaEventDisableTiming) != cudaSuccess)
        return CCC_ECUDA;
    r.ready = true;
  }
  *out = &r;
  return CCC_OK;
}

// 2-way tensor-core tally launch with the tile shape chosen by opts->tile;
// automatic = SM pairs (on GB300 the paired 256 x 256 tile ran the 20,000 x
// 16,384 panel in 6.43 ms against 7.73 ms for one-SM 128 x 256 tiles).
// FP4 operands (fp4_2way) run on the SM-pair tiles only.
static int launch_tally2_tc_auto(const Tally2Args &a, const ccc_opts *o, const uint8_t *op,
                                 int64_t rows_pad, int64_t kpad, int sms, cudaStream_t s) {
  const bool pair = o->tile != 1;
  return pair ? launch_tally2_tc_pair(a, op, rows_pad, kpad, sms, s, fp4_2way(o))
              : launch_tally2_tc(a, op, rows_pad, kpad, sms, s);
}

// The count operand rows of a 2-way tensor-core call, e2m1 or e4m3, row-major
// or (blocked_rows > 0) K-block-major, and, when w is set, the per-SNP factors
// (from the same read of the codes for e2m1 rows and for K-block-major rows).
static int unpack_2way(const ccc_panel *p, const ccc_opts *o, uint8_t *op, int64_t kpad,
                       int64_t rows_pad, cudaStream_t s, int64_t blocked_rows = 0,
                       float *w = nullptr) {
  if (fp4_2way(o))
    return launch_unpack_e2m1(p->geno, p->n_f, p->n_v, p->ld, op, kpad, rows_pad / 2, s,
                              blocked_rows, w, o->gamma);
  if (blocked_rows > 0)
    return launch_unpack_blocked(p->geno, p->n_f, p->n_v, p->ld, op, kpad, rows_pad / 2,
                                 blocked_rows, false, w, o->gamma, s);
  if (w != nullptr)
    CCC_TRY(launch_allele_counts(p->geno, p->n_f, p->n_v, p->ld, nullptr, w, o->gamma, s));
  return launch_unpack_e4m3(p->geno, p->n_f, p->n_v, p->ld, op, kpad, rows_pad / 2, s,
                            blocked_rows);
}

static bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice;
}

// K parts of a 2-way tensor-core call: opts->split when set (at most the K
// stages), else automatic: a panel whose triangle has at most half as many
// tiles as there are SM pairs, with at least 32 K stages, is split so that its
// (tile, part) units fill one or two waves of SM pairs best, two on a tie;
// each part keeps at least 16 K stages.  Measured on GB300 for 512 SNPs (10
// tiles, 76 SM pairs) x 1,000,000 individuals: 7 parts (one wave, 92% full)
// 0.486 ms, 14 parts (two waves, 92% full) 0.479 ms, 15 parts (two waves, 99%
// full) 0.456 ms; three or more waves were slower again (0.51-0.61 ms at 28-60
// parts), as each unit pays its pipeline fill and its partial-sum reductions.
static int k_split_tiles(int requested, int64_t tiles, int64_t kpad, int sms) {
  const int64_t nkb = kpad / 128;
  if (requested >= 1) return static_cast<int>(requested < nkb ? requested : nkb);
  const int64_t clusters = sms / 2;
  if (tiles < 1 || 2 * tiles > clusters || nkb < 32) return 1;
  const int64_t cap = nkb / 16;
  int64_t best = 1;
  double best_fill = 0.0;
  for (int64_t waves = 1; waves <= 2; ++waves) {
    int64_t split = waves * clusters / tiles;
    if (split > cap) split = cap;
    if (split < 1) continue;
    const int64_t units = tiles * split;
    const int64_t slots = (units + clusters - 1) / clusters * clusters;
    const double fill = static_cast<double>(units) / static_cast<double>(slots);
    if (fill >= best_fill) {
      best_fill = fill;
      best = split;
    }
  }
  return best > 1 ? static_cast<int>(best) : 1;
}

// K parts of a 2-way popcount call: opts->split when set (at most the 8-word
// stages), else automatic: a triangle of fewer 64-SNP tiles than four per SM is
// split into about 16 blocks per SM, each part keeping at least 64 words (4,096
// individuals).  Measured on GB300, 512 SNPs (36 tiles) x 1,000,000: 9 parts
// 12.3 ms, 18 parts 10.3, 36 parts 9.4, 72 parts 9.1.
static int popc_split(int requested, int64_t n_v, int64_t w64, int sms) {
  const int64_t stages = (w64 + 7) / 8;
  if (requested >= 1) return static_cast<int>(requested < stages ? requested : stages);
  const int64_t tiles = popc2_tiles(n_v);
  if (tiles < 1 || tiles >= 4 * static_cast<int64_t>(sms)) return 1;
  int64_t split = (16 * static_cast<int64_t>(sms) + tiles - 1) / tiles;
  if (split > stages / 8) split = stages / 8;
  return split > 1 ? static_cast<int>(split) : 1;
}

static int k_split(int requested, int64_t n_v, int64_t kpad, int sms) {
  return k_split_tiles(requested, tc2_pair_tiles(n_v, 0, (n_v + 127) / 128), kpad, sms);
}

// Thresholded output of a 2-way call (ccc2_filter); null for plain output.
struct FilterSpec {
  ccc_hit *hits;
  int64_t cap;
  int64_t *n_hits;
  float threshold;
};

// The 2-way sequence: counts (+ factors), operand preparation, tally kernel.
static int run_2way(const ccc_panel *p, int32_t *tally, float *out_ccc, const ccc_opts *o,
                    cudaStream_t s, const FilterSpec *filter = nullptr, int64_t i_begin = 0,
                    int64_t i_end = -1) {
  CCC_TRY(check_panel(p));
  CCC_TRY(check_opts2(o));
  if (filter == nullptr) {
    if (tally == nullptr || !aligned(tally, 16)) return CCC_EINVAL;
    if (out_ccc != nullptr && !aligned(out_ccc, 16)) return CCC_EINVAL;
  } else {
    if (filter->n_hits == nullptr || !aligned(filter->n_hits, 8) || filter->cap < 0) return CCC_EINVAL;
    if (filter->cap > 0 && (filter->hits == nullptr || !aligned(filter->hits, 8))) return CCC_EINVAL;
    if (!(filter->threshold == filter->threshold) || filter->threshold > 3.0e38f ||
        filter->threshold < -3.0e38f)
      return CCC_EINVAL;
  }
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  const bool fp4 = fp4_2way(o);
  const Layout L = make_layout(p->n_f, p->n_v, o->path, CCC_OP_2WAY, o->tile, fp4);
  CCC_TRY(check_workspace(o, L));
  CCC_TRY(clear_status(o, L, s));
  if (filter != nullptr &&
      cudaMemsetAsync(filter->n_hits, 0, sizeof(int64_t), s) != cudaSuccess)
    return CCC_ECUDA;
  if (p->n_v < 2) return CCC_OK;
  float *w = at<float>(o, L.w);
  const bool want_w = (out_ccc != nullptr || filter != nullptr) && o->norm == CCC_NORM_PERSNP;
  // With tensor-core operand rows the factors come with the unpack.
  const bool w_in_unpack = o->path == CCC_PATH_TC && o->tile != 3;
  if (want_w && !w_in_unpack)
    CCC_TRY(launch_allele_counts(p->geno, p->n_f, p->n_v, p->ld, nullptr, w, o->gamma, s));
  Tally2Args a;
  a.group = o->group;
  if (i_end >= 0) {
    a.i_begin = i_begin;
    a.i_end = i_end;
    a.pair0 = pair_index(i_begin, i_begin + 1, p->n_v);
  }
  if (filter != nullptr) {
    a.hits = filter->cap > 0 ? filter->hits : reinterpret_cast<ccc_hit *>(filter->n_hits);
    a.n_hits = reinterpret_cast<unsigned long long *>(filter->n_hits);
    a.cap = filter->cap;
    a.threshold = filter->threshold;
  }
  a.n_v = p->n_v;
  a.n_f = p->n_f;
  a.w = w;
  a.tally = tally;
  a.ccc = out_ccc;
  a.status = at<int32_t>(o, L.status);
  a.gamma = static_cast<float>(o->gamma);
  a.norm = o->norm;
  if (filter == nullptr)
    a.out_len = checked_out_len(i_end >= 0 ? pairs_in_rows(p->n_v, i_begin, i_end)
                                           : pairs_in_rows(p->n_v, 0, p->n_v));
  int rc;
  if (o->path == CCC_PATH_TC) {
    // tile 3: the tally kernel reads the packed panel and forms the count rows
    // in shared memory; otherwise they are unpacked into the operand matrix.
    const bool packed = o->tile == 3;
    uint8_t *op = packed ? nullptr : at<uint8_t>(o, L.op);
    // K stages are 128-byte runs of a row: 128 e4m3 or 256 e2m1 entries.
    const int split = (filter == nullptr && i_end < 0 && o->tile != 1 && on_device(tally))
                          ? k_split(o->split, p->n_v, fp4 ? L.kpad / 2 : L.kpad, dev.sms)
                          : 1;
    // The K-split kernel reads its operand K-block-major.
    if (!packed)
      CCC_TRY(unpack_2way(p, o, op, L.kpad, L.rows_pad, s, split > 1 ? L.rows_pad : 0,
                          want_w ? w : nullptr));
    if (split > 1) {
      // Partial tallies of the K parts are summed into the zeroed output; the
      // CCC values follow from the complete tallies.
      const size_t bytes = 16 * static_cast<size_t>(p->n_v) * static_cast<size_t>(p->n_v - 1) / 2;
      if (cudaMemsetAsync(tally, 0, bytes, s) != cudaSuccess) return CCC_ECUDA;
      const int slot = timing_begin(s);
      rc = packed ? launch_tally2_tc_pair_split_packed(a, p->geno, p->ld, split, dev.sms, s)
                  : launch_tally2_tc_pair_split(a, op, L.rows_pad, L.kpad, split, dev.sms, s, fp4);
      timing_end(slot, s);
      if (rc != CCC_OK || out_ccc == nullptr) return rc;
      return launch_metric2(tally, w, p->n_v, a.gamma, a.norm, out_ccc, s);
    }
    const int slot = timing_begin(s);
    rc = packed ? launch_tally2_tc_pair_packed(a, p->geno, p->ld, dev.sms, s)
                : launch_tally2_tc_auto(a, o, op, L.rows_pad, L.kpad, dev.sms, s);
    timing_end(slot, s);
    return rc;
  }
  uint64_t *planes = at<uint64_t>(o, L.planes);
  CCC_TRY(launch_planes(p->geno, p->n_f, p->n_v, p->ld, planes, L.w64, s));
  const int psplit = (filter == nullptr && i_end < 0 && on_device(tally))
                         ? popc_split(o->split, p->n_v, L.w64, dev.sms)
                         : 1;
  if (psplit > 1) {
    const size_t bytes = 16 * static_cast<size_t>(p->n_v) * static_cast<size_t>(p->n_v - 1) / 2;
    if (cudaMemsetAsync(tally, 0, bytes, s) != cudaSuccess) return CCC_ECUDA;
  }
  const int slot = timing_begin(s);
  rc = launch_tally2_popc(a, planes, L.w64, s, psplit);
  timing_end(slot, s);
  if (rc != CCC_OK || psplit == 1 || out_ccc == nullptr) return rc;
  return launch_metric2(tally, w, p->n_v, a.gamma, a.norm, out_ccc, s);
}

// A 3-way call after its checks: panel, options, stream, workspace layout and
// the kernel arguments (j_begin, j_end, tally, ccc set per slab range).
struct Run3 {
  const ccc_panel *p;
  const ccc_opts *o;
  cudaStream_t s;
  Layout L;
  DeviceInfo dev;
  Tally3Args a;
  bool fp4 = false;  // e2m1 operands (fp4_3way)
};

static int begin_3way(Run3 &R, const ccc_panel *p, const ccc_opts *o, cudaStream_t s) {
  CCC_TRY(check_panel(p));
  CCC_TRY(check_opts(o));
  R.fp4 = fp4_3way(o, p->n_f);
  if (o->operand == CCC_OPERAND_E2M1 && !R.fp4) return CCC_EUNSUPPORTED;
  if (p->n_v > 65535) return CCC_ERANGE;
  CCC_TRY(query_device(&R.dev));
  R.p = p;
  R.o = o;
  R.s = s;
  R.L = make_layout(p->n_f, p->n_v, o->path, CCC_OP_3WAY, o->tile, R.fp4);
  CCC_TRY(check_workspace(o, R.L));
  CCC_TRY(clear_status(o, R.L, s));
  R.a.n_v = p->n_v;
  R.a.n_f = p->n_f;
  R.a.w = at<float>(o, R.L.w);
  R.a.status = at<int32_t>(o, R.L.status);
  R.a.gamma = static_cast<float>(o->gamma);
  R.a.norm = o->norm;
  return CCC_OK;
}

static bool class_route(const ccc_opts *o) {
  return o->path == CCC_PATH_TC && (o->tile == 0 || o->tile == 3);
}

// Preparation shared by every slab range of a call: per-SNP factors, the e4m3
// operands (tensor cores) or bit planes (popcount), and for the genotype-class
// route the 2-way tallies r_ik of the pairs i < k with i < j_last - 1.
static int prep_3way(Run3 &R, bool want_ccc, int64_t j_last) {
  const ccc_panel *p = R.p;
  const ccc_opts *o = R.o;
  cudaStream_t s = R.s;
  const bool want_w = want_ccc && o->norm == CCC_NORM_PERSNP;
  float *w = at<float>(o, R.L.w);
  // e2m1 operand rows come with the factors from the same read of the codes.
  if (want_w && !(o->path == CCC_PATH_TC && R.fp4))
    CCC_TRY(launch_allele_counts(p->geno, p->n_f, p->n_v, p->ld, nullptr, w, o->gamma, s));
  if (o->path != CCC_PATH_TC)
    return launch_planes(p->geno, p->n_f, p->n_v, p->ld, at<uint64_t>(o, R.L.planes), R.L.w64, s);
  uint8_t *op = at<uint8_t>(o, R.L.op);
  if (R.fp4)
    CCC_TRY(launch_unpack_e2m1(p->geno, p->n_f, p->n_v, p->ld, op, R.L.kpad, R.L.rows_pad / 2, s,
                               0, want_w ? w : nullptr, o->gamma));
  else
    CCC_TRY(launch_unpack_e4m3(p->geno, p->n_f, p->n_v, p->ld, op, R.L.kpad, R.L.rows_pad / 2, s));
  if (!class_route(o)) return CCC_OK;
  const int64_t je = j_last < p->n_v - 1 ? j_last : p->n_v - 1;
  if (je < 2) return CCC_OK;
  Tally2Args a2;
  a2.n_v = p->n_v;
  a2.n_f = p->n_f;
  a2.w = nullptr;
  a2.tally = at<int32_t>(o, R.L.rtab);
  a2.ccc = nullptr;
  a2.status = R.a.status;
  a2.gamma = R.a.gamma;
  a2.norm = R.a.norm;
  a2.i_begin = 0;
  a2.i_end = je - 1;
  a2.pair0 = 0;
  a2.out_len = pairs_in_rows(p->n_v, 0, p->n_v);  // the table holds every pair
  return launch_tally2_tc_pair(a2, op, R.L.rows_pad, R.L.kpad, R.dev.sms, s, R.fp4);
}

// Tallies (and CCC values) of the slabs [R.a.j_begin, R.a.j_end) into
// R.a.tally / R.a.ccc (first triple = slab j_begin's first).
static int slabs_3way(Run3 &R) {
  const ccc_panel *p = R.p;
  const ccc_opts *o = R.o;
  const Layout &L = R.L;
  cudaStream_t s = R.s;
  const Tally3Args &a = R.a;
  if (slab_offset(a.j_end, p->n_v) == slab_offset(a.j_begin, p->n_v)) return CCC_OK;
  // Slab 0 has no i < j and slab n_v - 1 no k > j.
  const int64_t jb = a.j_begin > 1 ? a.j_begin : 1;
  const int64_t je = a.j_end < p->n_v - 1 ? a.j_end : p->n_v - 1;
  if (class_route(o)) {
    // Per batch of slabs: the compacted rows of the individuals with v_j
    // missing, the masked rows, the class kernel.  Batches alternate between
    // L.halves buffers; with two, batch b + 1 is prepared on a side stream
    // (which first waits for everything already queued on s) while batch b's
    // tally kernel runs.
    if (jb >= je) return CCC_OK;
    uint8_t *op = at<uint8_t>(o, L.op);
    int32_t *rtab = at<int32_t>(o, L.rtab);
    uint8_t *cbuf = at<uint8_t>(o, L.cbuf);
    int32_t *missing = at<int32_t>(o, L.missing);
    PrepRes *P = nullptr;
    cudaStream_t ps = s;
    if (L.halves == 2) {
      CCC_TRY(prep_res(R.dev.device, &P));
      ps = P->side;
      if (cudaEventRecord(P->fork, s) != cudaSuccess || cudaStreamWaitEvent(ps, P->fork, 0) != cudaSuccess)
        return CCC_ECUDA;
    }
    const size_t cbuf_half = static_cast<size_t>(L.cbuf_slabs) *
                             static_cast<size_t>(tc3_class_cbuf_rows(1, p->n_v) * tc3_class_cap());
    const int64_t op_rows = L.rows_pad + L.halves * L.mask_rows;
    int64_t j0 = jb;
    for (int b = 0; j0 < je; ++b) {
      // (A first batch of a quarter of the masked rows, so that less preparation
      // precedes the first class kernel, measured 14.04 against 14.13 ms per step
      // at 1,536 x 8,192 but 13.80 against 13.59 ms of class kernels: the extra
      // launch's last wave.  Not kept.)
      int64_t j1 = j0 + 1;
      while (j1 < je && j1 - j0 < L.cbuf_slabs &&
             tc3_class_mask_rows(j0, j1 + 1, p->n_v) <= L.mask_rows)
        ++j1;
      if (tc3_class_mask_rows(j0, j1, p->n_v) > L.mask_rows) return CCC_ERANGE;
      const int h = L.halves == 2 ? (b & 1) : 0;
      uint8_t *cb = cbuf + h * cbuf_half;
      int32_t *ms = missing + h * L.cbuf_slabs;
      const int64_t mrow0 = L.rows_pad + h * L.mask_rows;
      if (P != nullptr && b >= 2 && cudaStreamWaitEvent(ps, P->consumed[h], 0) != cudaSuccess)
        return CCC_ECUDA;
      CCC_TRY(launch_compact3(p->geno, p->n_f, p->n_v, p->ld, cb, ms, j0, j1, ps, R.fp4));
      CCC_TRY(launch_mask3c(p->geno, p->n_f, p->n_v, p->ld, op, L.kpad, mrow0, ms, j0, j1, ps,
                            R.fp4));
      if (P != nullptr && (cudaEventRecord(P->prepared[h], ps) != cudaSuccess ||
                           cudaStreamWaitEvent(s, P->prepared[h], 0) != cudaSuccess))
        return CCC_ECUDA;
      const int slot = timing_begin(s);
      const int rc = launch_tally3_class(a, op, op_rows, mrow0, L.kpad, rtab, cb, ms,
                                         at<uint32_t>(o, L.dscratch), j0, j1, R.dev.sms, s, R.fp4);
      timing_end(slot, s);
      if (rc != CCC_OK) return rc;
      if (P != nullptr && cudaEventRecord(P->consumed[h], s) != cudaSuccess) return CCC_ECUDA;
      j0 = j1;
    }
    return CCC_OK;
  }
  if (o->path == CCC_PATH_TC && o->tile == 2) {
    // Masked operands formed inside the tally kernel from the packed codes
    // (slower on GB300: 45.9 ms against 36.7 ms for the 1,536 x 8,192 panel,
    // because every k-block tile of a slab forms the same i-block operand again).
    const int slot = timing_begin(s);
    const int rc = launch_tally3_fused(a, p->geno, p->ld, at<uint8_t>(o, L.op), L.rows_pad, L.kpad,
                                       R.dev.sms, s);
    timing_end(slot, s);
    return rc;
  }
  if (o->path == CCC_PATH_TC) {
    uint8_t *op = at<uint8_t>(o, L.op);
    uint8_t *lop = at<uint8_t>(o, L.lop);
    int64_t j0 = jb;
    while (j0 < je) {
      int64_t j1 = j0 + 1;
      while (j1 < je && tc3_lop_rows(j0, j1 + 1) <= L.lop_rows) ++j1;
      if (tc3_lop_rows(j0, j1) > L.lop_rows) return CCC_ERANGE;
      CCC_TRY(launch_mask3(p->geno, p->n_f, p->n_v, p->ld, lop, L.kpad, j0, j1, s));
      const int slot = timing_begin(s);
      const int rc = launch_tally3_tc(a, op, L.rows_pad, L.kpad, lop, L.lop_rows, j0, j1, R.dev.sms, s);
      timing_end(slot, s);
      if (rc != CCC_OK) return rc;
      j0 = j1;
    }
    return CCC_OK;
  }
  const int slot = timing_begin(s);
  const int rc = launch_tally3_popc(a, at<uint64_t>(o, L.planes), L.w64, s);
  timing_end(slot, s);
  return rc;
}

// The 3-way sequence over slabs [j_begin, j_end): preparation, then the slabs.
static int run_3way(const ccc_panel *p, int64_t j_begin, int64_t j_end, int32_t *tally,
                    float *out_ccc, const ccc_opts *o, cudaStream_t s) {
  if (p == nullptr) return CCC_EINVAL;
  if (tally == nullptr || !aligned(tally, 16)) return CCC_EINVAL;
  if (out_ccc != nullptr && !aligned(out_ccc, 16)) return CCC_EINVAL;
  if (j_begin < 0 || j_end < j_begin || j_end > p->n_v) return CCC_EINVAL;
  Run3 R;
  CCC_TRY(begin_3way(R, p, o, s));
  if (slab_offset(j_end, p->n_v) == slab_offset(j_begin, p->n_v)) return CCC_OK;
  CCC_TRY(prep_3way(R, out_ccc != nullptr, j_end));
  R.a.j_begin = j_begin;
  R.a.j_end = j_end;
  R.a.tally = tally;
  R.a.ccc = out_ccc;
  R.a.out_len = checked_out_len(slab_offset(j_end, p->n_v) - slab_offset(j_begin, p->n_v));
  return slabs_3way(R);
}

// Workspace of a batch: [status][per panel: factors, operands (or bit planes)].
struct BatchLayout {
  size_t total = 0;
  size_t w[kMaxPanelsPerCall] = {}, op[kMaxPanelsPerCall] = {};
  int64_t kpad[kMaxPanelsPerCall] = {}, rows_pad[kMaxPanelsPerCall] = {}, w64[kMaxPanelsPerCall] = {};
};

// fp4: e2m1 operand rows (K padded to 256 entries, kpad / 2 bytes per row).
static int batch_layout(const ccc_panel *panels, int n, int path, bool fp4, BatchLayout *B) {
  size_t off = kAlign;
  for (int k = 0; k < n; ++k) {
    const ccc_panel &p = panels[k];
    B->w[k] = off;
    off = align_up(off + sizeof(float) * 2 * static_cast<size_t>(p.n_v), kAlign);
    if (path == CCC_PATH_TC) {
      B->kpad[k] = round_up(p.n_f, fp4 ? 256 : 128);
      B->rows_pad[k] = tc_rows_pad(p.n_v);
      off = align_up(off, 1024);
      B->op[k] = off;
      off = align_up(off + static_cast<size_t>(B->rows_pad[k]) *
                               static_cast<size_t>(fp4 ? B->kpad[k] / 2 : B->kpad[k]),
                     1024);
    } else {
      B->w64[k] = (p.n_f + 63) / 64;
      B->op[k] = off;
      off = align_up(off + 32 * static_cast<size_t>(p.n_v) * static_cast<size_t>(B->w64[k]), kAlign);
    }
  }
  B->total = off;
  return CCC_OK;
}

// Default solo-launch threshold of ccc2_batched, in SM-pair tiles.  On GB300
// (e4m3 operands) the 64-panel workload ran at 4.53e14 comparisons/s with
// 1024 (4.47e14 with 512, 4.1e14 with every panel in the persistent launch);
// ccc2_batched_tune measures the alternatives per batch shape.
constexpr int64_t kSoloTiles = 1024;

// K parts of the shared launch's panels (opts->split 0: automatic): when the
// launch holds fewer tiles than two per SM pair, every panel's tiles are split
// by the factor that brings the units to about two per SM pair, each part
// keeping at least 16 K stages; n >= 2: every panel into min(n, stages) parts.
static void batch_splits(const int64_t *tiles, const int64_t *stages, int m, int requested,
                         int sms, int *split) {
  int64_t total = 0;
  for (int x = 0; x < m; ++x) total += tiles[x];
  const int64_t clusters = sms / 2;
  int64_t f = 1;
  if (requested >= 2) f = requested;
  else if (requested == 0 && total > 0 && total < 2 * clusters)
    f = (2 * clusters + total - 1) / total;
  for (int x = 0; x < m; ++x) {
    int64_t p = f;
    const int64_t cap = requested >= 2 ? stages[x] : stages[x] / 16;
    if (p > cap) p = cap;
    split[x] = p > 1 ? static_cast<int>(p) : 1;
  }
}

static int run_batched(const ccc_panel *panels, int n, int32_t *const *tally, float *const *out_ccc,
                       const ccc_opts *o, cudaStream_t s) {
  CCC_TRY(check_opts2(o));
  if (o->tile == 3) return CCC_EINVAL;  // batched panels use the operand matrices
  if (panels == nullptr || tally == nullptr || n < 1 || n > kMaxPanelsPerCall) return CCC_EINVAL;
  for (int k = 0; k < n; ++k) {
    CCC_TRY(check_panel(&panels[k]));
    if (tally[k] == nullptr || !aligned(tally[k], 16)) return CCC_EINVAL;
    if (out_ccc != nullptr && (out_ccc[k] == nullptr || !aligned(out_ccc[k], 16))) return CCC_EINVAL;
  }
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  const bool fp4 = fp4_2way(o);
  static thread_local BatchLayout B;
  batch_layout(panels, n, o->path, fp4, &B);
  if (o->workspace == nullptr || !aligned(o->workspace, kAlign)) return CCC_EINVAL;
  if (o->workspace_bytes < B.total) return CCC_ENOSPACE;
  int32_t *status = at<int32_t>(o, 0);
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), s) != cudaSuccess) return CCC_ECUDA;
  static thread_local Tally2Args args[kMaxPanelsPerCall];
  static thread_local const uint8_t *ops[kMaxPanelsPerCall];
  static thread_local int order[kMaxPanelsPerCall];
  for (int k = 0; k < n; ++k) {
    const ccc_panel &p = panels[k];
    float *w = at<float>(o, B.w[k]);
    const bool want_w = out_ccc != nullptr && o->norm == CCC_NORM_PERSNP && p.n_v >= 2;
    if (want_w && o->path != CCC_PATH_TC)  // tensor cores: the factors come with the unpack
      CCC_TRY(launch_allele_counts(p.geno, p.n_f, p.n_v, p.ld, nullptr, w, o->gamma, s));
    Tally2Args a;
    a.n_v = p.n_v;
    a.n_f = p.n_f;
    a.w = w;
    a.tally = tally[k];
    a.ccc = out_ccc != nullptr ? out_ccc[k] : nullptr;
    a.status = status;
    a.gamma = static_cast<float>(o->gamma);
    a.norm = o->norm;
    a.group = o->group;
    a.out_len = checked_out_len(pairs_in_rows(p.n_v, 0, p.n_v));
    args[k] = a;
    if (p.n_v < 2) continue;
    if (o->path == CCC_PATH_TC) {
      // the operand rows (and factors) are unpacked below, in launch order
    } else {
      uint64_t *planes = at<uint64_t>(o, B.op[k]);
      CCC_TRY(launch_planes(p.geno, p.n_f, p.n_v, p.ld, planes, B.w64[k], s));
      const int slot = timing_begin(s);
      const int rc = launch_tally2_popc(a, planes, B.w64[k], s);
      timing_end(slot, s);
      if (rc != CCC_OK) return rc;
    }
  }
  if (o->path != CCC_PATH_TC) return CCC_OK;
  // Panel order: most tile work (tiles x K stages) first, or as given.
  for (int k = 0; k < n; ++k) order[k] = k;
  if (o->order == 0) {
    auto work = [&](int k) {
      const int64_t nv = panels[k].n_v;
      const int64_t nI = (nv + 63) / 64, nJ = (nv + 127) / 128;
      return (nI * nJ - (nI / 2) * (nI / 2 - 1) - (nI / 2) * (nI & 1)) * (B.kpad[k] / 128);
    };
    for (int x = 1; x < n; ++x)
      for (int y = x; y > 0 && work(order[y]) > work(order[y - 1]); --y) {
        const int t = order[y];
        order[y] = order[y - 1];
        order[y - 1] = t;
      }
  }
  // Operand rows of every panel, in launch order, on the side stream: each
  // tally launch waits only for its own panel's rows (the event's latest
  // record), so the unpacks of later panels run in the SMs that the earlier
  // tally launches leave idle in their last waves.
  PrepRes *P = nullptr;
  CCC_TRY(prep_res(dev.device, &P));
  cudaStream_t ps = P->side;
  if (cudaEventRecord(P->fork, s) != cudaSuccess || cudaStreamWaitEvent(ps, P->fork, 0) != cudaSuccess)
    return CCC_ECUDA;
  auto unpack_panel = [&](int k) -> int {
    const ccc_panel &p = panels[k];
    if (p.n_v < 2) return CCC_OK;
    const bool want_w = out_ccc != nullptr && o->norm == CCC_NORM_PERSNP;
    CCC_TRY(unpack_2way(&p, o, at<uint8_t>(o, B.op[k]), B.kpad[k], B.rows_pad[k], ps, 0,
                        want_w ? at<float>(o, B.w[k]) : nullptr));
    return cudaEventRecord(P->prepared[0], ps) == cudaSuccess ? CCC_OK : CCC_ECUDA;
  };
  // SM-pair tiles: a panel with at least `solo` tiles keeps every SM busy on its
  // own, and runs as its own launch (its operand blocks then have L2 to
  // themselves); the smaller panels share persistent launches.
  const int64_t solo = o->solo == 0 ? kSoloTiles : o->solo < 0 ? (int64_t(1) << 62) : o->solo;
  const int64_t stage_bytes = fp4 ? 256 : 128;  // entries per 128-byte K stage
  int nb = 0;
  if (o->tile != 1) {
    for (int x = 0; x < n; ++x) {
      const int k = order[x];
      const int64_t nB = (panels[k].n_v + 127) / 128;
      if (panels[k].n_v >= 2 && tc2_pair_tiles(panels[k].n_v, 0, nB) >= solo) {
        CCC_TRY(unpack_panel(k));
        if (cudaStreamWaitEvent(s, P->prepared[0], 0) != cudaSuccess) return CCC_ECUDA;
        const int slot = timing_begin(s);
        const int rc = launch_tally2_tc_pair(args[k], at<uint8_t>(o, B.op[k]), B.rows_pad[k],
                                             B.kpad[k], dev.sms, s, fp4);
        timing_end(slot, s);
        if (rc != CCC_OK) return rc;
      } else {
        order[nb++] = k;
      }
    }
  } else {
    nb = n;
  }
  for (int x = 0; x < nb; ++x) CCC_TRY(unpack_panel(order[x]));
  // Every unpack has been issued: the main stream joins the side stream here.
  if (cudaEventRecord(P->prepared[0], ps) != cudaSuccess ||
      cudaStreamWaitEvent(s, P->prepared[0], 0) != cudaSuccess)
    return CCC_ECUDA;
  static thread_local Tally2Args oargs[kMaxBatchPanels];
  static thread_local int64_t orows[kMaxBatchPanels], okpad[kMaxBatchPanels];
  static thread_local int64_t otiles[kMaxBatchPanels], ostages[kMaxBatchPanels];
  static thread_local int osplit[kMaxBatchPanels];
  for (int c0 = 0; c0 < nb; c0 += kMaxBatchPanels) {
    const int m = nb - c0 < kMaxBatchPanels ? nb - c0 : kMaxBatchPanels;
    for (int x = 0; x < m; ++x) {
      const int k = order[c0 + x];
      oargs[x] = args[k];
      ops[x] = at<uint8_t>(o, B.op[k]);
      orows[x] = B.rows_pad[k];
      okpad[x] = B.kpad[k];
      otiles[x] = panels[k].n_v >= 2 ? tc2_pair_tiles(panels[k].n_v, 0, (panels[k].n_v + 127) / 128)
                                     : 0;
      ostages[x] = B.kpad[k] / stage_bytes;
    }
    if (o->tile != 1) {
      batch_splits(otiles, ostages, m, o->split, dev.sms, osplit);
    } else {
      for (int x = 0; x < m; ++x) osplit[x] = 1;
    }
    // Split panels add their partial tallies into zeroed outputs.
    for (int x = 0; x < m; ++x)
      if (osplit[x] > 1 && oargs[x].n_v >= 2 &&
          cudaMemsetAsync(oargs[x].tally, 0,
                          16 * static_cast<size_t>(oargs[x].n_v) * static_cast<size_t>(oargs[x].n_v - 1) / 2,
                          s) != cudaSuccess)
        return CCC_ECUDA;
    const int slot = timing_begin(s);
    const int rc = o->tile == 1
                       ? launch_tally2_tc_batched(oargs, ops, orows, okpad, m, o->group, dev.sms, s)
                       : launch_tally2_tc_pair_batched(oargs, ops, orows, okpad, osplit, m,
                                                       o->group, dev.sms, s, fp4);
    timing_end(slot, s);
    if (rc != CCC_OK) return rc;
    // CCC values of the split panels from their summed tallies.
    for (int x = 0; x < m; ++x)
      if (osplit[x] > 1 && oargs[x].ccc != nullptr && oargs[x].n_v >= 2)
        CCC_TRY(launch_metric2(oargs[x].tally, oargs[x].w, oargs[x].n_v, oargs[x].gamma,
                               oargs[x].norm, oargs[x].ccc, s));
  }
  return CCC_OK;
}

// ---------------------------------------------------------------- markers with s states

static int check_panel_multi(const ccc_panel_multi *p) {
  if (p == nullptr || p->geno == nullptr) return CCC_EINVAL;
  if (p->n_f < 1 || p->n_v < 1 || p->n_states < 2 || p->n_states > 15) return CCC_EINVAL;
  if (p->ld < p->n_f || p->ld % 16 != 0 || !aligned(p->geno, 16)) return CCC_EINVAL;
  if (p->n_f > CCC_MAX_NF || p->n_v > kMaxNV) return CCC_ERANGE;
  return CCC_OK;
}

static int check_opts_multi(const ccc_opts *o) {
  CCC_TRY(check_opts(o));
  if (o->path != CCC_PATH_TC) return CCC_EUNSUPPORTED;
  return (o->tile == 0 || o->tile == 2) ? CCC_OK : CCC_EINVAL;
}

// e2m1 operands for markers with s states: automatic (or asked for) with at
// most 8 states and no K split; asked for with more states: refused.
static int multi_fp4(const ccc_opts *o, int s, int split, bool *fp4) {
  *fp4 = false;
  if (o->operand == CCC_OPERAND_E4M3) return CCC_OK;
  if (s > 8 || split > 1) return o->operand == CCC_OPERAND_E2M1 ? CCC_EUNSUPPORTED : CCC_OK;
  *fp4 = true;
  return CCC_OK;
}

// Workspace of the multi-allelic calls: [status][factors w[n_v][s]][operand rows].
struct MultiLayout {
  size_t status = 0, w = 0, op = 0, total = 0;
  int64_t kpad = 0, rows_pad = 0;
};

// fp4: e2m1 rows (kpad a multiple of 256, kpad / 2 bytes per row), never
// larger than the e4m3 rows the workspace size is given for.
static MultiLayout make_multi_layout(int64_t n_f, int64_t n_v, int s, bool with_op,
                                     bool fp4 = false) {
  MultiLayout L;
  size_t off = kAlign;
  L.w = off;
  off = align_up(off + sizeof(float) * static_cast<size_t>(n_v) * static_cast<size_t>(s), kAlign);
  if (with_op) {
    L.kpad = round_up(n_f, fp4 ? 256 : 128);
    L.rows_pad = multi_rows_pad(n_v, s);
    off = align_up(off, 1024);
    L.op = off;
    off = align_up(off + static_cast<size_t>(L.rows_pad) * static_cast<size_t>(fp4 ? L.kpad / 2 : L.kpad),
                   1024);
  }
  L.total = off;
  return L;
}

static int check_multi_workspace(const ccc_opts *o, const MultiLayout &L, cudaStream_t s) {
  if (o->workspace == nullptr || !aligned(o->workspace, kAlign)) return CCC_EINVAL;
  if (o->workspace_bytes < L.total) return CCC_ENOSPACE;
  return cudaMemsetAsync(at<int32_t>(o, L.status), 0, sizeof(int32_t), s) == cudaSuccess
             ? CCC_OK
             : CCC_ECUDA;
}

// Markers per 256-row operand block: phases on multiples of it waste no tile.
static int64_t multi_block_rows(int s) { return 8 * (32 / s); }

// The multi-allelic 2-way sequence: factors (PERSNP values), operand rows, tally
// kernel over the rows [i_begin, i_end) (all rows when i_end < 0).
static int run_multi(const ccc_panel_multi *p, int32_t *tally, float *out_ccc, const ccc_opts *o,
                     cudaStream_t s, int64_t i_begin = 0, int64_t i_end = -1) {
  CCC_TRY(check_panel_multi(p));
  CCC_TRY(check_opts_multi(o));
  if (tally == nullptr || !aligned(tally, 16)) return CCC_EINVAL;
  if (out_ccc != nullptr && !aligned(out_ccc, 16)) return CCC_EINVAL;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  const int ns = p->n_states;
  const MultiLayout L8 = make_multi_layout(p->n_f, p->n_v, ns, true);
  CCC_TRY(check_multi_workspace(o, L8, s));
  const bool whole = i_end < 0;
  if (whole) {
    i_begin = 0;
    i_end = p->n_v;
  }
  // An explicit E2M1 keeps the automatic K split off (it runs on e4m3 rows);
  // AUTO splits where that pays and takes e4m3 rows for it.
  const bool auto_split_off = o->operand == CCC_OPERAND_E2M1 && o->split == 0;
  const int split = whole && on_device(tally) && !auto_split_off
                        ? k_split_tiles(o->split, (L8.rows_pad / 256) * (L8.rows_pad / 256 + 1) / 2,
                                        L8.kpad, dev.sms)
                        : 1;
  bool fp4 = false;
  CCC_TRY(multi_fp4(o, ns, split, &fp4));
  const MultiLayout L = fp4 ? make_multi_layout(p->n_f, p->n_v, ns, true, true) : L8;
  if (p->n_v < 2) return CCC_OK;
  float *w = at<float>(o, L.w);
  if (out_ccc != nullptr && o->norm == CCC_NORM_PERSNP)
    CCC_TRY(launch_multi_counts(p->geno, p->n_f, p->n_v, p->ld, ns, nullptr, w, o->gamma, s));
  uint8_t *op = at<uint8_t>(o, L.op);
  CCC_TRY(launch_multi_unpack(p->geno, p->n_f, p->n_v, p->ld, ns, op, L.kpad, L.rows_pad, s, fp4));
  if (split > 1) {
    // Partial tallies of the K parts summed into the zeroed output; CCC values
    // from the complete tallies.
    const size_t bytes = 4 * static_cast<size_t>(ns) * ns * static_cast<size_t>(p->n_v) *
                         static_cast<size_t>(p->n_v - 1) / 2;
    if (cudaMemsetAsync(tally, 0, bytes, s) != cudaSuccess) return CCC_ECUDA;
    const int slot = timing_begin(s);
    const int rc = launch_tally2_multi(ns, p->n_v, w, tally, nullptr, at<int32_t>(o, L.status),
                                       static_cast<float>(o->gamma), o->norm, o->group, op,
                                       L.rows_pad, L.kpad, dev.sms, s, 0, p->n_v, 0, split);
    timing_end(slot, s);
    if (rc != CCC_OK || out_ccc == nullptr) return rc;
    return launch_metric2_multi(tally, w, p->n_v, ns, static_cast<float>(o->gamma), o->norm,
                                out_ccc, s);
  }
  const int slot = timing_begin(s);
  const int rc = launch_tally2_multi(ns, p->n_v, w, tally, out_ccc, at<int32_t>(o, L.status),
                                     static_cast<float>(o->gamma), o->norm, o->group, op,
                                     L.rows_pad, L.kpad, dev.sms, s, i_begin, i_end,
                                     pair_index(i_begin, i_begin + 1, p->n_v), 1, fp4);
  timing_end(slot, s);
  return rc;
}

// Largest phase of a multi-allelic split, in pairs.
static int64_t max_phase_pairs_multi(int64_t n_v, int s, int n_phases) {
  int64_t b[1025];
  if (n_phases > 1024) return -1;
  phase_bounds(n_v, n_phases, b, multi_block_rows(s));
  int64_t m = 0;
  for (int k = 0; k < n_phases; ++k) {
    const int64_t c = rows_count(n_v, b[k], b[k + 1]);
    if (c > m) m = c;
  }
  return m;
}

}  // namespace ccc

using namespace ccc;

extern "C" {




void ccc_opts_default(ccc_opts *opts) {
  if (opts == nullptr) return;
  memset(opts, 0, sizeof(*opts));
  opts->path = CCC_PATH_TC;
  opts->norm = CCC_NORM_PERSNP;
  opts->gamma = 2.0 / 3.0;
}

int ccc_workspace_size(const ccc_panel *panel, const ccc_opts *opts, int op, size_t *bytes) {
  if (bytes == nullptr) return CCC_EINVAL;
  CCC_TRY(check_opts(opts));
  if (panel == nullptr || panel->n_f < 1 || panel->n_v < 1) return CCC_EINVAL;
  if (panel->n_f > CCC_MAX_NF || panel->n_v > kMaxNV) return CCC_ERANGE;
  if (op != CCC_OP_2WAY && op != CCC_OP_3WAY && op != CCC_OP_METRIC) return CCC_EINVAL;
  const bool fp4 = (op == CCC_OP_2WAY && fp4_2way(opts)) ||
                   (op == CCC_OP_3WAY && fp4_3way(opts, panel->n_f));
  *bytes = make_layout(panel->n_f, panel->n_v, opts->path, op, opts->tile, fp4).total;
  return CCC_OK;
}

int ccc_allele_counts(const ccc_panel *panel, int32_t *counts, void *stream) {
  const NvtxRange nvtx_range("ccc_allele_counts");
  CCC_TRY(check_panel(panel));
  if (counts == nullptr || !aligned(counts, 4)) return CCC_EINVAL;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  return launch_allele_counts(panel->geno, panel->n_f, panel->n_v, panel->ld, counts, nullptr,
                              0.0, static_cast<cudaStream_t>(stream));
}

int ccc2_tally(const ccc_panel *panel, int32_t *tally, const ccc_opts *opts, void *stream) {
  const NvtxRange nvtx_range("ccc2_tally");
  return run_2way(panel, tally, nullptr, opts, static_cast<cudaStream_t>(stream));
}

int ccc2_tally_metric(const ccc_panel *panel, int32_t *tally, float *out_ccc, const ccc_opts *opts,
                      void *stream) {
  const NvtxRange nvtx_range("ccc2_tally_metric");
  if (out_ccc == nullptr) return CCC_EINVAL;
  return run_2way(panel, tally, out_ccc, opts, static_cast<cudaStream_t>(stream));
}

int ccc2_tally_metric_rows(const ccc_panel *panel, int64_t i_begin, int64_t i_end,
                           int32_t *tally, float *out_ccc, const ccc_opts *opts, void *stream) {
  const NvtxRange nvtx_range("ccc2_tally_metric_rows");
  if (panel == nullptr || i_begin < 0 || i_end < i_begin || i_end > panel->n_v) return CCC_EINVAL;
  if (out_ccc == nullptr) return CCC_EINVAL;
  if (i_begin == i_end || rows_count(panel->n_v, i_begin, i_end) == 0) {
    CCC_TRY(check_panel(panel));
    CCC_TRY(check_opts2(opts));
    return CCC_OK;
  }
  return run_2way(panel, tally, out_ccc, opts, static_cast<cudaStream_t>(stream), nullptr, i_begin,
                  i_end);
}

int64_t ccc2_rows_count(int64_t n_v, int64_t i_begin, int64_t i_end) {
  if (n_v < 1 || i_begin < 0 || i_end < i_begin || i_end > n_v) return -1;
  return rows_count(n_v, i_begin, i_end);
}

int ccc2_phase_bounds(int64_t n_v, int n_phases, int64_t *bounds) {
  if (bounds == nullptr || n_v < 1 || n_phases < 1 || n_phases > 1 << 20) return CCC_EINVAL;
  phase_bounds(n_v, n_phases, bounds);
  return CCC_OK;
}

namespace {

// Internal copy streams and events of ccc2_stream, one set per device.
struct StreamRes {
  bool ready = false;
  cudaStream_t copy[2] = {};
  cudaEvent_t computed[2] = {}, copied[2][2] = {};
};
StreamRes g_stream_res[64];

int stream_res(int dev, StreamRes **out) {
  StreamRes &r = g_stream_res[dev];
  if (!r.ready) {
    for (int k = 0; k < 2; ++k) {
      if (cudaStreamCreateWithFlags(&r.copy[k], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&r.computed[k], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&r.copied[k][0], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&r.copied[k][1], cudaEventDisableTiming) != cudaSuccess)
        return CCC_ECUDA;
    }
    r.ready = true;
  }
  *out = &r;
  return CCC_OK;
}

// Largest phase of a split, in pairs.
int64_t max_phase_pairs(int64_t n_v, int n_phases) {
  int64_t b[1025];
  if (n_phases > 1024) return -1;
  phase_bounds(n_v, n_phases, b);
  int64_t m = 0;
  for (int k = 0; k < n_phases; ++k) {
    const int64_t c = rows_count(n_v, b[k], b[k + 1]);
    if (c > m) m = c;
  }
  return m;
}

}  // namespace

int ccc2_stream_workspace_size(const ccc_panel *panel, int n_phases, const ccc_opts *opts,
                               size_t *bytes) {
  if (bytes == nullptr || panel == nullptr || n_phases < 2 || n_phases > 1024) return CCC_EINVAL;
  size_t base = 0;
  CCC_TRY(ccc_workspace_size(panel, opts, CCC_OP_2WAY, &base));
  const int64_t m = max_phase_pairs(panel->n_v, n_phases);
  *bytes = align_up(base, 1024) + 2 * align_up(static_cast<size_t>(m) * 32, 1024);
  return CCC_OK;
}

int ccc2_stream(const ccc_panel *p, int n_phases, int32_t *host_tally, float *host_ccc,
                const ccc_opts *o, void *stream) {
  const NvtxRange nvtx_range("ccc2_stream");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CCC_TRY(check_panel(p));
  CCC_TRY(check_opts2(o));
  if (host_tally == nullptr || n_phases < 2 || n_phases > 1024) return CCC_EINVAL;
  size_t need = 0;
  CCC_TRY(ccc2_stream_workspace_size(p, n_phases, o, &need));
  if (o->workspace == nullptr || !aligned(o->workspace, kAlign)) return CCC_EINVAL;
  if (o->workspace_bytes < need) return CCC_ENOSPACE;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return CCC_ECUDA;
  StreamRes *R = nullptr;
  CCC_TRY(stream_res(d, &R));
  const Layout L = make_layout(p->n_f, p->n_v, o->path, CCC_OP_2WAY, o->tile, fp4_2way(o));
  CCC_TRY(clear_status(o, L, s));
  if (p->n_v < 2) return CCC_OK;
  const bool want_ccc = host_ccc != nullptr;
  const int64_t slot_pairs = max_phase_pairs(p->n_v, n_phases);
  const size_t slot_bytes = align_up(static_cast<size_t>(slot_pairs) * 32, 1024);
  const size_t slot0 = align_up(L.total, 1024);
  // Preparation once for all phases.
  float *w = at<float>(o, L.w);
  const bool want_w = want_ccc && o->norm == CCC_NORM_PERSNP;
  uint8_t *op = nullptr;
  uint64_t *planes = nullptr;
  const bool packed = o->path == CCC_PATH_TC && o->tile == 3;
  if (want_w && (o->path != CCC_PATH_TC || packed))  // else the factors come with the unpack
    CCC_TRY(launch_allele_counts(p->geno, p->n_f, p->n_v, p->ld, nullptr, w, o->gamma, s));
  if (o->path == CCC_PATH_TC && !packed) {
    op = at<uint8_t>(o, L.op);
    CCC_TRY(unpack_2way(p, o, op, L.kpad, L.rows_pad, s, 0, want_w ? w : nullptr));
  } else if (o->path != CCC_PATH_TC) {
    planes = at<uint64_t>(o, L.planes);
    CCC_TRY(launch_planes(p->geno, p->n_f, p->n_v, p->ld, planes, L.w64, s));
  }
  int64_t bounds[1025];
  phase_bounds(p->n_v, n_phases, bounds);
  for (int ph = 0; ph < n_phases; ++ph) {
    const int64_t i0 = bounds[ph], i1 = bounds[ph + 1];
    const int64_t cnt = rows_count(p->n_v, i0, i1);
    if (cnt == 0) continue;
    const int k = ph & 1;
    int32_t *st = at<int32_t>(o, slot0 + k * slot_bytes);
    float *sc = reinterpret_cast<float *>(st + 4 * slot_pairs);
    if (ph >= 2) {  // the slot's previous copies must have finished
      if (cudaStreamWaitEvent(s, R->copied[k][0], 0) != cudaSuccess ||
          cudaStreamWaitEvent(s, R->copied[k][1], 0) != cudaSuccess)
        return CCC_ECUDA;
    }
    Tally2Args a;
    a.n_v = p->n_v;
    a.n_f = p->n_f;
    a.w = w;
    a.tally = st;
    a.ccc = want_ccc ? sc : nullptr;
    a.status = at<int32_t>(o, L.status);
    a.gamma = static_cast<float>(o->gamma);
    a.norm = o->norm;
    a.group = o->group;
    a.i_begin = i0;
    a.i_end = i1;
    a.pair0 = pair_index(i0, i0 + 1, p->n_v);
    a.out_len = checked_out_len(cnt);
    const int slot = timing_begin(s);
    const int rc = packed ? launch_tally2_tc_pair_packed(a, p->geno, p->ld, dev.sms, s)
                   : o->path == CCC_PATH_TC
                       ? launch_tally2_tc_auto(a, o, op, L.rows_pad, L.kpad, dev.sms, s)
                       : launch_tally2_popc(a, planes, L.w64, s);
    timing_end(slot, s);
    if (rc != CCC_OK) return rc;
    if (cudaEventRecord(R->computed[k], s) != cudaSuccess) return CCC_ECUDA;
    // Tallies on one copy stream, CCC values on the other.
    if (cudaStreamWaitEvent(R->copy[0], R->computed[k], 0) != cudaSuccess ||
        cudaMemcpyAsync(host_tally + 4 * a.pair0, st, static_cast<size_t>(cnt) * 16,
                        cudaMemcpyDeviceToHost, R->copy[0]) != cudaSuccess ||
        cudaEventRecord(R->copied[k][0], R->copy[0]) != cudaSuccess)
      return CCC_ECUDA;
    if (want_ccc) {
      if (cudaStreamWaitEvent(R->copy[1], R->computed[k], 0) != cudaSuccess ||
          cudaMemcpyAsync(host_ccc + 4 * a.pair0, sc, static_cast<size_t>(cnt) * 16,
                          cudaMemcpyDeviceToHost, R->copy[1]) != cudaSuccess)
        return CCC_ECUDA;
    }
    if (cudaEventRecord(R->copied[k][1], R->copy[1]) != cudaSuccess) return CCC_ECUDA;
  }
  for (int k = 0; k < 2; ++k)
    if (cudaEventRecord(R->copied[k][0], R->copy[0]) != cudaSuccess ||
        cudaEventRecord(R->copied[k][1], R->copy[1]) != cudaSuccess ||
        cudaStreamWaitEvent(s, R->copied[k][0], 0) != cudaSuccess ||
        cudaStreamWaitEvent(s, R->copied[k][1], 0) != cudaSuccess)
      return CCC_ECUDA;
  return CCC_OK;
}

namespace {

// Slab bounds with about equal triple counts.
void phase_bounds3(int64_t n_v, int n_phases, int64_t *bounds) {
  const int64_t total = slab_offset(n_v, n_v);
  bounds[0] = 0;
  int64_t j = 0;
  for (int p = 1; p < n_phases; ++p) {
    const double target = static_cast<double>(total) * p / n_phases;
    while (j < n_v && static_cast<double>(slab_offset(j, n_v)) < target) ++j;
    bounds[p] = j < bounds[p - 1] ? bounds[p - 1] : j;
  }
  bounds[n_phases] = n_v;
}

int64_t max_phase_triples(int64_t n_v, int n_phases) {
  int64_t b[1025];
  if (n_phases > 1024) return -1;
  phase_bounds3(n_v, n_phases, b);
  int64_t m = 0;
  for (int k = 0; k < n_phases; ++k) {
    const int64_t c = slab_offset(b[k + 1], n_v) - slab_offset(b[k], n_v);
    if (c > m) m = c;
  }
  return m;
}

}  // namespace

int ccc3_phase_bounds(int64_t n_v, int n_phases, int64_t *bounds) {
  if (bounds == nullptr || n_v < 1 || n_phases < 1 || n_phases > 1 << 20) return CCC_EINVAL;
  phase_bounds3(n_v, n_phases, bounds);
  return CCC_OK;
}

int ccc3_stream_workspace_size(const ccc_panel *panel, int n_phases, const ccc_opts *opts,
                               size_t *bytes) {
  if (bytes == nullptr || panel == nullptr || n_phases < 2 || n_phases > 1024) return CCC_EINVAL;
  size_t base = 0;
  CCC_TRY(ccc_workspace_size(panel, opts, CCC_OP_3WAY, &base));
  const int64_t m = max_phase_triples(panel->n_v, n_phases);
  *bytes = align_up(base, 1024) + 2 * align_up(static_cast<size_t>(m) * 64, 1024);
  return CCC_OK;
}

int ccc3_stream(const ccc_panel *p, int n_phases, int32_t *host_tally, float *host_ccc,
                const ccc_opts *o, void *stream) {
  const NvtxRange nvtx_range("ccc3_stream");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p == nullptr || host_tally == nullptr || n_phases < 2 || n_phases > 1024) return CCC_EINVAL;
  size_t need = 0;
  CCC_TRY(ccc3_stream_workspace_size(p, n_phases, o, &need));
  if (o->workspace == nullptr || !aligned(o->workspace, kAlign)) return CCC_EINVAL;
  if (o->workspace_bytes < need) return CCC_ENOSPACE;
  Run3 R;
  CCC_TRY(begin_3way(R, p, o, s));
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return CCC_ECUDA;
  StreamRes *S = nullptr;
  CCC_TRY(stream_res(d, &S));
  if (p->n_v < 3) return CCC_OK;
  const bool want_ccc = host_ccc != nullptr;
  CCC_TRY(prep_3way(R, want_ccc, p->n_v));
  const int64_t slot_trip = max_phase_triples(p->n_v, n_phases);
  const size_t slot_bytes = align_up(static_cast<size_t>(slot_trip) * 64, 1024);
  const size_t slot0 = align_up(R.L.total, 1024);
  int64_t bounds[1025];
  phase_bounds3(p->n_v, n_phases, bounds);
  for (int ph = 0; ph < n_phases; ++ph) {
    const int64_t j0 = bounds[ph], j1 = bounds[ph + 1];
    const int64_t t0 = slab_offset(j0, p->n_v);
    const int64_t cnt = slab_offset(j1, p->n_v) - t0;
    if (cnt == 0) continue;
    const int k = ph & 1;
    int32_t *st = at<int32_t>(o, slot0 + k * slot_bytes);
    float *sc = reinterpret_cast<float *>(st + 8 * slot_trip);
    if (ph >= 2) {  // the slot's previous copies must have finished
      if (cudaStreamWaitEvent(s, S->copied[k][0], 0) != cudaSuccess ||
          cudaStreamWaitEvent(s, S->copied[k][1], 0) != cudaSuccess)
        return CCC_ECUDA;
    }
    R.a.j_begin = j0;
    R.a.j_end = j1;
    R.a.tally = st;
    R.a.ccc = want_ccc ? sc : nullptr;
    R.a.out_len = checked_out_len(cnt);
    CCC_TRY(slabs_3way(R));
    if (cudaEventRecord(S->computed[k], s) != cudaSuccess) return CCC_ECUDA;
    if (cudaStreamWaitEvent(S->copy[0], S->computed[k], 0) != cudaSuccess ||
        cudaMemcpyAsync(host_tally + 8 * t0, st, static_cast<size_t>(cnt) * 32,
                        cudaMemcpyDeviceToHost, S->copy[0]) != cudaSuccess ||
        cudaEventRecord(S->copied[k][0], S->copy[0]) != cudaSuccess)
      return CCC_ECUDA;
    if (want_ccc) {
      if (cudaStreamWaitEvent(S->copy[1], S->computed[k], 0) != cudaSuccess ||
          cudaMemcpyAsync(host_ccc + 8 * t0, sc, static_cast<size_t>(cnt) * 32,
                          cudaMemcpyDeviceToHost, S->copy[1]) != cudaSuccess)
        return CCC_ECUDA;
    }
    if (cudaEventRecord(S->copied[k][1], S->copy[1]) != cudaSuccess) return CCC_ECUDA;
  }
  for (int k = 0; k < 2; ++k)
    if (cudaEventRecord(S->copied[k][0], S->copy[0]) != cudaSuccess ||
        cudaEventRecord(S->copied[k][1], S->copy[1]) != cudaSuccess ||
        cudaStreamWaitEvent(s, S->copied[k][0], 0) != cudaSuccess ||
        cudaStreamWaitEvent(s, S->copied[k][1], 0) != cudaSuccess)
      return CCC_ECUDA;
  return CCC_OK;
}

int ccc2_batched_workspace_size(const ccc_panel *panels, int n_panels, const ccc_opts *opts,
                                size_t *bytes) {
  if (bytes == nullptr || panels == nullptr || n_panels < 1 || n_panels > kMaxPanelsPerCall)
    return CCC_EINVAL;
  CCC_TRY(check_opts2(opts));
  for (int k = 0; k < n_panels; ++k) {
    if (panels[k].n_f < 1 || panels[k].n_v < 1) return CCC_EINVAL;
    if (panels[k].n_f > CCC_MAX_NF || panels[k].n_v > kMaxNV) return CCC_ERANGE;
  }
  static thread_local BatchLayout B;
  batch_layout(panels, n_panels, opts->path, fp4_2way(opts), &B);
  size_t total = B.total;
  if (opts->path == CCC_PATH_TC && opts->tile == 0 && fp4_2way(opts)) {
    // Automatic tiles: room for the e4m3 operands of the one-SM variant too,
    // which ccc2_batched_tune may try and choose.
    batch_layout(panels, n_panels, opts->path, false, &B);
    if (B.total > total) total = B.total;
  }
  *bytes = total;
  return CCC_OK;
}

int ccc2_batched(const ccc_panel *panels, int n_panels, int32_t *const *tally, float *const *ccc,
                 const ccc_opts *opts, void *stream) {
  const NvtxRange nvtx_range("ccc2_batched");
  return run_batched(panels, n_panels, tally, ccc, opts, static_cast<cudaStream_t>(stream));
}

int ccc2_batched_tune(const ccc_panel *panels, int n_panels, int32_t *const *tally, float *const *ccc,
                      ccc_opts *opts, void *stream) {
  const NvtxRange nvtx_range("ccc2_batched_tune");
  if (opts == nullptr || panels == nullptr || n_panels < 1 || n_panels > kMaxPanelsPerCall)
    return CCC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  // A batch whose panel sizes fall in already-tuned buckets takes the cached
  // schedule without the timing runs.
  const uint64_t key =
      tune_key(panels, n_panels, opts->path, opts->tile, opts->operand, dev.sms);
  auto apply = [](ccc_opts *o, const TuneChoice &c) {
    o->group = c.group;
    o->order = c.order;
    o->tile = c.tile;
    o->split = c.split;
    o->solo = c.solo;
  };
  TuneChoice cached;
  if (tune_lookup(key, &cached)) {
    apply(opts, cached);
    return run_batched(panels, n_panels, tally, ccc, opts, s);
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return CCC_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return CCC_ECUDA;
  }
  int rc = CCC_OK;
  // Whether a candidate's operands fit the caller's workspace.
  auto fits = [&](const TuneChoice &c) -> bool {
    ccc_opts o = *opts;
    apply(&o, c);
    static thread_local BatchLayout BL;
    batch_layout(panels, n_panels, o.path, fp4_2way(&o), &BL);
    return BL.total <= opts->workspace_bytes;
  };
  // One timed run of a candidate; -1 on an error (rc set).
  auto time_run = [&](const TuneChoice &c) -> float {
    ccc_opts o = *opts;
    apply(&o, c);
    cudaEventRecord(e0, s);
    rc = run_batched(panels, n_panels, tally, ccc, &o, s);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (rc == CCC_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      rc = CCC_ECUDA;
    return rc == CCC_OK ? ms : -1.f;
  };
  // Each choice in turn keeps the fastest candidate, the others fixed.
  TuneChoice best{8, 0, opts->tile == 1 ? 1 : 2, 0, static_cast<int>(kSoloTiles)};
  float best_ms = time_run(best);
  auto consider = [&](TuneChoice c) {
    if (rc != CCC_OK || !fits(c)) return;
    const float ms = time_run(c);
    if (rc == CCC_OK && ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  };
  if (opts->tile == 0) {
    TuneChoice c = best;
    c.tile = 1;
    consider(c);
  }
  if (best.tile == 2) {
    TuneChoice c = best;
    c.split = 1;
    consider(c);
    const int solos[3] = {-1, 512, 2048};
    const TuneChoice base = best;
    for (int k = 0; k < 3; ++k) {
      c = base;
      c.solo = solos[k];
      consider(c);
    }
  }
  const int groups[3] = {4, 8, 16};
  const TuneChoice base = best;
  for (int ord = 0; ord < 2; ++ord)
    for (int gi = 0; gi < 3; ++gi) {
      if (groups[gi] == base.group && ord == base.order) continue;
      TuneChoice c = base;
      c.group = groups[gi];
      c.order = ord;
      consider(c);
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CCC_OK) return rc;
  apply(opts, best);
  tune_store(key, best, best_ms);
  // Leave the outputs as the chosen schedule writes them (all schedules agree).
  return run_batched(panels, n_panels, tally, ccc, opts, s);
}

int ccc2_filter(const ccc_panel *panel, float threshold, ccc_hit *hits, int64_t cap,
                int64_t *n_hits, const ccc_opts *opts, void *stream) {
  const NvtxRange nvtx_range("ccc2_filter");
  FilterSpec f{hits, cap, n_hits, threshold};
  return run_2way(panel, nullptr, nullptr, opts, static_cast<cudaStream_t>(stream), &f);
}

int ccc2_metric(const int32_t *tally, const int32_t *counts, int64_t n_v, const ccc_opts *opts,
                float *out_ccc, void *stream) {
  const NvtxRange nvtx_range("ccc2_metric");
  CCC_TRY(check_opts(opts));
  if (n_v < 1 || n_v > kMaxNV) return CCC_EINVAL;
  if (tally == nullptr || counts == nullptr || out_ccc == nullptr) return CCC_EINVAL;
  if (!aligned(tally, 16) || !aligned(out_ccc, 16) || !aligned(counts, 4)) return CCC_EINVAL;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  const Layout L = make_layout(1, n_v, opts->path, CCC_OP_METRIC);
  CCC_TRY(check_workspace(opts, L));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CCC_TRY(clear_status(opts, L, s));
  if (n_v < 2) return CCC_OK;
  float *w = at<float>(opts, L.w);
  if (opts->norm == CCC_NORM_PERSNP) CCC_TRY(launch_factors_from_counts(counts, n_v, w, opts->gamma, s));
  return launch_metric2(tally, w, n_v, static_cast<float>(opts->gamma), opts->norm, out_ccc, s);
}

int ccc3_tally(const ccc_panel *panel, int64_t j_begin, int64_t j_end, int32_t *tally,
               const ccc_opts *opts, void *stream) {
  const NvtxRange nvtx_range("ccc3_tally");
  return run_3way(panel, j_begin, j_end, tally, nullptr, opts, static_cast<cudaStream_t>(stream));
}

int ccc3_tally_metric(const ccc_panel *panel, int64_t j_begin, int64_t j_end, int32_t *tally,
                      float *out_ccc, const ccc_opts *opts, void *stream) {
  const NvtxRange nvtx_range("ccc3_tally_metric");
  if (out_ccc == nullptr) return CCC_EINVAL;
  return run_3way(panel, j_begin, j_end, tally, out_ccc, opts, static_cast<cudaStream_t>(stream));
}

int ccc3_metric(const int32_t *tally, const int32_t *counts, int64_t n_v, int64_t j_begin,
                int64_t j_end, const ccc_opts *opts, float *out_ccc, void *stream) {
  const NvtxRange nvtx_range("ccc3_metric");
  CCC_TRY(check_opts(opts));
  if (n_v < 1 || n_v > kMaxNV || j_begin < 0 || j_end < j_begin || j_end > n_v) return CCC_EINVAL;
  if (tally == nullptr || counts == nullptr || out_ccc == nullptr) return CCC_EINVAL;
  if (!aligned(tally, 16) || !aligned(out_ccc, 16) || !aligned(counts, 4)) return CCC_EINVAL;
  if (j_end - j_begin > 65535) return CCC_ERANGE;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  const Layout L = make_layout(1, n_v, opts->path, CCC_OP_METRIC);
  CCC_TRY(check_workspace(opts, L));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CCC_TRY(clear_status(opts, L, s));
  float *w = at<float>(opts, L.w);
  if (opts->norm == CCC_NORM_PERSNP) CCC_TRY(launch_factors_from_counts(counts, n_v, w, opts->gamma, s));
  return launch_metric3(tally, w, n_v, j_begin, j_end, static_cast<float>(opts->gamma), opts->norm,
                        out_ccc, s);
}

int ccc_checksum(const void *words, int64_t count, int64_t base, uint64_t *out, void *stream) {
  const NvtxRange nvtx_range("ccc_checksum");
  if (out == nullptr || !aligned(out, 16) || count < 0 || base < 0) return CCC_EINVAL;
  if (count > 0 && (words == nullptr || !aligned(words, 4))) return CCC_EINVAL;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  return launch_checksum(static_cast<const uint32_t *>(words), count, base, out,
                         static_cast<cudaStream_t>(stream));
}

int ccc_check_bounded_wait(int32_t *status, int64_t limit_ns, void *stream) {
  if (status == nullptr || !aligned(status, 4)) return CCC_EINVAL;
  if (limit_ns < 1000000 || limit_ns > 2000000000) return CCC_EINVAL;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  return launch_wait_selftest(status, static_cast<uint64_t>(limit_ns),
                              static_cast<cudaStream_t>(stream));
}

int ccc_last_cuda_error(void) {
  if (g_cuda_error != 0) return g_cuda_error;
  return static_cast<int>(cudaPeekAtLastError());
}

int ccc_mma_rate(int kind, int n_cols, int n_mma, int clusters, int64_t *cycles, int32_t *bad,
                 void *stream) {
  if (kind < CCC_MMA_E4M3 || kind > CCC_MMA_E2M1_NVF4) return CCC_EINVAL;
  if (n_cols < 64 || n_cols > 256 || n_cols % 16 != 0) return CCC_EINVAL;
  if (n_mma < 1 || n_mma > 65536) return CCC_EINVAL;
  if (cycles == nullptr || !aligned(cycles, 8) || bad == nullptr || !aligned(bad, 4))
    return CCC_EINVAL;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  if (clusters < 1 || clusters > dev.sms / 2) return CCC_EINVAL;
  NvtxRange nvtx("ccc_mma_rate");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(bad, 0, sizeof(int32_t), s) != cudaSuccess) return CCC_ECUDA;
  return launch_mma_rate(kind, n_cols, n_mma, clusters, cycles, bad, s);
}

int ccc_popc_rate(int iters, int blocks, int64_t *cycles, uint64_t *sink, void *stream) {
  if (iters < 1 || iters > (1 << 24) || blocks < 1 || blocks > 65536) return CCC_EINVAL;
  if (cycles == nullptr || !aligned(cycles, 8) || sink == nullptr || !aligned(sink, 8))
    return CCC_EINVAL;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  NvtxRange nvtx("ccc_popc_rate");
  return launch_popc_rate(iters, blocks, cycles, sink, static_cast<cudaStream_t>(stream));
}

int ccc_status(const ccc_opts *opts, int32_t *status, void *stream) {
  if (opts == nullptr || status == nullptr || opts->workspace == nullptr) return CCC_EINVAL;
  if (opts->workspace_bytes < kAlign) return CCC_ENOSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(status, opts->workspace, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return CCC_ECUDA;
  return CCC_OK;
}

int64_t ccc2_index(int64_t i, int64_t j, int64_t n_v) {
  if (i < 0 || j <= i || j >= n_v) return -1;
  return pair_index(i, j, n_v);
}

int64_t ccc3_index(int64_t i, int64_t j, int64_t k, int64_t n_v) {
  if (i < 0 || j <= i || k <= j || k >= n_v) return -1;
  return slab_offset(j, n_v) + i * (n_v - 1 - j) + (k - j - 1);
}

int64_t ccc2_count(int64_t n_v) { return n_v < 2 ? 0 : n_v * (n_v - 1) / 2; }

int64_t ccc3_count(int64_t n_v, int64_t j_begin, int64_t j_end) {
  if (n_v < 1 || j_begin < 0 || j_end < j_begin || j_end > n_v) return -1;
  return slab_offset(j_end, n_v) - slab_offset(j_begin, n_v);
}

const char *ccc_strerror(int status) {
  switch (status) {
    case CCC_OK: return "ok";
    case CCC_EINVAL: return "invalid argument";
    case CCC_ERANGE: return "size out of the supported range";
    case CCC_EUNSUPPORTED: return "unsupported device or path";
    case CCC_ECUDA: return "CUDA call failed";
    case CCC_ETIMEOUT: return "device-side wait timed out";
    case CCC_ENOSPACE: return "workspace too small";
    case CCC_EBOUNDS: return "index out of bounds on the device (checked build)";
    default: return "unknown status";
  }
}

uint64_t ccc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int ccc_checked_shrink_outputs(int64_t n) {
#ifdef CCC_BOUNDS_CHECK
  if (n < 0) return CCC_EINVAL;
  g_checked_shrink.store(n, std::memory_order_relaxed);
  return CCC_OK;
#else
  (void)n;
  return CCC_EUNSUPPORTED;  // the normal build has no index checks
#endif
}

int ccc_tune_cache_clear(void) {
  tune_clear();
  return CCC_OK;
}

int ccc_timing_enable(int enable) {
  g_timing.on = enable != 0;
  return CCC_OK;
}

int ccc_timing_read(double *total_ms, int64_t *launches) {
  if (total_ms == nullptr || launches == nullptr) return CCC_EINVAL;
  double sum = 0.0;
  for (int k = 0; k < g_timing.used; ++k) {
    float ms = 0.f;
    if (cudaEventSynchronize(g_timing.ev[2 * k + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, g_timing.ev[2 * k], g_timing.ev[2 * k + 1]) != cudaSuccess)
      return CCC_ECUDA;
    sum += ms;
  }
  *total_ms = sum;
  *launches = g_timing.used;
  g_timing.used = 0;
  return CCC_OK;
}

int ccc_multi_workspace_size(const ccc_panel_multi *panel, const ccc_opts *opts, size_t *bytes) {
  if (bytes == nullptr || panel == nullptr) return CCC_EINVAL;
  CCC_TRY(check_opts_multi(opts));
  if (panel->n_f < 1 || panel->n_v < 1 || panel->n_states < 2 || panel->n_states > 15)
    return CCC_EINVAL;
  if (panel->n_f > CCC_MAX_NF || panel->n_v > kMaxNV) return CCC_ERANGE;
  *bytes = make_multi_layout(panel->n_f, panel->n_v, panel->n_states, true).total;
  return CCC_OK;
}

int ccc_multi_counts(const ccc_panel_multi *panel, int32_t *counts, void *stream) {
  const NvtxRange nvtx_range("ccc_multi_counts");
  CCC_TRY(check_panel_multi(panel));
  if (counts == nullptr || !aligned(counts, 4)) return CCC_EINVAL;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  return launch_multi_counts(panel->geno, panel->n_f, panel->n_v, panel->ld, panel->n_states,
                             counts, nullptr, 0.0, static_cast<cudaStream_t>(stream));
}

int ccc2_multi_tally(const ccc_panel_multi *panel, int32_t *tally, const ccc_opts *opts,
                     void *stream) {
  const NvtxRange nvtx_range("ccc2_multi_tally");
  return run_multi(panel, tally, nullptr, opts, static_cast<cudaStream_t>(stream));
}

int ccc2_multi_tally_metric(const ccc_panel_multi *panel, int32_t *tally, float *out_ccc,
                            const ccc_opts *opts, void *stream) {
  const NvtxRange nvtx_range("ccc2_multi_tally_metric");
  if (out_ccc == nullptr) return CCC_EINVAL;
  return run_multi(panel, tally, out_ccc, opts, static_cast<cudaStream_t>(stream));
}

int ccc2_multi_metric(const int32_t *tally, const int32_t *counts, int64_t n_v, int32_t n_states,
                      const ccc_opts *opts, float *out_ccc, void *stream) {
  const NvtxRange nvtx_range("ccc2_multi_metric");
  CCC_TRY(check_opts_multi(opts));
  if (n_v < 1 || n_v > kMaxNV || n_states < 2 || n_states > 15) return CCC_EINVAL;
  if (tally == nullptr || counts == nullptr || out_ccc == nullptr) return CCC_EINVAL;
  if (!aligned(tally, 4) || !aligned(out_ccc, 4) || !aligned(counts, 4)) return CCC_EINVAL;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const MultiLayout L = make_multi_layout(1, n_v, n_states, false);
  CCC_TRY(check_multi_workspace(opts, L, s));
  if (n_v < 2) return CCC_OK;
  float *w = at<float>(opts, L.w);
  if (opts->norm == CCC_NORM_PERSNP)
    CCC_TRY(launch_multi_factors(counts, n_v, n_states, w, opts->gamma, s));
  return launch_metric2_multi(tally, w, n_v, n_states, static_cast<float>(opts->gamma), opts->norm,
                              out_ccc, s);
}

int ccc2_multi_tally_metric_rows(const ccc_panel_multi *panel, int64_t i_begin, int64_t i_end,
                                 int32_t *tally, float *out_ccc, const ccc_opts *opts, void *stream) {
  const NvtxRange nvtx_range("ccc2_multi_tally_metric_rows");
  if (panel == nullptr || i_begin < 0 || i_end < i_begin || i_end > panel->n_v) return CCC_EINVAL;
  if (out_ccc == nullptr) return CCC_EINVAL;
  if (i_begin == i_end || rows_count(panel->n_v, i_begin, i_end) == 0) {
    CCC_TRY(check_panel_multi(panel));
    CCC_TRY(check_opts_multi(opts));
    return CCC_OK;
  }
  return run_multi(panel, tally, out_ccc, opts, static_cast<cudaStream_t>(stream), i_begin, i_end);
}

int ccc2_multi_phase_bounds(int64_t n_v, int32_t n_states, int n_phases, int64_t *bounds) {
  if (bounds == nullptr || n_v < 1 || n_states < 2 || n_states > 15 || n_phases < 1 ||
      n_phases > 1 << 20)
    return CCC_EINVAL;
  phase_bounds(n_v, n_phases, bounds, multi_block_rows(n_states));
  return CCC_OK;
}

int ccc2_multi_stream_workspace_size(const ccc_panel_multi *panel, int n_phases,
                                     const ccc_opts *opts, size_t *bytes) {
  if (bytes == nullptr || panel == nullptr || n_phases < 2 || n_phases > 1024) return CCC_EINVAL;
  size_t base = 0;
  CCC_TRY(ccc_multi_workspace_size(panel, opts, &base));
  const int64_t m = max_phase_pairs_multi(panel->n_v, panel->n_states, n_phases);
  const size_t ss = static_cast<size_t>(panel->n_states) * static_cast<size_t>(panel->n_states);
  *bytes = align_up(base, 1024) + 2 * align_up(static_cast<size_t>(m) * ss * 8, 1024);
  return CCC_OK;
}

int ccc2_multi_stream(const ccc_panel_multi *p, int n_phases, int32_t *host_tally, float *host_ccc,
                      const ccc_opts *o, void *stream) {
  const NvtxRange nvtx_range("ccc2_multi_stream");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CCC_TRY(check_panel_multi(p));
  CCC_TRY(check_opts_multi(o));
  if (host_tally == nullptr || n_phases < 2 || n_phases > 1024) return CCC_EINVAL;
  size_t need = 0;
  CCC_TRY(ccc2_multi_stream_workspace_size(p, n_phases, o, &need));
  if (o->workspace == nullptr || !aligned(o->workspace, kAlign)) return CCC_EINVAL;
  if (o->workspace_bytes < need) return CCC_ENOSPACE;
  DeviceInfo dev;
  CCC_TRY(query_device(&dev));
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return CCC_ECUDA;
  StreamRes *R = nullptr;
  CCC_TRY(stream_res(d, &R));
  const int ns = p->n_states;
  const int64_t ss = static_cast<int64_t>(ns) * ns;
  const MultiLayout L8 = make_multi_layout(p->n_f, p->n_v, ns, true);
  bool fp4 = false;
  CCC_TRY(multi_fp4(o, ns, 1, &fp4));
  const MultiLayout L = fp4 ? make_multi_layout(p->n_f, p->n_v, ns, true, true) : L8;
  if (cudaMemsetAsync(at<int32_t>(o, L.status), 0, sizeof(int32_t), s) != cudaSuccess)
    return CCC_ECUDA;
  if (p->n_v < 2) return CCC_OK;
  const bool want_ccc = host_ccc != nullptr;
  const int64_t slot_pairs = max_phase_pairs_multi(p->n_v, ns, n_phases);
  const size_t slot_bytes = align_up(static_cast<size_t>(slot_pairs * ss) * 8, 1024);
  const size_t slot0 = align_up(L8.total, 1024);  // as ccc2_multi_stream_workspace_size
  // Preparation once for all phases.
  float *w = at<float>(o, L.w);
  if (want_ccc && o->norm == CCC_NORM_PERSNP)
    CCC_TRY(launch_multi_counts(p->geno, p->n_f, p->n_v, p->ld, ns, nullptr, w, o->gamma, s));
  uint8_t *op = at<uint8_t>(o, L.op);
  CCC_TRY(launch_multi_unpack(p->geno, p->n_f, p->n_v, p->ld, ns, op, L.kpad, L.rows_pad, s, fp4));
  int64_t bounds[1025];
  phase_bounds(p->n_v, n_phases, bounds, multi_block_rows(ns));
  for (int ph = 0; ph < n_phases; ++ph) {
    const int64_t i0 = bounds[ph], i1 = bounds[ph + 1];
    const int64_t cnt = rows_count(p->n_v, i0, i1);
    if (cnt == 0) continue;
    const int k = ph & 1;
    int32_t *st = at<int32_t>(o, slot0 + k * slot_bytes);
    float *sc = reinterpret_cast<float *>(st + ss * slot_pairs);
    if (ph >= 2) {  // the slot's previous copies must have finished
      if (cudaStreamWaitEvent(s, R->copied[k][0], 0) != cudaSuccess ||
          cudaStreamWaitEvent(s, R->copied[k][1], 0) != cudaSuccess)
        return CCC_ECUDA;
    }
    const int64_t pair0 = pair_index(i0, i0 + 1, p->n_v);
    const int slot = timing_begin(s);
    const int rc = launch_tally2_multi(ns, p->n_v, w, st, want_ccc ? sc : nullptr,
                                       at<int32_t>(o, L.status), static_cast<float>(o->gamma),
                                       o->norm, o->group, op, L.rows_pad, L.kpad, dev.sms, s, i0, i1,
                                       pair0, 1, fp4);
    timing_end(slot, s);
    if (rc != CCC_OK) return rc;
    if (cudaEventRecord(R->computed[k], s) != cudaSuccess) return CCC_ECUDA;
    // Tallies on one copy stream, CCC values on the other.
    const size_t bytes = static_cast<size_t>(cnt * ss) * 4;
    if (cudaStreamWaitEvent(R->copy[0], R->computed[k], 0) != cudaSuccess ||
        cudaMemcpyAsync(host_tally + ss * pair0, st, bytes, cudaMemcpyDeviceToHost, R->copy[0]) !=
            cudaSuccess ||
        cudaEventRecord(R->copied[k][0], R->copy[0]) != cudaSuccess)
      return CCC_ECUDA;
    if (want_ccc) {
      if (cudaStreamWaitEvent(R->copy[1], R->computed[k], 0) != cudaSuccess ||
          cudaMemcpyAsync(host_ccc + ss * pair0, sc, bytes, cudaMemcpyDeviceToHost, R->copy[1]) !=
              cudaSuccess)
        return CCC_ECUDA;
    }
    if (cudaEventRecord(R->copied[k][1], R->copy[1]) != cudaSuccess) return CCC_ECUDA;
  }
  for (int k = 0; k < 2; ++k)
    if (cudaEventRecord(R->copied[k][0], R->copy[0]) != cudaSuccess ||
        cudaEventRecord(R->copied[k][1], R->copy[1]) != cudaSuccess ||
        cudaStreamWaitEvent(s, R->copied[k][0], 0) != cudaSuccess ||
        cudaStreamWaitEvent(s, R->copied[k][1], 0) != cudaSuccess)
      return CCC_ECUDA;
  return CCC_OK;
}

}  // extern "C"
