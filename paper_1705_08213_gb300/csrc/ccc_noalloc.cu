// ccc2_tally_metric_noalloc: the fused 2-way tensor-core call for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running inside a host
// framework that owns every device allocation through its own pool, plug-ins
// that are handed only their input and output buffers, and setups where
// allocation is forbidden after start-up (for instance while a stream is being
// recorded elsewhere, or under a strict memory budget).  They can still pass
// their inputs and outputs, but not a workspace.  This entry point therefore
// keeps its scratch (status word, per-SNP factors, e4m3 count operands) in a
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
//
// The computation is that of ccc2_tally_metric with opts->path == CCC_PATH_TC
// and the K split off: the tile variant opts->tile selects (the SM-pair
// kernel unless it is 1), on the same data layout, with bit-identical results;
// only the scratch addresses differ.
#include <mutex>

#include "ccc_launch.h"

namespace ccc {
namespace {

// Size of the built-in scratch: 32 MiB.
constexpr size_t kScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current).  Returns nullptr on failure.
void *scratch_address(int dev) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return nullptr;
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace
}  // namespace ccc

extern "C" int ccc2_tally_metric_noalloc(const ccc_panel *p, int32_t *tally, float *out_ccc,
                                         int32_t *status, const ccc_opts *o, void *stream) {
  using namespace ccc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Arguments: as for ccc2_tally_metric (the workspace fields of *o are
  // ignored); the tensor-core path only, unsplit, with the operand matrix in the
  // scratch (not tile 3).
  int rc = check_panel(p);
  if (rc != CCC_OK) return rc;
  rc = check_opts2(o);
  if (rc != CCC_OK) return rc;
  if (o->path != CCC_PATH_TC || o->tile == 3 || o->split > 1) return CCC_EINVAL;
  if (o->operand == CCC_OPERAND_E2M1) return CCC_EUNSUPPORTED;  // e4m3 operands in the scratch
  if (tally == nullptr || (reinterpret_cast<uintptr_t>(tally) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(out_ccc) & 15) != 0 ||
      (reinterpret_cast<uintptr_t>(status) & 3) != 0)
    return CCC_EINVAL;

  // Scratch layout: [status 256 B][factors n_v x 2 floats][e4m3 operands].
  const int64_t kpad = (p->n_f + 127) / 128 * 128;
  const int64_t rows_pad = (2 * p->n_v + 255) / 256 * 256 + 256;
  const size_t off_w = 256;
  const size_t off_op = up(off_w + sizeof(float) * 2 * static_cast<size_t>(p->n_v), 1024);
  const double need = static_cast<double>(off_op) + static_cast<double>(rows_pad) * kpad;
  if (need > static_cast<double>(kScratchBytes)) return CCC_ERANGE;

  int dev = 0, major = 0, minor = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CCC_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return CCC_EUNSUPPORTED;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CCC_ECUDA;
  if (major != 10 || minor != 3) return CCC_EUNSUPPORTED;
  uint8_t *scratch = static_cast<uint8_t *>(scratch_address(dev));
  if (scratch == nullptr) return CCC_ECUDA;

  int32_t *st = status != nullptr ? status : reinterpret_cast<int32_t *>(scratch);
  float *w = reinterpret_cast<float *>(scratch + off_w);
  uint8_t *op = scratch + off_op;
  // The status word must start at zero; everything else is rewritten in full.
  if (cudaMemsetAsync(st, 0, sizeof(int32_t), s) != cudaSuccess) return CCC_ECUDA;
  if (p->n_v < 2) return CCC_OK;

  if (out_ccc != nullptr && o->norm == CCC_NORM_PERSNP) {
    rc = launch_allele_counts(p->geno, p->n_f, p->n_v, p->ld, nullptr, w, o->gamma, s);
    if (rc != CCC_OK) return rc;
  }
  Tally2Args a;
  a.n_v = p->n_v;
  a.n_f = p->n_f;
  a.w = w;
  a.tally = tally;
  a.ccc = out_ccc;
  a.status = st;
  a.gamma = static_cast<float>(o->gamma);
  a.norm = o->norm;
  a.group = o->group;
  a.out_len = pairs_in_rows(p->n_v, 0, p->n_v);
  rc = launch_unpack_e4m3(p->geno, p->n_f, p->n_v, p->ld, op, kpad, rows_pad / 2, s);
  if (rc != CCC_OK) return rc;
  return o->tile == 1 ? launch_tally2_tc(a, op, rows_pad, kpad, sms, s)
                      : launch_tally2_tc_pair(a, op, rows_pad, kpad, sms, s);
}
