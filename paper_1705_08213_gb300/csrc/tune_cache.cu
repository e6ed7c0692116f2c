// Cache of the batched-schedule autotuner (see tune_cache.h).
//
// File format (CCC_TUNE_CACHE): one choice per line,
//   ccc-tune-v2 <key, 16 hex digits> <group> <order> <tile> <split> <solo> <milliseconds>
// appended as choices are made; when a key appears more than once the last
// line wins.  Lines that do not parse are ignored.
#include "tune_cache.h"

#include <inttypes.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

namespace ccc {
namespace {

std::mutex g_mu;
std::unordered_map<uint64_t, TuneChoice> g_cache;
bool g_file_loaded = false;

int bucket(int64_t x) {
  int b = 0;
  for (uint64_t v = x > 1 ? static_cast<uint64_t>(x - 1) : 0; v != 0; v >>= 1) ++b;
  return b;
}

uint64_t fnv1a(uint64_t h, uint64_t v) {
  for (int i = 0; i < 8; ++i) {
    h ^= (v >> (8 * i)) & 0xFFu;
    h *= 1099511628211ull;
  }
  return h;
}

bool valid_choice(const TuneChoice &c) {
  return (c.group == 4 || c.group == 8 || c.group == 16) && (c.order == 0 || c.order == 1) &&
         (c.tile == 1 || c.tile == 2) && (c.split == 0 || c.split == 1) &&
         (c.solo == -1 || (c.solo > 0 && c.solo <= (1 << 20)));
}

// Caller holds g_mu.
void load_file_locked() {
  if (g_file_loaded) return;
  g_file_loaded = true;
  const char *path = getenv("CCC_TUNE_CACHE");
  if (path == nullptr || path[0] == '\0') return;
  FILE *f = fopen(path, "r");
  if (f == nullptr) return;
  char line[256];
  while (fgets(line, sizeof line, f) != nullptr) {
    uint64_t key = 0;
    TuneChoice c{};
    float ms = 0.f;
    if (sscanf(line, "ccc-tune-v2 %" SCNx64 " %d %d %d %d %d %f", &key, &c.group, &c.order,
               &c.tile, &c.split, &c.solo, &ms) == 7 &&
        valid_choice(c))
      g_cache[key] = c;
  }
  fclose(f);
}

}  // namespace

uint64_t tune_key(const ccc_panel *panels, int n_panels, int path, int tile, int operand, int sms) {
  std::vector<std::pair<int, int>> b;
  b.reserve(static_cast<size_t>(n_panels));
  for (int k = 0; k < n_panels; ++k) b.emplace_back(bucket(panels[k].n_v), bucket(panels[k].n_f));
  std::sort(b.begin(), b.end());
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, 0x7475'6e65'7632ull);  // format tag
  h = fnv1a(h, static_cast<uint64_t>(path));
  h = fnv1a(h, static_cast<uint64_t>(tile));
  h = fnv1a(h, static_cast<uint64_t>(operand));
  h = fnv1a(h, static_cast<uint64_t>(sms));
  h = fnv1a(h, static_cast<uint64_t>(n_panels));
  for (const auto &p : b) h = fnv1a(h, (static_cast<uint64_t>(p.first) << 32) | static_cast<uint32_t>(p.second));
  return h;
}

bool tune_lookup(uint64_t key, TuneChoice *out) {
  std::lock_guard<std::mutex> lock(g_mu);
  load_file_locked();
  const auto it = g_cache.find(key);
  if (it == g_cache.end()) return false;
  *out = it->second;
  return true;
}

void tune_store(uint64_t key, TuneChoice choice, float ms) {
  if (!valid_choice(choice)) return;
  std::lock_guard<std::mutex> lock(g_mu);
  load_file_locked();
  g_cache[key] = choice;
  const char *path = getenv("CCC_TUNE_CACHE");
  if (path == nullptr || path[0] == '\0') return;
  FILE *f = fopen(path, "a");
  if (f == nullptr) return;  // an unwritable cache file only loses persistence
  fprintf(f, "ccc-tune-v2 %016" PRIx64 " %d %d %d %d %d %.4f\n", key, choice.group, choice.order,
          choice.tile, choice.split, choice.solo, static_cast<double>(ms));
  fclose(f);
}

void tune_clear() {
  std::lock_guard<std::mutex> lock(g_mu);
  g_cache.clear();
  g_file_loaded = false;
}

}  // namespace ccc
