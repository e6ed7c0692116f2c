// Cache of the batched-schedule autotuner (ccc2_batched_tune): the fastest
// schedule (tile variant, K-split policy, solo-launch threshold, group, order)
// per batch shape, kept for the process and, when the
// environment variable CCC_TUNE_CACHE names a file, in that file across
// processes.  Host code only.
#pragma once

#include <stdint.h>

#include "../../include/ccc.h"

namespace ccc {

// The ccc_opts fields a tuning run chooses.
struct TuneChoice {
  int group;  // 4, 8 or 16
  int order;  // 0 or 1
  int tile;   // 1 (one SM) or 2 (SM pairs)
  int split;  // 0 (automatic K split in the shared launch) or 1 (off)
  int solo;   // solo-launch threshold in SM-pair tiles (> 0), or -1 (none)
};

// Key of a batch: the multiset of its panels' (n_v, n_f) power-of-two buckets
// (bucket(x) = bit length of x - 1), with the path, the requested tile
// variant, the operand encoding and the device's SM count.  Panels whose
// sizes fall in the same buckets share a key.
uint64_t tune_key(const ccc_panel *panels, int n_panels, int path, int tile, int operand, int sms);

// The cached choice for key (loading the CCC_TUNE_CACHE file on first use).
bool tune_lookup(uint64_t key, TuneChoice *out);

// Remember a choice (and append it to the CCC_TUNE_CACHE file, if set).
void tune_store(uint64_t key, TuneChoice choice, float ms);

// Forget every choice held by the process (the file is left alone; it is read
// again on the next lookup).
void tune_clear();

}  // namespace ccc
