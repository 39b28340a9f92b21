// Host-side helpers shared by the single-box and the batch entry points.
#pragma once

#include <string>

#include "lbm_tau1.h"

namespace lbm {

// Message returned by lbm_tau1_last_error(NULL) (the calling thread's last failed create).
void set_create_error(const std::string& msg);

// lbm_tau1_stats from the RED_FIELDS raw sums of a reduction; LBM_EDIVERGED
// when a fluid node is non-finite or max |u + g/2| > 0.3.
lbm_status fill_stats(const double* raw, int64_t n_nodes, const double g[3], int64_t step, lbm_tau1_stats* out);

// Autotune cache (tune_cache.cu): a JSON file of chosen variants by key; an
// empty or NULL path turns it off.
void tune_cache_set_path(const char* path);
bool tune_cache_lookup(const std::string& key, int* variant, double* ms);
void tune_cache_store(const std::string& key, int variant, double ms);

}  // namespace lbm
