// ulp_autotune.cu -- picks the warp-tile height and resident blocks per SM of
// the persistent solvers for a given set of map sizes by timing short bounded
// solves of the caller's own maps (CUDA events around each solver launch).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ulp_host.h"

using namespace ulp;

extern "C" int ulp_autotune(int n, const int* H, const int* W, const ulp_map* maps, int precond, int precision,
                            int iters, const char* cache_path, ulp_options* best) {
  if (n < 1 || !H || !W || !maps || !best) return set_error(ULP_ERR_INVALID, "ulp_autotune: null argument");
  if (iters <= 0) iters = 40;
  ulp_options base;
  ulp_options_default(&base);
  base.precision = precision;
  base.profile = 1;
  base.outer_tol = 0.0;
  // candidate tile heights around "one tile per resident warp"
  int nsm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return set_error(ULP_ERR_CUDA, "ulp_autotune: no device");
  const int occ = solver_blocks_per_sm();
  std::vector<int> rows;
  for (int bps = 1; bps <= occ; ++bps) {
    const int r0 = default_tile_rows(n, H, W, nsm * bps * kWarps);
    for (int r : {r0 / 2, r0, 2 * r0, 8, 16, 32, 64})
      if (r >= 4 && r <= 64 && std::find(rows.begin(), rows.end(), r) == rows.end()) rows.push_back(r);
  }
  double best_us = 1e30;
  int best_r = 0, best_b = 0;
  std::vector<ulp_stats> st(n);
  for (int bps = 1; bps <= occ; ++bps) {
    for (int r : rows) {
      ulp_options o = base;
      o.tile_rows = r;
      o.blocks_per_sm = bps;
      ulp_plan p = nullptr;
      if (ulp_plan_create_batched(n, H, W, &o, &p) != ULP_OK) continue;
      // warm-up, then the timed call
      int rc = ulp_unwrap_batched(p, maps, precond, 1e-30, 1, iters, nullptr, st.data());
      ulp_counters c;
      ulp_plan_counters(p, 1, &c);
      rc = ulp_unwrap_batched(p, maps, precond, 1e-30, 1, iters, nullptr, st.data());
      if (rc >= 0 && ulp_plan_counters(p, 1, &c) == ULP_OK && c.timed_launches > 0) {
        const double us = 1e3 * c.solver_ms;
        if (us < best_us) {
          best_us = us;
          best_r = r;
          best_b = bps;
        }
      }
      ulp_plan_destroy(p);
    }
  }
  if (!best_r) return set_error(ULP_ERR_CUDA, "ulp_autotune: no candidate ran");
  *best = base;
  best->profile = 0;
  best->tile_rows = best_r;
  best->blocks_per_sm = best_b;
  if (cache_path && *cache_path) {
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    unsigned long long h = 1469598103934665603ull;  // FNV-1a over the sizes
    for (int m = 0; m < n; ++m) {
      h = (h ^ (unsigned)H[m]) * 1099511628211ull;
      h = (h ^ (unsigned)W[m]) * 1099511628211ull;
    }
    if (FILE* f = std::fopen(cache_path, "a")) {
      std::fprintf(f,
                   "{\"gpu\": \"%s\", \"precision\": %d, \"precond\": %d, \"maps\": %d, \"sizes_hash\": \"%016llx\", "
                   "\"tile_rows\": %d, \"blocks_per_sm\": %d, \"us_per_call\": %.1f, \"iterations\": %d}\n",
                   prop.name, precision, precond, n, h, best_r, best_b, best_us, iters);
      std::fclose(f);
    }
  }
  return ULP_OK;
}
