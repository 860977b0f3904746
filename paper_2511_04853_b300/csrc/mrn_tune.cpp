// Launch-shape cache consulted by every conversion (filled by mrn_autotune).
#include <mutex>
#include <unordered_map>

#include "mrn_internal.h"

namespace mrn {

namespace {
std::mutex g_tune_mu;
std::unordered_map<uint64_t, LaunchShape> g_tune_cache;
}  // namespace

LaunchShape tuned_shape(const ConvPlan& p) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune_cache.find(p.tune_key);
  return it == g_tune_cache.end() ? LaunchShape{} : it->second;
}

void store_tuned_shape(uint64_t key, const LaunchShape& s) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache[key] = s;
}

void clear_tuned_shapes() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
}

}  // namespace mrn

extern "C" int mrn_autotune_clear(void) {
  mrn::clear_tuned_shapes();
  return MRN_OK;
}
