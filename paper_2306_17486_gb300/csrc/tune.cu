// Launch-shape tuning table: values that override the launch heuristics of a kernel
// family for one layer height and batch, set by the autotuner (or left empty: the
// heuristics rule).
#include <map>
#include <mutex>
#include <tuple>

#include "problem.h"

namespace {

std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;   // (knob, layer height, batch) -> value

}  // namespace

namespace helm {

int tune_get(int knob, int height, int batch) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const std::tuple<int, int, int> keys[3] = {{knob, height, batch}, {knob, height, 0}, {knob, 0, 0}};
  for (const auto& k : keys) {
    auto it = g_tune.find(k);
    if (it != g_tune.end()) return it->second;
  }
  return 0;
}

}  // namespace helm

extern "C" {

int helm_tune_set(int knob, int height, int batch, int value) {
  if (knob < 0 || knob >= HELM_TUNE_KNOBS || height < 0 || batch < 0 || value < 0 || (height == 0 && batch != 0)) {
    helm::set_error("helm_tune_set: knob in [0, %d), height, batch, value >= 0, batch 0 when height is 0",
                    HELM_TUNE_KNOBS);
    return HELM_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (value == 0)
    g_tune.erase({knob, height, batch});
  else
    g_tune[{knob, height, batch}] = value;
  return HELM_OK;
}

int helm_tune_get(int knob, int height, int batch, int* value) {
  if (knob < 0 || knob >= HELM_TUNE_KNOBS || height < 0 || batch < 0 || !value) {
    helm::set_error("helm_tune_get: invalid argument");
    return HELM_EINVAL;
  }
  *value = helm::tune_get(knob, height, batch);
  return HELM_OK;
}

int helm_tune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
  return HELM_OK;
}

}  // extern "C"
