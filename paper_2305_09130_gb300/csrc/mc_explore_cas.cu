// The exploration pass with the CAS-first inserts (MC_PROBE_CAS_FIRST and
// MC_PROBE_CAS_CLEAR), instantiated apart from the split and one-call
// inserts (mc_kernels.cu) so that the two halves compile in parallel.
#include "mc_explore.cuh"

namespace mc {

const void* pick_explore_cas(int key_words, int tile, int rule, int scheme) {
  if (scheme == MC_PROBE_CAS_FIRST) {
    if (key_words == 1) return pick_rule<uint64_t, MC_PROBE_CAS_FIRST>(tile, rule);
    if (key_words == 2) return pick_rule<u128, MC_PROBE_CAS_FIRST>(tile, rule);
  }
  if (scheme == MC_PROBE_CAS_CLEAR) {
    if (key_words == 1) return pick_rule<uint64_t, MC_PROBE_CAS_CLEAR>(tile, rule);
    if (key_words == 2) return pick_rule<u128, MC_PROBE_CAS_CLEAR>(tile, rule);
  }
  return nullptr;
}

}  // namespace mc
