// Rollout kernels of the two 7-joint arms (every layout and placement).
#include "mppi_rollout.cuh"

namespace mppi {
int launch_rollout_na7(int mode, const RolloutArgs& a, int spc, cudaStream_t s) {
    return dispatch_rollout<7>(mode, a, spc, s);
}
int choose_spc_na7(int lps, int K, int unom_floats) { return choose_spc<7>(lps, K, unom_floats); }
MPPI_BOUNDS_READER(bounds_word_rollout7)
}  // namespace mppi
