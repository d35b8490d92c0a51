// Rollout kernels of the two planar 3-link arms (every layout and placement).
#include "mppi_rollout.cuh"

namespace mppi {
int launch_rollout_na3(int mode, const RolloutArgs& a, int spc, cudaStream_t s) {
    return dispatch_rollout<3>(mode, a, spc, s);
}
int choose_spc_na3(int lps, int K, int unom_floats) { return choose_spc<3>(lps, K, unom_floats); }
MPPI_BOUNDS_READER(bounds_word_rollout3)
}  // namespace mppi
