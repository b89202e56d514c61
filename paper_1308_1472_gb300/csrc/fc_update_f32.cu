// fc_update_f32.cu -- the fused patch update in FP32.
#include "fc_update_launch.cuh"

namespace fc {
template int launch_update<float>(const Env<float> &, List, int, int, int, cudaStream_t);
}  // namespace fc
