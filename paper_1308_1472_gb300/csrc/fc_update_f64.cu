// fc_update_f64.cu -- the fused patch update in FP64.
#include "fc_update_launch.cuh"

namespace fc {
template int launch_update<double>(const Env<double> &, List, int, int, int, cudaStream_t);
}  // namespace fc
