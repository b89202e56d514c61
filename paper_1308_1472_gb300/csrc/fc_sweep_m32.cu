// fc_sweep_m32.cu -- row-sweep kernels for 32 x 32 patches.
#include "fc_sweep.cuh"

namespace fc {
template int launch_sweep_m<float, 32>(const Env<float> &, List, int, int, cudaStream_t);
}  // namespace fc
