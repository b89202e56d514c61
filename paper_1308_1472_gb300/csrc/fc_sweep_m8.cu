// fc_sweep_m8.cu -- row-sweep kernels for 8 x 8 patches.
#include "fc_sweep.cuh"

namespace fc {
template int launch_sweep_m<float, 8>(const Env<float> &, List, int, int, cudaStream_t);
template int launch_sweep_m<double, 8>(const Env<double> &, List, int, int, cudaStream_t);
}  // namespace fc
