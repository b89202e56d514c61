// fc_sweep_m16.cu -- row-sweep kernels for 16 x 16 patches.
#include "fc_sweep.cuh"

namespace fc {
template int launch_sweep_m<float, 16>(const Env<float> &, List, int, int, cudaStream_t);
template int launch_sweep_m<double, 16>(const Env<double> &, List, int, int, cudaStream_t);
}  // namespace fc
