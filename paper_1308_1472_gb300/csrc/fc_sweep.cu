// fc_sweep.cu -- dispatch of the row-sweep update by patch size; the
// kernels (fc_sweep.cuh) are instantiated in fc_sweep_m8.cu, fc_sweep_m16.cu
// and fc_sweep_m32.cu so that they compile in parallel.
#include "fc_kernels.cuh"

namespace fc {

template <typename T, int M>
int launch_sweep_m(const Env<T> &e, List l, int fine_acc, int k, cudaStream_t s);

template <typename T>
int launch_sweep(const Env<T> &e, List l, int fine_acc, int k, cudaStream_t s)
{
    if (e.eq != FC_EQ_SWE || e.conn == FC_CONN_SPHERE || e.t2 || e.efix || k < 0 || k > 2) {
        set_error("the row-sweep update is for shallow water on the square, T1 without entropy fix");
        return FC_ERR_INVALID_ARG;
    }
    if (e.m == 8) return launch_sweep_m<T, 8>(e, l, fine_acc, k, s);
    if (e.m == 16) return launch_sweep_m<T, 16>(e, l, fine_acc, k, s);
    if constexpr (sizeof(T) == 4)
        if (e.m == 32) return launch_sweep_m<T, 32>(e, l, fine_acc, k, s);
    set_error("unsupported patch size %d for this precision / equation", e.m);
    return FC_ERR_UNIMPLEMENTED;
}

template int launch_sweep<float>(const Env<float> &, List, int, int, cudaStream_t);
template int launch_sweep<double>(const Env<double> &, List, int, int, cudaStream_t);

}  // namespace fc
