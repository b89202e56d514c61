// fc_update_ext.cu -- the one-CTA-per-patch fused update with the optional
// parts of the method compiled in: the T2 transverse variant (the limited
// second-order corrections split transversely with the fluctuations,
// LeVeque 1997) and the Harten-Hyman entropy fix of transonic rarefactions.
// A separate translation unit, so that the plain kernels keep their register
// budget and the library's translation units compile in parallel.
#include "fc_update.cuh"

namespace fc {

template <typename T, int M, int EQ, int V>
static int launch_ext_t(const Env<T> &e, List l, int ksub, int fine_acc, cudaStream_t s)
{
    using Lay = UpdLayout<T, M, EQ>;
    constexpr int NT = UpdCfg<M, V>::NT;
    static bool configured = false;
    if (!configured) {
        cudaError_t err = cudaFuncSetAttribute(k_update<T, M, EQ, NT, true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Lay::bytes);
        if (err != cudaSuccess) return cuda_status(err, "cudaFuncSetAttribute(k_update)");
        configured = true;
    }
    if (l.count <= 0) return FC_OK;
    FC_CUDA(launch_pdl(k_update<T, M, EQ, NT, true>, l.count, NT, Lay::bytes, s, e, l.idx, l.count, ksub, fine_acc));
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

template <typename T, int EQ>
static int launch_ext_eq(const Env<T> &e, List l, int ksub, int fine_acc, int variant, cudaStream_t s)
{
    const int v = variant & 1;
    if (e.m == 8) return v ? launch_ext_t<T, 8, EQ, 1>(e, l, ksub, fine_acc, s) : launch_ext_t<T, 8, EQ, 0>(e, l, ksub, fine_acc, s);
    if (e.m == 16) return v ? launch_ext_t<T, 16, EQ, 1>(e, l, ksub, fine_acc, s) : launch_ext_t<T, 16, EQ, 0>(e, l, ksub, fine_acc, s);
    if constexpr (sizeof(T) == 4 || EQ != FC_EQ_SWE)
        if (e.m == 32) return v ? launch_ext_t<T, 32, EQ, 1>(e, l, ksub, fine_acc, s) : launch_ext_t<T, 32, EQ, 0>(e, l, ksub, fine_acc, s);
    set_error("unsupported patch size %d for this precision / equation", e.m);
    return FC_ERR_UNIMPLEMENTED;
}

template <typename T>
int launch_update_ext(const Env<T> &e, List l, int ksub, int fine_acc, int variant, cudaStream_t s)
{
    if (is_sphere_conn(e.conn) || variant < 0 || variant > 1) {
        set_error("T2 and the entropy fix run on the square with launch variants 0 and 1");
        return FC_ERR_INVALID_ARG;
    }
    if (e.eq == FC_EQ_SWE) return launch_ext_eq<T, FC_EQ_SWE>(e, l, ksub, fine_acc, variant, s);
    return launch_ext_eq<T, FC_EQ_ADV>(e, l, ksub, fine_acc, variant, s);
}

template int launch_update_ext<float>(const Env<float> &, List, int, int, int, cudaStream_t);
template int launch_update_ext<double>(const Env<double> &, List, int, int, int, cudaStream_t);

}  // namespace fc
