// fc_noalloc.cu -- conservation sums for callers that cannot allocate device
// memory.
//
// Some callers of this library may not call cudaMalloc (or any allocating
// routine): for example a process that reserves its whole device-memory budget
// up front and hands out fixed buffers, or code that runs where an allocation
// would synchronise the device or fail under memory pressure.  For them this
// file provides fc_conservation_sums_noalloc: per-patch partial sums weighted
// by the cell areas of the unit square (the sums of fc_conservation_sums on the
// square and periodic square; the spheres' mapped areas are not known here)
// and a fixed-order final reduction, with the per-patch
// partials kept in a file-scope device array instead of library-allocated
// memory.  The caller passes the fields and levels (device memory) and a device
// output array.
//
// Scratch: g_partials holds kMaxPatches x kMaxFields doubles (3 MiB) on every
// GPU that loads this library, for as long as the library stays loaded.  All
// calls on a device share it; every call writes each partial it later reads,
// so nothing needs clearing between calls.  Calls whose GPU work overlaps in
// time (different streams, or different host threads on one device) race on
// the shared array and must not be issued that way.
#include <mutex>

#include "fc_internal.cuh"

#define FC_NOALLOC_MAX_PATCHES 131072
#define FC_NOALLOC_MAX_FIELDS 3

// the scratch: per-patch partial sums, FP64
static __device__ __align__(256) double g_partials[FC_NOALLOC_MAX_PATCHES * FC_NOALLOC_MAX_FIELDS];

namespace {

constexpr int64_t kMaxPatches = FC_NOALLOC_MAX_PATCHES;
constexpr int kMaxFields = FC_NOALLOC_MAX_FIELDS;
constexpr int kMaxDevices = 64;

// device address of g_partials, looked up once per device with that device
// current (host code only has a host-side stand-in for the symbol)
std::mutex g_mu;
double *g_addr[kMaxDevices] = {nullptr};

int partials_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fc::cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        fc::set_error("device ordinal %d beyond %d", dev, kMaxDevices);
        return FC_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return fc::cuda_status(e, "cudaGetSymbolAddress(g_partials)");
        g_addr[dev] = (double *)p;
    }
    *out = g_addr[dev];
    return FC_OK;
}

// per-patch sums of every field times the cell area; q is [leaf][field][m*m]
template <typename T>
__global__ void k_partials_noalloc(const T *q, const int *level, int n, int m, int F, double *part)
{
    __shared__ double red[kMaxFields][32];
    int p = blockIdx.x;
    if (p >= n) return;
    int mm = m * m;
    double acc[kMaxFields] = {0.0, 0.0, 0.0};
    for (int c = threadIdx.x; c < mm; c += blockDim.x)
        for (int f = 0; f < F; ++f) acc[f] += (double)q[((size_t)p * F + f) * mm + c];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int f = 0; f < F; ++f) {
        double v = acc[f];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[f][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < F) {
        double v = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) v += red[threadIdx.x][k];
        double dx = 1.0 / ((double)(1 << level[p]) * m);
        part[(size_t)p * F + threadIdx.x] = v * (dx * dx);
    }
}

// fixed-order reduction of the partials (one block)
__global__ void k_final_noalloc(const double *part, int n, int F, double *out)
{
    __shared__ double red[kMaxFields][1024];
    for (int f = 0; f < F; ++f) {
        double v = 0.0;
        for (int p = threadIdx.x; p < n; p += blockDim.x) v += part[(size_t)p * F + f];
        red[f][threadIdx.x] = v;
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int f = 0; f < F; ++f) red[f][threadIdx.x] += red[f][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < F) out[threadIdx.x] = red[threadIdx.x][0];
}

}  // namespace

extern "C" int fc_conservation_sums_noalloc(const void *q, const int32_t *level, int64_t n, int m, int nfields,
                                            int precision, double *sums, void *stream)
{
    if (!q || !level || !sums || n <= 0 || !(m == 8 || m == 16 || m == 32) ||
        (precision != FC_FP64 && precision != FC_FP32)) {
        fc::set_error("fc_conservation_sums_noalloc: invalid argument");
        return FC_ERR_INVALID_ARG;
    }
    if (n > kMaxPatches || nfields < 1 || nfields > kMaxFields) {
        fc::set_error("fc_conservation_sums_noalloc: %lld patches x %d fields exceeds the static scratch "
                      "of %lld patches x %d fields",
                      (long long)n, nfields, (long long)kMaxPatches, kMaxFields);
        return FC_ERR_CAPACITY;
    }
    double *part = nullptr;
    FC_TRY(partials_address(&part));
    cudaStream_t s = (cudaStream_t)stream;
    if (precision == FC_FP64)
        k_partials_noalloc<double><<<(int)n, 256, 0, s>>>((const double *)q, level, (int)n, m, nfields, part);
    else
        k_partials_noalloc<float><<<(int)n, 256, 0, s>>>((const float *)q, level, (int)n, m, nfields, part);
    FC_CUDA(cudaGetLastError());
    k_final_noalloc<<<1, 1024, 0, s>>>(part, (int)n, nfields, sums);
    FC_CUDA(cudaGetLastError());
    FC_CUDA(cudaStreamSynchronize(s));
    return FC_OK;
}
