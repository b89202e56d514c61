// fc_internal.cuh -- internals of libfc shared by its translation units.
//
// Data layout in HBM (one context):
//   leaves     int32 tree[n], level[n], x[n], y[n]  (SFC order)
//   keys       uint64 key[n] = tree << 60 | Morton(X, Y), X = x << (30 - level)
//   nbr        int32 [n][8][4] {kind, id0, id1, orient}
//   state      T q[3][F][n][m*m]  -- three buffers per cell: the start of the
//              coarse step and two scratch buffers for its substeps, so that a
//              retaken step and the time interpolation need no copies
//   tiles      T gr[ntile][F][(m+4)^2] -- complete ghost-filled tiles of the
//              patches that have a finer neighbour (sources of coarse-to-fine
//              interpolation), refilled at every substep time
//   registers  double reg[nslot][m][F] -- effective fluxes * dt through
//              coarse-fine sides (Sec. 4 fine-to-coarse correction)
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "../../include/fc.h"

namespace fc {

// the mapped spheres (six-tree cubed sphere, two-tree sphere): capacity-form
// scalar advection on per-patch geometry
__host__ __device__ inline bool is_sphere_conn(int conn) { return conn == FC_CONN_SPHERE || conn == FC_CONN_PILLOW; }

constexpr int kMaxBits = 30;           // Morton bits per axis
constexpr int kMaxLevels = 16;         // levels 0..15
constexpr int kTreeShift = 60;

// ---------------------------------------------------------------------------
// error reporting (thread-local message, status codes)
void set_error(const char *fmt, ...);
int cuda_status(cudaError_t e, const char *what);
#define FC_CUDA(call)                                                              \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return ::fc::cuda_status(e_, #call);                \
    } while (0)
// named range around a host-side phase of an entry point (NVTX; free when
// no profiling tool is attached)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

#define FC_TRY(call)                                                               \
    do {                                                                           \
        int r_ = (call);                                                           \
        if (r_ != FC_OK) return r_;                                                \
    } while (0)

// ---------------------------------------------------------------------------
// Programmatic dependent launch between the kernels of a step: a kernel
// launched with launch_pdl may be scheduled while the kernels it follows are
// still running.  It calls pdl_trigger() first, which lets the kernels after
// it be scheduled in turn, and pdl_wait() before it reads or writes anything
// that a kernel of the step writes (states, tiles, registers, step control),
// which waits until the kernels it follows have completed and their memory
// operations are visible.  Before the wait a kernel reads only the
// forest's tables (leaves, neighbour records, lists, slot maps), which no
// kernel of a step writes, so the order of the step is that of plain
// launches; what overlaps is the launch of the next grid and its reads of
// the tables.  pdl_begin() is both at once.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_begin()
{
    pdl_trigger();
    pdl_wait();
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args)
{
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Morton keys: bit spreading with masks (x in the even bits)
__host__ __device__ inline uint64_t spread_bits(uint32_t v)
{
    uint64_t x = v & 0x3fffffffu;
    x = (x | (x << 16)) & 0x0000ffff0000ffffULL;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffULL;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0fULL;
    x = (x | (x << 2)) & 0x3333333333333333ULL;
    x = (x | (x << 1)) & 0x5555555555555555ULL;
    return x;
}
__host__ __device__ inline uint32_t compact_bits(uint64_t x)
{
    x &= 0x5555555555555555ULL;
    x = (x | (x >> 1)) & 0x3333333333333333ULL;
    x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0fULL;
    x = (x | (x >> 4)) & 0x00ff00ff00ff00ffULL;
    x = (x | (x >> 8)) & 0x0000ffff0000ffffULL;
    x = (x | (x >> 16)) & 0x00000000ffffffffULL;
    return (uint32_t)x;
}
__host__ __device__ inline uint64_t leaf_key(int tree, int level, int x, int y)
{
    int s = kMaxBits - level;
    return ((uint64_t)tree << kTreeShift) | spread_bits((uint32_t)x << s) | (spread_bits((uint32_t)y << s) << 1);
}

// ---------------------------------------------------------------------------
// forest as seen by kernels
struct ForestDev {
    int n;
    int conn;
    const int *ctab;      // FC_CONN_TABLE: [ntrees][4][3] {tree, side, reversed}
    int ntrees;
    const int *tree, *level, *x, *y;
    const uint64_t *key;
    const int *nbr;       // [n][8][4]
};

// ---------------------------------------------------------------------------
// device step state (lives in device memory; advanced by the step-control
// kernel so that a sequence of steps can be launched without host round trips)
struct StepCtl {
    double dt;              // step being attempted (coarse step under subcycling)
    double t;               // time of the last accepted step
    double dt_fixed;        // > 0: fixed step
    double cfl;
    double last_dt, last_courant, next_dt;
    unsigned long long smax_bits[kMaxLevels];  // per-level max |s|, as double bits
    double dtl_d[kMaxLevels], dtdx_d[kMaxLevels];   // per-level step and dt/dx of the attempt
    float dtl_f[kMaxLevels], dtdx_f[kMaxLevels];
    int start_buf[kMaxLevels];                  // buffer holding each level's state
    int attempts;           // failed attempts of the current step
    int accepted;           // accepted steps since the counter was reset
    int retries;            // total retaken attempts
    int cfl_error;          // sticky: a step was accepted with Courant > 1
    int dry_error;          // sticky: h <= 0 met
    int nonfinite_error;
    int index_error;        // sticky: a neighbour lookup fell outside its patch
};

// buffer written by substep k (1-based) of a level that started the coarse
// step in buffer s, and the buffer that substep reads
__host__ __device__ inline int buf_out(int s, int k) { return (s + 1 + ((k - 1) & 1)) % 3; }
__host__ __device__ inline int buf_in(int s, int k) { return k == 1 ? s : (s + 1 + ((k - 2) & 1)) % 3; }

}  // namespace fc
