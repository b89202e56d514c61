// fc_cnn.cu -- learned refinement tagger: forward, backward and Adam kernels.
//
// The paper has no learned component; this network stands in for the Sec. 5
// tagging criterion and predicts its refine / coarsen flags several steps
// ahead.  Network: 3x3 valid convolutions 3 -> 16 -> 16 -> 2 with ReLU after
// the first two, global max pool per output channel -> two logits.  Loss:
// binary cross-entropy with logits, summed over the two outputs, mean over
// samples.
//
// Precision: in BF16 mode the weights, the input and both hidden activations
// are rounded to BF16 before they enter a product; every sum is accumulated in
// FP32; the master weights and Adam moments stay FP32.  With bf16 = 0 the same
// kernels run on FP32 values (used to check the gradients tightly).  BF16
// inference (fc_cnn_forward with bf16 = 1) runs on the tensor cores (namespace
// tc below); training uses the scalar kernels in both modes.
//
// One CTA per sample at a time (grid-stride over samples); the sample, the
// activations and the CTA's gradient partials live in shared memory; the
// per-CTA partials are reduced in a fixed order by a second kernel, so the
// gradient does not depend on scheduling.
#include <cuda_bf16.h>

#include "fc_internal.cuh"

namespace fc {
namespace cnn {

constexpr int C1 = 16, C2 = 16, C3 = 2;
constexpr int NW1 = C1 * 3 * 9, NB1 = C1, NW2 = C2 * C1 * 9, NB2 = C2, NW3 = C3 * C2 * 9, NB3 = C3;
constexpr int NPARAM = NW1 + NB1 + NW2 + NB2 + NW3 + NB3;   // 3058
constexpr int OW1 = 0, OB1 = OW1 + NW1, OW2 = OB1 + NB1, OB2 = OW2 + NW2, OW3 = OB2 + NB2, OB3 = OW3 + NW3;
constexpr int NT = 256;
constexpr int MAXS = 36;

__device__ __forceinline__ float rnd(float v, int bf16) { return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v; }

// valid 3x3 convolution of Ci channels of width S into Co channels
__device__ void conv_fwd(const float *x, int Ci, int S, const float *w, const float *b, int Co, float *y, bool relu,
                         int bf16)
{
    int So = S - 2, np = So * So;
    for (int t = threadIdx.x; t < Co * np; t += blockDim.x) {
        int o = t / np, pos = t - o * np, r = pos / So, c = pos - r * So;
        float acc = b[o];
        const float *wo = w + o * Ci * 9;
        for (int i = 0; i < Ci; ++i) {
            const float *xi = x + (i * S + r) * S + c;
            const float *wi = wo + i * 9;
            acc += wi[0] * xi[0] + wi[1] * xi[1] + wi[2] * xi[2];
            acc += wi[3] * xi[S] + wi[4] * xi[S + 1] + wi[5] * xi[S + 2];
            acc += wi[6] * xi[2 * S] + wi[7] * xi[2 * S + 1] + wi[8] * xi[2 * S + 2];
        }
        if (relu) acc = acc > 0.f ? acc : 0.f;
        y[t] = relu ? rnd(acc, bf16) : acc;
    }
}

struct Smem {
    float *w, *x, *a1, *a2, *z, *d2, *d1, *g;
    int *arg;
};

// shared-memory layout: forward part {w, x, a1, a2, z, arg[16]}, then the
// training part {d2, d1, g} that only the backward kernel allocates
__device__ Smem carve(float *base, int S)
{
    Smem s;
    int S1 = S - 2, S2 = S - 4, S3 = S - 6;
    s.w = base;
    s.x = s.w + NPARAM;
    s.a1 = s.x + 3 * S * S;
    s.a2 = s.a1 + C1 * S1 * S1;
    s.z = s.a2 + C2 * S2 * S2;
    s.arg = (int *)(s.z + C3 * S3 * S3);
    s.d2 = (float *)(s.arg + 16);
    s.d1 = s.d2 + C2 * S2 * S2;
    s.g = s.d1 + C1 * S1 * S1;
    return s;
}

__host__ __device__ inline size_t smem_bytes(int S, bool train)
{
    int S1 = S - 2, S2 = S - 4, S3 = S - 6;
    size_t f = NPARAM + 3 * S * S + C1 * S1 * S1 + C2 * S2 * S2 + C3 * S3 * S3 + 16;   // 16 ints for arg
    if (train) f += C2 * S2 * S2 + C1 * S1 * S1 + NPARAM;
    return f * sizeof(float);
}

// forward of one sample already staged in s.x; logits into lg[2], argmax into s.arg
__device__ void forward_one(const Smem &s, int S, int bf16, float *lg)
{
    int S1 = S - 2, S2 = S - 4, S3 = S - 6;
    conv_fwd(s.x, 3, S, s.w + OW1, s.w + OB1, C1, s.a1, true, bf16);
    __syncthreads();
    conv_fwd(s.a1, C1, S1, s.w + OW2, s.w + OB2, C2, s.a2, true, bf16);
    __syncthreads();
    conv_fwd(s.a2, C2, S2, s.w + OW3, s.w + OB3, C3, s.z, false, bf16);
    __syncthreads();
    // global max per channel (first maximum in raster order), one warp per channel
    int wp = threadIdx.x >> 5, lane = threadIdx.x & 31, n3 = S3 * S3;
    if (wp < C3) {
        float best = -3.0e38f;
        int bi = 0x7fffffff;
        for (int k = lane; k < n3; k += 32) {
            float v = s.z[wp * n3 + k];
            if (v > best || (v == best && k < bi)) { best = v; bi = k; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            float ob = __shfl_xor_sync(0xffffffffu, best, o);
            int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) {
            // non-finite logits leave no maximum: fall back to position 0
            s.arg[wp] = (bi >= 0 && bi < n3) ? bi : 0;
            lg[wp] = best;
        }
    }
    __syncthreads();
}

__device__ void stage(const Smem &s, const float *w, const float *x, int S, int bf16, bool weights)
{
    if (weights)
        for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) {
            bool bias = (k >= OB1 && k < OW2) || (k >= OB2 && k < OW3) || k >= OB3;
            s.w[k] = bias ? w[k] : rnd(w[k], bf16);       // biases are added in FP32
        }
    for (int k = threadIdx.x; k < 3 * S * S; k += blockDim.x) s.x[k] = rnd(x[k], bf16);
}

__global__ void k_cnn_forward(int n, int S, const float *w, const float *x, float *logits, int bf16)
{
    extern __shared__ __align__(16) float sm[];
    Smem s = carve(sm, S);
    __shared__ float lg[C3];
    bool first = true;
    for (int smp = blockIdx.x; smp < n; smp += gridDim.x) {
        stage(s, w, x + (size_t)smp * 3 * S * S, S, bf16, first);
        first = false;
        __syncthreads();
        forward_one(s, S, bf16, lg);
        if (threadIdx.x < C3) logits[2 * smp + threadIdx.x] = lg[threadIdx.x];
        __syncthreads();
    }
}

// gradient of the loss of the samples a CTA processes, into part[block][NPARAM]
// and the summed loss into lossp[block]
__global__ void k_cnn_backward(int n, int S, const float *w, const float *x, const float *targets, float *part,
                               float *lossp, int bf16)
{
    extern __shared__ __align__(16) float sm[];
    Smem s = carve(sm, S);
    __shared__ float lg[C3], dz[C3];
    __shared__ float lsum;
    int S1 = S - 2, S2 = S - 4, S3 = S - 6;
    int n1 = S1 * S1, n2 = S2 * S2;
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) s.g[k] = 0.f;
    if (threadIdx.x == 0) lsum = 0.f;
    bool first = true;
    for (int smp = blockIdx.x; smp < n; smp += gridDim.x) {
        stage(s, w, x + (size_t)smp * 3 * S * S, S, bf16, first);
        first = false;
        __syncthreads();
        forward_one(s, S, bf16, lg);
        if (threadIdx.x < C3) {
            float z = lg[threadIdx.x], y = targets[2 * smp + threadIdx.x];
            float sig = 1.f / (1.f + expf(-z));
            dz[threadIdx.x] = (sig - y) / (float)n;
            float l = fmaxf(z, 0.f) - y * z + log1pf(expf(-fabsf(z)));
            atomicAdd(&lsum, l / (float)n);
        }
        __syncthreads();
        // layer 3: only the argmax positions carry gradient
        for (int k = threadIdx.x; k < C2 * n2; k += blockDim.x) s.d2[k] = 0.f;
        __syncthreads();
        for (int k = threadIdx.x; k < C3 * C2 * 9; k += blockDim.x) {
            int o = k / (C2 * 9), rem = k - o * C2 * 9, i = rem / 9, t = rem - i * 9, ky = t / 3, kx = t - ky * 3;
            int p = s.arg[o], r = p / S3 + ky, c = p - (p / S3) * S3 + kx;
            float a = s.a2[(i * S2 + r) * S2 + c];
            s.g[OW3 + k] += dz[o] * a;
        }
        if (threadIdx.x < C3) s.g[OB3 + threadIdx.x] += dz[threadIdx.x];
        // d a2 = sum over the two argmax windows (serial per channel: disjoint
        // only when the windows do not overlap, so one thread per channel i)
        for (int i = threadIdx.x; i < C2; i += blockDim.x)
            for (int o = 0; o < C3; ++o) {
                int p = s.arg[o], r0 = p / S3, c0 = p - r0 * S3;
                for (int t = 0; t < 9; ++t) {
                    int ky = t / 3, kx = t - ky * 3;
                    s.d2[(i * S2 + r0 + ky) * S2 + c0 + kx] += dz[o] * s.w[OW3 + (o * C2 + i) * 9 + t];
                }
            }
        __syncthreads();
        for (int k = threadIdx.x; k < C2 * n2; k += blockDim.x)
            if (!(s.a2[k] > 0.f)) s.d2[k] = 0.f;
        __syncthreads();
        // layer 2: weights, bias, and d a1 (transposed convolution)
        for (int k = threadIdx.x; k < NW2; k += blockDim.x) {
            int o = k / (C1 * 9), rem = k - o * C1 * 9, i = rem / 9, t = rem - i * 9, ky = t / 3, kx = t - ky * 3;
            const float *d = s.d2 + o * n2;
            const float *a = s.a1 + i * n1;
            float acc = 0.f;
            for (int r = 0; r < S2; ++r)
                for (int c = 0; c < S2; ++c) {
                    float dv = d[r * S2 + c];
                    if (dv != 0.f) acc += dv * a[(r + ky) * S1 + c + kx];
                }
            s.g[OW2 + k] += acc;
        }
        for (int o = threadIdx.x; o < C2; o += blockDim.x) {
            float acc = 0.f;
            for (int k = 0; k < n2; ++k) acc += s.d2[o * n2 + k];
            s.g[OB2 + o] += acc;
        }
        for (int k = threadIdx.x; k < C1 * n1; k += blockDim.x) {
            int i = k / n1, pos = k - i * n1, y = pos / S1, xx = pos - y * S1;
            float acc = 0.f;
            if (s.a1[k] > 0.f) {
                for (int o = 0; o < C2; ++o)
                    for (int ky = 0; ky < 3; ++ky) {
                        int r = y - ky;
                        if (r < 0 || r >= S2) continue;
                        for (int kx = 0; kx < 3; ++kx) {
                            int c = xx - kx;
                            if (c < 0 || c >= S2) continue;
                            acc += s.d2[(o * S2 + r) * S2 + c] * s.w[OW2 + ((o * C1 + i) * 3 + ky) * 3 + kx];
                        }
                    }
            }
            s.d1[k] = acc;
        }
        __syncthreads();
        // layer 1: weights and bias
        for (int k = threadIdx.x; k < NW1; k += blockDim.x) {
            int o = k / 27, rem = k - o * 27, i = rem / 9, t = rem - i * 9, ky = t / 3, kx = t - ky * 3;
            const float *d = s.d1 + o * n1;
            const float *a = s.x + i * S * S;
            float acc = 0.f;
            for (int r = 0; r < S1; ++r)
                for (int c = 0; c < S1; ++c) {
                    float dv = d[r * S1 + c];
                    if (dv != 0.f) acc += dv * a[(r + ky) * S + c + kx];
                }
            s.g[OW1 + k] += acc;
        }
        for (int o = threadIdx.x; o < C1; o += blockDim.x) {
            float acc = 0.f;
            for (int k = 0; k < n1; ++k) acc += s.d1[o * n1 + k];
            s.g[OB1 + o] += acc;
        }
        __syncthreads();
    }
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) part[(size_t)blockIdx.x * NPARAM + k] = s.g[k];
    if (threadIdx.x == 0) lossp[blockIdx.x] = lsum;
}

__global__ void k_cnn_reduce(const float *part, const float *lossp, int nb, float *grad, float *loss)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPARAM) {
        float acc = 0.f;
        for (int b = 0; b < nb; ++b) acc += part[(size_t)b * NPARAM + k];
        grad[k] = acc;
    }
    if (k == 0) {
        float l = 0.f;
        for (int b = 0; b < nb; ++b) l += lossp[b];
        *loss = l;
    }
}

__global__ void k_cnn_adam(float *w, const float *g, float *m1, float *m2, float b1t, float b2t, float lr)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float gk = g[k];
    float a = b1 * m1[k] + (1.f - b1) * gk;
    float v = b2 * m2[k] + (1.f - b2) * gk * gk;
    m1[k] = a;
    m2[k] = v;
    float ah = a / (1.f - b1t), vh = v / (1.f - b2t);
    w[k] -= lr * ah / (sqrtf(vh) + eps);
}

inline int grid_for(int n) { int g = n < 304 ? n : 304; return g > 0 ? g : 1; }


// per-block, per-channel sums over network inputs x [n][3][SS] (fixed grid
// and order: deterministic): of x, or with DEV of (x - mean[channel])^2
constexpr int kStatBlocks = 256, kStatThreads = 256;
template <bool DEV>
__global__ void k_chan_sums(long long total, int SS, const float *x, const double *mean, double *part)
{
    __shared__ double red[3][kStatThreads];
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long g = (long long)blockIdx.x * kStatThreads + threadIdx.x; g < total;
         g += (long long)kStatBlocks * kStatThreads) {
        const int c = (int)((g / SS) % 3);
        double v = (double)x[g];
        if (DEV) { v -= mean[c]; v *= v; }
        acc[c] += v;
    }
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = acc[c];
    __syncthreads();
    for (int h = kStatThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < 3) part[(size_t)blockIdx.x * 3 + threadIdx.x] = red[threadIdx.x][0];
}

// the blocks' partial sums in block order, divided by the count per channel
__global__ void k_chan_final(const double *part, double count, double *out)
{
    if (threadIdx.x >= 3 || blockIdx.x) return;
    double s = 0.0;
    for (int b = 0; b < kStatBlocks; ++b) s += part[(size_t)b * 3 + threadIdx.x];
    out[threadIdx.x] = s / count;
}

// the input transform of fc_export_tiles, in place
__global__ void k_normalize(long long total, int SS, float *x, double ref, double s0, double s1, double s2)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const int f = (int)((g / SS) % 3);
    const double v = (double)x[g];
    x[g] = (float)(f == 0 ? (v - ref) * s0 : v * (f == 1 ? s1 : s2));
}

}  // namespace cnn

// ---------------------------------------------------------------------------
// BF16 forward on the tensor cores (tcgen05, accumulators in TMEM).
//
// The three valid 3x3 convolutions are dense contractions: per output
// position, sum over input channels and the nine taps.  Activations live in
// shared memory as BF16 in channel chunks of eight, [chunk][position][8]
// (16 bytes per position and chunk), with positions p = r * S + c over the
// input tile's full width S for every layer ("wide" positions: the columns
// past a layer's valid width hold values no valid output reads).  Then the
// A operand of tap (ky, kx) for output positions p0 .. p0 + 127 is the
// activation buffer itself, started at position p0 + ky * S + kx: in the
// canonical K-major layout without swizzle an 8 x 16-byte core matrix is 8
// consecutive positions of one chunk, the next 8 positions follow 128 bytes
// on (stride byte offset) and the second chunk of 8 channels a whole chunk
// further (leading byte offset).  So each tap is one MMA with M = 128
// positions, N = 16 output channels (the two of the last layer padded with
// zero weights), K = 16 input channels (the three of the first layer padded
// with zeros), and no im2col copy: nine MMAs per 128-position tile, one
// thread issuing them, completion on an mbarrier, then each warp reads its
// 32 TMEM lanes (positions), adds the bias, applies ReLU and rounds to BF16
// into the next buffer, or (last layer) folds the valid positions into the
// per-channel maximum.  Products of BF16 values are exact in FP32 and the
// sums accumulate in FP32, as in the scalar kernels; only the order of the
// sums differs.
namespace tc {

constexpr int NT = 128;                       // one thread per TMEM lane of an M = 128 tile
constexpr uint32_t kTmemCols = 32;            // allocation unit: two accumulators of 16 columns
// instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4
// in bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading (K direction) and
// stride (M / N direction) byte offsets between core matrices, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, int acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(kIdesc), "r"(acc) : "memory");
}
__device__ __forceinline__ void commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}
__device__ __forceinline__ bool try_wait(uint32_t mbar, uint32_t phase)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(ok) : "r"(mbar), "r"(phase) : "memory");
    return ok != 0;
}
// bounded wait for the mbarrier phase; false if it did not complete
__device__ __forceinline__ bool wait_phase(uint32_t mbar, uint32_t phase, long long limit)
{
    for (long long k = 0; k < limit; ++k)
        if (try_wait(mbar, phase)) return true;
    return false;
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    #pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// positions per activation buffer: the 128-position tiles of the first
// layer's rows (S - 2 rows of width S) plus the reach of the last tap
__host__ __device__ inline int npos(int S)
{
    const int t1 = ((S - 2) * S + 127) / 128;
    return (t1 * 128 + 2 * S + 2 + 7) / 8 * 8;
}
constexpr int kSliceBytes = 2 * 2 * 64 * 2;   // [N group][K chunk][8 x 8] BF16 of one tap
__host__ __device__ inline size_t act_bytes(int S) { return (size_t)2 * npos(S) * 16; }
__host__ __device__ inline size_t smem_bytes(int S)
{
    return 3 * act_bytes(S) + 3 * 9 * kSliceBytes + 64 * sizeof(float) + 64;
}

__device__ __forceinline__ uint32_t pack2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// weights of layer (Ci -> Co) as nine tap slices [N group][K chunk][8][8]
// BF16, zero past Ci and Co
__device__ void stage_weights(const float *w, int Ci, int Co, __nv_bfloat16 *sl)
{
    for (int k = threadIdx.x; k < 9 * 256; k += NT) {
        const int s = k >> 8, rem = k & 255, g = rem >> 7, kc = (rem >> 6) & 1, r = (rem >> 3) & 7, kk = rem & 7;
        const int o = 8 * g + r, i = 8 * kc + kk;
        const float v = (o < Co && i < Ci) ? w[(o * Ci + i) * 9 + s] : 0.f;
        sl[k] = __float2bfloat16_rn(v);
    }
}

// one convolution layer: nine tap MMAs per tile of 128 wide positions, into
// two accumulators in turn (TMEM columns 0-15 and 16-31, each with its own
// mbarrier), so the MMAs of tile t + 1 run while the warps read tile t out.
// Returns false if an MMA tile did not complete within the wait limit.
__device__ bool conv_layer(const unsigned char *in, const __nv_bfloat16 *wsl, int S, int tiles, uint32_t tmem,
                           uint32_t mbar0, uint32_t mbar1, uint32_t &phases, long long limit, unsigned char *out,
                           const float *bias, int S3, float *best, int *bidx)
{
    const int NP = npos(S), warp = threadIdx.x >> 5;
    const uint32_t lbo_a = (uint32_t)NP * 16, in_a = saddr(in), w_a = saddr(wsl);
    auto issue = [&](int t) {
        if (threadIdx.x == 0) {
            const uint32_t d = tmem + (uint32_t)(16 * (t & 1));
            #pragma unroll 1
            for (int s = 0; s < 9; ++s) {
                const int sh = t * 128 + (s / 3) * S + (s % 3);
                mma(d, sdesc(in_a + (uint32_t)sh * 16, lbo_a, 128), sdesc(w_a + s * kSliceBytes, 128, 256), s > 0);
            }
            commit((t & 1) ? mbar1 : mbar0);
        }
    };
    bool ok = true;
    fence_after();
    issue(0);
    for (int t = 0; t < tiles; ++t) {
        // the other accumulator was read out before the barrier that ended
        // the previous tile
        fence_after();
        if (t + 1 < tiles) issue(t + 1);
        const int b = t & 1;
        const uint32_t mb = b ? mbar1 : mbar0, mo = b ? mbar0 : mbar1;
        if (!wait_phase(mb, (phases >> b) & 1u, limit)) {
            // give the MMAs in flight a last bounded chance to finish before
            // the accumulators are freed, and report the timeout
            wait_phase(mb, (phases >> b) & 1u, 1ll << 22);
            if (t + 1 < tiles) wait_phase(mo, (phases >> (b ^ 1)) & 1u, 1ll << 22);
            ok = false;
        }
        phases ^= 1u << b;
        fence_after();
        if (__syncthreads_or(!ok)) return false;
        float v[16];
        ld16(tmem + (uint32_t)(16 * b) + ((uint32_t)(32 * warp) << 16), v);
        const int p = t * 128 + (int)threadIdx.x;
        if (out) {
            uint4 lo, hi;
            float a[16];
            #pragma unroll
            for (int k = 0; k < 16; ++k) a[k] = fmaxf(v[k] + bias[k], 0.f);
            lo.x = pack2(a[0], a[1]); lo.y = pack2(a[2], a[3]); lo.z = pack2(a[4], a[5]); lo.w = pack2(a[6], a[7]);
            hi.x = pack2(a[8], a[9]); hi.y = pack2(a[10], a[11]); hi.z = pack2(a[12], a[13]); hi.w = pack2(a[14], a[15]);
            *reinterpret_cast<uint4 *>(out + (size_t)p * 16) = lo;
            *reinterpret_cast<uint4 *>(out + (size_t)(NP + p) * 16) = hi;
        } else {
            const int r = p / S, c = p - r * S;
            if (r < S3 && c < S3) {
                const int kidx = r * S3 + c;
                #pragma unroll
                for (int o = 0; o < 2; ++o) {
                    const float z = v[o] + bias[o];
                    if (z > best[o] || (z == best[o] && kidx < bidx[o])) { best[o] = z; bidx[o] = kidx; }
                }
            }
        }
        fence_before();
        __syncthreads();
    }
    return true;
}

__global__ void __launch_bounds__(NT) k_cnn_forward_tc(int n, int S, const float *w, const float *x, float *logits,
                                                       int *err, long long limit)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int NP = npos(S);
    const size_t AB = act_bytes(S);
    unsigned char *act0 = sm, *act1 = sm + AB, *act2 = sm + 2 * AB;
    __nv_bfloat16 *wsl = reinterpret_cast<__nv_bfloat16 *>(sm + 3 * AB);
    float *bias = reinterpret_cast<float *>(sm + 3 * AB + 3 * 9 * kSliceBytes);
    float *redv = bias + 34;                                  // 4 warps x 2 channels
    int *redi = reinterpret_cast<int *>(redv + 8);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 3 * AB + 3 * 9 * kSliceBytes + 64 * sizeof(float));
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mbar + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S1 = S - 2, S2 = S - 4, S3 = S - 6;
    const int T1 = (S1 * S + 127) / 128, T2 = (S2 * S + 127) / 128, T3 = (S3 * S + 127) / 128;

    // zero the activation buffers once (padding positions and channels stay zero)
    for (size_t k = threadIdx.x; k < 3 * AB / 16; k += NT) reinterpret_cast<uint4 *>(sm)[k] = make_uint4(0, 0, 0, 0);
    stage_weights(w + cnn::OW1, 3, 16, wsl);
    stage_weights(w + cnn::OW2, 16, 16, wsl + 9 * 256);
    stage_weights(w + cnn::OW3, 16, 2, wsl + 18 * 256);
    for (int k = threadIdx.x; k < 16; k += NT) { bias[k] = w[cnn::OB1 + k]; bias[16 + k] = w[cnn::OB2 + k]; }
    if (threadIdx.x < 2) bias[32 + threadIdx.x] = w[cnn::OB3 + threadIdx.x];
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(mbar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(mbar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(saddr(tslot)),
                     "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t mb0 = saddr(mbar), mb1 = saddr(mbar + 1);
    uint32_t phases = 0u;                     // bit b: the phase accumulator b waits for
    bool ok = true;

    for (int smp = blockIdx.x; smp < n && ok; smp += gridDim.x) {
        // the sample as BF16 into chunk 0 of act0 (channels 3..7 zero)
        const float *xs = x + (size_t)smp * 3 * S * S;
        for (int p = threadIdx.x; p < S * S; p += NT) {
            uint4 e;
            e.x = pack2(xs[p], xs[S * S + p]);
            e.y = pack2(xs[2 * S * S + p], 0.f);
            e.z = 0u; e.w = 0u;
            *reinterpret_cast<uint4 *>(act0 + (size_t)p * 16) = e;
        }
        fence_async_smem();
        __syncthreads();
        float best[2] = {-3.0e38f, -3.0e38f};
        int bidx[2] = {0x7fffffff, 0x7fffffff};
        ok = conv_layer(act0, wsl, S, T1, tmem, mb0, mb1, phases, limit, act1, bias, S3, best, bidx);
        if (ok) {
            fence_async_smem();
            __syncthreads();
            ok = conv_layer(act1, wsl + 9 * 256, S, T2, tmem, mb0, mb1, phases, limit, act2, bias + 16, S3, best,
                            bidx);
        }
        if (ok) {
            fence_async_smem();
            __syncthreads();
            ok = conv_layer(act2, wsl + 18 * 256, S, T3, tmem, mb0, mb1, phases, limit, nullptr, bias + 32, S3,
                            best, bidx);
        }
        if (!ok) break;
        // per-channel maximum, first position in raster order among equals
        #pragma unroll
        for (int o = 0; o < 2; ++o) {
            float b = best[o];
            int bi = bidx[o];
            for (int d = 16; d > 0; d >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, b, d);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, d);
                if (ob > b || (ob == b && oi < bi)) { b = ob; bi = oi; }
            }
            if (lane == 0) { redv[warp * 2 + o] = b; redi[warp * 2 + o] = bi; }
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            const int o = threadIdx.x;
            float b = redv[o];
            int bi = redi[o];
            for (int q = 1; q < NT / 32; ++q) {
                const float ob = redv[2 * q + o];
                const int oi = redi[2 * q + o];
                if (ob > b || (ob == b && oi < bi)) { b = ob; bi = oi; }
            }
            logits[2 * smp + o] = b;
        }
        __syncthreads();
    }
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace tc

// failure flag of the tensor-core forward (a tile that did not complete
// within the wait limit) and the limit itself, in mbarrier polls
static __device__ int g_tc_err;
static long long g_tc_wait_limit = 1ll << 24;
}  // namespace fc

using namespace fc;

extern "C" {

int fc_cnn_input_stats(int n, int S, const float *x, double *stats, void *stream)
{
    if (n <= 0 || S < 1 || !x || !stats) {
        set_error("fc_cnn_input_stats: invalid argument");
        return FC_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long total = (long long)n * 3 * S * S;
    const double count = (double)n * S * S;
    double *buf = nullptr;
    FC_CUDA(cudaMallocAsync(&buf, sizeof(double) * (3 * cnn::kStatBlocks + 6), s));
    double *part = buf, *mean = buf + 3 * cnn::kStatBlocks, *var = mean + 3;
    cnn::k_chan_sums<false><<<cnn::kStatBlocks, cnn::kStatThreads, 0, s>>>(total, S * S, x, nullptr, part);
    cnn::k_chan_final<<<1, 32, 0, s>>>(part, count, mean);
    cnn::k_chan_sums<true><<<cnn::kStatBlocks, cnn::kStatThreads, 0, s>>>(total, S * S, x, mean, part);
    cnn::k_chan_final<<<1, 32, 0, s>>>(part, count, var);
    cudaError_t e = cudaGetLastError();
    double h[6];
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, mean, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return cuda_status(e, "fc_cnn_input_stats");
    for (int c = 0; c < 3; ++c) { stats[c] = h[c]; stats[3 + c] = sqrt(h[3 + c]); }
    FC_CUDA(cudaStreamSynchronize(s));
    return FC_OK;
}

int fc_cnn_normalize(int n, int S, float *x, const double *xform, void *stream)
{
    if (n <= 0 || S < 1 || !x || !xform) {
        set_error("fc_cnn_normalize: invalid argument");
        return FC_ERR_INVALID_ARG;
    }
    const long long total = (long long)n * 3 * S * S;
    cnn::k_normalize<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(total, S * S, x, xform[0],
                                                                                     xform[1], xform[2], xform[3]);
    FC_CUDA(cudaGetLastError());
    FC_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return FC_OK;
}


int fc_cnn_forward(int n, int S, const float *w, const float *x, float *logits, int bf16, void *stream)
{
    if (n <= 0 || S < 7 || S > cnn::MAXS || !w || !x || !logits) {
        set_error("fc_cnn_forward: invalid argument");
        return FC_ERR_INVALID_ARG;
    }
    if (bf16) {                    // BF16 inference on the tensor cores
        cudaStream_t s = (cudaStream_t)stream;
        const size_t sb = tc::smem_bytes(S);
        FC_CUDA(cudaFuncSetAttribute(tc::k_cnn_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
        int dev = 0, sms = 0, per = 0;
        FC_CUDA(cudaGetDevice(&dev));
        FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        FC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, tc::k_cnn_forward_tc, tc::NT, sb));
        const int grid = n < sms * (per > 0 ? per : 1) ? n : sms * (per > 0 ? per : 1);
        int *err = nullptr;
        FC_CUDA(cudaGetSymbolAddress((void **)&err, g_tc_err));
        FC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
        tc::k_cnn_forward_tc<<<grid, tc::NT, sb, s>>>(n, S, w, x, logits, err, g_tc_wait_limit);
        FC_CUDA(cudaGetLastError());
        int herr = 0;
        FC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        FC_CUDA(cudaStreamSynchronize(s));
        if (herr) {
            set_error("fc_cnn_forward: a tensor-core tile did not complete within the wait limit");
            return FC_ERR_TIMEOUT;
        }
        return FC_OK;
    }
    size_t sb = cnn::smem_bytes(S, false);
    FC_CUDA(cudaFuncSetAttribute(cnn::k_cnn_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    cnn::k_cnn_forward<<<cnn::grid_for(n), cnn::NT, sb, (cudaStream_t)stream>>>(n, S, w, x, logits, bf16);
    FC_CUDA(cudaGetLastError());
    FC_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return FC_OK;
}

int fc_cnn_loss_grad(int n, int S, const float *w, const float *x, const float *targets, float *grad,
                     float *loss, int bf16, void *stream)
{
    if (n <= 0 || S < 7 || S > cnn::MAXS || !w || !x || !targets || !grad || !loss) {
        set_error("fc_cnn_loss_grad: invalid argument");
        return FC_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int nb = cnn::grid_for(n);
    float *part = nullptr, *lossp = nullptr, *dloss = nullptr;
    FC_CUDA(cudaMallocAsync(&part, sizeof(float) * ((size_t)nb * cnn::NPARAM + 2 * nb + 2), s));
    lossp = part + (size_t)nb * cnn::NPARAM;
    dloss = lossp + nb;
    size_t sb = cnn::smem_bytes(S, true);
    cudaError_t e = cudaFuncSetAttribute(cnn::k_cnn_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
    if (e == cudaSuccess) {
        cnn::k_cnn_backward<<<nb, cnn::NT, sb, s>>>(n, S, w, x, targets, part, lossp, bf16);
        cnn::k_cnn_reduce<<<(cnn::NPARAM + 255) / 256, 256, 0, s>>>(part, lossp, nb, grad, dloss);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dloss, sizeof(float), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(part, s);
    if (e != cudaSuccess) return cuda_status(e, "fc_cnn_loss_grad");
    FC_CUDA(cudaStreamSynchronize(s));
    return FC_OK;
}

int fc_cnn_set_wait_limit(long long polls)
{
    if (polls < 0) { set_error("fc_cnn_set_wait_limit: negative limit"); return FC_ERR_INVALID_ARG; }
    g_tc_wait_limit = polls;
    return FC_OK;
}

int fc_cnn_adam(float *w, const float *grad, float *m1, float *m2, int step, float lr, void *stream)
{
    if (!w || !grad || !m1 || !m2 || step < 1) { set_error("fc_cnn_adam: invalid argument"); return FC_ERR_INVALID_ARG; }
    float b1t = powf(0.9f, (float)step), b2t = powf(0.999f, (float)step);
    cnn::k_cnn_adam<<<(cnn::NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, grad, m1, m2, b1t, b2t, lr);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

}  // extern "C"
