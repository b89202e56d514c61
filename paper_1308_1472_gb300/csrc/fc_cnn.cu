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
// kernels run on FP32 values (used to check the gradients tightly).
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

int fc_cnn_adam(float *w, const float *grad, float *m1, float *m2, int step, float lr, void *stream)
{
    if (!w || !grad || !m1 || !m2 || step < 1) { set_error("fc_cnn_adam: invalid argument"); return FC_ERR_INVALID_ARG; }
    float b1t = powf(0.9f, (float)step), b2t = powf(0.999f, (float)step);
    cnn::k_cnn_adam<<<(cnn::NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, grad, m1, m2, b1t, b2t, lr);
    FC_CUDA(cudaGetLastError());
    return FC_OK;
}

}  // extern "C"
