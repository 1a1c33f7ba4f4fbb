// Measured ceilings of the vote kernels on the current GPU: how many
// shared-memory reductions (red.shared.add.u32, the vote of Eq. 1 into a
// private copy, Sec. II.A) one GPU completes per second for the address
// patterns the vote kernels produce, and how fast a streaming kernel reads
// HBM.  The vote kernels are measured against these beside the HBM copy rate.
//
// Patterns (512 threads per CTA, one CTA per SM, 128 KB of shared words):
//  * interleaved: lane l of every warp on bank l (word 32 k + l) -- the
//    lane-interleaved private copies of the vote kernels, never a conflict;
//  * same word: every lane of a warp on one word with the constant
//    increment 1 (a flat image region voting into one bin);
//  * random: each lane on a random word of one 128 KB copy (a single shared
//    histogram under a noise image: random bank conflicts).
#include <cstdio>

#include "glcm.h"
#include "glcm_internal.cuh"

namespace glcm {
namespace {

constexpr int kCT = 512;          // threads per CTA
constexpr int kCWords = 32768;    // 128 KB of shared words
constexpr int kCPerIter = 16;     // reductions per thread per iteration

__device__ __forceinline__ void red1(uint32_t a)
{
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a));
}

template <int PATTERN>
__global__ void __launch_bounds__(kCT, 1) k_red_rate(int iters, unsigned* sink)
{
    extern __shared__ __align__(16) uint32_t h[];
    for (int i = threadIdx.x; i < kCWords; i += kCT)
        h[i] = 0u;
    __syncthreads();
    const uint32_t hb = (uint32_t)__cvta_generic_to_shared(h);
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t r[kCPerIter];
    uint32_t x = (threadIdx.x + 1u) * 2654435761u ^ (blockIdx.x + 1u) * 40503u;
#pragma unroll
    for (int i = 0; i < kCPerIter; ++i) {
        x ^= x << 13;
        x ^= x >> 17;
        x ^= x << 5;
        r[i] = x & (kCWords - 1);
    }
    for (int it = 0; it < iters; ++it) {
        const uint32_t row = ((uint32_t)it * kCPerIter + warp * 7u) * 32u;
#pragma unroll
        for (int i = 0; i < kCPerIter; ++i) {
            uint32_t w;
            if (PATTERN == 0)
                w = (row + (uint32_t)i * 32u + lane) & (kCWords - 1);
            else if (PATTERN == 1)
                w = (row + (uint32_t)i * 32u) & (kCWords - 1);
            else
                w = (r[i] + (uint32_t)it * 1031u) & (kCWords - 1);
            red1(hb + 4u * w);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        sink[blockIdx.x] = h[blockIdx.x & (kCWords - 1)];
}

__global__ void k_read_rate(const uint4* __restrict__ p, long long n, unsigned* sink)
{
    uint32_t acc = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const uint4 a = __ldcs(p + i), b = __ldcs(p + i + stride), c = __ldcs(p + i + 2 * stride),
                    d = __ldcs(p + i + 3 * stride);
        acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
    }
    for (; i < n; i += stride) {
        const uint4 a = __ldcs(p + i);
        acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
    if (acc == 0x9E3779B9u)  // never for the zeroed buffer; keeps the loads
        sink[0] = acc;
}

template <int PATTERN>
double red_rate(int sms, unsigned* sink, cudaEvent_t e0, cudaEvent_t e1)
{
    const size_t smem = (size_t)kCWords * 4;
    if (cudaFuncSetAttribute(k_red_rate<PATTERN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return -1.0;
    const int iters = 2048;
    k_red_rate<PATTERN><<<sms, kCT, smem>>>(64, sink);  // warm-up
    double best = 0.0;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        k_red_rate<PATTERN><<<sms, kCT, smem>>>(iters, sink);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess)
            return -1.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double reds = (double)sms * kCT * kCPerIter * iters;
        if (ms > 0.f && reds / (ms * 1e-3) > best)
            best = reds / (ms * 1e-3);
    }
    return best;
}

}  // namespace
}  // namespace glcm

extern "C" int glcm_measure_ceilings(int device, glcm_ceilings* out)
{
    using namespace glcm;
    if (!out)
        return GLCM_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GLCM_ERR_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess)
        return GLCM_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const size_t bytes = (size_t)1 << 30;
    unsigned* sink = nullptr;
    void* buf = nullptr;
    if (cudaMalloc(&sink, (size_t)sms * 4 + 64) != cudaSuccess || cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (sink)
            cudaFree(sink);
        return GLCM_ERR_NOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = GLCM_OK;
    out->sm_count = sms;
    out->red_interleaved_per_s = red_rate<0>(sms, sink, e0, e1);
    out->red_same_word_per_s = red_rate<1>(sms, sink, e0, e1);
    out->red_random_one_copy_per_s = red_rate<2>(sms, sink, e0, e1);
    cudaMemset(buf, 0, bytes);
    const long long n = (long long)(bytes / 16);
    k_read_rate<<<sms * 4, 512>>>(static_cast<const uint4*>(buf), n, sink);
    double best = 0.0;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        k_read_rate<<<sms * 4, 512>>>(static_cast<const uint4*>(buf), n, sink);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = GLCM_ERR_CUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms > 0.f && (double)bytes / (ms * 1e-3) / 1e9 > best)
            best = (double)bytes / (ms * 1e-3) / 1e9;
    }
    out->hbm_read_gbs = best;
    if (out->red_interleaved_per_s < 0 || out->red_same_word_per_s < 0 || out->red_random_one_copy_per_s < 0 ||
        cudaGetLastError() != cudaSuccess)
        rc = GLCM_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    return rc;
}
