// Flat-wrap pairs (GLCM_FLAT_WRAP): Eq. 2 read literally on the image as one
// row-major buffer pairs pixel p = y W + x with p + dy W + dx whenever that
// index lies in [0, W H).  The vote kernels count the pairs whose partner lies
// inside the image rectangle; the ones they leave out are exactly the anchors
// whose partner column x + dx leaves [0, W) -- |dx| columns at one side of
// every row (all columns when |dx| >= W).  Those are counted here, one thread
// per anchor, with global atomics: about |dx| H pixels per offset, a sliver of
// the image, so the rate of the atomics does not matter.
#include "glcm_internal.cuh"

namespace glcm {
namespace {

__device__ __forceinline__ uint32_t seam_px(const SeamJob& j, long long q)
{
    const long long y = q / j.W, x = q - y * j.W;
    const uint8_t* row = j.img + y * j.pitch;
    if (j.bpp == 1)
        return __ldg(row + x);
    return (uint32_t)__ldg(row + 2 * x) | ((uint32_t)__ldg(row + 2 * x + 1) << 8);
}

__device__ __forceinline__ uint32_t seam_level(const SeamJob& j, uint32_t v)
{
    return j.levels_mode ? v : (uint32_t)(((unsigned long long)v * (unsigned)j.levels) >> (8 * j.bpp));
}

// blockIdx.y: the job; blockIdx.x: a slice of its seam anchors.
__global__ void k_seam(const SeamJob* jobs, unsigned* err)
{
    const SeamJob j = jobs[blockIdx.y];
    const int cols = j.dx == 0 ? 0 : (j.dx > 0 ? min(j.dx, j.W) : min(-j.dx, j.W));
    const int x0 = j.dx > 0 ? j.W - cols : 0;
    const long long rows = (long long)max(0, j.y_end - j.y_begin);
    const long long n = rows * cols;
    const long long total = (long long)j.W * j.H;
    const long long off = (long long)j.dy * j.W + j.dx;
    const uint32_t N = (uint32_t)j.levels;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / cols;
        const int x = x0 + (int)(t - r * cols);
        const long long p = (j.y_begin + r) * (long long)j.W + x;
        const long long q = p + off;
        if (q < 0 || q >= total)
            continue;
        const uint32_t a = seam_level(j, seam_px(j, p)), b = seam_level(j, seam_px(j, q));
        if (a >= N || b >= N) {
            atomicOr(err, kErrRange);
            continue;
        }
        atomicAdd(j.out + a * N + b, 1u);
    }
}

}  // namespace

cudaError_t launch_seams(const SeamJob* jobs, int n_jobs, int blocks_per_job, unsigned* err, cudaStream_t s)
{
    for (int j0 = 0; j0 < n_jobs; j0 += 65535) {  // grid.y holds at most 65535 jobs
        const int nj = n_jobs - j0 < 65535 ? n_jobs - j0 : 65535;
        k_seam<<<dim3(blocks_per_job, nj), 256, 0, s>>>(jobs + j0, err);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace glcm
