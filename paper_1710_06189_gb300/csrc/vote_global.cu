// GLCM counts for N > 256 levels (up to 4096): Eq. 1 with the histogram in
// global memory.  N^2 bins no longer fit one CTA's shared memory (4 MB per
// offset at N = 1024), so every vote goes straight to the output counts in
// L2, aggregated within the warp first: lanes whose pair falls in the same
// bin (__match_any_sync on the bin) are counted by one global reduction of
// their number (the warp-aggregated atomics of this work's plan for large N;
// the paper's Scheme 1, Sec. I.B, votes with one global atomic per pair).
// On smooth images most lanes of a warp share bins and the reductions
// collapse; on noise images it is one reduction per pair at L2's atomic rate.
// A thread takes one anchor of one offset; pixels come through the
// read-only cache.
#include "glcm_internal.cuh"

namespace glcm {
namespace {

__device__ __forceinline__ uint32_t gpx(const SeamJob& j, int x, int y)
{
    const uint8_t* row = j.img + (long long)y * j.pitch;
    if (j.bpp == 1)
        return __ldg(row + x);
    return (uint32_t)__ldg(row + 2 * x) | ((uint32_t)__ldg(row + 2 * x + 1) << 8);
}

__device__ __forceinline__ uint32_t glevel(const SeamJob& j, uint32_t v)
{
    return j.levels_mode ? v : (uint32_t)(((unsigned long long)v * (unsigned)j.levels) >> (8 * j.bpp));
}

// blockIdx.y: the job (one offset of one image, anchor rows [y_begin, y_end));
// blockIdx.x: a slice of its anchors.  Every lane of a warp reaches the
// aggregation (a lane without a vote takes part with an unused bin value).
__global__ void k_vote_global(const SeamJob* jobs, unsigned* err)
{
    const SeamJob j = jobs[blockIdx.y];
    const long long rows = (long long)max(0, j.y_end - j.y_begin);
    const long long n = rows * j.W;
    const uint32_t N = (uint32_t)j.levels;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    bool bad = false;
    // tb: the warp's first anchor (the same for all its lanes, so the whole
    // warp iterates together).
    for (long long tb = blockIdx.x * (long long)blockDim.x + (threadIdx.x - lane); tb < n; tb += stride) {
        const long long t = tb + lane;
        uint32_t code = 0xFFFFFFFFu;  // no vote
        if (t < n) {
            const long long r = t / j.W;
            const int x = (int)(t - r * j.W), y = j.y_begin + (int)r;
            const int x2 = x + j.dx, y2 = y + j.dy;
            if (x2 >= 0 && x2 < j.W && y2 >= 0 && y2 < j.H) {
                const uint32_t a = glevel(j, gpx(j, x, y)), b = glevel(j, gpx(j, x2, y2));
                if (a < N && b < N)
                    code = a * N + b;
                else
                    bad = true;
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, code);
        if (code != 0xFFFFFFFFu && lane == __ffs(peers) - 1)
            atomicAdd(j.out + code, (uint32_t)__popc(peers));
    }
    if (bad)
        atomicOr(err, kErrRange);
}

}  // namespace

cudaError_t launch_vote_global(const SeamJob* jobs, int n_jobs, int blocks_per_job, unsigned* err, cudaStream_t s)
{
    for (int j0 = 0; j0 < n_jobs; j0 += 65535) {  // grid.y holds at most 65535 jobs
        const int nj = n_jobs - j0 < 65535 ? n_jobs - j0 : 65535;
        k_vote_global<<<dim3(blocks_per_job, nj), 256, 0, s>>>(jobs + j0, err);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace glcm
