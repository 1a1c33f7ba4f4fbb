// Column-walk GLCM votes (the kernel is described in vote_fast.cuh): the
// instances for rows that start on 16 bytes, and the host side of every
// launch -- shared-memory sizes and the choice of kernel instance.
#include "vote_fast.cuh"

namespace glcm {
namespace {

template <int BPP>
const void* fast_kernel_aligned(int log2n)
{
    switch (log2n) {
        case 1: return (const void*)k_glcm_vote_d1<BPP, 1, true>;
        case 2: return (const void*)k_glcm_vote_d1<BPP, 2, true>;
        case 3: return (const void*)k_glcm_vote_d1<BPP, 3, true>;
        case 4: return (const void*)k_glcm_vote_d1<BPP, 4, true>;
        case 5: return (const void*)k_glcm_vote_d1<BPP, 5, true>;
        default: return (const void*)k_glcm_vote_d1<BPP, 8, true>;
    }
}

SmemLimit g_fast_lim[2][2][9];  // [aligned][bpp - 1][log2n]

}  // namespace

// Shared words of one job's histograms.
int vote_fast_hist_words(int log2n, int mode)
{
    if (mode == kFastWide)
        return 32768;
    const int M = (1 << log2n) + 1;
    if (mode == kFastJoint)
        return M * M * M * 64;
    if (mode == kFastPair)
        return log2n == 4 ? 2 * 256 * 64 : 2 * M * M * 64;  // N = 16: byte codes, no outside level
    return M * M * 32;
}

// Dynamic shared memory of a launch whose largest job histogram has
// max_hist_words words (the joint merge's marginals follow it): room to
// align the histograms (fast_align), the histograms, the marginals, the
// chunk index, and ring_words per warp of row rings (distances > 1; for
// N = 16 the rings lie in the alignment padding).
size_t vote_fast_smem_bytes(int max_hist_words, int log2n, int ring_words)
{
    const size_t rings = fast_align(log2n) == 65536u ? 0 : (size_t)ring_words * kFW * 4;
    return (size_t)fast_align(log2n) + (size_t)(max_hist_words + kMargWords) * 4 + 16 + rings;
}

cudaError_t launch_vote_fast(const FastParams& p, int bpp, int log2n, bool aligned, int grid, size_t smem,
                             cudaStream_t s)
{
    if (p.n_chunks <= 0)
        return cudaSuccess;
    if (bpp < 1 || bpp > 2 || log2n < 1 || (log2n > 5 && log2n != 8))
        return cudaErrorInvalidValue;
    const void* fn = !aligned ? vote_fast_kernel_unaligned(bpp, log2n)
                              : (bpp == 1 ? fast_kernel_aligned<1>(log2n) : fast_kernel_aligned<2>(log2n));
    const cudaError_t e = g_fast_lim[aligned ? 1 : 0][bpp - 1][log2n].raise(fn, smem);
    if (e != cudaSuccess)
        return e;
    void* args[] = {const_cast<FastParams*>(&p)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kFT), args, smem, s);
}

}  // namespace glcm
