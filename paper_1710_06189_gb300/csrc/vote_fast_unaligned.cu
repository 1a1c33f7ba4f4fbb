// Column-walk GLCM votes (the kernel is described in vote_fast.cuh): the
// instances for rows at any byte address (odd widths of a contiguous image,
// views that start at odd columns), whose 16-byte loads are realigned.
#include "vote_fast.cuh"

namespace glcm {

const void* vote_fast_kernel_unaligned(int bpp, int log2n)
{
    if (bpp == 1) {
        switch (log2n) {
            case 1: return (const void*)k_glcm_vote_d1<1, 1, false>;
            case 2: return (const void*)k_glcm_vote_d1<1, 2, false>;
            case 3: return (const void*)k_glcm_vote_d1<1, 3, false>;
            case 4: return (const void*)k_glcm_vote_d1<1, 4, false>;
            case 5: return (const void*)k_glcm_vote_d1<1, 5, false>;
            default: return (const void*)k_glcm_vote_d1<1, 8, false>;
        }
    }
    switch (log2n) {
        case 1: return (const void*)k_glcm_vote_d1<2, 1, false>;
        case 2: return (const void*)k_glcm_vote_d1<2, 2, false>;
        case 3: return (const void*)k_glcm_vote_d1<2, 3, false>;
        case 4: return (const void*)k_glcm_vote_d1<2, 4, false>;
        case 5: return (const void*)k_glcm_vote_d1<2, 5, false>;
        default: return (const void*)k_glcm_vote_d1<2, 8, false>;
    }
}

}  // namespace glcm
