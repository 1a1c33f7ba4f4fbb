// Gray-level histogram of one image.
//
// Every pixel, quantized to N levels as for Eq. (1), casts one vote into bin
// q.  The paper notes (Sec. I, contribution 2) that its analysis of vote
// collisions carries over to the image histogram; here its remedy of private
// copies is taken to the limit: every lane of a CTA owns a copy of the N
// bins, laid out so that lane l's copy of bin q is word q * 32 + l, which is
// always in bank l.  No vote ever waits on another lane's, whatever the
// image (smooth, constant or noise).
//
// The image is read once with 16-byte streaming loads, four in flight per
// thread.  A contiguous image (pitch = row bytes) is one span that the whole
// grid strides over; a pitched one is cut into row segments that warps take
// in grid-stride order.  Bytes before the first and after the last 16-byte
// boundary of a span are read one element at a time, as is every element of
// a uint16 span that starts at an odd address.  Each CTA finally sums its 32
// copies of every bin with a warp reduction and adds the sum into the global
// histogram, which the host has zeroed.
//
// Algorithmic traffic: W * H * bytes-per-pixel read once, N * 4 bytes added
// per CTA; the roofline is the HBM read (the shared reductions, one per
// pixel, and the instructions that form their addresses run beside it).
#include "glcm_internal.cuh"

namespace glcm {
namespace {

constexpr int kHistThreads = 512;
constexpr int kHistMinBlocks = 2;
// Bytes a warp takes at a time from a pitched image's row (a multiple of 16).
constexpr long long kHistSegBytes = 4096;

template <int BPP>
struct Voter {
    uint32_t base;  // shared address of this lane's copy of bin 0
    uint32_t n;     // levels
    int mode;       // pixels already are levels
    bool bad;       // a pixel >= N was seen in levels mode

    __device__ __forceinline__ void vote(uint32_t v)
    {
        uint32_t q;
        if (mode) {
            if (v >= n) {
                bad = true;
                return;
            }
            q = v;
        } else {
            q = (v * n) >> (8 * BPP);
        }
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(base + q * 128u), "r"(1u));
    }

    __device__ __forceinline__ void word(uint32_t w)
    {
        if constexpr (BPP == 1) {
            vote(w & 0xFFu);
            vote((w >> 8) & 0xFFu);
            vote((w >> 16) & 0xFFu);
            vote(w >> 24);
        } else {
            vote(w & 0xFFFFu);
            vote(w >> 16);
        }
    }

    __device__ __forceinline__ void vec(const uint4& a)
    {
        word(a.x);
        word(a.y);
        word(a.z);
        word(a.w);
    }
};

// One pixel at p (little-endian for uint16; p may be odd).
template <int BPP>
__device__ __forceinline__ uint32_t load_px(const uint8_t* p)
{
    if constexpr (BPP == 1)
        return __ldg(p);
    else
        return (uint32_t)__ldg(p) | ((uint32_t)__ldg(p + 1) << 8);
}

// Votes of the nbytes bytes at s (a whole number of pixels), shared by a team
// of `team` threads of which this one is `rank`.
template <int BPP>
__device__ __forceinline__ void vote_span(Voter<BPP>& vt, const uint8_t* s, long long nbytes, long long rank,
                                          long long team)
{
    const uintptr_t sa = reinterpret_cast<uintptr_t>(s);
    if (BPP == 2 && (sa & 1)) {
        const long long ne = nbytes >> 1;
        for (long long k = rank; k < ne; k += team)
            vt.vote(load_px<BPP>(s + 2 * k));
        return;
    }
    // Head up to the first 16-byte boundary (a whole number of pixels: s is
    // pixel-aligned here), then whole vectors, then the tail.
    long long head = (long long)((16u - (unsigned)(sa & 15u)) & 15u);
    if (head > nbytes)
        head = nbytes;
    const long long nv = (nbytes - head) >> 4;
    const long long tail0 = head + nv * 16;
    const long long n_head = head / BPP, n_tail = (nbytes - tail0) / BPP;
    for (long long k = rank; k < n_head; k += team)
        vt.vote(load_px<BPP>(s + k * BPP));
    for (long long k = rank; k < n_tail; k += team)
        vt.vote(load_px<BPP>(s + tail0 + k * BPP));
    const uint4* v = reinterpret_cast<const uint4*>(s + head);
    long long i = rank;
    for (; i + 3 * team < nv; i += 4 * team) {
        const uint4 a = __ldcs(v + i);
        const uint4 b = __ldcs(v + i + team);
        const uint4 c = __ldcs(v + i + 2 * team);
        const uint4 d = __ldcs(v + i + 3 * team);
        vt.vec(a);
        vt.vec(b);
        vt.vec(c);
        vt.vec(d);
    }
    for (; i < nv; i += team)
        vt.vec(__ldcs(v + i));
}

template <int BPP>
__global__ void __launch_bounds__(kHistThreads, kHistMinBlocks) k_histogram(HistParams p)
{
    extern __shared__ uint32_t s_h[];  // [bin][lane], levels * 32 words
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
    for (int t = threadIdx.x; t < p.levels * 32; t += blockDim.x)
        s_h[t] = 0;
    __syncthreads();

    Voter<BPP> vt{(uint32_t)__cvta_generic_to_shared(s_h) + 4u * (uint32_t)lane, (uint32_t)p.levels,
                  p.levels_mode, false};
    if (p.flat) {
        vote_span<BPP>(vt, p.img, p.row_bytes, (long long)blockIdx.x * blockDim.x + threadIdx.x,
                       (long long)gridDim.x * blockDim.x);
    } else {
        for (long long u = (long long)blockIdx.x * warps + warp; u < p.units; u += (long long)gridDim.x * warps) {
            const long long r = u / p.segs, b0 = (u - r * p.segs) * p.seg_bytes;
            const long long nb = p.row_bytes - b0 < p.seg_bytes ? p.row_bytes - b0 : p.seg_bytes;
            vote_span<BPP>(vt, p.img + r * p.pitch + b0, nb, lane, 32);
        }
    }
    if (vt.bad)
        atomicOr(p.err, kErrRange);
    __syncthreads();

    for (int b = warp; b < p.levels; b += warps) {
        const uint32_t c = __reduce_add_sync(0xffffffffu, s_h[b * 32 + lane]);
        if (lane == 0 && c)
            atomicAdd(p.hist + b, c);
    }
}

}  // namespace

cudaError_t launch_histogram(const HistParams& p, int sm_count, cudaStream_t s)
{
    if (p.row_bytes <= 0 || (!p.flat && p.units <= 0))
        return cudaSuccess;
    const size_t smem = (size_t)p.levels * 32 * 4;
    const void* fn = p.bpp == 1 ? (const void*)k_histogram<1> : (const void*)k_histogram<2>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kHistThreads, smem);
    if (e != cudaSuccess)
        return e;
    const long long full = (long long)(occ > 0 ? occ : 1) * sm_count;
    // At least four vectors per thread (flat) or one segment per warp.
    const long long want = p.flat ? (p.row_bytes + (long long)kHistThreads * 64 - 1) / ((long long)kHistThreads * 64)
                                  : (p.units + kHistThreads / 32 - 1) / (kHistThreads / 32);
    const int grid = (int)(want < 1 ? 1 : (want < full ? want : full));
    if (p.bpp == 1)
        k_histogram<1><<<grid, kHistThreads, smem, s>>>(p);
    else
        k_histogram<2><<<grid, kHistThreads, smem, s>>>(p);
    return cudaGetLastError();
}

long long histogram_seg_bytes()
{
    return kHistSegBytes;
}

}  // namespace glcm
