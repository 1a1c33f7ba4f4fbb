// GLCM vote kernels: quantize -> partner lookup -> vote -> merge.
//
// What is computed (Sec. I.A, Eq. 1): for every anchor pixel (x, y) whose
// partner (x + dx, y + dy) lies inside the image, with i and j the levels of
// the two pixels, P[i][j] += 1.  Partner addressing follows Eq. 2 with no
// pairing across the border, bins follow Eq. 3 with the anchor as the row.
//
// How (the paper's Scheme 2 copy strategy, Sec. II.A, redone for sm_103a):
//  * Persistent CTAs (one or two per SM) pull work items -- a 16-byte-per-
//    lane column strip of one image and a band of rows -- from a global
//    counter.  Each warp takes rows of the band; each lane owns 16 bytes of
//    the row (16 uint8 or 8 uint16 pixels), read with one 128-bit
//    non-coherent load, quantized in registers to packed level bytes.
//  * The partner row of each distinct dy is read the same way; the 4 levels
//    left and right of a lane come from its neighbours by shuffle, so every
//    |dx| <= 4 partner is a byte extraction from registers.
//  * Votes go into R private copies of the job's histograms in shared
//    memory, interleaved so that copy c of bin b sits at word b*R + c and
//    lane l always uses copy l mod R: with R = 32 every lane of a warp hits
//    its own bank whatever the data (the paper's copies are contiguous, so
//    equal bins of different copies share a bank).  With `pack` = 2, two
//    offsets share a word as two 16-bit halves, halving the footprint; the
//    host bounds the votes per half between merges below 65536.
//  * Optional warp aggregation (__match_any_sync + one popc-weighted add per
//    distinct word) for single-copy histograms.
//  * The merge (Sec. II.A, last step) sums the copies and adds each non-zero
//    bin into the global uint32 counts once per CTA and job.
//  * When a single offset's N*N uint32 histogram cannot fit shared memory
//    (N = 256) the job votes straight into the global counts (L2 atomics).
//  * Image edges, unaligned images, |dx| > 4 and out-of-range pixels in
//    levels mode take a per-pixel path with full bounds checks.
#include "glcm_internal.cuh"

namespace glcm {
namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void red_shared_add(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

__device__ __forceinline__ void red_global_add(uint32_t* p, uint32_t v)
{
    asm volatile("red.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ uint4 ldg_v4(const uint8_t* p)
{
    return __ldg(reinterpret_cast<const uint4*>(p));
}

// Raw pixel read with no alignment assumption.
__device__ __forceinline__ uint32_t read_px(const VoteJob& j, int x, int y)
{
    const uint8_t* row = j.img + (long long)y * j.pitch;
    if (j.bpp == 1)
        return __ldg(row + x);
    const uint8_t* q = row + 2ll * x;
    return (uint32_t)__ldg(q) | ((uint32_t)__ldg(q + 1) << 8);
}

__device__ __forceinline__ uint32_t level_of(const VoteJob& j, uint32_t v)
{
    if (j.levels_mode)
        return v;
    return (uint32_t)(((unsigned long long)v * (unsigned)j.levels) >> (8 * j.bpp));
}

// 4 uint8 pixels -> 4 level bytes.  `bad` gets set if levels mode sees v >= N.
__device__ __forceinline__ uint32_t quant_u8x4(const VoteJob& j, uint32_t w, bool& bad)
{
    if (j.levels_mode) {
        if (j.levels < 256)
            bad |= __vcmpgeu4(w, 0x01010101u * (uint32_t)j.levels) != 0u;
        return w;
    }
    if (j.log2n >= 0) {
        const int s = 8 - j.log2n;
        return (w >> s) & (0x01010101u * (0xFFu >> s));
    }
    uint32_t r = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t v = (w >> (8 * b)) & 0xFFu;
        r |= ((v * (uint32_t)j.levels) >> 8) << (8 * b);
    }
    return r;
}

// 4 uint16 pixels (two words) -> 4 level bytes.
__device__ __forceinline__ uint32_t quant_u16x4(const VoteJob& j, uint32_t w0, uint32_t w1, bool& bad)
{
    if (j.levels_mode) {
        const uint32_t hi = __byte_perm(w0, w1, 0x7531);
        const uint32_t lo = __byte_perm(w0, w1, 0x6420);
        bad |= hi != 0u;
        if (j.levels < 256)
            bad |= __vcmpgeu4(lo, 0x01010101u * (uint32_t)j.levels) != 0u;
        return lo;
    }
    if (j.log2n >= 0 && j.log2n <= 8) {
        const uint32_t hi = __byte_perm(w0, w1, 0x7531);
        const int s = 8 - j.log2n;
        return (hi >> s) & (0x01010101u * (0xFFu >> s));
    }
    uint32_t r = 0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t w = b < 2 ? w0 : w1;
        const uint32_t v = (w >> (16 * (b & 1))) & 0xFFFFu;
        r |= (uint32_t)(((unsigned long long)v * (unsigned)j.levels) >> 16) << (8 * b);
    }
    return r;
}

// Load the levels of pixels [xl, xl + PX) of row y into LW words.  Only whole
// 4-pixel groups inside [0, W) are loaded (others read as 0 and are never
// used by the fast path).
template <int BPP>
__device__ __forceinline__ void load_levels(const VoteJob& j, int y, int xl, uint32_t (&L)[4 / BPP],
                                            bool& bad)
{
    constexpr int PX = 16 / BPP;
    constexpr int LW = PX / 4;
    const uint8_t* p = j.img + (long long)y * j.pitch + (long long)xl * BPP;
    if (xl + PX <= j.W) {
        const uint4 r = ldg_v4(p);
        if (BPP == 1) {
            L[0] = quant_u8x4(j, r.x, bad);
            L[1] = quant_u8x4(j, r.y, bad);
            L[2 % LW] = quant_u8x4(j, r.z, bad);
            L[3 % LW] = quant_u8x4(j, r.w, bad);
        } else {
            L[0] = quant_u16x4(j, r.x, r.y, bad);
            L[1] = quant_u16x4(j, r.z, r.w, bad);
        }
    } else {
#pragma unroll
        for (int w = 0; w < LW; ++w) {
            L[w] = 0;
            if (xl + 4 * w + 4 <= j.W) {
                if (BPP == 1) {
                    L[w] = quant_u8x4(j, __ldg(reinterpret_cast<const uint32_t*>(p + 4 * w)), bad);
                } else {
                    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p + 8 * w));
                    L[w] = quant_u16x4(j, q.x, q.y, bad);
                }
            }
        }
    }
}

// Levels of the 4 pixels starting at column x (x % 4 == 0, whole group inside).
template <int BPP>
__device__ __forceinline__ uint32_t load_group(const VoteJob& j, int y, int x, bool& bad)
{
    const uint8_t* p = j.img + (long long)y * j.pitch + (long long)x * BPP;
    if (BPP == 1)
        return quant_u8x4(j, __ldg(reinterpret_cast<const uint32_t*>(p)), bad);
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
    return quant_u16x4(j, q.x, q.y, bad);
}

struct HistRef {
    uint32_t base;    // shared byte address of copy c of this offset's first bin
    uint32_t inc;     // 1 or 1 << 16
    uint32_t stride;  // bytes between consecutive bins (4 * R)
};

// Vote the PX anchors of one lane for a compile-time dx, all pairs valid.
template <int BPP, int DX>
__device__ __forceinline__ void vote_fast(const uint32_t (&A)[4 / BPP], const uint32_t (&B)[4 / BPP + 2],
                                          int N, const HistRef& h)
{
    constexpr int PX = 16 / BPP;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const uint32_t i = (A[k >> 2] >> (8 * (k & 3))) & 0xFFu;
        const int pb = k + DX + 4;  // byte of the extended partner row
        const uint32_t jv = (B[pb >> 2] >> (8 * (pb & 3))) & 0xFFu;
        const uint32_t bin = i * (uint32_t)N + jv;
        red_shared_add(h.base + bin * h.stride, h.inc);
    }
}

template <int BPP, int DX>
__device__ __forceinline__ void vote_fast_agg(const uint32_t (&A)[4 / BPP], const uint32_t (&B)[4 / BPP + 2],
                                              int N, const HistRef& h, unsigned mask, int lane)
{
    constexpr int PX = 16 / BPP;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const uint32_t i = (A[k >> 2] >> (8 * (k & 3))) & 0xFFu;
        const int pb = k + DX + 4;
        const uint32_t jv = (B[pb >> 2] >> (8 * (pb & 3))) & 0xFFu;
        const uint32_t bin = i * (uint32_t)N + jv;
        const unsigned m = __match_any_sync(mask, bin);
        if ((__ffs(m) - 1) == lane)
            red_shared_add(h.base + bin * h.stride, h.inc * (uint32_t)__popc(m));
    }
}

template <int BPP, int DX>
__device__ __forceinline__ void vote_fast_global(const uint32_t (&A)[4 / BPP], const uint32_t (&B)[4 / BPP + 2],
                                                 int N, uint32_t* out, unsigned mask, int lane, int agg)
{
    constexpr int PX = 16 / BPP;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const uint32_t i = (A[k >> 2] >> (8 * (k & 3))) & 0xFFu;
        const int pb = k + DX + 4;
        const uint32_t jv = (B[pb >> 2] >> (8 * (pb & 3))) & 0xFFu;
        const uint32_t bin = i * (uint32_t)N + jv;
        if (agg) {
            const unsigned m = __match_any_sync(mask, bin);
            if ((__ffs(m) - 1) == lane)
                red_global_add(out + bin, (uint32_t)__popc(m));
        } else {
            red_global_add(out + bin, 1u);
        }
    }
}

// Per-pixel path with full checks (edges, unaligned images, wide dx, bad levels).
__device__ void vote_slow(const VoteJob& j, int dx, int dy, int y, int xl, int px, const HistRef& h,
                          uint32_t* gout, unsigned* err)
{
    const int yp = y + dy;
    if (y < 0 || y >= j.H || yp < 0 || yp >= j.H)
        return;
    const uint32_t N = (uint32_t)j.levels;
    for (int k = 0; k < px; ++k) {
        const int x = xl + k;
        if (x >= j.W)
            break;
        const int xp = x + dx;
        if (xp < 0 || xp >= j.W)
            continue;
        const uint32_t i = level_of(j, read_px(j, x, y));
        const uint32_t jv = level_of(j, read_px(j, xp, yp));
        if (i >= N || jv >= N) {
            atomicOr(err, kErrRange);
            continue;
        }
        const uint32_t bin = i * N + jv;
        if (gout)
            red_global_add(gout + bin, 1u);
        else
            red_shared_add(h.base + bin * h.stride, h.inc);
    }
}

template <int BPP>
__device__ __forceinline__ void dispatch_fast(int dx, const uint32_t (&A)[4 / BPP], const uint32_t (&B)[4 / BPP + 2],
                                              int N, const HistRef& h, uint32_t* gout, int agg,
                                              unsigned mask, int lane)
{
#define GLCM_CASE(D)                                                        \
    case D:                                                                 \
        if (gout)                                                           \
            vote_fast_global<BPP, D>(A, B, N, gout, mask, lane, agg);       \
        else if (agg)                                                       \
            vote_fast_agg<BPP, D>(A, B, N, h, mask, lane);                  \
        else                                                                \
            vote_fast<BPP, D>(A, B, N, h);                                  \
        break;
    switch (dx) {
        GLCM_CASE(-4)
        GLCM_CASE(-3)
        GLCM_CASE(-2)
        GLCM_CASE(-1)
        GLCM_CASE(0)
        GLCM_CASE(1)
        GLCM_CASE(2)
        GLCM_CASE(3)
        GLCM_CASE(4)
        default:
            break;
    }
#undef GLCM_CASE
}

// Sum the R copies of every word of the job's histograms into global counts,
// then zero them.  Called by the whole CTA between __syncthreads().
__device__ void flush_hist(const VoteJob& j, const VoteOffset* offs, uint32_t* hist)
{
    const int R = 1 << j.rshift;
    const int NN = j.levels * j.levels;
    const int groups = (j.n_off + j.pack - 1) / j.pack;
    const int rows = groups * NN;
    const int lane = threadIdx.x & 31;
    for (int w = threadIdx.x; w < rows; w += blockDim.x) {
        uint32_t lo = 0, hi = 0;
        uint32_t* base = hist + (long long)w * R;
        for (int r = 0; r < R; ++r) {
            const int c = (r + lane) & (R - 1);  // rotate so lanes hit distinct banks
            const uint32_t v = base[c];
            base[c] = 0u;
            if (j.pack == 2) {
                lo += v & 0xFFFFu;
                hi += v >> 16;
            } else {
                lo += v;
            }
        }
        const int g = w / NN;
        const int bin = w - g * NN;
        const int o0 = g * j.pack;
        if (lo)
            red_global_add(j.out + (long long)offs[j.off0 + o0].slot * NN + bin, lo);
        if (j.pack == 2 && hi && o0 + 1 < j.n_off)
            red_global_add(j.out + (long long)offs[j.off0 + o0 + 1].slot * NN + bin, hi);
    }
}

template <int BPP>
__device__ void process_item(const VoteJob& j, const VoteOffset* offs, const VoteItem& it, uint32_t* hist,
                             unsigned* err)
{
    constexpr int PX = 16 / BPP;
    constexpr int LW = PX / 4;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int xl = it.x0 + lane * PX;
    const int N = j.levels;
    const int NN = N * N;
    const bool global_direct = j.rshift < 0;
    const int R = global_direct ? 1 : (1 << j.rshift);
    const int c = lane & (R - 1);
    const uint32_t hbase = smem_u32(hist);
    // A lane may use registers for all its pairs when its 4-pixel halos exist.
    const bool lane_interior = j.aligned && xl >= 4 && xl + PX + 4 <= j.W;

    for (int y = it.y0 + warp; y < it.y1; y += nwarps) {
        bool bad_a = false;
        uint32_t A[LW];
        if (j.aligned)
            load_levels<BPP>(j, y, xl, A, bad_a);
        int cur_dy = 0x7fffffff;
        uint32_t B[LW + 2];
        bool bad_b = false;
        for (int o = 0; o < j.n_off; ++o) {
            const VoteOffset of = offs[j.off0 + o];
            const int yp = y + of.dy;
            if (yp < 0 || yp >= j.H)
                continue;
            HistRef h;
            uint32_t* gout = nullptr;
            if (global_direct) {
                gout = j.out + (long long)of.slot * NN;
                h.base = 0; h.inc = 1; h.stride = 0;
            } else {
                const int g = j.pack == 2 ? (o >> 1) : o;
                h.inc = (j.pack == 2 && (o & 1)) ? 0x10000u : 1u;
                h.stride = 4u * (uint32_t)R;
                h.base = hbase + 4u * (uint32_t)(g * NN * R + c);
            }
            const bool fast_dx = of.dx >= -kFastMaxDx && of.dx <= kFastMaxDx;
            if (j.aligned && of.dy != cur_dy) {
                // Partner row levels plus one 4-level halo word on each side.
                bad_b = false;
                uint32_t P[LW];
                if (of.dy == 0) {
#pragma unroll
                    for (int w = 0; w < LW; ++w) P[w] = A[w];
                    bad_b = bad_a;
                } else {
                    load_levels<BPP>(j, yp, xl, P, bad_b);
                }
                uint32_t left = __shfl_up_sync(0xffffffffu, P[LW - 1], 1);
                uint32_t right = __shfl_down_sync(0xffffffffu, P[0], 1);
                if (lane == 0 && xl >= 4)
                    left = load_group<BPP>(j, yp, xl - 4, bad_b);
                if (lane == 31 && xl + PX + 4 <= j.W)
                    right = load_group<BPP>(j, yp, xl + PX, bad_b);
                B[0] = left;
#pragma unroll
                for (int w = 0; w < LW; ++w) B[w + 1] = P[w];
                B[LW + 1] = right;
                cur_dy = of.dy;
            }
            // Neighbour halos may carry an out-of-range level: check them too.
            const bool bad_any = __any_sync(0xffffffffu, bad_b) || bad_a;
            const bool fast = lane_interior && fast_dx && !bad_a && !bad_b && !bad_any;
            const unsigned fmask = __ballot_sync(0xffffffffu, fast);
            if (fast) {
                dispatch_fast<BPP>(of.dx, A, B, N, h, gout, j.agg, fmask, lane);
            } else if (xl < j.W) {
                vote_slow(j, of.dx, of.dy, y, xl, PX, h, gout, err);
            }
        }
    }
}

template <int BPP>
__global__ void __launch_bounds__(kMaxThreads, 1) k_glcm_vote(VoteParams p)
{
    extern __shared__ __align__(16) uint32_t hist[];
    __shared__ int s_item, s_job;
    for (int i = threadIdx.x; i < p.max_hist_words; i += blockDim.x)
        hist[i] = 0u;
    int cur = -1;       // job whose partial histogram is in shared memory
    int acc = 0;        // rows per warp voted into 16-bit halves since the last merge
    __syncthreads();
    const int nwarps = blockDim.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            const int k = (int)atomicAdd(p.item_counter, 1u);
            int job = -1;
            if (k < p.n_items) {
                // Last job whose first item is <= k.
                int lo = 0, hi = p.n_jobs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (p.jobs[mid].item0 <= k)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                job = lo;
            }
            s_item = k;
            s_job = job;
        }
        __syncthreads();
        const int it_idx = s_item;
        if (it_idx >= p.n_items)
            break;
        const int job = s_job;
        const VoteJob j = p.jobs[job];
        VoteItem it;
        {
            const int local = it_idx - j.item0;
            const int band = local / j.n_strips;
            const int strip = local - band * j.n_strips;
            it.job = job;
            it.x0 = strip * 32 * (16 / j.bpp);
            it.y0 = j.y_begin + band * j.band_rows;
            it.y1 = min(j.y_end, it.y0 + j.band_rows);
        }
        const int rows_per_warp = (it.y1 - it.y0 + nwarps - 1) / nwarps;
        if (cur >= 0) {
            const VoteJob& cj = p.jobs[cur];
            bool need = cur != it.job;
            if (!need && cj.pack == 2 && cj.rshift >= 0) {
                // Bound the votes per 16-bit half: threads per copy x pixels.
                const long long per_half = (long long)(acc + rows_per_warp) * (16 / cj.bpp) *
                                           (blockDim.x >> cj.rshift);
                need = per_half > 65535;
            }
            if (need) {
                if (cj.rshift >= 0)
                    flush_hist(cj, p.offs, hist);
                __syncthreads();
                cur = -1;
                acc = 0;
            }
        }
        cur = it.job;
        acc += rows_per_warp;
        if (j.rshift >= 0 && j.hist_words > p.max_hist_words) {
            if (threadIdx.x == 0)
                atomicOr(p.err, kErrInternal);
        } else {
            process_item<BPP>(j, p.offs, it, hist, p.err);
        }
        __syncthreads();
    }
    if (cur >= 0 && p.jobs[cur].rshift >= 0)
        flush_hist(p.jobs[cur], p.offs, hist);
}

// Scheme 1 of the paper (Sec. I.B): one thread per anchor pixel, one global
// atomic per vote.  Kept as an ablation baseline.
__global__ void k_glcm_naive(const uint8_t* img, long long pitch, int W, int H, int bpp, int levels,
                             int levels_mode, int dx, int dy, uint32_t* out, unsigned* err)
{
    const long long n = (long long)W * H;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(t / W), x = (int)(t - (long long)y * W);
        const int x2 = x + dx, y2 = y + dy;
        if (x2 < 0 || x2 >= W || y2 < 0 || y2 >= H)
            continue;
        const uint8_t* r1 = img + (long long)y * pitch;
        const uint8_t* r2 = img + (long long)y2 * pitch;
        uint32_t v1, v2;
        if (bpp == 1) {
            v1 = r1[x];
            v2 = r2[x2];
        } else {
            v1 = r1[2 * x] | (r1[2 * x + 1] << 8);
            v2 = r2[2 * x2] | (r2[2 * x2 + 1] << 8);
        }
        uint32_t i = levels_mode ? v1 : (uint32_t)(((unsigned long long)v1 * levels) >> (8 * bpp));
        uint32_t j = levels_mode ? v2 : (uint32_t)(((unsigned long long)v2 * levels) >> (8 * bpp));
        if (i >= (uint32_t)levels || j >= (uint32_t)levels) {
            atomicOr(err, kErrRange);
            continue;
        }
        atomicAdd(out + i * levels + j, 1u);
    }
}

}  // namespace

int vote_max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Raise the dynamic shared-memory limit only when a launch needs more than
// before, so no attribute call happens while a stream is being captured.
template <int BPP>
static cudaError_t vote_prepare(size_t smem)
{
    static size_t set_to = 0;
    if (smem <= set_to)
        return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_glcm_vote<BPP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        set_to = smem;
    return e;
}

int vote_blocks_per_sm(int bpp, int threads, size_t smem)
{
    int n = 0;
    if (bpp == 1) {
        if (vote_prepare<1>(smem) != cudaSuccess)
            return 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_glcm_vote<1>, threads, smem);
    } else {
        if (vote_prepare<2>(smem) != cudaSuccess)
            return 1;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_glcm_vote<2>, threads, smem);
    }
    return n;
}

cudaError_t launch_vote(const VoteParams& p, int bpp, int grid, int threads, size_t smem, cudaStream_t s)
{
    cudaError_t e;
    if (bpp == 1) {
        if ((e = vote_prepare<1>(smem)) != cudaSuccess)
            return e;
        k_glcm_vote<1><<<grid, threads, smem, s>>>(p);
    } else {
        if ((e = vote_prepare<2>(smem)) != cudaSuccess)
            return e;
        k_glcm_vote<2><<<grid, threads, smem, s>>>(p);
    }
    return cudaGetLastError();
}

cudaError_t launch_naive(const uint8_t* img, long long pitch, int W, int H, int bpp, int levels, int levels_mode,
                         int dx, int dy, uint32_t* out, unsigned* err, cudaStream_t s)
{
    const long long n = (long long)W * H;
    int grid = (int)((n + 255) / 256);
    if (grid > 152 * 16)
        grid = 152 * 16;
    if (grid < 1)
        grid = 1;
    k_glcm_naive<<<grid, 256, 0, s>>>(img, pitch, W, H, bpp, levels, levels_mode, dx, dy, out, err);
    return cudaGetLastError();
}

}  // namespace glcm
