// GLCM vote kernels: quantize -> partner lookup -> vote -> merge.
//
// What is computed (Sec. I.A, Eq. 1): for every anchor pixel (x, y) whose
// partner (x + dx, y + dy) lies inside the image, with i and j the levels of
// the two pixels, P[i][j] += 1.  Partner addressing follows Eq. 2 with no
// pairing across the border, bins follow Eq. 3 with the anchor as the row.
//
// How (the paper's Scheme 2 copy strategy, Sec. II.A, redone for sm_103a):
//  * Persistent CTAs (one per SM, 1024 threads) each take a contiguous,
//    weight-balanced range of work items -- a strip of 32 lanes x 16 bytes
//    of one job and a band of rows -- so a CTA spans few jobs and merges
//    each once.  Each warp takes rows of the band; each lane owns 16 bytes of
//    a row (16 uint8 or 8 uint16 pixels), read with one 128-bit
//    non-coherent load and quantized in registers to packed level bytes.
//  * The partner row of each distinct dy is read the same way; the 4 levels
//    left and right of a lane come from its neighbours by shuffle, so every
//    |dx| <= 4 partner is a byte extraction from registers.
//  * Votes go into R private copies of the job's histograms in shared
//    memory, interleaved so that copy c of a bin is word c of the bin's
//    R-word row and lane l always uses copy l mod R: with R = 32 every lane
//    of a warp hits its own bank whatever the data (the paper's copies are
//    contiguous, so equal bins of different copies share a bank).
//    Layouts: (0) one R-word row per bin; (1) two offsets' rows interleaved
//    per bin (R = 32: a bin is 256 bytes, so a byte code c addresses its bin
//    as c << 8); (2) two offsets share each word as 16-bit halves -- the
//    host bounds the votes per half between merges below 65536.
//  * For N <= 16 (power of two) the 4 codes i*N + j of a word are formed
//    with one shift and one OR, and each vote is one byte permute, one add
//    and one shared-memory reduction.
//  * A job may count only the anchors whose level lies in [lv_lo, lv_lo +
//    lv_span): N = 256 histograms are split by anchor level so that each
//    part fits one CTA's shared memory.
//  * The merge (Sec. II.A, last step) sums the copies and adds each non-zero
//    bin into the global uint32 counts once per CTA and job.
//  * Warps touching an image edge vote with per-anchor validity masks;
//    unaligned images, |dx| > 4 and out-of-range pixels in levels mode take
//    a per-pixel path with full bounds checks.
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

// Levels of the 4 pixels starting at column x (x % 4 == 0); pixels outside
// [0, W) read as level 0 and are masked out by the callers.
template <int BPP>
__device__ __forceinline__ uint32_t load_group(const VoteJob& j, int y, int x, bool& bad)
{
    if (x < 0 || x >= j.W)
        return 0u;
    const uint8_t* p = j.img + (long long)y * j.pitch + (long long)x * BPP;
    if (x + 4 <= j.W) {
        if (BPP == 1)
            return quant_u8x4(j, __ldg(reinterpret_cast<const uint32_t*>(p)), bad);
        const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
        return quant_u16x4(j, q.x, q.y, bad);
    }
    // Ragged right edge: the 1..3 pixels inside, one at a time.
    uint32_t r = 0;
    for (int b = 0; b < 4 && x + b < j.W; ++b) {
        const uint32_t v = BPP == 1 ? (uint32_t)__ldg(p + b)
                                    : ((uint32_t)__ldg(p + 2 * b) | ((uint32_t)__ldg(p + 2 * b + 1) << 8));
        const uint32_t q = level_of(j, v);
        bad |= q >= (uint32_t)j.levels;
        r |= (q & 0xFFu) << (8 * b);
    }
    return r;
}

// Levels of pixels [xl, xl + PX) of row y as LW words (one 128-bit load when
// the whole lane lies inside the row).
template <int BPP>
__device__ __forceinline__ void load_levels(const VoteJob& j, int y, int xl, uint32_t (&L)[4 / BPP], bool& bad)
{
    constexpr int PX = 16 / BPP;
    constexpr int LW = PX / 4;
    if (xl + PX <= j.W) {
        const uint8_t* p = j.img + (long long)y * j.pitch + (long long)xl * BPP;
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
        for (int w = 0; w < LW; ++w)
            L[w] = load_group<BPP>(j, y, xl + 4 * w, bad);
    }
}

// Where offset o of a job votes: shared byte address of (bin 0, this lane's
// copy), bytes between bins, and the increment (1 or 1 << 16).
struct HistRef {
    uint32_t base;
    uint32_t stride;
    uint32_t inc;
};

__device__ __forceinline__ HistRef hist_ref(const VoteJob& j, int o, uint32_t hbase, int c)
{
    const uint32_t R = 1u << j.rshift;
    const uint32_t NNs = (uint32_t)j.lv_span * (uint32_t)j.levels;
    HistRef h;
    if (j.layout == 1) {
        h.base = hbase + 4u * (((uint32_t)(o >> 1) * NNs * 2u * R) + (uint32_t)(o & 1) * R + (uint32_t)c);
        h.stride = 8u * R;
        h.inc = 1u;
    } else if (j.layout == 2) {
        h.base = hbase + 4u * ((uint32_t)(o >> 1) * NNs * R + (uint32_t)c);
        h.stride = 4u * R;
        h.inc = (o & 1) ? 0x10000u : 1u;
    } else {
        h.base = hbase + 4u * ((uint32_t)o * NNs * R + (uint32_t)c);
        h.stride = 4u * R;
        h.inc = 1u;
    }
    return h;
}

// Fast vote of one lane's PX anchors for a compile-time dx.  With MASKED,
// only the anchors whose bit is set in `mask` vote (image edges).
template <int BPP, int DX, bool SPLIT, bool MASKED>
__device__ __forceinline__ void vote_fast(const uint32_t (&A)[4 / BPP], const uint32_t (&B)[4 / BPP + 2],
                                          uint32_t N, uint32_t lo, uint32_t span, const HistRef& h, uint32_t mask)
{
    constexpr int PX = 16 / BPP;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const uint32_t i = __byte_perm(A[k >> 2], 0u, 0x4440u | (uint32_t)(k & 3));
        const int t = k + DX + 4;  // byte of the extended partner row
        const uint32_t jv = __byte_perm(B[t >> 2], 0u, 0x4440u | (uint32_t)(t & 3));
        const bool on = !MASKED || ((mask >> k) & 1u);
        if (SPLIT) {
            const uint32_t ii = i - lo;
            if (on && ii < span)
                red_shared_add(h.base + (ii * N + jv) * h.stride, h.inc);
        } else if (on) {
            red_shared_add(h.base + (i * N + jv) * h.stride, h.inc);
        }
    }
}

// N <= 16, power of two, layout 1 with 32 copies: code = (i << L) | j is a
// byte and its bin starts at code << 8 bytes from the offset's base.
template <int BPP, int DX, bool MASKED>
__device__ __forceinline__ void vote_bytecode(const uint32_t (&A)[4 / BPP], const uint32_t (&B)[4 / BPP + 2],
                                             int L, uint32_t base, uint32_t mask)
{
    constexpr int LW = 4 / BPP;
#pragma unroll
    for (int m = 0; m < LW; ++m) {
        const int t = 4 * m + DX + 4;
        const int w0 = t >> 2, s = t & 3;
        const uint32_t pw = s == 0 ? B[w0] : __funnelshift_r(B[w0], B[w0 + 1], 8 * s);
        const uint32_t code = (A[m] << L) | pw;
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (!MASKED || ((mask >> (4 * m + b)) & 1u))
                red_shared_add(base + __byte_perm(code, 0u, 0x4404u | (uint32_t)(b << 4)), 1u);
    }
}

// Per-pixel path with full checks (unaligned images, wide dx, bad levels).
__device__ __forceinline__ void vote_slow(const VoteJob& j, int dx, int dy, int y, int xl, int px, const HistRef& h,
                          unsigned* err)
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
        const uint32_t ii = i - (uint32_t)j.lv_lo;
        if (ii >= (uint32_t)j.lv_span)
            continue;
        red_shared_add(h.base + (ii * N + jv) * h.stride, h.inc);
    }
}

template <int BPP, bool MASKED>
__device__ __forceinline__ void dispatch_fast(int dx, const uint32_t (&A)[4 / BPP], const uint32_t (&B)[4 / BPP + 2],
                                              const VoteJob& j, const HistRef& h, bool bytecode, uint32_t mask)
{
    const uint32_t N = (uint32_t)j.levels, lo = (uint32_t)j.lv_lo, span = (uint32_t)j.lv_span;
    const bool split = j.lv_span < j.levels;
#define GLCM_CASE(D)                                                        \
    case D:                                                                 \
        if (bytecode)                                                       \
            vote_bytecode<BPP, D, MASKED>(A, B, j.log2n, h.base, mask);     \
        else if (split)                                                     \
            vote_fast<BPP, D, true, MASKED>(A, B, N, lo, span, h, mask);    \
        else                                                                \
            vote_fast<BPP, D, false, MASKED>(A, B, N, lo, span, h, mask);   \
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

// Sum the R copies of every bin row of the job's histograms into the global
// counts, then zero them.  Called by the whole CTA between __syncthreads().
__device__ void flush_hist(const VoteJob& j, const VoteOffset* offs, uint32_t* hist)
{
    const int R = 1 << j.rshift;
    const int N = j.levels;
    const int NN = N * N;
    const int NNs = j.lv_span * N;
    const int rows = j.hist_words >> j.rshift;
    const int lane = threadIdx.x & 31;
    const int out_bin0 = j.lv_lo * N;
    for (int w = threadIdx.x; w < rows; w += blockDim.x) {
        uint32_t lo = 0, hi = 0;
        uint32_t* base = hist + (long long)w * R;
        for (int r = 0; r < R; ++r) {
            const int c = (r + lane) & (R - 1);  // rotate so lanes hit distinct banks
            const uint32_t v = base[c];
            base[c] = 0u;
            if (j.layout == 2) {
                lo += v & 0xFFFFu;
                hi += v >> 16;
            } else {
                lo += v;
            }
        }
        int o, bin;
        if (j.layout == 1) {
            const int pr = w >> 1;
            o = (pr / NNs) * 2 + (w & 1);
            bin = pr - (pr / NNs) * NNs;
        } else if (j.layout == 2) {
            o = (w / NNs) * 2;
            bin = w - (w / NNs) * NNs;
        } else {
            o = w / NNs;
            bin = w - o * NNs;
        }
        if (lo && o < j.n_off)
            red_global_add(j.out + (long long)offs[j.off0 + o].slot * NN + out_bin0 + bin, lo);
        if (j.layout == 2 && hi && o + 1 < j.n_off)
            red_global_add(j.out + (long long)offs[j.off0 + o + 1].slot * NN + out_bin0 + bin, hi);
    }
}

// Per-offset vote parameters of the current job, staged in shared memory.
struct OffInfo {
    int dx, dy;
    uint32_t base;    // shared byte address of (bin 0, copy 0)
    uint32_t inc;     // 1 or 1 << 16
};
constexpr int kMaxJobOffsets = 64;

// Raw (not yet quantized) bytes of one lane's row chunk and its halos.
struct RawRow {
    uint4 v;          // the lane's 16 bytes
    uint2 l, r;       // 4 pixels left / right of the lane (lanes 0 and 31 only)
};

// One warp's row task: anchor row y, lane columns [xl, xl + PX).
struct Task {
    int y, xl;
    bool valid;
};

template <int BPP>
__device__ __forceinline__ Task task_of(const VoteJob& j, int k0, int t)
{
    constexpr int PX = 16 / BPP;
    Task q;
    const int item = k0 + t / j.band_rows;
    const int rib = t - (t / j.band_rows) * j.band_rows;
    const int local = item - j.item0;
    const int band = local / j.n_strips;
    const int strip = local - band * j.n_strips;
    q.y = j.y_begin + band * j.band_rows + rib;
    q.xl = strip * 32 * PX + (threadIdx.x & 31) * PX;
    q.valid = q.y < j.y_end;
    return q;
}

// Issue the loads of a lane's full chunk (and lane 0/31 halos) of row y.
template <int BPP>
__device__ __forceinline__ void fetch_raw(const VoteJob& j, int y, int xl, RawRow& r)
{
    constexpr int PX = 16 / BPP;
    const int lane = threadIdx.x & 31;
    const uint8_t* row = j.img + (long long)y * j.pitch;
    r.v = make_uint4(0u, 0u, 0u, 0u);
    r.l = make_uint2(0u, 0u);
    r.r = make_uint2(0u, 0u);
    if (xl + PX <= j.W)
        r.v = ldg_v4(row + (long long)xl * BPP);
    if (lane == 0 && xl >= 4) {
        if (BPP == 1)
            r.l.x = __ldg(reinterpret_cast<const uint32_t*>(row + xl - 4));
        else
            r.l = __ldg(reinterpret_cast<const uint2*>(row + 2ll * (xl - 4)));
    }
    if (lane == 31 && xl + PX + 4 <= j.W) {
        if (BPP == 1)
            r.r.x = __ldg(reinterpret_cast<const uint32_t*>(row + xl + PX));
        else
            r.r = __ldg(reinterpret_cast<const uint2*>(row + 2ll * (xl + PX)));
    }
}

// Quantize a prefetched chunk into level words; lanes whose chunk is partial
// (right image edge) load their groups now, byte-exact.
template <int BPP>
__device__ __forceinline__ void levels_of_raw(const VoteJob& j, int y, int xl, const RawRow& r,
                                              uint32_t (&L)[4 / BPP], bool& bad)
{
    constexpr int PX = 16 / BPP;
    if (xl + PX <= j.W) {
        if (BPP == 1) {
            L[0] = quant_u8x4(j, r.v.x, bad);
            L[1 % (4 / BPP)] = quant_u8x4(j, r.v.y, bad);
            L[2 % (4 / BPP)] = quant_u8x4(j, r.v.z, bad);
            L[3 % (4 / BPP)] = quant_u8x4(j, r.v.w, bad);
        } else {
            L[0] = quant_u16x4(j, r.v.x, r.v.y, bad);
            L[1] = quant_u16x4(j, r.v.z, r.v.w, bad);
        }
    } else {
        load_levels<BPP>(j, y, xl, L, bad);
    }
}

template <int BPP>
__device__ __forceinline__ uint32_t halo_of_raw(const VoteJob& j, int y, int x, const uint2& raw, bool& bad)
{
    // Whole group inside the row: use the prefetched bytes; else exact loads.
    if (x >= 0 && x + 4 <= j.W)
        return BPP == 1 ? quant_u8x4(j, raw.x, bad) : quant_u16x4(j, raw.x, raw.y, bad);
    return load_group<BPP>(j, y, x, bad);
}

// Vote every offset of one row task.  A is the anchor row; PA/PB (raw) are
// the prefetched anchor row and first partner row (dy = dy1).
template <int BPP>
__device__ __forceinline__ void vote_task(const VoteJob& j, const OffInfo* s_off, int dy1, const Task& q,
                                          const RawRow& ra, const RawRow& rb, unsigned* err)
{
    constexpr int PX = 16 / BPP;
    constexpr int LW = PX / 4;
    const int lane = threadIdx.x & 31;
    const int xl = q.xl, y = q.y;
    const uint32_t cbytes = 4u * (uint32_t)(lane & ((1 << j.rshift) - 1));
    const uint32_t stride = (j.layout == 1 ? 8u : 4u) << j.rshift;
    const bool bytecode = j.bytecode != 0;
    const bool lane_interior = xl >= 4 && xl + PX + 4 <= j.W;
    const bool warp_interior = __all_sync(0xffffffffu, lane_interior);
    const int wrem = j.W - xl;
    bool bad_a = false;
    uint32_t A[LW];
    if (j.aligned)
        levels_of_raw<BPP>(j, y, xl, ra, A, bad_a);
    int cur_dy = 0x7fffffff;
    uint32_t B[LW + 2];
    bool bad_b = false;
    for (int o = 0; o < j.n_off; ++o) {
        const OffInfo of = s_off[o];
        const int yp = y + of.dy;
        if (yp < 0 || yp >= j.H)
            continue;
        HistRef h;
        h.base = of.base + cbytes;
        h.stride = stride;
        h.inc = of.inc;
        if (j.aligned && of.dy != cur_dy) {
            bad_b = false;
            uint32_t P[LW];
            uint32_t left, right;
            if (of.dy == 0) {
#pragma unroll
                for (int w = 0; w < LW; ++w)
                    P[w] = A[w];
                bad_b = bad_a;
                left = halo_of_raw<BPP>(j, yp, xl - 4, ra.l, bad_b);
                right = halo_of_raw<BPP>(j, yp, xl + PX, ra.r, bad_b);
            } else if (of.dy == dy1) {
                levels_of_raw<BPP>(j, yp, xl, rb, P, bad_b);
                left = halo_of_raw<BPP>(j, yp, xl - 4, rb.l, bad_b);
                right = halo_of_raw<BPP>(j, yp, xl + PX, rb.r, bad_b);
            } else {
                load_levels<BPP>(j, yp, xl, P, bad_b);
                left = load_group<BPP>(j, yp, xl - 4, bad_b);
                right = load_group<BPP>(j, yp, xl + PX, bad_b);
            }
            // Lanes 1..31 take their left halo from the lane before, lanes
            // 0..30 their right halo from the lane after.
            const uint32_t up = __shfl_up_sync(0xffffffffu, P[LW - 1], 1);
            const uint32_t down = __shfl_down_sync(0xffffffffu, P[0], 1);
            B[0] = lane == 0 ? left : up;
#pragma unroll
            for (int w = 0; w < LW; ++w)
                B[w + 1] = P[w];
            B[LW + 1] = lane == 31 ? right : down;
            cur_dy = of.dy;
        }
        bool fast = j.aligned && of.dx >= -kFastMaxDx && of.dx <= kFastMaxDx;
        if (j.levels_mode) {
            // Neighbour halos may carry an out-of-range level: check them too.
            const bool bad_any = __any_sync(0xffffffffu, bad_b || bad_a);
            fast = fast && !bad_any;
        }
        if (fast && warp_interior) {
            dispatch_fast<BPP, false>(of.dx, A, B, j, h, bytecode, 0u);
        } else if (fast) {
            // Anchors k with xl + k < W and 0 <= xl + k + dx < W.
            const int lo_k = max(0, -of.dx - xl);
            const int hi_k = min(min(PX, wrem), wrem - of.dx);
            const uint32_t mask = hi_k > lo_k ? (((1u << hi_k) - 1u) & ~((1u << lo_k) - 1u)) : 0u;
            dispatch_fast<BPP, true>(of.dx, A, B, j, h, bytecode, mask);
        } else if (xl < j.W) {
            vote_slow(j, of.dx, of.dy, y, xl, PX, h, err);
        }
    }
}

// All row tasks of items [ka, kb) of one job: warp w takes tasks w, w + nwarps,
// ...; the loads of its next task are issued before it votes the current one.
template <int BPP>
__device__ __forceinline__ void vote_segment(const VoteJob& j, int ka, int kb, const OffInfo* s_off, int dy1,
                                             unsigned* err)
{
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int n_tasks = (kb - ka) * j.band_rows;
    int t = warp;
    if (t >= n_tasks)
        return;
    Task q = task_of<BPP>(j, ka, t);
    RawRow ra, rb;
    const bool pre_b = dy1 != 0;
    if (q.valid && j.aligned) {
        fetch_raw<BPP>(j, q.y, q.xl, ra);
        if (pre_b && q.y + dy1 >= 0 && q.y + dy1 < j.H)
            fetch_raw<BPP>(j, q.y + dy1, q.xl, rb);
    }
    for (; t < n_tasks; t += nwarps) {
        const int tn = t + nwarps;
        Task qn;
        qn.valid = false;
        RawRow na, nb;
        if (tn < n_tasks) {
            qn = task_of<BPP>(j, ka, tn);
            if (qn.valid && j.aligned) {
                fetch_raw<BPP>(j, qn.y, qn.xl, na);
                if (pre_b && qn.y + dy1 >= 0 && qn.y + dy1 < j.H)
                    fetch_raw<BPP>(j, qn.y + dy1, qn.xl, nb);
            }
        }
        if (q.valid)
            vote_task<BPP>(j, s_off, dy1, q, ra, rb, err);
        q = qn;
        ra = na;
        rb = nb;
    }
}

// First item whose starting weight is >= w (items of a job all weigh w_item).
__device__ int item_at(const VoteParams& p, double w)
{
    if (w <= 0.0)
        return 0;
    if (w >= p.total_w)
        return p.n_items;
    int lo = 0, hi = p.n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.jobs[mid].w0 <= w)
            lo = mid;
        else
            hi = mid - 1;
    }
    const VoteJob& j = p.jobs[lo];
    long long k = (long long)ceil((w - j.w0) / (double)j.w_item);
    k = k < 0 ? 0 : (k > j.n_job_items ? j.n_job_items : k);
    return j.item0 + (int)k;
}

// Persistent CTAs with a static, weight-balanced partition: CTA b votes the
// contiguous item range covering weights [W b / G, W (b + 1) / G), so it
// touches only the few jobs that range spans and merges each once.
template <int BPP, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_glcm_vote(VoteParams p)
{
    extern __shared__ __align__(16) uint32_t hist[];
    __shared__ int s_k0, s_k1, s_job, s_dy1;
    __shared__ OffInfo s_off[kMaxJobOffsets];
    for (int i = threadIdx.x; i < p.max_hist_words; i += blockDim.x)
        hist[i] = 0u;
    if (threadIdx.x == 0) {
        const double W = p.total_w;
        s_k0 = item_at(p, W * (double)blockIdx.x / (double)gridDim.x);
        s_k1 = blockIdx.x + 1 == gridDim.x ? p.n_items
                                            : item_at(p, W * (double)(blockIdx.x + 1) / (double)gridDim.x);
        int lo = 0, hi = p.n_jobs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.jobs[mid].item0 <= s_k0)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_job = lo;
    }
    __syncthreads();
    const int k1 = s_k1;
    int k = s_k0;
    int job = s_job;
    const uint32_t hbase = smem_u32(hist);
    const int nwarps = blockDim.x >> 5;
    while (k < k1) {
        while (job + 1 < p.n_jobs && p.jobs[job + 1].item0 <= k)
            ++job;
        const VoteJob j = p.jobs[job];
        const int seg_end = min(k1, j.item0 + j.n_job_items);
        if (j.hist_words > p.max_hist_words || j.n_off > kMaxJobOffsets) {
            if (threadIdx.x == 0)
                atomicOr(p.err, kErrInternal);
            k = seg_end;
            continue;
        }
        // Stage the job's offsets (previous readers finished at the last barrier).
        if (threadIdx.x < j.n_off) {
            const VoteOffset vo = p.offs[j.off0 + threadIdx.x];
            const HistRef h = hist_ref(j, threadIdx.x, hbase, 0);
            s_off[threadIdx.x] = OffInfo{vo.dx, vo.dy, h.base, h.inc};
        }
        if (threadIdx.x == 0) {
            int d1 = 0;
            for (int o = 0; o < j.n_off && d1 == 0; ++o)
                d1 = p.offs[j.off0 + o].dy;
            s_dy1 = d1;
        }
        __syncthreads();
        // Items per merge: unbounded for 32-bit counters; 16-bit halves stay
        // below 65536 votes (rows per warp x pixels x threads per copy).
        int step = seg_end - k;
        if (j.layout == 2) {
            const long long rows_ok = 65535ll / ((16 / BPP) * (long long)(blockDim.x >> j.rshift));
            step = (int)max(1ll, min((long long)step, rows_ok * nwarps / j.band_rows));
        }
        for (int ka = k; ka < seg_end; ka += step) {
            const int kb = min(seg_end, ka + step);
            vote_segment<BPP>(j, ka, kb, s_off, s_dy1, p.err);
            __syncthreads();
            flush_hist(j, p.offs, hist);
            __syncthreads();
        }
        k = seg_end;
    }
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

// Raise the dynamic shared-memory limit only when a launch needs more than
// before, so no attribute call happens while a stream is being captured.
template <int BPP, int MAXT>
cudaError_t vote_prepare(size_t smem)
{
    static size_t set_to = 0;
    if (smem <= set_to)
        return cudaSuccess;
    cudaError_t e =
        cudaFuncSetAttribute(k_glcm_vote<BPP, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        set_to = smem;
    return e;
}

// Two register budgets: up to 1024 threads at 64 registers, or up to 512
// threads at 128 registers.
template <int BPP>
cudaError_t vote_launch_t(const VoteParams& p, int grid, int threads, size_t smem, cudaStream_t s, int* occ)
{
    cudaError_t e;
    if (threads > 512) {
        if ((e = vote_prepare<BPP, 1024>(smem)) != cudaSuccess)
            return e;
        if (occ)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_glcm_vote<BPP, 1024>, threads, smem);
        k_glcm_vote<BPP, 1024><<<grid, threads, smem, s>>>(p);
    } else {
        if ((e = vote_prepare<BPP, 512>(smem)) != cudaSuccess)
            return e;
        if (occ)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_glcm_vote<BPP, 512>, threads, smem);
        k_glcm_vote<BPP, 512><<<grid, threads, smem, s>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace

int vote_max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

int vote_blocks_per_sm(int bpp, int threads, size_t smem)
{
    int n = 0;
    cudaError_t e = bpp == 1 ? vote_launch_t<1>(VoteParams{}, 0, threads, smem, nullptr, &n)
                             : vote_launch_t<2>(VoteParams{}, 0, threads, smem, nullptr, &n);
    return e == cudaSuccess ? n : 1;
}

cudaError_t launch_vote(const VoteParams& p, int bpp, int grid, int threads, size_t smem, cudaStream_t s)
{
    return bpp == 1 ? vote_launch_t<1>(p, grid, threads, smem, s, nullptr)
                    : vote_launch_t<2>(p, grid, threads, smem, s, nullptr);
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
