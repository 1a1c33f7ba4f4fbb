// GLCM vote kernels: stage -> quantize -> partner lookup -> vote -> merge.
//
// What is computed (Sec. I.A, Eq. 1): for every anchor pixel (x, y) whose
// partner (x + dx, y + dy) lies inside the image, with i and j the levels of
// the two pixels, P[i][j] += 1.  Partner addressing follows Eq. 2 with no
// pairing across the border, bins follow Eq. 3 with the anchor as the row.
//
// How (the paper's Scheme 2 copy strategy, Sec. II.A, and its image
// partitioning with halo, Sec. III, redone for sm_103a):
//  * Work items are tiles: a strip of 512 bytes of a band of anchor rows of
//    one job (one image x one group of offsets x one anchor-level range).
//    Items are grouped host-side into chunks of consecutive items of one job;
//    persistent CTAs (one per SM) take chunk b first and then claim chunks
//    from a global counter, merging their histograms only when the job
//    changes.
//  * A tile is staged into shared memory by TMA bulk copies
//    (cp.async.bulk, one per row: 16 halo bytes + 512 + 16 halo bytes, plus
//    the halo rows the offsets' dy need), double-buffered and completed on
//    an mbarrier, so the copy of the next tile overlaps the votes of the
//    current one.  Images whose base or pitch is not 16-byte aligned are
//    staged by plain loads into the same layout.
//  * Each lane reads its 16 bytes of a row (16 uint8 or 8 uint16 pixels) and
//    the 4 pixels on each side from shared memory and quantizes them in
//    registers to packed level bytes (a shift and a mask per word for
//    power-of-two N); the partner words of an offset are one byte permute
//    each of the partner row's words.
//  * Votes go into R private copies of the job's histograms in shared
//    memory, interleaved so that copy c of a bin is word c of the bin's
//    R-word row and lane l uses copy l mod R: with R = 32 every lane of a
//    warp hits its own bank whatever the data (the paper's copies are
//    contiguous, so equal bins of different copies share a bank).
//    Layouts: (0) one R-word row per bin; (1) two offsets' rows interleaved
//    per bin (R = 32: a bin is 256 bytes, so a byte code c addresses its bin
//    as c << 8); (2) two offsets share each word as 16-bit halves -- the
//    merge comes before any half can reach 65536; (3) one offset's N bins of
//    anchor level i share H = ceil(N / 2) words as 16-bit halves, so the
//    65536 bins of N = 256 fit one CTA (128 KB) and an image takes one pass
//    per offset instead of one per offset and anchor-level part.  Partner
//    level j goes to position k = (j - i + floor(H / 2)) mod N: the lower
//    half of column k for k < H, the upper half of column k - H otherwise,
//    so the bins near the diagonal (flat regions, where many lanes hit one
//    word) take the constant increment 1.  Column kk of anchor level i is
//    word i * H + (kk + i) mod H: rotating each row spreads the lanes of a
//    smooth region (same kk, different i) over the banks, and a merge still
//    reads and writes along rows.  For power-of-two N the columns and half
//    bits of four votes come from byte-wise arithmetic on the packed level
//    words.  Every few tiles a spill pass
//    moves each half that reached 2^14 into the global counts, so no half
//    can wrap in between.  Layout 3 is compiled into its own kernel
//    instance (PACKED), so launches without it run the plain vote loop.
//  * For N <= 16 (power of two) the 4 codes i*N + j of a word come from one
//    shift and one OR; a vote is a byte permute, an add and a reduction.
//  * The merge (Sec. II.A, last step) sums the copies and adds each non-zero
//    bin into the global uint32 counts once per CTA and job.
//  * Edge lanes vote under per-anchor validity masks; |dx| > 4 and
//    out-of-range pixels in levels mode take a per-pixel path with full
//    bounds checks.  Every wait is bounded and reports a timeout bit.
#include "glcm_internal.cuh"

namespace glcm {
namespace {

constexpr int kStripBytes = 512;
constexpr int kHaloBytes = 16;
constexpr int kRowBytes = kStripBytes + 2 * kHaloBytes;
constexpr int kMaxJobOffsets = 64;
constexpr long long kTileWaitLimit = 1ll << 22;  // try_wait polls before a tile wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void red_shared_add(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Predicated reduction (no branch around it).
__device__ __forceinline__ void red_shared_add_if(uint32_t addr, uint32_t v, uint32_t on)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p red.shared.add.u32 [%0], %1;\n\t}" ::"r"(addr), "r"(v),
        "r"(on));
}

__device__ __forceinline__ void red_global_add(uint32_t* p, uint32_t v)
{
    asm volatile("red.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---- mbarrier + bulk copy (TMA) -------------------------------------------

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for phase `parity` of `bar`; false (and the timeout bit) if
// the limit is hit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* err)
{
    for (long long it = 0; it < kTileWaitLimit; ++it)
        if (mbar_try_wait(bar, parity))
            return true;
    atomicOr(err, kErrTimeout);
    return false;
}

// ---- levels ----------------------------------------------------------------

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

// Quantization of a job, set once per tile: N a power of two and pixels not
// already levels -- a shift and a mask per packed word.
struct Quant {
    bool fast;
    uint32_t shift, mask;
};

__device__ __forceinline__ Quant quant_of(const VoteJob& j)
{
    Quant q;
    q.fast = !j.levels_mode && j.log2n >= 0;
    q.shift = q.fast ? (uint32_t)(8 - j.log2n) : 0u;
    q.mask = 0x01010101u * (0xFFu >> q.shift);
    return q;
}

// 4 uint8 pixels -> 4 level bytes.  `bad` gets set if levels mode sees v >= N.
__device__ __forceinline__ uint32_t quant_u8x4(const VoteJob& j, const Quant& q, uint32_t w, bool& bad)
{
    if (q.fast)
        return (w >> q.shift) & q.mask;
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
__device__ __forceinline__ uint32_t quant_u16x4(const VoteJob& j, const Quant& q, uint32_t w0, uint32_t w1,
                                                bool& bad)
{
    if (q.fast)
        return (__byte_perm(w0, w1, 0x7531) >> q.shift) & q.mask;
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

// A staged row of the tile as this lane sees it: levels of its PX pixels
// (LW words) with one 4-level halo word on each side.
template <int BPP>
__device__ __forceinline__ void row_levels(const VoteJob& j, const Quant& q, const uint8_t* trow, int lane,
                                           uint32_t (&A)[4 / BPP], uint32_t& left, uint32_t& right, bool& bad)
{
    const uint8_t* c = trow + kHaloBytes + 16 * lane;
    const uint4 v = *reinterpret_cast<const uint4*>(c);
    if (BPP == 1) {
        A[0] = quant_u8x4(j, q, v.x, bad);
        A[1 % (4 / BPP)] = quant_u8x4(j, q, v.y, bad);
        A[2 % (4 / BPP)] = quant_u8x4(j, q, v.z, bad);
        A[3 % (4 / BPP)] = quant_u8x4(j, q, v.w, bad);
        left = quant_u8x4(j, q, *reinterpret_cast<const uint32_t*>(c - 4), bad);
        right = quant_u8x4(j, q, *reinterpret_cast<const uint32_t*>(c + 16), bad);
    } else {
        A[0] = quant_u16x4(j, q, v.x, v.y, bad);
        A[1] = quant_u16x4(j, q, v.z, v.w, bad);
        const uint2 l = *reinterpret_cast<const uint2*>(c - 8);
        const uint2 r = *reinterpret_cast<const uint2*>(c + 16);
        left = quant_u16x4(j, q, l.x, l.y, bad);
        right = quant_u16x4(j, q, r.x, r.y, bad);
    }
}

// Anchor levels only (no halos needed).
template <int BPP>
__device__ __forceinline__ void anchor_levels(const VoteJob& j, const Quant& q, const uint8_t* trow, int lane,
                                              uint32_t (&A)[4 / BPP], bool& bad)
{
    const uint4 v = *reinterpret_cast<const uint4*>(trow + kHaloBytes + 16 * lane);
    if (BPP == 1) {
        A[0] = quant_u8x4(j, q, v.x, bad);
        A[1 % (4 / BPP)] = quant_u8x4(j, q, v.y, bad);
        A[2 % (4 / BPP)] = quant_u8x4(j, q, v.z, bad);
        A[3 % (4 / BPP)] = quant_u8x4(j, q, v.w, bad);
    } else {
        A[0] = quant_u16x4(j, q, v.x, v.y, bad);
        A[1] = quant_u16x4(j, q, v.z, v.w, bad);
    }
}

// Partner level words aligned with the anchor words: PW[m] holds the levels
// of the partners of anchors 4m .. 4m + 3 for horizontal offset dx in
// [-4, 4].  Byte t = 4m + dx + 4 of the extended row [left, B..., right] is
// the partner of anchor byte 4m; with t0 = dx + 4 = 4 hi + sh (hi in {0, 1},
// sh in [0, 4]) it is byte sh of the word pair (B[m + hi], B[m + hi + 1]),
// so each word is one byte permute with selector 0x3210 + 0x1111 sh.  hi and
// the selector are set once per offset.
__device__ __forceinline__ int2 partner_sel(int dx)
{
    const int t0 = dx + 4;
    const int hi = t0 >= 4 ? 1 : 0;
    return make_int2(hi, 0x3210 + 0x1111 * (t0 - 4 * hi));
}

template <int BPP>
__device__ __forceinline__ void partner_words(int2 ps, const uint32_t (&B)[4 / BPP + 2], uint32_t (&PW)[4 / BPP])
{
    constexpr int LW = 4 / BPP;
#pragma unroll
    for (int m = 0; m < LW; ++m) {
        const uint32_t lo = ps.x ? B[m + 1] : B[m];
        const uint32_t hi = ps.x ? B[m + 2] : B[m + 1];
        PW[m] = __byte_perm(lo, hi, (uint32_t)ps.y);
    }
}

// Byte-wise arithmetic on four packed levels, no carry or borrow between
// bytes: (x - y) mod 256, and (d + q) mod 256 for q < 128.
__device__ __forceinline__ uint32_t bytes_sub(uint32_t x, uint32_t y)
{
    return ((x | 0x80808080u) - (y & 0x7F7F7F7Fu)) ^ ((x ^ ~y) & 0x80808080u);
}

__device__ __forceinline__ uint32_t bytes_add_small(uint32_t d, uint32_t qq)
{
    return ((d & 0x7F7F7F7Fu) + qq) ^ (d & 0x80808080u);
}

// Where offset o of a job votes: shared byte address of (bin 0, copy 0),
// bytes between bins (between words in layout 3), and the increment (1 or
// 1 << 16; layout 3 picks it per vote).
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
    } else if (j.layout == 3) {
        const uint32_t Hh = ((uint32_t)j.levels + 1u) >> 1;
        h.base = hbase + 4u * ((uint32_t)o * (uint32_t)j.lv_span * Hh * R + (uint32_t)c);
        h.stride = 4u * R;
        h.inc = 0u;
    } else {
        h.base = hbase + 4u * ((uint32_t)o * NNs * R + (uint32_t)c);
        h.stride = 4u * R;
        h.inc = 1u;
    }
    return h;
}

// Votes of one lane's PX anchors against partner words PW.  FULL: every
// anchor votes; else only those whose bit is set in `mask` (image edges).
// BYTECODE: N <= 16 power of two, 32 interleaved copies, one byte per code.
// SPLIT: only anchors with level in [lo, lo + span) vote.
// INC1: the increment is the constant 1 (every layout but the upper halves of
// layout 2), which lets lanes of a warp that hit the same word be combined
// into one update instead of serializing.
// PACK: layout 3 (P2: N is a power of two).
template <int BPP, bool BYTECODE, bool SPLIT, bool FULL, bool INC1, bool PACK = false, bool P2 = false>
__device__ __forceinline__ void vote_words(const VoteJob& j, const uint32_t (&A)[4 / BPP],
                                           const uint32_t (&PW)[4 / BPP], const HistRef& h, uint32_t mask)
{
    constexpr int LW = 4 / BPP;
    if (BYTECODE) {
        const int L = j.log2n;
#pragma unroll
        for (int m = 0; m < LW; ++m) {
            const uint32_t code = (A[m] << L) | PW[m];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t addr = h.base + __byte_perm(code, 0u, 0x4404u | (uint32_t)(b << 4));
                if (FULL)
                    red_shared_add(addr, 1u);
                else
                    red_shared_add_if(addr, 1u, (mask >> (4 * m + b)) & 1u);
            }
        }
        return;
    }
    const uint32_t N = (uint32_t)j.levels, lo = (uint32_t)j.lv_lo, span = (uint32_t)j.lv_span;
    if constexpr (PACK && P2 && !SPLIT) {
        // Power-of-two N, whole level range: the packed column (j + q) mod H
        // and the half bit (bit log2(H) of (j - i + q) mod N) of four votes at
        // a time, byte-wise (N divides 256, so byte arithmetic mod 256 keeps
        // the low bits right).  A warp row with no upper-half vote among its
        // active votes reduces with the constant 1, the others with a per-vote
        // increment.
        const uint32_t Hh = N >> 1, q = Hh >> 1, lh = (uint32_t)j.log2n - 1u;
        const uint32_t Mh = (Hh - 1u) * 0x01010101u, qq = q * 0x01010101u;
        uint32_t U4[LW], anyu = 0u, addr[4 * LW];
#pragma unroll
        for (int m = 0; m < LW; ++m) {
            const uint32_t C4 = ((PW[m] & Mh) + qq) & Mh;
            U4[m] = (bytes_add_small(bytes_sub(PW[m], A[m]), qq) >> lh) & 0x01010101u;
            // Active votes of this word as bytes (the 4 mask bits spread to bits 0, 8, 16, 24).
            const uint32_t act = FULL ? 0x01010101u : (((mask >> (4 * m)) & 0xFu) * 0x00204081u) & 0x01010101u;
            anyu |= U4[m] & act;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t i = __byte_perm(A[m], 0u, 0x4440u | (uint32_t)b);
                const uint32_t c = __byte_perm(C4, 0u, 0x4440u | (uint32_t)b);
                addr[4 * m + b] = h.base + (i * Hh + c) * h.stride;
            }
        }
        // All addresses first, then the reductions back to back: lanes that
        // share a word in a flat region combine best that way (measured).
        if (!__any_sync(0xffffffffu, anyu != 0u)) {
#pragma unroll
            for (int v = 0; v < 4 * LW; ++v) {
                if (FULL)
                    red_shared_add(addr[v], 1u);
                else
                    red_shared_add_if(addr[v], 1u, (mask >> v) & 1u);
            }
        } else {
#pragma unroll
            for (int v = 0; v < 4 * LW; ++v) {
                const uint32_t up = (U4[v >> 2] >> (8 * (v & 3))) & 1u;
                const uint32_t on = FULL ? 1u : ((mask >> v) & 1u);
                red_shared_add_if(addr[v], up ? 0x10000u : 1u, on);
            }
        }
        return;
    } else if constexpr (PACK) {
        // Addresses and upper-half bits of the lane's votes first; a warp row
        // with no upper-half vote (flat and smooth regions) reduces with the
        // constant 1, so lanes that hit one word combine, the others with a
        // per-vote increment.
        const uint32_t Hh = (N + 1u) >> 1, q = Hh >> 1;
        const uint32_t lh = P2 ? (uint32_t)j.log2n - 1u : 0u;  // log2(H)
        const uint32_t cq = q - lo;                              // mod H below (P2)
        uint32_t addr[4 * LW];
        uint32_t upm = 0u, onm = FULL ? 0xFFFFFFFFu : mask;
#pragma unroll
        for (int m = 0; m < LW; ++m) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t i = __byte_perm(A[m], 0u, 0x4440u | (uint32_t)b);
                const uint32_t jv = __byte_perm(PW[m], 0u, 0x4440u | (uint32_t)b);
                const uint32_t ii = SPLIT ? i - lo : i;
                if (SPLIT && ii >= span)
                    onm &= ~(1u << (4 * m + b));
                const uint32_t t = jv + q - i;
                uint32_t up, c;
                if (P2) {
                    // H divides N: (k mod H + ii) mod H = (j + q - lo) mod H,
                    // and the half is bit log2(H) of j - i + q.
                    up = (t >> lh) & 1u;
                    c = (jv + cq) & (Hh - 1u);
                } else {
                    uint32_t k = (int)t < 0 ? t + N : t;
                    k = k >= N ? k - N : k;
                    up = k >= Hh ? 1u : 0u;
                    c = (up ? k - Hh : k) + ii;
                    c = c >= Hh ? c - Hh : c;
                    c = c >= Hh ? c - Hh : c;
                }
                upm |= up << (4 * m + b);
                addr[4 * m + b] = h.base + (ii * Hh + c) * h.stride;
            }
        }
        if (!__any_sync(0xffffffffu, (upm & onm) != 0u)) {
#pragma unroll
            for (int v = 0; v < 4 * LW; ++v) {
                if (FULL && !SPLIT)
                    red_shared_add(addr[v], 1u);
                else
                    red_shared_add_if(addr[v], 1u, (onm >> v) & 1u);
            }
        } else {
#pragma unroll
            for (int v = 0; v < 4 * LW; ++v)
                red_shared_add_if(addr[v], ((upm >> v) & 1u) ? 0x10000u : 1u, (onm >> v) & 1u);
        }
        return;
    } else {
#pragma unroll
        for (int m = 0; m < LW; ++m) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t i = __byte_perm(A[m], 0u, 0x4440u | (uint32_t)b);
                const uint32_t jv = __byte_perm(PW[m], 0u, 0x4440u | (uint32_t)b);
                const uint32_t ii = SPLIT ? i - lo : i;
                const uint32_t addr = h.base + (ii * N + jv) * h.stride;
                const uint32_t inc = INC1 ? 1u : h.inc;
                if (FULL && !SPLIT) {
                    red_shared_add(addr, inc);
                } else {
                    uint32_t on = FULL ? 1u : ((mask >> (4 * m + b)) & 1u);
                    if (SPLIT)
                        on &= ii < span ? 1u : 0u;
                    red_shared_add_if(addr, inc, on);
                }
            }
        }
    }
}

template <int BPP, bool SPLIT, bool FULL>
__device__ __forceinline__ void vote_words_packed(const VoteJob& j, const uint32_t (&A)[4 / BPP],
                                                  const uint32_t (&PW)[4 / BPP], const HistRef& h, uint32_t mask)
{
    if (j.log2n >= 0)
        vote_words<BPP, false, SPLIT, FULL, false, true, true>(j, A, PW, h, mask);
    else
        vote_words<BPP, false, SPLIT, FULL, false, true, false>(j, A, PW, h, mask);
}

template <int BPP, bool INC1, bool PACKED>
__device__ __forceinline__ void vote_words_inc(const VoteJob& j, const uint32_t (&A)[4 / BPP],
                                               const uint32_t (&PW)[4 / BPP], const HistRef& h, uint32_t mask,
                                               bool full)
{
    const bool split = j.lv_span < j.levels;
    if (PACKED && j.layout == 3) {
        if (split) {
            if (full)
                vote_words_packed<BPP, true, true>(j, A, PW, h, mask);
            else
                vote_words_packed<BPP, true, false>(j, A, PW, h, mask);
        } else {
            if (full)
                vote_words_packed<BPP, false, true>(j, A, PW, h, mask);
            else
                vote_words_packed<BPP, false, false>(j, A, PW, h, mask);
        }
    } else if (j.bytecode) {
        if (full)
            vote_words<BPP, true, false, true, true>(j, A, PW, h, mask);
        else
            vote_words<BPP, true, false, false, true>(j, A, PW, h, mask);
    } else if (split) {
        if (full)
            vote_words<BPP, false, true, true, INC1>(j, A, PW, h, mask);
        else
            vote_words<BPP, false, true, false, INC1>(j, A, PW, h, mask);
    } else {
        if (full)
            vote_words<BPP, false, false, true, INC1>(j, A, PW, h, mask);
        else
            vote_words<BPP, false, false, false, INC1>(j, A, PW, h, mask);
    }
}

template <int BPP, bool PACKED>
__device__ __forceinline__ void vote_words_dispatch(const VoteJob& j, const uint32_t (&A)[4 / BPP],
                                                    const uint32_t (&PW)[4 / BPP], const HistRef& h,
                                                    uint32_t mask, bool full)
{
    if (h.inc == 1u || (PACKED && j.layout == 3))
        vote_words_inc<BPP, true, PACKED>(j, A, PW, h, mask, full);
    else
        vote_words_inc<BPP, false, PACKED>(j, A, PW, h, mask, full);
}

// Per-pixel path with full checks (|dx| > 4, bad levels): reads the image.
__device__ __noinline__ void vote_slow(const VoteJob* __restrict__ jp, int dx, int dy, int y, int xl, int px,
                                       HistRef h, unsigned* err)
{
    const VoteJob& j = *jp;
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
        if (j.layout == 3) {
            const uint32_t Hh = (N + 1u) >> 1;
            const uint32_t k = (jv + N + (Hh >> 1) - i) % N;
            const bool up = k >= Hh;
            const uint32_t c = ((up ? k - Hh : k) + ii) % Hh;
            red_shared_add(h.base + (ii * Hh + c) * h.stride, up ? 0x10000u : 1u);
        } else {
            red_shared_add(h.base + (ii * N + jv) * h.stride, h.inc);
        }
    }
}

// Sum the R copies of every bin row of the job's histograms into the global
// counts, then zero them.  Called by the whole CTA between __syncthreads().
__device__ void flush_hist(const VoteJob& j, const VoteOffset* offs, uint32_t* hist)
{
    const int R = 1 << j.rshift;
    const int N = j.levels;
    const long long NN = (long long)N * N;
    const int NNs = j.lv_span * N;
    const int rows = j.hist_words >> j.rshift;
    const int lane = threadIdx.x & 31;
    const int out_bin0 = j.lv_lo * N;
    // Row w of the histograms is bin `bin` of offset group g: layout 1 pairs
    // two offsets' rows (w = 2 (g NNs + bin) + parity), the others have one
    // row per bin.  Advanced incrementally, without a division per row.
    const int per = j.layout == 1 ? 2 : 1;
    const int par = (int)threadIdx.x % per;
    const int step = (int)blockDim.x / per;
    int u = (int)threadIdx.x / per;
    int g = u / NNs, bin = u - g * NNs;
    int cur_o = -1;
    uint32_t* dst_lo = nullptr;
    uint32_t* dst_hi = nullptr;
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
        const int o = j.layout == 1 ? 2 * g + par : (j.layout == 2 ? 2 * g : g);
        if (o != cur_o) {
            cur_o = o;
            dst_lo = o < j.n_off ? j.out + (long long)offs[j.off0 + o].slot * NN + out_bin0 : nullptr;
            dst_hi = (j.layout == 2 && o + 1 < j.n_off)
                         ? j.out + (long long)offs[j.off0 + o + 1].slot * NN + out_bin0
                         : nullptr;
        }
        if (lo && dst_lo)
            red_global_add(dst_lo + bin, lo);
        if (hi && dst_hi)
            red_global_add(dst_hi + bin, hi);
        bin += step;
        while (bin >= NNs) {
            bin -= NNs;
            ++g;
        }
    }
}

// Partner level of position k in anchor level i's packed row (layout 3).
__device__ __forceinline__ int packed_partner(int k, int i, int N, int Hh)
{
    int jv = k + i - (Hh >> 1);
    jv = jv < 0 ? jv + N : jv;
    return jv >= N ? jv - N : jv;
}

// Layout 3: the same for packed halves.  Row w of the job's words is word
// (g * span + ii) * H + c of offset g, anchor level lv_lo + ii: positions
// kk = (c - ii) mod H (lower half) and kk + H (upper half).  Advanced
// incrementally, without a division per row.
__device__ void flush_hist_packed(const VoteJob& j, const VoteOffset* offs, uint32_t* hist)
{
    const int R = 1 << j.rshift;
    const int N = j.levels, Hh = (N + 1) >> 1, span = j.lv_span;
    const long long NN = (long long)N * N;
    const int rows = j.hist_words >> j.rshift;
    const int lane = threadIdx.x & 31;
    const int T = (int)blockDim.x;
    const int sq = T / Hh, sr = T - sq * Hh;
    const int q0 = (int)threadIdx.x / Hh;
    int c = (int)threadIdx.x - q0 * Hh;
    int g = q0 / span;
    int ii = q0 - g * span;
    const bool p2 = j.log2n >= 0;
    int cur_g = -1;
    uint32_t* dst = nullptr;
    for (int w = threadIdx.x; w < rows; w += T) {
        uint32_t lo = 0, hi = 0;
        uint32_t* base = hist + (long long)w * R;
        for (int r = 0; r < R; ++r) {
            const int cc = (r + lane) & (R - 1);  // rotate so lanes hit distinct banks
            const uint32_t v = base[cc];
            base[cc] = 0u;
            lo += v & 0xFFFFu;
            hi += v >> 16;
        }
        if (g != cur_g) {
            cur_g = g;
            dst = g < j.n_off ? j.out + (long long)offs[j.off0 + g].slot * NN + (long long)j.lv_lo * N : nullptr;
        }
        if (dst && (lo | hi)) {
            const int lvl = j.lv_lo + ii;
            int kk;
            if (p2) {
                kk = (c - ii) & (Hh - 1);
            } else {
                kk = c - ii % Hh;
                kk += kk < 0 ? Hh : 0;
            }
            if (lo)
                red_global_add(dst + ii * N + packed_partner(kk, lvl, N, Hh), lo);
            if (hi && kk + Hh < N)
                red_global_add(dst + ii * N + packed_partner(kk + Hh, lvl, N, Hh), hi);
        }
        if (w + T < rows) {
            c += sr;
            ii += sq;
            if (c >= Hh) {
                c -= Hh;
                ++ii;
            }
            while (ii >= span) {
                ii -= span;
                ++g;
            }
        }
    }
}

// Layout 3 spill threshold: a half at or above 2^14 is moved to the global
// counts, so the halves left are below 2^14 and the next tiles may add up to
// 65535 - 16383 = 49152 votes to a half before the next spill.
constexpr uint32_t kSpillMask = 0xC000C000u;
constexpr int kSpillVotes = 49152;

__device__ void spill_word(const VoteJob& j, const VoteOffset* offs, uint32_t* hist, int w)
{
    const uint32_t v = hist[w];
    if ((v & kSpillMask) == 0u)
        return;
    const int N = j.levels, Hh = (N + 1) >> 1;
    const int row = w >> j.rshift;
    const int q = row / Hh, c = row - q * Hh;
    const int g = q / j.lv_span, ii = q - g * j.lv_span;
    int kk = c - ii % Hh;
    kk += kk < 0 ? Hh : 0;
    if (g >= j.n_off)
        return;
    const int lvl = j.lv_lo + ii;
    uint32_t* dst = j.out + (long long)offs[j.off0 + g].slot * ((long long)N * N) + (long long)lvl * N;
    uint32_t keep = v;
    if (v & (kSpillMask & 0xFFFFu)) {
        red_global_add(dst + packed_partner(kk, lvl, N, Hh), v & 0xFFFFu);
        keep &= 0xFFFF0000u;
    }
    if ((v & (kSpillMask & 0xFFFF0000u)) && kk + Hh < N) {
        red_global_add(dst + packed_partner(kk + Hh, lvl, N, Hh), v >> 16);
        keep &= 0xFFFFu;
    }
    hist[w] = keep;
}

// Layout 3: spill the halves at or above 2^14 (one 16-byte read per four
// words; almost every word is below).  Called by the whole CTA between
// __syncthreads().
__device__ void spill_hist_packed(const VoteJob& j, const VoteOffset* offs, uint32_t* hist)
{
    const int words = j.hist_words;
    const uint4* h4 = reinterpret_cast<const uint4*>(hist);
    for (int q = threadIdx.x; q < (words >> 2); q += blockDim.x) {
        const uint4 v = h4[q];
        if (((v.x | v.y | v.z | v.w) & kSpillMask) == 0u)
            continue;
        for (int e = 0; e < 4; ++e)
            spill_word(j, offs, hist, 4 * q + e);
    }
    for (int w = (words & ~3) + (int)threadIdx.x; w < words; w += blockDim.x)
        spill_word(j, offs, hist, w);
}

template <bool PACKED>
__device__ __forceinline__ void flush_any(const VoteJob& j, const VoteOffset* offs, uint32_t* hist)
{
    if (PACKED && j.layout == 3)
        flush_hist_packed(j, offs, hist);
    else
        flush_hist(j, offs, hist);
}

// ---- tiles -------------------------------------------------------------------

struct Tile {
    int x0;          // first anchor column
    int y0, y1;      // anchor rows
    int ty0, ty1;    // image rows staged (anchor rows plus the dy halo)
};

__device__ __forceinline__ Tile tile_of(const VoteJob& j, int k)
{
    Tile t;
    const int local = k - j.item0;
    const int band = local / j.n_strips;
    const int strip = local - band * j.n_strips;
    t.x0 = strip * (kStripBytes / j.bpp);
    t.y0 = j.y_begin + band * j.band_rows;
    t.y1 = min(j.y_end, t.y0 + j.band_rows);
    t.ty0 = max(0, t.y0 + j.dy_min);
    t.ty1 = min(j.H, t.y1 + j.dy_max);
    return t;
}

// Issue the bulk copies of a tile into `buf` (warp 0): each staged row is the
// 16-byte-aligned byte range [x0*bpp - 16, x0*bpp + 528) clipped to the row's
// 16-byte-rounded width.  Lane 0 announces the byte count first.
__device__ __forceinline__ void issue_tile(const VoteJob& j, const Tile& t, uint8_t* buf, uint64_t* bar)
{
    const int lane = threadIdx.x & 31;
    const int xb = t.x0 * j.bpp - kHaloBytes;
    const int row_end = ((j.W * j.bpp) + 15) & ~15;
    const int cb0 = max(0, xb), cb1 = min(row_end, xb + kRowBytes);
    const int bytes = max(0, cb1 - cb0);
    const int rows = max(0, t.ty1 - t.ty0);
    if (lane == 0)
        mbar_arrive_expect_tx(bar, (uint32_t)(bytes * rows));
    __syncwarp();
    if (bytes > 0) {
        for (int r = lane; r < rows; r += 32) {
            const uint8_t* src = j.img + (long long)(t.ty0 + r) * j.pitch + cb0;
            bulk_copy_g2s(buf + r * kRowBytes + (cb0 - xb), src, (uint32_t)bytes, bar);
        }
    }
}

// Unaligned images: the whole CTA copies the tile with plain loads.
__device__ void fill_tile_plain(const VoteJob& j, const Tile& t, uint8_t* buf)
{
    const int xb = t.x0 * j.bpp - kHaloBytes;
    const int row_bytes = j.W * j.bpp;
    const int rows = max(0, t.ty1 - t.ty0);
    for (int e = threadIdx.x; e < rows * kRowBytes; e += blockDim.x) {
        const int r = e / kRowBytes, b = e - r * kRowBytes;
        const int col = xb + b;
        uint8_t v = 0;
        if (col >= 0 && col < row_bytes)
            v = __ldg(j.img + (long long)(t.ty0 + r) * j.pitch + col);
        buf[e] = v;
    }
}

// Votes of one staged tile: warp w takes anchor rows y0 + w, y0 + w + nwarps, ...
template <int BPP, bool PACKED>
__device__ __forceinline__ void vote_tile(const VoteJob& j, const VoteJob* jg, const Tile& t, const uint8_t* buf,
                                          const HistRef* s_off_h, const int4* s_off_d, unsigned* err)
{
    constexpr int PX = 16 / BPP;
    constexpr int LW = PX / 4;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int xl = t.x0 + lane * PX;
    const uint32_t cbytes = 4u * (uint32_t)(lane & ((1 << j.rshift) - 1));
    const bool lane_interior = xl >= 4 && xl + PX + 4 <= j.W;
    const bool full = __all_sync(0xffffffffu, lane_interior);
    const int wrem = j.W - xl;
    const Quant q = quant_of(j);
    for (int y = t.y0 + warp; y < t.y1; y += nwarps) {
        bool bad_a = false;
        uint32_t A[LW];
        anchor_levels<BPP>(j, q, buf + (y - t.ty0) * kRowBytes, lane, A, bad_a);
        int cur_dy = 0x7fffffff;
        uint32_t B[LW + 2];
        bool bad_b = false;
        for (int o = 0; o < j.n_off; ++o) {
            const int4 d = s_off_d[o];  // dx, dy, partner word pair, byte selector
            const int yp = y + d.y;
            if (yp < 0 || yp >= j.H)
                continue;
            HistRef h = s_off_h[o];
            h.base += cbytes;
            if (d.y != cur_dy) {
                bad_b = false;
                uint32_t P[LW];
                row_levels<BPP>(j, q, buf + (yp - t.ty0) * kRowBytes, lane, P, B[0], B[LW + 1], bad_b);
#pragma unroll
                for (int w = 0; w < LW; ++w)
                    B[w + 1] = P[w];
                cur_dy = d.y;
            }
            bool fast = d.x >= -kFastMaxDx && d.x <= kFastMaxDx;
            if (j.levels_mode) {
                // A neighbour's halo may carry an out-of-range level: check all.
                fast = fast && !__any_sync(0xffffffffu, bad_a || bad_b);
            }
            if (fast) {
                uint32_t PW[LW];
                partner_words<BPP>(make_int2(d.z, d.w), B, PW);
                uint32_t mask = 0xFFFFu;
                if (!full) {
                    // Anchors k with xl + k < W and 0 <= xl + k + dx < W.
                    const int lo_k = max(0, -d.x - xl);
                    const int hi_k = min(min(PX, wrem), wrem - d.x);
                    mask = hi_k > lo_k ? (((1u << hi_k) - 1u) & ~((1u << lo_k) - 1u)) : 0u;
                }
                vote_words_dispatch<BPP, PACKED>(j, A, PW, h, mask, full);
            } else if (xl < j.W) {
                vote_slow(jg, d.x, d.y, y, xl, PX, h, err);
            }
        }
    }
}

// Jobs whose offsets span too many rows to stage: per-pixel votes only.
template <int BPP>
__device__ void vote_tile_unstaged(const VoteJob& j, const VoteJob* jg, const Tile& t, const HistRef* s_off_h,
                                   const int4* s_off_d, unsigned* err)
{
    constexpr int PX = 16 / BPP;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int xl = t.x0 + lane * PX;
    const uint32_t cbytes = 4u * (uint32_t)(lane & ((1 << j.rshift) - 1));
    if (xl >= j.W)
        return;
    for (int y = t.y0 + warp; y < t.y1; y += nwarps)
        for (int o = 0; o < j.n_off; ++o) {
            HistRef h = s_off_h[o];
            h.base += cbytes;
            vote_slow(jg, s_off_d[o].x, s_off_d[o].y, y, xl, PX, h, err);
        }
}

// Persistent CTAs pull chunks -- runs of consecutive items of one job, sized
// on the host so that a chunk's votes outweigh its merge -- from a global
// counter.  Chunks are ordered job by job, so a CTA usually stays on one job
// for several chunks and merges only when its job changes; pulling them
// dynamically balances images whose contention makes items cost very
// different times.  Dynamic shared memory: two tile buffers, then the
// histograms.
template <int BPP, int MAXT, bool PACKED>
__global__ void __launch_bounds__(MAXT, 1) k_glcm_vote(VoteParams p)
{
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int s_chunk, s_ok;
    __shared__ HistRef s_off_h[kMaxJobOffsets];
    __shared__ int4 s_off_d[kMaxJobOffsets];
    uint8_t* tiles = smem;
    uint32_t* hist = reinterpret_cast<uint32_t*>(smem + 2 * p.tile_bytes);
    for (int i = threadIdx.x; i < p.max_hist_words; i += blockDim.x)
        hist[i] = 0u;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_ok = 1;
    }
    __syncthreads();
    const uint32_t hbase = smem_u32(hist);
    const int nwarps = blockDim.x >> 5;
    uint32_t uses[2] = {0u, 0u};  // completed phases per tile buffer
    int cur = -1;                 // job whose partial histograms are in shared memory
    long long acc_rows = 0;       // rows per warp voted into 16-bit halves since the last merge
    int spill_rows = 0;           // anchor rows voted into packed halves (layout 3) since the last spill
    // Chunk b goes to CTA b; later chunks are claimed from the counter.
    bool first = true;
    for (;;) {
        if (threadIdx.x == 0)
            s_chunk = first ? (int)blockIdx.x : (int)gridDim.x + (int)atomicAdd(p.item_counter, 1u);
        first = false;
        __syncthreads();
        const int c = s_chunk;
        if (c >= p.n_chunks)
            break;
        const int3 ch = p.chunks[c];
        const VoteJob* jg = p.jobs + ch.x;
        const VoteJob j = *jg;
        const int tile_need = j.staged ? (j.band_rows + j.dy_max - j.dy_min) * kRowBytes : 0;
        if (j.hist_words > p.max_hist_words || j.n_off > kMaxJobOffsets || tile_need > p.tile_bytes) {
            if (threadIdx.x == 0)
                atomicOr(p.err, kErrInternal);
            __syncthreads();
            continue;
        }
        const long long rows_ok =
            j.layout == 2 ? 65535ll / ((16 / BPP) * (long long)(blockDim.x >> j.rshift)) : (1ll << 62);
        const long long chunk_rows = (long long)(ch.z - ch.y) * j.band_rows / nwarps + 1;
        if (cur >= 0 && (cur != ch.x || acc_rows + chunk_rows > rows_ok)) {
            flush_any<PACKED>(p.jobs[cur], p.offs, hist);
            __syncthreads();
            cur = -1;
        }
        if (cur != ch.x) {
            if (threadIdx.x < j.n_off) {
                const VoteOffset vo = p.offs[j.off0 + threadIdx.x];
                s_off_h[threadIdx.x] = hist_ref(j, threadIdx.x, hbase, 0);
                const int2 ps = partner_sel(vo.dx);  // used only for |dx| <= kFastMaxDx
                s_off_d[threadIdx.x] = make_int4(vo.dx, vo.dy, ps.x, ps.y);
            }
            __syncthreads();
            cur = ch.x;
            acc_rows = 0;
            spill_rows = 0;
        }
        // Layout 3: anchor rows between spills (votes per half per CTA row:
        // PX anchors of each of the 32 / R lanes that share a copy).
        const int rows_spill = kSpillVotes * (1 << j.rshift) / (32 * (16 / BPP));
        // Items per merge inside the chunk (16-bit halves only).
        int step = ch.z - ch.y;
        if (j.layout == 2)
            step = (int)max(1ll, min((long long)step, rows_ok * nwarps / j.band_rows));
        const bool tma = j.staged && j.aligned;
        for (int ka = ch.y; ka < ch.z; ka += step) {
            const int kb = min(ch.z, ka + step);
            if (ka > ch.y) {
                flush_hist(j, p.offs, hist);
                __syncthreads();
            }
            if (tma && threadIdx.x < 32)
                issue_tile(j, tile_of(j, ka), tiles, &s_bar[0]);
            for (int kk = ka; kk < kb; ++kk) {
                const int b = (kk - ka) & 1;
                uint8_t* buf = tiles + b * p.tile_bytes;
                const Tile t = tile_of(j, kk);
                if (PACKED && j.layout == 3) {
                    const int rows_t = t.y1 - t.y0;
                    if (spill_rows + rows_t > rows_spill) {
                        spill_hist_packed(j, p.offs, hist);
                        __syncthreads();
                        spill_rows = 0;
                    }
                    spill_rows += rows_t;
                }
                if (!j.staged) {
                    vote_tile_unstaged<BPP>(j, jg, t, s_off_h, s_off_d, p.err);
                    __syncthreads();
                    continue;
                }
                if (tma) {
                    // Prefetch the next tile into the other buffer (its last
                    // readers passed the barrier at the end of the previous item).
                    if (kk + 1 < kb && threadIdx.x < 32)
                        issue_tile(j, tile_of(j, kk + 1), tiles + (b ^ 1) * p.tile_bytes, &s_bar[b ^ 1]);
                    if (!mbar_wait_bounded(&s_bar[b], uses[b] & 1u, p.err))
                        s_ok = 0;
                    uses[b]++;
                } else {
                    fill_tile_plain(j, t, buf);
                    // Plain stores before a later bulk copy reuses the buffer.
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncthreads();
                }
                if (s_ok)
                    vote_tile<BPP, PACKED>(j, jg, t, buf, s_off_h, s_off_d, p.err);
                __syncthreads();
            }
        }
        acc_rows += chunk_rows;
    }
    if (cur >= 0)
        flush_any<PACKED>(p.jobs[cur], p.offs, hist);
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

// Raise the dynamic shared-memory limit on the current device only when a
// launch needs more than before (see SmemLimit).
template <int BPP, int MAXT, bool PACKED>
cudaError_t vote_prepare(size_t smem)
{
    static SmemLimit lim;
    return lim.raise((const void*)k_glcm_vote<BPP, MAXT, PACKED>, smem);
}

// Two register budgets: up to 1024 threads at 64 registers, or up to 512
// threads at 128 registers.
template <int BPP, bool PACKED>
cudaError_t vote_launch_t(const VoteParams& p, int grid, int threads, size_t smem, cudaStream_t s, int* occ)
{
    cudaError_t e;
    if (threads > 512) {
        if ((e = vote_prepare<BPP, 1024, PACKED>(smem)) != cudaSuccess)
            return e;
        if (occ)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_glcm_vote<BPP, 1024, PACKED>, threads,
                                                                 smem);
        k_glcm_vote<BPP, 1024, PACKED><<<grid, threads, smem, s>>>(p);
    } else {
        if ((e = vote_prepare<BPP, 512, PACKED>(smem)) != cudaSuccess)
            return e;
        if (occ)
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k_glcm_vote<BPP, 512, PACKED>, threads,
                                                                 smem);
        k_glcm_vote<BPP, 512, PACKED><<<grid, threads, smem, s>>>(p);
    }
    return cudaGetLastError();
}

template <bool PACKED>
cudaError_t vote_launch_b(const VoteParams& p, int bpp, int grid, int threads, size_t smem, cudaStream_t s,
                          int* occ)
{
    return bpp == 1 ? vote_launch_t<1, PACKED>(p, grid, threads, smem, s, occ)
                    : vote_launch_t<2, PACKED>(p, grid, threads, smem, s, occ);
}

}  // namespace

int vote_max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

int vote_row_bytes() { return kRowBytes; }

int vote_blocks_per_sm(int bpp, int threads, size_t smem, bool packed)
{
    int n = 0;
    cudaError_t e = packed ? vote_launch_b<true>(VoteParams{}, bpp, 0, threads, smem, nullptr, &n)
                           : vote_launch_b<false>(VoteParams{}, bpp, 0, threads, smem, nullptr, &n);
    return e == cudaSuccess ? n : 1;
}

cudaError_t launch_vote(const VoteParams& p, int bpp, int grid, int threads, size_t smem, cudaStream_t s,
                        bool packed)
{
    return packed ? vote_launch_b<true>(p, bpp, grid, threads, smem, s, nullptr)
                  : vote_launch_b<false>(p, bpp, grid, threads, smem, s, nullptr);
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
