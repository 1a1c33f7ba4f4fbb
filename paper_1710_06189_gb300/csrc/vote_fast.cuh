// Column-walk GLCM votes for the offsets at chessboard distance 1.
//
// What is computed (Sec. I.A, Eq. 1, partner by Eq. 2 without wrapping, bin
// by Eq. 3): the counts P[i][j] of every offset at distance 1, which is one
// of the canonical offsets k = 0: (1, 0), 1: (1, -1), 2: (0, -1),
// 3: (-1, -1) -- partner to the right or in the row above -- or the
// opposite of one, whose counts are the transpose (Eq. 1 with anchor and
// partner swapped).  So one histogram per canonical offset serves both
// directions, and the merge writes it as counted, transposed, or both.
//
// How, on sm_103a (the paper's private copies, Sec. II.A, and its halo
// rows, Sec. III, redone for this GPU):
//  * A work item is a strip of 32 lanes x 16 bytes of a band of rows; one
//    warp walks down it.  Each lane keeps the levels of its 16 bytes (16
//    uint8 or 8 uint16 pixels) of the previous row in registers, so a
//    partner in the row above costs nothing, and a partner to the left or
//    right is one byte permute; the neighbour lanes' edge words come by
//    shuffle, the strip's outer edges by one 4- or 8-byte load.  Rows are
//    read with 16-byte loads, kPF rows in flight per lane; the first row of
//    a band also loads the row above it (the halo of Eq. 8).
//  * Pixels outside the image (past the right edge, left of column 0, above
//    row 0) get the level N, one past the last.  Their votes go to bins of
//    row or column N, which the merge ignores: no edge masks, no per-pixel
//    bounds checks, every lane of an interior strip votes unconditionally.
//    With M = N + 1 levels a bin of one offset is a * M + b.
//  * Votes go into 32 lane-interleaved private copies (copy c of a bin is
//    word 32 * bin + c; lane l uses copy l), so the lanes of a warp never
//    share a bank whatever the image.  A vote is one byte permute that
//    places the bin code above the lane's byte offset, and one reduction
//    with the constant increment 1 (equal words of different lanes combine).
//  * N <= 8 with all four offsets: the four votes of an anchor are fused
//    into two, of the joint codes (a, j0, j1) and (a, j2, j3) (M^3 bins each,
//    interleaved); the merge marginalizes them.  Half the reductions, which
//    bound this kernel.
//  * N = 16: one vote per offset with the byte code a * 16 + j; two offsets
//    interleaved per bin row.  Here every byte value is a bin, so there is
//    no outside level: the warps of the first and last strip of a row vote
//    under per-pixel masks, the top row skips the offsets into the row above.
//  * N = 32: a job holds up to two offsets as the 16-bit halves of each word
//    (increment 1 or 65536), so 32 copies still fit; the merge comes before
//    any half can reach 65536.
//  * N = 256: a job counts one offset's GLCM rows [128 h, 128 h + 128) (anchor
//    levels, or partner levels for a transposed offset) in one copy of 32768
//    32-bit counters (128 KB), laid out as those rows of the output.  A vote
//    is one byte permute for row * 256 + column, one multiply-add for the
//    address and one unconditional reduction: a vote of the other row half
//    goes to a spare word of its lane past the 128 KB (one unsigned min), as
//    a reduction predicated per lane costs a divergent branch; four offsets
//    take eight jobs.  The merge is a single bulk reduction of the 128 KB into the
//    output rows (cp.reduce.async.bulk ... add.u32, done at L2), not one
//    global atomic per bin.
//  * Persistent CTAs (one per SM, 16 warps) pull chunks of consecutive items
//    of one job from a counter and merge their histograms into the global
//    counts only when their job changes (Sec. II.A's final merge).
//  * Rows that start on 16 bytes (the usual case) and rows at any byte
//    address are separate kernel instances, compiled in separate files
//    (vote_fast.cu, vote_fast_unaligned.cu): the realigning loads cost
//    registers that the aligned loop must not spend.
#pragma once

#include "glcm_internal.cuh"

namespace glcm {
namespace {

constexpr int kFT = 512;            // threads per CTA
constexpr int kFW = kFT / 32;       // warps per CTA
constexpr int kPF = 4;              // rows in flight per lane
constexpr int kMargWords = 4 * 64;  // joint-code merge: 4 offsets x N^2 (N <= 8)
static_assert(kMargWords >= 32, "N = 256 jobs use the first 32 marginal words as spare words");

// Alignment of the histograms' shared address: 64 KB for N = 16 (a byte
// code's vote address is one byte permute with the region's upper bytes),
// else 256 bytes (the base folded into 16-bit codes).
__host__ __device__ constexpr uint32_t fast_align(int log2n)
{
    return log2n == 4 ? 65536u : 256u;
}
// 16-bit halves: anchor rows a lane may vote between merges (16 votes per
// row into one copy at most: 4000 * 16 < 65536).
constexpr unsigned kHalfRows = 4000;

__device__ __forceinline__ void red1(uint32_t a)
{
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(a));
}

// Reduction if bit `bit` of a lane's anchor mask is set (edge strips of N = 16).
__device__ __forceinline__ void red1_if(uint32_t a, uint32_t mask, uint32_t bit)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b32 t;\n\tand.b32 t, %1, %2;\n\tsetp.ne.u32 p, t, 0;\n\t"
        "@p red.shared.add.u32 [%0], 1;\n\t}" ::"r"(a),
        "r"(mask), "r"(bit));
}

// N = 256: reduction at address a (hb + the byte offset of the code within
// the job's 128 rows, hb < 131072) if it lies inside the rows, else into
// `spare`, the lane's own word past the rows (never read).  A code of the
// other half lies above the spare words, or -- for the upper half's job --
// below hb, which wraps around to above them (unsigned); so one min picks.
// No predicate: a predicated reduction whose predicate differs between
// lanes costs a divergent branch around it.
__device__ __forceinline__ void red_row(uint32_t a, uint32_t spare)
{
    red1(min(a, spare));
}

// ... and only if bit `bit` of the lane's anchor mask is set (edge strips).
__device__ __forceinline__ void red_row_if(uint32_t a, uint32_t spare, uint32_t mask, uint32_t bit)
{
    red1((mask & bit) ? min(a, spare) : spare);
}

__device__ __forceinline__ void red_hi(uint32_t a)
{
    asm volatile("red.shared.add.u32 [%0], 65536;" ::"r"(a));
}

__device__ __forceinline__ void red_global(uint32_t* p, uint32_t v)
{
    asm volatile("red.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bytes of the four pixels of a word that lie past the right edge: `rem` is
// W minus the word's first pixel.
__device__ __forceinline__ uint32_t outside_mask(int rem)
{
    return rem >= 4 ? 0u : (rem <= 0 ? 0xFFFFFFFFu : (0xFFFFFFFFu << (8 * rem)));
}

// 16 bytes from any address p, of which the first `need` (1..16) belong to
// the row: the aligned 16-byte block holding p and, only when a needed byte
// lies in it, the next one, shifted into place.  A block read always holds a
// byte of the row, so it lies within the row's allocation (an aligned block
// never crosses a page).
__device__ __forceinline__ uint4 load16_any(const uint8_t* p, int need)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const uint32_t off = (uint32_t)(a & 15u);
    const uint4* b = reinterpret_cast<const uint4*>(a - off);
    const uint4 x = __ldg(b);
    if (off == 0)
        return x;
    uint4 y = make_uint4(0u, 0u, 0u, 0u);
    if ((int)off + need > 16)
        y = __ldg(b + 1);
    const uint32_t q = off >> 2, sh = 8u * (off & 3u);
    // Words q .. q + 4 of (x, y), chosen without dynamic indexing.
    const uint32_t w0 = q == 0 ? x.x : (q == 1 ? x.y : (q == 2 ? x.z : x.w));
    const uint32_t w1 = q == 0 ? x.y : (q == 1 ? x.z : (q == 2 ? x.w : y.x));
    const uint32_t w2 = q == 0 ? x.z : (q == 1 ? x.w : (q == 2 ? y.x : y.y));
    const uint32_t w3 = q == 0 ? x.w : (q == 1 ? y.x : (q == 2 ? y.y : y.z));
    const uint32_t w4 = q == 0 ? y.x : (q == 1 ? y.y : (q == 2 ? y.z : y.w));
    return make_uint4(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh), __funnelshift_r(w2, w3, sh),
                      __funnelshift_r(w3, w4, sh));
}

// 16-bit lanes of a packed word: bytes 0, 1 (lo) or 2, 3 (hi).
__device__ __forceinline__ uint32_t spread_lo(uint32_t w) { return __byte_perm(w, 0u, 0x4140); }
__device__ __forceinline__ uint32_t spread_hi(uint32_t w) { return __byte_perm(w, 0u, 0x4342); }

// Four pixels -> four packed levels q = v >> (bits - log2 N).
template <int BPP, int LOG2N>
__device__ __forceinline__ uint32_t qword(uint32_t a, uint32_t b)
{
    constexpr uint32_t S = 8 - LOG2N;
    constexpr uint32_t MK = (0xFFu >> S) * 0x01010101u;
    if constexpr (BPP == 1)
        return (a >> S) & MK;
    else
        return (__byte_perm(a, b, 0x7531) >> S) & MK;
}

// Partner words of anchor word m of the current row C (right edge word CR)
// and the row D above, P (edge words PL, PR), for canonical offset K at
// distance D: (D, 0), (D, -D), (0, -D), (-D, -D).  sr / sl are the byte
// permutes that shift a word pair D pixels right / left (right_sel(D),
// left_sel(D)); D <= 4, so a partner never lies beyond the neighbour word.
template <int K, int LW>
__device__ __forceinline__ uint32_t partner(int m, const uint32_t (&C)[LW], uint32_t CR, const uint32_t (&P)[LW],
                                            uint32_t PL, uint32_t PR, uint32_t sr, uint32_t sl)
{
    if constexpr (K == 0)
        return __byte_perm(C[m], m + 1 < LW ? C[m + 1] : CR, sr);
    else if constexpr (K == 1)
        return __byte_perm(P[m], m + 1 < LW ? P[m + 1] : PR, sr);
    else if constexpr (K == 2)
        return P[m];
    else
        return __byte_perm(m > 0 ? P[m - 1] : PL, P[m], sl);
}

// Byte-permute selectors: bytes D .. D + 3 of the pair (w, next word), and
// bytes 4 - D .. 7 - D of the pair (previous word, w).
__device__ __forceinline__ uint32_t right_sel(uint32_t D)
{
    return D * 0x1111u + 0x3210u;
}

__device__ __forceinline__ uint32_t left_sel(uint32_t D)
{
    return 0x7654u - D * 0x1111u;
}

// ---- votes of one row ------------------------------------------------------

// N <= 8, all four offsets: joint codes (a*M + j0)*M + j1 and (a*M + j2)*M + j3.
// Bin row of code c: 64 words, the first 32 the (j0, j1) copies, the next 32
// the (j2, j3) copies.
template <int LW, int LOG2N>
__device__ __forceinline__ void votes_joint(const uint32_t (&C)[LW], uint32_t CR, const uint32_t (&P)[LW],
                                            uint32_t PL, uint32_t PR, uint32_t sr, uint32_t sl, uint32_t hb, uint32_t l4)
{
    constexpr uint32_t M = (1u << LOG2N) + 1u, M2 = M * M;
    const uint32_t l4b = l4 + 128u;
    // hb / 256 added to both 16-bit codes, so a byte permute gives the whole
    // address hb + code * 256 + lane * 4 (hb is a multiple of 256).
    const uint32_t hp = (hb >> 8) * 0x00010001u;
#pragma unroll
    for (int m = 0; m < LW; ++m) {
        // Packed bytes j0*M + j1 <= N*M + N < 256: no carries between bytes.
        const uint32_t ta = partner<0>(m, C, CR, P, PL, PR, sr, sl) * M + partner<1>(m, C, CR, P, PL, PR, sr, sl);
        const uint32_t tb = partner<2>(m, C, CR, P, PL, PR, sr, sl) * M + partner<3>(m, C, CR, P, PL, PR, sr, sl);
        const uint32_t alo = spread_lo(C[m]) * M2 + hp, ahi = spread_hi(C[m]) * M2 + hp;
        const uint32_t ca0 = alo + spread_lo(ta), ca1 = ahi + spread_hi(ta);
        const uint32_t cb0 = alo + spread_lo(tb), cb1 = ahi + spread_hi(tb);
        // Address hb + code*256 + lane*4 (+128): the 16-bit code above the lane byte.
        red1(__byte_perm(ca0, l4, 0x5104));
        red1(__byte_perm(cb0, l4b, 0x5104));
        red1(__byte_perm(ca0, l4, 0x5324));
        red1(__byte_perm(cb0, l4b, 0x5324));
        red1(__byte_perm(ca1, l4, 0x5104));
        red1(__byte_perm(cb1, l4b, 0x5104));
        red1(__byte_perm(ca1, l4, 0x5324));
        red1(__byte_perm(cb1, l4b, 0x5324));
    }
}

// One offset K, N <= 8: byte codes a*M + j (<= 80).  Region K >> 1 of
// M*M bin rows of 64 words; offset K & 1 uses words 32 (K & 1) .. + 31.
template <int K, int LW, int LOG2N>
__device__ __forceinline__ void votes_one8(const uint32_t (&A9)[LW], const uint32_t (&C)[LW], uint32_t CR,
                                           const uint32_t (&P)[LW], uint32_t PL, uint32_t PR, uint32_t sr, uint32_t sl, uint32_t hb,
                                           uint32_t l4)
{
    constexpr uint32_t M = (1u << LOG2N) + 1u;
    const uint32_t base = hb + (uint32_t)(K >> 1) * (M * M * 256u);
    const uint32_t lq = l4 + (uint32_t)(K & 1) * 128u;
#pragma unroll
    for (int m = 0; m < LW; ++m) {
        const uint32_t code = A9[m] + partner<K>(m, C, CR, P, PL, PR, sr, sl);
        red1(base + __byte_perm(code, lq, 0x5504));
        red1(base + __byte_perm(code, lq, 0x5514));
        red1(base + __byte_perm(code, lq, 0x5524));
        red1(base + __byte_perm(code, lq, 0x5534));
    }
}

// One offset K, N = 16: byte codes a*16 + j in region K >> 1 (256 bin rows of
// 64 words, 64 KB), offset K & 1 at words 32 (K & 1) .. + 31.  EDGE: only the
// anchors whose bit is set in `mask` vote (bit 4m + b: byte b of word m).
template <int K, int LW, bool EDGE>
__device__ __forceinline__ void votes_one16(const uint32_t (&A16)[LW], const uint32_t (&C)[LW], uint32_t CR,
                                            const uint32_t (&P)[LW], uint32_t PL, uint32_t PR, uint32_t sr, uint32_t sl, uint32_t hb,
                                            uint32_t l4, uint32_t mask)
{
    // hb is a multiple of 65536 here: the region's address hb + (K >> 1) *
    // 65536 has a zero low half, so one byte permute of the code byte, the
    // lane byte and the region's upper bytes gives the whole address.
    const uint32_t x = hb + (uint32_t)(K >> 1) * 65536u + l4 + (uint32_t)(K & 1) * 128u;
#pragma unroll
    for (int m = 0; m < LW; ++m) {
        const uint32_t code = A16[m] | partner<K>(m, C, CR, P, PL, PR, sr, sl);
        const uint32_t a0 = __byte_perm(code, x, 0x7604);
        const uint32_t a1 = __byte_perm(code, x, 0x7614);
        const uint32_t a2 = __byte_perm(code, x, 0x7624);
        const uint32_t a3 = __byte_perm(code, x, 0x7634);
        // In an edge strip only a few words have a masked-out anchor: the
        // others take the unmasked votes, decided for the whole warp.
        if (EDGE && !__all_sync(0xffffffffu, ((mask >> (4 * m)) & 0xFu) == 0xFu)) {
            red1_if(a0, mask, 1u << (4 * m));
            red1_if(a1, mask, 1u << (4 * m + 1));
            red1_if(a2, mask, 1u << (4 * m + 2));
            red1_if(a3, mask, 1u << (4 * m + 3));
        } else {
            red1(a0);
            red1(a1);
            red1(a2);
            red1(a3);
        }
    }
}

// One offset K, N = 32: 16-bit codes a*33 + j (<= 1088) in 1089 rows of 32
// words; byte offset code*128 + lane*4 = (code*256 + lane*8) / 2.  HI: the
// offset counts in the upper halves.
template <int K, int LW, bool HI>
__device__ __forceinline__ void votes_one32(const uint32_t (&Alo)[LW], const uint32_t (&Ahi)[LW],
                                            const uint32_t (&C)[LW], uint32_t CR, const uint32_t (&P)[LW],
                                            uint32_t PL, uint32_t PR, uint32_t sr, uint32_t sl, uint32_t hb, uint32_t l8)
{
#pragma unroll
    for (int m = 0; m < LW; ++m) {
        const uint32_t w = partner<K>(m, C, CR, P, PL, PR, sr, sl);
        const uint32_t c0 = Alo[m] + spread_lo(w), c1 = Ahi[m] + spread_hi(w);
        // Alo / Ahi carry hb / 128: these are whole addresses.
        const uint32_t a0 = __byte_perm(c0, l8, 0x5104) >> 1;
        const uint32_t a1 = __byte_perm(c0, l8, 0x5324) >> 1;
        const uint32_t a2 = __byte_perm(c1, l8, 0x5104) >> 1;
        const uint32_t a3 = __byte_perm(c1, l8, 0x5324) >> 1;
        if (HI) {
            red_hi(a0);
            red_hi(a1);
            red_hi(a2);
            red_hi(a3);
        } else {
            red1(a0);
            red1(a1);
            red1(a2);
            red1(a3);
        }
    }
}

template <int K, int LW>
__device__ __forceinline__ void votes_one32_sel(bool hi, const uint32_t (&Alo)[LW], const uint32_t (&Ahi)[LW],
                                                const uint32_t (&C)[LW], uint32_t CR, const uint32_t (&P)[LW],
                                                uint32_t PL, uint32_t PR, uint32_t sr, uint32_t sl, uint32_t hb, uint32_t l8)
{
    if (hi)
        votes_one32<K, LW, true>(Alo, Ahi, C, CR, P, PL, PR, sr, sl, hb, l8);
    else
        votes_one32<K, LW, false>(Alo, Ahi, C, CR, P, PL, PR, sr, sl, hb, l8);
}

// One offset k, N = 256: code x = row * 256 + column with row the anchor
// level (tr: the partner level) -- one byte permute of the column word and
// the row's 16-bit spread ([r0, 0, r1, 0]) -- counted at byte 4 x - 4 * 32768 h
// of the job's rows (rbase = -4 * 32768 h).  The job's offset is a run-time
// value: its partner word is one byte permute of operands and selector
// chosen per offset (warp-uniform selects, no branch per row).
template <int LW, bool EDGE>
__device__ __forceinline__ void votes_wide(int k, bool tr, const uint32_t (&C)[LW], uint32_t CR,
                                           const uint32_t (&P)[LW], uint32_t PL, uint32_t PR, uint32_t sr, uint32_t sl, uint32_t hb,
                                           uint32_t rbase, uint32_t spare, uint32_t mask)
{
    const uint32_t sel = k == 3 ? sl : (k == 2 ? 0x3210u : sr);
#pragma unroll
    for (int m = 0; m < LW; ++m) {
        const uint32_t cur = k == 0 ? C[m] : P[m];
        const uint32_t nxt = k == 0 ? (m + 1 < LW ? C[m + 1] : CR) : (m + 1 < LW ? P[m + 1] : PR);
        const uint32_t prv = m > 0 ? P[m - 1] : PL;
        const uint32_t w = __byte_perm(k == 3 ? prv : cur, k == 3 ? P[m] : nxt, sel);
        const uint32_t col = tr ? C[m] : w;
        const uint32_t rw = tr ? w : C[m];
        const uint32_t slo = spread_lo(rw), shi = spread_hi(rw);
        const uint32_t r0 = 4u * __byte_perm(col, slo, 0x5540) + rbase;  // hb + byte offset
        const uint32_t r1 = 4u * __byte_perm(col, slo, 0x5561) + rbase;
        const uint32_t r2 = 4u * __byte_perm(col, shi, 0x5542) + rbase;
        const uint32_t r3 = 4u * __byte_perm(col, shi, 0x5563) + rbase;
        if (EDGE && !__all_sync(0xffffffffu, ((mask >> (4 * m)) & 0xFu) == 0xFu)) {
            red_row_if(r0, spare, mask, 1u << (4 * m));
            red_row_if(r1, spare, mask, 1u << (4 * m + 1));
            red_row_if(r2, spare, mask, 1u << (4 * m + 2));
            red_row_if(r3, spare, mask, 1u << (4 * m + 3));
        } else {
            red_row(r0, spare);
            red_row(r1, spare);
            red_row(r2, spare);
            red_row(r3, spare);
        }
    }
}

// Masks of an edge strip's anchors for N = 16 (bit 4m + b: pixel 4m + b of
// the lane): anchors inside the image, with a partner to the right inside
// it, with a partner to the left inside it.
struct EdgeMasks {
    uint32_t in, right, left;
};

template <int LW, int LOG2N, bool EDGE>
__device__ __forceinline__ void vote_row(const FastJob& j, const uint32_t (&C)[LW], uint32_t CR,
                                         const uint32_t (&P)[LW], uint32_t PL, uint32_t PR, uint32_t sr, uint32_t sl, uint32_t hb,
                                         uint32_t l4, bool top, const EdgeMasks& em)
{
    const int pr = j.present;
    if constexpr (LOG2N <= 3) {
        if (j.mode == kFastJoint) {
            votes_joint<LW, LOG2N>(C, CR, P, PL, PR, sr, sl, hb, l4);
            return;
        }
        constexpr uint32_t M = (1u << LOG2N) + 1u;
        uint32_t A9[LW];
#pragma unroll
        for (int m = 0; m < LW; ++m)
            A9[m] = C[m] * M;  // packed bytes a*M <= 72
        if (pr & 1)
            votes_one8<0, LW, LOG2N>(A9, C, CR, P, PL, PR, sr, sl, hb, l4);
        if (pr & 2)
            votes_one8<1, LW, LOG2N>(A9, C, CR, P, PL, PR, sr, sl, hb, l4);
        if (pr & 4)
            votes_one8<2, LW, LOG2N>(A9, C, CR, P, PL, PR, sr, sl, hb, l4);
        if (pr & 8)
            votes_one8<3, LW, LOG2N>(A9, C, CR, P, PL, PR, sr, sl, hb, l4);
    } else if constexpr (LOG2N == 8) {
        // One offset and orientation per job, fixed for this loop instance.
        const uint32_t rbase = hb - 4u * 32768u * (uint32_t)j.row_half;
        const int k = (pr & 1) ? 0 : ((pr & 2) ? 1 : ((pr & 4) ? 2 : 3));
        if (top && k != 0)
            return;  // no row above the image's first row
        // Spare words: the lane's word of the 32 after the job's 32768.
        votes_wide<LW, EDGE>(k, j.transposed != 0, C, CR, P, PL, PR, sr, sl, hb, rbase, hb + 131072u + l4,
                             k == 2 ? em.in : (k == 3 ? em.left : em.right));
    } else if constexpr (LOG2N == 4) {
        uint32_t A16[LW];
#pragma unroll
        for (int m = 0; m < LW; ++m)
            A16[m] = C[m] << 4;  // packed bytes a*16 <= 240
        if (pr & 1)
            votes_one16<0, LW, EDGE>(A16, C, CR, P, PL, PR, sr, sl, hb, l4, em.right);
        if (top)
            return;  // no row above the image's first row
        if (pr & 2)
            votes_one16<1, LW, EDGE>(A16, C, CR, P, PL, PR, sr, sl, hb, l4, em.right);
        if (pr & 4)
            votes_one16<2, LW, EDGE>(A16, C, CR, P, PL, PR, sr, sl, hb, l4, em.in);
        if (pr & 8)
            votes_one16<3, LW, EDGE>(A16, C, CR, P, PL, PR, sr, sl, hb, l4, em.left);
    } else {
        constexpr uint32_t M = (1u << LOG2N) + 1u;
        uint32_t Alo[LW], Ahi[LW];
#pragma unroll
        for (int m = 0; m < LW; ++m) {
            // hb / 128 (hb a multiple of 256) added to both 16-bit codes.
            Alo[m] = spread_lo(C[m]) * M + (hb >> 7) * 0x00010001u;
            Ahi[m] = spread_hi(C[m]) * M + (hb >> 7) * 0x00010001u;
        }
        const uint32_t l8 = 2u * l4;
        const int hk = j.half_hi;
        if (pr & 1)
            votes_one32_sel<0, LW>(hk == 0, Alo, Ahi, C, CR, P, PL, PR, sr, sl, hb, l8);
        if (pr & 2)
            votes_one32_sel<1, LW>(hk == 1, Alo, Ahi, C, CR, P, PL, PR, sr, sl, hb, l8);
        if (pr & 4)
            votes_one32_sel<2, LW>(hk == 2, Alo, Ahi, C, CR, P, PL, PR, sr, sl, hb, l8);
        if (pr & 8)
            votes_one32_sel<3, LW>(hk == 3, Alo, Ahi, C, CR, P, PL, PR, sr, sl, hb, l8);
    }
}

// ---- one work item: a warp walks down its strip ------------------------------

// EDGE: the strip holds the image's first or last column (pixels outside
// the image get the outside level N, or for N = 16 the anchors are masked);
// interior strips need neither.  ALIGNED: every row starts on 16 bytes, so a
// lane's bytes are one 16-byte load (a separate instance: the realigning
// loads of other images cost registers the aligned loop does not spend).
// ring: this warp's row history for distances D > 1 -- D slots of 32 lanes
// x (LW level words + the lane's halo word), word-major so that each lane
// keeps to its own bank; unused for D = 1 (the row above stays in registers).
template <int BPP, int LOG2N, bool EDGE, bool ALIGNED>
__device__ __forceinline__ void walk_strip(const FastJob& j, int x0, int y0, int y1, uint32_t hb, uint32_t* ring)
{
    constexpr int PX = 16 / BPP, LW = 4 / BPP;
    constexpr uint32_t N = 1u << LOG2N;
    constexpr bool OUTLEVEL = LOG2N <= 3 || LOG2N == 5;  // the outside level N exists
    constexpr bool MASKED = !OUTLEVEL;                      // edge strips vote under masks
    constexpr uint32_t D4 = (N & 0xFFu) * 0x01010101u;  // four pixels outside the image
    const int lane = threadIdx.x & 31;
    const int xl = x0 + lane * PX, xe = x0 + 32 * PX;
    const bool on = xl < j.W;
    uint32_t om[LW];
#pragma unroll
    for (int m = 0; m < LW; ++m)
        om[m] = EDGE ? outside_mask(j.W - (xl + 4 * m)) : 0u;
    const uint32_t omr = EDGE ? outside_mask(j.W - xe) : 0u;
    const int D = j.dist;  // partner distance, 1 .. 4
    const uint32_t sr = right_sel((uint32_t)D), sl = left_sel((uint32_t)D);
    EdgeMasks em{0xFFFFu, 0xFFFFu, 0xFFFFu};
    if (EDGE && MASKED) {
        const int nin = max(0, min(PX, j.W - xl));           // pixels of the lane inside the image
        const int nright = max(0, min(PX, j.W - D - xl));    // ... with a partner D to the right
        em.in = (1u << nin) - 1u;
        em.right = (1u << nright) - 1u;
        em.left = em.in & (xl == 0 ? ~((1u << D) - 1u) : ~0u);  // ... and D to the left
    }
    const bool has_l = lane == 0 && x0 > 0;
    const bool has_r = lane == 31 && xe < j.W;
    const bool has_h = has_l || has_r;
    // A 16-byte block with at least one byte of the row lies inside the row's
    // allocation (base and pitch are 16-byte aligned), as do the 4 pixels
    // before a strip's first pixel and the 4 after its end when they exist.
    const uint8_t* col = j.img + (long long)(on ? xl : 0) * BPP;
    const uint8_t* hcol = j.img + (long long)(has_l ? x0 - 4 : (has_r ? xe : 0)) * BPP;
    const uint32_t l4 = 4u * (uint32_t)lane;

    uint4 qv[kPF];
    uint2 qh[kPF];
    // Bytes of the row from the lane's first pixel, and from the halo's first pixel.
    const int need = min(16, (j.W - (on ? xl : 0)) * BPP);
    const int hneed = has_l ? 4 * BPP : min(4, j.W - xe) * BPP;
    auto load_row = [&](int y, uint4& v, uint2& h) {
        const long long ro = (long long)y * j.pitch;
        v = make_uint4(0u, 0u, 0u, 0u);
        h = make_uint2(0u, 0u);
        if constexpr (ALIGNED) {
            if (on)
                v = __ldg(reinterpret_cast<const uint4*>(col + ro));
            if (has_h) {
                if constexpr (BPP == 1)
                    h.x = __ldg(reinterpret_cast<const uint32_t*>(hcol + ro));
                else
                    h = __ldg(reinterpret_cast<const uint2*>(hcol + ro));
            }
        } else {
            // Rows at any byte address: realigned loads.
            if (on)
                v = load16_any(col + ro, need);
            if (has_h) {
                const uint4 t = load16_any(hcol + ro, hneed);
                h = make_uint2(t.x, t.y);
            }
        }
    };
    auto levels = [&](const uint4& v, const uint2& h, uint32_t (&L)[LW], uint32_t& ll, uint32_t& lr, uint32_t& hqo) {
        if constexpr (BPP == 1) {
            L[0] = qword<1, LOG2N>(v.x, 0u);
            L[1 % LW] = qword<1, LOG2N>(v.y, 0u);
            L[2 % LW] = qword<1, LOG2N>(v.z, 0u);
            L[3 % LW] = qword<1, LOG2N>(v.w, 0u);
        } else {
            L[0] = qword<2, LOG2N>(v.x, v.y);
            L[1] = qword<2, LOG2N>(v.z, v.w);
        }
        if constexpr (EDGE && OUTLEVEL) {
#pragma unroll
            for (int m = 0; m < LW; ++m)
                L[m] = (L[m] & ~om[m]) | (D4 & om[m]);
        }
        uint32_t hq = qword<BPP, LOG2N>(h.x, h.y);
        if constexpr (EDGE && OUTLEVEL)
            hq = lane == 31 ? ((hq & ~omr) | (D4 & omr)) : hq;
        const uint32_t up = __shfl_up_sync(0xffffffffu, L[LW - 1], 1);
        const uint32_t dn = __shfl_down_sync(0xffffffffu, L[0], 1);
        ll = lane == 0 ? (has_l ? hq : D4) : up;
        lr = lane == 31 ? (has_r ? hq : D4) : dn;
        hqo = hq;
    };

    uint32_t P[LW], PL = D4, PR = D4;
#pragma unroll
    for (int m = 0; m < LW; ++m)
        P[m] = D4;
    const int ys = max(0, y0 - D);  // the D rows above the band are its halo
    int slot = 0;                   // ring slot of row y: (y - ys) mod D
#pragma unroll
    for (int k = 0; k < kPF; ++k)
        if (ys + k < y1)
            load_row(ys + k, qv[k], qh[k]);
    for (int yb = ys; yb < y1; yb += kPF) {
#pragma unroll
        for (int k = 0; k < kPF; ++k) {
            const int y = yb + k;
            if (y >= y1)
                break;
            const uint4 v = qv[k];
            const uint2 h = qh[k];
            if (y + kPF < y1)
                load_row(y + kPF, qv[k], qh[k]);
            uint32_t C[LW], CL, CR, hq;
            levels(v, h, C, CL, CR, hq);
            if (D > 1) {
                // Row y - D from the ring slot, which then takes row y; rows
                // y < D have the outside level above them (no partner: their
                // votes land in ignored bins, or are skipped under masks).
                uint32_t* rs = ring + slot * ((LW + 1) * 32) + lane;
                if (y >= D) {
#pragma unroll
                    for (int m = 0; m < LW; ++m)
                        P[m] = rs[m * 32];
                    const uint32_t hp = rs[LW * 32];
                    const uint32_t up = __shfl_up_sync(0xffffffffu, P[LW - 1], 1);
                    const uint32_t dn = __shfl_down_sync(0xffffffffu, P[0], 1);
                    PL = lane == 0 ? (has_l ? hp : D4) : up;
                    PR = lane == 31 ? (has_r ? hp : D4) : dn;
                } else {
#pragma unroll
                    for (int m = 0; m < LW; ++m)
                        P[m] = D4;
                    PL = D4;
                    PR = D4;
                }
#pragma unroll
                for (int m = 0; m < LW; ++m)
                    rs[m * 32] = C[m];
                rs[LW * 32] = hq;
                slot = slot + 1 == D ? 0 : slot + 1;
            }
            // (masked edge strips vote with all lanes -- lanes outside the
            // image have empty masks -- since their word masks are decided
            // warp-wide.)  Rows y < D have no partner row above.
            if (y >= y0 && (on || (EDGE && MASKED)))
                vote_row<LW, LOG2N, EDGE>(j, C, CR, P, PL, PR, sr, sl, hb, l4, y < D, em);
            if (D == 1) {
#pragma unroll
                for (int m = 0; m < LW; ++m)
                    P[m] = C[m];
                PL = CL;
                PR = CR;
            }
        }
    }
}

// Items of a job: first the edge strips (the first and the last) of every
// band, then the interior strips (1 .. n_strips - 2), so that a chunk's
// items, one per warp, cost about the same and no warp waits long at the
// chunk's barrier for an edge strip, and a job's last chunks -- a launch's
// tail -- are its cheaper interior ones.
template <int BPP, int LOG2N, bool ALIGNED>
__device__ __forceinline__ void walk_item(const FastJob& j, int item, uint32_t hb, uint32_t* ring)
{
    constexpr int PX = 16 / BPP;
    const int n_int = max(0, j.n_strips - 2);
    const int n_edge = min(2, j.n_strips);
    const int n_bands = (j.y_end - j.y_begin + j.band - 1) / j.band;
    int local = item - j.item0;
    int band, strip;
    if (local < n_edge * n_bands) {
        band = local / n_edge;
        strip = (local - band * n_edge) == 0 ? 0 : j.n_strips - 1;
    } else {
        local -= n_edge * n_bands;
        band = local / n_int;
        strip = 1 + (local - band * n_int);
    }
    const int x0 = strip * 32 * PX;
    const int y0 = j.y_begin + band * j.band;
    const int y1 = min(j.y_end, y0 + j.band);
    if (y0 >= y1)
        return;
    // Edge strips: the first, and every strip whose partners D pixels past
    // its right end can leave the image (the last, and the one before it
    // when the last holds fewer than D pixels).
    if (strip == 0 || x0 + 32 * PX + j.dist > j.W)
        walk_strip<BPP, LOG2N, true, ALIGNED>(j, x0, y0, y1, hb, ring);
    else
        walk_strip<BPP, LOG2N, false, ALIGNED>(j, x0, y0, y1, hb, ring);
}

// ---- merge -------------------------------------------------------------------

// Sum of the 32 copies of bin row `row` (32 words), cleared: eight 16-byte
// reads, rotated by lane so the rows of consecutive lanes spread over all
// banks (four wavefronts per warp read, the least for 512 bytes).
__device__ __forceinline__ uint32_t take_row(uint32_t* h, int row)
{
    const int lane = threadIdx.x & 31;
    uint4* b = reinterpret_cast<uint4*>(h + row * 32);
    uint32_t s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int w = (c + lane) & 7;
        const uint4 v = b[w];
        s += (v.x + v.y) + (v.z + v.w);
        b[w] = make_uint4(0u, 0u, 0u, 0u);
    }
    return s;
}

__device__ __forceinline__ void take_row_halves(uint32_t* h, int row, uint32_t& lo, uint32_t& hi)
{
    const int lane = threadIdx.x & 31;
    uint4* b = reinterpret_cast<uint4*>(h + row * 32);
    lo = hi = 0u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int w = (c + lane) & 7;
        const uint4 v = b[w];
        lo += (v.x & 0xFFFFu) + (v.y & 0xFFFFu) + (v.z & 0xFFFFu) + (v.w & 0xFFFFu);
        hi += (v.x >> 16) + (v.y >> 16) + (v.z >> 16) + (v.w >> 16);
        b[w] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Count v of canonical offset k at bin (a, b) into the job's outputs.
__device__ __forceinline__ void emit(const FastJob& j, int k, uint32_t a, uint32_t b, uint32_t v)
{
    const uint32_t N = 1u << j.log2n;
    const long long NN = (long long)N * N;
    if (j.slot[k] >= 0)
        red_global(j.out + j.slot[k] * NN + a * N + b, v);
    if (j.slot_t[k] >= 0)
        red_global(j.out + j.slot_t[k] * NN + b * N + a, v);
}

template <int LOG2N>
__device__ void flush_t(const FastJob& j, uint32_t* hist, uint32_t* marg)
{
    constexpr uint32_t N = 1u << LOG2N, M = N + 1u, M2 = M * M;
    const int tid = threadIdx.x;
    if constexpr (LOG2N == 8) {
        // Every thread's reductions visible to the bulk-copy (async) proxy,
        // then one bulk reduction of the 128 counted rows into the output.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            int k = 0;
            while (k < kFastOffsets - 1 && !((j.present >> k) & 1))
                ++k;
            uint32_t* dst = j.out + (long long)j.slot[k] * 65536 + (long long)j.row_half * 32768;
            asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u32 [%0], [%1], %2;" ::"l"(dst),
                         "r"((uint32_t)__cvta_generic_to_shared(hist)), "r"(131072u)
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
        }
        __syncthreads();
        uint4* z = reinterpret_cast<uint4*>(hist);
        for (int i = tid; i < 32768 / 4; i += kFT)
            z[i] = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    if (LOG2N <= 3 && j.mode == kFastJoint) {
        constexpr int rows = 2 * (int)(M * M2);
        for (int r = tid; r < rows; r += kFT) {
            const uint32_t s = take_row(hist, r);
            if (s) {
                const uint32_t code = (uint32_t)r >> 1, q = (uint32_t)r & 1u;
                const uint32_t a = code / M2, t = code - a * M2, ja = t / M, jb = t - ja * M;
                if (a < N) {
                    if (ja < N)
                        atomicAdd(marg + (2u * q) * N * N + a * N + ja, s);
                    if (jb < N)
                        atomicAdd(marg + (2u * q + 1u) * N * N + a * N + jb, s);
                }
            }
        }
        __syncthreads();
        for (int e = tid; e < 4 * (int)(N * N); e += kFT) {
            const uint32_t v = marg[e];
            if (v) {
                marg[e] = 0u;
                const int k = e / (int)(N * N);
                const uint32_t ij = (uint32_t)e - (uint32_t)k * N * N;
                emit(j, k, ij / N, ij % N, v);
            }
        }
    } else if (LOG2N <= 4) {
        // Region K >> 1 of MB^2 bin rows of 64 words (N = 16: codes a*16 + j,
        // no outside level), each as two rows of 32: row = 2 (region MB^2 + code) + (K & 1).
        constexpr uint32_t MB = LOG2N == 4 ? N : M, MB2 = MB * MB;
        constexpr int rows = 4 * (int)MB2;
        for (int r = tid; r < rows; r += kFT) {
            const int k = 2 * (r / (2 * (int)MB2)) + (r & 1);
            if (!((j.present >> k) & 1))
                continue;
            const uint32_t s = take_row(hist, r);
            if (s) {
                const uint32_t code = (uint32_t)(r % (2 * (int)MB2)) >> 1;
                const uint32_t a = code / MB, b = code - a * MB;
                if (a < N && b < N)
                    emit(j, k, a, b, s);
            }
        }
    } else {
        constexpr int rows = (int)M2;
        int klo = -1, khi = j.half_hi;
        for (int k = 0; k < kFastOffsets; ++k)
            if (((j.present >> k) & 1) && k != khi) {
                klo = k;
                break;
            }
        for (int r = tid; r < rows; r += kFT) {
            uint32_t lo, hi;
            take_row_halves(hist, r, lo, hi);
            if (lo | hi) {
                const uint32_t a = (uint32_t)r / M, b = (uint32_t)r - a * M;
                if (a < N && b < N) {
                    if (lo && klo >= 0)
                        emit(j, klo, a, b, lo);
                    if (hi && khi >= 0)
                        emit(j, khi, a, b, hi);
                }
            }
        }
    }
}

// Persistent CTAs: chunk b to CTA b first, then chunks from the counter.
// (Taking the first chunk from the counter too, for CTAs that start late
// beside another kernel, measured slower: a lone 4096^2 N = 32 image 28.9 ->
// 32.0 us, the contention step 0.431 -> 0.433 ms.)
// One kernel instance per pixel type, N and row alignment (every job of a
// launch has them).
// Dynamic shared memory: the histograms (max_hist_words), the joint merge's
// marginals, then the chunk index.
template <int BPP, int LOG2N, bool ALIGNED>
__global__ void __launch_bounds__(kFT, 1) k_glcm_vote_d1(FastParams p)
{
    extern __shared__ __align__(16) uint32_t sh[];
    // The histograms start at a shared address that is a multiple of
    // fast_align(LOG2N), so that vote addresses need no add (see the votes).
    const uint32_t base0 = (uint32_t)__cvta_generic_to_shared(sh);
    const uint32_t pad = (fast_align(LOG2N) - (base0 & (fast_align(LOG2N) - 1u))) & (fast_align(LOG2N) - 1u);
    uint32_t* hist = sh + pad / 4u;
    const uint32_t hb = base0 + pad;
    if (LOG2N == 8 && hb >= 131072u) {  // the N = 256 votes' wrap-around needs hb < 128 KB
        if (threadIdx.x == 0)
            atomicOr(p.err, kErrInternal);
        return;
    }
    uint32_t* marg = hist + p.max_hist_words;
    int* s_chunk = reinterpret_cast<int*>(marg + kMargWords);
    // Row rings of distances D > 1, ring_words per warp: after the chunk
    // index, or for N = 16 in the padding before the 64 KB-aligned
    // histograms (the dynamic shared memory starts near 0, so the padding is
    // almost 64 KB; the launch's size counts no ring then).
    const bool ring_in_pad = fast_align(LOG2N) == 65536u;
    if (ring_in_pad && (uint32_t)p.ring_words * kFW * 4u > pad) {
        if (threadIdx.x == 0)
            atomicOr(p.err, kErrInternal);
        return;
    }
    uint32_t* ring = (ring_in_pad ? sh : marg + kMargWords + 4) + (threadIdx.x >> 5) * p.ring_words;
    {
        uint4* z = reinterpret_cast<uint4*>(hist);
        for (int i = threadIdx.x; i < (p.max_hist_words + kMargWords) / 4; i += kFT)
            z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    int cur = -1;
    unsigned acc_rows = 0;
    bool first = true;
    for (;;) {
        if (threadIdx.x == 0)
            *s_chunk = first ? (int)blockIdx.x : (int)gridDim.x + (int)atomicAdd(p.chunk_counter, 1u);
        first = false;
        __syncthreads();
        const int c = *s_chunk;
        if (c >= p.n_chunks)
            break;
        const int3 ch = p.chunks[c];
        const FastJob j = p.jobs[ch.x];
        const unsigned rows_w = (unsigned)((ch.z - ch.y + kFW - 1) / kFW) * (unsigned)(j.band + 1);
        if (cur >= 0 && (cur != ch.x || (j.mode == kFastHalf && acc_rows + rows_w > kHalfRows))) {
            flush_t<LOG2N>(p.jobs[cur], hist, marg);
            __syncthreads();
            cur = -1;
        }
        if (cur != ch.x) {
            cur = ch.x;
            acc_rows = 0;
        }
        acc_rows += rows_w;
        if (j.hist_words > p.max_hist_words || j.log2n != LOG2N || j.bpp != BPP || (j.aligned != 0) != ALIGNED ||
            (j.mode == kFastHalf && rows_w > kHalfRows) || j.dist < 1 || j.dist > 4 ||
            (j.dist > 1 && j.dist * (4 / BPP + 1) * 32 > p.ring_words)) {
            if (threadIdx.x == 0)
                atomicOr(p.err, kErrInternal);
        } else {
            for (int it = ch.y + warp; it < ch.z; it += kFW)
                walk_item<BPP, LOG2N, ALIGNED>(j, it, hb, ring);
        }
        __syncthreads();
    }
    if (cur >= 0)
        flush_t<LOG2N>(p.jobs[cur], hist, marg);
    if (LOG2N == 8 && threadIdx.x == 0)
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // the bulk reductions have landed
}

}  // namespace
}  // namespace glcm
