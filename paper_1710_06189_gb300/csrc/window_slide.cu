// Sliding-window local GLCMs and texture maps, updated incrementally.
//
// Each win x win window (top-left pixel (wx * stride, wy * stride)) gets the
// GLCM of Eq. 1 over the pairs with both pixels inside it, per offset, and
// four float32 maps per offset: contrast, angular second moment, inverse
// difference moment and entropy of its normalized GLCM (Haralick's f2, f1,
// f5 and f9; of S = P + P^T with GLCM_SYMMETRIC).
//
// Moving a window `stride` columns to the right removes the pairs of the
// anchor columns that leave it and adds those of the columns that enter it
// (the voting step after Eq. 3 run both ways); the other columns' pairs are
// shared.  Each lane owns one task -- a row of consecutive windows along x,
// for one offset -- and keeps that offset's counts in 8-bit counters in
// shared memory, interleaved so that lane l's counter word k is word
// 32 k + l, always bank l: no lane ever waits on another.  Beside the counts
// a lane keeps the sums the four maps need, updated with every vote:
//   T = sum S, A = sum S^2, C = sum S (i - j)^2            (exact integers)
//   E = sum S ln S, I = sum S / (1 + (i - j)^2)             (fixed point 2^-40)
// so each window's maps cost O(1) -- contrast C / T, ASM A / T^2, IDM I / T,
// entropy ln T - E / T -- and never a scan of its N^2 bins.  Adding one to a
// bin of count c changes sum S ln S by g(c) = (c + 1) ln(c + 1) - c ln c,
// read from a table made once on the host in float64 and rounded to 2^-40:
// the sums are exact sums of rounded terms.  T ln T is the prefix sum of the
// same terms, so T * entropy = T ln T - sum S ln S is an exact integer
// difference (0 for a constant window) and the maps need no float64 on the
// device (float64 is slow on this GPU): each is one float32 division.
//
// One CTA covers `tasks` consecutive window rows and `seg` windows of each;
// it stages the levels of the pixels they span in shared memory once.
#include <cmath>
#include <type_traits>

#include "glcm_internal.cuh"

namespace glcm {
namespace {

constexpr int kSlideWarps = 8;
constexpr int kSlideThreads = 32 * kSlideWarps;
constexpr int kGTab = kSlideG;      // g(c) for c < 512 (S <= 2 * 255 + 1)
constexpr double kFix = 1099511627776.0;  // 2^40
constexpr uint8_t kBad = 0xFF;      // a pixel >= N (levels mode)

__device__ __forceinline__ uint32_t slide_px(const WindowParams& p, int x, int y)
{
    const uint8_t* row = p.img + (long long)y * p.pitch;
    if (p.bpp == 1)
        return __ldg(row + x);
    return (uint32_t)__ldg(row + 2 * x) | ((uint32_t)__ldg(row + 2 * x + 1) << 8);
}

struct SlideSums {
    int T, A, C;
    long long E, I;
};

// LPW lanes per task: one per offset (n_off <= LPW), the rest idle.
template <int LPW>
__global__ void __launch_bounds__(kSlideThreads) k_window_slide(WindowParams p, int seg, int RH, int RW, int RWp,
                                                                int hw, int vec_counts)
{
    constexpr int TPW = 32 / LPW;  // tasks per warp
    extern __shared__ __align__(16) unsigned char sm[];
    long long* Gt = reinterpret_cast<long long*>(sm);
    long long* PGt = Gt + kGTab;       // t ln t, t <= 512
    long long* Ht = PGt + kGTab + 1;
    uint8_t* tile = reinterpret_cast<uint8_t*>(Ht + 32);
    uint32_t* hist = reinterpret_cast<uint32_t*>(tile + (((size_t)RH * RWp + 15) & ~(size_t)15));
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int S = p.stride, N = p.levels, NN = N * N;
    const int tasks = kSlideWarps * TPW;

    for (int c = tid; c < kSlideTableWords; c += kSlideThreads)
        Gt[c] = p.slide_tables[c];
    const int wx0 = blockIdx.x * seg, wy0 = blockIdx.y * tasks;
    const int px0 = wx0 * S, py0 = wy0 * S;
    for (int t = tid; t < RH * RW; t += kSlideThreads) {
        const int r = t / RW, c = t - r * RW;
        const int x = px0 + c, y = py0 + r;
        uint8_t v = kBad;
        if (x < p.W && y < p.H) {
            const uint32_t raw = slide_px(p, x, y);
            const uint32_t q = p.levels_mode ? raw
                                             : (uint32_t)(((unsigned long long)raw * (unsigned)N) >> (8 * p.bpp));
            v = q < (uint32_t)N ? (uint8_t)q : kBad;
        }
        tile[r * RWp + c] = v;
    }
    __syncthreads();

    const int task = warp * TPW + lane / LPW, o = lane % LPW;
    const int wy = wy0 + task;
    const int n_w = min(seg, p.nwx - wx0);
    if (o >= p.n_off || wy >= p.nwy || n_w <= 0)
        return;  // no CTA-wide synchronization follows
    const int dx = p.dx[o], dy = p.dy[o];
    const int axlo = max(0, -dx), axhi = p.win - max(0, dx);
    const int aylo = max(0, -dy), ayhi = p.win - max(0, dy);
    uint32_t* hl = hist + warp * (hw * 32) + lane;  // counter b: byte b & 3 of hl[(b >> 2) * 32]
    for (int k = 0; k < hw; ++k)
        hl[k * 32] = 0u;
    const int sym = p.symmetric;
    const int tstep = dy * RWp + dx;  // tile offset from anchor to partner
    SlideSums s{0, 0, 0, 0ll, 0ll};
    bool bad = false;

    // One vote of the pair at tile index a (anchor), added (SG = +1) or removed
    // (SG = -1).  Branch-free, so the lanes of a warp never split on i == j:
    // with S the symmetric count before the vote (c + c^T; 2c on the
    // diagonal) the pair moves two unit steps -- S(i, j) and S(j, i), or S(i, i)
    // twice -- so sum S^2 changes by 2 (2 S + 1) + 2 [i == j] when added and
    // by 2 (1 - 2 S) + 2 [i == j] when removed, and sum S ln S by
    // g(S) + g(S + [i == j]), or -(g(S - 1) + g(S - 1 - [i == j])).
    auto vote = [&](uint32_t i, uint32_t j, auto sg_tag) {
        constexpr int SG = decltype(sg_tag)::value;
        if (i == kBad || j == kBad) {
            bad = true;
            return;
        }
        const uint32_t b = i * (uint32_t)N + j;
        uint32_t* w = hl + (b >> 2) * 32;
        const uint32_t sh = (b & 3u) * 8u;
        const uint32_t word = *w;
        const int c = (int)((word >> sh) & 0xFFu);
        const int d = (int)i - (int)j;
        const long long h = Ht[d < 0 ? -d : d];
        if (sym) {
            const uint32_t bt = j * (uint32_t)N + i;
            const int ct = (int)((hl[(bt >> 2) * 32] >> ((bt & 3u) * 8u)) & 0xFFu);
            const int Sv = c + ct;
            const int dg = i == j ? 1 : 0;
            if (SG > 0) {
                s.A += 2 * (2 * Sv + 1) + 2 * dg;
                s.E += Gt[Sv] + Gt[Sv + dg];
            } else {
                s.A += 2 * (1 - 2 * Sv) + 2 * dg;
                s.E -= Gt[Sv - 1] + Gt[Sv - 1 - dg];
            }
            s.T += 2 * SG;
            s.C += 2 * SG * d * d;
            s.I += 2 * SG * h;
        } else {
            s.A += 2 * SG * c + 1;
            s.E += SG > 0 ? Gt[c] : -Gt[c - 1];
            s.T += SG;
            s.C += SG * d * d;
            s.I += SG * h;
        }
        *w = word + (SG > 0 ? (1u << sh) : (0u - (1u << sh)));
    };
    using Add = std::integral_constant<int, 1>;
    using Rem = std::integral_constant<int, -1>;
    // Votes of n anchors in a row from tile index a0: the levels of four
    // anchors and their partners are read before their votes, so those reads
    // overlap instead of waiting behind each vote's counter update.
    auto vote_run = [&](int a0, int n, auto sg_tag) {
        for (int k0 = 0; k0 < n; k0 += 4) {
            uint32_t ii[4], jj[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int a = a0 + k0 + (k0 + q < n ? q : 0);
                ii[q] = tile[a];
                jj[q] = tile[a + tstep];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (k0 + q < n)
                    vote(ii[q], jj[q], sg_tag);
        }
    };
    const long long plane = (long long)p.nwy * p.nwx;
    auto emit = [&](int wx) {
        const long long win_id = (long long)wy * p.nwx + wx;
        if (p.counts) {
            uint32_t* dst = p.counts + (win_id * p.n_off + o) * NN;
            if (vec_counts) {
                for (int k = 0; k < hw; ++k) {
                    const uint32_t w = hl[k * 32];
                    reinterpret_cast<uint4*>(dst)[k] =
                        make_uint4(w & 0xFFu, (w >> 8) & 0xFFu, (w >> 16) & 0xFFu, w >> 24);
                }
            } else {
                for (int b = 0; b < NN; ++b)
                    dst[b] = (hl[(b >> 2) * 32] >> ((b & 3) * 8)) & 0xFFu;
            }
        }
        if (p.maps) {
            float con = 0.f, asmv = 0.f, idm = 0.f, ent = 0.f;
            if (s.T > 0) {
                // Exact integers (C, A, T^2 < 2^24) or exact fixed-point sums
                // scaled by a power of two: one rounding each, then a division.
                const float T = (float)s.T;
                const float inv_fix = 1.0f / (float)kFix;
                con = __fdiv_rn((float)s.C, T);
                asmv = __fdiv_rn((float)s.A, __fmul_rn(T, T));
                idm = __fdiv_rn(__fmul_rn(__ll2float_rn(s.I), inv_fix), T);
                ent = __fdiv_rn(__fmul_rn(__ll2float_rn(PGt[s.T] - s.E), inv_fix), T);
            }
            p.maps[(0ll * p.n_off + o) * plane + win_id] = con;
            p.maps[(1ll * p.n_off + o) * plane + win_id] = asmv;
            p.maps[(2ll * p.n_off + o) * plane + win_id] = idm;
            p.maps[(3ll * p.n_off + o) * plane + win_id] = ent;
        }
    };

    const int Y0 = task * S;  // the window's top row in the tile
    // First window of the row: every pair.
    for (int y = aylo; y < ayhi; ++y)
        vote_run((Y0 + y) * RWp + axlo, axhi - axlo, Add{});
    emit(wx0);
    // Slides: the anchor columns [X0 + axlo, X0 + axhi) become [X1 + axlo, X1 + axhi).
    for (int k = 1; k < n_w; ++k) {
        const int X0 = (k - 1) * S, X1 = k * S;
        const int r_end = min(X0 + axhi, X1 + axlo);
        const int a_beg = max(X0 + axhi, X1 + axlo);
        for (int y = aylo; y < ayhi; ++y) {
            const int row = (Y0 + y) * RWp;
            vote_run(row + X0 + axlo, r_end - (X0 + axlo), Rem{});
            vote_run(row + a_beg, X1 + axhi - a_beg, Add{});
        }
        emit(wx0 + k);
    }
    if (bad)
        atomicOr(p.err, kErrRange);
}

}  // namespace

void window_slide_tables(long long* out)
{
    long long* G = out;
    long long* PG = out + kSlideG;
    long long* H = PG + kSlideG + 1;
    PG[0] = 0;
    for (int c = 0; c < kSlideG; ++c) {
        const double cd = (double)c;
        const double g = (cd + 1.0) * std::log(cd + 1.0) - (c > 0 ? cd * std::log(cd) : 0.0);
        G[c] = std::llrint(g * kFix);
        PG[c + 1] = PG[c] + G[c];
    }
    for (int d = 0; d < 32; ++d)
        H[d] = std::llrint(kFix / (1.0 + (double)d * d));
}

// The incremental kernel, when the windows fit it: N <= 16, at most 8
// offsets, at most 255 pairs per window and offset (8-bit counters) and a
// staged tile that fits shared memory.  Returns cudaErrorNotSupported
// otherwise (the caller then recounts every window).
cudaError_t launch_windows_slide(const WindowParams& p, cudaStream_t s)
{
    if (p.nwx <= 0 || p.nwy <= 0)
        return cudaSuccess;
    if (p.levels > 16 || p.n_off < 1 || p.n_off > 8 || !p.slide_tables)
        return cudaErrorNotSupported;
    for (int o = 0; o < p.n_off; ++o)
        if ((long long)(p.win - abs(p.dx[o])) * (p.win - abs(p.dy[o])) > 255)
            return cudaErrorNotSupported;
    const int lpw = p.n_off <= 1 ? 1 : (p.n_off <= 2 ? 2 : (p.n_off <= 4 ? 4 : 8));
    const int tasks = kSlideWarps * (32 / lpw);
    const int NN = p.levels * p.levels;
    const int hw = (NN + 3) / 4;
    const size_t hist_bytes = (size_t)kSlideWarps * hw * 32 * 4;
    const size_t fixed = (size_t)kSlideTableWords * 8 + hist_bytes;
    const int RH = (tasks - 1) * p.stride + p.win;
    // Windows per task: as many as keep the tile within 96 KB (a slide costs
    // what a first window costs once per task), at least one, and enough
    // CTAs to cover the GPU twice.
    const size_t tile_budget = 96 * 1024;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int row_blocks = (p.nwy + tasks - 1) / tasks;
    int seg = 64;
    while (seg > 4 && (long long)row_blocks * ((p.nwx + seg - 1) / seg) < 2ll * sms)
        seg /= 2;
    int RW = (seg - 1) * p.stride + p.win;
    while (seg > 1 && (size_t)RH * RW > tile_budget) {
        --seg;
        RW = (seg - 1) * p.stride + p.win;
    }
    if ((size_t)RH * RW > tile_budget)
        return cudaErrorNotSupported;
    // Tile row pitch: rows `stride` apart (the tasks of a warp) start in
    // different banks.
    int RWp = RW;
    while ((((long long)p.stride * RWp / 4) & 1) == 0 && RWp < RW + 128)
        ++RWp;
    const size_t smem = fixed + (((size_t)RH * RWp + 15) & ~(size_t)15);
    if (smem > (size_t)vote_max_smem_optin())
        return cudaErrorNotSupported;
    int vec = (NN % 4 == 0 && (reinterpret_cast<uintptr_t>(p.counts) & 15) == 0) ? 1 : 0;
    const void* fn = lpw == 1 ? (const void*)k_window_slide<1>
                              : (lpw == 2 ? (const void*)k_window_slide<2>
                                          : (lpw == 4 ? (const void*)k_window_slide<4> : (const void*)k_window_slide<8>));
    static SmemLimit lim[4];
    const int li = lpw == 1 ? 0 : (lpw == 2 ? 1 : (lpw == 4 ? 2 : 3));
    const cudaError_t e = lim[li].raise(fn, smem);
    if (e != cudaSuccess)
        return e;
    const dim3 grid((p.nwx + seg - 1) / seg, row_blocks);
    int seg_a = seg, RH_a = RH, RW_a = RW, RWp_a = RWp, hw_a = hw;
    WindowParams pc = p;
    void* args[] = {&pc, &seg_a, &RH_a, &RW_a, &RWp_a, &hw_a, &vec};
    return cudaLaunchKernel(fn, grid, dim3(kSlideThreads), args, smem, s);
}

}  // namespace glcm
