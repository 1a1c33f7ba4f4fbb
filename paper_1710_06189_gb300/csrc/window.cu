// Sliding-window local GLCMs and texture maps.
//
// Each win x win window (top-left pixel at (wx*stride, wy*stride)) gets its
// own GLCM of Eq. (1) over the pairs whose two pixels both lie inside the
// window, for every offset, and optionally four float32 maps per offset:
// contrast, angular second moment, inverse difference moment and entropy
// (Haralick's f2, f1, f5 and f9 of the window's normalized GLCM).
//
// One CTA covers a block of 8 x 4 windows and stages the pixels they span,
// quantized to levels, in shared memory once; each warp then owns one window
// and keeps its histograms in shared memory with 8- or 16-bit counters
// packed into words (a window of 15 x 15 has at most 225 pairs per offset).
// The counter width is a template parameter and power-of-two N takes shifts,
// so no vote, count or map bin needs an integer division.
#include "glcm_internal.cuh"

namespace glcm {
namespace {

constexpr int kWX = 8, kWY = 4;  // windows per CTA
constexpr int kWinThreads = 32 * kWX * kWY;
constexpr uint16_t kBadLevel = 0xFFFFu;

__device__ __forceinline__ uint32_t px_at(const WindowParams& p, int x, int y)
{
    const uint8_t* row = p.img + (long long)y * p.pitch;
    if (p.bpp == 1)
        return __ldg(row + x);
    return (uint32_t)__ldg(row + 2 * x) | ((uint32_t)__ldg(row + 2 * x + 1) << 8);
}

// Row and column of bin b of an N x N GLCM (l2 = log2 N, or -1).
__device__ __forceinline__ void bin_ij(int b, int N, int l2, int& i, int& j)
{
    if (l2 >= 0) {
        i = b >> l2;
        j = b & (N - 1);
    } else {
        i = b / N;
        j = b - i * N;
    }
}

template <int CB>
__global__ void __launch_bounds__(kWinThreads) k_window_glcm(WindowParams p, int hist_words)
{
    constexpr int kPwLog = CB == 8 ? 2 : (CB == 16 ? 1 : 0);  // log2(counters per word)
    constexpr uint32_t kPwMask = (1u << kPwLog) - 1u;
    constexpr uint32_t cmask = CB == 32 ? 0xFFFFFFFFu : ((1u << CB) - 1u);
    extern __shared__ __align__(16) uint32_t sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.stride, Wn = p.win, N = p.levels, NN = N * N;
    const int RW = (kWX - 1) * S + Wn, RH = (kWY - 1) * S + Wn;
    const int rx0 = blockIdx.x * kWX * S, ry0 = blockIdx.y * kWY * S;
    uint16_t* lv = reinterpret_cast<uint16_t*>(sm);
    const int lv_words = (RW * RH + 1) / 2;
    uint32_t* hist = sm + lv_words + warp * hist_words;

    for (int t = threadIdx.x; t < RW * RH; t += blockDim.x) {
        const int ly = t / RW, lx = t - ly * RW;
        const int x = rx0 + lx, y = ry0 + ly;
        uint16_t v = kBadLevel;
        if (x < p.W && y < p.H) {
            const uint32_t raw = px_at(p, x, y);
            const uint32_t q = p.levels_mode ? raw
                                             : (uint32_t)(((unsigned long long)raw * (unsigned)N) >> (8 * p.bpp));
            v = q < (uint32_t)N ? (uint16_t)q : kBadLevel;
        }
        lv[t] = v;
    }
    __syncthreads();

    const int wxl = warp % kWX, wyl = warp / kWX;
    const int wx = blockIdx.x * kWX + wxl, wy = blockIdx.y * kWY + wyl;
    if (wx >= p.nwx || wy >= p.nwy)
        return;
    for (int k = lane; k < hist_words; k += 32)
        hist[k] = 0u;
    __syncwarp();
    const int lx0 = wxl * S, ly0 = wyl * S;
    const int l2 = (N & (N - 1)) == 0 ? __ffs(N) - 1 : -1;
    const uint32_t hist_base = static_cast<uint32_t>(__cvta_generic_to_shared(hist));
    bool bad = false;
    // Anchor t = lane + 32k of the window as (ay, ax), stepped without divisions.
    const int q32 = 32 / Wn, r32 = 32 - q32 * Wn;
    int ay = lane / Wn, ax = lane - ay * Wn;
    for (int t = lane; t < Wn * Wn; t += 32) {
        const uint32_t i = lv[(ly0 + ay) * RW + lx0 + ax];
        for (int o = 0; o < p.n_off; ++o) {
            const int bx = ax + p.dx[o], by = ay + p.dy[o];
            if (bx < 0 || bx >= Wn || by < 0 || by >= Wn)
                continue;
            const uint32_t jv = lv[(ly0 + by) * RW + lx0 + bx];
            if (i >= (uint32_t)N || jv >= (uint32_t)N) {
                bad = true;
                continue;
            }
            const uint32_t idx = (uint32_t)(o * NN) + i * (uint32_t)N + jv;
            const uint32_t word = idx >> kPwLog;
            const uint32_t sh = (idx & kPwMask) * CB;
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(hist_base + 4u * word), "r"(1u << sh));
        }
        ax += r32;
        ay += q32;
        if (ax >= Wn) {
            ax -= Wn;
            ++ay;
        }
    }
    if (bad)
        atomicOr(p.err, kErrRange);
    __syncwarp();

    const long long win_id = (long long)wy * p.nwx + wx;
    auto count_of = [&](uint32_t idx) { return (hist[idx >> kPwLog] >> ((idx & kPwMask) * CB)) & cmask; };
    for (int o = 0; o < p.n_off; ++o) {
        // Counts out and the window's total for this offset.
        unsigned long long tot = 0;
        for (int b = lane; b < NN; b += 32) {
            const uint32_t c = count_of((uint32_t)(o * NN + b));
            tot += c;
            if (p.counts)
                p.counts[(win_id * p.n_off + o) * NN + b] = c;
        }
        for (int s = 16; s > 0; s >>= 1)
            tot += __shfl_xor_sync(0xffffffffu, tot, s);
        if (!p.maps)
            continue;
        const float Tf = p.symmetric ? 2.f * (float)tot : (float)tot;
        const float invT = tot > 0 ? __frcp_rn(Tf) : 0.f;  // p = c / T as c * (1 / T): within 1.5 ulp
        float con = 0.f, asmv = 0.f, idm = 0.f, ent = 0.f;
        if (tot > 0) {
            for (int b = lane; b < NN; b += 32) {
                int i, j;
                bin_ij(b, N, l2, i, j);
                uint32_t c = count_of((uint32_t)(o * NN + b));
                if (p.symmetric)
                    c += count_of((uint32_t)(o * NN + j * N + i));
                if (!c)
                    continue;
                const float pv = __fmul_rn((float)c, invT);
                const float d2 = (float)((i - j) * (i - j));
                con = __fadd_rn(con, __fmul_rn(d2, pv));
                asmv = __fadd_rn(asmv, __fmul_rn(pv, pv));
                idm = __fadd_rn(idm, __fmul_rn(pv, __frcp_rn(__fadd_rn(1.f, d2))));
                ent = __fsub_rn(ent, __fmul_rn(pv, logf(pv)));
            }
        }
        for (int s = 16; s > 0; s >>= 1) {
            con += __shfl_xor_sync(0xffffffffu, con, s);
            asmv += __shfl_xor_sync(0xffffffffu, asmv, s);
            idm += __shfl_xor_sync(0xffffffffu, idm, s);
            ent += __shfl_xor_sync(0xffffffffu, ent, s);
        }
        if (lane == 0) {
            const long long plane = (long long)p.nwy * p.nwx;
            p.maps[(0ll * p.n_off + o) * plane + win_id] = con;
            p.maps[(1ll * p.n_off + o) * plane + win_id] = asmv;
            p.maps[(2ll * p.n_off + o) * plane + win_id] = idm;
            p.maps[(3ll * p.n_off + o) * plane + win_id] = ent;
        }
    }
}

}  // namespace

cudaError_t launch_windows(const WindowParams& p, cudaStream_t s)
{
    if (p.nwx <= 0 || p.nwy <= 0)
        return cudaSuccess;
    // Windows that fit the incremental kernel slide (window_slide.cu).
    const cudaError_t es = launch_windows_slide(p, s);
    if (es != cudaErrorNotSupported)
        return es;
    long long maxpairs = (long long)p.win * p.win;
    const int cbits = maxpairs <= 255 ? 8 : (maxpairs <= 65535 ? 16 : 32);
    const long long bins = (long long)p.n_off * p.levels * p.levels;
    const int hist_words = (int)((bins * cbits + 31) / 32);
    const int RW = (kWX - 1) * p.stride + p.win, RH = (kWY - 1) * p.stride + p.win;
    const size_t smem = (size_t)((RW * RH + 1) / 2) * 4 + (size_t)hist_words * 4 * kWX * kWY;
    if (smem > (size_t)vote_max_smem_optin())
        return cudaErrorInvalidConfiguration;
    static SmemLimit lim[3];
    const int ci = cbits == 8 ? 0 : (cbits == 16 ? 1 : 2);
    {
        const void* fn = cbits == 8 ? (const void*)k_window_glcm<8>
                                    : (cbits == 16 ? (const void*)k_window_glcm<16> : (const void*)k_window_glcm<32>);
        const cudaError_t e = lim[ci].raise(fn, smem);
        if (e != cudaSuccess)
            return e;
    }
    dim3 grid((p.nwx + kWX - 1) / kWX, (p.nwy + kWY - 1) / kWY);
    if (cbits == 8)
        k_window_glcm<8><<<grid, kWinThreads, smem, s>>>(p, hist_words);
    else if (cbits == 16)
        k_window_glcm<16><<<grid, kWinThreads, smem, s>>>(p, hist_words);
    else
        k_window_glcm<32><<<grid, kWinThreads, smem, s>>>(p, hist_words);
    return cudaGetLastError();
}

}  // namespace glcm
