// GLCM epilogue: symmetrize, normalize and the 14 Haralick features.
//
// The paper names Haralick's fourteen statistics as the use of each GLCM
// (Sec. I, introduction) without defining them; the definitions used are the
// textbook ones (see the header for the list).  One CTA handles one GLCM.
//
// Precision plan (the counts stay exact integers throughout):
//  * All marginals (rows, columns, i+j and |i-j| sums) and the total T are
//    exact 64-bit integer sums of the counts; moments that are integer
//    combinations (contrast, sum average, means of the sum and difference
//    distributions) are exact integers divided once by T.
//  * Every other sum is float32 with Kahan compensation per thread and a
//    two-sum (error-free) block reduction; no fused multiply-add contraction
//    is allowed in those sums (__fadd_rn / __fmul_rn).
//  * Correlation (f3) and sum of squares (f4) come from exact integer
//    moments: T^2 var = T sum i^2 r_i - (sum i r_i)^2 and T^2 cov =
//    T sum i j S(i, j) - (sum i r_i)(sum j c_j) in 128-bit integers, turned
//    into float64 once by one thread (float64 is slow on this GPU, so no
//    thread does float64 arithmetic per cell).
//  * f12 and f13 are functions of the mutual information
//    I = HX + HY - HXY (= HXY1 - HXY = HXY2 - HXY, since HXY1 = HXY2 =
//    HX + HY).  I is summed as sum q * phi(x) with q = p_x p_y,
//    x = p/q - 1 = (S*T - r*c)/(r*c) from an exact integer numerator and
//    phi(x) = (1+x) ln(1+x) - x >= 0 (a series for small |x|), so no term
//    cancels another and tiny I stays accurate in float32.
//  * f14 is the second largest singular value of A = D_x^-1/2 P D_y^-1/2
//    (its square is the second eigenvalue of Q).  The known top pair
//    (singular value 1, vectors sqrt(p_x), sqrt(p_y)) is removed exactly:
//    A'(i,j) = (S*T - r*c) / (T sqrt(r c)), and the largest singular value
//    of A' is found by Golub-Kahan-Lanczos bidiagonalization with full
//    reorthogonalization in float32, stopped when its top Ritz value
//    settles (exact after min(rows, cols) steps).  Supports of at most 32
//    levels instead square G = A'^T A' (or A' A'^T) repeatedly with the
//    whole block and take a Rayleigh quotient: a few dozen barrier-separated
//    steps instead of a serial chain of Lanczos steps in one warp.
//  * Symmetric GLCMs with 128 < N <= 256 (A' symmetric, too large for one
//    CTA's shared memory as a full matrix) are spread over a cluster of
//    eight CTAs (k_haralick_cluster, below): each keeps 32 rows of A' in
//    shared memory, and max |eigenvalue| of A' -- its largest singular
//    value -- comes from symmetric Lanczos without reorthogonalization: in
//    finite precision the extreme Ritz values still converge (lost
//    orthogonality only adds copies of converged values), so no basis has
//    to be stored.
#include <cmath>

#include "glcm_internal.cuh"

namespace glcm {
namespace {

constexpr int kNumFeat = 14;
constexpr int kMaxLanczos = 96;
// A' and the Lanczos vectors stay in shared memory up to these sizes
// (covers supports up to 128 x 128); larger ones use global scratch.
constexpr int kSmemAFloats = 128 * 128;
constexpr int kSmemUVFloats = (2 * kMaxLanczos + 1) * 128;
constexpr int kColGroups = 4;
constexpr int kMaxSymSteps = 384;
constexpr int kMaxLevelsPerLane = 256 / 32;  // N <= 256
// Repeated squaring for supports of at most 32 levels: row stride (16-byte
// rows, conflict-free float4 reads), minimum and maximum squarings, floats.
constexpr int kSqLD = 36;
constexpr int kSqMin = 13;
constexpr int kSqMax = 30;
constexpr int kSqFloats = 96 * kSqLD + 64;

struct DF {  // float value hi + lo (unevaluated sum)
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    const float l = __fadd_rn(__fadd_rn(a.lo, b.lo), e);
    DF r;
    two_sum(s, l, r.hi, r.lo);
    return r;
}

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ DF df() const { return DF{s, -c}; }
};

// phi(x) = (1 + x) ln(1 + x) - x for x >= -1 (phi >= 0, phi(-1) = 1).
__device__ __forceinline__ float phi(float x)
{
    if (x <= -1.f)
        return 1.f;
    if (fabsf(x) < 0.0625f) {
        // With u = -x: phi = sum_{n>=2} u^n / (n (n - 1)), kept through u^8.
        const float u = -x;
        float t = 1.f / 56.f;
        t = __fadd_rn(__fmul_rn(t, u), 1.f / 42.f);
        t = __fadd_rn(__fmul_rn(t, u), 1.f / 30.f);
        t = __fadd_rn(__fmul_rn(t, u), 1.f / 20.f);
        t = __fadd_rn(__fmul_rn(t, u), 1.f / 12.f);
        t = __fadd_rn(__fmul_rn(t, u), 1.f / 6.f);
        t = __fadd_rn(__fmul_rn(t, u), 0.5f);
        return __fmul_rn(__fmul_rn(x, x), t);
    }
    return __fsub_rn(__fmul_rn(__fadd_rn(1.f, x), log1pf(x)), x);
}

template <int K>
__device__ void block_reduce_df(DF (&v)[K], DF* scratch /* K * 32 */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            DF t;
            t.hi = __shfl_down_sync(0xffffffffu, v[k].hi, o);
            t.lo = __shfl_down_sync(0xffffffffu, v[k].lo, o);
            v[k] = df_add(v[k], t);
        }
        if (lane == 0)
            scratch[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            DF a = lane < nw ? scratch[k * 32 + lane] : DF{0.f, 0.f};
            for (int o = 16; o > 0; o >>= 1) {
                DF t;
                t.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
                t.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
                a = df_add(a, t);
            }
            if (lane == 0)
                scratch[k * 32] = a;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k)
        v[k] = scratch[k * 32];
    __syncthreads();
}

// Signed 128-bit integer to double (the two 64-bit halves, rounded once each).
__device__ __forceinline__ double i128_to_double(__int128 v)
{
    const bool neg = v < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const double d = (double)(unsigned long long)(u >> 64) * 18446744073709551616.0 + (double)(unsigned long long)u;
    return neg ? -d : d;
}

__device__ __forceinline__ unsigned long long cell(const uint32_t* C, int N, int i, int j, int sym)
{
    unsigned long long s = __ldg(C + i * N + j);
    if (sym)
        s += __ldg(C + j * N + i);
    return s;
}

// m / T for exact integer sums: the integer quotient plus the remainder's
// fraction, so an integral mean comes out exact however large T is (a float
// quotient of the two rounded integers can miss it by an ulp).
__device__ __forceinline__ float ratio_u64(unsigned long long m, unsigned long long T)
{
    const unsigned long long q = m / T;
    return __fadd_rn((float)q, __fdiv_rn((float)(m - q * T), (float)T));
}

__device__ __forceinline__ float neg_plogp(float p)
{
    return p > 0.f ? -__fmul_rn(p, logf(p)) : 0.f;
}

__device__ __forceinline__ float warp_sum(float s)
{
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Sum over the block; every thread gets the result.
__device__ float block_sum(float s, float* s_red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    s = warp_sum(s);
    if (lane == 0)
        s_red[warp] = s;
    __syncthreads();
    // Every warp reduces the partials the same way; lane 0's total is
    // broadcast so that all threads hold the same value.
    float t = lane < nw ? s_red[lane] : 0.f;
    t = __shfl_sync(0xffffffffu, warp_sum(t), 0);
    __syncthreads();
    return t;
}

// y = A x for the m x n column-major A (leading dim m); x, y in shared memory.
// Warps own 32-row blocks and split the columns into kColGroups strided
// groups, four independent products in flight per lane.
__device__ void matvec(const float* __restrict__ A, int m, int n, const float* x, float* y, float* part)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rbs = (m + 31) >> 5;
    const int groups = max(1, min(kColGroups, nw / rbs));
    for (int w = warp; w < rbs * groups; w += nw) {
        const int rb = w % rbs, g = w / rbs;
        const int r = rb * 32 + lane;
        if (r >= m)
            continue;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int c = g;
        for (; c + 3 * groups < n; c += 4 * groups) {
            a0 = fmaf(A[(long long)c * m + r], x[c], a0);
            a1 = fmaf(A[(long long)(c + groups) * m + r], x[c + groups], a1);
            a2 = fmaf(A[(long long)(c + 2 * groups) * m + r], x[c + 2 * groups], a2);
            a3 = fmaf(A[(long long)(c + 3 * groups) * m + r], x[c + 3 * groups], a3);
        }
        for (; c < n; c += groups)
            a0 = fmaf(A[(long long)c * m + r], x[c], a0);
        part[g * 256 + r] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        float s = 0.f;
        for (int g = 0; g < groups; ++g)
            s += part[g * 256 + r];
        y[r] = s;
    }
    __syncthreads();
}

// x = A^T y: one warp per column, lanes over the rows.
__device__ void matvec_t(const float* __restrict__ A, int m, int n, const float* y, float* x)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int c = warp; c < n; c += nw) {
        const float* col = A + (long long)c * m;
        float a0 = 0.f, a1 = 0.f;
        int r = lane;
        for (; r + 32 < m; r += 64) {
            a0 = fmaf(col[r], y[r], a0);
            a1 = fmaf(col[r + 32], y[r + 32], a1);
        }
        if (r < m)
            a0 = fmaf(col[r], y[r], a0);
        const float s = warp_sum(a0 + a1);
        if (lane == 0)
            x[c] = s;
    }
    __syncthreads();
}

// v -= sum_i <v, Q_i> Q_i over rows i < k of Q (len-long rows), twice.
__device__ void reorth(float* v, const float* __restrict__ Q, int k, int len, float* s_coef)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = warp; i < k; i += nw) {
            const float* q = Q + (long long)i * len;
            float s = 0.f;
            for (int r = lane; r < len; r += 32)
                s = fmaf(v[r], q[r], s);
            s = warp_sum(s);
            if (lane == 0)
                s_coef[i] = s;
        }
        __syncthreads();
        for (int r = threadIdx.x; r < len; r += blockDim.x) {
            // Four independent chains so that the loads of a group issue together.
            float a0 = v[r], a1 = 0.f, a2 = 0.f, a3 = 0.f;
            const float* q = Q + r;
            int i = 0;
            for (; i + 3 < k; i += 4) {
                a0 = fmaf(-s_coef[i], q[(long long)i * len], a0);
                a1 = fmaf(-s_coef[i + 1], q[(long long)(i + 1) * len], a1);
                a2 = fmaf(-s_coef[i + 2], q[(long long)(i + 2) * len], a2);
                a3 = fmaf(-s_coef[i + 3], q[(long long)(i + 3) * len], a3);
            }
            for (; i < k; ++i)
                a0 = fmaf(-s_coef[i], q[(long long)i * len], a0);
            v[r] = (a0 + a1) + (a2 + a3);
        }
        __syncthreads();
    }
}

// Number of eigenvalues below x of the (L+1) x (L+1) zero-diagonal
// tridiagonal matrix with off-diagonals ab[0..L) (Sturm sequence).
__device__ __forceinline__ int sturm_below(const float* ab, int L, float x)
{
    int cnt = 0;
    float q = -x;
    if (q < 0.f)
        ++cnt;
    for (int t = 0; t < L; ++t) {
        const float b = ab[t];
        if (q == 0.f)
            q = -1e-30f;
        q = -x - __fdividef(b * b, q);
        if (q < 0.f)
            ++cnt;
    }
    return cnt;
}

// One multisection round of one end of a spectrum by the warps [w0, w0 + nw)
// (mine: the calling warp is one of them) over the points x(0) < ... <
// x(32 nw - 1) inside the bracket [a, b]: each point tests whether every
// eigenvalue (upper) or none (lower) lies below it, and the bracket shrinks
// to the interval between the two neighbouring points where the answer
// changes.  Every thread of the block calls (one barrier); a and b are
// meaningful in the calling warps.  msk: 32 words, not reused by the next
// round.
template <class F, class X>
__device__ __forceinline__ void multisect_round(F below, int n_eig, X x, float& a, float& b, bool upper, bool mine,
                                                int w0, int nw, unsigned* msk)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int P = 32 * nw;
    if (mine) {
        const int c = below(x((warp - w0) * 32 + lane));
        const unsigned m = __ballot_sync(0xffffffffu, upper ? c >= n_eig : c == 0);
        if (lane == 0)
            msk[warp - w0 + (upper ? 0 : 16)] = m;
    }
    __syncthreads();
    if (mine) {
        const unsigned* mk = msk + (upper ? 0 : 16);
        float na, nb;
        if (upper) {
            int idx = P;  // first point above every eigenvalue
            for (int w = nw - 1; w >= 0; --w)
                if (mk[w])
                    idx = 32 * w + __ffs(mk[w]) - 1;
            na = idx == 0 ? a : x(idx - 1);
            nb = idx == P ? b : x(idx);
        } else {
            int idx = -1;  // last point below every eigenvalue
            for (int w = 0; w < nw; ++w)
                if (mk[w])
                    idx = 32 * w + 31 - __clz(mk[w]);
            na = idx < 0 ? a : x(idx);
            nb = idx == P - 1 ? b : x(idx + 1);
        }
        a = na;
        b = nb;
    }
}

// Multisection of one end of a spectrum by the warps [w0, w0 + nw): `rounds`
// rounds, each splitting the bracket evenly into 32 nw + 1 parts.  A fixed
// number of rounds, so that every thread of the block passes the same
// barriers; the returned midpoint is meaningful in the calling warps.
// s_msk: 2 x 32 words.
template <class F>
__device__ float block_multisect(F below, int n_eig, float a, float b, bool upper, int w0, int nw, int rounds,
                                 unsigned (*s_msk)[32])
{
    const int warp = threadIdx.x >> 5;
    const bool mine = warp >= w0 && warp < w0 + nw;
    const float den = (float)(32 * nw + 1);
    for (int r = 0; r < rounds; ++r) {
        auto even = [=](int pt) { return a + (b - a) * (float)(pt + 1) / den; };
        multisect_round(below, n_eig, even, a, b, upper, mine, w0, nw, s_msk[r & 1]);
    }
    return 0.5f * (a + b);
}

// The Golub-Kahan bidiagonal matrix after k steps has diagonal alpha_i =
// ab[2i] and superdiagonal beta_i = ab[2i+1]; its singular values are the
// non-negative eigenvalues of the zero-diagonal tridiagonal matrix with
// off-diagonals alpha_0, beta_0, alpha_1, ... (eigenvalues +-sigma).
// Largest singular value of that bidiagonal matrix by the whole block: three
// rounds of 32 nw-way multisection of [0, 2 max(ab)] (the largest
// eigenvalue of the zero-diagonal tridiagonal matrix); every thread returns it.
__device__ float gk_sigma_max_block(const float* ab, int steps, unsigned (*s_msk)[32])
{
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int L = 2 * steps - 1;
    if (L <= 0)
        return 0.f;
    float hi = 0.f;
    for (int t = lane; t < L; t += 32)
        hi = fmaxf(hi, ab[t]);
    for (int o = 16; o > 0; o >>= 1)
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    hi *= 2.f;
    auto below = [=](float x) { return sturm_below(ab, L, x); };
    return block_multisect(below, L + 1, 0.f, hi, true, 0, nw < 16 ? nw : 16, 3, s_msk);
}

// Largest singular value of the m x n matrix A (column-major, leading
// dimension m; 2 <= m, n <= 32) by the whole block, through repeated
// squaring.  G = A^T A or A A^T (the smaller, order d) has sigma_max^2 as its
// top eigenvalue.  X_0 = G / tr(G) and X_{s+1} = X_s^2 / tr(X_s)^2 keep every
// entry of the positive semidefinite X_s within [0, 1] in magnitude and its
// top eigenvalue at least 1/d^2, while each other eigenvector's weight
// shrinks as (lambda_k / lambda_1)^(2^s) against the top one: X_s tends to
// the projector onto G's top eigenvector(s).  The Rayleigh quotient of G at
// X's column with the largest diagonal entry then gives lambda_1, with an
// error second order in the residual weights.  Squaring stops after at
// least kSqMin steps once tr(X) moved by less than 1e-6 of itself (float
// rounding alone moves it by about 1e-7): the trace stays put only when the
// residual weights are negligible or the gap lambda_1 - lambda_2 is below
// about 3e-3 / 2^kSqMin of lambda_1 (the quotient lies between the two), so
// the error stays within a few float roundings either way.
// Buffers: three 32 x kSqLD matrices and two diagonals (kSqFloats floats,
// 16-byte aligned).  Returns sigma_max in every thread.
// One squaring X' = X^2 * sc of the symmetric D x D block (rows kSqLD floats
// apart; entries beyond the support are zero): warp w takes rows w, w + nw,
// ... (two rows at a time for D = 32, sharing the loads of X's rows k), lane
// b column b, so a row k is read without bank conflicts and X[a][k] is a
// broadcast.  The new diagonal goes to dn.
template <int D>
__device__ __forceinline__ void square_step(const float* __restrict__ X, float* __restrict__ Xn, float* dn,
                                            float sc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (D == 32 && nw == 16) {
        const int a0 = warp, a1 = warp + 16;
        float p0 = 0.f, p1 = 0.f, q0 = 0.f, q1 = 0.f;
#pragma unroll
        for (int k = 0; k < 32; k += 2) {
            const float xk0 = X[k * kSqLD + lane], xk1 = X[(k + 1) * kSqLD + lane];
            p0 = fmaf(X[a0 * kSqLD + k], xk0, p0);
            p1 = fmaf(X[a0 * kSqLD + k + 1], xk1, p1);
            q0 = fmaf(X[a1 * kSqLD + k], xk0, q0);
            q1 = fmaf(X[a1 * kSqLD + k + 1], xk1, q1);
        }
        const float v0 = (p0 + p1) * sc, v1 = (q0 + q1) * sc;
        Xn[a0 * kSqLD + lane] = v0;
        Xn[a1 * kSqLD + lane] = v1;
        if (lane == a0)
            dn[a0] = v0;
        if (lane == a1)
            dn[a1] = v1;
        return;
    }
    for (int a = warp; a < D; a += nw) {
        if (lane < D) {
            float p0 = 0.f, p1 = 0.f;
#pragma unroll
            for (int k = 0; k < D; k += 2) {
                p0 = fmaf(X[a * kSqLD + k], X[k * kSqLD + lane], p0);
                p1 = fmaf(X[a * kSqLD + k + 1], X[(k + 1) * kSqLD + lane], p1);
            }
            const float v = (p0 + p1) * sc;
            Xn[a * kSqLD + lane] = v;
            if (a == lane)
                dn[a] = v;
        }
    }
}

__device__ float sigma_max_squaring(const float* A, int m, int n, float* buf, float* s_out)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int d = min(m, n);
    const bool ata = n <= m;
    // G, then X in two buffers (X_s in buffer s & 1), then their diagonals.
    float* G = buf;
    auto Xb = [&](int c) { return buf + (32 + 32 * c) * kSqLD; };
    auto Db = [&](int c) { return buf + 96 * kSqLD + 32 * c; };
    // Everything is 32 x 32 with zero padding beyond d: fixed, unrolled loops.
    for (int t = threadIdx.x; t < kSqFloats; t += blockDim.x)
        buf[t] = 0.f;
    __syncthreads();
    // For A^T A the lanes read columns of A m floats apart, one bank when m is
    // a multiple of 32: the columns are first copied 33 floats apart into the
    // second X buffer (unused until the first squaring rewrites it whole).
    const float* Ac = A;
    int lda = m;
    if (ata) {
        float* Ap = Xb(1);
        for (int t = threadIdx.x; t < n * m; t += blockDim.x) {
            const int c = t / m, r = t - c * m;
            Ap[c * 33 + r] = A[t];
        }
        __syncthreads();
        Ac = Ap;
        lda = 33;
    }
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        const int a = t >> 5, b = t & 31;
        if (a < d && b < d) {
            float acc = 0.f;
            if (ata) {
                for (int r = 0; r < m; ++r)
                    acc = fmaf(Ac[a * lda + r], Ac[b * lda + r], acc);
            } else {
                for (int c = 0; c < n; ++c)
                    acc = fmaf(A[c * m + a], A[c * m + b], acc);
            }
            G[a * kSqLD + b] = acc;
        }
    }
    __syncthreads();
    // Traces are summed in the same fixed order by every thread, so every
    // thread takes the same decisions.
    auto trace32 = [](const float* v, int stride) {
        float p[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 32; ++k)
            p[k & 3] += v[k * stride];
        return (p[0] + p[1]) + (p[2] + p[3]);
    };
    const float tr = trace32(G, kSqLD + 1);
    if (!(tr > 0.f))
        return 0.f;
    const float inv = 1.f / tr;
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        const int a = t >> 5, b = t & 31;
        const float v = G[a * kSqLD + b] * inv;
        Xb(0)[a * kSqLD + b] = v;
        if (a == b)
            Db(0)[a] = v;
    }
    __syncthreads();
    int cur = 0;
    float prev = 2.f;
    for (int step = 0; step < kSqMax; ++step) {
        // tr X by a warp sum in every warp: the same value in every thread.
        const float trc = warp_sum(lane < 32 ? Db(cur)[lane] : 0.f);
        if (step >= kSqMin && fabsf(trc - prev) <= 1e-6f * trc)
            break;
        prev = trc;
        const float sc = 1.f / (trc * trc);
        if (d <= 8)
            square_step<8>(Xb(cur), Xb(cur ^ 1), Db(cur ^ 1), sc);
        else if (d <= 16)
            square_step<16>(Xb(cur), Xb(cur ^ 1), Db(cur ^ 1), sc);
        else
            square_step<32>(Xb(cur), Xb(cur ^ 1), Db(cur ^ 1), sc);
        __syncthreads();
        cur ^= 1;
    }
    // Column c of X with the largest diagonal entry (every thread, same
    // order), then x^T G x and x^T x for x = column c (X is symmetric) over the
    // whole block: product (a, k) by thread a * 32 + k, fixed-order sums.
    const float* dgc = Db(cur);
    int c = 0;
    for (int k = 1; k < d; ++k)
        c = dgc[k] > dgc[c] ? k : c;
    const float* Xf = Xb(cur);
    float gx = 0.f, xx = 0.f;
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
        const int a = t >> 5, k = t & 31;
        // (Beyond the support the squarings wrote nothing; the second X
        // buffer may still hold the copy of A's columns there.)
        const float xa = a < d ? Xf[a * kSqLD + c] : 0.f, xk = k < d ? Xf[k * kSqLD + c] : 0.f;
        gx = fmaf(G[a * kSqLD + k] * xa, xk, gx);
        if (k == 0)
            xx = fmaf(xa, xa, xx);
    }
    for (int o = 16; o > 0; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        xx += __shfl_xor_sync(0xffffffffu, xx, o);
    }
    float* part = Db(cur ^ 1);  // 32 floats free here
    if (lane == 0 && warp < 16) {
        part[2 * warp] = gx;
        part[2 * warp + 1] = xx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float sg = 0.f, sx = 0.f;
        const int nw = min((int)(blockDim.x >> 5), 16);
        for (int w = 0; w < nw; ++w) {
            sg += part[2 * w];
            sx += part[2 * w + 1];
        }
        *s_out = sqrtf(fmaxf(0.f, sg / sx));
    }
    __syncthreads();
    return *s_out;
}

struct LanczosWork {
    float* xs;    // n floats, shared
    float* ys;    // m floats, shared
    float* part;  // kColGroups * 256 floats, shared
    float* U;     // kMaxLanczos x m (shared or global)
    float* V;     // (kMaxLanczos + 1) x n
    float* coef;  // kMaxLanczos + 1, shared
    float* red;   // 32, shared
    float* ab;    // 2 kMaxLanczos + 2, shared
    float* sig;   // shared scalar
    int* stop;    // shared scalar
    unsigned (*msk)[32];  // shared 2 x 32 words for the multisection
};

// Golub-Kahan-Lanczos bidiagonalization of the m x n matrix A with full
// reorthogonalization; returns the top Ritz value (largest singular value).
__device__ float lanczos_sigma_max(const float* A, int m, int n, const LanczosWork& w)
{
    const int K = min(kMaxLanczos, min(m, n));
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const float v = 1.f + 0.01f * (float)((c * 37) % 11);  // fixed start vector
        w.xs[c] = v;
    }
    if (threadIdx.x == 0) {
        *w.sig = -1.f;
        *w.stop = 0;
    }
    __syncthreads();
    {
        float s = 0.f;
        for (int c = threadIdx.x; c < n; c += blockDim.x)
            s = fmaf(w.xs[c], w.xs[c], s);
        const float inv = rsqrtf(block_sum(s, w.red));
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            w.xs[c] *= inv;
            w.V[c] = w.xs[c];
        }
        __syncthreads();
    }
    int steps = 0;
    float beta = 0.f;
    for (int k = 0; k < K; ++k) {
        // u_k = A v_k - beta_k u_{k-1}, reorthogonalized.
        matvec(A, m, n, w.xs, w.ys, w.part);
        if (k > 0)
            for (int r = threadIdx.x; r < m; r += blockDim.x)
                w.ys[r] = fmaf(-beta, w.U[(long long)(k - 1) * m + r], w.ys[r]);
        __syncthreads();
        reorth(w.ys, w.U, k, m, w.coef);
        float s = 0.f;
        for (int r = threadIdx.x; r < m; r += blockDim.x)
            s = fmaf(w.ys[r], w.ys[r], s);
        const float alpha = sqrtf(block_sum(s, w.red));
        if (threadIdx.x == 0)
            w.ab[2 * k] = alpha;
        if (!(alpha > 1e-30f))
            break;
        const float ia = 1.f / alpha;
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            w.ys[r] *= ia;
            w.U[(long long)k * m + r] = w.ys[r];
        }
        __syncthreads();
        steps = k + 1;
        // v_{k+1} = A^T u_k - alpha_k v_k, reorthogonalized.
        matvec_t(A, m, n, w.ys, w.xs);
        for (int c = threadIdx.x; c < n; c += blockDim.x)
            w.xs[c] = fmaf(-alpha, w.V[(long long)k * n + c], w.xs[c]);
        __syncthreads();
        reorth(w.xs, w.V, k + 1, n, w.coef);
        s = 0.f;
        for (int c = threadIdx.x; c < n; c += blockDim.x)
            s = fmaf(w.xs[c], w.xs[c], s);
        beta = sqrtf(block_sum(s, w.red));
        if (threadIdx.x == 0)
            w.ab[2 * k + 1] = beta;
        if (!(beta > 1e-30f) || k + 1 == K)
            break;
        const float ib = 1.f / beta;
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            w.xs[c] *= ib;
            w.V[(long long)(k + 1) * n + c] = w.xs[c];
        }
        // Every 8 steps: stop once the top Ritz value moved by < 1e-7.
        __syncthreads();
        if (((k + 1) & 7) == 0) {
            const float sg = gk_sigma_max_block(w.ab, k + 1, w.msk);
            if (threadIdx.x == 0) {
                *w.stop = (k + 1 >= 16 && fabsf(sg - *w.sig) <= 1e-7f) ? 1 : 0;
                *w.sig = sg;
            }
            __syncthreads();
            if (*w.stop)
                break;
        }
    }
    __syncthreads();
    return gk_sigma_max_block(w.ab, steps, w.msk);
}

// Eigenvalues below x of the L x L symmetric tridiagonal matrix with
// diagonal al[] and off-diagonal be[] (Sturm sequence).
__device__ __forceinline__ int tri_count_below(const float* al, const float* be, int L, float x)
{
    int cnt = 0;
    float d = al[0] - x;
    if (d < 0.f)
        ++cnt;
    for (int t = 1; t < L; ++t) {
        if (d == 0.f)
            d = -1e-30f;
        d = (al[t] - x) - __fdividef(be[t - 1] * be[t - 1], d);
        if (d < 0.f)
            ++cnt;
    }
    return cnt;
}

// Both ends of a growing tridiagonal matrix as last bracketed: estimates
// (bracket midpoints), max |eigenvalue|, the bound on the inner side of each
// bracket, and each end's move at that check.
struct TriEnds {
    float top, bot, absmax, top_in, bot_in, dtop, dbot;
};

// max(|lambda_max|, |lambda_min|) of the L x L symmetric tridiagonal matrix
// with diagonal al[] and off-diagonal be[], into e (every thread of the
// block calls; e is written by thread 0 and read after the last barrier).
// The first half of the warps brackets the top end, the second half the
// bottom end, inside the Gershgorin interval.  Cold: four rounds of even
// multisection.  Warm, when e holds the ends of the matrix's leading
// (L - k) x (L - k) block: by Cauchy interlacing the top end can only rise
// and the bottom end only fall as rows are added, so each lies on the outer
// side of the previous bracket's inner bound.  The first round then puts
// half of its points evenly within a reach of that bound (four times the
// end's last move, at least 1e-5 of max |eigenvalue|), where a converging end
// lands, and the other half geometrically out to the Gershgorin bound; one
// even round follows.
__device__ void tri_ends_block(const float* al, const float* be, int L, bool warm, TriEnds& e,
                               unsigned (*s_msk)[32])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int half = nw / 2 < 16 ? nw / 2 : 16;
    float lo = 3.4e38f, hi = -3.4e38f;
    for (int t = lane; t < L; t += 32) {
        const float b0 = t > 0 ? fabsf(be[t - 1]) : 0.f, b1 = t + 1 < L ? fabsf(be[t]) : 0.f;
        lo = fminf(lo, al[t] - b0 - b1);
        hi = fmaxf(hi, al[t] + b0 + b1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (L <= 0)
        lo = hi = 0.f;
    auto below = [=](float x) { return tri_count_below(al, be, L, x); };
    const bool up = warp < half, mine = warp < 2 * half;
    const int w0 = up ? 0 : half;
    float a = lo, b = hi;
    int rounds = 4;
    if (warm) {
        // The inner bound moves in by a little more than the counts'
        // rounding, so that the end cannot lie on its inner side.
        const float v = e.absmax, eps = 1e-6f * v + 1e-30f;
        const float in = up ? fminf(fmaxf(e.top_in - eps, lo), hi) : fmaxf(fminf(e.bot_in + eps, hi), lo);
        const float span = up ? hi - in : in - lo;
        const float R = fminf(fmaxf(4.f * (up ? e.dtop : e.dbot), 1e-5f * v) + 1e-30f, span);
        const float lg = R > 0.f ? log2f(span / R) : 0.f;
        const int H = 16 * half, P = 32 * half;
        // Distance from the inner bound of the q-th point outward.
        auto off = [=](int q) {
            return q < H ? R * (float)(q + 1) / (float)H : R * exp2f(lg * (float)(q + 1 - H) / (float)H);
        };
        auto warm_x = [=](int pt) { return up ? in + off(pt) : in - off(P - 1 - pt); };
        if (up)
            a = in;
        else
            b = in;
        multisect_round(below, L, warm_x, a, b, up, mine, w0, half, s_msk[0]);
        rounds = 1;
    }
    const float den = (float)(32 * half + 1);
    for (int r = warm ? 1 : 0; r < (warm ? 1 : 0) + rounds; ++r) {
        auto even = [=](int pt) { return a + (b - a) * (float)(pt + 1) / den; };
        multisect_round(below, L, even, a, b, up, mine, w0, half, s_msk[r & 1]);
    }
    if (mine && warp == w0 && lane == 0) {
        const float mid = 0.5f * (a + b);
        if (up) {
            e.dtop = warm ? mid - e.top : 0.f;
            e.top = mid;
            e.top_in = a;
        } else {
            e.dbot = warm ? e.bot - mid : 0.f;
            e.bot = mid;
            e.bot_in = b;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        e.absmax = fmaxf(fabsf(e.top), fabsf(e.bot));
    __syncthreads();
}

// The 14 features from the exact totals and moments (m: sum i r_i,
// sum j c_j, sum k^2 d_k, sum k s_k, sum k d_k, sum i^2 r_i, sum j^2 c_j),
// the exact sum of i j S(i, j) and the ten compensated sums v (ASM, entropy,
// mutual information, IDM, sum variance, sum entropy, difference variance,
// difference entropy, HX, HY).  One thread.
__device__ void write_features(float* feat, unsigned long long T, const unsigned long long* m,
                               unsigned long long cij, const DF (&v)[10], float f6, float mcc)
{
    const float Tf = (float)T;
    // f3 and f4 from exact integer moments: T^2 var_x = T sum i^2 r_i -
    // (sum i r_i)^2, T^2 cov = T sum i j S(i, j) - (sum i r_i)(sum j c_j).
    const __int128 Ti = (__int128)T;
    const __int128 vxn = Ti * (__int128)m[5] - (__int128)m[0] * (__int128)m[0];
    const __int128 vyn = Ti * (__int128)m[6] - (__int128)m[1] * (__int128)m[1];
    const __int128 cvn = Ti * (__int128)cij - (__int128)m[0] * (__int128)m[1];
    const double Td = (double)T;
    const double varx = i128_to_double(vxn) / (Td * Td);
    const double vxy = i128_to_double(vxn) * i128_to_double(vyn);
    const float mi = fmaxf(0.f, v[2].hi + v[2].lo);
    const float hx = v[8].hi + v[8].lo, hy = v[9].hi + v[9].lo;
    const float hmax = fmaxf(hx, hy);
    feat[0] = v[0].hi + v[0].lo;
    feat[1] = (float)m[2] / Tf;
    feat[2] = vxy > 0.0 ? (float)(i128_to_double(cvn) / sqrt(vxy)) : 1.f;
    feat[3] = (float)varx;
    feat[4] = v[3].hi + v[3].lo;
    feat[5] = f6;
    feat[6] = v[4].hi + v[4].lo;
    feat[7] = v[5].hi + v[5].lo;
    feat[8] = v[1].hi + v[1].lo;
    feat[9] = v[6].hi + v[6].lo;
    feat[10] = v[7].hi + v[7].lo;
    feat[11] = hmax > 0.f ? -mi / hmax : 0.f;
    feat[12] = sqrtf(fmaxf(0.f, -expm1f(-2.f * mi)));
    feat[13] = mcc;
}

// Dynamic shared memory layout for a launch whose largest N is `N`.
struct FeatLayout {
    size_t marg, maps, dscr, xs, ys, part, a, uv, total;
};

__host__ __device__ inline FeatLayout feat_layout(int N)
{
    FeatLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    const int K = N < kMaxLanczos ? N : kMaxLanczos;
    const long long nn = (long long)N * N;
    const long long uv = (2ll * K + 1) * N;
    L.marg = take((size_t)5 * N * 8);
    L.maps = take((size_t)2 * N * 4);
    L.dscr = take(10 * 32 * sizeof(DF));
    L.xs = take((size_t)N * 4);
    L.ys = take((size_t)N * 4);
    L.part = take((size_t)kColGroups * 256 * 4);
    L.a = take((size_t)(nn < kSmemAFloats ? nn : kSmemAFloats) * 4);
    // At least kSqFloats: the squaring path for supports <= 32.
    const long long uvf = uv < kSmemUVFloats ? uv : kSmemUVFloats;
    L.uv = take((size_t)(uvf > kSqFloats ? uvf : kSqFloats) * 4);
    L.total = o;
    return L;
}

constexpr int kFeatSmallPerSM = 4;  // CTAs per SM of the N <= 32 instance

// MINB: CTAs per SM the register budget allows -- 1 for the 512-thread
// launch, more for the 256-thread one of GLCMs with N <= 32 (a short,
// barrier-bound epilogue: more CTAs per SM hide each other's waits).  The
// arithmetic is the same in every instance.
template <int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB) k_haralick(FeatParams p, int maxN)
{
    const FeatJob J = p.jobs[blockIdx.x];
    const int N = J.levels;
    const int NN = N * N;
    const int sym = J.symmetric;
    const uint32_t* C = J.counts;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FeatLayout Lo = feat_layout(maxN);
    unsigned long long* rs = reinterpret_cast<unsigned long long*>(smem_raw + Lo.marg);  // N
    unsigned long long* cs = rs + N;                                                    // N
    unsigned long long* ss = cs + N;                                                    // 2N
    unsigned long long* ds = ss + 2 * N;                                                // N
    int* rmap = reinterpret_cast<int*>(smem_raw + Lo.maps);                             // N
    int* cmap = rmap + N;                                                               // N
    DF* dscr = reinterpret_cast<DF*>(smem_raw + Lo.dscr);
    __shared__ unsigned long long s_T, s_m[7], s_cij;
    __shared__ int s_nr, s_nc, s_stop;
    __shared__ float s_red[32], s_coef[kMaxLanczos + 1], s_ab[2 * kMaxLanczos + 2], s_sig;
    __shared__ unsigned s_msk[2][32];

    for (int k = threadIdx.x; k < 5 * N; k += blockDim.x)
        rs[k] = 0ull;
    if (threadIdx.x == 0)
        s_cij = 0ull;
    __syncthreads();
    // Exact integer marginals of P.  Warp w takes rows w, w + nwarps, ...; the
    // row sum is a warp reduction, the other marginals shared atomics.  For
    // S = P + P^T they follow from P's without reading P^T: the row (= column)
    // sums of S are P's row plus column sums, and the i+j and |i-j| sums of S
    // are twice P's.
    for (int i = warp; i < N; i += blockDim.x >> 5) {
        // All of the row's loads are issued before the first atomic.
        uint32_t v[kMaxLevelsPerLane];
#pragma unroll
        for (int u = 0; u < kMaxLevelsPerLane; ++u) {
            const int j = lane + 32 * u;
            v[u] = j < N ? __ldg(C + i * N + j) : 0u;
        }
        unsigned long long rsum = 0;
#pragma unroll
        for (int u = 0; u < kMaxLevelsPerLane; ++u) {
            const int j = lane + 32 * u;
            const unsigned long long s = v[u];
            if (s) {
                rsum += s;
                atomicAdd(&cs[j], s);
                atomicAdd(&ss[i + j], s);
                atomicAdd(&ds[i > j ? i - j : j - i], s);
            }
        }
        for (int o = 16; o > 0; o >>= 1)
            rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
        if (lane == 0)
            rs[i] = rsum;
    }
    __syncthreads();
    if (sym) {
        for (int k = threadIdx.x; k < 2 * N - 1; k += blockDim.x) {
            if (k < N) {
                const unsigned long long t = rs[k] + cs[k];
                rs[k] = t;
                cs[k] = t;
                ds[k] *= 2ull;
            }
            ss[k] *= 2ull;
        }
        __syncthreads();
    }
    // Totals, integer moments and the support maps (warp 0).
    if (warp == 0) {
        unsigned long long T = 0, m_i = 0, m_j = 0, c2 = 0, m_s = 0, m_d = 0, q_i = 0, q_j = 0;
        int nr = 0, nc = 0;
        for (int k0 = 0; k0 < 2 * N; k0 += 32) {
            const int k = k0 + lane;
            const bool inN = k < N;
            const unsigned long long r = inN ? rs[k] : 0ull, c = inN ? cs[k] : 0ull, d = inN ? ds[k] : 0ull;
            const unsigned long long sv = k < 2 * N - 1 ? ss[k] : 0ull;
            T += r;
            m_i += (unsigned long long)k * r;
            m_j += (unsigned long long)k * c;
            c2 += (unsigned long long)k * k * d;
            q_i += (unsigned long long)k * k * r;
            q_j += (unsigned long long)k * k * c;
            m_d += (unsigned long long)k * d;
            m_s += (unsigned long long)k * sv;
            const unsigned rb = __ballot_sync(0xffffffffu, r != 0ull);
            const unsigned cb = __ballot_sync(0xffffffffu, c != 0ull);
            const unsigned below = (1u << lane) - 1u;
            if (inN) {
                rmap[k] = r ? nr + __popc(rb & below) : -1;
                cmap[k] = c ? nc + __popc(cb & below) : -1;
            }
            nr += __popc(rb);
            nc += __popc(cb);
        }
        for (int o = 16; o > 0; o >>= 1) {
            T += __shfl_xor_sync(0xffffffffu, T, o);
            m_i += __shfl_xor_sync(0xffffffffu, m_i, o);
            m_j += __shfl_xor_sync(0xffffffffu, m_j, o);
            c2 += __shfl_xor_sync(0xffffffffu, c2, o);
            m_s += __shfl_xor_sync(0xffffffffu, m_s, o);
            m_d += __shfl_xor_sync(0xffffffffu, m_d, o);
            q_i += __shfl_xor_sync(0xffffffffu, q_i, o);
            q_j += __shfl_xor_sync(0xffffffffu, q_j, o);
        }
        if (lane == 0) {
            s_T = T;
            s_m[0] = m_i;
            s_m[1] = m_j;
            s_m[2] = c2;
            s_m[3] = m_s;
            s_m[4] = m_d;
            s_m[5] = q_i;
            s_m[6] = q_j;
            s_nr = nr;
            s_nc = nc;
        }
    }
    __syncthreads();
    const unsigned long long T = s_T;
    float* feat = J.features;
    if (T == 0ull) {
        for (int t = threadIdx.x; t < NN && J.normalized; t += blockDim.x)
            J.normalized[t] = 0.f;
        if (feat && threadIdx.x < kNumFeat)
            feat[threadIdx.x] = 0.f;
        return;
    }
    const float Tf = (float)T;
    if (!feat) {
        // Normalize only.
        for (int t = threadIdx.x; t < NN && J.normalized; t += blockDim.x) {
            const int i = t / N, j = t - (t / N) * N;
            J.normalized[t] = __fdiv_rn((float)cell(C, N, i, j, sym), Tf);
        }
        return;
    }
    const int nr = s_nr, nc = s_nc;
    const int K = min(kMaxLanczos, min(nr, nc));
    // A' and the Lanczos vectors: shared memory when they fit, else scratch.
    float* gwork = p.work ? p.work + (long long)blockIdx.x * p.work_stride : nullptr;
    const bool a_smem = (long long)nr * nc <= kSmemAFloats && (long long)nr * nc <= (long long)maxN * maxN;
    const long long uv_need = (long long)K * nr + (long long)(K + 1) * nc;
    const bool uv_smem = uv_need <= kSmemUVFloats &&
                         uv_need <= (long long)(2 * min(maxN, kMaxLanczos) + 1) * maxN;
    float* A = a_smem ? reinterpret_cast<float*>(smem_raw + Lo.a) : gwork;
    float* UV = uv_smem ? reinterpret_cast<float*>(smem_raw + Lo.uv)
                        : (gwork ? gwork + (long long)maxN * maxN : nullptr);
    const bool have_work = A != nullptr && UV != nullptr;

    // Cell pass: normalized output, f1, f9, MI terms, covariance, A'.
    Kahan k_asm, k_ent, k_mi;
    unsigned long long cij = 0;  // sum of i j S(i, j), exact
    for (int t = threadIdx.x; t < NN; t += blockDim.x) {
        const int i = t / N, j = t - (t / N) * N;
        const unsigned long long s = cell(C, N, i, j, sym);
        const float pv = __fdiv_rn((float)s, Tf);
        if (J.normalized)
            J.normalized[t] = pv;
        if (s) {
            k_asm.add(__fmul_rn(pv, pv));
            k_ent.add(neg_plogp(pv));
            cij += (unsigned long long)(i * j) * s;
        }
        const unsigned long long r = rs[i], c = cs[j];
        if (r && c) {
            // Exact numerator S*T - r*c while T < 2^31 (all products < 2^62).
            const float rc = __fmul_rn((float)r, (float)c);
            float numf;
            if (T < (1ull << 31))
                numf = (float)((long long)(s * T) - (long long)(r * c));
            else
                numf = __fsub_rn(__fmul_rn((float)s, Tf), rc);
            const float x = __fdiv_rn(numf, rc);
            const float q = __fmul_rn(__fdiv_rn((float)r, Tf), __fdiv_rn((float)c, Tf));
            k_mi.add(__fmul_rn(q, phi(x)));
            if (have_work) {
                const float a = __fdiv_rn(numf, __fmul_rn(Tf, sqrtf(rc)));
                A[(long long)cmap[j] * nr + rmap[i]] = a;
            }
        }
    }

    // Marginal passes (length N or 2N-1).
    Kahan k_idm, k_svar, k_sent, k_dvar, k_dent, k_hx, k_hy;
    const float f6 = ratio_u64(s_m[3], T);
    const float mean_d = ratio_u64(s_m[4], T);
    for (int k = threadIdx.x; k < 2 * N - 1; k += blockDim.x) {
        const float ps = __fdiv_rn((float)ss[k], Tf);
        const float dk = __fsub_rn((float)k, f6);
        k_svar.add(__fmul_rn(__fmul_rn(dk, dk), ps));
        k_sent.add(neg_plogp(ps));
        if (k < N) {
            const float pd = __fdiv_rn((float)ds[k], Tf);
            k_idm.add(__fdiv_rn(pd, (float)(1 + k * k)));
            const float dd2 = __fsub_rn((float)k, mean_d);
            k_dvar.add(__fmul_rn(__fmul_rn(dd2, dd2), pd));
            k_dent.add(neg_plogp(pd));
            k_hx.add(neg_plogp(__fdiv_rn((float)rs[k], Tf)));
            k_hy.add(neg_plogp(__fdiv_rn((float)cs[k], Tf)));
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        cij += __shfl_xor_sync(0xffffffffu, cij, o);
    if (lane == 0 && cij)
        atomicAdd(&s_cij, cij);  // complete after the block reduction's barriers
    DF v[10] = {k_asm.df(), k_ent.df(), k_mi.df(), k_idm.df(), k_svar.df(),
                k_sent.df(), k_dvar.df(), k_dent.df(), k_hx.df(), k_hy.df()};
    block_reduce_df<10>(v, dscr);

    float mcc = 0.f;
    if (nr >= 2 && nr <= 32 && nc <= 32 && a_smem) {
        // Small supports: repeated squaring by the whole block.
        mcc = sigma_max_squaring(A, nr, nc, reinterpret_cast<float*>(smem_raw + Lo.uv), &s_sig);
    } else if (nr >= 2 && have_work) {
        LanczosWork w;
        w.xs = reinterpret_cast<float*>(smem_raw + Lo.xs);
        w.ys = reinterpret_cast<float*>(smem_raw + Lo.ys);
        w.part = reinterpret_cast<float*>(smem_raw + Lo.part);
        w.U = UV;
        w.V = UV + (long long)K * nr;
        w.coef = s_coef;
        w.red = s_red;
        w.ab = s_ab;
        w.sig = &s_sig;
        w.stop = &s_stop;
        w.msk = s_msk;
        mcc = lanczos_sigma_max(A, nr, nc, w);
    }
    if (!have_work && nr >= 2 && threadIdx.x == 0)
        atomicOr(p.err, kErrInternal);

    if (threadIdx.x == 0)
        write_features(feat, T, s_m, s_cij, v, f6, mcc);
}


// ---- Symmetric GLCMs with 128 < N <= 256: one cluster of CTAs per GLCM -----
//
// S = P + P^T, padded to order 256 with zero rows and columns, is split by
// rows over the kClu CTAs of a thread-block cluster: CTA r owns rows
// [32 r, 32 r + 32).  It stages those rows of P and the same columns of P
// (rows of P^T) in shared memory and forms exact integer partial sums of P's
// marginals from them -- one index per thread, no atomics -- then reads the
// other CTAs' partial sums from their shared memory (distributed shared
// memory).  Every CTA thus holds the full marginals and the same totals, so
// every branch below goes the same way in all of them and they all pass the
// same cluster barriers.  Each CTA does the cell pass of its rows (normalized
// output, f1, f9, the mutual-information terms, sum i j S) and keeps its rows
// of A' in shared memory.  f14 is max |eigenvalue| of A' by symmetric Lanczos
// without reorthogonalization: each step multiplies the CTA's rows of A' by
// the current vector, and one cluster barrier exchanges the pieces of the
// result and of its dot product with the vector, written by plain stores
// into every CTA's shared memory.  Sums across CTAs are taken in rank order, and CTA 0
// writes the features, so a GLCM's features do not depend on its batch.

constexpr int kClu = 8;                  // CTAs per GLCM
constexpr int kCR = 32;                  // rows of S per CTA
constexpr int kCN = kClu * kCR;          // padded order of S
constexpr int kCluThreads = 512;
constexpr int kCluWarps = kCluThreads / 32;
// Partial sums of P over a CTA's rows: column sums, i + j sums, |i - j|
// sums, then the row sums of its own rows.
constexpr int kPartCS = 0, kPartSS = kCN, kPartDS = 3 * kCN, kPartRS = 4 * kCN;
constexpr int kPartWords = 4 * kCN + kCR;

struct CluSmem {
    uint32_t pb[kCR * kCN];               // P rows of this CTA; then A' rows (float)
    uint32_t pt[kCN * (kCR + 1)];         // pt[j * 33 + c] = P(j, 32 r + c)
    unsigned long long part[kPartWords];  // read by every CTA of the cluster
    unsigned long long rs[kCN];           // row sums of S (= column sums)
    unsigned long long ss[2 * kCN];       // i + j sums of S
    unsigned long long ds[kCN];           // |i - j| sums of S
    unsigned long long mom[7], T, cij, fin_cij[kClu];
    float qv[2][kCN];                     // Lanczos vectors q_k and q_(k-1) (by step parity)
    __align__(16) float w[2][kCN];        // A' q - beta q_prev, pieces written by every CTA (by step parity)
    __align__(16) float stg[kCR];         // this CTA's entries of A' q - beta q_prev
    float al[kMaxSymSteps], be[kMaxSymSteps];
    TriEnds te;                           // ends of the tridiagonal matrix at the last check
    DF fin[kClu][10];                     // CTA 0: each CTA's compensated sums
    DF dscr[10 * 32];
    float red[32];
    unsigned msk[2][32];
    int nr, stop;
};

__device__ __forceinline__ uint32_t clu_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t clu_id()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

// Address in CTA `rank`'s shared memory of the variable at p in this CTA's.
__device__ __forceinline__ uint32_t clu_addr(const void* p, uint32_t rank)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void clu_st(uint32_t a, float v)
{
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

__device__ __forceinline__ void clu_st4(uint32_t a, float4 v)
{
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ void clu_st64(uint32_t a, unsigned long long v)
{
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(a), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long clu_ld64(uint32_t a)
{
    unsigned long long v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return v;
}

// Every thread of every CTA of the cluster; stores before it (local or into
// other CTAs) are visible to all of them after it.
__device__ __forceinline__ void clu_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The same barrier for a warp whose stores nobody reads across it: it
// arrives without release ordering (no fence), and still waits with acquire.
__device__ __forceinline__ void clu_sync_relaxed()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long s)
{
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// max |eigenvalue| of A' (rows of this CTA in A, row stride kCN) by symmetric
// Lanczos without reorthogonalization from a fixed zero-mean pseudo-random
// start: w' = A' q - beta q_prev, alpha = w' . q, w = w' - alpha q,
// beta = |w|, q = w / beta; every 8 steps (after 16) the tridiagonal
// matrix's extreme eigenvalues are bracketed, each check after the first
// starting from the last one's brackets, and the iteration stops once
// max |eigenvalue| moved by less than 4e-7 of itself.
// Warp v of the CTA owns rows 2 v and 2 v + 1 of the CTA's 32, held in
// registers (lane l: columns l + 32 u); q and the previous q alternate
// between two shared buffers by step parity.  A step: every warp multiplies
// its rows by q, forms its two entries of w' and writes them into every
// CTA; one cluster barrier; warp 0 of every CTA reads all of w' and forms
// alpha, beta and the next q from the same numbers in the same order, so all
// CTAs hold the same vector and tridiagonal matrix and take the same
// decisions; one CTA barrier.  A CTA a step ahead cannot overwrite a w'
// buffer another still reads: w' alternates by step parity too, and every
// CTA reads its buffer before it arrives at the next cluster barrier.
__device__ float clu_lanczos(CluSmem& sm, const float* A, int N, uint32_t r)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int j = lane >> 4;                       // this lane's row of the warp's two ...
    const int gi = (int)r * kCR + 2 * warp + j;    // ... as an index of A'
    float a0[kCN / 32], a1[kCN / 32];
#pragma unroll
    for (int u = 0; u < kCN / 32; ++u) {
        a0[u] = A[(2 * warp) * kCN + lane + 32 * u];
        a1[u] = A[(2 * warp + 1) * kCN + lane + 32 * u];
    }
    // Warp 0 keeps q in registers too (lane l: entries l + 32 u).
    float q[kCN / 32];
    if (warp == 0) {
        float ss = 0.f;
#pragma unroll
        for (int u = 0; u < kCN / 32; ++u) {
            // A near-constant start would be almost orthogonal to the top
            // eigenvectors of a deflated A' and could stall on a lower one.
            const int c = lane + 32 * u;
            const unsigned hs = (unsigned)c * 2654435761u + 12345u;
            q[u] = c < N ? (float)hs * 2.3283064e-10f - 0.5f : 0.f;
            ss = fmaf(q[u], q[u], ss);
        }
        const float inv = rsqrtf(warp_sum(ss));
#pragma unroll
        for (int u = 0; u < kCN / 32; ++u) {
            q[u] *= inv;
            sm.qv[0][lane + 32 * u] = q[u];
            sm.qv[1][lane + 32 * u] = 0.f;
        }
        if (lane == 0) {
            sm.te.absmax = -1.f;
            sm.stop = 0;
        }
    }
    __syncthreads();
    float beta = 0.f;
    int L = 0, checked = 0;
    for (int k = 0; k < kMaxSymSteps; ++k) {
        const int par = k & 1;
        float y0 = 0.f, y1 = 0.f;
#pragma unroll
        for (int u = 0; u < kCN / 32; ++u) {
            const float qc = sm.qv[par][lane + 32 * u];
            y0 = fmaf(a0[u], qc, y0);
            y1 = fmaf(a1[u], qc, y1);
        }
        // Lanes 0-15 sum row 2 v, lanes 16-31 row 2 v + 1.
        float y = (j ? y1 : y0) + __shfl_xor_sync(0xffffffffu, j ? y0 : y1, 16);
        for (int o = 8; o > 0; o >>= 1)
            y += __shfl_xor_sync(0xffffffffu, y, o);
        const float wv = fmaf(-beta, sm.qv[par ^ 1][gi], y);
        if ((lane & 15) == 0)
            sm.stg[2 * warp + j] = wv;
        __syncthreads();
        if (warp == 0) {
            // Lane l: entries [8 (l / 8), 8 (l / 8) + 8) of this CTA's 32, into CTA l % 8.
            const int c = lane & 7, e = 8 * (lane >> 3);
            const uint32_t dst = clu_addr(&sm.w[par][(int)r * kCR + e], (uint32_t)c);
            clu_st4(dst, *reinterpret_cast<const float4*>(&sm.stg[e]));
            clu_st4(dst + 16u, *reinterpret_cast<const float4*>(&sm.stg[e + 4]));
            clu_sync();
        } else {
            clu_sync_relaxed();  // these warps wrote nothing another CTA reads
        }
        if (warp == 0) {
            float wc[kCN / 32], d = 0.f;
#pragma unroll
            for (int u = 0; u < kCN / 32; ++u) {
                wc[u] = sm.w[par][lane + 32 * u];
                d = fmaf(wc[u], q[u], d);
            }
            const float alpha = warp_sum(d);
            float s2 = 0.f;
#pragma unroll
            for (int u = 0; u < kCN / 32; ++u) {
                wc[u] = fmaf(-alpha, q[u], wc[u]);
                s2 = fmaf(wc[u], wc[u], s2);
            }
            const float bn = sqrtf(warp_sum(s2));
            if (lane == 0) {
                sm.al[k] = alpha;
                sm.be[k] = bn;
            }
            if (bn > 1e-30f) {
                const float ib = 1.f / bn;
#pragma unroll
                for (int u = 0; u < kCN / 32; ++u) {
                    q[u] = wc[u] * ib;
                    sm.qv[par ^ 1][lane + 32 * u] = q[u];
                }
            }
        }
        __syncthreads();
        const float bn = sm.be[k];
        L = k + 1;
        if (!(bn > 1e-30f))
            break;  // invariant subspace: the tridiagonal matrix is exact
        beta = bn;
        if ((L & 7) == 0 && L >= 16) {
            const float prev = sm.te.absmax;
            tri_ends_block(sm.al, sm.be, L, checked > 0, sm.te, sm.msk);
            checked = L;
            if (tid == 0)
                sm.stop = fabsf(sm.te.absmax - prev) <= 4e-7f * sm.te.absmax ? 1 : 0;
            __syncthreads();
            if (sm.stop)
                break;
        }
    }
    __syncthreads();
    if (checked != L)
        tri_ends_block(sm.al, sm.be, L, false, sm.te, sm.msk);
    return sm.te.absmax;
}

__global__ void __cluster_dims__(kClu, 1, 1) __launch_bounds__(kCluThreads, 1)
    k_haralick_cluster(FeatParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CluSmem& sm = *reinterpret_cast<CluSmem*>(smem_raw);
    const uint32_t r = clu_rank();
    const FeatJob J = p.jobs[clu_id()];
    const int N = J.levels;
    const uint32_t* P = J.counts;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = (int)r * kCR;

    // Stage P's rows [i0, i0 + 32) and columns [i0, i0 + 32), zero outside N.
    {
        uint32_t v[kCR * kCN / kCluThreads];
#pragma unroll
        for (int u = 0; u < kCR * kCN / kCluThreads; ++u) {
            const int e = tid + u * kCluThreads, i = i0 + (e >> 8), j = e & 255;
            v[u] = (i < N && j < N) ? __ldg(P + i * N + j) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kCR * kCN / kCluThreads; ++u)
            sm.pb[tid + u * kCluThreads] = v[u];
#pragma unroll
        for (int u = 0; u < kCR * kCN / kCluThreads; ++u) {
            const int e = tid + u * kCluThreads, j = e >> 5, i = i0 + (e & 31);
            v[u] = (i < N && j < N) ? __ldg(P + j * N + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kCR * kCN / kCluThreads; ++u) {
            const int e = tid + u * kCluThreads;
            sm.pt[(e >> 5) * (kCR + 1) + (e & 31)] = v[u];
        }
    }
    if (tid == 0)
        sm.cij = 0ull;
    __syncthreads();
    // Partial marginals of P over this CTA's rows (level i = i0 + rr): row
    // sums by warps; column, i + j and |i - j| sums one index per thread
    // (consecutive indices read consecutive words: no bank conflict).
    for (int rr = warp; rr < kCR; rr += kCluWarps) {
        unsigned long long s = 0;
#pragma unroll
        for (int u = 0; u < kCN / 32; ++u)
            s += sm.pb[rr * kCN + lane + 32 * u];
        s = warp_sum_u64(s);
        if (lane == 0)
            sm.part[kPartRS + rr] = s;
    }
    if (tid < kCN) {
        const int x = tid;
        unsigned long long cs = 0, ds = 0;
        for (int rr = 0; rr < kCR; ++rr) {
            const int i = i0 + rr;
            cs += sm.pb[rr * kCN + x];
            if (i + x < kCN)
                ds += sm.pb[rr * kCN + i + x];
            if (x > 0 && i - x >= 0)
                ds += sm.pb[rr * kCN + i - x];
        }
        sm.part[kPartCS + x] = cs;
        sm.part[kPartDS + x] = ds;
    }
    for (int x = tid; x < 2 * kCN; x += kCluThreads) {
        unsigned long long s = 0;
        for (int rr = 0; rr < kCR; ++rr) {
            const int j = x - (i0 + rr);
            if (j >= 0 && j < kCN)
                s += sm.pb[rr * kCN + j];
        }
        sm.part[kPartSS + x] = s;
    }
    clu_sync();
    // Marginals of S = P + P^T from every CTA's partial sums: row (= column)
    // sums are P's row plus column sums, the i + j and |i - j| sums twice P's.
    for (int x = tid; x < 4 * kCN; x += kCluThreads) {
        unsigned long long s = 0;
        for (int c = 0; c < kClu; ++c)
            s += clu_ld64(clu_addr(&sm.part[x], (uint32_t)c));
        if (x < kPartSS) {
            s += clu_ld64(clu_addr(&sm.part[kPartRS + (x & (kCR - 1))], (uint32_t)(x / kCR)));
            sm.rs[x] = s;
        } else if (x < kPartDS) {
            sm.ss[x - kPartSS] = 2ull * s;
        } else {
            sm.ds[x - kPartDS] = 2ull * s;
        }
    }
    clu_sync();  // no CTA reads another's partial sums after this
    // Totals and exact moments (warp 0 of every CTA, the same values).
    if (warp == 0) {
        unsigned long long T = 0, m_i = 0, c2 = 0, m_s = 0, m_d = 0, q_i = 0;
        int nr = 0;
        for (int k0 = 0; k0 < 2 * kCN; k0 += 32) {
            const int k = k0 + lane;
            const bool in = k < kCN;
            const unsigned long long rv = in ? sm.rs[k] : 0ull, d = in ? sm.ds[k] : 0ull, sv = sm.ss[k];
            T += rv;
            m_i += (unsigned long long)k * rv;
            q_i += (unsigned long long)k * k * rv;
            c2 += (unsigned long long)k * k * d;
            m_d += (unsigned long long)k * d;
            m_s += (unsigned long long)k * sv;
            nr += __popc(__ballot_sync(0xffffffffu, rv != 0ull));
        }
        T = warp_sum_u64(T);
        m_i = warp_sum_u64(m_i);
        q_i = warp_sum_u64(q_i);
        c2 = warp_sum_u64(c2);
        m_d = warp_sum_u64(m_d);
        m_s = warp_sum_u64(m_s);
        if (lane == 0) {
            sm.T = T;
            sm.mom[0] = m_i;
            sm.mom[1] = m_i;
            sm.mom[2] = c2;
            sm.mom[3] = m_s;
            sm.mom[4] = m_d;
            sm.mom[5] = q_i;
            sm.mom[6] = q_i;
            sm.nr = nr;
        }
    }
    __syncthreads();
    const unsigned long long T = sm.T;
    if (T == 0ull) {
        for (int e = tid; e < kCR * kCN && J.normalized; e += kCluThreads) {
            const int i = i0 + (e >> 8), j = e & 255;
            if (i < N && j < N)
                J.normalized[(size_t)i * N + j] = 0.f;
        }
        if (r == 0 && tid < kNumFeat)
            J.features[tid] = 0.f;
        return;  // every CTA of the cluster returns here
    }
    const float Tf = (float)T;
    // Cell pass over this CTA's rows: warp w rows w and w + 16, lane l
    // columns l + 32 u.  A' overwrites the staged row of P cell by cell.
    float* A = reinterpret_cast<float*>(sm.pb);
    Kahan k_asm, k_ent, k_mi;
    unsigned long long cij = 0;
    for (int rr = warp; rr < kCR; rr += kCluWarps) {
        const int i = i0 + rr;
#pragma unroll 2
        for (int u = 0; u < kCN / 32; ++u) {
            const int j = lane + 32 * u;
            float a = 0.f;
            if (i < N && j < N) {
                const unsigned long long sv =
                    (unsigned long long)sm.pb[rr * kCN + j] + sm.pt[j * (kCR + 1) + rr];
                const float pv = __fdiv_rn((float)sv, Tf);
                if (J.normalized)
                    J.normalized[(size_t)i * N + j] = pv;
                if (sv) {
                    k_asm.add(__fmul_rn(pv, pv));
                    k_ent.add(neg_plogp(pv));
                    cij += (unsigned long long)(i * j) * sv;
                }
                const unsigned long long ri = sm.rs[i], cj = sm.rs[j];
                if (ri && cj) {
                    // Exact numerator S*T - r*c while T < 2^31 (products < 2^62).
                    const float rc = __fmul_rn((float)ri, (float)cj);
                    float numf;
                    if (T < (1ull << 31))
                        numf = (float)((long long)(sv * T) - (long long)(ri * cj));
                    else
                        numf = __fsub_rn(__fmul_rn((float)sv, Tf), rc);
                    const float x = __fdiv_rn(numf, rc);
                    const float q = __fmul_rn(__fdiv_rn((float)ri, Tf), __fdiv_rn((float)cj, Tf));
                    k_mi.add(__fmul_rn(q, phi(x)));
                    a = __fdiv_rn(numf, __fmul_rn(Tf, sqrtf(rc)));
                }
            }
            A[rr * kCN + j] = a;
        }
    }
    // Terms of the marginal distributions, indices [64 r, 64 r + 64).
    Kahan k_idm, k_svar, k_sent, k_dvar, k_dent, k_hx, k_hy;
    const float f6 = ratio_u64(sm.mom[3], T);
    const float mean_d = ratio_u64(sm.mom[4], T);
    for (int k = (int)r * 64 + tid; tid < 64 && k < 2 * N - 1; k += kCluThreads) {
        const float ps = __fdiv_rn((float)sm.ss[k], Tf);
        const float dk = __fsub_rn((float)k, f6);
        k_svar.add(__fmul_rn(__fmul_rn(dk, dk), ps));
        k_sent.add(neg_plogp(ps));
        if (k < N) {
            const float pd = __fdiv_rn((float)sm.ds[k], Tf);
            k_idm.add(__fdiv_rn(pd, (float)(1 + k * k)));
            const float dd2 = __fsub_rn((float)k, mean_d);
            k_dvar.add(__fmul_rn(__fmul_rn(dd2, dd2), pd));
            k_dent.add(neg_plogp(pd));
            const float pr = neg_plogp(__fdiv_rn((float)sm.rs[k], Tf));
            k_hx.add(pr);
            k_hy.add(pr);
        }
    }
    cij = warp_sum_u64(cij);
    if (lane == 0 && cij)
        atomicAdd(&sm.cij, cij);  // complete after the block reduction's barriers
    DF v[10] = {k_asm.df(), k_ent.df(), k_mi.df(), k_idm.df(), k_svar.df(),
                k_sent.df(), k_dvar.df(), k_dent.df(), k_hx.df(), k_hy.df()};
    block_reduce_df<10>(v, sm.dscr);
    // This CTA's sums into CTA 0 (read there after the last cluster barrier).
    if (tid < 10) {
        const uint32_t a = clu_addr(&sm.fin[r][tid], 0u);
        clu_st(a, v[tid].hi);
        clu_st(a + 4u, v[tid].lo);
    } else if (tid == 10) {
        clu_st64(clu_addr(&sm.fin_cij[r], 0u), sm.cij);
    }
    __syncthreads();
    float mcc = 0.f;
    if (sm.nr >= 2)
        mcc = clu_lanczos(sm, A, N, r);
    clu_sync();  // the last access to another CTA's shared memory precedes this
    if (r != 0)
        return;
    if (tid == 0) {
        DF tot[10];
        unsigned long long cij_t = 0;
        for (int k = 0; k < 10; ++k)
            tot[k] = sm.fin[0][k];
        cij_t = sm.fin_cij[0];
        for (int c = 1; c < kClu; ++c) {
            for (int k = 0; k < 10; ++k)
                tot[k] = df_add(tot[k], sm.fin[c][k]);
            cij_t += sm.fin_cij[c];
        }
        write_features(J.features, T, sm.mom, cij_t, tot, f6, mcc);
    }
}
}  // namespace

// Global scratch per GLCM for supports too large for shared memory: A' (N^2)
// followed by the Lanczos vectors.
long long features_work_floats(int levels)
{
    const int K = levels < kMaxLanczos ? levels : kMaxLanczos;
    return (long long)levels * levels + (2ll * K + 1) * levels + 64;
}

size_t features_smem_bytes(int max_levels)
{
    return feat_layout(max_levels).total;
}

// A launch at scheduling priority `priority` (0: the stream's own; lower
// numbers are more urgent): the attribute stays with the kernel node when
// the launch is captured into a graph.
template <class... Params, class... Args>
cudaError_t launch_prio(void (*kernel)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, int priority,
                        Args... args)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = priority;
    cfg.attrs = attr;
    cfg.numAttrs = priority != 0 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Symmetric feature jobs with 128 < N <= 256: one cluster of kClu CTAs each.
cudaError_t launch_features_cluster(const FeatParams& p, cudaStream_t s, int priority)
{
    if (p.n_jobs <= 0)
        return cudaSuccess;
    static SmemLimit lim;
    const cudaError_t e = lim.raise((const void*)k_haralick_cluster, sizeof(CluSmem));
    if (e != cudaSuccess)
        return e;
    return launch_prio(k_haralick_cluster, dim3(p.n_jobs * kClu), dim3(kCluThreads), sizeof(CluSmem), s, priority, p);
}

// threads: kFeatThreads, or kFeatThreadsSmall for jobs with N <= 32 (their
// epilogue is short and barrier-bound: two such CTAs share an SM).  The
// block size depends on a job's N only, so its features do not depend on
// the batch it is in.
cudaError_t launch_features(const FeatParams& p, int max_levels, cudaStream_t s, int threads, int priority)
{
    if (p.n_jobs <= 0)
        return cudaSuccess;
    if (threads != kFeatThreads && (threads != kFeatThreadsSmall || max_levels > kSmallFeatLevels))
        return cudaErrorInvalidValue;
    const size_t smem = features_smem_bytes(max_levels);
    if (threads == kFeatThreadsSmall) {
        static SmemLimit lim_small;
        const cudaError_t e = lim_small.raise((const void*)k_haralick<kFeatThreadsSmall, kFeatSmallPerSM>, smem);
        if (e != cudaSuccess)
            return e;
        return launch_prio(k_haralick<kFeatThreadsSmall, kFeatSmallPerSM>, dim3(p.n_jobs), dim3(threads), smem, s,
                           priority, p, max_levels);
    }
    static SmemLimit lim;
    const cudaError_t e = lim.raise((const void*)k_haralick<kFeatThreads, 1>, smem);
    if (e != cudaSuccess)
        return e;
    return launch_prio(k_haralick<kFeatThreads, 1>, dim3(p.n_jobs), dim3(threads), smem, s, priority, p, max_levels);
}

}  // namespace glcm
