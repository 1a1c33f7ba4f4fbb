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
//  * The means, variances and covariance behind correlation (f3) and sum of
//    squares (f4) are float64 -- the one float64 step.
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
//    of A' is found with one-sided (Hestenes) Jacobi rotations in float32.
#include <cmath>

#include "glcm_internal.cuh"

namespace glcm {
namespace {

constexpr int kFeatThreads = 512;
constexpr int kNumFeat = 14;
constexpr int kSmemA = 64;  // support up to 64x64 keeps A' in shared memory

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

template <int K>
__device__ void block_reduce_d(double (&v)[K], double* scratch)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        for (int o = 16; o > 0; o >>= 1)
            v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
        if (lane == 0)
            scratch[k * 32 + warp] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double a = lane < nw ? scratch[k * 32 + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1)
                a += __shfl_down_sync(0xffffffffu, a, o);
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

__device__ __forceinline__ unsigned long long cell(const uint32_t* C, int N, int i, int j, int sym)
{
    unsigned long long s = C[i * N + j];
    if (sym)
        s += C[j * N + i];
    return s;
}

__device__ __forceinline__ float neg_plogp(float p)
{
    return p > 0.f ? -__fmul_rn(p, logf(p)) : 0.f;
}

// Largest singular value of the m x n matrix A (column-major, leading dim m)
// by one-sided Jacobi: rotate column pairs until all are orthogonal, then
// the column norms are the singular values.
__device__ float jacobi_sigma_max(float* A, int m, int n, int* s_flag, float* s_red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (n <= 0 || m <= 0)
        return 0.f;
    const int np = (n + 1) & ~1;  // even number of players (one dummy if odd)
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (threadIdx.x == 0)
            *s_flag = 0;
        __syncthreads();
        for (int step = 0; step < np - 1; ++step) {
            for (int k = warp; k < np / 2; k += nw) {
                int a, b;
                if (k == 0) {
                    a = 0;
                    b = (step % (np - 1)) + 1;
                } else {
                    a = ((step + k) % (np - 1)) + 1;
                    b = ((step + np - 1 - k) % (np - 1)) + 1;
                }
                if (a >= n || b >= n)
                    continue;
                float* ca = A + (long long)a * m;
                float* cb = A + (long long)b * m;
                float al = 0.f, be = 0.f, ga = 0.f;
                for (int r = lane; r < m; r += 32) {
                    const float x = ca[r], y = cb[r];
                    al = fmaf(x, x, al);
                    be = fmaf(y, y, be);
                    ga = fmaf(x, y, ga);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                if (fabsf(ga) > 4e-7f * sqrtf(al * be) && fabsf(ga) > 1e-30f) {
                    const float zeta = (be - al) / (2.f * ga);
                    const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    const float cs = rsqrtf(1.f + t * t);
                    const float sn = cs * t;
                    for (int r = lane; r < m; r += 32) {
                        const float x = ca[r], y = cb[r];
                        ca[r] = cs * x - sn * y;
                        cb[r] = sn * x + cs * y;
                    }
                    if (lane == 0)
                        *s_flag = 1;
                }
            }
            __syncthreads();
        }
        const int rotated = *s_flag;
        __syncthreads();
        if (!rotated)
            break;
    }
    // Column norms, maximum.
    float best = 0.f;
    for (int k = warp; k < n; k += nw) {
        const float* ck = A + (long long)k * m;
        float s = 0.f;
        for (int r = lane; r < m; r += 32)
            s = fmaf(ck[r], ck[r], s);
        for (int o = 16; o > 0; o >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, o);
        best = fmaxf(best, s);
    }
    if (lane == 0)
        s_red[warp] = best;
    __syncthreads();
    float m2 = 0.f;
    for (int w = 0; w < nw; ++w)
        m2 = fmaxf(m2, s_red[w]);
    __syncthreads();
    return sqrtf(m2);
}

// Largest singular value of the m x n matrix A (column-major, leading dim m,
// in global scratch) by Golub-Kahan-Lanczos bidiagonalization with full
// reorthogonalization, then bisection (Sturm counts) on the 2K x 2K
// zero-diagonal tridiagonal matrix whose eigenvalues are +-sigma(B_K).
// U (kMaxLanczos x m) and V ((kMaxLanczos + 1) x n) live after A.
constexpr int kMaxLanczos = 96;

__device__ float block_dot(const float* x, const float* y, int len, float* s_red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float s = 0.f;
    for (int r = threadIdx.x; r < len; r += blockDim.x)
        s = fmaf(x[r], y[r], s);
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0)
        s_red[warp] = s;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < nw; ++w)
        t += s_red[w];
    __syncthreads();
    return t;
}

// x -= sum_i <x, Q_i> Q_i over the first k rows of Q (twice, classical GS).
__device__ void reorth(float* x, const float* Q, int k, int len, float* s_coef, float* s_red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int pass = 0; pass < 2; ++pass) {
        for (int i = warp; i < k; i += nw) {
            const float* q = Q + (long long)i * len;
            float s = 0.f;
            for (int r = lane; r < len; r += 32)
                s = fmaf(x[r], q[r], s);
            for (int o = 16; o > 0; o >>= 1)
                s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0)
                s_coef[i] = s;
        }
        __syncthreads();
        for (int r = threadIdx.x; r < len; r += blockDim.x) {
            float v = x[r];
            for (int i = 0; i < k; ++i)
                v = fmaf(-s_coef[i], Q[(long long)i * len + r], v);
            x[r] = v;
        }
        __syncthreads();
    }
    (void)s_red;
}

// Largest singular value of the K x K upper bidiagonal matrix with
// diagonal alpha_k = ab[2k] and superdiagonal beta_k = ab[2k+1]: bisection
// with Sturm counts on the zero-diagonal tridiagonal matrix whose
// off-diagonals are alpha_0, beta_0, alpha_1, ... (eigenvalues +-sigma).
__device__ float gk_sigma_max(const float* ab, int steps)
{
    const int L = 2 * steps - 1;
    if (L <= 0)
        return 0.f;
    float hi = 0.f;
    for (int t = 0; t < L; ++t)
        hi = fmaxf(hi, ab[t]);
    hi *= 2.f;
    float lo = 0.f;
    for (int it = 0; it < 60; ++it) {
        const float x = 0.5f * (lo + hi);
        int cnt = 0;
        float q = -x;
        if (q < 0.f)
            ++cnt;
        for (int t = 0; t < L; ++t) {
            const float b = ab[t];
            if (q == 0.f)
                q = -1e-30f;
            q = -x - b * b / q;
            if (q < 0.f)
                ++cnt;
        }
        if (cnt >= L + 1)
            hi = x;  // all eigenvalues below x
        else
            lo = x;
    }
    return 0.5f * (lo + hi);
}

__device__ float lanczos_sigma_max(const float* A, int m, int n, float* U, float* V, float* s_coef, float* s_red,
                                   float* s_ab, float* s_sig, int* s_stop)
{
    const int K = min(kMaxLanczos, min(m, n));
    float* v0 = V;
    for (int c = threadIdx.x; c < n; c += blockDim.x)
        v0[c] = 1.f + 0.01f * (float)((c * 37) % 11);  // fixed, not orthogonal to anything special
    __syncthreads();
    float nv = sqrtf(block_dot(v0, v0, n, s_red));
    for (int c = threadIdx.x; c < n; c += blockDim.x)
        v0[c] /= nv;
    __syncthreads();
    int steps = 0;
    float beta = 0.f;
    for (int k = 0; k < K; ++k) {
        float* uk = U + (long long)k * m;
        const float* vk = V + (long long)k * n;
        // u = A v_k - beta_k u_{k-1}
        for (int r = threadIdx.x; r < m; r += blockDim.x) {
            float s = 0.f;
            for (int c = 0; c < n; ++c)
                s = fmaf(A[(long long)c * m + r], vk[c], s);
            if (k > 0)
                s = fmaf(-beta, U[(long long)(k - 1) * m + r], s);
            uk[r] = s;
        }
        __syncthreads();
        reorth(uk, U, k, m, s_coef, s_red);
        const float alpha = sqrtf(block_dot(uk, uk, m, s_red));
        if (threadIdx.x == 0)
            s_ab[2 * k] = alpha;
        if (!(alpha > 1e-30f))
            break;
        for (int r = threadIdx.x; r < m; r += blockDim.x)
            uk[r] /= alpha;
        __syncthreads();
        steps = k + 1;
        // v = A^T u_k - alpha_k v_k
        float* vn = V + (long long)(k + 1) * n;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int c = warp; c < n; c += nw) {
            const float* col = A + (long long)c * m;
            float s = 0.f;
            for (int r = lane; r < m; r += 32)
                s = fmaf(col[r], uk[r], s);
            for (int o = 16; o > 0; o >>= 1)
                s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0)
                vn[c] = s - alpha * vk[c];
        }
        __syncthreads();
        reorth(vn, V, k + 1, n, s_coef, s_red);
        beta = sqrtf(block_dot(vn, vn, n, s_red));
        if (threadIdx.x == 0)
            s_ab[2 * k + 1] = beta;
        if (!(beta > 1e-30f) || k + 1 == K)
            break;
        // Every 8 steps: stop once the top Ritz value moved by < 1e-7.
        if (((k + 1) & 7) == 0) {
            if (threadIdx.x == 0) {
                const float sg = gk_sigma_max(s_ab, k + 1);
                *s_stop = (k + 1 >= 16 && fabsf(sg - *s_sig) <= 1e-7f) ? 1 : 0;
                *s_sig = sg;
            }
            __syncthreads();
            if (*s_stop)
                break;
        }
        for (int c = threadIdx.x; c < n; c += blockDim.x)
            vn[c] /= beta;
        __syncthreads();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        *s_sig = gk_sigma_max(s_ab, steps);
    __syncthreads();
    return *s_sig;
}

__global__ void __launch_bounds__(kFeatThreads) k_haralick(FeatParams p)
{
    const FeatJob J = p.jobs[blockIdx.x];
    const int N = J.levels;
    const int NN = N * N;
    const int sym = J.symmetric;
    const uint32_t* C = J.counts;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* rs = reinterpret_cast<unsigned long long*>(smem_raw);  // N
    unsigned long long* cs = rs + N;                                           // N
    unsigned long long* ss = cs + N;                                           // 2N
    unsigned long long* ds = ss + 2 * N;                                       // N
    int* rmap = reinterpret_cast<int*>(ds + N);                                // N (row -> support idx)
    int* cmap = rmap + N;                                                      // N
    DF* dscr = reinterpret_cast<DF*>(cmap + N);                                // 10 * 32
    double* dd = reinterpret_cast<double*>(dscr + 10 * 32);                     // 6 * 32
    float* fa = reinterpret_cast<float*>(dd + 6 * 32);                         // kSmemA^2
    __shared__ unsigned long long s_T, s_m[6];
    __shared__ int s_nr, s_nc, s_flag;
    __shared__ float s_red[32];

    for (int k = threadIdx.x; k < 5 * N; k += blockDim.x)
        rs[k] = 0ull;
    __syncthreads();
    for (int t = threadIdx.x; t < NN; t += blockDim.x) {
        const int i = t / N, j = t - (t / N) * N;
        const unsigned long long s = cell(C, N, i, j, sym);
        if (s) {
            atomicAdd(&rs[i], s);
            atomicAdd(&cs[j], s);
            atomicAdd(&ss[i + j], s);
            atomicAdd(&ds[i > j ? i - j : j - i], s);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long T = 0, m_i = 0, m_j = 0, c2 = 0, m_s = 0, m_d = 0;
        int nr = 0, nc = 0;
        for (int k = 0; k < N; ++k) {
            T += rs[k];
            m_i += (unsigned long long)k * rs[k];
            m_j += (unsigned long long)k * cs[k];
            c2 += (unsigned long long)k * k * ds[k];
            m_d += (unsigned long long)k * ds[k];
            rmap[k] = rs[k] ? nr++ : -1;
            cmap[k] = cs[k] ? nc++ : -1;
        }
        for (int k = 0; k < 2 * N - 1; ++k)
            m_s += (unsigned long long)k * ss[k];
        s_T = T;
        s_m[0] = m_i; s_m[1] = m_j; s_m[2] = c2; s_m[3] = m_s; s_m[4] = m_d;
        s_nr = nr;
        s_nc = nc;
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
    const double Td = (double)T;
    const double mux = (double)s_m[0] / Td, muy = (double)s_m[1] / Td;
    const int nr = s_nr, nc = s_nc;
    // A' storage: shared memory when the support is small, else global scratch.
    float* A = (nr <= kSmemA && nc <= kSmemA) ? fa : (p.work + (long long)blockIdx.x * p.work_stride);
    const bool have_work = (nr <= kSmemA && nc <= kSmemA) || p.work != nullptr;

    // Cell pass: normalized output, f1, f9, MI terms, covariance, A'.
    Kahan k_asm, k_ent, k_mi;
    double cov = 0.0;
    for (int t = threadIdx.x; t < NN; t += blockDim.x) {
        const int i = t / N, j = t - (t / N) * N;
        const unsigned long long s = cell(C, N, i, j, sym);
        const float pv = __fdiv_rn((float)s, Tf);
        if (J.normalized)
            J.normalized[t] = pv;
        if (s) {
            k_asm.add(__fmul_rn(pv, pv));
            k_ent.add(neg_plogp(pv));
            cov += ((double)i - mux) * ((double)j - muy) * (double)s;
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
    double vx = 0.0, vy = 0.0;
    const float f6 = __fdiv_rn((float)s_m[3], Tf);
    const float mean_d = __fdiv_rn((float)s_m[4], Tf);
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
            vx += ((double)k - mux) * ((double)k - mux) * (double)rs[k];
            vy += ((double)k - muy) * ((double)k - muy) * (double)cs[k];
        }
    }
    DF v[10] = {k_asm.df(), k_ent.df(), k_mi.df(), k_idm.df(), k_svar.df(),
                k_sent.df(), k_dvar.df(), k_dent.df(), k_hx.df(), k_hy.df()};
    block_reduce_df<10>(v, dscr);
    double dv[3] = {cov, vx, vy};
    block_reduce_d<3>(dv, dd);

    float mcc = 0.f;
    if (nr >= 2 && have_work) {
        if (nr <= kSmemA && nc <= kSmemA) {
            mcc = jacobi_sigma_max(A, nr, nc, &s_flag, s_red);
        } else {
            float* Uw = A + (long long)nr * nc;
            float* Vw = Uw + (long long)kMaxLanczos * nr;
            __shared__ float s_coef[kMaxLanczos + 1];
            __shared__ float s_ab[2 * kMaxLanczos + 2];
            __shared__ float s_sg;
            __shared__ int s_stop;
            if (threadIdx.x == 0) {
                s_sg = -1.f;
                s_stop = 0;
            }
            __syncthreads();
            mcc = lanczos_sigma_max(A, nr, nc, Uw, Vw, s_coef, s_red, s_ab, &s_sg, &s_stop);
        }
    }
    if (!have_work && threadIdx.x == 0)
        atomicOr(p.err, kErrInternal);

    if (threadIdx.x == 0 && feat) {
        const double varx = dv[1] / Td, vary = dv[2] / Td;
        const double sdx = sqrt(varx), sdy = sqrt(vary);
        const float mi = fmaxf(0.f, v[2].hi + v[2].lo);
        const float hx = v[8].hi + v[8].lo, hy = v[9].hi + v[9].lo;
        const float hmax = fmaxf(hx, hy);
        feat[0] = v[0].hi + v[0].lo;
        feat[1] = (float)s_m[2] / Tf;
        feat[2] = (sdx * sdy > 0.0) ? (float)((dv[0] / Td) / (sdx * sdy)) : 1.f;
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
}

}  // namespace

long long features_work_floats(int levels)
{
    return (long long)levels * levels + (long long)(2 * kMaxLanczos + 2) * levels + 64;
}

size_t features_smem_bytes(int max_levels)
{
    const int N = max_levels;
    return (size_t)5 * N * 8 + (size_t)2 * N * 4 + 10 * 32 * sizeof(DF) + 6 * 32 * 8 +
           (size_t)kSmemA * kSmemA * 4 + 64;
}

cudaError_t launch_features(const FeatParams& p, int max_levels, cudaStream_t s)
{
    if (p.n_jobs <= 0)
        return cudaSuccess;
    const size_t smem = features_smem_bytes(max_levels);
    static size_t set_to = 0;
    if (smem > set_to) {
        cudaError_t e = cudaFuncSetAttribute(k_haralick, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        set_to = smem;
    }
    k_haralick<<<p.n_jobs, kFeatThreads, smem, s>>>(p);
    return cudaGetLastError();
}

}  // namespace glcm
