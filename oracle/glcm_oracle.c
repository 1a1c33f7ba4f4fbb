/*
 * Plain CPU oracle for the gray-level co-occurrence matrix (GLCM).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the CUDA library must compute.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA path, and the CUDA path never
 * calls it.
 *
 * Definition followed (Sec. I.A, Eq. 1; partner from Eq. 2; one vote per
 * pair as in the voting step after Eq. 3):
 *
 *   for every anchor pixel (x, y) whose partner (x + dx, y + dy) lies inside
 *   the W x H image (no wrap from one row into the next), with
 *   i = level(x, y) and j = level(x + dx, y + dy):   P[i * N + j] += 1
 *
 * Row index y grows downwards, so the paper's 0/45/90/135 degree directions
 * at distance d are (d,0), (d,-d), (0,-d), (-d,-d).
 *
 * Levels: with `levels_mode` = 0 a pixel v of b bits maps to
 * floor(v * N / 2^b) (the paper reduces gray levels to 8, 16 or 32 without
 * giving the mapping, Sec. I.A); with `levels_mode` = 1 the pixel already is
 * a level and must be < N.  A pair that touches a pixel >= N in that mode is
 * not counted and is reported in the return value.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

static unsigned read_pixel(const unsigned char *img, size_t pitch, int bpp, int x, int y)
{
    const unsigned char *row = img + (size_t)y * pitch;
    if (bpp == 1)
        return row[x];
    uint16_t v;
    memcpy(&v, row + 2 * (size_t)x, 2);
    return v;
}

static unsigned level_of(unsigned v, int bpp, int n_levels, int levels_mode)
{
    if (levels_mode)
        return v;
    return (unsigned)(((uint64_t)v * (uint64_t)n_levels) >> (8 * bpp));
}

/* GLCM of one offset over the whole image.  P has N*N entries, row-major
 * [i][j], i = anchor level.  Returns the number of pairs skipped because a
 * pixel was out of range in levels mode (0 otherwise), or -1 on bad args. */
long long oracle_glcm(const void *image, int W, int H, size_t pitch, int bpp,
                      int n_levels, int levels_mode, int dx, int dy, uint32_t *P)
{
    if (!image || !P || W < 0 || H < 0 || (bpp != 1 && bpp != 2) || n_levels < 1)
        return -1;
    const unsigned char *img = (const unsigned char *)image;
    long long skipped = 0;
    memset(P, 0, sizeof(uint32_t) * (size_t)n_levels * (size_t)n_levels);
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int x2 = x + dx, y2 = y + dy;
            if (x2 < 0 || x2 >= W || y2 < 0 || y2 >= H)
                continue;
            unsigned i = level_of(read_pixel(img, pitch, bpp, x, y), bpp, n_levels, levels_mode);
            unsigned j = level_of(read_pixel(img, pitch, bpp, x2, y2), bpp, n_levels, levels_mode);
            if (i >= (unsigned)n_levels || j >= (unsigned)n_levels) {
                ++skipped;
                continue;
            }
            P[(size_t)i * n_levels + j] += 1u;
        }
    }
    return skipped;
}

/* GLCMs of several offsets: P has n_off blocks of N*N.  dxy holds
 * dx0, dy0, dx1, dy1, ...  Returns the total skipped count or -1. */
long long oracle_glcm_multi(const void *image, int W, int H, size_t pitch, int bpp,
                            int n_levels, int levels_mode, int n_off, const int *dxy,
                            uint32_t *P)
{
    long long total = 0;
    for (int o = 0; o < n_off; ++o) {
        long long s = oracle_glcm(image, W, H, pitch, bpp, n_levels, levels_mode,
                                  dxy[2 * o], dxy[2 * o + 1],
                                  P + (size_t)o * n_levels * n_levels);
        if (s < 0)
            return -1;
        total += s;
    }
    return total;
}

/* Local GLCM of one win x win window whose top-left pixel is (x0, y0): only
 * pairs with both pixels inside the window are counted. */
static long long window_glcm(const unsigned char *img, size_t pitch, int bpp, int n_levels,
                             int levels_mode, int x0, int y0, int win, int dx, int dy,
                             uint32_t *P)
{
    long long skipped = 0;
    memset(P, 0, sizeof(uint32_t) * (size_t)n_levels * (size_t)n_levels);
    for (int y = y0; y < y0 + win; ++y) {
        for (int x = x0; x < x0 + win; ++x) {
            int x2 = x + dx, y2 = y + dy;
            if (x2 < x0 || x2 >= x0 + win || y2 < y0 || y2 >= y0 + win)
                continue;
            unsigned i = level_of(read_pixel(img, pitch, bpp, x, y), bpp, n_levels, levels_mode);
            unsigned j = level_of(read_pixel(img, pitch, bpp, x2, y2), bpp, n_levels, levels_mode);
            if (i >= (unsigned)n_levels || j >= (unsigned)n_levels) {
                ++skipped;
                continue;
            }
            P[(size_t)i * n_levels + j] += 1u;
        }
    }
    return skipped;
}

/* Sliding-window GLCMs for a list of windows.  Window w is the one whose
 * top-left pixel is (wx[w] * stride, wy[w] * stride); it must lie inside the
 * image.  Output: n_win x n_off x N x N counts.  Returns skipped or -1. */
long long oracle_window_glcm(const void *image, int W, int H, size_t pitch, int bpp,
                             int n_levels, int levels_mode, int win, int stride,
                             int n_off, const int *dxy, int n_win, const int *wx,
                             const int *wy, uint32_t *out)
{
    if (!image || !out || win < 1 || stride < 1)
        return -1;
    const unsigned char *img = (const unsigned char *)image;
    long long total = 0;
    size_t nn = (size_t)n_levels * n_levels;
    for (int w = 0; w < n_win; ++w) {
        int x0 = wx[w] * stride, y0 = wy[w] * stride;
        if (x0 < 0 || y0 < 0 || x0 + win > W || y0 + win > H)
            return -1;
        for (int o = 0; o < n_off; ++o) {
            long long s = window_glcm(img, pitch, bpp, n_levels, levels_mode, x0, y0, win,
                                      dxy[2 * o], dxy[2 * o + 1],
                                      out + ((size_t)w * n_off + o) * nn);
            total += s;
        }
    }
    return total;
}

/* Gray-level histogram of the whole image: h[q] counts the pixels whose level
 * is q (the one-pixel statistic whose voting the paper's contention analysis
 * also covers, Sec. I, contribution 2).  h has N entries.  A pixel >= N in
 * levels mode is not counted; returns how many were skipped, or -1 on bad
 * arguments. */
long long oracle_histogram(const void *image, int W, int H, size_t pitch, int bpp,
                           int n_levels, int levels_mode, uint32_t *h)
{
    if (!image || !h || W < 0 || H < 0 || (bpp != 1 && bpp != 2) || n_levels < 1)
        return -1;
    const unsigned char *img = (const unsigned char *)image;
    long long skipped = 0;
    memset(h, 0, sizeof(uint32_t) * (size_t)n_levels);
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            unsigned q = level_of(read_pixel(img, pitch, bpp, x, y), bpp, n_levels, levels_mode);
            if (q >= (unsigned)n_levels) {
                ++skipped;
                continue;
            }
            h[q] += 1u;
        }
    }
    return skipped;
}

/* Flat-wrap GLCM of one offset: Eq. 2 taken literally on the image as one
 * row-major buffer of W * H pixels (the paper addresses the partner of pixel
 * p as p + d for 0 degrees and p + d (N - 1), p + d N, p + d (N + 1) for the
 * others, with N the image width, Sec. I.A, and pads stripes the same way,
 * Eq. 9).  Pixel p = y W + x pairs with p + dy W + dx whenever that index
 * lies in [0, W H), so a pair may run from the end of one row into another.
 * Returns the skipped count (levels mode) or -1 on bad arguments. */
long long oracle_glcm_flat(const void *image, int W, int H, size_t pitch, int bpp,
                           int n_levels, int levels_mode, int dx, int dy, uint32_t *P)
{
    if (!image || !P || W < 1 || H < 1 || (bpp != 1 && bpp != 2) || n_levels < 1)
        return -1;
    const unsigned char *img = (const unsigned char *)image;
    long long skipped = 0;
    const long long n = (long long)W * H;
    const long long off = (long long)dy * W + dx;
    memset(P, 0, sizeof(uint32_t) * (size_t)n_levels * (size_t)n_levels);
    for (long long p = 0; p < n; ++p) {
        const long long q = p + off;
        if (q < 0 || q >= n)
            continue;
        unsigned i = level_of(read_pixel(img, pitch, bpp, (int)(p % W), (int)(p / W)), bpp, n_levels, levels_mode);
        unsigned j = level_of(read_pixel(img, pitch, bpp, (int)(q % W), (int)(q / W)), bpp, n_levels, levels_mode);
        if (i >= (unsigned)n_levels || j >= (unsigned)n_levels) {
            ++skipped;
            continue;
        }
        P[(size_t)i * n_levels + j] += 1u;
    }
    return skipped;
}

long long oracle_glcm_flat_multi(const void *image, int W, int H, size_t pitch, int bpp,
                                 int n_levels, int levels_mode, int n_off, const int *dxy,
                                 uint32_t *P)
{
    long long total = 0;
    for (int o = 0; o < n_off; ++o) {
        long long s = oracle_glcm_flat(image, W, H, pitch, bpp, n_levels, levels_mode,
                                       dxy[2 * o], dxy[2 * o + 1],
                                       P + (size_t)o * n_levels * n_levels);
        if (s < 0)
            return -1;
        total += s;
    }
    return total;
}
