/*
 * glcm.h -- C ABI of libglcm, a GB300 (sm_103a) library for the gray-level
 * co-occurrence matrix (GLCM) of "Computation of gray-level co-occurrence
 * matrix based on CUDA and its optimization" (Hong, Zheng, Pan, 2017).
 *
 * What is computed (Sec. I.A, Eq. 1): for an image f and an offset (dx, dy),
 *
 *     P[i][j] = #{ (x, y) : f(x, y) has level i, f(x + dx, y + dy) has level j }
 *
 * over every anchor (x, y) whose partner (x + dx, y + dy) lies inside the
 * image.  x is the column, y the row (growing downwards), so the paper's
 * directions 0/45/90/135 degrees at distance d (Eq. 2) are (d, 0), (d, -d),
 * (0, -d), (-d, -d); diagonal distances are chessboard steps.  Pairs never
 * wrap from one row into the next.  The bin of a pair is i * N + j with i
 * the anchor's level (Eq. 3), one vote per pair, exact uint32 counts.
 *
 * Levels: a pixel v of b bits (b = 8 or 16) has level floor(v * N / 2^b)
 * (the paper reduces images to N = 8, 16 or 32 levels without giving the
 * mapping, Sec. I.A); with GLCM_INPUT_LEVELS the pixel already is its level
 * and must be < N.
 *
 * Pointers.  Every image, count, normalized, feature or map pointer may be a
 * host pointer (pageable or pinned) or a device pointer of the context's
 * device; the library tells them apart with cudaPointerGetAttributes.  The
 * caller owns all of them.  An image is `height` rows of `pitch_bytes` bytes
 * each, pixels little-endian for uint16.
 *
 * Synchronicity.  A context created with a CUDA stream enqueues its work on
 * that stream and returns as soon as everything is enqueued when all the
 * call's pointers are device pointers; the caller synchronizes (the stream,
 * or glcm_synchronize, which also reports device-detected errors).  Calls
 * that read or write host memory, and every call on a context created
 * without a stream, return after the results are in place.
 *
 * Errors.  Every function returns a glcm_status (0 = success); nothing is
 * thrown across the ABI.  glcm_last_error() gives a message for the last
 * failure on a context.  Pixels >= N in levels mode are skipped (their pairs
 * are not counted) and the call, or the next glcm_synchronize, returns
 * GLCM_ERR_RANGE; the kernels never trap.
 */
#ifndef GLCM_H
#define GLCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct glcm_ctx glcm_ctx;

typedef enum {
    GLCM_OK = 0,
    GLCM_ERR_ARG = -1,         /* invalid argument                                */
    GLCM_ERR_RANGE = -2,       /* a pixel >= N in GLCM_INPUT_LEVELS mode          */
    GLCM_ERR_NOMEM = -3,       /* device or pinned memory could not be obtained   */
    GLCM_ERR_UNSUPPORTED = -4, /* valid request outside what is implemented       */
    GLCM_ERR_CUDA = -5,        /* a CUDA runtime call failed                      */
    GLCM_ERR_TIMEOUT = -6,     /* a bounded device or host wait gave up           */
    GLCM_ERR_BUSY = -7         /* admission refused: HBM budget or slots exhausted */
} glcm_status;

enum { GLCM_U8 = 0, GLCM_U16 = 1 };

enum {
    GLCM_SYMMETRIC = 1,    /* normalized / features use S = P + P^T           */
    GLCM_NORMALIZE = 2,    /* write p = S / sum(S) as float32                 */
    GLCM_INPUT_LEVELS = 4, /* pixels are levels already (must be < N)         */
    GLCM_FLAT_WRAP = 8     /* pair along the flat row-major buffer (below)    */
};

/* GLCM_FLAT_WRAP: Eq. 2 read literally on the image as one row-major buffer
 * of width * height pixels (the paper addresses partners by adding d, d (N-1),
 * d N or d (N+1) to a pixel's index, N the image width, Sec. I.A, and pads
 * its stripes the same way, Eq. 9).  Pixel p = y * width + x pairs with
 * p + dy * width + dx whenever that index lies in [0, width * height), so
 * pairs also run from the end of a row into another row; the default (no
 * flag) counts only partners inside the image rectangle.  The extra pairs are
 * exactly those whose partner column x + dx leaves [0, width).  Accepted by
 * glcm_compute, glcm_compute_batch, glcm_enqueue_batch and the server. */

#define GLCM_MAX_LEVELS 256        /* normalized GLCMs, features, windows, histograms */
#define GLCM_MAX_COUNT_LEVELS 4096 /* counts alone (glcm_compute, batches, server)    */
#define GLCM_MAX_OFFSETS 64
#define GLCM_N_FEATURES 14
#define GLCM_N_WINDOW_MAPS 4
#define GLCM_MAX_WINDOW_OFFSETS 8

typedef struct {
    int dx, dy; /* partner of anchor (x, y) is (x + dx, y + dy) */
} glcm_offset;

/* One image of a batch (glcm_compute_batch). */
typedef struct {
    const void *image;          /* height rows of pitch_bytes                      */
    int width, height;
    size_t pitch_bytes;
    int dtype;                  /* GLCM_U8 or GLCM_U16                             */
    int levels;                 /* N, 2..256 (..4096 without normalized/features)  */
    const glcm_offset *offsets; /* n_offsets entries (host memory)                 */
    int n_offsets;              /* 1..GLCM_MAX_OFFSETS                             */
    int flags;                  /* GLCM_SYMMETRIC | GLCM_INPUT_LEVELS | GLCM_FLAT_WRAP */
    uint32_t *counts;           /* n_offsets x N x N, required                     */
    float *normalized;          /* n_offsets x N x N or NULL                       */
    float *features;            /* n_offsets x 14 or NULL                          */
} glcm_desc;

/* Create a context on CUDA device `device`.  `hbm_budget_bytes` caps the
 * device memory the context may hold for staging and scratch (0 = 1 GiB).
 * `cuda_stream` is a cudaStream_t to enqueue on, or NULL for a private
 * stream with synchronous calls.  *out receives the context (owned by the
 * caller, released with glcm_destroy).
 * Errors: GLCM_ERR_ARG (out NULL, bad device), GLCM_ERR_CUDA, GLCM_ERR_NOMEM. */
int glcm_create(glcm_ctx **out, int device, size_t hbm_budget_bytes, void *cuda_stream);

/* Wait for all work enqueued by the context, free everything it owns.
 * NULL is accepted.  Returns GLCM_OK or GLCM_ERR_CUDA. */
int glcm_destroy(glcm_ctx *ctx);

/* Message for the last failure on ctx ("" if none); valid until the next
 * call on ctx.  With ctx == NULL: the last failure of glcm_create. */
const char *glcm_last_error(const glcm_ctx *ctx);

/* (dx, dy) of distance d >= 1 at theta in {0, 45, 90, 135} degrees, the
 * directions of Eq. 2: (d,0), (d,-d), (0,-d), (-d,-d).  GLCM_ERR_ARG for
 * any other theta or d < 1. */
int glcm_offset_from_angle(int d, int theta_deg, glcm_offset *out);

/* GLCMs of one image for n_offsets offsets (Eq. 1, all offsets fused in
 * one pass over the image).
 *   image       height rows of pitch_bytes; pitch_bytes >= width * bytes per pixel
 *   levels      N in 2..256; up to GLCM_MAX_COUNT_LEVELS (4096, e.g. 1024 for
 *               full-range uint16) for counts alone -- those GLCMs vote straight
 *               into the output counts in L2 (warp-aggregated global
 *               reductions; N^2 bins do not fit shared memory) and GLCM_NORMALIZE
 *               returns GLCM_ERR_UNSUPPORTED
 *   offsets     host array of n_offsets (1..64) offsets, |dx| < 65536, |dy| < 65536
 *   flags       GLCM_SYMMETRIC, GLCM_NORMALIZE, GLCM_INPUT_LEVELS, GLCM_FLAT_WRAP
 *   counts      out: n_offsets x N x N uint32, row-major [offset][i][j]; always
 *               the plain (non-symmetric) counts P
 *   normalized  out (or NULL): n_offsets x N x N float32, p = S / sum(S) with
 *               S = P + P^T if GLCM_SYMMETRIC else P; all zero for an empty GLCM.
 *               Written only when GLCM_NORMALIZE is set.
 * Host images are streamed to the device in row stripes with halo rows on a
 * side stream, overlapped with the votes of earlier stripes (Sec. III,
 * Eqs. 7-9).
 * Errors: GLCM_ERR_ARG, GLCM_ERR_RANGE, GLCM_ERR_NOMEM (image staging over
 * budget), GLCM_ERR_CUDA. */
int glcm_compute(glcm_ctx *ctx, const void *image, int width, int height, size_t pitch_bytes,
                 int dtype, int levels, const glcm_offset *offsets, int n_offsets, int flags,
                 uint32_t *counts, float *normalized);

/* The 14 Haralick texture features (named by the paper, Sec. I, as the use
 * of each GLCM) of n_glcm count matrices.
 *   counts    n_glcm x N x N uint32 (as written by glcm_compute)
 *   flags     GLCM_SYMMETRIC: features of S = P + P^T, else of P
 *   features  out: n_glcm x 14 float32 in the order asm, contrast,
 *             correlation, sum of squares, inverse difference moment, sum
 *             average, sum variance, sum entropy, entropy, difference
 *             variance, difference entropy, information measures of
 *             correlation 1 and 2, maximal correlation coefficient.
 *             Natural logarithms; correlation is 1 when a marginal has zero
 *             variance; an empty GLCM gives all zeros.
 * float32 arithmetic with compensated sums; the correlation means and
 * variances in float64.
 * Errors: GLCM_ERR_ARG, GLCM_ERR_CUDA. */
int glcm_features(glcm_ctx *ctx, const uint32_t *counts, int levels, int n_glcm, int flags,
                  float *features);

/* A batch of images (multispectral bands, many images of uneven sizes, all
 * their offsets) in one persistent vote launch plus one epilogue launch,
 * replayed from a cached CUDA graph when the same batch (same pointers,
 * sizes and flags) comes again.  Per desc: counts always, normalized if
 * non-NULL (GLCM_NORMALIZE implied), features if non-NULL.  Each desc's
 * results equal those of a glcm_compute + glcm_features on that image alone.
 * Host images (and host results) may be mixed with device ones: host images
 * are copied once into device staging on a side stream in up to four groups
 * of consecutive images, each group's votes starting as soon as its copies
 * are in (Sec. III's overlap of copies with earlier votes).  Images whose
 * features are asked for at N > 64 come first, as one group, and their
 * epilogue overlaps the votes of the rest.  Registered (pinned) host images
 * are read by a copy kernel on a few SMs, which the vote launches leave free
 * while later groups are still copying; other host memory goes through
 * cudaMemcpyAsync / cudaMemcpy2DAsync.  The call returns after the host
 * results are written.  Results do not depend on the grouping.
 * Errors: as glcm_compute, per the first failing desc. */
int glcm_compute_batch(glcm_ctx *ctx, const glcm_desc *descs, int n);

/* The same batch as glcm_compute_batch, launched directly (no graph is
 * captured or cached) and never synchronized: the call returns once the
 * table upload, the vote launches and the epilogue launch are enqueued on the
 * context's stream.  For batches whose composition changes every call (a
 * serving loop).  All pointers are device pointers; the caller keeps them
 * valid until the stream has passed the work, and glcm_synchronize reports
 * device-detected errors.
 * Errors: GLCM_ERR_ARG (host pointers, bad descs), GLCM_ERR_NOMEM, GLCM_ERR_CUDA. */
int glcm_enqueue_batch(glcm_ctx *ctx, const glcm_desc *descs, int n);

/* Local GLCMs of sliding win x win windows whose top-left pixels are
 * (u*stride, v*stride), u < nwx = (width - win)/stride + 1,
 * v < nwy = (height - win)/stride + 1; each window's GLCM counts the pairs
 * with both pixels inside the window.
 *   offsets   1..8 offsets with |dx|, |dy| < win
 *   counts    out (or NULL): nwy x nwx x n_offsets x N x N uint32
 *   maps      out (or NULL): 4 x n_offsets x nwy x nwx float32 -- contrast,
 *             angular second moment, inverse difference moment, entropy of
 *             each window's normalized GLCM (symmetric with GLCM_SYMMETRIC)
 * Errors: GLCM_ERR_ARG, GLCM_ERR_UNSUPPORTED (window histograms larger than
 * shared memory), GLCM_ERR_RANGE, GLCM_ERR_CUDA. */
int glcm_windows(glcm_ctx *ctx, const void *image, int width, int height, size_t pitch_bytes,
                 int dtype, int levels, int win, int stride, const glcm_offset *offsets,
                 int n_offsets, int flags, uint32_t *counts, float *maps);

/* One sliding-window job of a batch (glcm_compute_batch_windows): the
 * arguments of glcm_windows, all buffers device memory. */
typedef struct {
    const void *image;          /* height rows of pitch_bytes (device)            */
    int width, height;
    size_t pitch_bytes;
    int dtype;                  /* GLCM_U8 or GLCM_U16                             */
    int levels;                 /* N, 2..256                                       */
    int win, stride;            /* window side and step (glcm_windows)             */
    const glcm_offset *offsets; /* 1..GLCM_MAX_WINDOW_OFFSETS (host memory)        */
    int n_offsets;
    int flags;                  /* GLCM_SYMMETRIC | GLCM_INPUT_LEVELS              */
    uint32_t *counts;           /* nwy x nwx x n_offsets x N x N or NULL (device)  */
    float *maps;                /* 4 x n_offsets x nwy x nwx or NULL (device)      */
} glcm_window_desc;

/* A batch of images (as glcm_compute_batch, device buffers only) and of
 * sliding-window jobs (as glcm_windows) in one CUDA-graph launch: the first
 * call runs them directly and captures the graph -- the window kernels, then
 * the batch's persistent vote launches and epilogue -- and later calls with
 * the same descriptors (pointers, sizes, flags) replay it, so a whole
 * workload of many images and window maps costs one launch (the paper's
 * launch-shape rules, Eqs. 4-6, give way to one captured schedule).  Results
 * equal those of glcm_compute_batch and glcm_windows.  n or n_win may be 0.
 * Errors: GLCM_ERR_ARG (host buffers, bad descs), GLCM_ERR_UNSUPPORTED,
 * GLCM_ERR_NOMEM, GLCM_ERR_RANGE, GLCM_ERR_CUDA. */
int glcm_compute_batch_windows(glcm_ctx *ctx, const glcm_desc *descs, int n, const glcm_window_desc *wins,
                               int n_win);

/* Gray-level histogram of one image: hist[q] = the number of pixels whose
 * level (quantized as for glcm_compute) is q.  The one-pixel statistic to
 * which the paper's analysis of vote collisions also applies (Sec. I,
 * contribution 2).
 *   image, width, height, pitch_bytes, dtype, levels   as for glcm_compute
 *   flags   GLCM_INPUT_LEVELS (others ignored)
 *   hist    out: levels uint32 (host or device pointer), overwritten
 * In GLCM_INPUT_LEVELS mode a pixel >= levels is not counted and the call
 * returns GLCM_ERR_RANGE (after the kernel, or at glcm_synchronize for device
 * buffers on a caller's stream).
 * Errors: GLCM_ERR_ARG (also more than 2^32 - 1 pixels), GLCM_ERR_UNSUPPORTED
 * (levels > 256), GLCM_ERR_RANGE, GLCM_ERR_NOMEM, GLCM_ERR_CUDA. */
int glcm_histogram(glcm_ctx *ctx, const void *image, int width, int height, size_t pitch_bytes,
                   int dtype, int levels, int flags, uint32_t *hist);

/* Wait for the context's stream; report device-detected errors of the work
 * enqueued since the last check (GLCM_ERR_RANGE, GLCM_ERR_TIMEOUT) and
 * clear them. */
int glcm_synchronize(glcm_ctx *ctx);

/* Kernel timing: when enabled, CUDA events bracket every vote-kernel launch
 * and glcm_get_timing returns the summed device milliseconds of the vote
 * kernels completed since the last reset, how many vote launches that was,
 * and how many kernels the context launched in total.  Reading synchronizes
 * the context's stream. */
int glcm_set_timing(glcm_ctx *ctx, int enable);
int glcm_get_timing(glcm_ctx *ctx, double *vote_ms, long long *vote_launches,
                    long long *kernel_launches, int reset);

/* Vote-kernel configuration for one (levels, offsets, pixel type) class, as
 * chosen by the autotuner: threads per CTA (64..1024, multiple of 32), log2
 * of the private histogram copies per CTA (0..5; copy c serves lanes with
 * lane % copies == c), the shared-memory layout (0: one row of copies per
 * bin; 1: two offsets' rows interleaved per bin; 2: two offsets as 16-bit
 * halves of one word; 3: one offset's partner levels j and j + ceil(N/2) as
 * 16-bit halves of one word, so that N = 256 takes one pass per offset; 4:
 * the column-walk kernel, which every offset at chessboard distance 1 of an
 * image with N a power of two up to 32 takes by default -- threads and
 * copies are then fixed), and anchor rows per work item (0 = derived).
 * Offsets that do not fit one CTA's shared memory together are split over
 * several passes, and a histogram whose one level row does not fit is
 * rejected.  A layout of 0..3 sends the class's distance-1 offsets to the
 * general kernel too.  threads <= 0 removes the override.
 * Errors: GLCM_ERR_ARG. */
int glcm_set_vote_config(glcm_ctx *ctx, int levels, int n_offsets, int dtype, int threads,
                         int log2_copies, int layout, int band_rows);

/* Scheme 1 of the paper (Sec. I.B): one thread per pixel and one global
 * atomic per vote, one offset.  Ablation baseline with the same inputs and
 * outputs as glcm_compute for one offset (device pointers only). */
int glcm_compute_naive(glcm_ctx *ctx, const void *image, int width, int height,
                       size_t pitch_bytes, int dtype, int levels, glcm_offset offset, int flags,
                       uint32_t *counts);

/* GLCM counts of one device image without allocating anything (the paper has
 * no counterpart; this is a deployment variant of glcm_compute).
 *
 * For callers that cannot call cudaMalloc while they run: real-time or
 * embedded pipelines that reserve all memory up front, code running inside a
 * custom allocator or memory pool that forbids nested allocation, and threads
 * that must not block on the allocator.  glcm_create and the context entry
 * points allocate tables and scratch on first use; this call does not.  It
 * needs no context.
 *
 * The vote kernel's scratch (job, offset and chunk tables, the chunk counter,
 * the error word; about 113 KB) is one fixed static device array present on
 * every device that loads the library until the process exits.  Every call
 * looks up the array's device address in the current context
 * (cudaGetSymbolAddress, which allocates nothing); the first call on a device
 * also loads the library's device code there, so make it before any stream
 * capture.  Every call reuses the array and clears the counter and error word
 * it needs.  Calls are serialized by a process-wide mutex and each waits for
 * its own work, but calls that overlap on the GPU through the same array (for
 * example from another copy of the library in the same process) would race.
 *
 *   image      device pointer of the current device, height rows of pitch_bytes
 *   offsets    host array of n_offsets (1..64) offsets
 *   flags      GLCM_INPUT_LEVELS only (counts are always the plain P;
 *              GLCM_FLAT_WRAP returns GLCM_ERR_UNSUPPORTED)
 *   counts     device pointer, out: n_offsets x N x N uint32 (as glcm_compute)
 *   cuda_stream  stream to run on (NULL: the legacy default stream); the call
 *              returns after the counts are complete
 *   errbuf     optional buffer for a message (errbuf_len bytes)
 * Limits: at most GLCM_NOALLOC_MAX_JOBS histogram passes (offset groups x
 * anchor-level parts) and GLCM_NOALLOC_MAX_CHUNKS scheduling chunks (chunks
 * are made coarser to fit); larger requests return GLCM_ERR_UNSUPPORTED.
 * Errors: GLCM_ERR_ARG (host pointers, bad sizes), GLCM_ERR_RANGE,
 * GLCM_ERR_UNSUPPORTED, GLCM_ERR_CUDA, GLCM_ERR_TIMEOUT. */
#define GLCM_NOALLOC_MAX_JOBS 128
#define GLCM_NOALLOC_MAX_CHUNKS 8192
int glcm_compute_noalloc(const void *image, int width, int height, size_t pitch_bytes, int dtype,
                         int levels, const glcm_offset *offsets, int n_offsets, int flags,
                         uint32_t *counts, void *cuda_stream, char *errbuf, size_t errbuf_len);

/* ---- Measured ceilings ---------------------------------------------------
 *
 * The rates the vote kernels are held against, measured on `device` by
 * microbenchmarks (the paper weighs its copy strategy by the serialization of
 * colliding votes, Sec. I.B and Sec. II.A; these are that serialization's
 * limits on this GPU).  Shared-memory reductions (red.shared.add.u32, one
 * per vote) per second over the whole GPU, one 512-thread CTA per SM, for
 *   red_interleaved_per_s      lane l of every warp on bank l (the
 *                              lane-interleaved private copies: no conflict)
 *   red_same_word_per_s        every lane of a warp on one word, increment 1
 *   red_random_one_copy_per_s  each lane on a random word of one 128 KB copy
 * and hbm_read_gbs, the best of five streaming 16-byte-load reads of a 1 GiB
 * buffer (GB/s, 1e9 bytes).  Allocates 1 GiB for the duration of the call.
 * Errors: GLCM_ERR_ARG (bad device, out NULL), GLCM_ERR_NOMEM, GLCM_ERR_CUDA. */
typedef struct {
    int sm_count;
    double red_interleaved_per_s;
    double red_same_word_per_s;
    double red_random_one_copy_per_s;
    double hbm_read_gbs;
} glcm_ceilings;

int glcm_measure_ceilings(int device, glcm_ceilings *out);

/* ---- Serving: continuous batching of host requests ----------------------
 *
 * A server owns a device-memory arena of hbm_budget_bytes, `lanes` contexts
 * (one CUDA stream each), a copy stream and one scheduler thread.  The paper
 * overlaps the host-to-device copy of image stripes with the votes of
 * earlier stripes over CUDA streams (Sec. III, Eqs. 7-9); the server applies
 * the same overlap across requests.  Its scheduler repeatedly
 *   - admits queued requests in arrival order while their device footprint
 *     (pitched image + counts + normalized + features) fits in the free
 *     arena, and enqueues their image copies on the copy stream;
 *   - gives the admitted requests not yet launched to the next idle lane as
 *     one batch (at most max_batch requests and, past its first request, at
 *     most 256 MiB of images, so that a burst votes batch by batch while the
 *     later batches still copy): the lane waits for those copies, runs the
 *     batch's votes and epilogue, and copies the results to the requests'
 *     host buffers;
 *   - retires finished batches, frees their arena space and wakes waiters.
 * So requests that arrive while others are on the GPU join the next batch as
 * lanes and memory free up, and copies overlap earlier batches' kernels.
 * Each result equals that of glcm_compute (+ glcm_features) on the request
 * alone.  Requests with GLCM_INPUT_LEVELS run as batches of one so that a
 * GLCM_ERR_RANGE belongs to that request. */
typedef struct glcm_server glcm_server;

typedef struct {
    long long submitted, completed, failed;
    long long batches;          /* batches launched                              */
    long long max_batch;        /* most requests in one batch                    */
    long long kernel_launches;  /* kernels the lanes launched                    */
    long long queue_peak;       /* most requests waiting for admission           */
    size_t arena_bytes;         /* arena size                                    */
    size_t arena_peak;          /* most arena bytes in use at once               */
} glcm_server_counters;

/* Create a server on `device`: an arena of hbm_budget_bytes (0 = 4 GiB),
 * `lanes` compute streams (1..8; 0 = 2), at most max_batch requests per
 * batch (0 = 256) and at most max_queue requests waiting for admission
 * (0 = 4096).  Errors: GLCM_ERR_ARG, GLCM_ERR_NOMEM, GLCM_ERR_CUDA. */
int glcm_server_create(glcm_server **out, int device, size_t hbm_budget_bytes, int lanes, int max_batch,
                       int max_queue);

/* Queue one request.  `request` is a glcm_desc whose image, counts and
 * (optional) normalized and features pointers are HOST pointers -- pinned
 * memory lets copies overlap; pageable memory works but blocks the
 * scheduler during its copies.  The offsets are copied; the buffers must
 * stay valid until the request completes.  *ticket receives its id (>= 1).
 * Errors: GLCM_ERR_ARG (bad desc, device pointers), GLCM_ERR_NOMEM
 * (footprint larger than the whole arena), GLCM_ERR_BUSY (admission queue
 * full; retry later). */
int glcm_server_submit(glcm_server *s, const glcm_desc *request, long long *ticket);

/* Wait up to timeout_ms (< 0: no limit; 0: just check) for a request.  When
 * it has completed, returns its status (GLCM_OK or the error that failed
 * it), writes the milliseconds from its submission to its completion into
 * *latency_ms (may be NULL) and forgets the ticket.  Returns GLCM_ERR_BUSY if
 * it is still in flight, GLCM_ERR_ARG for an unknown ticket. */
int glcm_server_wait(glcm_server *s, long long ticket, int timeout_ms, double *latency_ms);

/* Counters since creation.  Errors: GLCM_ERR_ARG. */
int glcm_server_stats(glcm_server *s, glcm_server_counters *out);

/* Message for the last failure of a server call or request ("" if none);
 * with s == NULL, of the last glcm_server_create. */
const char *glcm_server_last_error(const glcm_server *s);

/* Finish every admitted request, fail the ones still queued with
 * GLCM_ERR_BUSY, stop the scheduler and free everything.  NULL is accepted. */
int glcm_server_destroy(glcm_server *s);

#ifdef __cplusplus
}
#endif

#endif /* GLCM_H */
