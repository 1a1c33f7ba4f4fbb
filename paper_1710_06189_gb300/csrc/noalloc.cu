// glcm_compute_noalloc: GLCM counts of one device image with no allocation.
//
// Who needs it: code that must not allocate device memory while it runs --
// a real-time or embedded pipeline that reserves all memory up front, a
// caller inside a custom allocator or memory pool that forbids nested
// cudaMalloc, code holding a lock that cudaMalloc could contend on, or a
// host thread that must never block on the allocator.  The context-based
// entry points allocate (tables, staging, scratch) on first use; this one
// does not.
//
// How: the vote kernel's scratch -- its job, offset and chunk tables, the
// chunk counter and the error word -- lives in one file-scope
// `static __device__` array of fixed size (kScratchBytes, about 113 KB),
// present on every device that loads the library until the process exits.
// Host code cannot use that array's name as a device address, so every call
// looks the address up with cudaGetSymbolAddress in the current device's
// context (a lookup: it allocates nothing).  The address is not kept between
// calls, because it belongs to one context: after cudaDeviceReset, or under
// another context on the same device, a kept address would point at memory
// that no longer holds the array.  The first call on a device also loads the
// library's device code into that context (set-up), so it should come before
// any stream capture.  Planning uses fixed host arrays, never the heap.  Every call reuses the array, so the counter and error word are
// cleared on each call; a process-wide mutex serializes calls and each call
// waits for its own work, but two callers sharing the array from different
// processes or library copies would race.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "glcm.h"
#include "glcm_internal.cuh"

using namespace glcm;

namespace {

constexpr int kNaMaxJobs = GLCM_NOALLOC_MAX_JOBS;
constexpr int kNaMaxChunks = GLCM_NOALLOC_MAX_CHUNKS;
constexpr int kNaThreads = 512;
constexpr int kNaBand = 32;
constexpr int kNaTileRows = 48;

struct NaScratch {
    VoteJob jobs[kNaMaxJobs];
    VoteOffset offs[GLCM_MAX_OFFSETS];
    int3 chunks[kNaMaxChunks];
    unsigned words[64];  // [0] error bits, [1] chunk counter
};
constexpr size_t kScratchBytes = sizeof(NaScratch);

static __device__ __align__(256) unsigned char g_na_scratch[kScratchBytes];

std::mutex g_na_mutex;
NaScratch g_na_host;  // host-side plan, copied into the device array

int na_fail(char* errbuf, size_t len, int code, const char* msg)
{
    if (errbuf && len > 0) {
        strncpy(errbuf, msg, len - 1);
        errbuf[len - 1] = '\0';
    }
    return code;
}

int ilog2_or(int n)
{
    for (int k = 0; k < 31; ++k)
        if ((1 << k) == n)
            return k;
    return -1;
}

// Jobs needed for one configuration (same rules as the context planner).
struct NaShape {
    int groups_per_job, span, jobs;
};

// Bin rows per anchor level: layout 3 packs two partner levels per word.
long long na_level_rows(int layout, int levels) { return layout == 3 ? (levels + 1) / 2 : levels; }
int na_group_offsets(int layout) { return layout == 0 || layout == 3 ? 1 : 2; }

NaShape na_shape(long long budget, int levels, int n_off, int layout, int rshift)
{
    const long long wrow = (layout == 1 ? 2ll : 1ll) << rshift;
    const int opg = na_group_offsets(layout);
    const int groups = (n_off + opg - 1) / opg;
    const long long per_level = na_level_rows(layout, levels) * wrow;
    const long long per_group = (long long)levels * per_level;
    NaShape s{1, 0, 0};
    if (per_group <= budget) {
        s.groups_per_job = (int)(budget / per_group < groups ? budget / per_group : groups);
        s.span = levels;
        s.jobs = (groups + s.groups_per_job - 1) / s.groups_per_job;
    } else {
        s.span = (int)(budget / per_level);
        if (s.span < 1)
            return NaShape{1, 0, 0};
        s.jobs = groups * ((levels + s.span - 1) / s.span);
    }
    return s;
}

}  // namespace

extern "C" int glcm_compute_noalloc(const void* image, int width, int height, size_t pitch_bytes, int dtype,
                                    int levels, const glcm_offset* offsets, int n_offsets, int flags,
                                    uint32_t* counts, void* cuda_stream, char* errbuf, size_t errbuf_len)
{
    if (!image || !counts || !offsets)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_ARG, "image, offsets and counts are required");
    if (width < 1 || height < 1 || width >= (1 << 30) || height >= (1 << 30))
        return na_fail(errbuf, errbuf_len, GLCM_ERR_ARG, "width and height must be in 1..2^30-1");
    if (dtype != GLCM_U8 && dtype != GLCM_U16)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_ARG, "dtype must be GLCM_U8 or GLCM_U16");
    const int bpp = dtype == GLCM_U8 ? 1 : 2;
    if (pitch_bytes < (size_t)width * bpp)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_ARG, "pitch_bytes < width * bytes per pixel");
    if (levels > GLCM_MAX_LEVELS)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_UNSUPPORTED, "levels > 256");
    if (levels < 2)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_ARG, "levels must be in 2..256");
    if (n_offsets < 1 || n_offsets > GLCM_MAX_OFFSETS)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_ARG, "need 1..64 offsets");
    for (int k = 0; k < n_offsets; ++k)
        if (offsets[k].dx <= -65536 || offsets[k].dx >= 65536 || offsets[k].dy <= -65536 || offsets[k].dy >= 65536)
            return na_fail(errbuf, errbuf_len, GLCM_ERR_ARG, "offset out of range");
    if (flags & GLCM_FLAT_WRAP)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_UNSUPPORTED, "GLCM_FLAT_WRAP is not supported here");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_CUDA, "no current CUDA device");
    for (const void* ptr : {image, static_cast<const void*>(counts)}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev) {
            cudaGetLastError();
            return na_fail(errbuf, errbuf_len, GLCM_ERR_ARG,
                           "image and counts must be device memory of the current device");
        }
    }
    std::lock_guard<std::mutex> guard(g_na_mutex);
    // The device address of the static scratch in the current context.
    NaScratch* dscr = nullptr;
    {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return na_fail(errbuf, errbuf_len, GLCM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        }
        dscr = static_cast<NaScratch*>(p);
    }
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);

    // Plan into fixed host arrays (the same rules as the context planner).
    int optin = 0, sms = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long budget = (optin - 2 * kNaTileRows * vote_row_bytes() - 4096) / 4;
    // The context planner's cost model (default_cfg): ~2 per pass over the
    // image, per offset voted in a pass ~1.5 plus the copy count's conflict
    // factor, plus ~1.5 for packed halves or ~2 for two offsets in halves.
    static const double conflict[6] = {2.2, 2.0, 1.8, 1.6, 1.4, 1.0};
    int rshift = 0, layout = 0;
    double best = 1e30;
    for (int r = 5; r >= 0; --r)
        for (int lay : {1, 0, 2, 3}) {
            if (lay == 2 && 65535ll * (1 << r) / (16ll * kNaThreads) < 64)
                continue;
            const NaShape s = na_shape(budget, levels, n_offsets, lay, r);
            if (s.jobs <= 0)
                continue;
            const int parts = (levels + s.span - 1) / s.span;
            const double per_off = 1.5 + conflict[r] + (lay == 3 ? 1.5 : 0.0) + (lay == 2 ? 2.0 : 0.0);
            const double cost = 2.0 * s.jobs + (double)n_offsets * parts * per_off;
            if (cost < best - 1e-9) {
                best = cost;
                rshift = r;
                layout = lay;
            }
        }
    const NaShape shape = na_shape(budget, levels, n_offsets, layout, rshift);
    if (shape.jobs <= 0)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_UNSUPPORTED, "histograms do not fit shared memory");
    NaScratch& h = g_na_host;
    int order[GLCM_MAX_OFFSETS];
    for (int k = 0; k < n_offsets; ++k)
        order[k] = k;
    for (int a = 1; a < n_offsets; ++a)  // stable insertion sort by dy
        for (int b = a; b > 0 && offsets[order[b]].dy < offsets[order[b - 1]].dy; --b) {
            const int t = order[b];
            order[b] = order[b - 1];
            order[b - 1] = t;
        }
    const int PX = 16 / bpp;
    const int strip_px = 32 * PX;
    const int n_strips = (width + strip_px - 1) / strip_px;
    const int n_bands = (height + kNaBand - 1) / kNaBand;
    const int opg = na_group_offsets(layout);
    const int per_job = shape.groups_per_job * opg;
    const int log2n = ilog2_or(levels);
    const bool aligned = ((reinterpret_cast<uintptr_t>(image) | (uintptr_t)pitch_bytes) & 15) == 0;
    int n_jobs = 0, n_off_used = 0, n_items = 0, tile_rows = 0, max_words = 0;
    for (int o0 = 0; o0 < n_offsets;) {
        int cnt = 1;
        int dmin = offsets[order[o0]].dy < 0 ? offsets[order[o0]].dy : 0;
        int dmax = offsets[order[o0]].dy > 0 ? offsets[order[o0]].dy : 0;
        while (o0 + cnt < n_offsets && cnt < per_job) {
            const int d = offsets[order[o0 + cnt]].dy;
            const int nmin = d < dmin ? d : dmin, nmax = d > dmax ? d : dmax;
            if (nmax - nmin > kMaxDySpan && dmax - dmin <= kMaxDySpan)
                break;
            dmin = nmin;
            dmax = nmax;
            ++cnt;
        }
        for (int k = o0; k < o0 + cnt; ++k) {
            VoteOffset vo{};
            vo.dx = offsets[order[k]].dx;
            vo.dy = offsets[order[k]].dy;
            vo.slot = order[k];
            h.offs[n_off_used + (k - o0)] = vo;
        }
        for (int lv = 0; lv < levels; lv += shape.span) {
            if (n_jobs >= kNaMaxJobs)
                return na_fail(errbuf, errbuf_len, GLCM_ERR_UNSUPPORTED,
                               "request needs more jobs than the static scratch holds (GLCM_NOALLOC_MAX_JOBS)");
            const int span = shape.span < levels - lv ? shape.span : levels - lv;
            VoteJob j{};
            j.img = static_cast<const uint8_t*>(image);
            j.pitch = (long long)pitch_bytes;
            j.W = width;
            j.H = height;
            j.bpp = bpp;
            j.levels = levels;
            j.log2n = log2n;
            j.levels_mode = (flags & GLCM_INPUT_LEVELS) ? 1 : 0;
            j.aligned = aligned ? 1 : 0;
            j.n_off = cnt;
            j.off0 = n_off_used;
            j.rshift = rshift;
            j.layout = layout;
            j.lv_lo = lv;
            j.lv_span = span;
            j.bytecode = (layout == 1 && rshift == 5 && span == levels && log2n >= 0 && levels <= 16) ? 1 : 0;
            j.hist_words = (int)((long long)((cnt + opg - 1) / opg) * span * na_level_rows(layout, levels) *
                                 ((layout == 1 ? 2 : 1) << rshift));
            j.item0 = n_items;
            j.n_job_items = n_strips * n_bands;
            const double votes_per_item = (double)kNaBand * strip_px * cnt * span / levels;
            const double want = (10.0 * (2.0 * j.hist_words + 64.0)) / (votes_per_item > 1.0 ? votes_per_item : 1.0);
            j.chunk_items = want < 1.0 ? 1 : (want > j.n_job_items ? j.n_job_items : (int)want + 1);
            j.n_strips = n_strips;
            j.band_rows = kNaBand;
            j.y_begin = 0;
            j.y_end = height;
            j.dy_min = dmin;
            j.dy_max = dmax;
            j.staged = (dmax - dmin <= kMaxDySpan) ? 1 : 0;
            j.out = counts;
            if (j.staged && kNaBand + dmax - dmin > tile_rows)
                tile_rows = kNaBand + dmax - dmin;
            if (j.hist_words > max_words)
                max_words = j.hist_words;
            n_items += j.n_job_items;
            h.jobs[n_jobs++] = j;
        }
        n_off_used += cnt;
        o0 += cnt;
    }
    // Chunks; if there are more than the scratch holds, make them coarser.
    {
        const int cap = n_items / (3 * sms) > 1 ? n_items / (3 * sms) : 1;  // >= ~3 chunks per CTA
        for (int jb = 0; jb < n_jobs; ++jb)
            if (h.jobs[jb].chunk_items > cap)
                h.jobs[jb].chunk_items = cap;
    }
    // Coarser chunks (items per chunk times `scale`, at most a whole job)
    // until the chunks fit; every job needs at least one, and the jobs fit.
    auto chunks_at = [&](long long scale) {
        long long n = 0;
        for (int jb = 0; jb < n_jobs; ++jb) {
            const long long ci = h.jobs[jb].chunk_items * scale < h.jobs[jb].n_job_items
                                     ? h.jobs[jb].chunk_items * scale
                                     : h.jobs[jb].n_job_items;
            n += (h.jobs[jb].n_job_items + ci - 1) / ci;
        }
        return n;
    };
    long long scale = 1;
    while (chunks_at(scale) > kNaMaxChunks)
        scale *= 2;
    int n_chunks = 0;
    for (int jb = 0; jb < n_jobs; ++jb) {
        VoteJob& j = h.jobs[jb];
        if (scale > 1)
            j.chunk_items = (int)(j.chunk_items * scale < j.n_job_items ? j.chunk_items * scale : j.n_job_items);
        for (int k = 0; k < j.n_job_items; k += j.chunk_items) {
            if (n_chunks >= kNaMaxChunks)
                return na_fail(errbuf, errbuf_len, GLCM_ERR_UNSUPPORTED,
                               "request needs more chunks than the static scratch holds (GLCM_NOALLOC_MAX_CHUNKS)");
            const int e = k + j.chunk_items < j.n_job_items ? k + j.chunk_items : j.n_job_items;
            h.chunks[n_chunks++] = make_int3(jb, j.item0 + k, j.item0 + e);
        }
    }

    // Upload the plan into the static scratch, clear the counts, the chunk
    // counter and the error word, vote, and wait for the result.
    const size_t nn = (size_t)levels * levels;
#define NA_CK(call)                                                                               \
    do {                                                                                          \
        const cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                                  \
            char m_[256];                                                                         \
            snprintf(m_, sizeof m_, "%s failed: %s", #call, cudaGetErrorString(e_));              \
            return na_fail(errbuf, errbuf_len, GLCM_ERR_CUDA, m_);                                \
        }                                                                                         \
    } while (0)
    NA_CK(cudaMemcpyAsync(dscr->jobs, h.jobs, sizeof(VoteJob) * n_jobs, cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemcpyAsync(dscr->offs, h.offs, sizeof(VoteOffset) * n_off_used, cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemcpyAsync(dscr->chunks, h.chunks, sizeof(int3) * n_chunks, cudaMemcpyHostToDevice, stream));
    NA_CK(cudaMemsetAsync(dscr->words, 0, sizeof(dscr->words), stream));
    NA_CK(cudaMemsetAsync(counts, 0, n_offsets * nn * sizeof(uint32_t), stream));
    VoteParams vp{};
    vp.jobs = dscr->jobs;
    vp.n_jobs = n_jobs;
    vp.offs = dscr->offs;
    vp.n_items = n_items;
    vp.chunks = dscr->chunks;
    vp.n_chunks = n_chunks;
    vp.tile_bytes = tile_rows * vote_row_bytes();
    vp.max_hist_words = max_words;
    vp.item_counter = &dscr->words[1];
    vp.err = &dscr->words[0];
    size_t smem = 2 * (size_t)tile_rows * vote_row_bytes() + (size_t)max_words * 4;
    if (smem < 16)
        smem = 16;
    int per_sm = vote_blocks_per_sm(bpp, kNaThreads, smem, layout == 3);
    per_sm = per_sm < 1 ? 1 : per_sm;
    int grid = sms * per_sm;
    grid = grid < n_chunks ? grid : n_chunks;
    grid = grid < 1 ? 1 : grid;
    NA_CK(launch_vote(vp, bpp, grid, kNaThreads, smem, stream, layout == 3));
    unsigned err_bits = 0;
    NA_CK(cudaMemcpyAsync(&err_bits, &dscr->words[0], sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    NA_CK(cudaStreamSynchronize(stream));
#undef NA_CK
    if (err_bits & kErrInternal)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_CUDA, "a kernel index check failed");
    if (err_bits & kErrTimeout)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_TIMEOUT, "a bounded device wait gave up");
    if (err_bits & kErrRange)
        return na_fail(errbuf, errbuf_len, GLCM_ERR_RANGE, "a pixel >= levels in GLCM_INPUT_LEVELS mode; its pairs were skipped");
    na_fail(errbuf, errbuf_len, GLCM_OK, "");
    return GLCM_OK;
}
