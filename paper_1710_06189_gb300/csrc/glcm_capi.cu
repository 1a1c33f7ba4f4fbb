// C ABI of libglcm (declared in include/glcm.h): contexts, argument checks,
// work planning, the host-image stripe pipeline (Sec. III, Eqs. 7-9), batch
// launches with a CUDA-graph cache, and kernel timing.
#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <unordered_map>
#include <vector>

#include "glcm.h"
#include "glcm_internal.cuh"

using namespace glcm;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct VoteCfg {
    int threads = 512;
    int rshift = 5;     // log2 private copies
    int layout = 1;     // see VoteJob::layout; 4: the column-walk kernel for offsets at distance 1
    int band_rows = 0;  // 0: derived from the launch size
};

struct TimedPair {
    cudaEvent_t a, b;
};

struct GraphEntry {
    cudaGraph_t graph = nullptr;  // kept alive: its nodes address the exec's event records
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t ev_start = nullptr, ev_stop = nullptr;
    cudaEvent_t cap_a = nullptr, cap_b = nullptr;  // events recorded at capture
    DevBuf jobs, offs, feat;
    DevBuf jobs2, offs2, feat2;  // second part of a split batch
    int n_vote_kernels = 0;
    int n_kernels = 0;
};

// Jobs of the column-walk kernel for one (pixel type, N, row alignment): one
// launch.
struct FastClass {
    int bpp = 1, log2n = 1;
    bool aligned = true;  // every row of every job starts on 16 bytes
    int max_dist = 1;     // largest partner distance of the class's jobs (row rings when > 1)
    std::vector<FastJob> jobs;
    std::vector<int3> chunks;  // (class-local job, first item, end item)
    int n_items = 0;
    int max_hist_words = 0;
    size_t jobs_off = 0, chunks_off = 0;  // byte offsets in the uploaded jobs buffer
};

// Host-side plan of one vote launch.
struct VotePlan {
    std::vector<VoteJob> jobs;
    std::vector<VoteOffset> offs;
    int n_items = 0;
    std::vector<int3> chunks;  // (job, first item, end item), job-major
    size_t chunk_off = 0;      // byte offset of this plan's chunks in the jobs buffer
    int max_hist_words = 0;
    int tile_rows = 0;  // max staged tile rows over the plan's jobs
    int threads = 0;    // max over the plan's jobs
    int bpp = 1;
    int max_ctas = 0;   // grid cap (0: every SM), leaves SMs to a concurrent kernel
    std::vector<FastClass> fast;  // column-walk launches (offsets at distance 1)
    std::vector<SeamJob> seams;   // flat-wrap pairs across row ends (GLCM_FLAT_WRAP)
    size_t seams_off = 0;         // byte offset of the seam table in the jobs buffer
    std::vector<SeamJob> globals; // N > 256: every pair of one offset voted into global counts
    size_t globals_off = 0;
};

bool plan_empty(const VotePlan& p) { return p.jobs.empty() && p.fast.empty() && p.globals.empty(); }

}  // namespace

struct glcm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;
    cudaStream_t side_stream = nullptr;  // epilogues overlapped with votes in split batches
    cudaStream_t epi_stream = nullptr;   // light groups' epilogues in host-buffer batches
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr;
    // Column-walk classes of one vote launch group voted side by side, and
    // their epilogues after them (one stream per number of levels).
    cudaStream_t cls_stream[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_cls_fork = nullptr, ev_cls_vote[4] = {}, ev_cls_done[4] = {};
    size_t budget = 0, used = 0;
    int sm_count = 0, smem_optin = 0;
    int prio_high = 0;  // the device's most urgent stream priority (class epilogues)
    int sm_reserve = 0;  // SMs every vote launch leaves free (to a concurrent copy kernel)
    unsigned* d_words = nullptr;  // [0] error bits, [1] general vote chunk counter, [2..31] column-walk counters
    DevBuf jobs, offs, feat, work, img, counts, norm, featout, maps;
    DevBuf slide_tab;             // fixed-point tables of the incremental window kernel
    bool slide_tab_ready = false;
    DevBuf hb_img, hb_out;        // host-buffer batches: staged images, device results
    std::vector<std::array<DevBuf, 3>> hb_tab;  // host-buffer batches: tables per group
    void* h_stage = nullptr;      // pinned table staging
    size_t h_stage_cap = 0;
    cudaEvent_t ev_stage = nullptr;
    std::vector<cudaEvent_t> stripe_events;
    std::string err;
    bool timing = false;
    std::vector<TimedPair> pool, pending;
    double vote_ms = 0;
    long long vote_launches = 0, kernel_launches = 0;
    std::map<long long, VoteCfg> overrides;
    std::unordered_map<std::string, GraphEntry> graphs;
};

namespace {

int fail(glcm_ctx* c, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(glcm_ctx* c, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, GLCM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)            \
    do {                     \
        int r_ = (expr);     \
        if (r_ != GLCM_OK)   \
            return r_;       \
    } while (0)

bool fault_injected(const char* what)
{
    const char* f = getenv("GLCM_FAULT");
    return f && strcmp(f, what) == 0;
}

int ensure(glcm_ctx* ctx, DevBuf& b, size_t bytes)
{
    if (bytes == 0)
        bytes = 16;
    if (b.cap >= bytes)
        return GLCM_OK;
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    want = (want + 255) & ~(size_t)255;
    if (fault_injected("alloc") || ctx->used - b.cap + want > ctx->budget) {
        if (!fault_injected("alloc") && ctx->used - b.cap + bytes <= ctx->budget)
            want = (bytes + 255) & ~(size_t)255;
        else
            return fail(ctx, GLCM_ERR_NOMEM, "device scratch of %zu bytes exceeds the budget (%zu of %zu used)",
                        bytes, ctx->used, ctx->budget);
    }
    if (b.p) {
        cudaStreamSynchronize(ctx->stream);
        if (ctx->side_stream)
            cudaStreamSynchronize(ctx->side_stream);
        if (ctx->epi_stream)
            cudaStreamSynchronize(ctx->epi_stream);
        for (cudaStream_t cs : ctx->cls_stream)
            if (cs)
                cudaStreamSynchronize(cs);
        cudaFree(b.p);
        ctx->used -= b.cap;
        b.p = nullptr;
        b.cap = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GLCM_ERR_NOMEM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    b.cap = want;
    ctx->used += want;
    return GLCM_OK;
}

int ensure_stage(glcm_ctx* ctx, size_t bytes)
{
    if (ctx->h_stage_cap >= bytes)
        return GLCM_OK;
    if (ctx->h_stage) {
        cudaEventSynchronize(ctx->ev_stage);
        cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        ctx->h_stage_cap = 0;
    }
    size_t want = std::max<size_t>(bytes, 1 << 16);
    if (cudaMallocHost(&ctx->h_stage, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, GLCM_ERR_NOMEM, "cudaMallocHost(%zu) failed", want);
    }
    ctx->h_stage_cap = want;
    return GLCM_OK;
}

bool is_device_ptr(const void* p)
{
    if (!p)
        return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int ilog2_exact(int n)
{
    for (int k = 0; k < 31; ++k)
        if ((1 << k) == n)
            return k;
    return -1;
}

long long cfg_key(int levels, int n_off, int bpp)
{
    return ((long long)levels << 20) | ((long long)n_off << 4) | bpp;
}

// Staged tiles: at most kTileRows rows (anchor band + dy halo) of
// vote_row_bytes() bytes each, two buffers per CTA.  64 anchor rows per item
// (4 per warp at 512 threads) were measured 3-5 % faster than 32 at every N;
// the histogram budget left (about 35 K words) still holds N = 256 packed.
constexpr int kTileRows = 80;
constexpr int kDefaultBand = 64;

int hist_budget_words(const glcm_ctx* ctx)
{
    // Leave room for the two tile buffers, static shared memory and the
    // per-block reservation.
    return (ctx->smem_optin - 2 * kTileRows * vote_row_bytes() - 4096) / 4;
}

// Offsets per histogram group, words per bin row of a group, and bin rows
// per anchor level (layout 3 packs partner levels j and j + ceil(N/2)).
int group_offsets(int layout) { return layout == 0 || layout == 3 ? 1 : 2; }
long long group_row_words(int layout, int rshift) { return (layout == 1 ? 2ll : 1ll) << rshift; }
long long level_rows(int layout, int levels) { return layout == 3 ? (levels + 1) / 2 : levels; }

// How one image's offsets are split into jobs for a configuration: groups per
// job, and anchor-level span per job (span < N splits the levels).
struct JobShape {
    int groups_per_job = 1, span = 0, jobs = 0;
};

JobShape job_shape(const glcm_ctx* ctx, int levels, int n_off, int layout, int rshift)
{
    JobShape s;
    const long long budget = hist_budget_words(ctx);
    const long long wrow = group_row_words(layout, rshift);
    const int opg = group_offsets(layout);
    const int groups = (n_off + opg - 1) / opg;
    const long long per_level = level_rows(layout, levels) * wrow;
    const long long per_group = (long long)levels * per_level;
    if (per_group <= budget) {
        s.groups_per_job = (int)std::min<long long>(groups, budget / per_group);
        s.span = levels;
        s.jobs = (groups + s.groups_per_job - 1) / s.groups_per_job;
    } else {
        s.groups_per_job = 1;
        s.span = (int)(budget / per_level);
        if (s.span < 1)
            return JobShape{1, 0, 0};
        s.jobs = groups * ((levels + s.span - 1) / s.span);
    }
    return s;
}

// Default vote configuration (used when the autotuner has not set one for a
// class) from a cost model in units of one conflict-free shared-memory
// reduction per pixel, calibrated on timing probes of the kernel: every pass
// over the image costs ~2 (tile staging and anchor levels); every offset voted
// in a pass ~1.5 (partner words and dispatch) plus the bank-conflict factor of
// the copy count (32 interleaved copies never conflict; a single copy costs
// ~2x over the benchmark's image mix) plus ~1.5 for packed halves (layout 3, more arithmetic
// per vote) or ~2 for two offsets in 16-bit halves (layout 2: merges every
// few rows, no constant increment for the upper halves).  A level-split job
// votes all its offsets in every part.
VoteCfg default_cfg(const glcm_ctx* ctx, int levels, int n_off)
{
    static const double conflict[6] = {2.2, 2.0, 1.8, 1.6, 1.4, 1.0};  // by log2 copies
    VoteCfg best;
    double best_cost = 1e30;
    for (int r = 5; r >= 0; --r) {
        for (int layout : {1, 0, 2, 3}) {
            if (layout == 2 && 65535ll * (1 << r) / (16ll * 512) < 64)
                continue;  // 16-bit halves would force a merge every few rows
            const JobShape s = job_shape(ctx, levels, n_off, layout, r);
            if (s.jobs <= 0)
                continue;
            const int parts = (levels + s.span - 1) / s.span;
            const double per_off = 1.5 + conflict[r] + (layout == 3 ? 1.5 : 0.0) + (layout == 2 ? 2.0 : 0.0);
            const double cost = 2.0 * s.jobs + (double)n_off * parts * per_off;
            if (cost < best_cost - 1e-9) {
                best_cost = cost;
                best.rshift = r;
                best.layout = layout;
            }
        }
    }
    return best;
}

VoteCfg get_cfg(const glcm_ctx* ctx, int levels, int n_off, int bpp)
{
    auto it = ctx->overrides.find(cfg_key(levels, n_off, bpp));
    if (it != ctx->overrides.end())
        return it->second;
    return default_cfg(ctx, levels, n_off);
}

struct ImageSpec {
    const uint8_t* img;  // device
    long long pitch;
    int W, H, bpp, levels, levels_mode;
    const glcm_offset* offsets;
    int n_off;
    uint32_t* out;       // device counts, n_off*N*N
    int y_begin, y_end;  // anchor rows of this launch
    int flat = 0;        // GLCM_FLAT_WRAP: also the pairs across row ends
};

// Append the jobs of one image to a plan.  Jobs run in the order
// (superband, offset group, level part): when an image needs several passes
// each pass re-reads at most one superband (<= 24 MB), which stays in L2.
int plan_image_general(glcm_ctx* ctx, const ImageSpec& s, VotePlan& plan, const std::vector<int>& idx)
{
    const int n_gen = (int)idx.size();
    if (n_gen == 0)
        return GLCM_OK;
    VoteCfg cfg = get_cfg(ctx, s.levels, s.n_off, s.bpp);
    if (cfg.layout == 4)
        cfg = default_cfg(ctx, s.levels, n_gen);
    const int T = std::max(plan.threads, cfg.threads);
    plan.threads = T;
    plan.bpp = s.bpp;
    const int nwarps = T / 32;
    const int PX = 16 / s.bpp;
    const JobShape shape = job_shape(ctx, s.levels, n_gen, cfg.layout, cfg.rshift);
    if (shape.jobs <= 0)
        return fail(ctx, GLCM_ERR_ARG, "vote config cannot hold one level row of the histogram");
    // Offsets sorted by dy so a partner row is loaded once per distinct dy.
    std::vector<int> order(idx);
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return s.offsets[a].dy < s.offsets[b].dy; });
    const int opg = group_offsets(cfg.layout);
    const int per_job = shape.groups_per_job * opg;
    const int rows = s.y_end - s.y_begin;
    const int strip_px = 32 * PX;
    const int n_strips = std::max(1, (s.W + strip_px - 1) / strip_px);
    // Default band: 64 anchor rows, or 32 when that leaves a small image fewer
    // than 16 items (a 512 x 512 image would run on 8 CTAs).
    int band = cfg.band_rows > 0 ? cfg.band_rows : kDefaultBand;
    if (cfg.band_rows <= 0 && (long long)n_strips * ((rows + band - 1) / band) < 16)
        band = kDefaultBand / 2;
    band = std::min(band, kTileRows - kMaxDySpan);
    if (cfg.layout == 2) {
        // votes per 16-bit half per item: ceil(band/nwarps) * PX * (T / R) <= 65535
        const long long max_rows_per_warp = 65535ll * (1 << cfg.rshift) / ((long long)PX * T);
        if (max_rows_per_warp < 1)
            return fail(ctx, GLCM_ERR_ARG, "vote config cannot bound 16-bit counters");
        band = (int)std::min<long long>(band, max_rows_per_warp * nwarps);
    }
    if (cfg.layout == 3) {
        // An item must fit between two spills: 49152 votes per half, PX per
        // anchor row of each lane sharing a copy.
        const long long rows_spill = 49152ll * (1 << cfg.rshift) / (32ll * PX);
        band = (int)std::min<long long>(band, rows_spill);
    }
    band = std::max(1, band);
    // Superbands only when the image takes several passes.
    const int passes = ((n_gen + per_job - 1) / per_job) * ((s.levels + shape.span - 1) / shape.span);
    int sb_rows = rows;
    if (passes > 1) {
        const long long row_bytes = (long long)s.W * s.bpp;
        const long long want = std::max<long long>(band, (24ll << 20) / std::max<long long>(1, row_bytes));
        sb_rows = (int)std::min<long long>(rows, ((want + band - 1) / band) * band);
    }
    for (int sb0 = s.y_begin; sb0 < s.y_end; sb0 += sb_rows) {
        const int sb1 = std::min(s.y_end, sb0 + sb_rows);
        const int n_bands = (sb1 - sb0 + band - 1) / band;
        for (int o0 = 0; o0 < n_gen;) {
            // Up to per_job consecutive offsets (sorted by dy) whose dy range,
            // with 0, spans at most kMaxDySpan rows; a lone wider offset is
            // voted unstaged.
            int cnt = 1;
            int dmin = std::min(0, s.offsets[order[o0]].dy), dmax = std::max(0, s.offsets[order[o0]].dy);
            while (o0 + cnt < n_gen && cnt < per_job) {
                const int d = s.offsets[order[o0 + cnt]].dy;
                const int nmin = std::min(dmin, d), nmax = std::max(dmax, d);
                if (nmax - nmin > kMaxDySpan && dmax - dmin <= kMaxDySpan)
                    break;
                dmin = nmin;
                dmax = nmax;
                ++cnt;
            }
            for (int lv = 0; lv < s.levels; lv += shape.span) {
                const int span = std::min(shape.span, s.levels - lv);
                VoteJob j{};
                j.img = s.img;
                j.pitch = s.pitch;
                j.W = s.W;
                j.H = s.H;
                j.bpp = s.bpp;
                j.levels = s.levels;
                j.log2n = ilog2_exact(s.levels);
                j.levels_mode = s.levels_mode;
                j.aligned = ((reinterpret_cast<uintptr_t>(s.img) | (uintptr_t)s.pitch) & 15) == 0;
                j.n_off = cnt;
                j.off0 = (int)plan.offs.size();
                j.rshift = cfg.rshift;
                j.layout = cfg.layout;
                j.lv_lo = lv;
                j.lv_span = span;
                j.bytecode = (cfg.layout == 1 && cfg.rshift == 5 && span == s.levels && j.log2n >= 0 &&
                              s.levels <= 16)
                                 ? 1
                                 : 0;
                const int groups = (cnt + opg - 1) / opg;
                j.hist_words = (int)((long long)groups * span * level_rows(cfg.layout, s.levels) *
                                     group_row_words(cfg.layout, cfg.rshift));
                j.item0 = plan.n_items;
                j.n_job_items = n_strips * n_bands;
                // Weight of an item: pixel loads plus expected votes (offsets x
                // the share of anchor levels this job counts).
                {
                    // Chunk = enough items that their votes are ~10x the merge
                    // (reading and clearing the job's shared histograms).
                    const double votes_per_item = (double)band * strip_px * cnt * span / s.levels;
                    const double merge = 2.0 * j.hist_words + 64.0;
                    const double want = std::ceil(10.0 * merge / std::max(1.0, votes_per_item));
                    j.chunk_items = (int)std::max(1.0, std::min<double>(n_strips * n_bands, want));
                }
                j.n_strips = n_strips;
                j.band_rows = band;
                j.y_begin = sb0;
                j.y_end = sb1;
                j.dy_min = dmin;
                j.dy_max = dmax;
                j.staged = (dmax - dmin <= kMaxDySpan) ? 1 : 0;
                j.out = s.out;
                if (j.staged)
                    plan.tile_rows = std::max(plan.tile_rows, band + dmax - dmin);
                for (int k = o0; k < o0 + cnt; ++k) {
                    VoteOffset vo{};
                    vo.dx = s.offsets[order[k]].dx;
                    vo.dy = s.offsets[order[k]].dy;
                    vo.slot = order[k];
                    plan.offs.push_back(vo);
                }
                plan.max_hist_words = std::max(plan.max_hist_words, j.hist_words);
                plan.n_items += n_strips * n_bands;
                if (n_strips * n_bands > 0)
                    plan.jobs.push_back(j);
                else
                    plan.offs.resize(j.off0);
            }
            o0 += cnt;
        }
    }
    return GLCM_OK;
}


// Canonical offset (0: (1, 0), 1: (1, -1), 2: (0, -1), 3: (-1, -1)) of an
// offset at chessboard distance 1 and whether it is the opposite one (its
// counts are the canonical counts transposed); -1 for any other offset.
// Canonical offset of the column walk: (D, 0) -> 0, (D, -D) -> 1, (0, -D) -> 2,
// (-D, -D) -> 3 at a distance D of 1 .. 4, or the opposite of one (its
// counts are the transpose); -1 for any other offset.  dist: D.
int canonical_fast(int dx, int dy, int& dist, bool& transposed)
{
    transposed = false;
    dist = std::max(std::abs(dx), std::abs(dy));
    if (dist < 1 || dist > 4 || (dx != 0 && std::abs(dx) != dist) || (dy != 0 && std::abs(dy) != dist))
        return -1;
    if (dy > 0 || (dy == 0 && dx < 0)) {
        dx = -dx;
        dy = -dy;
        transposed = true;
    }
    if (dy == 0)
        return 0;
    return dx == dist ? 1 : (dx == 0 ? 2 : 3);
}

FastClass& fast_class(VotePlan& plan, int bpp, int log2n, bool aligned)
{
    for (FastClass& c : plan.fast)
        if (c.bpp == bpp && c.log2n == log2n && c.aligned == aligned)
            return c;
    plan.fast.emplace_back();
    plan.fast.back().bpp = bpp;
    plan.fast.back().log2n = log2n;
    plan.fast.back().aligned = aligned;
    return plan.fast.back();
}

// CTAs of a vote launch: every SM but the context's reserve (left to a
// concurrent copy kernel), and at most max_ctas when that is given.
int launch_ctas(const glcm_ctx* ctx, int max_ctas = 0)
{
    int c = std::max(1, ctx->sm_count - ctx->sm_reserve);
    if (max_ctas > 0)
        c = std::min(c, max_ctas);
    return std::max(1, c);
}

// SMs the later groups of a host-buffer batch leave to the expensive
// epilogues of its first groups (n_glcm GLCMs) while they vote.  (A device
// batch's light part votes on every SM: its heavy epilogue is launched
// first and takes its SMs before the light CTAs queue for them.)
int split_reserve(const glcm_ctx* ctx, int n_glcm)
{
    return std::min(n_glcm, ctx->sm_count / 4);
}

// Items per chunk of the column-walk kernel: one per warp of a CTA.
constexpr int kFastChunkItems = 16;

// Column-walk jobs of one image for the canonical offsets in `present`
// (slot / slot_t: the output GLCMs of each canonical offset as counted and
// transposed).  Items and chunks are made by finalize_fast; a band height
// configured for the class (the autotuner's tile shape) is kept.
void plan_image_fast(const glcm_ctx* ctx, const ImageSpec& s, VotePlan& plan, int dist, int present,
                     const int (&slot)[4], const int (&slot_t)[4])
{
    int band_override = 0;
    {
        auto it = ctx->overrides.find(cfg_key(s.levels, s.n_off, s.bpp));
        if (it != ctx->overrides.end() && it->second.layout == 4)
            band_override = std::min(it->second.band_rows, 1024);
    }
    const int log2n = ilog2_exact(s.levels);
    const bool aligned = ((reinterpret_cast<uintptr_t>(s.img) | (uintptr_t)s.pitch) & 15) == 0;
    FastClass& fc = fast_class(plan, s.bpp, log2n, aligned);
    const int PX = 16 / s.bpp;
    const int n_strips = (s.W + 32 * PX - 1) / (32 * PX);
    if (s.y_end <= s.y_begin || n_strips <= 0)
        return;
    struct Group {
        int mode, present, half_hi, row_half, transposed, slot;
    };
    std::vector<Group> groups;
    if (log2n == 8) {
        // N = 256: one job per offset, orientation and half of the GLCM's rows.
        for (int k = 0; k < 4; ++k)
            for (int t = 0; t < 2; ++t) {
                const int sl = t ? slot_t[k] : slot[k];
                if (sl >= 0)
                    for (int h = 0; h < 2; ++h)
                        groups.push_back({kFastWide, 1 << k, -1, h, t, sl});
            }
    } else if (log2n <= 3 && present == 15) {
        groups.push_back({kFastJoint, 15, -1, 0, 0, -1});
    } else if (log2n <= 4) {
        groups.push_back({kFastPair, present, -1, 0, 0, -1});
    } else {
        int pending = -1;
        for (int k = 0; k < 4; ++k) {
            if (!((present >> k) & 1))
                continue;
            if (pending < 0) {
                pending = k;
            } else {
                groups.push_back({kFastHalf, (1 << pending) | (1 << k), k, 0, 0, -1});
                pending = -1;
            }
        }
        if (pending >= 0)
            groups.push_back({kFastHalf, 1 << pending, -1, 0, 0, -1});
    }
    for (const Group& g : groups) {
        FastJob j{};
        j.img = s.img;
        j.pitch = s.pitch;
        j.W = s.W;
        j.H = s.H;
        j.bpp = s.bpp;
        j.log2n = log2n;
        j.mode = g.mode;
        j.present = g.present;
        j.half_hi = g.half_hi;
        j.row_half = g.row_half;
        j.transposed = g.transposed;
        j.aligned = aligned ? 1 : 0;
        for (int k = 0; k < 4; ++k) {
            const bool in = (g.present >> k) & 1;
            j.slot[k] = in ? (g.mode == kFastWide ? g.slot : slot[k]) : -1;
            j.slot_t[k] = in && g.mode != kFastWide ? slot_t[k] : -1;
        }
        j.hist_words = vote_fast_hist_words(log2n, g.mode);
        j.n_strips = n_strips;
        j.band = band_override;  // 0: set by finalize_fast
        j.y_begin = s.y_begin;
        j.y_end = s.y_end;
        j.dist = dist;
        j.out = s.out;
        fc.max_hist_words = std::max(fc.max_hist_words, j.hist_words);
        fc.max_dist = std::max(fc.max_dist, dist);
        fc.jobs.push_back(j);
    }
}

// Bands, items and chunks of every column-walk class of a plan.  One band
// height per class (4..64 rows), chosen for the shortest launch on `ctas`
// CTAs: with c(b) chunks of kFastChunkItems items (one item per warp, chunks
// never span jobs) a CTA takes ceil(c(b) / ctas) chunks, each costing about
// b rows plus the row above the band and the item's start, so b minimizes
// ceil(c(b) / ctas) * (b + kItemRowsExtra).  (Rounding b up from rows per
// warp can leave one chunk more than CTAs, and one CTA twice the work.)
constexpr int kItemRowsExtra = 3;

void finalize_fast(VotePlan& plan, int ctas)
{
    ctas = std::max(1, ctas);
    for (FastClass& fc : plan.fast) {
        auto chunks_for = [&](int b) {
            long long c = 0;
            for (const FastJob& j : fc.jobs) {
                const int bj = j.band > 0 ? j.band : b;
                const long long items = (long long)j.n_strips * ((j.y_end - j.y_begin + bj - 1) / bj);
                c += (items + kFastChunkItems - 1) / kFastChunkItems;
            }
            return c;
        };
        int band = 64;
        long long best = -1;
        for (int b = 4; b <= 64; ++b) {
            const long long per_cta = (chunks_for(b) + ctas - 1) / ctas;
            const long long cost = per_cta * (b + kItemRowsExtra);
            if (best < 0 || cost < best) {
                best = cost;
                band = b;
            }
        }
        fc.n_items = 0;
        fc.chunks.clear();
        for (int jb = 0; jb < (int)fc.jobs.size(); ++jb) {
            FastJob& j = fc.jobs[jb];
            if (j.band <= 0)
                j.band = band;
            j.item0 = fc.n_items;
            j.n_items = j.n_strips * ((j.y_end - j.y_begin + j.band - 1) / j.band);
            for (int i = 0; i < j.n_items; i += kFastChunkItems)
                fc.chunks.push_back(make_int3(jb, j.item0 + i, j.item0 + std::min(j.n_items, i + kFastChunkItems)));
            fc.n_items += j.n_items;
        }
    }
}

// Append the jobs of one image to a plan: offsets at chessboard distance 1 of
// a uint8/uint16 image with N in {2, 4, 8, 16, 32, 256} (levels quantized
// here, not given) go to the column-walk kernel unless the autotuner chose a
// general layout for the class; the others to the general vote kernel.
int plan_image(glcm_ctx* ctx, const ImageSpec& s, VotePlan& plan, int target_items)
{
    if (s.levels > GLCM_MAX_LEVELS) {
        // N > 256: every offset votes into global counts (vote_global.cu).
        const long long nn = (long long)s.levels * s.levels;
        for (int k = 0; k < s.n_off; ++k) {
            const SeamJob g{s.img, s.pitch, s.W, s.H, s.bpp, s.levels, s.levels_mode,
                            s.offsets[k].dx, s.offsets[k].dy, s.y_begin, s.y_end, s.out + k * nn};
            plan.globals.push_back(g);
            if (s.flat && s.offsets[k].dx != 0)
                plan.seams.push_back(g);
        }
        return GLCM_OK;
    }
    const int log2n = ilog2_exact(s.levels);
    const bool aligned = ((reinterpret_cast<uintptr_t>(s.img) | (uintptr_t)s.pitch) & 15) == 0;
    auto it = ctx->overrides.find(cfg_key(s.levels, s.n_off, s.bpp));
    const bool tuned_general = it != ctx->overrides.end() && it->second.layout != 4;
    // N = 256 merges by bulk reductions into the output rows: 16-byte aligned counts.
    const bool out_aligned = (reinterpret_cast<uintptr_t>(s.out) & 15) == 0;
    const bool eligible = !tuned_general && ((log2n >= 1 && log2n <= 5) || (log2n == 8 && out_aligned)) &&
                          !s.levels_mode && s.y_end > s.y_begin;
    (void)aligned;  // rows at any byte address are realigned by the kernel
    std::vector<int> gen;
    // Column-walk offsets grouped by distance D (index D - 1): one set of
    // jobs per distance.
    int present[4] = {0, 0, 0, 0};
    int slot[4][4], slot_t[4][4];
    for (int d = 0; d < 4; ++d)
        for (int c = 0; c < 4; ++c)
            slot[d][c] = slot_t[d][c] = -1;
    for (int k = 0; k < s.n_off; ++k) {
        bool tr = false;
        int dist = 0;
        const int c = eligible ? canonical_fast(s.offsets[k].dx, s.offsets[k].dy, dist, tr) : -1;
        int* dst = c < 0 ? nullptr : (tr ? &slot_t[dist - 1][c] : &slot[dist - 1][c]);
        if (dst && *dst < 0) {
            *dst = k;
            present[dist - 1] |= 1 << c;
        } else {
            gen.push_back(k);  // any other offset, or a repeat of one already placed
        }
    }
    (void)target_items;
    for (int d = 0; d < 4; ++d)
        if (present[d])
            plan_image_fast(ctx, s, plan, d + 1, present[d], slot[d], slot_t[d]);
    if (s.flat) {
        // Flat-wrap: the pairs whose partner column leaves [0, W), added after the votes.
        const long long nn = (long long)s.levels * s.levels;
        for (int k = 0; k < s.n_off; ++k)
            if (s.offsets[k].dx != 0)
                plan.seams.push_back(SeamJob{s.img, s.pitch, s.W, s.H, s.bpp, s.levels, s.levels_mode,
                                             s.offsets[k].dx, s.offsets[k].dy, s.y_begin, s.y_end,
                                             s.out + k * nn});
    }
    return plan_image_general(ctx, s, plan, gen);
}

int check_image_args(glcm_ctx* ctx, const void* image, int width, int height, size_t pitch, int dtype,
                     int levels, const glcm_offset* offsets, int n_offsets)
{
    if (!image)
        return fail(ctx, GLCM_ERR_ARG, "image is NULL");
    if (width < 1 || height < 1)
        return fail(ctx, GLCM_ERR_ARG, "width and height must be >= 1 (got %d x %d)", width, height);
    if (dtype != GLCM_U8 && dtype != GLCM_U16)
        return fail(ctx, GLCM_ERR_ARG, "dtype must be GLCM_U8 or GLCM_U16");
    const int bpp = dtype == GLCM_U8 ? 1 : 2;
    if (pitch < (size_t)width * bpp)
        return fail(ctx, GLCM_ERR_ARG, "pitch_bytes %zu < width * %d", pitch, bpp);
    if (levels > GLCM_MAX_COUNT_LEVELS)
        return fail(ctx, GLCM_ERR_UNSUPPORTED, "levels %d > %d", levels, GLCM_MAX_COUNT_LEVELS);
    if (levels < 2)
        return fail(ctx, GLCM_ERR_ARG, "levels must be in 2..256 (got %d)", levels);
    if (!offsets || n_offsets < 1 || n_offsets > GLCM_MAX_OFFSETS)
        return fail(ctx, GLCM_ERR_ARG, "need 1..%d offsets (got %d)", GLCM_MAX_OFFSETS, n_offsets);
    for (int k = 0; k < n_offsets; ++k)
        if (offsets[k].dx <= -65536 || offsets[k].dx >= 65536 || offsets[k].dy <= -65536 || offsets[k].dy >= 65536)
            return fail(ctx, GLCM_ERR_ARG, "offset %d out of range", k);
    return GLCM_OK;
}

int target_items(const glcm_ctx* ctx)
{
    return ctx->sm_count * 4;
}

// Whether a plan needs the vote kernel instance with packed halves (layout 3).
bool plan_packed(const VotePlan& plan)
{
    for (const VoteJob& j : plan.jobs)
        if (j.layout == 3)
            return true;
    return false;
}

size_t vote_smem(const VotePlan& plan)
{
    return std::max<size_t>(16, 2 * (size_t)plan.tile_rows * vote_row_bytes() + (size_t)plan.max_hist_words * 4);
}

int grid_for(const glcm_ctx* ctx, const VotePlan& plan)
{
    const size_t smem = vote_smem(plan);
    const int per_sm = std::max(1, vote_blocks_per_sm(plan.bpp, plan.threads, smem, plan_packed(plan)));
    int ctas = std::max(1, ctx->sm_count - ctx->sm_reserve) * per_sm;
    if (plan.max_ctas > 0)
        ctas = std::min(ctas, plan.max_ctas * per_sm);
    return std::max(1, std::min((int)plan.chunks.size(), ctas));
}

// Split every job of a plan into chunks of chunk_items consecutive items,
// capped so that the launch has at least ~4 chunks per CTA to balance
// (measured against 1, 2, 3 and 6).
void build_chunks(VotePlan& plan, int ctas)
{
    plan.chunks.clear();
    const int cap = std::max(1, plan.n_items / std::max(1, 4 * ctas));
    for (int jb = 0; jb < (int)plan.jobs.size(); ++jb) {
        const VoteJob& j = plan.jobs[jb];
        const int cs = std::max(1, std::min(j.chunk_items, cap));
        for (int k = 0; k < j.n_job_items; k += cs)
            plan.chunks.push_back(make_int3(jb, j.item0 + k, j.item0 + std::min(j.n_job_items, k + cs)));
    }
}

// Upload a plan's tables into the given device buffers (through pinned staging).
// The chunk table follows the jobs in `djobs`, 16-byte aligned.
int upload_tables(glcm_ctx* ctx, const VotePlan& plan, const std::vector<FeatJob>& feats, DevBuf& djobs,
                  DevBuf& doffs, DevBuf& dfeat)
{
    const size_t bj0 = (plan.jobs.size() * sizeof(VoteJob) + 15) & ~(size_t)15;
    // Column-walk tables after the general chunks: every class's jobs back to
    // back (one array over all classes, which the zeroing kernel walks), then
    // every class's chunks.
    size_t bj = (bj0 + plan.chunks.size() * sizeof(int3) + 15) & ~(size_t)15;
    for (const FastClass& c : plan.fast) {
        const_cast<FastClass&>(c).jobs_off = bj;
        bj += c.jobs.size() * sizeof(FastJob);
    }
    bj = (bj + 15) & ~(size_t)15;
    for (const FastClass& c : plan.fast) {
        const_cast<FastClass&>(c).chunks_off = bj;
        bj += c.chunks.size() * sizeof(int3);
    }
    bj = (bj + 15) & ~(size_t)15;
    const_cast<VotePlan&>(plan).seams_off = bj;
    bj += plan.seams.size() * sizeof(SeamJob);
    bj = (bj + 15) & ~(size_t)15;
    const_cast<VotePlan&>(plan).globals_off = bj;
    bj += plan.globals.size() * sizeof(SeamJob);
    const size_t bo = plan.offs.size() * sizeof(VoteOffset);
    const size_t bf = feats.size() * sizeof(FeatJob);
    TRY(ensure(ctx, djobs, bj));
    TRY(ensure(ctx, doffs, bo));
    TRY(ensure(ctx, dfeat, bf));
    const size_t total = ((bj + 255) & ~(size_t)255) + ((bo + 255) & ~(size_t)255) + bf;
    cudaEventSynchronize(ctx->ev_stage);
    TRY(ensure_stage(ctx, total));
    uint8_t* h = static_cast<uint8_t*>(ctx->h_stage);
    const size_t oo = (bj + 255) & ~(size_t)255;
    const size_t of = oo + ((bo + 255) & ~(size_t)255);
    if (!plan.jobs.empty())
        memcpy(h, plan.jobs.data(), plan.jobs.size() * sizeof(VoteJob));
    if (!plan.chunks.empty())
        memcpy(h + bj0, plan.chunks.data(), plan.chunks.size() * sizeof(int3));
    const_cast<VotePlan&>(plan).chunk_off = bj0;
    for (const FastClass& c : plan.fast) {
        if (!c.jobs.empty())
            memcpy(h + c.jobs_off, c.jobs.data(), c.jobs.size() * sizeof(FastJob));
        if (!c.chunks.empty())
            memcpy(h + c.chunks_off, c.chunks.data(), c.chunks.size() * sizeof(int3));
    }
    if (!plan.seams.empty())
        memcpy(h + plan.seams_off, plan.seams.data(), plan.seams.size() * sizeof(SeamJob));
    if (!plan.globals.empty())
        memcpy(h + plan.globals_off, plan.globals.data(), plan.globals.size() * sizeof(SeamJob));
    if (bo)
        memcpy(h + oo, plan.offs.data(), bo);
    if (bf)
        memcpy(h + of, feats.data(), bf);
    if (bj)
        CK(cudaMemcpyAsync(djobs.p, h, bj, cudaMemcpyHostToDevice, ctx->stream));
    if (bo)
        CK(cudaMemcpyAsync(doffs.p, h + oo, bo, cudaMemcpyHostToDevice, ctx->stream));
    if (bf)
        CK(cudaMemcpyAsync(dfeat.p, h + of, bf, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaEventRecord(ctx->ev_stage, ctx->stream));
    return GLCM_OK;
}

// Zero the jobs' output GLCMs and the vote kernel's chunk counter.  (A kernel
// rather than memsets: on the copy engines a memset would queue behind the
// image copies of a host-buffer batch.)
__global__ void k_clear_word(unsigned* w) { *w = 0u; }

__global__ void k_zero_words(uint32_t* p, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        p[k] = 0u;
}

// Zero n words on `st` with a kernel (see k_zero_job_outputs for why).
int zero_words(glcm_ctx* ctx, uint32_t* p, long long n, cudaStream_t st)
{
    const int grid = (int)std::min<long long>(std::max<long long>(1, (n + 255) / 256), 4ll * ctx->sm_count);
    k_zero_words<<<grid, 256, 0, st>>>(p, n);
    CK(cudaGetLastError());
    ctx->kernel_launches += 1;
    return GLCM_OK;
}

// Chunk counters in the context's device words: [1] the general vote kernel,
// [2 + c] column-walk class c.
constexpr int kCounterWords = 32;  // the context's 128 bytes of device words
constexpr int kMaxFastClasses = kCounterWords - 2;

// Blocks x in [0, n_gen) zero general job x's outputs, blocks x in [n_gen,
// n_gen + n_fast) the outputs of column-walk job x - n_gen, each in
// kZeroSlices slices (blockIdx.y); an N = 256 job zeroes only the 128 rows it
// counts (its twin job for the other half zeroes the rest).  Block (0, 0)
// also clears the chunk counters.
constexpr int kZeroSlices = 8;

__device__ __forceinline__ void zero_slice(uint32_t* dst, long long n)
{
    const long long per = (n + kZeroSlices - 1) / kZeroSlices;
    const long long lo = per * blockIdx.y, hi = lo + per < n ? lo + per : n;
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x)
        dst[e] = 0u;
}

__global__ void k_zero_job_outputs(const VoteJob* jobs, int n_gen, const VoteOffset* offs, const FastJob* fjobs,
                                   unsigned* counters)
{
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x < kCounterWords - 1)
        counters[threadIdx.x] = 0u;
    if ((int)blockIdx.x < n_gen) {
        const VoteJob j = jobs[blockIdx.x];
        const long long NN = (long long)j.levels * j.levels;
        for (int o = 0; o < j.n_off; ++o)
            zero_slice(j.out + offs[j.off0 + o].slot * NN, NN);
        return;
    }
    const FastJob& f = fjobs[blockIdx.x - n_gen];
    const long long NN = 1ll << (2 * f.log2n);
    for (int k = 0; k < kFastOffsets; ++k)
        for (int t = 0; t < 2; ++t) {
            const int sl = t ? f.slot_t[k] : f.slot[k];
            if (sl < 0)
                continue;
            if (f.mode == kFastWide)
                zero_slice(f.out + sl * NN + (long long)f.row_half * (NN / 2), NN / 2);
            else
                zero_slice(f.out + sl * NN, NN);
        }
}

// Zero the N x N counts of every N > 256 job (blockIdx.y: the job).
__global__ void k_zero_global_outputs(const SeamJob* jobs)
{
    const SeamJob j = jobs[blockIdx.y];
    const long long nn = (long long)j.levels * j.levels;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x)
        j.out[e] = 0u;
}

__global__ void k_clear_counters(unsigned* counters)
{
    if (threadIdx.x < kCounterWords - 1)
        counters[threadIdx.x] = 0u;
}

TimedPair take_pair(glcm_ctx* ctx)
{
    if (ctx->pool.empty()) {
        TimedPair p;
        cudaEventCreate(&p.a);
        cudaEventCreate(&p.b);
        return p;
    }
    TimedPair p = ctx->pool.back();
    ctx->pool.pop_back();
    return p;
}

// Enqueue zero (optional) + vote for a plan whose tables are at djobs/doffs.
// Column-walk classes of a vote launch group voted side by side: group g
// (one number of levels) on ctx->cls_stream[g], largest first; used ==
// false when everything votes on one stream.
struct ClassStreams {
    bool used = false;
    int n = 0;
    int levels[4] = {0, 0, 0, 0};
};

// Groups of a plan's column-walk classes by number of levels, the most
// work first (pixels walked, one walk per job; then the larger N, whose
// votes and epilogue cost more), so that the cheapest class's votes and
// epilogue end the launch; false when the plan votes anything else or has
// more than four numbers of levels.
bool class_groups(const VotePlan& plan, ClassStreams& cs, std::vector<int>& group_of)
{
    if (!plan.jobs.empty() || !plan.globals.empty() || !plan.seams.empty() || plan.fast.size() < 2)
        return false;
    std::vector<std::pair<long long, int>> work;  // (work, levels)
    for (const FastClass& c : plan.fast) {
        long long w = 0;
        for (const FastJob& j : c.jobs)
            w += (long long)j.W * (j.y_end - j.y_begin);
        w = w * 512 + c.log2n;  // ties: the larger N first
        const int lv = 1 << c.log2n;
        auto it = std::find_if(work.begin(), work.end(), [&](const std::pair<long long, int>& x) { return x.second == lv; });
        if (it == work.end())
            work.push_back({w, lv});
        else
            it->first += w;
    }
    if (work.size() < 2 || work.size() > 4)
        return false;
    std::stable_sort(work.begin(), work.end(),
                     [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) { return a.first > b.first; });
    cs.n = (int)work.size();
    for (int g = 0; g < cs.n; ++g)
        cs.levels[g] = work[g].second;
    group_of.assign(plan.fast.size(), 0);
    for (size_t ci = 0; ci < plan.fast.size(); ++ci)
        for (int g = 0; g < cs.n; ++g)
            if (cs.levels[g] == 1 << plan.fast[ci].log2n)
                group_of[ci] = g;
    return true;
}

int enqueue_vote(glcm_ctx* ctx, const VotePlan& plan, const DevBuf& djobs, const DevBuf& doffs, const int3* dchunks,
                 bool zero, bool capturing, GraphEntry* ge, cudaStream_t st = nullptr, ClassStreams* cs = nullptr)
{
    if (plan_empty(plan))
        return GLCM_OK;
    if (!st)
        st = ctx->stream;
    if ((int)plan.fast.size() > kMaxFastClasses)
        return fail(ctx, GLCM_ERR_UNSUPPORTED, "more column-walk classes than chunk counters");
    int n_fast_jobs = 0;
    for (const FastClass& c : plan.fast)
        n_fast_jobs += (int)c.jobs.size();
    const FastJob* fjobs0 =
        plan.fast.empty() ? nullptr
                          : reinterpret_cast<const FastJob*>(static_cast<uint8_t*>(djobs.p) + plan.fast[0].jobs_off);
    const SeamJob* gjobs =
        plan.globals.empty() ? nullptr
                             : reinterpret_cast<const SeamJob*>(static_cast<uint8_t*>(djobs.p) + plan.globals_off);
    if (zero && !plan.globals.empty()) {
        for (size_t g0 = 0; g0 < plan.globals.size(); g0 += 65535) {
            const int ng = (int)std::min<size_t>(65535, plan.globals.size() - g0);
            k_zero_global_outputs<<<dim3(64, ng), 256, 0, st>>>(gjobs + g0);
            CK(cudaGetLastError());
            ctx->kernel_launches += capturing ? 0 : 1;
            if (ge)
                ge->n_kernels++;
        }
    }
    if (zero && plan.jobs.empty() && plan.fast.empty()) {
        k_clear_counters<<<1, 32, 0, st>>>(ctx->d_words + 1);
    } else if (zero) {
        k_zero_job_outputs<<<dim3((int)plan.jobs.size() + n_fast_jobs, kZeroSlices), 256, 0, st>>>(
            static_cast<const VoteJob*>(djobs.p), (int)plan.jobs.size(), static_cast<const VoteOffset*>(doffs.p),
            fjobs0, ctx->d_words + 1);
    } else {
        k_clear_counters<<<1, 32, 0, st>>>(ctx->d_words + 1);
    }
    CK(cudaGetLastError());
    ctx->kernel_launches += capturing ? 0 : 1;
    if (ge)
        ge->n_kernels++;
    VoteParams vp{};
    vp.jobs = static_cast<const VoteJob*>(djobs.p);
    vp.n_jobs = (int)plan.jobs.size();
    vp.offs = static_cast<const VoteOffset*>(doffs.p);
    vp.n_items = plan.n_items;
    vp.chunks = dchunks;
    vp.n_chunks = (int)plan.chunks.size();
    vp.max_hist_words = plan.max_hist_words;
    vp.tile_bytes = plan.tile_rows * vote_row_bytes();
    vp.item_counter = ctx->d_words + 1;
    vp.err = ctx->d_words;
    const size_t smem = vote_smem(plan);
    const int grid = plan.jobs.empty() ? 1 : grid_for(ctx, plan);
    TimedPair tp{};
    const bool time_it = ctx->timing && !capturing;
    if (time_it) {
        tp = take_pair(ctx);
        CK(cudaEventRecord(tp.a, st));
    }
    int n_launch = 0;
    // Classes side by side: each group forks from the stream after the
    // zeroing; the stream then waits for every group's votes.
    std::vector<int> group_of;
    const bool par = cs && class_groups(plan, *cs, group_of);
    std::vector<size_t> order(plan.fast.size());
    for (size_t ci = 0; ci < order.size(); ++ci)
        order[ci] = ci;
    if (par) {
        cs->used = true;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return group_of[a] < group_of[b]; });
        CK(cudaEventRecord(ctx->ev_cls_fork, st));
        for (int g = 0; g < cs->n; ++g)
            CK(cudaStreamWaitEvent(ctx->cls_stream[g], ctx->ev_cls_fork, 0));
    }
    for (size_t ci : order) {
        const FastClass& c = plan.fast[ci];
        if (c.chunks.empty())
            continue;
        FastParams fp{};
        fp.jobs = reinterpret_cast<const FastJob*>(static_cast<uint8_t*>(djobs.p) + c.jobs_off);
        fp.chunks = reinterpret_cast<const int3*>(static_cast<uint8_t*>(djobs.p) + c.chunks_off);
        fp.n_chunks = (int)c.chunks.size();
        fp.max_hist_words = c.max_hist_words;
        fp.chunk_counter = ctx->d_words + 2 + ci;
        fp.err = ctx->d_words;
        fp.ring_words = c.max_dist > 1 ? c.max_dist * (4 / c.bpp + 1) * 32 : 0;
        const size_t fsmem = vote_fast_smem_bytes(c.max_hist_words, c.log2n, fp.ring_words);
        int ctas = std::max(1, ctx->sm_count - ctx->sm_reserve);
        if (plan.max_ctas > 0)
            ctas = std::min(ctas, plan.max_ctas);
        CK(launch_vote_fast(fp, c.bpp, c.log2n, c.aligned, std::max(1, std::min(fp.n_chunks, ctas)), fsmem,
                            par ? ctx->cls_stream[group_of[ci]] : st));
        ++n_launch;
    }
    if (par)
        for (int g = 0; g < cs->n; ++g) {
            CK(cudaEventRecord(ctx->ev_cls_vote[g], ctx->cls_stream[g]));
            CK(cudaStreamWaitEvent(st, ctx->ev_cls_vote[g], 0));
        }
    if (!plan.jobs.empty()) {
        CK(launch_vote(vp, plan.bpp, grid, plan.threads, smem, st, plan_packed(plan)));
        ++n_launch;
    }
    if (!plan.globals.empty()) {
        long long most = 1;
        for (const SeamJob& gj : plan.globals)
            most = std::max<long long>(most, (long long)gj.W * (gj.y_end - gj.y_begin));
        const int bpj = (int)std::max<long long>(1, std::min<long long>(4ll * ctx->sm_count, (most + 8191) / 8192));
        CK(launch_vote_global(gjobs, (int)plan.globals.size(), bpj, ctx->d_words, st));
        ++n_launch;
    }
    if (!plan.seams.empty()) {
        long long most = 1;
        for (const SeamJob& sj : plan.seams)
            most = std::max<long long>(most, (long long)std::min(std::abs(sj.dx), sj.W) * (sj.y_end - sj.y_begin));
        const int bpj = (int)std::max<long long>(1, std::min<long long>(ctx->sm_count, (most + 4095) / 4096));
        const SeamJob* sjobs =
            reinterpret_cast<const SeamJob*>(static_cast<uint8_t*>(djobs.p) + plan.seams_off);
        CK(launch_seams(sjobs, (int)plan.seams.size(), bpj, ctx->d_words, st));
        if (!capturing)
            ctx->kernel_launches += 1;
        if (ge)
            ge->n_kernels++;
    }
    if (time_it) {
        CK(cudaEventRecord(tp.b, st));
        ctx->pending.push_back(tp);
    }
    if (!capturing) {
        ctx->kernel_launches += n_launch;
        ctx->vote_launches += n_launch;
    }
    if (ge) {
        ge->n_kernels += n_launch;
        ge->n_vote_kernels += n_launch;
    }
    return GLCM_OK;
}

// Capture-time timing events around a graph's vote kernels; the graph's
// event nodes are re-pointed per replay.
int capture_mark(glcm_ctx* ctx, GraphEntry* ge, bool start)
{
    if (!ge || !ctx->timing)
        return GLCM_OK;
    if (!ge->cap_a) {
        CK(cudaEventCreate(&ge->cap_a));
        CK(cudaEventCreate(&ge->cap_b));
    }
    CK(cudaEventRecordWithFlags(start ? ge->cap_a : ge->cap_b, ctx->stream, cudaEventRecordExternal));
    return GLCM_OK;
}

// Feature jobs in launch order (feat_job_group): one small CTA each (N <=
// 32), one CTA each, one cluster of CTAs each (symmetric, 128 < N <= 256).
// Each job names its own outputs, so the order changes nothing else.
// Feature jobs by number of levels, then launch group: the jobs of one
// number of levels are contiguous (an epilogue can follow its class's votes)
// and the runs of one launch group long.
void order_feats(std::vector<FeatJob>& feats)
{
    std::stable_sort(feats.begin(), feats.end(), [](const FeatJob& a, const FeatJob& b) {
        return a.levels != b.levels ? a.levels < b.levels : feat_job_group(a) < feat_job_group(b);
    });
}

int enqueue_features(glcm_ctx* ctx, const std::vector<FeatJob>& feats, const DevBuf& dfeat, int max_levels,
                     bool capturing, GraphEntry* ge, cudaStream_t st = nullptr, int priority = 0)
{
    if (feats.empty())
        return GLCM_OK;
    if (!st)
        st = ctx->stream;
    // One launch per run of jobs of one launch group.
    size_t g0 = 0;
    while (g0 < feats.size()) {
        const int grp = feat_job_group(feats[g0]);
        size_t g1 = g0;
        int gmax = 2;
        bool any_feat = false;
        while (g1 < feats.size() && feat_job_group(feats[g1]) == grp) {
            gmax = std::max(gmax, feats[g1].levels);
            any_feat |= feats[g1].features != nullptr;
            ++g1;
        }
        if (gmax > max_levels)
            return fail(ctx, GLCM_ERR_CUDA, "internal: a feature job beyond the launch's levels");
        FeatParams fp{};
        fp.jobs = static_cast<const FeatJob*>(dfeat.p) + g0;
        fp.n_jobs = (int)(g1 - g0);
        fp.err = ctx->d_words;
        if (grp == 2) {
            CK(launch_features_cluster(fp, st, priority));
        } else {
            if (gmax > 64 && any_feat) {
                const long long per = features_work_floats(gmax);
                TRY(ensure(ctx, ctx->work, (size_t)fp.n_jobs * (size_t)per * sizeof(float)));
                fp.work = static_cast<float*>(ctx->work.p);
                fp.work_stride = per;
            }
            CK(launch_features(fp, gmax, st, grp == 0 ? kFeatThreadsSmall : kFeatThreads, priority));
        }
        if (!capturing)
            ctx->kernel_launches += 1;
        if (ge)
            ge->n_kernels++;
        g0 = g1;
    }
    return GLCM_OK;
}

// Read (and clear) the device error word after synchronizing the stream.
int collect_device_errors(glcm_ctx* ctx)
{
    CK(cudaStreamSynchronize(ctx->stream));
    unsigned w = 0;
    CK(cudaMemcpy(&w, ctx->d_words, sizeof w, cudaMemcpyDeviceToHost));
    if (w) {
        CK(cudaMemset(ctx->d_words, 0, sizeof(unsigned)));
        if (w & kErrInternal)
            return fail(ctx, GLCM_ERR_CUDA, "a kernel index check failed (error bits 0x%x)", w);
        if (w & kErrTimeout)
            return fail(ctx, GLCM_ERR_TIMEOUT, "a bounded device wait gave up (error bits 0x%x)", w);
        if (w & kErrRange)
            return fail(ctx, GLCM_ERR_RANGE, "a pixel >= levels in GLCM_INPUT_LEVELS mode; its pairs were skipped");
    }
    return GLCM_OK;
}

// Image rows from host memory to the device (see copy_rows_to_device).  The
// destination rows are 16-byte aligned; unit k of a row is destination bytes
// [16k, 16k + 16).  A row that starts on a 16-byte boundary is copied one
// aligned 16-byte block per unit; otherwise a unit comes from two aligned
// blocks realigned by funnel shifts.  Only blocks that hold at least one byte
// of the row are read, so no read leaves the pages of the caller's rows;
// destination bytes past row_bytes (up to the next 16) are don't-care padding.
// Each thread keeps kCopyUnroll units in flight (the reads cross the
// chip-to-chip link, so bytes in flight set the rate).
constexpr int kCopyUnroll = 4;

__device__ __forceinline__ uint4 load_row_unit(const uint8_t* src, size_t spitch, size_t row_bytes, long long r,
                                               size_t u)
{
    const uintptr_t row = reinterpret_cast<uintptr_t>(src) + (uintptr_t)(r * (long long)spitch);
    const uintptr_t first = row + 16 * u;
    const unsigned off = (unsigned)(first & 15);
    if (off == 0)
        return *reinterpret_cast<const uint4*>(first);
    const uintptr_t b0 = first & ~(uintptr_t)15;
    const uintptr_t last_blk = (row + row_bytes - 1) & ~(uintptr_t)15;
    const uint4 x = *reinterpret_cast<const uint4*>(b0);
    const uint4 y = b0 + 16 <= last_blk ? *reinterpret_cast<const uint4*>(b0 + 16) : make_uint4(0, 0, 0, 0);
    const uint32_t w[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
    const unsigned q = off >> 2, sh = 8 * (off & 3);
    uint32_t o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        // words q + i and q + i + 1 of the 8, selected without dynamic indexing
        uint32_t lo = w[i], hi = w[i + 1];
        if (q == 1) {
            lo = w[i + 1];
            hi = w[i + 2];
        } else if (q == 2) {
            lo = w[i + 2];
            hi = w[i + 3];
        } else if (q == 3) {
            lo = w[i + 3];
            hi = i + 4 < 8 ? w[i + 4] : 0u;
        }
        o[i] = __funnelshift_r(lo, hi, sh);
    }
    return make_uint4(o[0], o[1], o[2], o[3]);
}

__global__ void k_copy_rows(uint8_t* __restrict__ dst, size_t dpitch, const uint8_t* __restrict__ src, size_t spitch,
                            size_t row_bytes, int rows)
{
    const size_t units = (row_bytes + 15) / 16;
    const long long total = (long long)units * rows;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; k0 < total; k0 += kCopyUnroll * stride) {
        uint4 v[kCopyUnroll];
        long long at[kCopyUnroll];
#pragma unroll
        for (int e = 0; e < kCopyUnroll; ++e) {
            const long long k = k0 + e * stride;
            at[e] = -1;
            if (k < total) {
                const long long r = total <= 0xFFFFFFFFll ? (long long)((unsigned)k / (unsigned)units)
                                                           : k / (long long)units;
                const size_t u = (size_t)(k - r * (long long)units);
                v[e] = load_row_unit(src, spitch, row_bytes, r, u);
                at[e] = r * (long long)dpitch + 16 * (long long)u;
            }
        }
#pragma unroll
        for (int e = 0; e < kCopyUnroll; ++e)
            if (at[e] >= 0)
                *reinterpret_cast<uint4*>(dst + at[e]) = v[e];
    }
}

}  // namespace

// Host-to-device copy of `rows` image rows.  Registered (pinned) host memory
// that the device can address is read by a copy kernel on a few SMs (16-byte
// aligned reads, realigned on the device): on GB300
// (host memory behind the chip-to-chip link) copy-engine transfers from host
// memory held back the kernels of other streams until every queued transfer
// had finished, while a copy kernel overlaps them (the vote launches that
// run beside it leave it a few SMs).  Other host memory takes
// cudaMemcpyAsync (one flat copy when both sides have the same pitch) or
// cudaMemcpy2DAsync, as does every copy when allow_kernel is false.
cudaError_t glcm::copy_rows_to_device(void* dst, size_t dpitch, const void* src, size_t spitch, size_t row_bytes,
                                      int rows, cudaStream_t st, bool allow_kernel, int max_ctas)
{
    if (rows <= 0 || row_bytes == 0)
        return cudaSuccess;
    cudaPointerAttributes pa;
    if (allow_kernel && cudaPointerGetAttributes(&pa, src) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer) {
        // The destination side must allow 16-byte stores; the source side may
        // start anywhere.
        const uintptr_t b = reinterpret_cast<uintptr_t>(dst);
        if ((b | dpitch) % 16 == 0 && dpitch >= ((row_bytes + 15) & ~(size_t)15)) {
            const long long units = (long long)((row_bytes + 15) / 16) * rows;
            const int grid = (int)std::max<long long>(1, std::min<long long>(max_ctas, (units + 511) / 512));
            k_copy_rows<<<grid, 512, 0, st>>>(static_cast<uint8_t*>(dst), dpitch,
                                              static_cast<const uint8_t*>(pa.devicePointer), spitch, row_bytes, rows);
            return cudaGetLastError();
        }
    }
    cudaGetLastError();
    if (dpitch == spitch)
        return cudaMemcpyAsync(dst, src, spitch * (size_t)(rows - 1) + row_bytes, cudaMemcpyHostToDevice, st);
    return cudaMemcpy2DAsync(dst, dpitch, src, spitch, row_bytes, rows, cudaMemcpyHostToDevice, st);
}

void glcm::set_vote_sm_reserve(glcm_ctx* ctx, int sms)
{
    if (ctx)
        ctx->sm_reserve = std::max(0, std::min(sms, ctx->sm_count - 1));
}

namespace {

// Copy a host image into device staging, in row stripes on the copy stream;
// returns the device image.  stripe_rows[k] are the row ends of the copies.
int stage_host_image(glcm_ctx* ctx, const void* image, int width, int height, size_t pitch, int bpp,
                     DevBuf& dst, size_t& dpitch, const std::vector<int>& cuts)
{
    dpitch = (((size_t)width * bpp) + 15) & ~(size_t)15;
    TRY(ensure(ctx, dst, dpitch * height));
    int prev = 0;
    while (ctx->stripe_events.size() < cuts.size()) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->stripe_events.push_back(e);
    }
    for (size_t k = 0; k < cuts.size(); ++k) {
        const int r1 = cuts[k];
        if (r1 > prev) {
            CK(copy_rows_to_device(static_cast<uint8_t*>(dst.p) + (size_t)prev * dpitch, dpitch,
                                   static_cast<const uint8_t*>(image) + (size_t)prev * pitch, pitch,
                                   (size_t)width * bpp, r1 - prev, ctx->copy_stream));
        }
        CK(cudaEventRecord(ctx->stripe_events[k], ctx->copy_stream));
        prev = std::max(prev, r1);
    }
    return GLCM_OK;
}

std::string batch_key(const glcm_desc* d, int n, const glcm_ctx* ctx)
{
    std::string k;
    k.reserve((size_t)n * 96);
    char buf[160];
    for (int i = 0; i < n; ++i) {
        snprintf(buf, sizeof buf, "%p,%d,%d,%zu,%d,%d,%d,%p,%p,%p|", d[i].image, d[i].width, d[i].height,
                 d[i].pitch_bytes, d[i].dtype, d[i].levels, d[i].flags, (void*)d[i].counts,
                 (void*)d[i].normalized, (void*)d[i].features);
        k += buf;
        for (int o = 0; o < d[i].n_offsets; ++o) {
            snprintf(buf, sizeof buf, "%d:%d;", d[i].offsets[o].dx, d[i].offsets[o].dy);
            k += buf;
        }
    }
    k += ctx->timing ? "T" : "U";
    for (const auto& kv : ctx->overrides) {
        snprintf(buf, sizeof buf, "#%lld:%d,%d,%d,%d", kv.first, kv.second.threads, kv.second.rshift,
                 kv.second.layout, kv.second.band_rows);
        k += buf;
    }
    return k;
}

void destroy_graph(GraphEntry& g)
{
    if (g.exec)
        cudaGraphExecDestroy(g.exec);
    if (g.graph)
        cudaGraphDestroy(g.graph);
    if (g.cap_a)
        cudaEventDestroy(g.cap_a);
    if (g.cap_b)
        cudaEventDestroy(g.cap_b);
    for (DevBuf* b : {&g.jobs, &g.offs, &g.feat, &g.jobs2, &g.offs2, &g.feat2})
        if (b->p)
            cudaFree(b->p);
}

}  // namespace

// ---------------------------------------------------------------------------
// Public API
// ---------------------------------------------------------------------------

extern "C" int glcm_offset_from_angle(int d, int theta_deg, glcm_offset* out)
{
    if (!out || d < 1)
        return GLCM_ERR_ARG;
    switch (theta_deg) {
        case 0: *out = {d, 0}; return GLCM_OK;
        case 45: *out = {d, -d}; return GLCM_OK;
        case 90: *out = {0, -d}; return GLCM_OK;
        case 135: *out = {-d, -d}; return GLCM_OK;
        default: return GLCM_ERR_ARG;
    }
}

extern "C" const char* glcm_last_error(const glcm_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

extern "C" int glcm_create(glcm_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream)
{
    glcm_ctx* ctx = nullptr;
    if (!out)
        return fail(nullptr, GLCM_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, GLCM_ERR_ARG, "no CUDA device %d", device);
    }
    if (cudaSetDevice(device) != cudaSuccess)
        return fail(nullptr, GLCM_ERR_CUDA, "cudaSetDevice(%d) failed", device);
    ctx = new glcm_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)1 << 30;
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&ctx->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    {
        int least = 0, greatest = 0;
        if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess)
            ctx->prio_high = greatest;
    }
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return fail(nullptr, GLCM_ERR_CUDA, "cudaStreamCreate failed");
        }
        ctx->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->epi_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_join2, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_stage, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->ev_cls_fork, cudaEventDisableTiming) != cudaSuccess) {
        glcm_destroy(ctx);
        return fail(nullptr, GLCM_ERR_CUDA, "stream/event creation failed");
    }
    for (int i = 0; i < 4; ++i)
        if (cudaStreamCreateWithFlags(&ctx->cls_stream[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_cls_vote[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ctx->ev_cls_done[i], cudaEventDisableTiming) != cudaSuccess) {
            glcm_destroy(ctx);
            return fail(nullptr, GLCM_ERR_CUDA, "stream/event creation failed");
        }
    if (fault_injected("alloc") || cudaMalloc(&ctx->d_words, 128) != cudaSuccess) {
        cudaGetLastError();
        ctx->d_words = nullptr;
        glcm_destroy(ctx);
        return fail(nullptr, GLCM_ERR_NOMEM, "could not allocate the context's device words");
    }
    cudaMemset(ctx->d_words, 0, 128);
    cudaDeviceSynchronize();
    *out = ctx;
    return GLCM_OK;
}

extern "C" int glcm_destroy(glcm_ctx* ctx)
{
    if (!ctx)
        return GLCM_OK;
    cudaSetDevice(ctx->device);
    if (ctx->stream)
        cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_stream)
        cudaStreamSynchronize(ctx->copy_stream);
    if (ctx->side_stream)
        cudaStreamSynchronize(ctx->side_stream);
    if (ctx->epi_stream)
        cudaStreamSynchronize(ctx->epi_stream);
    for (cudaStream_t cs : ctx->cls_stream)
        if (cs)
            cudaStreamSynchronize(cs);
    for (auto& kv : ctx->graphs)
        destroy_graph(kv.second);
    for (DevBuf* b : {&ctx->jobs, &ctx->offs, &ctx->feat, &ctx->work, &ctx->img, &ctx->counts, &ctx->norm,
                      &ctx->featout, &ctx->maps, &ctx->hb_img, &ctx->hb_out, &ctx->slide_tab})
        if (b->p)
            cudaFree(b->p);
    for (auto& t : ctx->hb_tab)
        for (DevBuf& b : t)
            if (b.p)
                cudaFree(b.p);
    if (ctx->d_words)
        cudaFree(ctx->d_words);
    if (ctx->h_stage)
        cudaFreeHost(ctx->h_stage);
    for (auto& p : ctx->pool) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : ctx->stripe_events)
        cudaEventDestroy(e);
    if (ctx->ev_stage)
        cudaEventDestroy(ctx->ev_stage);
    if (ctx->copy_stream)
        cudaStreamDestroy(ctx->copy_stream);
    if (ctx->side_stream)
        cudaStreamDestroy(ctx->side_stream);
    if (ctx->epi_stream)
        cudaStreamDestroy(ctx->epi_stream);
    if (ctx->ev_join2)
        cudaEventDestroy(ctx->ev_join2);
    if (ctx->ev_fork)
        cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join)
        cudaEventDestroy(ctx->ev_join);
    for (int i = 0; i < 4; ++i) {
        if (ctx->cls_stream[i])
            cudaStreamDestroy(ctx->cls_stream[i]);
        if (ctx->ev_cls_vote[i])
            cudaEventDestroy(ctx->ev_cls_vote[i]);
        if (ctx->ev_cls_done[i])
            cudaEventDestroy(ctx->ev_cls_done[i]);
    }
    if (ctx->ev_cls_fork)
        cudaEventDestroy(ctx->ev_cls_fork);
    if (ctx->own_stream && ctx->stream)
        cudaStreamDestroy(ctx->stream);
    delete ctx;
    return GLCM_OK;
}

extern "C" int glcm_synchronize(glcm_ctx* ctx)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    return collect_device_errors(ctx);
}

extern "C" int glcm_set_timing(glcm_ctx* ctx, int enable)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    ctx->timing = enable != 0;
    return GLCM_OK;
}

extern "C" int glcm_get_timing(glcm_ctx* ctx, double* vote_ms, long long* vote_launches, long long* kernel_launches,
                               int reset)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    CK(cudaStreamSynchronize(ctx->stream));
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p.a, p.b));
        ctx->vote_ms += ms;
        ctx->pool.push_back(p);
    }
    ctx->pending.clear();
    if (vote_ms)
        *vote_ms = ctx->vote_ms;
    if (vote_launches)
        *vote_launches = ctx->vote_launches;
    if (kernel_launches)
        *kernel_launches = ctx->kernel_launches;
    if (reset) {
        ctx->vote_ms = 0;
        ctx->vote_launches = 0;
        ctx->kernel_launches = 0;
    }
    return GLCM_OK;
}

extern "C" int glcm_set_vote_config(glcm_ctx* ctx, int levels, int n_offsets, int dtype, int threads,
                                    int log2_copies, int layout, int band_rows)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    const int bpp = dtype == GLCM_U16 ? 2 : 1;
    const long long key = cfg_key(levels, n_offsets, bpp);
    if (threads <= 0) {
        ctx->overrides.erase(key);
        return GLCM_OK;
    }
    if (threads % 32 || threads < 64 || threads > kMaxThreads || log2_copies < 0 || log2_copies > 5 ||
        layout < 0 || layout > 4 || levels < 2 || levels > GLCM_MAX_LEVELS || n_offsets < 1 || band_rows < 0)
        return fail(ctx, GLCM_ERR_ARG, "invalid vote config");
    if (layout == 4) {
        // The column-walk kernel: N a power of two up to 32; threads and
        // copies are fixed by the kernel, band_rows (0 = derived) is its item height.
        const int l2 = ilog2_exact(levels);
        if (l2 < 1 || (l2 > 5 && l2 != 8))
            return fail(ctx, GLCM_ERR_ARG, "the column-walk kernel needs N in {2, 4, 8, 16, 32, 256}");
        VoteCfg c;
        c.threads = 512;
        c.rshift = 5;
        c.layout = 4;
        c.band_rows = band_rows;
        ctx->overrides[key] = c;
        return GLCM_OK;
    }
    if (job_shape(ctx, levels, n_offsets, layout, log2_copies).jobs <= 0)
        return fail(ctx, GLCM_ERR_ARG, "one level row of the histograms does not fit shared memory");
    if (layout == 2 && 65535ll * (1 << log2_copies) / ((16 / bpp) * (long long)threads) < 1)
        return fail(ctx, GLCM_ERR_ARG, "16-bit counters cannot be bounded with this config");
    VoteCfg c;
    c.threads = threads;
    c.rshift = log2_copies;
    c.layout = layout;
    c.band_rows = band_rows;
    ctx->overrides[key] = c;
    return GLCM_OK;
}

extern "C" int glcm_compute(glcm_ctx* ctx, const void* image, int width, int height, size_t pitch_bytes, int dtype,
                            int levels, const glcm_offset* offsets, int n_offsets, int flags, uint32_t* counts,
                            float* normalized)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    TRY(check_image_args(ctx, image, width, height, pitch_bytes, dtype, levels, offsets, n_offsets));
    if (!counts)
        return fail(ctx, GLCM_ERR_ARG, "counts is NULL");
    const int bpp = dtype == GLCM_U8 ? 1 : 2;
    const bool dev_img = is_device_ptr(image);
    const bool dev_counts = is_device_ptr(counts);
    const bool want_norm = (flags & GLCM_NORMALIZE) && normalized;
    if (want_norm && levels > GLCM_MAX_LEVELS)
        return fail(ctx, GLCM_ERR_UNSUPPORTED, "normalized GLCMs need levels <= %d", GLCM_MAX_LEVELS);
    const bool dev_norm = want_norm && is_device_ptr(normalized);
    const size_t nn = (size_t)levels * levels;
    uint32_t* d_counts = counts;
    if (!dev_counts) {
        TRY(ensure(ctx, ctx->counts, n_offsets * nn * 4));
        d_counts = static_cast<uint32_t*>(ctx->counts.p);
    }
    float* d_norm = normalized;
    if (want_norm && !dev_norm) {
        TRY(ensure(ctx, ctx->norm, n_offsets * nn * 4));
        d_norm = static_cast<float*>(ctx->norm.p);
    }
    int dymin = 0, dymax = 0;
    bool wide_wrap = false;  // a flat-wrap offset reaching a whole row or more sideways
    for (int k = 0; k < n_offsets; ++k) {
        dymin = std::min(dymin, offsets[k].dy);
        dymax = std::max(dymax, offsets[k].dy);
        wide_wrap |= std::abs(offsets[k].dx) >= width;
    }
    const bool flat = (flags & GLCM_FLAT_WRAP) != 0;
    // A flat-wrap pair that leaves a row to the right lands one row further down.
    if (flat)
        dymax += 1;

    // Stripes (Sec. III): anchor rows [r_k, r_{k+1}); stripe k's copy ends at
    // r_{k+1} + max(dy, 0) so its partner rows are on the device.
    std::vector<int> anchors_cut;
    int n_stripes = 1;
    if (!dev_img) {
        const long long bytes = (long long)height * width * bpp;
        n_stripes = (int)std::max<long long>(1, std::min<long long>(8, bytes / (4ll << 20)));
        n_stripes = std::min(n_stripes, height);
        if (flat && wide_wrap)
            n_stripes = 1;
    }
    for (int k = 1; k <= n_stripes; ++k)
        anchors_cut.push_back((int)((long long)height * k / n_stripes));
    const uint8_t* d_img = static_cast<const uint8_t*>(image);
    size_t dpitch = pitch_bytes;
    if (!dev_img) {
        std::vector<int> copy_cut;
        for (int r : anchors_cut)
            copy_cut.push_back(std::min(height, r + dymax));
        TRY(stage_host_image(ctx, image, width, height, pitch_bytes, bpp, ctx->img, dpitch, copy_cut));
        d_img = static_cast<const uint8_t*>(ctx->img.p);
    }
    // Zero the counts once, then one vote launch per stripe.
    TRY(zero_words(ctx, d_counts, (long long)n_offsets * nn, ctx->stream));
    int r0 = 0;
    for (int k = 0; k < n_stripes; ++k) {
        const int r1 = anchors_cut[k];
        if (!dev_img)
            CK(cudaStreamWaitEvent(ctx->stream, ctx->stripe_events[k], 0));
        VotePlan plan;
        ImageSpec s{d_img, (long long)dpitch, width, height, bpp, levels, (flags & GLCM_INPUT_LEVELS) ? 1 : 0,
                    offsets, n_offsets, d_counts, r0, r1, flat ? 1 : 0};
        TRY(plan_image(ctx, s, plan, target_items(ctx)));
        finalize_fast(plan, launch_ctas(ctx));
        build_chunks(plan, ctx->sm_count);
        std::vector<FeatJob> none;
        TRY(upload_tables(ctx, plan, none, ctx->jobs, ctx->offs, ctx->feat));
        TRY(enqueue_vote(ctx, plan, ctx->jobs, ctx->offs,
                         reinterpret_cast<const int3*>(static_cast<uint8_t*>(ctx->jobs.p) + plan.chunk_off), false,
                         false, nullptr));
        r0 = r1;
    }
    if (want_norm) {
        std::vector<FeatJob> fj(n_offsets);
        for (int o = 0; o < n_offsets; ++o)
            fj[o] = FeatJob{d_counts + o * nn, d_norm + o * nn, nullptr, levels, (flags & GLCM_SYMMETRIC) ? 1 : 0};
        VotePlan empty;
        TRY(upload_tables(ctx, empty, fj, ctx->jobs, ctx->offs, ctx->feat));
        TRY(enqueue_features(ctx, fj, ctx->feat, levels, false, nullptr));
    }
    if (!dev_counts)
        CK(cudaMemcpyAsync(counts, d_counts, n_offsets * nn * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (want_norm && !dev_norm)
        CK(cudaMemcpyAsync(normalized, d_norm, n_offsets * nn * 4, cudaMemcpyDeviceToHost, ctx->stream));
    const bool sync = ctx->own_stream || !dev_img || !dev_counts || (want_norm && !dev_norm);
    if (sync)
        return collect_device_errors(ctx);
    return GLCM_OK;
}

extern "C" int glcm_compute_naive(glcm_ctx* ctx, const void* image, int width, int height, size_t pitch_bytes,
                                  int dtype, int levels, glcm_offset offset, int flags, uint32_t* counts)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    TRY(check_image_args(ctx, image, width, height, pitch_bytes, dtype, levels, &offset, 1));
    if (!is_device_ptr(image) || !is_device_ptr(counts))
        return fail(ctx, GLCM_ERR_ARG, "glcm_compute_naive takes device pointers only");
    const size_t nn = (size_t)levels * levels;
    TRY(zero_words(ctx, counts, (long long)nn, ctx->stream));
    CK(launch_naive(static_cast<const uint8_t*>(image), (long long)pitch_bytes, width, height,
                    dtype == GLCM_U8 ? 1 : 2, levels, (flags & GLCM_INPUT_LEVELS) ? 1 : 0, offset.dx, offset.dy,
                    counts, ctx->d_words, ctx->stream));
    ctx->kernel_launches += 1;
    if (ctx->own_stream)
        return collect_device_errors(ctx);
    return GLCM_OK;
}

extern "C" int glcm_features(glcm_ctx* ctx, const uint32_t* counts, int levels, int n_glcm, int flags,
                             float* features)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (levels > GLCM_MAX_LEVELS && levels <= GLCM_MAX_COUNT_LEVELS)
        return fail(ctx, GLCM_ERR_UNSUPPORTED, "features need levels <= %d", GLCM_MAX_LEVELS);
    if (!counts || !features || n_glcm < 0 || levels < 2 || levels > GLCM_MAX_LEVELS)
        return fail(ctx, GLCM_ERR_ARG, "glcm_features: bad arguments");
    if (n_glcm == 0)
        return GLCM_OK;
    const size_t nn = (size_t)levels * levels;
    const bool dev_c = is_device_ptr(counts), dev_f = is_device_ptr(features);
    const uint32_t* d_c = counts;
    float* d_f = features;
    if (!dev_c) {
        TRY(ensure(ctx, ctx->counts, n_glcm * nn * 4));
        CK(cudaMemcpyAsync(ctx->counts.p, counts, n_glcm * nn * 4, cudaMemcpyHostToDevice, ctx->stream));
        d_c = static_cast<const uint32_t*>(ctx->counts.p);
    }
    if (!dev_f) {
        TRY(ensure(ctx, ctx->featout, (size_t)n_glcm * GLCM_N_FEATURES * 4));
        d_f = static_cast<float*>(ctx->featout.p);
    }
    std::vector<FeatJob> fj(n_glcm);
    for (int g = 0; g < n_glcm; ++g)
        fj[g] = FeatJob{d_c + g * nn, nullptr, d_f + (size_t)g * GLCM_N_FEATURES, levels,
                        (flags & GLCM_SYMMETRIC) ? 1 : 0};
    VotePlan empty;
    TRY(upload_tables(ctx, empty, fj, ctx->jobs, ctx->offs, ctx->feat));
    TRY(enqueue_features(ctx, fj, ctx->feat, levels, false, nullptr));
    if (!dev_f)
        CK(cudaMemcpyAsync(features, d_f, (size_t)n_glcm * GLCM_N_FEATURES * 4, cudaMemcpyDeviceToHost,
                           ctx->stream));
    if (ctx->own_stream || !dev_c || !dev_f)
        return collect_device_errors(ctx);
    return GLCM_OK;
}

namespace {

// Build the plan and feature jobs of a batch whose images and outputs are on
// the device.
int plan_batch(glcm_ctx* ctx, const glcm_desc* descs, int n, VotePlan& plan, std::vector<FeatJob>& feats,
               int& max_levels, int ctas)
{
    max_levels = 2;
    long long total_rows_strips = 0;
    for (int i = 0; i < n; ++i) {
        const int PX = descs[i].dtype == GLCM_U8 ? 16 : 8;
        total_rows_strips += (long long)descs[i].height * ((descs[i].width + 32 * PX - 1) / (32 * PX));
    }
    for (int i = 0; i < n; ++i) {
        const glcm_desc& d = descs[i];
        const int bpp = d.dtype == GLCM_U8 ? 1 : 2;
        if ((d.normalized || d.features) && d.levels > GLCM_MAX_LEVELS)
            return fail(ctx, GLCM_ERR_UNSUPPORTED, "desc %d: normalized GLCMs and features need levels <= %d", i,
                        GLCM_MAX_LEVELS);
        // Work items in proportion to this image's share of the batch.
        const long long rs = (long long)d.height * ((d.width + 32 * (16 / bpp) - 1) / (32 * (16 / bpp)));
        const int tgt = (int)std::max<long long>(1, (long long)target_items(ctx) * 4 * rs /
                                                        std::max<long long>(1, total_rows_strips));
        ImageSpec s{static_cast<const uint8_t*>(d.image), (long long)d.pitch_bytes, d.width, d.height, bpp,
                    d.levels, (d.flags & GLCM_INPUT_LEVELS) ? 1 : 0, d.offsets, d.n_offsets, d.counts, 0,
                    d.height, (d.flags & GLCM_FLAT_WRAP) ? 1 : 0};
        TRY(plan_image(ctx, s, plan, tgt));
        if (d.normalized || d.features)
            max_levels = std::max(max_levels, d.levels);  // the epilogue's shared-memory layout
        const size_t nn = (size_t)d.levels * d.levels;
        if (d.normalized || d.features) {
            for (int o = 0; o < d.n_offsets; ++o)
                feats.push_back(FeatJob{d.counts + o * nn, d.normalized ? d.normalized + o * nn : nullptr,
                                        d.features ? d.features + (size_t)o * GLCM_N_FEATURES : nullptr, d.levels,
                                        (d.flags & GLCM_SYMMETRIC) ? 1 : 0});
        }
    }
    finalize_fast(plan, ctas);
    order_feats(feats);
    return GLCM_OK;
}


// A device batch split by pixel type (the vote kernel is templated on it),
// with its tables uploaded: p8's jobs, offsets and chunks first, then p16's.
struct SplitBatch {
    VotePlan p8, p16;
    std::vector<FeatJob> feats;
    int max_levels = 2;
    DevBuf j16, o16;                       // views into the uploaded tables
    const int3* c8 = nullptr;
    const int3* c16 = nullptr;
};

// ctas: the CTAs the batch's column-walk launches will have (its chunks are
// cut for exactly that many); 0: every SM the context's launches use.
int prepare_batch(glcm_ctx* ctx, const glcm_desc* descs, int n, SplitBatch& sb, DevBuf& djobs, DevBuf& doffs,
                  DevBuf& dfeat, int ctas = 0)
{
    VotePlan plan;
    TRY(plan_batch(ctx, descs, n, plan, sb.feats, sb.max_levels, ctas > 0 ? ctas : launch_ctas(ctx)));
    for (int pass = 0; pass < 2; ++pass) {
        VotePlan& dst = pass == 0 ? sb.p8 : sb.p16;
        dst.threads = plan.threads;
        dst.bpp = pass == 0 ? 1 : 2;
        for (const VoteJob& j : plan.jobs) {
            if (j.bpp != dst.bpp)
                continue;
            VoteJob c = j;
            const int cnt_items = (c.n_strips) * ((c.y_end - c.y_begin + c.band_rows - 1) / c.band_rows);
            c.off0 = (int)dst.offs.size();
            for (int k = 0; k < j.n_off; ++k)
                dst.offs.push_back(plan.offs[j.off0 + k]);
            c.item0 = dst.n_items;
            dst.n_items += cnt_items;
            dst.max_hist_words = std::max(dst.max_hist_words, c.hist_words);
            if (c.staged)
                dst.tile_rows = std::max(dst.tile_rows, c.band_rows + c.dy_max - c.dy_min);
            dst.jobs.push_back(c);
        }
    }
    // The column-walk classes and the flat-wrap seams (either pixel type)
    // launch with the uint8 part.
    sb.p8.fast = plan.fast;
    sb.p8.seams = plan.seams;
    sb.p8.globals = plan.globals;
    VotePlan all;
    all.fast = plan.fast;
    all.seams = plan.seams;
    all.globals = plan.globals;
    all.jobs = sb.p8.jobs;
    all.jobs.insert(all.jobs.end(), sb.p16.jobs.begin(), sb.p16.jobs.end());
    for (size_t k = sb.p8.jobs.size(); k < all.jobs.size(); ++k)
        all.jobs[k].off0 += (int)sb.p8.offs.size();
    all.offs = sb.p8.offs;
    all.offs.insert(all.offs.end(), sb.p16.offs.begin(), sb.p16.offs.end());
    build_chunks(sb.p8, ctx->sm_count);
    build_chunks(sb.p16, ctx->sm_count);
    all.chunks = sb.p8.chunks;
    all.chunks.insert(all.chunks.end(), sb.p16.chunks.begin(), sb.p16.chunks.end());
    TRY(upload_tables(ctx, all, sb.feats, djobs, doffs, dfeat));
    for (size_t c = 0; c < all.fast.size(); ++c) {
        sb.p8.fast[c].jobs_off = all.fast[c].jobs_off;
        sb.p8.fast[c].chunks_off = all.fast[c].chunks_off;
    }
    sb.p8.seams_off = all.seams_off;
    sb.p8.globals_off = all.globals_off;
    sb.j16.p = static_cast<VoteJob*>(djobs.p) + sb.p8.jobs.size();
    sb.o16.p = doffs.p;  // p16's off0 are already shifted past p8's offsets
    sb.c8 = reinterpret_cast<const int3*>(static_cast<uint8_t*>(djobs.p) + all.chunk_off);
    sb.c16 = sb.c8 + sb.p8.chunks.size();
    return GLCM_OK;
}

// The epilogue of a prepared batch part on ctx->stream; when its column-walk
// classes voted side by side (cs), the GLCMs of each number of levels follow
// their class's votes on its stream, at the device's most urgent priority
// (an SM freed by a vote CTA goes to them before the other classes' pending
// vote CTAs: the epilogues of the early classes do not pile up at the end),
// and the stream waits for all of them.
int enqueue_epilogue(glcm_ctx* ctx, const SplitBatch& sb, const DevBuf& dfeat, bool capturing, GraphEntry* ge,
                     const ClassStreams& cs)
{
    if (!cs.used)
        return enqueue_features(ctx, sb.feats, dfeat, sb.max_levels, capturing, ge);
    size_t done = 0;
    for (int g = 0; g < cs.n; ++g) {
        size_t a = 0;
        while (a < sb.feats.size() && sb.feats[a].levels != cs.levels[g])
            ++a;
        size_t b = a;
        while (b < sb.feats.size() && sb.feats[b].levels == cs.levels[g])
            ++b;
        if (b > a) {
            const std::vector<FeatJob> part(sb.feats.begin() + (long)a, sb.feats.begin() + (long)b);
            DevBuf view;
            view.p = static_cast<FeatJob*>(dfeat.p) + a;
            TRY(enqueue_features(ctx, part, view, sb.max_levels, capturing, ge, ctx->cls_stream[g], ctx->prio_high));
            done += b - a;
        }
        CK(cudaEventRecord(ctx->ev_cls_done[g], ctx->cls_stream[g]));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_cls_done[g], 0));
    }
    if (done != sb.feats.size())
        return fail(ctx, GLCM_ERR_CUDA, "internal: a feature job of no voted class");
    return GLCM_OK;
}

// Enqueue a prepared batch: zero + vote per pixel type, then the epilogue.
int enqueue_batch(glcm_ctx* ctx, const SplitBatch& sb, const DevBuf& djobs, const DevBuf& doffs, const DevBuf& dfeat,
                  bool capturing, GraphEntry* ge)
{
    if (capturing)
        TRY(capture_mark(ctx, ge, true));
    ClassStreams cs;
    if (!plan_empty(sb.p8))
        TRY(enqueue_vote(ctx, sb.p8, djobs, doffs, sb.c8, true, capturing, ge, nullptr,
                         plan_empty(sb.p16) ? &cs : nullptr));
    if (!plan_empty(sb.p16))
        TRY(enqueue_vote(ctx, sb.p16, sb.j16, sb.o16, sb.c16, true, capturing, ge));
    if (capturing)
        TRY(capture_mark(ctx, ge, false));
    return enqueue_epilogue(ctx, sb, dfeat, capturing, ge, cs);
}

// A batch split in two: the images whose epilogue is expensive (features of
// N > 64) vote first; their epilogue then runs on the side stream on a few
// SMs while the rest of the batch votes on the others, and the rest's
// epilogue follows.
int enqueue_batch_split(glcm_ctx* ctx, const SplitBatch& h, const DevBuf* th, SplitBatch& r, const DevBuf* tr,
                        bool capturing, GraphEntry* ge)
{
    if (capturing)
        TRY(capture_mark(ctx, ge, true));
    if (!plan_empty(h.p8))
        TRY(enqueue_vote(ctx, h.p8, th[0], th[1], h.c8, true, capturing, ge));
    if (!plan_empty(h.p16))
        TRY(enqueue_vote(ctx, h.p16, h.j16, h.o16, h.c16, true, capturing, ge));
    CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->side_stream, ctx->ev_fork, 0));
    TRY(enqueue_features(ctx, h.feats, th[2], h.max_levels, capturing, ge, ctx->side_stream));
    // The rest votes on every SM: the heavy epilogue, launched first, has
    // taken its SMs before the rest's CTAs queue for them.
    r.p8.max_ctas = r.p16.max_ctas = 0;
    ClassStreams cs;
    if (!plan_empty(r.p8))
        TRY(enqueue_vote(ctx, r.p8, tr[0], tr[1], r.c8, true, capturing, ge, nullptr,
                         plan_empty(r.p16) ? &cs : nullptr));
    if (!plan_empty(r.p16))
        TRY(enqueue_vote(ctx, r.p16, r.j16, r.o16, r.c16, true, capturing, ge));
    if (capturing)
        TRY(capture_mark(ctx, ge, false));
    TRY(enqueue_epilogue(ctx, r, tr[2], capturing, ge, cs));
    CK(cudaEventRecord(ctx->ev_join, ctx->side_stream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    return GLCM_OK;
}

// A batch with host buffers.  Every host image is copied once into device
// staging on the copy stream, in groups of about equal bytes; each group's
// votes start as soon as its own copies are in, so the copies of later
// groups overlap the votes of earlier ones (the paper overlaps the copies of
// image parts with the votes of earlier parts over streams, Sec. III).
// Images with expensive epilogues (features of N > 64) come first, and their
// groups' epilogues run on the side stream on a few SMs reserved from the
// votes.  Results come back to the host buffers once, at the end.
constexpr int kCopySMs = 8;

int run_host_batch(glcm_ctx* ctx, const glcm_desc* descs_in, int n)
{
    std::vector<glcm_desc> descs;
    descs.reserve(n);
    int n_heavy_glcm = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < n; ++i) {
            const bool heavy = descs_in[i].features && descs_in[i].levels > 64;
            if (heavy == (pass == 0)) {
                descs.push_back(descs_in[i]);
                n_heavy_glcm += heavy ? descs_in[i].n_offsets : 0;
            }
        }
    std::vector<glcm_desc> dd(descs);
    std::vector<size_t> img_off(n), dpitch(n);
    std::vector<char> host_img(n);
    size_t ib = 0, ob = 0;
    auto r256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    struct OutMap {
        size_t counts, norm, feat;
    };
    std::vector<OutMap> om(n);
    for (int i = 0; i < n; ++i) {
        const glcm_desc& d = descs[i];
        const int bpp = d.dtype == GLCM_U8 ? 1 : 2;
        host_img[i] = !is_device_ptr(d.image);
        dpitch[i] = (((size_t)d.width * bpp) + 15) & ~(size_t)15;
        img_off[i] = ib;
        if (host_img[i])
            ib += r256(dpitch[i] * d.height);
        const size_t nn = (size_t)d.levels * d.levels;
        om[i].counts = om[i].norm = om[i].feat = (size_t)-1;
        if (!is_device_ptr(d.counts)) {
            om[i].counts = ob;
            ob += r256(d.n_offsets * nn * 4);
        }
        if (d.normalized && !is_device_ptr(d.normalized)) {
            om[i].norm = ob;
            ob += r256(d.n_offsets * nn * 4);
        }
        if (d.features && !is_device_ptr(d.features)) {
            om[i].feat = ob;
            ob += r256((size_t)d.n_offsets * GLCM_N_FEATURES * 4);
        }
    }
    TRY(ensure(ctx, ctx->hb_img, ib));
    TRY(ensure(ctx, ctx->hb_out, ob));
    uint8_t* gi = static_cast<uint8_t*>(ctx->hb_img.p);
    uint8_t* go = static_cast<uint8_t*>(ctx->hb_out.p);
    for (int i = 0; i < n; ++i) {
        if (host_img[i]) {
            dd[i].image = gi + img_off[i];
            dd[i].pitch_bytes = dpitch[i];
        }
        if (om[i].counts != (size_t)-1)
            dd[i].counts = reinterpret_cast<uint32_t*>(go + om[i].counts);
        if (om[i].norm != (size_t)-1)
            dd[i].normalized = reinterpret_cast<float*>(go + om[i].norm);
        if (om[i].feat != (size_t)-1)
            dd[i].features = reinterpret_cast<float*>(go + om[i].feat);
    }
    // Groups of consecutive images, each voting as soon as its copies are in.
    // Host-to-device copies run at about 210 GB/s whatever moves them, so the
    // aim is to keep votes going while the rest copies in: the heavy images
    // (epilogue at N > 64, first in the order) form the first group -- their
    // votes cost several times their copy time -- and the light images follow
    // in three groups (55 / 25 / 20 % of their bytes), the last short so that
    // the exposed tail after the last copy stays small.  Without heavy images
    // the cuts are at 1/4, 5/8 and 7/8 of the bytes.  (Measured against 3, 4
    // and 6 groups of equal bytes, and 6 with small first groups.)
    std::vector<int> gend;
    {
        int n_heavy = 0;
        size_t heavy_bytes = 0, total = 0;
        for (int i = 0; i < n; ++i) {
            const size_t b = host_img[i] ? r256(dpitch[i] * descs[i].height) : 0;
            total += b;
            if (descs[i].features && descs[i].levels > 64) {
                ++n_heavy;
                heavy_bytes += b;
            }
        }
        std::vector<size_t> cuts;  // cumulative byte targets of the group ends but the last
        if (n_heavy > 0 && n_heavy < n) {
            cuts.push_back(heavy_bytes);
            cuts.push_back(heavy_bytes + (total - heavy_bytes) * 55 / 100);
            cuts.push_back(heavy_bytes + (total - heavy_bytes) * 80 / 100);
        } else {
            cuts.push_back(total / 4);
            cuts.push_back(total * 5 / 8);
            cuts.push_back(total * 7 / 8);
        }
        size_t acc = 0;
        size_t c = 0;
        for (int i = 0; i < n; ++i) {
            acc += host_img[i] ? r256(dpitch[i] * descs[i].height) : 0;
            if (i == n - 1) {
                gend.push_back(i + 1);
                break;
            }
            if (c < cuts.size() && acc >= cuts[c]) {
                gend.push_back(i + 1);
                while (c < cuts.size() && acc >= cuts[c])
                    ++c;
            }
        }
    }
    while (ctx->stripe_events.size() < gend.size()) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->stripe_events.push_back(e);
    }
    if (ctx->hb_tab.size() < gend.size())
        ctx->hb_tab.resize(gend.size());
    int first = 0;
    for (size_t g = 0; g < gend.size(); ++g) {
        for (int i = first; i < gend[g]; ++i) {
            if (!host_img[i])
                continue;
            const int bpp = descs[i].dtype == GLCM_U8 ? 1 : 2;
            CK(copy_rows_to_device(gi + img_off[i], dpitch[i], descs[i].image, descs[i].pitch_bytes,
                                   (size_t)descs[i].width * bpp, descs[i].height, ctx->copy_stream));
        }
        CK(cudaEventRecord(ctx->stripe_events[g], ctx->copy_stream));
        first = gend[g];
    }
    // Plans and tables of every group while the copies run (the copies go
    // through a copy kernel for registered memory, so the tables' small
    // uploads do not queue behind them on a copy engine).
    const int reserve = split_reserve(ctx, n_heavy_glcm);
    std::vector<SplitBatch> sbs(gend.size());
    first = 0;
    for (size_t g = 0; g < gend.size(); ++g) {
        auto& tab = ctx->hb_tab[g];
        // While later groups' copies are in flight, kCopySMs SMs stay free for the
        // copy kernel: a vote CTA fills its SM's register file, so without them
        // the copies stall behind the votes (measured).
        const int copy_sms = g + 1 < gend.size() ? kCopySMs : 0;
        const int group_ctas = ctx->sm_count - reserve - copy_sms;
        TRY(prepare_batch(ctx, dd.data() + first, gend[g] - first, sbs[g], tab[0], tab[1], tab[2],
                          launch_ctas(ctx, group_ctas)));
        if (reserve + copy_sms > 0)
            sbs[g].p8.max_ctas = sbs[g].p16.max_ctas = group_ctas;
        first = gend[g];
    }
    // Results of images [i0, i1) to the caller's host buffers on stream st.
    auto read_back = [&](int i0, int i1, cudaStream_t st) -> int {
        for (int i = i0; i < i1; ++i) {
            const size_t nn = (size_t)descs[i].levels * descs[i].levels;
            if (om[i].counts != (size_t)-1)
                CK(cudaMemcpyAsync(descs[i].counts, dd[i].counts, descs[i].n_offsets * nn * 4,
                                   cudaMemcpyDeviceToHost, st));
            if (om[i].norm != (size_t)-1)
                CK(cudaMemcpyAsync(descs[i].normalized, dd[i].normalized, descs[i].n_offsets * nn * 4,
                                   cudaMemcpyDeviceToHost, st));
            if (om[i].feat != (size_t)-1)
                CK(cudaMemcpyAsync(descs[i].features, dd[i].features,
                                   (size_t)descs[i].n_offsets * GLCM_N_FEATURES * 4, cudaMemcpyDeviceToHost, st));
        }
        return GLCM_OK;
    };
    bool forked = false;
    first = 0;
    for (size_t g = 0; g < gend.size(); ++g) {
        CK(cudaStreamWaitEvent(ctx->stream, ctx->stripe_events[g], 0));
        auto& tab = ctx->hb_tab[g];
        SplitBatch& sb = sbs[g];
        if (!plan_empty(sb.p8))
            TRY(enqueue_vote(ctx, sb.p8, tab[0], tab[1], sb.c8, true, false, nullptr));
        if (!plan_empty(sb.p16))
            TRY(enqueue_vote(ctx, sb.p16, sb.j16, sb.o16, sb.c16, true, false, nullptr));
        // Every group's epilogue and read-back off the vote stream, so the next
        // group's vote does not wait behind them and only the last group's
        // read-back is exposed: heavy groups on the side stream, light ones on
        // their own stream, so a light epilogue does not queue behind a heavy
        // one (their tables are per group; light epilogues use no global scratch).
        bool group_heavy = false;
        for (int i = first; i < gend[g]; ++i)
            group_heavy |= descs[i].features && descs[i].levels > 64;
        cudaStream_t es = group_heavy ? ctx->side_stream : ctx->epi_stream;
        CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
        CK(cudaStreamWaitEvent(es, ctx->ev_fork, 0));
        TRY(enqueue_features(ctx, sb.feats, tab[2], sb.max_levels, false, nullptr, es));
        TRY(read_back(first, gend[g], es));
        forked = true;
        first = gend[g];
    }
    if (forked) {
        CK(cudaEventRecord(ctx->ev_join, ctx->side_stream));
        CK(cudaEventRecord(ctx->ev_join2, ctx->epi_stream));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join2, 0));
    }
    return collect_device_errors(ctx);
}

}  // namespace

namespace {

int check_window_args(glcm_ctx* ctx, const void* image, int width, int height, size_t pitch_bytes, int dtype,
                      int levels, int win, int stride, const glcm_offset* offsets, int n_offsets, const void* counts,
                      const void* maps)
{
    TRY(check_image_args(ctx, image, width, height, pitch_bytes, dtype, levels, offsets, n_offsets));
    if (levels > GLCM_MAX_LEVELS)
        return fail(ctx, GLCM_ERR_UNSUPPORTED, "window GLCMs need levels <= %d", GLCM_MAX_LEVELS);
    if (n_offsets > GLCM_MAX_WINDOW_OFFSETS)
        return fail(ctx, GLCM_ERR_ARG, "at most %d window offsets", GLCM_MAX_WINDOW_OFFSETS);
    if (win < 1 || stride < 1 || win > width || win > height)
        return fail(ctx, GLCM_ERR_ARG, "window %d / stride %d do not fit %d x %d", win, stride, width, height);
    for (int k = 0; k < n_offsets; ++k)
        if (abs(offsets[k].dx) >= win || abs(offsets[k].dy) >= win)
            return fail(ctx, GLCM_ERR_ARG, "offset %d does not fit the window", k);
    if (!counts && !maps)
        return fail(ctx, GLCM_ERR_ARG, "need counts or maps");
    return GLCM_OK;
}

// Kernel parameters of a window job whose image and outputs are on the
// device (uploads the incremental kernel's tables once per context).
int window_params(glcm_ctx* ctx, const uint8_t* d_img, size_t dpitch, int width, int height, int dtype, int levels,
                  int win, int stride, const glcm_offset* offsets, int n_offsets, int flags, uint32_t* d_c,
                  float* d_m, WindowParams& wp)
{
    wp = WindowParams{};
    wp.img = d_img;
    wp.pitch = (long long)dpitch;
    wp.W = width;
    wp.H = height;
    wp.bpp = dtype == GLCM_U8 ? 1 : 2;
    wp.levels = levels;
    wp.levels_mode = (flags & GLCM_INPUT_LEVELS) ? 1 : 0;
    wp.win = win;
    wp.stride = stride;
    wp.nwx = (width - win) / stride + 1;
    wp.nwy = (height - win) / stride + 1;
    wp.n_off = n_offsets;
    for (int k = 0; k < n_offsets; ++k) {
        wp.dx[k] = offsets[k].dx;
        wp.dy[k] = offsets[k].dy;
    }
    wp.symmetric = (flags & GLCM_SYMMETRIC) ? 1 : 0;
    wp.counts = d_c;
    wp.maps = d_m;
    wp.err = ctx->d_words;
    if (!ctx->slide_tab_ready) {
        std::vector<long long> tab(kSlideTableWords);
        window_slide_tables(tab.data());
        TRY(ensure(ctx, ctx->slide_tab, tab.size() * sizeof(long long)));
        CK(cudaMemcpy(ctx->slide_tab.p, tab.data(), tab.size() * sizeof(long long), cudaMemcpyHostToDevice));
        ctx->slide_tab_ready = true;
    }
    wp.slide_tables = static_cast<const long long*>(ctx->slide_tab.p);
    return GLCM_OK;
}

int enqueue_windows(glcm_ctx* ctx, const std::vector<WindowParams>& wins, cudaStream_t st, bool capturing,
                    GraphEntry* ge)
{
    for (const WindowParams& wp : wins) {
        const cudaError_t e = launch_windows(wp, st);
        if (e == cudaErrorInvalidConfiguration) {
            cudaGetLastError();
            return fail(ctx, GLCM_ERR_UNSUPPORTED, "window histograms do not fit shared memory");
        }
        CK(e);
        if (!capturing)
            ctx->kernel_launches += 1;
        if (ge)
            ge->n_kernels++;
    }
    return GLCM_OK;
}

}  // namespace

// A device-resident batch (and window jobs, run first) replayed from a
// cached CUDA graph: the first call runs directly (setting every kernel
// attribute) and captures the graph; later calls with the same batch
// (pointers, sizes, flags; wkey for the window jobs) launch it.
int run_graph_batch(glcm_ctx* ctx, const glcm_desc* descs, int n, const std::vector<WindowParams>& wins,
                    const std::string& wkey)
{
    const std::string key = batch_key(descs, n, ctx) + wkey;
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        if (ctx->graphs.size() >= 16) {
            cudaStreamSynchronize(ctx->stream);
            for (auto& kv : ctx->graphs)
                destroy_graph(kv.second);
            ctx->graphs.clear();
        }
        GraphEntry ge;
        SplitBatch sb, sb2;
        // Expensive epilogues (features of N > 64) overlap the other images'
        // votes when the batch has both kinds.
        std::vector<glcm_desc> heavy, rest;
        for (int i = 0; i < n; ++i)
            (descs[i].features && descs[i].levels > 64 ? heavy : rest).push_back(descs[i]);
        const bool split = !heavy.empty() && !rest.empty();
        // One direct run produces this call's results and sets every kernel
        // attribute before capture.
        int rc0;
        if (split) {
            int n_heavy_glcm = 0;
            for (const glcm_desc& d : heavy)
                n_heavy_glcm += d.n_offsets;
            rc0 = prepare_batch(ctx, heavy.data(), (int)heavy.size(), sb, ge.jobs, ge.offs, ge.feat);
            if (rc0 == GLCM_OK)
                rc0 = prepare_batch(ctx, rest.data(), (int)rest.size(), sb2, ge.jobs2, ge.offs2, ge.feat2,
                                    launch_ctas(ctx));
        } else if (n > 0) {
            rc0 = prepare_batch(ctx, descs, n, sb, ge.jobs, ge.offs, ge.feat);
        } else {
            rc0 = GLCM_OK;
        }
        const DevBuf th[3] = {ge.jobs, ge.offs, ge.feat};
        const DevBuf tr[3] = {ge.jobs2, ge.offs2, ge.feat2};
        if (rc0 == GLCM_OK)
            rc0 = enqueue_windows(ctx, wins, ctx->stream, false, nullptr);
        if (rc0 == GLCM_OK && n > 0)
            rc0 = split ? enqueue_batch_split(ctx, sb, th, sb2, tr, false, nullptr)
                        : enqueue_batch(ctx, sb, ge.jobs, ge.offs, ge.feat, false, nullptr);
        if (rc0 == GLCM_OK)
            rc0 = collect_device_errors(ctx);
        if (rc0 != GLCM_OK) {
            cudaStreamSynchronize(ctx->stream);
            cudaStreamSynchronize(ctx->side_stream);
            for (cudaStream_t cs : ctx->cls_stream)
                cudaStreamSynchronize(cs);
            destroy_graph(ge);
            return rc0;
        }
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue_windows(ctx, wins, ctx->stream, true, &ge);
        if (rc == GLCM_OK && n > 0)
            rc = split ? enqueue_batch_split(ctx, sb, th, sb2, tr, true, &ge)
                       : enqueue_batch(ctx, sb, ge.jobs, ge.offs, ge.feat, true, &ge);
        cudaError_t ce = cudaStreamEndCapture(ctx->stream, &graph);
        if (rc != GLCM_OK) {
            if (graph)
                cudaGraphDestroy(graph);
            destroy_graph(ge);
            return rc;
        }
        CK(ce);
        ce = cudaGraphInstantiate(&ge.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
        if (ce == cudaSuccess && ctx->timing) {
            // Find the event-record nodes that bracket the first vote kernel.
            size_t nnodes = 0;
            cudaGraphGetNodes(graph, nullptr, &nnodes);
            std::vector<cudaGraphNode_t> nodes(nnodes);
            cudaGraphGetNodes(graph, nodes.data(), &nnodes);
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                cudaGraphNodeGetType(nd, &t);
                if (t == cudaGraphNodeTypeEventRecord) {
                    cudaEvent_t ev = nullptr;
                    cudaGraphEventRecordNodeGetEvent(nd, &ev);
                    if (ev == ge.cap_a)
                        ge.ev_start = nd;
                    else if (ev == ge.cap_b)
                        ge.ev_stop = nd;
                }
            }
        }
        ge.graph = graph;
        if (ce != cudaSuccess) {
            destroy_graph(ge);
            return fail(ctx, GLCM_ERR_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ce));
        }
        it = ctx->graphs.emplace(key, ge).first;
        // The direct run above already produced this batch's results.
        return ctx->own_stream ? collect_device_errors(ctx) : GLCM_OK;
    }
    GraphEntry& ge = it->second;
    TimedPair tp{};
    const bool timed = ctx->timing && ge.ev_start && ge.ev_stop;
    if (timed) {
        tp = take_pair(ctx);
        CK(cudaGraphExecEventRecordNodeSetEvent(ge.exec, ge.ev_start, tp.a));
        CK(cudaGraphExecEventRecordNodeSetEvent(ge.exec, ge.ev_stop, tp.b));
    }
    CK(cudaGraphLaunch(ge.exec, ctx->stream));
    if (timed)
        ctx->pending.push_back(tp);
    ctx->kernel_launches += ge.n_kernels;
    ctx->vote_launches += ge.n_vote_kernels;
    if (ctx->own_stream)
        return collect_device_errors(ctx);
    return GLCM_OK;
}

extern "C" int glcm_compute_batch(glcm_ctx* ctx, const glcm_desc* descs, int n)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (n < 0 || (n > 0 && !descs))
        return fail(ctx, GLCM_ERR_ARG, "bad batch");
    if (n == 0)
        return GLCM_OK;
    bool all_dev = true, any_dev = false;
    for (int i = 0; i < n; ++i) {
        const glcm_desc& d = descs[i];
        TRY(check_image_args(ctx, d.image, d.width, d.height, d.pitch_bytes, d.dtype, d.levels, d.offsets,
                             d.n_offsets));
        if (!d.counts)
            return fail(ctx, GLCM_ERR_ARG, "desc %d: counts is NULL", i);
        const bool dv = is_device_ptr(d.image) && is_device_ptr(d.counts) &&
                        (!d.normalized || is_device_ptr(d.normalized)) && (!d.features || is_device_ptr(d.features));
        all_dev &= dv;
        any_dev |= dv;
    }
    if (!all_dev && n > 1)
        return run_host_batch(ctx, descs, n);
    if (!all_dev) {
        // One image with host buffers: the stripe pipeline.
        for (int i = 0; i < n; ++i) {
            const glcm_desc& d = descs[i];
            const int fl = d.flags | (d.normalized ? GLCM_NORMALIZE : 0);
            TRY(glcm_compute(ctx, d.image, d.width, d.height, d.pitch_bytes, d.dtype, d.levels, d.offsets,
                             d.n_offsets, fl, d.counts, d.normalized));
            if (d.features)
                TRY(glcm_features(ctx, d.counts, d.levels, d.n_offsets, d.flags & GLCM_SYMMETRIC, d.features));
        }
        return GLCM_OK;
    }
    return run_graph_batch(ctx, descs, n, {}, std::string());
}

extern "C" int glcm_enqueue_batch(glcm_ctx* ctx, const glcm_desc* descs, int n)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (n < 0 || (n > 0 && !descs))
        return fail(ctx, GLCM_ERR_ARG, "bad batch");
    if (n == 0)
        return GLCM_OK;
    for (int i = 0; i < n; ++i) {
        const glcm_desc& d = descs[i];
        TRY(check_image_args(ctx, d.image, d.width, d.height, d.pitch_bytes, d.dtype, d.levels, d.offsets,
                             d.n_offsets));
        if (!d.counts)
            return fail(ctx, GLCM_ERR_ARG, "desc %d: counts is NULL", i);
        if (!is_device_ptr(d.image) || !is_device_ptr(d.counts) || (d.normalized && !is_device_ptr(d.normalized)) ||
            (d.features && !is_device_ptr(d.features)))
            return fail(ctx, GLCM_ERR_ARG, "desc %d: glcm_enqueue_batch takes device pointers only", i);
    }
    SplitBatch sb;
    TRY(prepare_batch(ctx, descs, n, sb, ctx->jobs, ctx->offs, ctx->feat));
    return enqueue_batch(ctx, sb, ctx->jobs, ctx->offs, ctx->feat, false, nullptr);
}

extern "C" int glcm_histogram(glcm_ctx* ctx, const void* image, int width, int height, size_t pitch_bytes,
                              int dtype, int levels, int flags, uint32_t* hist)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    const glcm_offset unit{1, 0};
    TRY(check_image_args(ctx, image, width, height, pitch_bytes, dtype, levels, &unit, 1));
    if (levels > GLCM_MAX_LEVELS)
        return fail(ctx, GLCM_ERR_UNSUPPORTED, "histograms need levels <= %d", GLCM_MAX_LEVELS);
    if (!hist)
        return fail(ctx, GLCM_ERR_ARG, "hist is NULL");
    if ((long long)width * height > 0xFFFFFFFFll)
        return fail(ctx, GLCM_ERR_ARG, "more than 2^32 - 1 pixels (uint32 counts)");
    const int bpp = dtype == GLCM_U8 ? 1 : 2;
    const bool dev_img = is_device_ptr(image);
    const bool dev_h = is_device_ptr(hist);
    const uint8_t* d_img = static_cast<const uint8_t*>(image);
    size_t dpitch = pitch_bytes;
    if (!dev_img) {
        std::vector<int> cut{height};
        TRY(stage_host_image(ctx, image, width, height, pitch_bytes, bpp, ctx->img, dpitch, cut));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->stripe_events[0], 0));
        d_img = static_cast<const uint8_t*>(ctx->img.p);
    }
    uint32_t* d_h = hist;
    if (!dev_h) {
        TRY(ensure(ctx, ctx->counts, (size_t)levels * 4));
        d_h = static_cast<uint32_t*>(ctx->counts.p);
    }
    CK(cudaMemsetAsync(d_h, 0, (size_t)levels * 4, ctx->stream));
    const long long row_bytes = (long long)width * bpp;
    HistParams hp{};
    hp.img = d_img;
    hp.pitch = (long long)dpitch;
    hp.flat = (dpitch == (size_t)row_bytes || height == 1) ? 1 : 0;
    hp.row_bytes = hp.flat ? row_bytes * height : row_bytes;
    hp.seg_bytes = histogram_seg_bytes();
    hp.segs = (row_bytes + hp.seg_bytes - 1) / hp.seg_bytes;
    hp.units = hp.segs * height;
    hp.bpp = bpp;
    hp.levels = levels;
    hp.levels_mode = (flags & GLCM_INPUT_LEVELS) ? 1 : 0;
    hp.hist = d_h;
    hp.err = ctx->d_words;
    CK(launch_histogram(hp, ctx->sm_count, ctx->stream));
    ctx->kernel_launches += 1;
    if (!dev_h)
        CK(cudaMemcpyAsync(hist, d_h, (size_t)levels * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->own_stream || !dev_img || !dev_h)
        return collect_device_errors(ctx);
    return GLCM_OK;
}


extern "C" int glcm_windows(glcm_ctx* ctx, const void* image, int width, int height, size_t pitch_bytes, int dtype,
                            int levels, int win, int stride, const glcm_offset* offsets, int n_offsets, int flags,
                            uint32_t* counts, float* maps)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    TRY(check_window_args(ctx, image, width, height, pitch_bytes, dtype, levels, win, stride, offsets, n_offsets,
                          counts, maps));
    const int bpp = dtype == GLCM_U8 ? 1 : 2;
    const int nwx = (width - win) / stride + 1, nwy = (height - win) / stride + 1;
    const size_t nn = (size_t)levels * levels;
    const size_t n_counts = (size_t)nwx * nwy * n_offsets * nn;
    const size_t n_maps = (size_t)GLCM_N_WINDOW_MAPS * n_offsets * nwx * nwy;
    const bool dev_img = is_device_ptr(image);
    const bool dev_c = counts && is_device_ptr(counts);
    const bool dev_m = maps && is_device_ptr(maps);
    const uint8_t* d_img = static_cast<const uint8_t*>(image);
    size_t dpitch = pitch_bytes;
    if (!dev_img) {
        std::vector<int> cut{height};
        TRY(stage_host_image(ctx, image, width, height, pitch_bytes, bpp, ctx->img, dpitch, cut));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->stripe_events[0], 0));
        d_img = static_cast<const uint8_t*>(ctx->img.p);
    }
    uint32_t* d_c = counts;
    float* d_m = maps;
    if (counts && !dev_c) {
        TRY(ensure(ctx, ctx->counts, n_counts * 4));
        d_c = static_cast<uint32_t*>(ctx->counts.p);
    }
    if (maps && !dev_m) {
        TRY(ensure(ctx, ctx->maps, n_maps * 4));
        d_m = static_cast<float*>(ctx->maps.p);
    }
    WindowParams wp{};
    TRY(window_params(ctx, d_img, dpitch, width, height, dtype, levels, win, stride, offsets, n_offsets, flags, d_c,
                      d_m, wp));
    (void)bpp;
    (void)nwx;
    (void)nwy;
    TRY(enqueue_windows(ctx, std::vector<WindowParams>{wp}, ctx->stream, false, nullptr));
    if (counts && !dev_c)
        CK(cudaMemcpyAsync(counts, d_c, n_counts * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (maps && !dev_m)
        CK(cudaMemcpyAsync(maps, d_m, n_maps * 4, cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->own_stream || !dev_img || (counts && !dev_c) || (maps && !dev_m))
        return collect_device_errors(ctx);
    return GLCM_OK;
}

extern "C" int glcm_compute_batch_windows(glcm_ctx* ctx, const glcm_desc* descs, int n, const glcm_window_desc* wins,
                                          int n_win)
{
    if (!ctx)
        return GLCM_ERR_ARG;
    cudaSetDevice(ctx->device);
    if (n < 0 || n_win < 0 || (n > 0 && !descs) || (n_win > 0 && !wins))
        return fail(ctx, GLCM_ERR_ARG, "bad batch");
    for (int i = 0; i < n; ++i) {
        const glcm_desc& d = descs[i];
        TRY(check_image_args(ctx, d.image, d.width, d.height, d.pitch_bytes, d.dtype, d.levels, d.offsets,
                             d.n_offsets));
        if (!d.counts)
            return fail(ctx, GLCM_ERR_ARG, "desc %d: counts is NULL", i);
        if (!is_device_ptr(d.image) || !is_device_ptr(d.counts) || (d.normalized && !is_device_ptr(d.normalized)) ||
            (d.features && !is_device_ptr(d.features)))
            return fail(ctx, GLCM_ERR_ARG, "desc %d: glcm_compute_batch_windows takes device buffers only", i);
    }
    std::vector<WindowParams> wps(n_win);
    std::string wkey = "W";
    for (int k = 0; k < n_win; ++k) {
        const glcm_window_desc& w = wins[k];
        TRY(check_window_args(ctx, w.image, w.width, w.height, w.pitch_bytes, w.dtype, w.levels, w.win, w.stride,
                              w.offsets, w.n_offsets, w.counts, w.maps));
        if (!is_device_ptr(w.image) || (w.counts && !is_device_ptr(w.counts)) || (w.maps && !is_device_ptr(w.maps)))
            return fail(ctx, GLCM_ERR_ARG, "window %d: glcm_compute_batch_windows takes device buffers only", k);
        TRY(window_params(ctx, static_cast<const uint8_t*>(w.image), w.pitch_bytes, w.width, w.height, w.dtype,
                          w.levels, w.win, w.stride, w.offsets, w.n_offsets, w.flags, w.counts, w.maps, wps[k]));
        char buf[256];
        snprintf(buf, sizeof buf, "%p,%d,%d,%zu,%d,%d,%d,%d,%d,%p,%p|", w.image, w.width, w.height, w.pitch_bytes,
                 w.dtype, w.levels, w.win, w.stride, w.flags, (void*)w.counts, (void*)w.maps);
        wkey += buf;
        for (int o = 0; o < w.n_offsets; ++o) {
            snprintf(buf, sizeof buf, "%d:%d;", w.offsets[o].dx, w.offsets[o].dy);
            wkey += buf;
        }
    }
    if (n == 0 && n_win == 0)
        return GLCM_OK;
    return run_graph_batch(ctx, descs, n, wps, wkey);
}
