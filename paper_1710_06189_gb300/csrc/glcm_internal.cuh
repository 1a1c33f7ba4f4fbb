// Internal structures shared by the host planner (glcm_capi.cu) and the
// kernels.  Not part of the public ABI (include/glcm.h is).
#pragma once
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

struct glcm_ctx;  // the context (glcm_capi.cu; opaque in the public header)

namespace glcm {

// Fast-path horizontal reach: a lane holds its own pixels plus one word of
// quantized levels (4 levels) from each neighbouring lane.
constexpr int kFastMaxDx = 4;
// Largest dy_max - dy_min a staged job may have (tile halo rows).
constexpr int kMaxDySpan = 16;
constexpr int kMaxThreads = 1024;
// Bounded spin limit for any device-side wait (none on the vote path today;
// kept for the persistent serving kernels).
constexpr long long kSpinLimit = 1ll << 26;

// Device error bits written into the context's error word.
enum : unsigned {
    kErrRange = 1u,     // a pixel >= N in levels mode (pair skipped)
    kErrInternal = 2u,  // an index check failed inside a kernel (access skipped)
    kErrTimeout = 4u,   // a bounded wait gave up
};

// One histogram target: one image and the group of offsets voted together.
struct VoteJob {
    const uint8_t* img;
    long long pitch;   // bytes between rows
    int W, H;
    int bpp;           // 1 (uint8) or 2 (uint16)
    int levels;        // N
    int log2n;         // log2(N) if N is a power of two, else -1
    int levels_mode;   // pixels already are levels (< N)
    int aligned;       // base and pitch are 16-byte aligned
    int n_off;         // offsets in this job
    int off0;          // first entry in the offsets table
    int rshift;        // log2(copies): R = 1 << rshift private copies
    int layout;        // 0: R words per bin; 1: two offsets' R words interleaved
                       // per bin; 2: two offsets as 16-bit halves of R words;
                       // 3: partner levels j and j + ceil(N/2) of one offset as
                       // 16-bit halves of R words
    int bytecode;      // N <= 16 power of two, layout 1, R = 32, no level split
    int lv_lo, lv_span;  // anchor levels [lv_lo, lv_lo + lv_span) counted
    int hist_words;    // shared words this job uses
    int item0;         // first work item of this job in the launch
    int n_job_items;   // work items of this job
    int chunk_items;   // items per scheduling chunk
    int n_strips;      // column strips of 32 lanes x 16 bytes
    int band_rows;     // anchor rows per work item
    int y_begin, y_end;  // anchor rows voted by this job ([0, H) for a whole image)
    int dy_min, dy_max;  // min(0, dy) and max(0, dy) over the job's offsets
    int staged;          // tiles go through shared memory (dy_max - dy_min <= kMaxDySpan)
    uint32_t* out;     // counts: offset slot s at out + s*N*N
};

struct VoteOffset {
    int dx, dy;
    int slot;          // output GLCM index within the job
    int pad;
};

// A work item: one column strip (32 lanes x 16 bytes) of one job and a band
// of anchor rows; item k of job j is strip (k - item0) % n_strips of band
// (k - item0) / n_strips.
struct VoteItem {
    int job, x0, y0, y1;
};

struct VoteParams {
    const VoteJob* jobs;
    int n_jobs;
    const VoteOffset* offs;
    int n_items;
    const int3* chunks;      // (job, first item, end item), job-major order
    int n_chunks;
    int tile_bytes;          // one staged tile buffer (two are allocated)
    int max_hist_words;
    unsigned* item_counter;  // chunk counter, zeroed before each launch
    unsigned* err;           // error bits (kErr*)
};

// Column-walk vote kernel (vote_fast.cu) for offsets at chessboard distance 1.
// The canonical offsets are k = 0: (1, 0), 1: (1, -1), 2: (0, -1), 3: (-1, -1)
// (partner to the right or in the row above); every offset at distance 1 is
// one of them or its opposite, whose GLCM is the transpose (an anchor of one
// is the partner of the other).
constexpr int kFastOffsets = 4;
enum : int {
    kFastJoint = 0,  // N <= 8, all four offsets: two joint votes per anchor
    kFastPair = 1,   // N <= 16: one vote per anchor and offset, two offsets per bin row
    kFastHalf = 2,   // N = 32: up to two offsets as 16-bit halves of one word
    kFastWide = 3,   // N = 256: one offset, 128 rows of the GLCM as 32-bit counters
};

struct FastJob {
    const uint8_t* img;
    long long pitch;   // bytes between rows
    int W, H;
    int bpp;           // 1 or 2
    int log2n;         // N = 2^log2n: 1..5, or 8
    int mode;          // kFast*
    int present;       // bit k: canonical offset k is voted by this job
    int half_hi;       // kFastHalf: the offset (k) counted in the upper halves, or -1
    int aligned;       // base and pitch 16-byte aligned (one 16-byte load per lane and row)
    int row_half;      // kFastWide: GLCM rows [128 row_half, 128 row_half + 128) are counted
    int transposed;    // kFastWide: count the transpose (rows are partner levels)
    int slot[kFastOffsets];    // output GLCM of canonical offset k, or -1
    int slot_t[kFastOffsets];  // output GLCM that receives its transpose, or -1
    int hist_words;    // shared words of the job's histograms
    int item0;         // first item of this job in the launch
    int n_items;       // items: n_strips column strips x bands of band rows
    int n_strips;
    int band;
    int y_begin, y_end;  // anchor rows voted by this job
    int dist;          // partner distance D (1 .. 4): offsets (D, 0), (D, -D), (0, -D), (-D, -D)
    uint32_t* out;     // counts: GLCM s at out + s*N*N
};

struct FastParams {
    const FastJob* jobs;
    const int3* chunks;       // (job, first item, end item), job-major order
    int n_chunks;
    int max_hist_words;
    unsigned* chunk_counter;  // zeroed before each launch
    unsigned* err;
    int ring_words;           // shared words per warp for the row rings of distances > 1 (0: none)
};

// Flat-wrap pairs of one offset (GLCM_FLAT_WRAP): the anchors of rows
// [y_begin, y_end) whose partner column x + dx leaves [0, W), paired along the
// row-major buffer (seam.cu).
struct SeamJob {
    const uint8_t* img;
    long long pitch;
    int W, H, bpp, levels, levels_mode;
    int dx, dy;
    int y_begin, y_end;
    uint32_t* out;  // this offset's N x N counts
};

// Epilogue: symmetrize / normalize / Haralick features for one GLCM.
struct FeatJob {
    const uint32_t* counts;  // N*N
    float* normalized;       // N*N or null
    float* features;         // 14 or null
    int levels;
    int symmetric;
};

struct FeatParams {
    const FeatJob* jobs;
    int n_jobs;
    float* work;             // scratch for large-N singular value sweeps
    long long work_stride;   // floats per job in `work`
    unsigned* err;
};

// Sliding-window local GLCMs.
struct WindowParams {
    const uint8_t* img;
    long long pitch;
    int W, H, bpp, levels, levels_mode;
    int win, stride, nwx, nwy;
    int n_off;
    int dx[8], dy[8];
    int symmetric;
    uint32_t* counts;   // nwy*nwx*n_off*N*N or null
    float* maps;        // 4*n_off*nwy*nwx or null  [map][offset][wy][wx]
    unsigned* err;
    const long long* slide_tables;  // kSlideTableWords fixed-point terms (incremental kernel) or null
};

// Fixed-point tables of the incremental window kernel (scale 2^40), made on
// the host in float64: g(c) = (c + 1) ln(c + 1) - c ln c for c < 512, its
// prefix sums t ln t for t <= 512, and 1 / (1 + d^2) for d < 32.
constexpr int kSlideG = 512;
constexpr int kSlideTableWords = kSlideG + (kSlideG + 1) + 32;
void window_slide_tables(long long* out);

// Gray-level histogram of one image (histogram.cu).
struct HistParams {
    const uint8_t* img;
    long long pitch;      // bytes between rows (pitched mode)
    long long row_bytes;  // bytes of one row, or of the whole image when flat
    long long seg_bytes;  // row segment a warp takes (pitched mode; multiple of 16)
    long long segs;       // segments per row (pitched mode)
    long long units;      // rows * segs (pitched mode)
    int flat;             // the image is one contiguous span of row_bytes
    int bpp, levels, levels_mode;
    uint32_t* hist;       // levels counts, zeroed before the launch and added into
    unsigned* err;
};

// The dynamic shared-memory limit of one kernel, raised per device
// (cudaFuncSetAttribute applies to the current device's context): the
// attribute is set only when a launch needs more than was set on the current
// device before, so once an uncaptured launch of a size has run, no attribute
// call happens inside a later stream capture.  Thread-safe.
class SmemLimit {
public:
    static constexpr int kMaxDevices = 64;
    cudaError_t raise(const void* fn, size_t smem)
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess)
            return e;
        if (dev < 0 || dev >= kMaxDevices)
            return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        std::lock_guard<std::mutex> g(m_);
        if (smem <= set_[dev])
            return cudaSuccess;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            set_[dev] = smem;
        return e;
    }

private:
    std::mutex m_;
    size_t set_[kMaxDevices] = {};
};

// Launchers (defined in the .cu files).
// packed: some job of the launch uses layout 3 (a separate kernel instance).
cudaError_t launch_vote(const VoteParams& p, int bpp, int grid, int threads, size_t smem,
                        cudaStream_t s, bool packed = false);
// Column-walk votes: one launch per pixel type and N (every job of the launch
// has them).
cudaError_t launch_vote_fast(const FastParams& p, int bpp, int log2n, bool aligned, int grid, size_t smem,
                             cudaStream_t s);
size_t vote_fast_smem_bytes(int max_hist_words, int log2n, int ring_words);
int vote_fast_hist_words(int log2n, int mode);
// The column-walk kernel for rows at any byte address (vote_fast_unaligned.cu).
const void* vote_fast_kernel_unaligned(int bpp, int log2n);
cudaError_t launch_seams(const SeamJob* jobs, int n_jobs, int blocks_per_job, unsigned* err, cudaStream_t s);
// N > 256: every in-rectangle pair of each job (one offset of one image, its
// rows [y_begin, y_end)) voted into global counts (vote_global.cu).
cudaError_t launch_vote_global(const SeamJob* jobs, int n_jobs, int blocks_per_job, unsigned* err, cudaStream_t s);
cudaError_t launch_naive(const uint8_t* img, long long pitch, int W, int H, int bpp, int levels,
                         int levels_mode, int dx, int dy, uint32_t* out, unsigned* err,
                         cudaStream_t s);
// Threads per epilogue CTA: kFeatThreads, or kFeatThreadsSmall for the jobs
// with N <= kSmallFeatLevels.
constexpr int kFeatThreads = 512;
constexpr int kFeatThreadsSmall = 256;
constexpr int kSmallFeatLevels = 32;
// priority: 0, or a stream priority for this launch alone (lower is more urgent).
cudaError_t launch_features(const FeatParams& p, int max_levels, cudaStream_t s, int threads, int priority = 0);
// Symmetric feature jobs with 128 < N <= 256, one cluster of CTAs per GLCM.
cudaError_t launch_features_cluster(const FeatParams& p, cudaStream_t s, int priority = 0);
inline bool feat_job_clustered(const FeatJob& f)
{
    return f.features != nullptr && f.symmetric && f.levels > 128 && f.levels <= 256;
}
// Launch group of a feature job: 0 one small CTA (N <= 32), 1 one CTA,
// 2 a cluster of CTAs.
inline int feat_job_group(const FeatJob& f)
{
    return feat_job_clustered(f) ? 2 : (f.levels <= kSmallFeatLevels ? 0 : 1);
}
size_t features_smem_bytes(int max_levels);
long long features_work_floats(int levels);
cudaError_t launch_windows(const WindowParams& p, cudaStream_t s);
// The incremental window kernel (window_slide.cu); cudaErrorNotSupported when
// the windows do not fit it.
cudaError_t launch_windows_slide(const WindowParams& p, cudaStream_t s);
cudaError_t launch_histogram(const HistParams& p, int sm_count, cudaStream_t s);
long long histogram_seg_bytes();
int vote_max_smem_optin();
int vote_blocks_per_sm(int bpp, int threads, size_t smem, bool packed = false);
int vote_row_bytes();
// Host image rows to the device on `st` (a copy kernel for registered host
// memory, else cudaMemcpy(2D)Async); defined in glcm_capi.cu.
// max_ctas caps the copy kernel's grid.
cudaError_t copy_rows_to_device(void* dst, size_t dpitch, const void* src, size_t spitch, size_t row_bytes, int rows,
                                cudaStream_t st, bool allow_kernel = true, int max_ctas = 24);
// Every vote launch of `ctx` leaves `sms` SMs free (for a concurrent copy
// kernel; a vote CTA fills its SM's register file); defined in glcm_capi.cu.
void set_vote_sm_reserve(::glcm_ctx* ctx, int sms);

}  // namespace glcm
