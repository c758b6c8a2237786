// hmi_internal.cuh -- device data structures and launch entry points shared by
// the CUDA translation units of libhmi.so.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "hmi.h"
#include "hmi_queue.h"

namespace hmi {

// ---------------------------------------------------------------------------
// Geometry constants
// ---------------------------------------------------------------------------
constexpr int kChunkPx = 16;       // pixels per classification unit (48 frame bytes)
constexpr int kWordPx = 32;        // pixels per mask bit word
constexpr int kBlock = 32;         // connected-component block: 32 rows x 32 px
constexpr int kSlots = 256;        // max 8-connected components in a 32x32 block
constexpr int kMorphTW = 8;        // morphology tile width in words (256 px)
constexpr int kMorphRows = 32;     // morphology tile height (one CC block row)
constexpr int kMaxHalo = 32;       // 2 * (open_iters + close_iters) <= 32
constexpr int kStripMaxHalo = 8;   // register strips handle halos up to 8 rows
constexpr int kTickMaxHalo = 4;    // ... and up to 4 rows inside the persistent tick
constexpr int kMaxDim = 8192;
constexpr int kMaxBatch = 4096;
constexpr uint32_t kLoopLimit = 1u << 22;  // bound on every device-side retry loop

// device error flags (StreamState::err / batch error word)
constexpr uint32_t kErrUnionLoop = 1u;
constexpr uint32_t kErrFindLoop = 2u;
constexpr uint32_t kErrSlots = 4u;
constexpr uint32_t kErrRoot = 8u;
constexpr uint32_t kErrBounds = 32u;   // debug builds: an index failed its bounds check

// Bounds check of a computed index in debug builds (compiled with HMI_DEBUG):
// false, with kErrBounds recorded in *err, when cond fails, so that the caller
// skips the access; the kernel goes on (no trap).  Always true otherwise.
#ifdef HMI_DEBUG
#define HMI_IN_BOUNDS(cond, err) ((cond) ? true : (atomicOr((err), kErrBounds), false))
#else
#define HMI_IN_BOUNDS(cond, err) true
#endif

// One 8-connected component of a 32x32 block, later the accumulator of its
// whole component when it is the root.  64 bytes.
struct __align__(16) Comp {
    uint32_t key;                 // smallest linear index y*w + x of its pixels
    uint32_t area;
    unsigned long long sx, sy;    // sums of x and y
    int32_t x0, y0, x1, y1;       // inclusive box
    uint32_t top, bot, left, right;  // its pixels on the block's 4 borders
    uint32_t pad[2];
};
static_assert(sizeof(Comp) == 64, "Comp layout");

// Mutable per-stream state in device memory.
struct __align__(16) StreamState {
    unsigned long long sy;        // luma sum of the frame being processed (0 between frames)
    unsigned long long syref;     // reference luma of the background
    unsigned long long best;      // packed (area, ~key) argmax (0 between frames)
    unsigned long long learn_luma;  // luma total over the learning frames
    uint32_t gain;                // Q16 gain of the last frame
    uint32_t gain_p[3];           // Q16 gain of the frame of each tick phase (kPhases)
    uint32_t err;                 // kErr* flags
    int32_t click;
    int32_t hist_count;
    int32_t hist_head;
    int32_t frames;               // frames processed since learning
    uint32_t lframes;             // frames whose gain was computed since learning
    uint32_t lframe_p[3];         // the number of the frame of each tick phase (kPhases)
    int32_t track_valid, track_x, track_y;   // tracked point: last valid pointer's rounded centroid
    uint32_t nlearn;              // learning frames of the background (set when the band is formed)
    uint32_t last_phase;          // tick phase of the last finished frame (its bits give the labels)
    hmi_event event;              // the Interface module's event of the last frame
    hmi_pointer last;             // pointer of the last frame
};

// Gaussian mixture background of a stream (bg_model 1): 6 K fields of uint16
// per pixel, W[k] (Q15), M[k][c] (Q8), V[k] (Q4), C[k], stored by tiles of 32
// pixels of a row (one mask word): tile (y, x / 32) holds, field after field,
// the 32 pixels' values, so that a warp's pixel state is one contiguous block
// and every field is at a fixed offset from it.
struct MixView {
    uint16_t *planes;
    int K;                        // components per pixel; 0: a band stream
    int tiles_x;                  // tiles per row (the row's mask words)
    int rate_n, bg_pct;           // N (rates 1/min(., N)) and T in percent
    uint32_t lam_a, lam_b;        // match iff lam_a * d2 <= lam_b * V (kd^2, 3 kn^2 4096)
    uint32_t v_init, v_min;       // 16 sigma0^2 and 16 sigma_min^2
    unsigned long long recip_n;   // recip40(2N): rounded division by N in one multiply
};

// First entry of the 32-pixel tile holding pixel (x, y) of a mixture.
__host__ __device__ inline size_t mix_tile(const MixView &G, int x, int y)
{
    return ((size_t)y * G.tiles_x + (size_t)(x >> 5)) * (size_t)(6 * G.K) * 32u;
}

// Division by a divisor shared by many numerators, by one multiply: with
// R = ceil(2^40 / d) and 2 <= d < 2^18, 2^40 <= R d <= 2^40 + 2^18, so
// floor(n R / 2^40) = floor(n / d) for every n < 2^22 (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994,
// Theorem 4.2 with N = 22, l = 18).
__host__ __device__ inline unsigned long long recip40(uint32_t d)
{
    return ((1ull << 40) + d - 1) / d;
}

// Read-only description of a stream as the kernels see it.
struct DevStream {
    int w, h;
    int nwords;                   // ceil(w / 32): bit words per row == CC blocks per block-row
    int bh;                       // ceil(h / 32): CC block rows
    int tiles_x;                  // ceil(nwords / kMorphTW)
    int strips_x;                 // ceil(nwords / 30): register-strip tiles per block-row
    int fpitch;                   // bytes per row of the band (and of the staging frame)
    uint32_t cpr_magic;           // ceil(2^32 / (2 * nwords)): row of chunk u = umulhi(u, magic)
    int gray_tol;
    int open_iters, close_iters;
    uint32_t gain_min, gain_max, min_area;
    int click_on, click_off, click_window;
    // hue arc per sector (0: R max, 1: G max, 2: B max) as two half-open
    // intervals of N = 512 (t + d) + d:  d*A <= N < d*B
    int hueA[3][2], hueB[3][2];
    uint8_t *lo, *hi;             // background band, pitch fpitch, RGB interleaved
    // re-learning (relearn_frames 0: off): window parameters and the sums,
    // pixel-major RGB over rows of rpitch pixels (a multiple of 16)
    int relearn_period, relearn_frames, relearn_min, rpitch;
    int bg_kn, bg_kd, bg_delta;   // band parameters (k = kn / kd, margin delta)
    int track_max_dist;           // 0: the hand is the largest blob; else tracked
    const hmi_interface *ui;      // zones and wheel (all zero: none)
    MixView mix;                  // Gaussian mixture (mix.K 0: the band test)
    uint16_t *rS;                 // sum of corrected values, per pixel-channel
    uint32_t *rQ;                 // sum of their squares
    uint8_t *rmin, *rmax;         // their min and max
    uint8_t *rcnt;                // background frames counted, per pixel
    uint32_t *raw[3];             // raw AND mask bits, (bh*32) x nwords words, by tick phase
    // bits, count and flag are those of one tick phase (the plan keeps a
    // descriptor table per phase; *_p hold every phase's buffers)
    uint32_t *bits;               // mask bits after morphology, same layout
    Comp *comp;                   // bh*nwords*kSlots records
    uint32_t *parent;             // union-find parent per record
    uint32_t *count;              // components per CC block
    uint32_t *flag;               // per CC block: listed for components this tick
    uint32_t *bits_p[3], *count_p[3], *flag_p[3];
    StreamState *st;
    uint32_t *hist;               // click_window areas (ring)
};

// Row of chunk u of a stream with cpr chunks per row: with m = ceil(2^32 / cpr)
// = (2^32 + e) / cpr, 0 <= e < cpr, u m / 2^32 = u / cpr + u e / (cpr 2^32),
// and the second term stays below 1 / cpr whenever u cpr < 2^32, so the high
// word of u m is floor(u / cpr).  Here u < h cpr and cpr <= 512, h <= 8192.
__device__ __forceinline__ int chunk_row(uint32_t u, uint32_t magic)
{
    return (int)__umulhi(u, magic);
}

// Per-tick pointers of one stream.
struct TickIO {
    const uint8_t *frame;         // frame of this tick
    long long frame_pitch;        // bytes between rows of `frame`
    const uint8_t *src;           // a pinned host frame (device-accessible address, dense
                                  // rows of 3 w bytes, w a multiple of 16) that k_luma
                                  // copies into `frame` as it sums it; null: none
    uint8_t *mask;                // h*w mask out (device) or null
    hmi_pointer *ptr_out;         // pointer out (device) or null
};

// Everything a tick's kernels need, passed by value.
struct BatchDev {
    const DevStream *ds;
    const TickIO *io;
    int n;
    unsigned long long total_chunks;          // sum h * 2 * nwords
    uint32_t total_tiles;                     // sum bh * tiles_x
    uint32_t total_blocks;                    // sum bh * nwords
    const unsigned long long *chunk_prefix;   // n + 1 entries
    const uint32_t *tile_prefix;              // n + 1
    const uint32_t *strip_prefix;             // n + 1
    uint32_t total_strips;                    // sum bh * strips_x
    int max_halo;                             // largest 2 * (open + close) of the batch
    int uniform_halo;                         // the common 2 * (open + close), or -1
    const uint32_t *block_prefix;             // n + 1
    uint32_t *done;                           // last-block counters [4]
    const int4 *pieces;                       // (stream, chunk begin, chunk end, 0)
    int npieces;                              // pieces of the per-pixel kernels
    uint32_t *err;                            // batch error word: OR of the streams' flags
    uint32_t *cc_count;                       // non-empty blocks listed this tick
    uint2 *cc_list;                           // (stream, block) of each, total_blocks slots
    uint32_t *skin_count;                     // chunks queued for the skin tests this tick
    uint2 *skin_list;                         // ((stream << 16) | bits, chunk), total_chunks slots
    int phase;                                // tick phase (slot mod kPhases): selects raw[],
                                              // gain_p[] and the skin queue, so that up to
                                              // kPhases consecutive ticks can be in flight
    // launch shape (host side; chosen by the plan's tuning)
    int relearn;                              // some stream of the batch re-learns
    int any_band;                             // some stream has the band test
    int any_mix;                              // bit K: some stream has a K-component mixture
    uint32_t loop_limit;                      // steps of every bounded device loop (0: kLoopLimit)
    int merge_threads;                        // threads of a stream's merge CTA (256, 512, 1024)
    // tick form of the per-pixel kernels: 0 the chain, 1 the persistent tick
    // (queue below), 2 the cooperative per-pixel stage (counters done[2..3])
    int fused;
    const int4 *items;                        // work queue, in order
    int nitems;
    TickSync *sync;                           // per stream
    uint32_t *tick_head;                      // next item to take
    uint32_t *tick_exit;                      // CTAs that have left the launch
    int luma_ctas_per_sm;                     // 0: as many as fit (also the persistent grid)
    int skin_ctas_per_sm;
    int cc_ctas_per_sm;
};

// Consecutive ticks in flight at once at most (pipelined ticks), and so the
// number of copies of the per-tick state they would otherwise share.
constexpr int kPhases = 3;

// Threads per CTA of every kernel of a tick.
constexpr int kThreads = 256;

// Records `status` as the calling thread's last error (hmi_last_error) and
// returns it (hmi_api.cu).
int set_error(int status);

// An NVTX range over a host scope (a learning call, a tick, a server round,
// the enqueue of a tick kernel), so that a timeline tool shows the stages.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Name of tick kernel k (kernel order of a tick, see kTickKernels).
inline const char *tick_kernel_name(int k)
{
    static const char *names[] = {"hmi luma",    "hmi classify",  "hmi mixture",
                                  "hmi relearn", "hmi relearn band", "hmi skin",
                                  "hmi morphology", "hmi block components", "hmi merge"};
    return (k >= 0 && k < 9) ? names[k] : "hmi kernel";
}

// ---------------------------------------------------------------------------
// Launchers (hmi_frame.cu, hmi_cc.cu, hmi_learn.cu)
// ---------------------------------------------------------------------------
// The kernels of one tick, in order: 0 luma (and gains), 1 classify (band
// test), 2 mixture test and update (no launch without mixture streams), 3
// re-learning sums and 4 re-learned bands (no launch unless a stream of the
// batch re-learns), 5 skin (gray and hue tests), 6 morphology, 7 block
// components (none on the generic morphology path, which labels its blocks
// itself), 8 finish.
constexpr int kTickKernels = 9;
constexpr int kTickTail = 5;       // first kernel of the latency-bound tail (skin)
static_assert(kTickKernels == HMI_TICK_KERNELS, "tick kernel count");
cudaError_t launch_luma(const BatchDev &b, cudaStream_t cs, int num_sms);
cudaError_t launch_classify(const BatchDev &b, cudaStream_t cs, int num_sms);
cudaError_t launch_skin(const BatchDev &b, cudaStream_t cs, int num_sms);
cudaError_t launch_relearn(const BatchDev &b, cudaStream_t cs, int num_sms);
cudaError_t launch_relearn_band(const BatchDev &b, cudaStream_t cs, int num_sms);
cudaError_t launch_mix(const BatchDev &b, cudaStream_t cs, int num_sms);
// The mixture update of nf dense learning frames (h*w*3 bytes each), frame i
// being frame number t0 + i + 1 of the stream.
cudaError_t launch_mix_learn(const uint8_t *frames, int nf, uint32_t t0, int w, int h,
                             const MixView &mix, cudaStream_t cs);

// Frame f (counted from 1 after learning) is in a re-learning window iff
// (f - 1) mod period >= period - frames; the window ends with f mod period == 0.
__host__ __device__ inline bool relearn_window(uint32_t f, int period, int frames)
{
    return frames > 0 && period > 0 && f > 0 && (int)((f - 1) % (uint32_t)period) >= period - frames;
}
cudaError_t launch_morph(const BatchDev &b, cudaStream_t cs, int num_sms);
// The persistent tick (hmi_tick.cu), and the CTAs per SM its grid has for a
// requested number (0: as many as fit).
cudaError_t launch_tick(const BatchDev &b, cudaStream_t cs, int num_sms);
int tick_ctas_per_sm(int requested);
cudaError_t launch_block_cc(const BatchDev &b, cudaStream_t cs, int num_sms);
cudaError_t launch_finish(const BatchDev &b, cudaStream_t cs);
cudaError_t launch_tick_kernel(int k, const BatchDev &b, cudaStream_t cs, int num_sms);
cudaError_t launch_labels(const DevStream *ds_dev, const DevStream &ds, int32_t *labels,
                          cudaStream_t cs);

cudaError_t launch_learn_accum(const uint8_t *frames, int nf, long long npx, uint32_t *S,
                               uint32_t *Q, uint8_t *vmin, uint8_t *vmax, int first,
                               StreamState *st, cudaStream_t cs);
// One learning frame of a stream, for k_learn_batch: frame (device-accessible,
// packed rows, npx % 4 == 0, 4-byte aligned), the stream's sums, first frame
// or not, and its first quad (4 pixels) in the launch.
struct LearnItem {
    const uint8_t *frame;
    uint32_t *S, *Q;
    uint8_t *vmin, *vmax;
    StreamState *st;
    unsigned long long quad0;
    int first;
};
cudaError_t launch_learn_batch(const LearnItem *items, int nitems, unsigned long long total_quads,
                               cudaStream_t cs);
cudaError_t launch_learn_band(const uint32_t *S, const uint32_t *Q, const uint8_t *vmin,
                              const uint8_t *vmax, int n, int kn, int kd, int delta, int w,
                              int h, int fpitch, uint8_t *lo, uint8_t *hi, StreamState *st,
                              cudaStream_t cs);
cudaError_t launch_stats(const uint32_t *S, const uint32_t *Q, int n, long long count,
                         float *mean, float *stdv, cudaStream_t cs);

}  // namespace hmi
