/*
 * hmi.h -- C ABI of the GB300 hand-isolation library (libhmi.so).
 *
 * The library implements the per-frame path of the contactless interface of
 * Magoules & Zou (arXiv 1907.04393): learn a background with no hand in view
 * (Sec. 2, initialisation step), then for every camera frame correct the
 * brightness (Sec. 2, Sec. 3.2), build the three thresholded images and AND
 * them (Sec. 3.1 (i)-(iii)), clean the mask with erosion/dilation (Sec. 3.1),
 * and turn the hand zone into a pointer with a click state (Sec. 2, Mouse and
 * Interface modules).  Every step runs in hand-written sm_103a CUDA kernels;
 * there is no CPU fallback.
 *
 * Conventions (all calls):
 *   - Return value: HMI_OK (0) or a negative HMI_ERR_* status.  Functions that
 *     return a pointer return NULL on error; hmi_last_error() then gives the
 *     status (thread-local).
 *   - Frames are packed RGB8: h rows of 3*w bytes, pixel (x, y) at byte
 *     3*(y*w + x), channels in the order R, G, B.  Masks are h*w bytes (0/1),
 *     labels h*w int32.
 *   - Buffers passed in are owned by the caller.  A buffer may live in host
 *     memory (pageable or pinned) or in device memory of the stream's GPU;
 *     the library tells them apart with cudaPointerGetAttributes.  The library
 *     owns all per-stream device state.
 *   - Host frames are copied to the device (pinned host memory copies
 *     fastest); device frames whose width is a multiple of 16 and whose
 *     address is 16-byte aligned are read in place.
 *   - Synchronous calls return when results are in the caller's buffers.
 *     The *_async calls only enqueue work on the given CUDA stream
 *     (a cudaStream_t passed as void*, NULL = the legacy default stream) and
 *     require device buffers.
 *   - One hmi_stream is used by one host thread at a time.  Device-side errors
 *     (a bounded wait or bounded loop that ran out) surface as
 *     HMI_ERR_DEVICE_TIMEOUT on the next synchronous call on that stream.
 *   - Limits: 1 <= w, h <= 8192; 1 <= n (learning frames) <= 65535.
 */
#ifndef HMI_H
#define HMI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HMI_API __attribute__((visibility("default")))
#else
#define HMI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define HMI_OK 0
#define HMI_ERR_INVALID_ARG (-1)    /* null/odd pointer, size or parameter out of range */
#define HMI_ERR_NOT_LEARNED (-2)    /* processing before hmi_learn_background */
#define HMI_ERR_NO_MEMORY (-3)      /* device or host allocation failed, or admission refused */
#define HMI_ERR_DEVICE (-4)         /* a CUDA call failed */
#define HMI_ERR_DEVICE_TIMEOUT (-5) /* a bounded device-side wait/loop gave up */
#define HMI_LEARNING 1              /* server result only: the frame was taken as one of the
                                     * stream's background-learning frames (not an error;
                                     * its pointer is the empty pointer) */

/* Opaque per-camera stream: geometry, parameters, learned background model,
 * click state and device work buffers.  Created by hmi_create_stream. */
typedef struct hmi_stream hmi_stream;

/* User-adjustable thresholds (Sec. 2: the FIZI settings can be changed by
 * the user; Sec. 3.1: tolerance S and hue thresholds alpha1, alpha2 are set
 * by the user).  Defaults in brackets, set by hmi_default_params. */
typedef struct {
    uint32_t gain_min_q16;  /* [32768]  lower clamp of the brightness gain, Q16 (0.5) */
    uint32_t gain_max_q16;  /* [131072] upper clamp of the brightness gain, Q16 (2.0) */
    uint32_t min_area;      /* [50]     pointer valid iff the hand blob has >= min_area pixels */
    uint16_t hue_lo;        /* [1472]   alpha1, hue units (1536 per turn, 256 per 60 deg) */
    uint16_t hue_hi;        /* [256]    alpha2; hue_lo > hue_hi means the arc wraps through red */
    uint16_t click_window;  /* [30]     valid frames remembered for the click reference area (<= 1024) */
    uint8_t gray_tol;       /* [15]     S: pixels with max(RGB) - min(RGB) < S are gray, removed */
    uint8_t bg_margin;      /* [2]      delta added outside the learned background band */
    uint8_t bg_k_num;       /* [5]      band half-width k = bg_k_num / bg_k_den standard deviations */
    uint8_t bg_k_den;       /* [2]      (1..15; numerator 0..15) */
    uint8_t open_iters;     /* [1]      openings (erode, dilate) for noise removal */
    uint8_t close_iters;    /* [1]      closings (dilate, erode) to connect zones; open+close <= 16 */
    uint8_t click_on_pct;   /* [80]     click when 100*area < on_pct * reference area */
    uint8_t click_off_pct;  /* [90]     release when 100*area > off_pct * reference area */
    /* Re-learning (Sec. 3.3: part of the learning is restarted from time to
     * time as the lighting drifts).  Off when relearn_frames is 0.  Otherwise the last
     * relearn_frames frames of every relearn_period frames (counted from 1
     * after learning) add the gain-corrected values of their background
     * pixels to per-pixel sums; after the window each pixel counted at least
     * relearn_min times gets the band of those sums (the learning formula,
     * n = its count) and the sums restart.  1 <= relearn_min <= relearn_frames
     * <= relearn_period. */
    uint8_t relearn_frames; /* [0]      frames of a re-learning window (0: off) */
    uint8_t relearn_min;    /* [0]      background frames a pixel needs in a window */
    uint16_t relearn_period;/* [0]      frames from one window's end to the next */
    /* Tracking (Sec. 2: the Mouse module tracks the hand zone).  0: the hand
     * is the largest blob.  Otherwise, once a valid pointer has been seen,
     * the hand is the blob of at least min_area pixels whose bounding box is
     * nearest (L1 distance, 0 inside) the previous valid pointer's rounded
     * centroid, if within this many pixels (ties: larger area, then smaller
     * label); else the largest blob. */
    uint16_t track_max_dist;/* [0]      pixels */
    /* Background model (Sec. 2: FIZI's background is learned with advanced
     * machine learning; Sec. 3.3 cites Lee's adaptive Gaussian
     * mixture learning).  bg_model 0: the learned band above.  bg_model 1:
     * per pixel, mix_k Gaussian components over the gain-corrected RGB value,
     * each a weight W (Q15), a mean per channel M (Q8), one variance V
     * shared by the channels (Q4: level^2 * 16) and a match count C (0:
     * empty), kept in fitness order.  For frame t (counted from 1 over the
     * learning frames, which the mixture learns from an empty model, then the
     * running frames): the value matches the first non-empty component with
     * bg_k_den^2 * sum (256 c' - M)^2 <= 3 * bg_k_num^2 * V * 4096 (the mean
     * squared channel deviation within lambda^2 V, lambda = bg_k_num /
     * bg_k_den, as the band reads k per channel); on a running frame it is
     * background iff it matched component j and the weights before j sum to
     * at most mix_bg_pct percent of all weights (model before the update).
     * Update (Lee's rates, every division rounded half away from zero): the
     * matched component's C grows by one and, with r = min(C, mix_rate_n),
     * M moves by (256 c' - M) / r and V by (D / 3 - V) / r (D the squared
     * distance in Q4; V clamped to [16 mix_sigma_min^2, 65535]); with no
     * match the last component becomes (M = 256 c', V = 16 mix_sigma0^2,
     * C = 1, W = 0); then with m = min(t, mix_rate_n) every W moves by
     * (32768 [the matched or new one] or 0 [the others] - W) / m; finally
     * the components are stably re-sorted, non-empty ones first by
     * W / sqrt(V) (a before b iff W_a^2 V_b > W_b^2 V_a), empty ones last.
     * Requires relearn_frames 0 and bg_k_num >= 1; the band is still formed
     * from the learning frames (hmi_get_band) but not used. */
    uint8_t bg_model;       /* [0]      0: learned band, 1: Gaussian mixture */
    uint8_t mix_k;          /* [3]      components per pixel, 1..4 */
    uint8_t mix_bg_pct;     /* [70]     T: background share of the weights, 1..100 */
    uint8_t mix_sigma0;     /* [15]     standard deviation of a new component, 1..63 */
    uint8_t mix_sigma_min;  /* [2]      lower bound of a standard deviation, 1..mix_sigma0 */
    uint8_t mix_pad;        /* [0]      must be 0 */
    uint16_t mix_rate_n;    /* [256]    N: the learning rate alpha is 1 / N, 1..65535 */
} hmi_params;

/* The Mouse module's pointer (Sec. 2): position of the hand zone and
 * whether it is clicked.  With no foreground at all: valid 0, area 0,
 * label -1, box -1, x = y = -1. */
typedef struct {
    int32_t valid;    /* 1 iff the largest blob has at least min_area pixels */
    int32_t click;    /* click state after this frame (0/1) */
    float x, y;       /* centroid of the largest blob, pixel centres at integers */
    uint32_t area;    /* pixels in the largest blob */
    int32_t x0, y0;   /* inclusive bounding box of the largest blob */
    int32_t x1, y1;
    int32_t label;    /* the blob's label: smallest linear index y*w + x of its pixels */
} hmi_pointer;

/* Fill *p with the documented defaults.  HMI_ERR_INVALID_ARG if p is NULL. */
HMI_API int hmi_default_params(hmi_params *p);

/* Create a stream for w x h frames on the current CUDA device (Sec. 2,
 * initialisation: reading the configuration).  p may be NULL (defaults).
 * Allocates all device state up front.  NULL on error (invalid size or
 * parameters: HMI_ERR_INVALID_ARG; allocation: HMI_ERR_NO_MEMORY). */
HMI_API hmi_stream *hmi_create_stream(int w, int h, const hmi_params *p);

/* Release a stream and all of its device memory (NULL is a no-op).
 * Any batch that contains the stream must be destroyed first. */
HMI_API void hmi_destroy_stream(hmi_stream *s);

/* Learn the background model from n user-free frames (Sec. 2: FIZI's
 * background is learned before the hand enters; Sec. 3.1 (i): per-pixel
 * minimum and maximum).  frames: n consecutive packed RGB8 frames
 * (n*h*w*3 bytes), host or device.  Per pixel and channel the library keeps
 * the exact sums S, Q and the min / max, derives the background band and the
 * reference luma used by the brightness correction, and resets the click
 * state.  Replaces any earlier model. */
HMI_API int hmi_learn_background(hmi_stream *s, const uint8_t *frames, int n);

/* Run the whole per-frame path on one frame (Sec. 2 running step; Sec. 3.1,
 * 3.2): brightness gain, background / gray / hue masks, AND, morphology,
 * 8-connected components, largest blob, pointer and click state.
 * frame: h*w*3 bytes (host or device).  mask_out: h*w bytes or NULL.
 * pointer_out: one hmi_pointer or NULL.  HMI_ERR_NOT_LEARNED before learning. */
HMI_API int hmi_process_frame(hmi_stream *s, const uint8_t *frame, uint8_t *mask_out,
                      hmi_pointer *pointer_out);

/* Same work enqueued on cuda_stream; frame, mask_out and pointer_out must be
 * device memory (mask_out and pointer_out may be NULL). */
HMI_API int hmi_process_frame_async(hmi_stream *s, const uint8_t *frame, uint8_t *mask_out,
                            hmi_pointer *pointer_out, void *cuda_stream);

/* One frame for each of n streams (1 <= n <= 4096, all on the same device,
 * each stream at most once), processed by single launches that cover every
 * stream.  frames[i], masks[i] belong to s[i]; masks (or masks[i]) and
 * ptrs may be NULL.  ptrs, when given, is an array of n hmi_pointer.
 * The launch plan for a given list of streams is built on first use and
 * reused while the same list is passed again. */
HMI_API int hmi_process_batch(hmi_stream *const *s, int n, const uint8_t *const *frames,
                      uint8_t *const *masks, hmi_pointer *ptrs);

/* A reusable launch plan over a fixed list of streams (the batched form of
 * hmi_process_batch).  hmi_batch_create returns NULL on error. */
typedef struct hmi_batch hmi_batch;
HMI_API hmi_batch *hmi_batch_create(hmi_stream *const *s, int n);
HMI_API void hmi_batch_destroy(hmi_batch *b);

/* Concurrency of a launch plan.  The streams of a batch are dealt into
 * `groups` groups of about equal pixel count; each group's kernels form their
 * own chain, and the chains of a tick overlap (each group's luma pass starts
 * after the previous group's), so the bandwidth-bound passes of one group run
 * beside the latency-bound tail of another.  Default: min(2, n).  Changing it
 * rebuilds the plan (waits for the device).  Results do not depend on it. */
HMI_API int hmi_batch_set_groups(hmi_batch *b, int groups);
HMI_API int hmi_batch_get_groups(const hmi_batch *b);

/* Failure detection: the bound on every bounded device loop and wait of the
 * batch's ticks (union-find steps of the component merge, the persistent
 * tick's waits for a stream's earlier steps).  0 restores the default, 2^22.
 * A loop that runs out sets the stream's error flag and lets the tick end;
 * the next synchronous call returns HMI_ERR_DEVICE_TIMEOUT (that frame's
 * results are not to be trusted) and clears it.  Re-makes the plan (waits for
 * the device).  Lowering it lets a test make a loop run out without any fault. */
HMI_API int hmi_batch_set_loop_limit(hmi_batch *b, uint32_t limit);

/* Process one frame per stream of the batch.  Synchronous form: buffers may be
 * host or device; frames[i] is the frame of the i-th stream given at creation.
 * masks / ptrs as in hmi_process_batch.  A frame in pinned (page-locked) host
 * memory whose stream width is a multiple of 16 and whose address is 16-byte
 * aligned is read over the host link by the luma pass itself, which stores it
 * into a device staging frame as it sums it (one pass, no copy engine); other
 * host frames are copied first.  The batch remembers the pinned buffers it has
 * seen: they must stay pinned while the batch may be given them. */
HMI_API int hmi_batch_process(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
                      hmi_pointer *ptrs);

/* Asynchronous form on cuda_stream: every buffer must be device memory, except
 * frames, which may also be pinned host memory read in the luma pass as above
 * (stream width a multiple of 16, 16-byte aligned; other host frames:
 * HMI_ERR_INVALID_ARG); such a frame must stay valid and unchanged until
 * cuda_stream has passed the call.  ptrs (device, n entries) may be NULL.
 * With use_graph != 0 the tick is replayed from a CUDA graph captured on first
 * use. */
HMI_API int hmi_batch_process_async(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
                            hmi_pointer *ptrs, void *cuda_stream, int use_graph);

/* Launch shape of a batch's ticks.  piece_chunks: 16-pixel chunks per CTA
 * work piece of the per-pixel kernels (the tile; a multiple of 32 in
 * 32..65536, default 512); luma_ctas_per_sm: CTAs per SM of the luma pass,
 * and of the persistent tick below (0 = as many as fit, else 1..32);
 * skin_ctas_per_sm, cc_ctas_per_sm: grid of the gray/hue pass and of the
 * block-component pass, in CTAs per SM (1..32, default 8); groups: stream
 * groups of plain ticks (0 = one when every stream can use the persistent
 * tick, else min(2, n); or 1..64); pipeline_depth: stages of a pipelined
 * tick (2 or 3, see hmi_batch_process_pipelined; default 2).
 * fused (default 0): with 1, a group whose streams all use the background band
 * (bg_model 0) with the same open_iters + close_iters, at most 2, runs the
 * per-pixel part of its tick (kernels 0, 1, 5 and 6 below) in one persistent
 * launch, whose CTAs take work items from a queue in order (per stream: luma
 * sums, then band / gray / hue tests, then morphology strips), each item
 * waiting (bounded) only for the stream's items of the step before; with 2,
 * such a group (open_iters + close_iters at most 4) runs them in one
 * cooperative launch of three phases (luma sums; gains and band / gray / hue
 * tests; morphology strips) separated by grid barriers with bounded waits; 0
 * runs the chain of kernels of HMI_TICK_KERNELS.  queue_lag: queue positions
 * between a stream's last item of one step and its first of the next
 * (0 = twice the persistent grid, else 1..2^20).  merge_threads: threads of
 * the CTA that merges one stream's block components into its pointer (the
 * merge schedule: 256, 512 or 1024; 0 = 512).  Results never depend on the
 * tuning. */
typedef struct {
    int32_t piece_chunks;
    int32_t luma_ctas_per_sm;
    int32_t skin_ctas_per_sm;
    int32_t cc_ctas_per_sm;
    int32_t groups;
    int32_t pipeline_depth;
    int32_t fused;
    int32_t queue_lag;
    int32_t merge_threads;
} hmi_tuning;

/* Replace the batch's launch shape (re-makes the plan; waits for the device).
 * HMI_ERR_INVALID_ARG for values out of range. */
HMI_API int hmi_batch_set_tuning(hmi_batch *b, const hmi_tuning *t);
HMI_API int hmi_batch_get_tuning(const hmi_batch *b, hmi_tuning *t);

/* Search the launch shape (Sec. 3.3: the GPU computation is autotuned):
 * time `ticks` ticks (2..10000) of frames (device memory, one per stream) for
 * each candidate (after untimed ticks that build every per-tick graph): the
 * tick form and the piece size together, then one parameter at a time (the
 * luma, skin and block-component grids, the merge CTA size, then the pipeline
 * depth for pipelined ticks or the group count for plain ticks); keep the
 * fastest, apply it and return it in *best with its time per tick in
 * microseconds (either may be NULL).  pipelined != 0 times pipelined
 * ticks (one group), else plain graph ticks.  The streams' click state and
 * pointer history are restored afterwards; their last labels are those of the
 * last tuning tick. */
HMI_API int hmi_batch_autotune(hmi_batch *b, const uint8_t *const *frames, int ticks, int pipelined,
                               hmi_tuning *best, double *best_tick_us);

/* Pipelined ticks, for plans with one group (HMI_ERR_INVALID_ARG otherwise;
 * see hmi_batch_set_groups).  A tick is split into D stages (D = the tuning's
 * pipeline_depth): with D = 2, {gains, background band test, re-learning}
 * (bandwidth-bound) and {gray and hue tests, morphology, components, pointer}
 * (latency-bound); with D = 3, {gains}, {band test, re-learning} and the same
 * last stage.  Each call
 * enqueues the first stage of its own frames and, beside it on the device,
 * stage j of the frames of the call j calls earlier, so D ticks overlap.
 * Buffers as in hmi_batch_process_async.  The results of a call (its masks
 * and ptrs) are complete once cuda_stream has passed the (D-1)-th pipelined
 * call after it on the batch, or hmi_batch_flush; its frames must stay valid
 * and unchanged until then.  Every other processing call on the batch (and
 * any change of its tuning) flushes first.  Results equal those of
 * hmi_batch_process_async on the same frames. */
HMI_API int hmi_batch_process_pipelined(hmi_batch *b, const uint8_t *const *frames,
                                        uint8_t *const *masks, hmi_pointer *ptrs,
                                        void *cuda_stream, int use_graph);
/* Enqueue the pending stage 2 (if any) on cuda_stream. */
HMI_API int hmi_batch_flush(hmi_batch *b, void *cuda_stream);

/* Kernel timing of a batch's ticks.  A tick runs HMI_TICK_KERNELS kernels in
 * this order: 0 luma sums and gains, 1 background band test (the per-pixel
 * HBM pass), 2 Gaussian mixture test and update (launched only when a stream
 * of the batch has bg_model 1), 3 re-learning sums and 4 re-learned bands
 * (launched only when a stream of the batch re-learns; they act on streams
 * inside a window), 5 gray and hue tests of out-of-band pixels, 6
 * morphology, 7 block components, 8 merge and pointer.  hmi_batch_profile(b, max_ticks)
 * starts recording CUDA events between the kernels for each of the next
 * max_ticks ticks (0 stops); the plan must have one group
 * (HMI_ERR_INVALID_ARG otherwise), so that every launch is timed alone.
 * hmi_batch_profile_kernels waits for them and gives the number of ticks timed
 * and, for the first n_kernels kernels (1..HMI_TICK_KERNELS), the sum of their
 * durations in milliseconds; hmi_batch_profile_read gives that sum for kernel
 * 1 alone.  With the persistent tick or the cooperative stage
 * (hmi_tuning.fused 1 or 2), kernel 0 is the whole per-pixel stage (kernels
 * 0, 1, 5 and 6), kernels 1, 2, 5 and 6 launch nothing, and
 * hmi_batch_profile_read gives kernel 0. */
#define HMI_TICK_KERNELS 9
HMI_API int hmi_batch_profile(hmi_batch *b, int max_ticks);
HMI_API int hmi_batch_profile_kernels(hmi_batch *b, int *ticks, double *ms, int n_kernels);
HMI_API int hmi_batch_profile_read(hmi_batch *b, int *ticks, double *total_ms);

/* FP32 mean and standard deviation of the learned background per pixel and
 * channel (h*w*3 floats each, host or device; either may be NULL):
 * mean = S/n, std = sqrt((n*Q - S^2)/n^2), each step one IEEE operation. */
HMI_API int hmi_get_background_stats(const hmi_stream *s, float *mean, float *std);

/* Labels of the last processed frame (h*w int32, host or device): -1 for
 * background, else the smallest linear index of the pixel's 8-connected
 * component (Mouse module, Sec. 2).  Computed on demand from the last mask. */
HMI_API int hmi_get_labels(const hmi_stream *s, int32_t *labels);

/* Headless Interface module (Sec. 2: fed by the Mouse module, it finds
 * which interface zone holds the pointer; each zone maps to an event)
 * and driving wheel (Sec. 4: the hand rotates about a virtual wheel to
 * steer left and right; speed is the third control).  Per frame, from the
 * valid pointer's rounded centroid p = floor((2 sum + area) / (2 area)) per
 * axis: zone = the first listed inclusive rectangle containing p; on_wheel
 * iff r_in^2 <= |p - c|^2 <= r_out^2 around the wheel centre c; steer = the
 * clockwise angle of p around c from the top, as a "diamond" pseudo-angle of
 * 4096 units per turn (1024 per quadrant: 1024 u / (u + v) in the first,
 * u = dx, v = -dy, floor division; likewise in the others), wrapped to
 * (-2048, 2048]; left / right = on the wheel and steer beyond -/+ dead_zone;
 * throttle = on the wheel and the click state (closed hand).  With no valid
 * pointer: zone = event = -1, the wheel fields 0.  frame is the number of
 * frames processed since learning, this one included. */
#define HMI_MAX_ZONES 16
typedef struct {
    int32_t x0, y0, x1, y1;  /* inclusive pixel rectangle */
    int32_t event;           /* the caller's event id */
} hmi_zone;

typedef struct {
    int32_t nzones;          /* 0 .. HMI_MAX_ZONES */
    hmi_zone zones[HMI_MAX_ZONES];
    int32_t wheel_on;        /* 0: no wheel */
    int32_t wheel_cx, wheel_cy;
    int32_t wheel_r_in, wheel_r_out;   /* 0 <= r_in <= r_out <= 65535 */
    int32_t dead_zone;       /* 0 .. 2048, pseudo-angle units */
} hmi_interface;

typedef struct {
    int32_t zone;            /* index of the activated zone, or -1 */
    int32_t event;           /* its event id, or -1 */
    int32_t on_wheel, steer, left, right, throttle;
    int32_t frame;           /* frames processed when the event was made */
} hmi_event;

/* Install the stream's interface (copied; waits for the device).  It applies
 * to the frames processed after the call.  HMI_ERR_INVALID_ARG out of range. */
HMI_API int hmi_set_interface(hmi_stream *s, const hmi_interface *ui);
/* The event of the stream's last processed frame (host or device pointer). */
HMI_API int hmi_get_event(const hmi_stream *s, hmi_event *out);

/* The background band in use (Sec. 3.1 (i)): lo and hi are h*w*3 bytes each
 * (host or device; pixel-major RGB), the learned band or, with re-learning,
 * the band as last re-formed.  HMI_ERR_NOT_LEARNED before learning. */
HMI_API int hmi_get_band(const hmi_stream *s, uint8_t *lo, uint8_t *hi);

/* The Gaussian mixture of a bg_model 1 stream (the state after the last
 * frame): out receives 6 * mix_k planes of h*w uint16 each (host or device),
 * in the order W[k], M[k][c] (k-major, c = R, G, B), V[k], C[k], k in the
 * stream's fitness order.  HMI_ERR_INVALID_ARG for a band stream,
 * HMI_ERR_NOT_LEARNED before learning. */
HMI_API int hmi_get_mixture(const hmi_stream *s, uint16_t *out);

/* Checkpoint of the learned model.  Export copies (each pointer may be NULL;
 * host or device) the per pixel-channel sums S, Q (uint32, h*w*3), min/max
 * and the derived band lo/hi (uint8, h*w*3, packed like the frame), the
 * reference luma and the number of learning frames.  Import installs S, Q,
 * min, max (all required) for n frames with reference luma syref, derives the
 * band with the stream's parameters and resets the click state, exactly as
 * learning from frames with those sums would.  HMI_ERR_NOT_LEARNED on export
 * before any learning.  A mixture stream (bg_model 1) exports its learning
 * sums like any stream, but refuses import (HMI_ERR_INVALID_ARG): its
 * mixture is learned from frames only. */
HMI_API int hmi_export_background(const hmi_stream *s, uint32_t *S, uint32_t *Q, uint8_t *vmin,
                                  uint8_t *vmax, uint8_t *lo, uint8_t *hi, uint64_t *syref,
                                  int *n);
HMI_API int hmi_import_background(hmi_stream *s, const uint32_t *S, const uint32_t *Q,
                                  const uint8_t *vmin, const uint8_t *vmax, int n, uint64_t syref);

/* Brightness gain (Q16) applied to the last processed frame, or an error. */
HMI_API int hmi_get_last_gain(const hmi_stream *s, uint32_t *gain_q16);

/* Bytes of device memory held by a stream created with these arguments
 * (the figure that admission control budgets).  0 on invalid arguments. */
HMI_API size_t hmi_stream_device_bytes(int w, int h, const hmi_params *p);

/* ---------------------------------------------------------------------------
 * Serving: many camera streams that come and go, frames arriving on their own
 * clocks.  A server admits a stream only while the device memory of all its
 * streams stays within a budget, keeps every admitted stream's state resident,
 * and runs a dispatcher thread that continuously batches: whenever frames are
 * pending it runs one tick over all admitted streams, taking at most one
 * frame (the oldest) per stream to process, so each stream's frames stay in
 * order; a stream still learning online gives up to four queued learning
 * frames to a round, added to its sums in arrival order.  A round is issued
 * while the previous one is still on the device, and its results are posted
 * once its device work has finished.  Results carry the submit and completion
 * times (hmi_server_now_ns clock).  All calls are thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct hmi_server hmi_server;

typedef struct {
    int32_t stream_id;   /* as returned by hmi_server_admit */
    int32_t status;      /* HMI_OK, HMI_LEARNING or the tick's error status */
    uint64_t tag;        /* the caller's tag from hmi_server_submit */
    uint64_t submit_ns;  /* when hmi_server_submit accepted the frame */
    uint64_t done_ns;    /* when the result became available */
    hmi_pointer pointer; /* the frame's pointer (Mouse module output) */
} hmi_server_result;

/* device_budget_bytes: cap on the sum of hmi_stream_device_bytes of admitted
 * streams; max_queue: frames a stream may have pending (1..64).  Creation maps
 * the library's stream-memory pool up to the budget (at most a quarter of the
 * free device memory), so that admitting a burst of streams later allocates
 * nothing new from the CUDA driver. */
HMI_API hmi_server *hmi_server_create(size_t device_budget_bytes, int max_queue);
HMI_API void hmi_server_destroy(hmi_server *srv);
/* Create a stream (Sec. 2, initialisation) and reserve its device bytes in
 * the budget; HMI_ERR_NO_MEMORY when they would exceed it (admission refused).
 * With learn_frames non-NULL the background is learned now from n contiguous
 * host frames (h*w*3 bytes each).  With learn_frames NULL the stream learns
 * online: the first n frames submitted to it are the user-free learning frames
 * (Sec. 2: FIZI's background is learned with no hand in view), each
 * accumulated by the dispatcher as it arrives and returned with status
 * HMI_LEARNING; the band is formed after the n-th, and later frames are
 * processed.  n: 1..65535. */
HMI_API int hmi_server_admit(hmi_server *srv, int w, int h, const hmi_params *p,
                             const uint8_t *learn_frames, int n, int *stream_id);
/* Retire a stream once its pending frames have been processed. */
HMI_API int hmi_server_release(hmi_server *srv, int stream_id);
/* Queue one host frame (h*w*3 bytes, copied before return).  HMI_ERR_NO_MEMORY
 * when the stream already has max_queue frames pending. */
HMI_API int hmi_server_submit(hmi_server *srv, int stream_id, const uint8_t *frame, uint64_t tag);
/* Same, without the copy: the server reads `frame` when the stream's tick
 * runs, so the caller keeps it valid and unchanged until the frame's result
 * has been returned by hmi_server_poll (pinned host memory is fastest). */
HMI_API int hmi_server_submit_ref(hmi_server *srv, int stream_id, const uint8_t *frame, uint64_t tag);
/* Up to max_results finished frames (waiting at most wait_us for the first);
 * returns how many were written, or a negative status. */
HMI_API int hmi_server_poll(hmi_server *srv, hmi_server_result *out, int max_results, int wait_us);
/* Device bytes admitted, ticks run and frames processed so far. */
HMI_API int hmi_server_stats(hmi_server *srv, size_t *bytes_admitted, uint64_t *ticks,
                             uint64_t *frames);
HMI_API uint64_t hmi_server_now_ns(void);

/* Per-round record of the dispatcher (the server's own timing trace).  A
 * round first creates newly admitted streams, retires released ones and
 * re-makes the plan when they changed (setup), then takes at most one
 * pending frame per stream and processes them; rounds that only did setup
 * are recorded too (frames = learning = 0). */
typedef struct {
    uint64_t start_ns;     /* round start */
    uint64_t setup_ns;     /* setup finished, frames taken from the queues */
    uint64_t issued_ns;    /* every copy and kernel of the round issued */
    uint64_t done_ns;      /* device work finished and results posted */
    int32_t frames;        /* frames processed by the round's tick */
    int32_t learning;      /* learning frames accumulated in the round */
    int32_t streams;       /* streams in the plan */
    int32_t replanned;     /* 1 if the plan was re-made in the setup */
    int32_t created;       /* streams created in the setup */
    int32_t retired;       /* streams retired in the setup */
} hmi_server_round;

/* Copy up to max_rounds of the most recent rounds (oldest first; the server
 * keeps the last 16384) into out; returns how many were written. */
HMI_API int hmi_server_rounds(hmi_server *srv, hmi_server_round *out, int max_rounds);

/* Brightness gain of one frame without any device allocation.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate
 * device memory, such as a real-time loop in which a cudaMalloc could stall the
 * device, or a host program that owns all device memory through its own pool.
 * It returns, in *gain_out (device memory, one uint32), the same clamped Q16
 * gain round(syref / SY) that hmi_process_frame applies, SY being the frame's
 * integer luma sum.  frame: h rows of 3*w bytes that the current device can
 * read (its device memory, managed memory, or pinned / registered host memory);
 * gain_out: device or managed memory of the current device, 4-byte aligned.
 * Anything else, and syref > 255*w*h (larger than any frame of this size can
 * sum to), is rejected with HMI_ERR_INVALID_ARG before any work is enqueued;
 * every error is also recorded for hmi_last_error.  The work runs on
 * cuda_stream (NULL = legacy default stream); the result is ready when that
 * stream reaches this point.
 * Scratch: a fixed 32 KiB array built into the library, one copy per GPU that
 * loads it, kept until the process exits.  Frames of more than 4,194,304
 * sixteen-pixel row chunks (h * ceil(w/16); 8192 x 8192 is the largest square)
 * and w or h beyond 8192 are rejected with HMI_ERR_INVALID_ARG.  A call outside
 * a stream capture looks up the current device's scratch address afresh; a
 * call made while cuda_stream is capturing reuses the address found by the
 * last call outside one, so make at least one call on the device before any
 * capture (and one after a device reset before capturing again).  All calls
 * share the scratch: calls that overlap on the GPU race and must be serialised
 * by the caller.  Calls no allocator. */
HMI_API int hmi_frame_gain_noalloc(const uint8_t *frame, int w, int h, uint64_t syref,
                                   uint32_t gain_min_q16, uint32_t gain_max_q16,
                                   uint32_t *gain_out, void *cuda_stream);

/* Status of the last failed call on this thread, and a text for a status. */
HMI_API int hmi_last_error(void);
HMI_API const char *hmi_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* HMI_H */
