// hmi_host.h -- host-side definitions shared by the translation units of the
// C ABI: the stream (hmi_stream), the launch plan (hmi_batch) with its stream
// groups, the device arena layout of a stream, and the plan and stream
// helpers that the server (hmi_server.cu) calls on top of the batch
// implementation (hmi_api.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "hmi_internal.cuh"

namespace hmi {

constexpr int kRing = 12;         // per-tick pointer slots of a launch plan (a multiple of kPhases)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Byte offsets of a stream's buffers inside its device arena.
struct Layout {
    int w, h, nwords, bh, tiles_x, strips_x, fpitch;
    size_t frame_ph[kPhases];     // staging frames for pinned host frames, by tick phase
    size_t npx, frame, lo, hi, S, Q, vmin, vmax, raw[kPhases], bits[kPhases], comp, parent,
        count[kPhases], flag[kPhases], mask, st, hist, ds, ptr, ui, total;
    // re-learning sums (only with re-learning on): rows of rpitch pixels
    int rpitch;
    size_t rS, rQ, rmin, rmax, rcnt, rpx;
    // Gaussian mixture (bg_model 1 only): mbytes of 32-pixel tiles, nwords
    // per row, 6 mix_k uint16 fields of 32 pixels each
    int mix_k;
    size_t mix, mbytes;
};

// Records `status` as this thread's last error (hmi_last_error) and returns
// it; the CUDA form clears the sticky error first and reports HMI_ERR_DEVICE.
int fail(int status);
int cuda_fail(cudaError_t e);

}  // namespace hmi

// Return the library's status for a failed CUDA call from the enclosing
// function.
#define HMI_CUDA(call)                               \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

using namespace hmi;

struct hmi_batch;
struct hmi_stream;
// learning from frames without preparing the single-frame plan (the server's)
extern "C" int learn_background(hmi_stream *s, const uint8_t *frames, int n);

struct hmi_stream {
    int dev = 0;
    int w = 0, h = 0;
    hmi_params p{};
    Layout L{};
    uint8_t *arena = nullptr;
    DevStream ds{};          // host copy (the buffers of tick phase 0)
    DevStream ds_phase[kPhases]{};   // host copies of the descriptor of each tick phase
    DevStream *d_ds = nullptr;       // device copies, kPhases of them
    StreamState *st = nullptr;
    uint8_t *d_frame = nullptr, *d_mask = nullptr;
    uint32_t *d_S = nullptr, *d_Q = nullptr;
    uint8_t *d_vmin = nullptr, *d_vmax = nullptr;
    hmi_pointer *d_ptr = nullptr;
    int learned = 0;
    int n_learn = 0;
    bool pooled = false;         // arena from the library's memory pool
    bool used = false;           // has been given frames (learning must wait for its work)
    cudaStream_t cs = nullptr;
    hmi_batch *self = nullptr;   // one-stream plan of hmi_process_frame, made on first use
};

// One chain of tick kernels over a subset of the batch's streams.
struct Group {
    int off = 0, cnt = 0;         // range in the permuted stream order
    BatchDev bd{};                // io, phase and skin queue are set per tick slot
    uint32_t *skin_count_p[kPhases] = {};   // skin queue of each tick phase
    uint2 *skin_list_p[kPhases] = {};
    uint32_t *cc_count_p[kPhases] = {};     // listed blocks of each tick phase
    uint2 *cc_list_p[kPhases] = {};
    cudaStream_t cs = nullptr;    // branch stream (also joins graph capture)
    cudaEvent_t ev_luma = nullptr, ev_done = nullptr;
};

struct hmi_batch {
    int dev = 0;
    int n = 0;
    hmi_tuning tune{};            // launch shape of the plan
    uint32_t loop_limit = 0;      // bound of the device loops (0: kLoopLimit)
    int cap = 0;                  // streams the per-batch buffers hold
    size_t plan_cap = 0;          // bytes of the plan table buffer
    std::vector<hmi_stream *> s;  // user order
    std::vector<int> pos;         // user index -> permuted position
    std::vector<Group> groups;
    uint8_t *arena = nullptr;     // per-batch device buffers
    uint8_t *plan = nullptr;      // per-plan device tables
    const DevStream *ds_tab = nullptr;   // in plan: kPhases tables of n descriptors
    TickIO *h_io = nullptr;       // pinned mirrors, kRing x n, permuted order
    TickIO *d_io = nullptr;       // device copies, kRing x n
    hmi_pointer *d_ptrs = nullptr;  // n pointers for the synchronous form, user order
    uint32_t *d_err = nullptr;    // batch error word (device)
    uint32_t *h_err = nullptr;    // pinned
    cudaEvent_t slot_ev[kRing] = {};
    bool slot_used[kRing] = {};
    int next = 0;
    cudaStream_t cs = nullptr;    // origin stream of the synchronous form and of graph capture
    cudaEvent_t ev_fork = nullptr;
    int num_sms = 1;
    cudaGraphExec_t graph[kRing] = {};     // plain tick graphs
    // profiling tick graphs (single group): an event-record node before the
    // first kernel and after each, retargeted to the tick's events at launch;
    // the source graph is kept alive for its node handles
    cudaGraph_t pgraph_src[kRing] = {};
    cudaGraphExec_t pgraph[kRing] = {};
    cudaGraphNode_t ev_node[kRing][kTickKernels + 1] = {};
    cudaEvent_t dummy_ev[kTickKernels + 1] = {};
    // pipelined ticks (single group): slots of the ticks still in flight,
    // newest first (pend[j] has run stages 0 .. j and runs stage j + 1 next),
    // the depth they were started with, an event at the end of the last
    // pipelined call, a second branch stream and the branches' end events,
    // and per slot the graph of a full pipelined call
    int npend = 0;
    int pend[kPhases - 1] = {};
    int pend_depth = 0;
    cudaEvent_t pipe_ev = nullptr;
    cudaStream_t cs2 = nullptr;
    cudaEvent_t side_done[kPhases - 1] = {};
    cudaGraphExec_t pipe_graph[kRing] = {};
    // profiling of the classification kernel (single-group plans)
    std::vector<cudaEvent_t> prof_ev;
    int prof_max = 0, prof_used = 0;
    // device buffers already validated (skips a pointer-attribute query per
    // buffer per tick); bounded, cleared when full
    std::unordered_set<const void *> seen;
    bool seen_device(const void *p) const { return seen.count(p) != 0; }
    void remember_device(const void *p)
    {
        if (seen.size() >= 65536) seen.clear();
        seen.insert(p);
    }
    // pinned host buffers already validated, with their device-accessible
    // address (the caller keeps them pinned while the batch uses them)
    std::unordered_map<const void *, const uint8_t *> pinned;
    const uint8_t *pinned_dev(const void *p)
    {
        auto it = pinned.find(p);
        if (it != pinned.end()) return it->second;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return nullptr;
        if (pinned.size() >= 65536) pinned.clear();
        const uint8_t *d = static_cast<const uint8_t *>(at.devicePointer);
        pinned.emplace(p, d);
        return d;
    }
};

namespace hmi {

// The library's stream-ordered memory pool of device `dev` (null: none).
cudaMemPool_t arena_pool(int dev);
// A stream of w x h on the current device, its arena ordered after `order`.
hmi_stream *create_stream_on(int w, int h, const hmi_params *p, cudaStream_t order);
// A launch plan over n learned streams in ngroups groups (0: by the streams),
// its re-plan over another set of streams, and its release.
hmi_batch *batch_new(hmi_stream *const *s, int n, int ngroups);
int batch_replan(hmi_batch *b, hmi_stream *const *s, int n, int ngroups);
int batch_free(hmi_batch *b);
// The next free per-tick slot of a plan (waits for its last tick), and one
// tick of the plan in that slot on cs (through its graph or not).
int acquire_slot(hmi_batch *b);
int run_tick(hmi_batch *b, int slot, cudaStream_t cs, bool use_graph);
// Enqueue on cs: the reset of a stream's mixture, and the band of its n
// learning frames from the accumulated sums.
cudaError_t enqueue_mix_reset(hmi_stream *s, cudaStream_t cs);
cudaError_t enqueue_band(hmi_stream *s, int n, cudaStream_t cs);


// Plans: the device tables of a plan for ng groups and their release, the
// groups a set of streams gets by default, and whether all streams of a plan
// have learned their background.
int plan_build(hmi_batch *b, int ng);
void plan_free(hmi_batch *b);
int default_groups(hmi_stream *const *s, int n, const hmi_tuning &t);
bool all_learned(hmi_batch *b);
// The asynchronous and pipelined forms of a tick (the C entry points after
// their argument checks), and the end of the pipelined ticks still in flight.
int batch_async(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks, hmi_pointer *ptrs,
                void *cuda_stream, int use_graph);
int batch_pipelined(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks, hmi_pointer *ptrs,
                    void *cuda_stream, int use_graph);
int flush_pending(hmi_batch *b, cudaStream_t cs);
// Launch shapes (hmi_tune.cu): a shape's validity, a re-plan with a shape,
// and the search of the autotuner.
bool tuning_ok(const hmi_tuning &t);
int batch_retune(hmi_batch *b, const hmi_tuning &t);
int batch_autotune(hmi_batch *b, const uint8_t *const *frames, int ticks, bool pipelined,
                   hmi_tuning *best_out, double *best_us_out);

}  // namespace hmi
