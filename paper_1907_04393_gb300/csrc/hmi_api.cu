// hmi_api.cu -- host implementation of the C ABI declared in include/hmi.h.
//
// A stream owns one device arena (all of its buffers, taken from a
// library-owned stream-ordered memory pool at creation) and, once learned, a
// one-stream launch plan.  A launch plan (hmi_batch) owns the device tables
// the tick kernels read (stream descriptors, work pieces, prefix sums), a ring
// of per-tick pointer slots (pinned host mirror + device copy + event), and
// optionally one CUDA graph per slot that replays the whole tick: the slot's
// pointer upload, then the luma (which also brings pinned host frames over),
// band test or mixture, re-learning, gray/hue, morphology + block components
// and per-stream finish (merge, resolve, pointer, interface event) kernels.
//
// In order below: layouts and the pool; plans (build, re-plan, groups,
// graphs, pipelined stages); ticks (slot preparation, synchronous,
// asynchronous and pipelined forms, tuning and autotuning); learning; the
// server (admission, rounds, batched learning); the exported C functions.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "hmi_internal.cuh"
#include "hmi_queue.h"

using namespace hmi;

namespace {

thread_local int g_last_error = HMI_OK;

int fail(int status)
{
    g_last_error = status;
    return status;
}

int cuda_fail(cudaError_t e)
{
    (void)cudaGetLastError();
    (void)e;
    return fail(HMI_ERR_DEVICE);
}

}  // namespace

// Thread-local status of the last failed call, for the other translation units.
int hmi::set_error(int status) { return fail(status); }

namespace {

#define HMI_CUDA(call)                               \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

constexpr int kRing = 12;         // per-tick pointer slots of a launch plan (a multiple of kPhases)
// Default launch shape (hmi_tuning): 16-px chunks per CTA piece of the
// per-pixel kernels (512 = 8192 px), luma CTAs per SM (0 = as many as fit),
// skin-test and block-component CTAs per SM, stream groups (0 = by the
// streams, see default_groups), stages of a pipelined tick, the persistent
// tick off (the chain of kernels measured faster on the 64-stream batch), its
// queue lag chosen from the grid, 512 threads per stream merge.
constexpr hmi_tuning kDefaultTuning = {512, 0, 8, 8, 0, 2, 0, 0, 0};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool params_valid(const hmi_params &p)
{
    if (p.hue_lo >= 1536 || p.hue_hi >= 1536) return false;
    if (p.bg_k_den < 1 || p.bg_k_den > 15 || p.bg_k_num > 15) return false;
    if (p.open_iters + p.close_iters > 16) return false;
    if (p.gain_min_q16 > p.gain_max_q16 || p.gain_max_q16 > (1u << 24)) return false;
    if (p.click_window > 1024) return false;
    if (p.relearn_frames > 0 &&
        (p.relearn_min < 1 || p.relearn_min > p.relearn_frames || p.relearn_period < p.relearn_frames))
        return false;
    if (p.bg_model > 1 || p.mix_pad != 0) return false;
    if (p.bg_model == 1 &&
        (p.mix_k < 1 || p.mix_k > 4 || p.mix_bg_pct < 1 || p.mix_bg_pct > 100 || p.mix_sigma0 < 1 ||
         p.mix_sigma0 > 63 || p.mix_sigma_min < 1 || p.mix_sigma_min > p.mix_sigma0 ||
         p.mix_rate_n < 1 || p.bg_k_num < 1 || p.relearn_frames != 0))
        return false;
    return true;
}

// Hue arc [lo, hi] (mod 1536) as, per sector, up to two intervals of
// q = floor(N / 2d) in [0, 512] with h = base - 256 + q; stored as the
// half-open bounds of N: 2d*a <= N < 2d*(b + 1).  Empty: a = b = 513.
void hue_intervals(int lo, int hi, int A[3][2], int B[3][2])
{
    for (int sec = 0; sec < 3; ++sec) {
        const int base = 512 * sec;
        int nint = 0;
        A[sec][0] = A[sec][1] = B[sec][0] = B[sec][1] = 2 * 513;
        int q = 0;
        while (q <= 512 && nint < 2) {
            auto in_arc = [&](int qq) {
                int h = ((base - 256 + qq) % 1536 + 1536) % 1536;
                return lo <= hi ? (h >= lo && h <= hi) : (h >= lo || h <= hi);
            };
            while (q <= 512 && !in_arc(q)) ++q;
            if (q > 512) break;
            int a = q;
            while (q <= 512 && in_arc(q)) ++q;
            A[sec][nint] = 2 * a;
            B[sec][nint] = 2 * q;   // q is one past the run
            ++nint;
        }
    }
}

struct Arena {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    }
};

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

Layout make_layout(int w, int h, const hmi_params &p)
{
    Layout L;
    L.w = w;
    L.h = h;
    L.nwords = (w + 31) / 32;
    L.bh = (h + 31) / 32;
    L.tiles_x = (L.nwords + kMorphTW - 1) / kMorphTW;
    L.strips_x = (L.nwords + 29) / 30;   // strips of 30 words x 16 rows
    L.fpitch = (int)align_up((size_t)w, 16) * 3;
    L.npx = (size_t)w * h;
    const size_t nblk = (size_t)L.bh * L.nwords;
    const size_t bitrows = (size_t)L.bh * 32 * L.nwords * 4;
    Arena a;
    L.frame = a.take((size_t)h * L.fpitch + 64);
    L.frame_ph[0] = L.frame;
    for (int k = 1; k < kPhases; ++k) L.frame_ph[k] = a.take((size_t)h * L.fpitch + 64);
    L.lo = a.take((size_t)h * L.fpitch + 64);
    L.hi = a.take((size_t)h * L.fpitch + 64);
    L.S = a.take(L.npx * 3 * 4);
    L.Q = a.take(L.npx * 3 * 4);
    L.vmin = a.take(L.npx * 3);
    L.vmax = a.take(L.npx * 3);
    for (int k = 0; k < kPhases; ++k) L.raw[k] = a.take(bitrows);   // one per tick phase
    for (int k = 0; k < kPhases; ++k) L.bits[k] = a.take(bitrows);
    L.comp = a.take(nblk * kSlots * sizeof(Comp));
    L.parent = a.take(nblk * kSlots * 4);
    for (int k = 0; k < kPhases; ++k) {
        L.count[k] = a.take(nblk * 4);
        L.flag[k] = a.take(nblk * 4);
    }
    L.mask = a.take(L.npx);
    L.st = a.take(sizeof(StreamState));
    L.hist = a.take((size_t)std::max<int>(p.click_window, 1) * 4);
    L.ds = a.take(sizeof(DevStream) * kPhases);   // one descriptor per tick phase
    L.ptr = a.take(sizeof(hmi_pointer));
    L.ui = a.take(sizeof(hmi_interface));
    L.rpitch = (int)align_up((size_t)w, 16);
    L.rpx = p.relearn_frames > 0 ? (size_t)h * L.rpitch : 0;
    L.rS = L.rQ = L.rmin = L.rmax = L.rcnt = 0;
    if (L.rpx) {
        L.rS = a.take(L.rpx * 3 * 2);
        L.rQ = a.take(L.rpx * 3 * 4);
        L.rmin = a.take(L.rpx * 3);
        L.rmax = a.take(L.rpx * 3);
        L.rcnt = a.take(L.rpx);
    }
    L.mix_k = p.bg_model == 1 ? p.mix_k : 0;
    L.mbytes = (size_t)h * L.nwords * 32 * 6 * L.mix_k * 2;
    L.mix = L.mix_k ? a.take(L.mbytes) : 0;
    L.total = a.off;
    return L;
}

// Stream state comes from a stream-ordered memory pool owned by the library
// (one per device, memory kept while any stream lives), so that creating and
// destroying streams, as a server admitting and retiring cameras does, needs
// neither the CUDA driver's allocator nor a device-wide synchronisation of its own.
struct ArenaPools {
    std::mutex mu;
    cudaMemPool_t pool[64] = {};
    int state[64] = {};              // 0 unknown, 1 pool, 2 no pool support
    std::atomic<int> live[64] = {};
};
ArenaPools g_pools;

cudaMemPool_t arena_pool(int dev)
{
    if (dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_pools.mu);
    if (g_pools.state[dev] == 0) {
        int ok = 0;
        cudaDeviceGetAttribute(&ok, cudaDevAttrMemoryPoolsSupported, dev);
        cudaMemPoolProps pr;
        memset(&pr, 0, sizeof(pr));
        pr.allocType = cudaMemAllocationTypePinned;
        pr.location.type = cudaMemLocationTypeDevice;
        pr.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (ok && cudaMemPoolCreate(&pool, &pr) == cudaSuccess) {
            uint64_t keep = ~0ull;   // released only when the last stream goes
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            g_pools.pool[dev] = pool;
            g_pools.state[dev] = 1;
        } else {
            (void)cudaGetLastError();
            g_pools.state[dev] = 2;
        }
    }
    return g_pools.pool[dev];
}

bool is_device_ptr(const void *p)
{
    if (p == nullptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

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

namespace {

std::mutex g_cache_mu;
hmi_batch *g_cache = nullptr;    // plan reused by hmi_process_batch

// The descriptor a tick of phase k uses: its own bit mask, block counts and flags.
DevStream phase_view(const DevStream &D, int k)
{
    DevStream V = D;
    V.bits = D.bits_p[k];
    V.count = D.count_p[k];
    V.flag = D.flag_p[k];
    return V;
}

void fill_devstream(hmi_stream *s)
{
    DevStream &D = s->ds;
    const Layout &L = s->L;
    uint8_t *a = s->arena;
    D.w = s->w;
    D.h = s->h;
    D.nwords = L.nwords;
    D.bh = L.bh;
    D.tiles_x = L.tiles_x;
    D.strips_x = L.strips_x;
    D.fpitch = L.fpitch;
    D.cpr_magic = (uint32_t)(((1ull << 32) + 2ull * L.nwords - 1) / (2ull * L.nwords));
    D.gray_tol = s->p.gray_tol;
    D.open_iters = s->p.open_iters;
    D.close_iters = s->p.close_iters;
    D.gain_min = s->p.gain_min_q16;
    D.gain_max = s->p.gain_max_q16;
    D.min_area = s->p.min_area;
    D.click_on = s->p.click_on_pct;
    D.click_off = s->p.click_off_pct;
    D.click_window = s->p.click_window;
    hue_intervals(s->p.hue_lo, s->p.hue_hi, D.hueA, D.hueB);
    D.lo = a + L.lo;
    D.hi = a + L.hi;
    for (int k = 0; k < kPhases; ++k) D.raw[k] = reinterpret_cast<uint32_t *>(a + L.raw[k]);
    for (int k = 0; k < kPhases; ++k) {
        D.bits_p[k] = reinterpret_cast<uint32_t *>(a + L.bits[k]);
        D.count_p[k] = reinterpret_cast<uint32_t *>(a + L.count[k]);
        D.flag_p[k] = reinterpret_cast<uint32_t *>(a + L.flag[k]);
    }
    D.bits = D.bits_p[0];
    D.count = D.count_p[0];
    D.flag = D.flag_p[0];
    D.comp = reinterpret_cast<Comp *>(a + L.comp);
    D.parent = reinterpret_cast<uint32_t *>(a + L.parent);
    D.st = reinterpret_cast<StreamState *>(a + L.st);
    D.hist = reinterpret_cast<uint32_t *>(a + L.hist);
    D.bg_kn = s->p.bg_k_num;
    D.bg_kd = s->p.bg_k_den;
    D.bg_delta = s->p.bg_margin;
    D.track_max_dist = s->p.track_max_dist;
    D.ui = reinterpret_cast<const hmi_interface *>(a + L.ui);
    D.relearn_frames = L.rpx ? s->p.relearn_frames : 0;
    D.relearn_min = s->p.relearn_min;
    D.relearn_period = s->p.relearn_period;
    D.rpitch = L.rpitch;
    D.rS = L.rpx ? reinterpret_cast<uint16_t *>(a + L.rS) : nullptr;
    D.rQ = L.rpx ? reinterpret_cast<uint32_t *>(a + L.rQ) : nullptr;
    D.rmin = L.rpx ? a + L.rmin : nullptr;
    D.rmax = L.rpx ? a + L.rmax : nullptr;
    D.rcnt = L.rpx ? a + L.rcnt : nullptr;
    MixView &M = D.mix;
    M.K = L.mix_k;
    M.planes = L.mix_k ? reinterpret_cast<uint16_t *>(a + L.mix) : nullptr;
    M.tiles_x = L.nwords;
    M.rate_n = s->p.mix_rate_n;
    M.bg_pct = s->p.mix_bg_pct;
    M.lam_a = (uint32_t)s->p.bg_k_den * s->p.bg_k_den;
    M.lam_b = 3u * s->p.bg_k_num * s->p.bg_k_num * 4096u;
    M.v_init = 16u * s->p.mix_sigma0 * s->p.mix_sigma0;
    M.v_min = 16u * s->p.mix_sigma_min * s->p.mix_sigma_min;
    M.recip_n = recip40(2u * s->p.mix_rate_n);
}

void plan_free_graphs(hmi_batch *b)
{
    for (int i = 0; i < kRing; ++i) {
        if (b->graph[i]) cudaGraphExecDestroy(b->graph[i]);
        if (b->pgraph[i]) cudaGraphExecDestroy(b->pgraph[i]);
        if (b->pipe_graph[i]) cudaGraphExecDestroy(b->pipe_graph[i]);
        b->pipe_graph[i] = nullptr;
        if (b->pgraph_src[i]) cudaGraphDestroy(b->pgraph_src[i]);
        b->graph[i] = b->pgraph[i] = nullptr;
        b->pgraph_src[i] = nullptr;
        for (auto &nd : b->ev_node[i]) nd = nullptr;
    }
}

void group_destroy(Group &g)
{
    if (g.cs) cudaStreamDestroy(g.cs);
    if (g.ev_luma) cudaEventDestroy(g.ev_luma);
    if (g.ev_done) cudaEventDestroy(g.ev_done);
    g.cs = nullptr;
    g.ev_luma = g.ev_done = nullptr;
}

void plan_free(hmi_batch *b)
{
    plan_free_graphs(b);
    for (auto &g : b->groups) group_destroy(g);
    b->groups.clear();
    if (b->plan) cudaFree(b->plan);
    b->plan = nullptr;
    b->plan_cap = 0;
}

int flush_pending(hmi_batch *b, cudaStream_t cs);

int batch_free(hmi_batch *b)
{
    if (!b) return HMI_OK;
    cudaSetDevice(b->dev);
    if (b->cs && b->npend > 0) flush_pending(b, b->cs);
    if (b->cs) cudaStreamSynchronize(b->cs);
    for (int i = 0; i < kRing; ++i)
        if (b->slot_ev[i]) cudaEventSynchronize(b->slot_ev[i]);
    cudaDeviceSynchronize();
    plan_free(b);
    for (int i = 0; i < kRing; ++i)
        if (b->slot_ev[i]) cudaEventDestroy(b->slot_ev[i]);
    for (auto &e : b->dummy_ev)
        if (e) cudaEventDestroy(e);
    for (auto e : b->prof_ev) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->pipe_ev) cudaEventDestroy(b->pipe_ev);
    for (auto e : b->side_done)
        if (e) cudaEventDestroy(e);
    if (b->cs2) cudaStreamDestroy(b->cs2);
    if (b->cs) cudaStreamDestroy(b->cs);
    if (b->arena) cudaFree(b->arena);
    if (b->h_io) cudaFreeHost(b->h_io);
    if (b->h_err) cudaFreeHost(b->h_err);
    delete b;
    return HMI_OK;
}

// Build the launch plan with `ng` stream groups: streams are dealt to groups
// by pixel count (largest first, to the least-loaded group); each group gets
// its own descriptor array, prefix tables, work pieces, counters and
// component list, and its own branch stream.
int plan_build(hmi_batch *b, int ng)
{
    const int n = b->n;
    ng = std::max(1, std::min(ng, n));
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (long long)b->s[x]->w * b->s[x]->h > (long long)b->s[y]->w * b->s[y]->h;
    });
    std::vector<std::vector<int>> members(ng);
    std::vector<long long> load(ng, 0);
    for (int i : order) {
        const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        members[g].push_back(i);
        load[g] += (long long)b->s[i]->w * b->s[i]->h;
    }
    std::vector<int> perm;
    // branch streams and events of an earlier plan are reused
    std::vector<Group> old = std::move(b->groups);
    b->groups.assign(ng, Group());
    for (int g = 0; g < (int)old.size(); ++g) {
        if (g < ng) {
            b->groups[g].cs = old[g].cs;
            b->groups[g].ev_luma = old[g].ev_luma;
            b->groups[g].ev_done = old[g].ev_done;
        } else {
            group_destroy(old[g]);
        }
    }
    for (int g = 0; g < ng; ++g) {
        std::sort(members[g].begin(), members[g].end());
        b->groups[g].off = (int)perm.size();
        b->groups[g].cnt = (int)members[g].size();
        for (int i : members[g]) perm.push_back(i);
    }
    b->pos.assign(n, 0);
    for (int p = 0; p < n; ++p) b->pos[perm[p]] = p;

    struct Tables {
        std::vector<unsigned long long> cpre;
        std::vector<uint32_t> tpre, bpre, spre;
        std::vector<int4> pieces;
        int max_halo = 0, uniform_halo = 0;
        bool any_mix = false;
        size_t o_c, o_t, o_b, o_s, o_done, o_p, o_ccn[kPhases], o_ccl[kPhases], o_skn[kPhases], o_skl[kPhases];
        // persistent tick: work queue and per-stream progress
        bool fused = false;
        std::vector<int4> items;
        std::vector<TickSync> sync;
        size_t o_items = 0, o_sync = 0, o_head = 0;
    };
    const long long tick_grid = (long long)b->num_sms * tick_ctas_per_sm(b->tune.luma_ctas_per_sm);
    std::vector<Tables> T(ng);
    Arena a;
    const size_t o_ds = a.take(sizeof(DevStream) * n * kPhases);   // a descriptor table per tick phase
    for (int g = 0; g < ng; ++g) {
        Tables &t = T[g];
        const int m = b->groups[g].cnt;
        t.cpre.assign(m + 1, 0);
        t.tpre.assign(m + 1, 0);
        t.bpre.assign(m + 1, 0);
        t.spre.assign(m + 1, 0);
        t.uniform_halo = -2;
        for (int k = 0; k < m; ++k) {
            const hmi_stream *st = b->s[perm[b->groups[g].off + k]];
            const Layout &L = st->L;
            const int chunks = L.h * 2 * L.nwords;
            t.cpre[k + 1] = t.cpre[k] + (unsigned long long)chunks;
            t.tpre[k + 1] = t.tpre[k] + (uint32_t)(L.bh * L.tiles_x);
            t.spre[k + 1] = t.spre[k] + (uint32_t)(((L.h + kStripRows - 1) / kStripRows) * L.strips_x);
            t.bpre[k + 1] = t.bpre[k] + (uint32_t)(L.bh * L.nwords);
            const int halo = 2 * (st->p.open_iters + st->p.close_iters);
            t.max_halo = std::max(t.max_halo, halo);
            t.uniform_halo = (t.uniform_halo == -2 || t.uniform_halo == halo) ? halo : -1;
            for (int c = 0; c < chunks; c += b->tune.piece_chunks)
                t.pieces.push_back(make_int4(k, c, std::min(chunks, c + b->tune.piece_chunks), 0));
            if (L.mix_k) t.any_mix = true;
        }
        t.fused = b->tune.fused && !t.any_mix && t.uniform_halo >= 0 && t.uniform_halo <= kTickMaxHalo;
        if (t.fused) {
            std::vector<int> ch(m), sp(m);
            for (int k = 0; k < m; ++k) {
                const Layout &L = b->s[perm[b->groups[g].off + k]]->L;
                ch[k] = L.h * 2 * L.nwords;
                sp[k] = ((L.h + kStripRows - 1) / kStripRows) * L.strips_x;   // morphology strips
            }
            const long long lag = b->tune.queue_lag > 0 ? b->tune.queue_lag : 2 * tick_grid;
            t.items = tick_queue(ch, sp, b->tune.piece_chunks, lag, &t.sync);
            t.o_items = a.take(sizeof(int4) * t.items.size());
            t.o_sync = a.take(sizeof(TickSync) * m);
            t.o_head = a.take(sizeof(uint32_t) * 2);
        }
        t.o_c = a.take(sizeof(unsigned long long) * (m + 1));
        t.o_t = a.take(sizeof(uint32_t) * (m + 1));
        t.o_b = a.take(sizeof(uint32_t) * (m + 1));
        t.o_s = a.take(sizeof(uint32_t) * (m + 1));
        t.o_done = a.take(sizeof(uint32_t) * 4);
        t.o_p = a.take(sizeof(int4) * std::max<size_t>(t.pieces.size(), 1));
        for (int k = 0; k < kPhases; ++k) {
            t.o_ccn[k] = a.take(sizeof(uint32_t));
            t.o_ccl[k] = a.take(sizeof(uint2) * std::max<size_t>(t.bpre[m], 1));
            t.o_skn[k] = a.take(sizeof(uint32_t));
            t.o_skl[k] = a.take(sizeof(uint2) * std::max<size_t>(t.cpre[m], 1));
        }
    }
    if (a.off > b->plan_cap) {   // grow the table buffer; a smaller plan reuses it
        if (b->plan) cudaFree(b->plan);
        b->plan = nullptr;
        b->plan_cap = 0;
        const size_t want = std::max(a.off, b->plan_cap + b->plan_cap / 2);
        if (cudaMalloc(&b->plan, want) != cudaSuccess) {
            (void)cudaGetLastError();
            for (auto &g : b->groups) group_destroy(g);
            b->groups.clear();
            return fail(HMI_ERR_NO_MEMORY);
        }
        b->plan_cap = want;
    }
    // Tables go up in stream order on the batch's own stream, from host
    // vectors that live until the synchronisation at the end.
    uint8_t *A = b->plan;
    cudaStream_t up = b->cs;
    std::vector<DevStream> ds((size_t)n * kPhases);
    for (int k = 0; k < kPhases; ++k)
        for (int p = 0; p < n; ++p) ds[(size_t)k * n + p] = b->s[perm[p]]->ds_phase[k];
    bool ok = cudaMemsetAsync(A, 0, a.off, up) == cudaSuccess &&
              cudaMemcpyAsync(A + o_ds, ds.data(), sizeof(DevStream) * n * kPhases, cudaMemcpyHostToDevice, up) == cudaSuccess;
    b->ds_tab = reinterpret_cast<const DevStream *>(A + o_ds);
    for (int g = 0; ok && g < ng; ++g) {
        Tables &t = T[g];
        Group &G = b->groups[g];
        const int m = G.cnt;
        ok = cudaMemcpyAsync(A + t.o_c, t.cpre.data(), sizeof(unsigned long long) * (m + 1), cudaMemcpyHostToDevice, up) == cudaSuccess &&
             cudaMemcpyAsync(A + t.o_t, t.tpre.data(), sizeof(uint32_t) * (m + 1), cudaMemcpyHostToDevice, up) == cudaSuccess &&
             cudaMemcpyAsync(A + t.o_b, t.bpre.data(), sizeof(uint32_t) * (m + 1), cudaMemcpyHostToDevice, up) == cudaSuccess &&
             cudaMemcpyAsync(A + t.o_s, t.spre.data(), sizeof(uint32_t) * (m + 1), cudaMemcpyHostToDevice, up) == cudaSuccess &&
             cudaMemcpyAsync(A + t.o_p, t.pieces.data(), sizeof(int4) * t.pieces.size(), cudaMemcpyHostToDevice, up) == cudaSuccess &&
             (!t.fused ||
              (cudaMemcpyAsync(A + t.o_items, t.items.data(), sizeof(int4) * t.items.size(), cudaMemcpyHostToDevice, up) == cudaSuccess &&
               cudaMemcpyAsync(A + t.o_sync, t.sync.data(), sizeof(TickSync) * m, cudaMemcpyHostToDevice, up) == cudaSuccess)) &&
             (G.cs || cudaStreamCreateWithFlags(&G.cs, cudaStreamNonBlocking) == cudaSuccess) &&
             (G.ev_luma || cudaEventCreateWithFlags(&G.ev_luma, cudaEventDisableTiming) == cudaSuccess) &&
             (G.ev_done || cudaEventCreateWithFlags(&G.ev_done, cudaEventDisableTiming) == cudaSuccess);
        BatchDev &bd = G.bd;
        bd.ds = reinterpret_cast<const DevStream *>(A + o_ds) + G.off;
        bd.io = nullptr;
        bd.n = m;
        bd.total_chunks = t.cpre[m];
        bd.total_tiles = t.tpre[m];
        bd.total_blocks = t.bpre[m];
        bd.chunk_prefix = reinterpret_cast<const unsigned long long *>(A + t.o_c);
        bd.tile_prefix = reinterpret_cast<const uint32_t *>(A + t.o_t);
        bd.block_prefix = reinterpret_cast<const uint32_t *>(A + t.o_b);
        bd.strip_prefix = reinterpret_cast<const uint32_t *>(A + t.o_s);
        bd.total_strips = t.spre[m];
        bd.max_halo = t.max_halo;
        bd.uniform_halo = t.uniform_halo;
        bd.done = reinterpret_cast<uint32_t *>(A + t.o_done);
        bd.pieces = reinterpret_cast<const int4 *>(A + t.o_p);
        bd.npieces = (int)t.pieces.size();
        bd.err = b->d_err;
        for (int k = 0; k < kPhases; ++k) {
            G.cc_count_p[k] = reinterpret_cast<uint32_t *>(A + t.o_ccn[k]);
            G.cc_list_p[k] = reinterpret_cast<uint2 *>(A + t.o_ccl[k]);
            G.skin_count_p[k] = reinterpret_cast<uint32_t *>(A + t.o_skn[k]);
            G.skin_list_p[k] = reinterpret_cast<uint2 *>(A + t.o_skl[k]);
        }
        bd.skin_count = G.skin_count_p[0];
        bd.skin_list = G.skin_list_p[0];
        bd.cc_count = G.cc_count_p[0];
        bd.cc_list = G.cc_list_p[0];
        bd.phase = 0;
        bd.relearn = bd.any_band = bd.any_mix = 0;
        for (int k = 0; k < m; ++k) {
            const hmi_stream *sk = b->s[perm[G.off + k]];
            if (sk->L.rpx) bd.relearn = 1;
            if (sk->L.mix_k) bd.any_mix |= 1 << sk->L.mix_k;
            else bd.any_band = 1;
        }
        bd.fused = t.fused ? 1 : 0;
        bd.items = t.fused ? reinterpret_cast<const int4 *>(A + t.o_items) : nullptr;
        bd.nitems = t.fused ? (int)t.items.size() : 0;
        bd.sync = t.fused ? reinterpret_cast<TickSync *>(A + t.o_sync) : nullptr;
        bd.tick_head = t.fused ? reinterpret_cast<uint32_t *>(A + t.o_head) : nullptr;
        bd.tick_exit = t.fused ? bd.tick_head + 1 : nullptr;
        bd.loop_limit = b->loop_limit ? b->loop_limit : kLoopLimit;
        bd.merge_threads = b->tune.merge_threads ? b->tune.merge_threads : 512;
        bd.luma_ctas_per_sm = b->tune.luma_ctas_per_sm;
        bd.skin_ctas_per_sm = b->tune.skin_ctas_per_sm;
        bd.cc_ctas_per_sm = b->tune.cc_ctas_per_sm;
    }
    ok = ok && cudaStreamSynchronize(up) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        plan_free(b);
        return fail(HMI_ERR_DEVICE);
    }
    return HMI_OK;
}

bool streams_ok(hmi_stream *const *s, int n)
{
    if (!s || n < 1 || n > kMaxBatch) return false;
    for (int i = 0; i < n; ++i) {
        if (!s[i] || s[i]->dev != s[0]->dev) return false;
        for (int j = 0; j < i; ++j)
            if (s[j] == s[i]) return false;
    }
    return true;
}

// Per-batch buffers for `cap` streams: kRing tick tables (device and pinned
// mirror), the pointers of the synchronous form and the error word.
bool batch_alloc_io(hmi_batch *b, int cap)
{
    if (b->arena) cudaFree(b->arena);
    if (b->h_io) cudaFreeHost(b->h_io);
    b->arena = nullptr;
    b->h_io = nullptr;
    b->cap = 0;
    Arena a;
    const size_t o_io = a.take(sizeof(TickIO) * cap * kRing);
    const size_t o_ptr = a.take(sizeof(hmi_pointer) * cap);
    const size_t o_err = a.take(sizeof(uint32_t));
    if (cudaMalloc(&b->arena, a.off) != cudaSuccess || cudaMemset(b->arena, 0, a.off) != cudaSuccess ||
        cudaMallocHost(&b->h_io, sizeof(TickIO) * cap * kRing) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    memset(b->h_io, 0, sizeof(TickIO) * cap * kRing);
    b->d_io = reinterpret_cast<TickIO *>(b->arena + o_io);
    b->d_ptrs = reinterpret_cast<hmi_pointer *>(b->arena + o_ptr);
    b->d_err = reinterpret_cast<uint32_t *>(b->arena + o_err);
    b->cap = cap;
    return true;
}

// Stream groups of a plan left at groups = 0: one when every stream can run
// in the persistent tick (band streams: a group's persistent launch already
// fills the GPU), else two overlapping chains.
int default_groups(hmi_stream *const *s, int n, const hmi_tuning &t)
{
    bool fusable = t.fused != 0;
    for (int i = 0; i < n && fusable; ++i)
        fusable = s[i]->L.mix_k == 0 && 2 * (s[i]->p.open_iters + s[i]->p.close_iters) <= kTickMaxHalo;
    return fusable ? 1 : std::min(2, n);
}

hmi_batch *batch_new(hmi_stream *const *s, int n, int ngroups)
{
    if (!streams_ok(s, n)) {
        fail(HMI_ERR_INVALID_ARG);
        return nullptr;
    }
    hmi_batch *b = new (std::nothrow) hmi_batch();
    if (!b) {
        fail(HMI_ERR_NO_MEMORY);
        return nullptr;
    }
    b->dev = s[0]->dev;
    b->n = n;
    b->s.assign(s, s + n);
    b->tune = kDefaultTuning;
    b->tune.groups = ngroups;
    if (cudaSetDevice(b->dev) != cudaSuccess) {
        delete b;
        cuda_fail(cudaErrorInvalidDevice);
        return nullptr;
    }
    bool ok = batch_alloc_io(b, n) &&
              cudaMallocHost(&b->h_err, sizeof(uint32_t)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->pipe_ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->cs2, cudaStreamNonBlocking) == cudaSuccess;
    for (auto &e : b->side_done)
        ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < kRing; ++i)
        ok = cudaEventCreateWithFlags(&b->slot_ev[i], cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i <= kTickKernels; ++i) ok = cudaEventCreate(&b->dummy_ev[i]) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        batch_free(b);
        fail(HMI_ERR_NO_MEMORY);
        return nullptr;
    }
    *b->h_err = 0;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
    b->num_sms = sms > 0 ? sms : 1;
    if (plan_build(b, ngroups) != HMI_OK) {
        const int st = g_last_error;
        batch_free(b);
        fail(st);
        return nullptr;
    }
    return b;
}

// Kernels of one tick with the slot's pointer table.  Each group runs its
// chain (luma, classify, morphology, block components, finish) on its own
// branch; group g starts its luma after group g-1's luma, so the HBM-bound
// passes of later groups overlap the latency-bound tail of earlier ones.
// With one group, event records (or event nodes) bracket the classify kernel.
// Launch parameters of group G for the tick in `slot`: its pointer table, and
// the tick phase (slot mod kPhases; slots are taken in turn and the ring is a
// multiple of kPhases) that picks the raw bits, the gains and the skin queue,
// so that up to kPhases consecutive ticks never share them.
BatchDev tick_dev(const hmi_batch *b, const Group &G, int slot)
{
    static_assert(kRing % kPhases == 0, "consecutive slots must have distinct phases");
    BatchDev bd = G.bd;
    bd.io = b->d_io + (size_t)slot * b->n + G.off;
    bd.phase = slot % kPhases;
    bd.ds = b->ds_tab + (size_t)bd.phase * b->n + G.off;   // this phase's bit mask, counts, flags
    bd.skin_count = G.skin_count_p[bd.phase];
    bd.skin_list = G.skin_list_p[bd.phase];
    bd.cc_count = G.cc_count_p[bd.phase];
    bd.cc_list = G.cc_list_p[bd.phase];
    return bd;
}

cudaError_t upload_io(hmi_batch *b, int slot, cudaStream_t cs)
{
    return cudaMemcpyAsync(b->d_io + (size_t)slot * b->n, b->h_io + (size_t)slot * b->n,
                           sizeof(TickIO) * b->n, cudaMemcpyHostToDevice, cs);
}

// Tick kernels k0 .. k1 - 1 of a single-group plan, with an event after each
// (and one before the first) when ev is given.
cudaError_t enqueue_kernels(hmi_batch *b, int slot, cudaStream_t cs, int k0, int k1, const cudaEvent_t *ev,
                            bool capture)
{
    const BatchDev bd = tick_dev(b, b->groups[0], slot);
    const unsigned flags = capture ? cudaEventRecordExternal : 0;
    cudaError_t e;
    if (ev && (e = cudaEventRecordWithFlags(ev[k0], cs, flags)) != cudaSuccess) return e;
    for (int k = k0; k < k1; ++k) {
        NvtxRange range(tick_kernel_name(k));
        if ((e = launch_tick_kernel(k, bd, cs, b->num_sms)) != cudaSuccess) return e;
        if (ev && (e = cudaEventRecordWithFlags(ev[k + 1], cs, flags)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t enqueue_tick(hmi_batch *b, int slot, cudaStream_t cs, const cudaEvent_t *ev, bool capture)
{
    cudaError_t e;
    if ((e = upload_io(b, slot, cs)) != cudaSuccess) return e;
    const int ng = (int)b->groups.size();
    if (ng == 1) return enqueue_kernels(b, slot, cs, 0, kTickKernels, ev, capture);
    if ((e = cudaEventRecord(b->ev_fork, cs)) != cudaSuccess) return e;
    for (int g = 0; g < ng; ++g) {
        Group &G = b->groups[g];
        const BatchDev bd = tick_dev(b, G, slot);
        if ((e = cudaStreamWaitEvent(G.cs, b->ev_fork, 0)) != cudaSuccess) return e;
        if (g > 0 && (e = cudaStreamWaitEvent(G.cs, b->groups[g - 1].ev_luma, 0)) != cudaSuccess) return e;
        if ((e = launch_tick_kernel(0, bd, G.cs, b->num_sms)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(G.ev_luma, G.cs)) != cudaSuccess) return e;
        for (int k = 1; k < kTickKernels; ++k)
            if ((e = launch_tick_kernel(k, bd, G.cs, b->num_sms)) != cudaSuccess) return e;
        if ((e = cudaEventRecord(G.ev_done, G.cs)) != cudaSuccess) return e;
    }
    for (int g = 0; g < ng; ++g)
        if ((e = cudaStreamWaitEvent(cs, b->groups[g].ev_done, 0)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Stages of a pipelined tick: the first kernel of each of its `depth` stages,
// then kTickKernels.  Depth 2: {luma, band test, mixture, re-learning}
// {gray/hue, morphology, blocks, finish}; depth 3: {luma} {band test, mixture,
// re-learning} {gray/hue .. finish}.  The first stages are bandwidth-bound, the last is
// latency-bound; the band is only read and re-formed in the middle stage.
void stage_bounds(int depth, int *first, bool fused)
{
    constexpr int kTail = kTickTail;   // first kernel of the latency-bound tail (gray/hue tests)
    if (fused) {   // {persistent tick, re-learning} {block components, merge}; a third stage
        first[0] = 0;   // would part re-learning from the band test it follows
        first[1] = kTail;
        first[2] = kTickKernels;
        first[3] = kTickKernels;
    } else if (depth >= 3) {
        first[0] = 0;
        first[1] = 1;
        first[2] = kTail;
        first[3] = kTickKernels;
    } else {
        first[0] = 0;
        first[1] = kTail;
        first[2] = kTickKernels;
    }
}

// One pipelined call (single group): stage 0 of `slot` on cs and, beside it,
// stage j + 1 of the in-flight tick pend[j] on branch stream j; cs then waits
// for the branches.  Concurrent stages belong to consecutive ticks, whose
// phases differ, so they touch disjoint per-tick state.
cudaError_t enqueue_pipelined(hmi_batch *b, int slot, const int *pend, int npend, int depth, cudaStream_t cs)
{
    int first[kPhases + 1];
    stage_bounds(depth, first, b->groups[0].bd.fused != 0);
    cudaStream_t side[kPhases - 1] = {b->groups[0].cs, b->cs2};
    cudaError_t e;
    if (npend > 0 && (e = cudaEventRecord(b->ev_fork, cs)) != cudaSuccess) return e;
    for (int j = 0; j < npend; ++j) {
        if ((e = cudaStreamWaitEvent(side[j], b->ev_fork, 0)) != cudaSuccess) return e;
        if ((e = enqueue_kernels(b, pend[j], side[j], first[j + 1], first[j + 2], nullptr, false)) != cudaSuccess)
            return e;
        if ((e = cudaEventRecord(b->side_done[j], side[j])) != cudaSuccess) return e;
    }
    if ((e = upload_io(b, slot, cs)) != cudaSuccess) return e;
    if ((e = enqueue_kernels(b, slot, cs, first[0], first[1], nullptr, false)) != cudaSuccess) return e;
    for (int j = 0; j < npend; ++j)
        if ((e = cudaStreamWaitEvent(cs, b->side_done[j], 0)) != cudaSuccess) return e;
    return cudaSuccess;
}

// Graph of a full pipelined call in `slot` (every earlier stage in flight:
// the ticks of the depth - 1 slots before it).
int build_pipe_graph(hmi_batch *b, int slot, int depth)
{
    int pend[kPhases - 1];
    for (int j = 0; j + 1 < depth; ++j) pend[j] = (slot + kRing - 1 - j) % kRing;
    cudaGraph_t g = nullptr;
    HMI_CUDA(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_pipelined(b, slot, pend, depth - 1, depth, b->cs);
    cudaError_t e2 = cudaStreamEndCapture(b->cs, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e != cudaSuccess ? e : e2);
    }
    e = cudaGraphInstantiate(&b->pipe_graph[slot], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->pipe_graph[slot] = nullptr;
        return cuda_fail(e);
    }
    return HMI_OK;
}

// Run the remaining stages of the in-flight pipelined ticks on cs, oldest
// first.
int flush_pending(hmi_batch *b, cudaStream_t cs)
{
    if (b->npend == 0) return HMI_OK;
    int first[kPhases + 1];
    stage_bounds(b->pend_depth, first, b->groups[0].bd.fused != 0);
    const int npend = b->npend;
    b->npend = 0;
    HMI_CUDA(cudaStreamWaitEvent(cs, b->pipe_ev, 0));
    for (int j = npend - 1; j >= 0; --j) {
        HMI_CUDA(enqueue_kernels(b, b->pend[j], cs, first[j + 1], kTickKernels, nullptr, false));
        HMI_CUDA(cudaEventRecord(b->slot_ev[b->pend[j]], cs));
    }
    return HMI_OK;
}

// Capture one tick into a graph: the plain form, or (profiling, single group)
// the form with event-record nodes around each kernel.
int build_graph(hmi_batch *b, int slot, bool profiling)
{
    cudaGraph_t g = nullptr;
    HMI_CUDA(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_tick(b, slot, b->cs, profiling ? b->dummy_ev : nullptr, true);
    cudaError_t e2 = cudaStreamEndCapture(b->cs, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e != cudaSuccess ? e : e2);
    }
    if (profiling) {
        size_t nn = 0;
        cudaGraphGetNodes(g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
        for (auto nd : nodes) {
            cudaGraphNodeType t;
            cudaGraphNodeGetType(nd, &t);
            if (t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            cudaGraphEventRecordNodeGetEvent(nd, &ev);
            for (int k = 0; k <= kTickKernels; ++k)
                if (ev == b->dummy_ev[k]) b->ev_node[slot][k] = nd;
        }
        for (int k = 0; k <= kTickKernels; ++k)
            if (!b->ev_node[slot][k]) {
                cudaGraphDestroy(g);
                return fail(HMI_ERR_DEVICE);
            }
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e);
    }
    if (profiling) {
        b->pgraph[slot] = x;
        b->pgraph_src[slot] = g;
    } else {
        b->graph[slot] = x;
        cudaGraphDestroy(g);
    }
    return HMI_OK;
}

// Fill slot pointers for one tick (permuted order).  Frames and masks not
// usable in place are staged through the stream's own buffers; returns which
// masks need a copy out.
int prepare_slot(hmi_batch *b, int slot, const uint8_t *const *frames, uint8_t *const *masks,
                 bool async_mode, cudaStream_t cs, std::vector<int> *mask_copy)
{
    TickIO *io = b->h_io + (size_t)slot * b->n;
    for (int i = 0; i < b->n; ++i) {
        hmi_stream *s = b->s[i];
        s->used = true;
        TickIO &t = io[b->pos[i]];
        const uint8_t *f = frames[i];
        if (!f) return fail(HMI_ERR_INVALID_ARG);
        bool dev = b->seen_device(f);
        if (!dev) {
            dev = is_device_ptr(f);
            if (dev) b->remember_device(f);
        }
        // a pinned host frame with 16-pixel rows: k_luma copies it into the
        // tick phase's staging frame while it sums it (no copy engine, one
        // pass over the host link)
        const uint8_t *pin = (!dev && (s->w % 16) == 0) ? b->pinned_dev(f) : nullptr;
        if (pin && (reinterpret_cast<uintptr_t>(pin) & 15u) != 0) pin = nullptr;
        t.src = pin;
        if (async_mode && !dev && !pin) return fail(HMI_ERR_INVALID_ARG);
        if (dev && (s->w % 16) == 0 && (reinterpret_cast<uintptr_t>(f) & 15u) == 0) {
            t.frame = f;
            t.frame_pitch = 3LL * s->w;
        } else if (pin) {
            t.frame = s->arena + s->L.frame_ph[slot % kPhases];
            t.frame_pitch = s->L.fpitch;   // 3 w: w is a multiple of 16
        } else {
            if (3 * (size_t)s->w == (size_t)s->L.fpitch) {
                HMI_CUDA(cudaMemcpyAsync(s->d_frame, f, 3 * (size_t)s->w * s->h, cudaMemcpyDefault, cs));
            } else {
                HMI_CUDA(cudaMemcpy2DAsync(s->d_frame, s->L.fpitch, f, 3 * (size_t)s->w, 3 * (size_t)s->w,
                                           s->h, cudaMemcpyDefault, cs));
            }
            t.frame = s->d_frame;
            t.frame_pitch = s->L.fpitch;
        }
        uint8_t *m = (masks != nullptr) ? masks[i] : nullptr;
        if (m == nullptr) {
            t.mask = nullptr;
        } else if (b->seen_device(m) || is_device_ptr(m)) {
            b->remember_device(m);
            t.mask = m;
        } else {
            if (async_mode) return fail(HMI_ERR_INVALID_ARG);
            t.mask = s->d_mask;
            if (mask_copy) mask_copy->push_back(i);
        }
    }
    return HMI_OK;
}

int acquire_slot(hmi_batch *b)
{
    const int slot = b->next;
    b->next = (b->next + 1) % kRing;
    if (b->slot_used[slot]) {
        cudaError_t e = cudaEventSynchronize(b->slot_ev[slot]);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return slot;
}

int run_tick(hmi_batch *b, int slot, cudaStream_t cs, bool use_graph)
{
    const cudaEvent_t *ev = nullptr;
    if (b->prof_used < b->prof_max && b->groups.size() == 1) {
        ev = b->prof_ev.data() + (size_t)(kTickKernels + 1) * b->prof_used;
        b->prof_used++;
    }
    if (use_graph && ev) {
        if (!b->pgraph[slot]) {
            int st = build_graph(b, slot, true);
            if (st != HMI_OK) return st;
        }
        for (int k = 0; k <= kTickKernels; ++k)
            HMI_CUDA(cudaGraphExecEventRecordNodeSetEvent(b->pgraph[slot], b->ev_node[slot][k], ev[k]));
        HMI_CUDA(cudaGraphLaunch(b->pgraph[slot], cs));
    } else if (use_graph) {
        if (!b->graph[slot]) {
            int st = build_graph(b, slot, false);
            if (st != HMI_OK) return st;
        }
        HMI_CUDA(cudaGraphLaunch(b->graph[slot], cs));
    } else {
        HMI_CUDA(enqueue_tick(b, slot, cs, ev, false));
    }
    HMI_CUDA(cudaEventRecord(b->slot_ev[slot], cs));
    b->slot_used[slot] = true;
    return HMI_OK;
}

bool all_learned(hmi_batch *b)
{
    for (auto s : b->s)
        if (!s->learned) return false;
    return true;
}

int batch_sync(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
               hmi_pointer *ptrs)
{
    NvtxRange range("hmi tick (synchronous)");
    if (!b || !frames) return fail(HMI_ERR_INVALID_ARG);
    if (!all_learned(b)) return fail(HMI_ERR_NOT_LEARNED);
    HMI_CUDA(cudaSetDevice(b->dev));
    int st0 = flush_pending(b, b->cs);
    if (st0 != HMI_OK) return st0;
    int slot = acquire_slot(b);
    if (slot < 0) return slot;
    std::vector<int> mcopy;
    int st = prepare_slot(b, slot, frames, masks, false, b->cs, &mcopy);
    if (st != HMI_OK) return st;
    TickIO *io = b->h_io + (size_t)slot * b->n;
    for (int i = 0; i < b->n; ++i) io[b->pos[i]].ptr_out = b->d_ptrs + i;
    st = run_tick(b, slot, b->cs, false);
    if (st != HMI_OK) return st;
    for (int i : mcopy) {
        hmi_stream *s = b->s[i];
        HMI_CUDA(cudaMemcpyAsync(masks[i], s->d_mask, (size_t)s->w * s->h, cudaMemcpyDefault, b->cs));
    }
    if (ptrs) HMI_CUDA(cudaMemcpyAsync(ptrs, b->d_ptrs, sizeof(hmi_pointer) * b->n, cudaMemcpyDefault, b->cs));
    HMI_CUDA(cudaMemcpyAsync(b->h_err, b->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, b->cs));
    HMI_CUDA(cudaStreamSynchronize(b->cs));
    if (*b->h_err) {
        const uint32_t e = *b->h_err;
        *b->h_err = 0;
        HMI_CUDA(cudaMemset(b->d_err, 0, sizeof(uint32_t)));
        return fail((e & kErrBounds) ? HMI_ERR_DEVICE : HMI_ERR_DEVICE_TIMEOUT);
    }
    return HMI_OK;
}

int batch_async(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
                hmi_pointer *ptrs, void *cuda_stream, int use_graph)
{
    NvtxRange range("hmi tick (asynchronous)");
    if (!b || !frames) return fail(HMI_ERR_INVALID_ARG);
    if (!all_learned(b)) return fail(HMI_ERR_NOT_LEARNED);
    if (ptrs && !is_device_ptr(ptrs)) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(b->dev));
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    int st = flush_pending(b, cs);
    if (st != HMI_OK) return st;
    int slot = acquire_slot(b);
    if (slot < 0) return slot;
    st = prepare_slot(b, slot, frames, masks, true, cs, nullptr);
    if (st != HMI_OK) return st;
    TickIO *io = b->h_io + (size_t)slot * b->n;
    for (int i = 0; i < b->n; ++i) io[b->pos[i]].ptr_out = ptrs ? ptrs + i : nullptr;
    return run_tick(b, slot, cs, use_graph != 0);
}

int batch_pipelined(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
                    hmi_pointer *ptrs, void *cuda_stream, int use_graph)
{
    NvtxRange range("hmi tick (pipelined)");
    if (!b || !frames || b->groups.size() != 1) return fail(HMI_ERR_INVALID_ARG);
    if (!all_learned(b)) return fail(HMI_ERR_NOT_LEARNED);
    if (ptrs && !is_device_ptr(ptrs)) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(b->dev));
    cudaStream_t cs = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int slot = acquire_slot(b);
    if (slot < 0) return slot;
    int st = prepare_slot(b, slot, frames, masks, true, cs, nullptr);
    if (st != HMI_OK) return st;
    TickIO *io = b->h_io + (size_t)slot * b->n;
    for (int i = 0; i < b->n; ++i) io[b->pos[i]].ptr_out = ptrs ? ptrs + i : nullptr;
    const int depth = b->tune.pipeline_depth;
    const int npend = b->npend;
    int pend[kPhases - 1];
    for (int j = 0; j < npend; ++j) pend[j] = b->pend[j];
    bool full = npend == depth - 1;
    for (int j = 0; j < npend; ++j) full = full && pend[j] == (slot + kRing - 1 - j) % kRing;
    if (npend > 0) HMI_CUDA(cudaStreamWaitEvent(cs, b->pipe_ev, 0));
    if (use_graph && full) {
        if (!b->pipe_graph[slot]) {
            st = build_pipe_graph(b, slot, depth);
            if (st != HMI_OK) return st;
        }
        HMI_CUDA(cudaGraphLaunch(b->pipe_graph[slot], cs));
    } else {
        HMI_CUDA(enqueue_pipelined(b, slot, pend, npend, depth, cs));
    }
    HMI_CUDA(cudaEventRecord(b->slot_ev[slot], cs));
    b->slot_used[slot] = true;
    for (int j = 0; j < npend; ++j) HMI_CUDA(cudaEventRecord(b->slot_ev[pend[j]], cs));
    HMI_CUDA(cudaEventRecord(b->pipe_ev, cs));
    // pend[j] has now run stage j + 1; it stays in flight while stages remain
    b->pend[0] = slot;
    int k = 1;
    for (int j = 0; j < npend && k < depth - 1; ++j)
        if (j + 2 < depth) b->pend[k++] = pend[j];
    b->npend = std::min(k, depth - 1);
    b->pend_depth = depth;
    return HMI_OK;
}

bool tuning_ok(const hmi_tuning &t)
{
    return t.piece_chunks >= 32 && t.piece_chunks <= 65536 && t.piece_chunks % 32 == 0 &&
           t.luma_ctas_per_sm >= 0 && t.luma_ctas_per_sm <= 32 && t.skin_ctas_per_sm >= 1 &&
           t.skin_ctas_per_sm <= 32 && t.cc_ctas_per_sm >= 1 && t.cc_ctas_per_sm <= 32 &&
           t.groups >= 0 && t.groups <= 64 && t.pipeline_depth >= 2 && t.pipeline_depth <= kPhases &&
           (t.fused == 0 || t.fused == 1) && t.queue_lag >= 0 && t.queue_lag <= (1 << 20) &&
           (t.merge_threads == 0 || t.merge_threads == 256 || t.merge_threads == 512 ||
            t.merge_threads == 1024);
}

// Apply a launch shape: the plan is re-made with the device idle.
int batch_retune(hmi_batch *b, const hmi_tuning &t)
{
    if (!b || !tuning_ok(t)) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(b->dev));
    const int st = flush_pending(b, b->cs);
    if (st != HMI_OK) return st;
    HMI_CUDA(cudaDeviceSynchronize());
    plan_free(b);
    for (int i = 0; i < kRing; ++i) b->slot_used[i] = false;
    b->tune = t;
    return plan_build(b, t.groups > 0 ? t.groups : default_groups(b->s.data(), b->n, t));
}

// Microseconds per tick of `ticks` ticks of `frames` with the current plan
// (pipelined or plain graph ticks on the batch's own stream, masks and
// pointers not written), after three untimed ticks.
int time_ticks(hmi_batch *b, const uint8_t *const *frames, int ticks, bool pipelined, double *us)
{
    auto one = [&]() {
        return pipelined ? batch_pipelined(b, frames, nullptr, nullptr, b->cs, 1)
                         : batch_async(b, frames, nullptr, nullptr, b->cs, 1);
    };
    for (int i = 0; i < 3; ++i) {
        const int st = one();
        if (st != HMI_OK) return st;
    }
    int st = flush_pending(b, b->cs);
    if (st != HMI_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(cudaErrorMemoryAllocation);
    }
    cudaEventRecord(e0, b->cs);
    for (int i = 0; i < ticks && st == HMI_OK; ++i) st = one();
    if (st == HMI_OK) st = flush_pending(b, b->cs);
    cudaEventRecord(e1, b->cs);
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != HMI_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e);
    *us = 1e3 * ms / ticks;
    return HMI_OK;
}

int batch_autotune(hmi_batch *b, const uint8_t *const *frames, int ticks, bool pipelined,
                   hmi_tuning *best_out, double *best_us_out)
{
    NvtxRange range("hmi autotune");
    if (!b || !frames || ticks < 2 || ticks > 10000) return fail(HMI_ERR_INVALID_ARG);
    if (!all_learned(b)) return fail(HMI_ERR_NOT_LEARNED);
    HMI_CUDA(cudaSetDevice(b->dev));
    int st = flush_pending(b, b->cs);
    if (st != HMI_OK) return st;
    HMI_CUDA(cudaDeviceSynchronize());
    // the streams' click state, pointer history and adaptive background
    // (band, re-learning sums, mixture), put back afterwards
    std::vector<std::pair<void *, size_t>> keep;
    for (hmi_stream *s : b->s) {
        const Layout &L = s->L;
        keep.emplace_back(s->st, sizeof(StreamState));
        keep.emplace_back(s->ds.hist, sizeof(uint32_t) * std::max<int>(s->p.click_window, 1));
        keep.emplace_back(s->arena + L.lo, (size_t)L.h * L.fpitch);
        keep.emplace_back(s->arena + L.hi, (size_t)L.h * L.fpitch);
        if (L.rpx) {
            keep.emplace_back(s->arena + L.rS, L.rpx * 3 * 2);
            keep.emplace_back(s->arena + L.rQ, L.rpx * 3 * 4);
            keep.emplace_back(s->arena + L.rmin, L.rpx * 3);
            keep.emplace_back(s->arena + L.rmax, L.rpx * 3);
            keep.emplace_back(s->arena + L.rcnt, L.rpx);
        }
        if (L.mix_k) keep.emplace_back(s->arena + L.mix, L.mbytes);
    }
    size_t total = 0;
    for (auto &k : keep) total += k.second;
    uint8_t *save = nullptr;
    HMI_CUDA(cudaMalloc(&save, total));
    size_t off = 0;
    for (auto &k : keep) {
        cudaMemcpyAsync(save + off, k.first, k.second, cudaMemcpyDeviceToDevice, b->cs);
        off += k.second;
    }
    const hmi_tuning start = b->tune;
    hmi_tuning cur = start;
    if (pipelined) cur.groups = 1;
    double cur_us = 0.0;
    st = batch_retune(b, cur);
    if (st == HMI_OK) st = time_ticks(b, frames, ticks, pipelined, &cur_us);
    // one parameter at a time, each over its candidate values
    struct Axis {
        int32_t hmi_tuning::*field;
        std::vector<int32_t> values;
    };
    std::vector<Axis> axes = {{&hmi_tuning::fused, {0, 1}},
                              {&hmi_tuning::piece_chunks, {128, 256, 512, 1024, 2048}},
                              {&hmi_tuning::luma_ctas_per_sm, {0, 2, 3, 4, 6}},
                              {&hmi_tuning::skin_ctas_per_sm, {4, 8, 16}},
                              {&hmi_tuning::cc_ctas_per_sm, {4, 8, 16}},
                              {&hmi_tuning::merge_threads, {256, 512, 1024}}};
    if (pipelined) axes.push_back({&hmi_tuning::pipeline_depth, {2, 3}});
    else axes.push_back({&hmi_tuning::groups, {1, 2, 3}});
    for (const Axis &ax : axes) {
        for (int32_t v : ax.values) {
            if (st != HMI_OK || cur.*ax.field == v) continue;
            hmi_tuning cand = cur;
            cand.*ax.field = v;
            double us = 0.0;
            st = batch_retune(b, cand);
            if (st == HMI_OK) st = time_ticks(b, frames, ticks, pipelined, &us);
            if (st == HMI_OK && us < cur_us) {
                cur = cand;
                cur_us = us;
            }
        }
    }
    const int st_apply = batch_retune(b, st == HMI_OK ? cur : start);
    cudaDeviceSynchronize();
    off = 0;
    for (auto &k : keep) {
        cudaMemcpy(k.first, save + off, k.second, cudaMemcpyDeviceToDevice);
        off += k.second;
    }
    cudaFree(save);
    if (st != HMI_OK) return st;
    if (st_apply != HMI_OK) return st_apply;
    if (best_out) *best_out = cur;
    if (best_us_out) *best_us_out = cur_us;
    return HMI_OK;
}

int batch_set_groups(hmi_batch *b, int ng)
{
    if (!b || ng < 1 || ng > 64) return fail(HMI_ERR_INVALID_ARG);
    hmi_tuning t = b->tune;
    t.groups = ng;
    return batch_retune(b, t);
}

// Give a stream's arena back (stream-ordered for pooled arenas) and destroy
// its CUDA stream; the pool is trimmed when the device's last stream goes.
void release_arena(hmi_stream *s)
{
    if (s->arena) {
        if (s->pooled) {
            cudaFreeAsync(s->arena, s->cs);
            cudaStreamSynchronize(s->cs);
            if (--g_pools.live[s->dev] == 0) cudaMemPoolTrimTo(g_pools.pool[s->dev], 0);
        } else {
            cudaFree(s->arena);
        }
        s->arena = nullptr;
    }
    if (s->cs) {
        cudaStreamSynchronize(s->cs);
        cudaStreamDestroy(s->cs);
        s->cs = nullptr;
    }
}

// A stream whose device state is allocated and initialised in the order of
// CUDA stream `order` (no host synchronisation: usable by work enqueued on
// `order`, and by any work once `order` has been synchronised), or, with
// order NULL, on its own CUDA stream and synchronised before returning.
hmi_stream *create_stream_on(int w, int h, const hmi_params *p, cudaStream_t order)
{
    hmi_params d;
    hmi_default_params(&d);
    const hmi_params &pp = p ? *p : d;
    if (w < 1 || h < 1 || w > kMaxDim || h > kMaxDim || !params_valid(pp)) {
        fail(HMI_ERR_INVALID_ARG);
        return nullptr;
    }
    hmi_stream *s = new (std::nothrow) hmi_stream();
    if (!s) {
        fail(HMI_ERR_NO_MEMORY);
        return nullptr;
    }
    s->w = w;
    s->h = h;
    s->p = pp;
    s->L = make_layout(w, h, pp);
    if (cudaGetDevice(&s->dev) != cudaSuccess) {
        delete s;
        cuda_fail(cudaErrorNoDevice);
        return nullptr;
    }
    if (cudaStreamCreateWithFlags(&s->cs, cudaStreamNonBlocking) != cudaSuccess) {
        (void)cudaGetLastError();
        delete s;
        fail(HMI_ERR_DEVICE);
        return nullptr;
    }
    cudaStream_t cs = order ? order : s->cs;
    cudaMemPool_t pool = arena_pool(s->dev);
    cudaError_t ae = pool ? cudaMallocFromPoolAsync(reinterpret_cast<void **>(&s->arena), s->L.total, pool, cs)
                          : cudaMalloc(&s->arena, s->L.total);
    if (ae != cudaSuccess) {
        (void)cudaGetLastError();
        cudaStreamDestroy(s->cs);
        delete s;
        fail(HMI_ERR_NO_MEMORY);
        return nullptr;
    }
    s->pooled = pool != nullptr;
    if (s->pooled) g_pools.live[s->dev]++;
    uint8_t *a = s->arena;
    s->d_frame = a + s->L.frame;
    s->d_mask = a + s->L.mask;
    s->d_S = reinterpret_cast<uint32_t *>(a + s->L.S);
    s->d_Q = reinterpret_cast<uint32_t *>(a + s->L.Q);
    s->d_vmin = a + s->L.vmin;
    s->d_vmax = a + s->L.vmax;
    s->st = reinterpret_cast<StreamState *>(a + s->L.st);
    s->d_ds = reinterpret_cast<DevStream *>(a + s->L.ds);
    s->d_ptr = reinterpret_cast<hmi_pointer *>(a + s->L.ptr);
    fill_devstream(s);
    for (int k = 0; k < kPhases; ++k) s->ds_phase[k] = phase_view(s->ds, k);
    bool ok = cudaMemsetAsync(s->arena, 0, s->L.total, cs) == cudaSuccess &&
              cudaMemcpyAsync(s->d_ds, s->ds_phase, sizeof(DevStream) * kPhases, cudaMemcpyHostToDevice, cs) == cudaSuccess &&
              (order != nullptr || cudaStreamSynchronize(cs) == cudaSuccess);
    if (!ok) {
        (void)cudaGetLastError();
        if (order) cudaStreamSynchronize(order);
        release_arena(s);
        delete s;
        fail(HMI_ERR_NO_MEMORY);
        return nullptr;
    }
    return s;
}

hmi_batch *self_plan(hmi_stream *s)
{
    if (!s->self) {
        hmi_stream *one = s;
        if (cudaSetDevice(s->dev) != cudaSuccess) {
            cuda_fail(cudaErrorInvalidDevice);
            return nullptr;
        }
        s->self = batch_new(&one, 1, 1);
    }
    return s->self;
}

// Re-plan an idle batch (no tick in flight) over another set of streams,
// reusing its buffers, branch streams and events where they are large enough,
// so that a plan can follow streams joining and leaving without allocating on
// every change.  The batch's error word is cleared.
int batch_replan(hmi_batch *b, hmi_stream *const *s, int n, int ngroups)
{
    if (!b || !streams_ok(s, n) || s[0]->dev != b->dev) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(b->dev));
    plan_free_graphs(b);
    if (n > b->cap && !batch_alloc_io(b, std::min(kMaxBatch, std::max(n, 2 * b->cap)))) {
        plan_free(b);
        return fail(HMI_ERR_NO_MEMORY);
    }
    b->n = n;
    b->s.assign(s, s + n);
    for (int i = 0; i < kRing; ++i) b->slot_used[i] = false;
    b->next = 0;
    b->seen.clear();
    b->tune.groups = ngroups;
    HMI_CUDA(cudaMemsetAsync(b->d_err, 0, sizeof(uint32_t), b->cs));
    return plan_build(b, ngroups);
}

// An empty Gaussian mixture (every plane zero: no component), before its
// learning frames.
cudaError_t enqueue_mix_reset(hmi_stream *s, cudaStream_t cs)
{
    if (!s->L.mix_k) return cudaSuccess;
    return cudaMemsetAsync(s->arena + s->L.mix, 0, s->L.mbytes, cs);
}

// Band of a stream from its learned sums after n frames (Sec. 3.1 (i)), in
// the padded row layout; the padding bytes are zeroed first.
cudaError_t enqueue_band(hmi_stream *s, int n, cudaStream_t cs)
{
    const size_t bytes = (size_t)s->h * s->L.fpitch;
    cudaError_t e = cudaSuccess;
    if (s->L.rpx) {   // the re-learning sums restart with the learned band
        const Layout &L = s->L;
        e = cudaMemsetAsync(s->arena + L.rS, 0, L.rpx * 3 * 2, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->arena + L.rQ, 0, L.rpx * 3 * 4, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->arena + L.rmin, 0xff, L.rpx * 3, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->arena + L.rmax, 0, L.rpx * 3, cs);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->arena + L.rcnt, 0, L.rpx, cs);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(s->arena + s->L.lo, 0, bytes, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->arena + s->L.hi, 0, bytes, cs);
    if (e == cudaSuccess)
        e = launch_learn_band(s->d_S, s->d_Q, s->d_vmin, s->d_vmax, n, s->p.bg_k_num, s->p.bg_k_den,
                              s->p.bg_margin, s->w, s->h, s->L.fpitch, s->arena + s->L.lo,
                              s->arena + s->L.hi, s->st, cs);
    return e;
}


// ===========================================================================
// Server: admission by device-memory budget, resident streams, continuous
// batching by a dispatcher thread (one tick over all admitted streams per
// round, streams without a pending frame marked inactive by a null frame).
// ===========================================================================
struct SrvFrame {
    const uint8_t *host = nullptr;   // pinned copy, or the caller's buffer
    size_t bytes = 0;
    uint64_t tag = 0, submit_ns = 0;
    bool owned = false;              // host is a pooled copy to give back
};

struct SrvStream {
    hmi_stream *s = nullptr;         // null until the dispatcher has created it
    int w = 0, h = 0;
    hmi_params p{};
    size_t bytes = 0;
    bool pending = false;            // admitted, creation left to the dispatcher
    bool failed = false;             // creation failed: queued frames are returned as errors
    bool releasing = false;
    int learn_n = 0, learn_done = 0;   // online learning: frames wanted / taken
    std::deque<SrvFrame> q;
};

struct SrvTake {
    SrvFrame f;
    SrvStream *ss = nullptr;
    bool learning = false;
    const uint8_t *src = nullptr;   // a pinned frame the luma pass reads itself
};

hmi_pointer empty_pointer()
{
    hmi_pointer p;
    memset(&p, 0, sizeof(p));
    p.x = p.y = -1.0f;
    p.x0 = p.y0 = p.x1 = p.y1 = -1;
    p.label = -1;
    return p;
}

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

}  // namespace

struct hmi_server {
    int dev = 0;
    size_t budget = 0, used = 0;
    int max_queue = 8;
    std::mutex mu;
    std::condition_variable work_cv, done_cv;
    std::map<int, SrvStream> streams;
    int next_id = 1;
    std::deque<hmi_server_result> done;
    std::map<size_t, std::vector<uint8_t *>> pool;   // free pinned buffers by size
    bool stop = false, dirty = false;
    std::thread worker;
    // dispatcher-only state
    hmi_batch *plan = nullptr;
    std::vector<int> plan_ids;
    cudaStream_t cs = nullptr;
    // per-round buffers, two sets: a round is posted after the next one has
    // been issued (its pointers, error word and learning table stay put)
    hmi_pointer *h_ptrs[2] = {}, *d_ptrs[2] = {};
    int ptr_cap = 0;
    LearnItem *h_items[2] = {}, *d_items = nullptr;   // a round's learning frames
    int item_cap = 0;
    uint32_t *h_err[2] = {};      // the plan's error word after each round (pinned)
    cudaEvent_t ev[2] = {};       // end of each round's device work
    int next_buf = 0;
    struct Flight {               // a round issued to the device, not yet posted
        std::vector<SrvTake> take;
        std::vector<int> ids;     // stream ids of the plan's streams, in plan order
        hmi_server_round rec;
        bool any_active = false;
        int status = HMI_OK;
        int buf = 0;
    };
    std::deque<Flight> flights;   // oldest first, at most two
    uint64_t ticks = 0, frames = 0;
    std::vector<hmi_server_round> rounds;   // ring of kRoundLog records (under mu)
    uint64_t rounds_written = 0;
};

namespace {

uint8_t *pool_get(hmi_server *v, size_t bytes)
{
    auto &fl = v->pool[bytes];
    if (!fl.empty()) {
        uint8_t *p = fl.back();
        fl.pop_back();
        return p;
    }
    uint8_t *p = nullptr;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

// A dispatcher round is issued (copies, learning, tick and the read-back of
// pointers and the error word, all on the server's CUDA stream, closed by an
// event) and posted later, once its event has completed, so that the next
// round's host work and issue overlap this round's device work.  Rounds that
// change the set of streams (creation, retirement, re-plan) wait until no
// round is in flight.
void complete_round(hmi_server *v);

// Post every round in flight (waiting for the device).
void drain_rounds(hmi_server *v)
{
    while (!v->flights.empty()) complete_round(v);
}

// Whether the next round has setup work (streams to create or retire, or a
// plan to re-make).
bool setup_pending(hmi_server *v)
{
    std::unique_lock<std::mutex> lk(v->mu);
    if (v->dirty) return true;
    for (auto &kv : v->streams) {
        const SrvStream &ss = kv.second;
        if (ss.pending || ss.failed || (ss.releasing && ss.q.empty())) return true;
    }
    return false;
}

// One dispatcher round; returns false when there was nothing to do.
constexpr int kRoundLog = 16384;

void log_round(hmi_server *v, const hmi_server_round &rec)   // under v->mu
{
    if (v->rounds.size() < (size_t)kRoundLog) v->rounds.push_back(rec);
    else v->rounds[v->rounds_written % kRoundLog] = rec;
    v->rounds_written += 1;
}

bool server_issue(hmi_server *v)
{
    NvtxRange range("hmi server round: issue");
    if (!v->flights.empty() && setup_pending(v)) drain_rounds(v);
    // Setup (creating, retiring streams, re-making the plan) is applied only
    // with no round in flight: a round's kernels read the plan's tables and
    // its streams' arenas until it is posted.  Only this thread issues rounds,
    // so `idle` holds for the whole call; setup that an admission or release
    // asks for meanwhile waits for the next idle round (the check above drains
    // for it).
    const bool idle = v->flights.empty();
    std::vector<SrvTake> take;
    std::vector<hmi_stream *> dead;
    std::vector<int> replan_ids;
    std::vector<hmi_stream *> replan_s;
    hmi_server_round rec;
    memset(&rec, 0, sizeof(rec));
    rec.start_ns = now_ns();
    std::vector<SrvStream *> creates;
    {
        std::unique_lock<std::mutex> lk(v->mu);
        // retire released streams whose queues are empty, and streams whose
        // creation failed (their frames come back with the error)
        bool posted = false;
        for (auto it = v->streams.begin(); it != v->streams.end();) {
            SrvStream &ss = it->second;
            if (ss.failed) {
                for (const SrvFrame &f : ss.q) {
                    hmi_server_result r;
                    memset(&r, 0, sizeof(r));
                    r.stream_id = it->first;
                    r.status = HMI_ERR_NO_MEMORY;
                    r.tag = f.tag;
                    r.submit_ns = f.submit_ns;
                    r.done_ns = now_ns();
                    r.pointer = empty_pointer();
                    v->done.push_back(r);
                    if (f.owned) v->pool[f.bytes].push_back(const_cast<uint8_t *>(f.host));
                    posted = true;
                }
                ss.q.clear();
            }
            if (idle && (ss.releasing || ss.failed) && ss.q.empty() && !ss.pending) {
                if (ss.s) dead.push_back(ss.s);
                v->used -= ss.bytes;
                it = v->streams.erase(it);
                v->dirty = true;
            } else {
                if (ss.pending && idle) {
                    creates.push_back(&ss);
                    ss.pending = false;
                }
                ++it;
            }
        }
        if (posted) v->done_cv.notify_all();
    }
    rec.created = (int32_t)creates.size();
    rec.retired = (int32_t)dead.size();
    if (!creates.empty()) {
        // device state of newly admitted streams, in the order of this
        // thread's CUDA stream (all later work on them runs on it too)
        std::vector<hmi_stream *> made(creates.size());
        for (size_t k = 0; k < creates.size(); ++k)
            made[k] = create_stream_on(creates[k]->w, creates[k]->h, &creates[k]->p, v->cs);
        std::unique_lock<std::mutex> lk(v->mu);
        for (size_t k = 0; k < creates.size(); ++k) {
            creates[k]->s = made[k];
            creates[k]->failed = made[k] == nullptr;
        }
        v->dirty = true;
    }
    {
        std::unique_lock<std::mutex> lk(v->mu);
        if (v->dirty && idle) {
            rec.replanned = 1;
            replan_ids.clear();
            for (auto &kv : v->streams) {
                if (!kv.second.s) continue;
                replan_ids.push_back(kv.first);
                replan_s.push_back(kv.second.s);
            }
            v->dirty = false;
        }
    }
    if (rec.replanned) {
        // Re-made in place with the lock released (no tick is in flight
        // between rounds, and only this thread erases streams), so that
        // admissions and submissions are not held up by it.
        v->plan_ids = replan_ids;
        if (!replan_s.empty()) {
            if (!v->plan)
                v->plan = batch_new(replan_s.data(), (int)replan_s.size(), 1);
            else if (batch_replan(v->plan, replan_s.data(), (int)replan_s.size(), 1) != HMI_OK) {
                batch_free(v->plan);
                v->plan = nullptr;
            }
        }
    }
    for (auto *d : dead) hmi_destroy_stream(d);   // no plan refers to them now
    {
        std::unique_lock<std::mutex> lk(v->mu);
        take.resize(v->plan_ids.size());
        bool any = false;
        for (size_t i = 0; i < v->plan_ids.size(); ++i) {
            auto it = v->streams.find(v->plan_ids[i]);
            if (it == v->streams.end()) continue;   // cannot happen: only this thread erases
            SrvStream &st = it->second;
            take[i].ss = &st;   // map nodes stay put
            if (!st.q.empty()) {
                take[i].f = st.q.front();
                st.q.pop_front();
                any = true;
            }
        }
        rec.setup_ns = now_ns();
        if (!any) {
            if (rec.replanned || rec.created || rec.retired) {
                rec.issued_ns = rec.done_ns = rec.setup_ns;
                rec.streams = (int32_t)v->plan_ids.size();
                log_round(v, rec);
            }
            return rec.replanned != 0;
        }
    }
    hmi_batch *b = v->plan;
    const int n = b ? b->n : 0;
    int status = b ? HMI_OK : HMI_ERR_NO_MEMORY;
    if (status == HMI_OK && (v->ptr_cap < n || v->item_cap < n)) drain_rounds(v);   // buffers in use
    // per-round buffers grow geometrically (streams join a few at a time, and
    // every allocation may wait for the device)
    const int cap = std::max(n, std::max(256, 2 * std::max(v->ptr_cap, v->item_cap)));
    if (status == HMI_OK && v->ptr_cap < n) {
        bool ok = true;
        for (int k = 0; k < 2; ++k) {
            cudaFreeHost(v->h_ptrs[k]);
            cudaFree(v->d_ptrs[k]);
            v->h_ptrs[k] = nullptr;
            v->d_ptrs[k] = nullptr;
            ok = ok && cudaMallocHost(&v->h_ptrs[k], sizeof(hmi_pointer) * cap) == cudaSuccess &&
                 cudaMalloc(&v->d_ptrs[k], sizeof(hmi_pointer) * cap) == cudaSuccess;
        }
        v->ptr_cap = ok ? cap : 0;
        if (!ok) status = HMI_ERR_NO_MEMORY;
    }
    const int buf = v->next_buf;
    // All of the round's host-to-device copies go first, back to back on the
    // copy engine: a learning frame densely into its stream's frame buffer, a
    // frame to process at the buffer's pitch.  Then the learning kernels (the
    // band is formed after a stream's last learning frame), then one tick over
    // the plan, in which learning streams are inactive (null frame).
    bool any_active = false;
    for (int i = 0; i < n && status == HMI_OK; ++i) {
        const SrvFrame &f = take[i].f;
        if (!f.host) continue;
        SrvStream *ss = take[i].ss;
        hmi_stream *s = ss->s;
        take[i].learning = ss->learn_done < ss->learn_n;
        any_active = any_active || !take[i].learning;
        take[i].src = nullptr;
        // a pinned frame needs no copy: the luma pass reads a frame to process
        // (16-pixel rows, 16-byte aligned), the batched learning kernel a
        // learning frame (pixels a multiple of 4, 4-byte aligned)
        const bool rows16 = (s->w % 16) == 0, quads = ((size_t)s->w * s->h) % 4 == 0;
        if (take[i].learning ? quads : rows16) {
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, f.host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                at.devicePointer != nullptr &&
                (reinterpret_cast<uintptr_t>(at.devicePointer) & (take[i].learning ? 3u : 15u)) == 0) {
                take[i].src = static_cast<const uint8_t *>(at.devicePointer);
                continue;
            }
            (void)cudaGetLastError();
        }
        cudaError_t e;
        if (take[i].learning || 3 * (size_t)s->w == (size_t)s->L.fpitch)
            e = cudaMemcpyAsync(s->d_frame, f.host, f.bytes, cudaMemcpyHostToDevice, v->cs);
        else
            e = cudaMemcpy2DAsync(s->d_frame, s->L.fpitch, f.host, 3 * (size_t)s->w, 3 * (size_t)s->w, s->h,
                                  cudaMemcpyHostToDevice, v->cs);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            status = HMI_ERR_DEVICE;
        }
    }
    // learning frames: their sums in one launch for the whole round (a burst
    // of new streams learns at once), except frames the batch cannot take
    if (status == HMI_OK && v->item_cap < n) {
        cudaFreeHost(v->h_items[0]);
        cudaFreeHost(v->h_items[1]);
        cudaFree(v->d_items);
        v->h_items[0] = v->h_items[1] = nullptr;
        v->d_items = nullptr;
        v->item_cap = 0;
        if (cudaMallocHost(&v->h_items[0], sizeof(LearnItem) * cap) == cudaSuccess &&
            cudaMallocHost(&v->h_items[1], sizeof(LearnItem) * cap) == cudaSuccess &&
            cudaMalloc(&v->d_items, sizeof(LearnItem) * cap) == cudaSuccess)
            v->item_cap = cap;
        else
            status = HMI_ERR_NO_MEMORY;
    }
    int nitems = 0;
    unsigned long long quads = 0;
    for (int i = 0; i < n && status == HMI_OK; ++i) {
        if (!take[i].f.host || !take[i].learning) continue;
        SrvStream *ss = take[i].ss;
        hmi_stream *s = ss->s;
        const uint8_t *fr = take[i].src ? take[i].src : s->d_frame;
        const long long npx = (long long)s->w * s->h;
        cudaError_t e = cudaSuccess;
        if (ss->learn_done == 0)
            e = cudaMemsetAsync(&s->st->learn_luma, 0, sizeof(unsigned long long), v->cs);
        if (e == cudaSuccess && npx % 4 == 0 && (reinterpret_cast<uintptr_t>(fr) & 3u) == 0) {
            v->h_items[buf][nitems++] = LearnItem{fr, s->d_S, s->d_Q, s->d_vmin, s->d_vmax, s->st, quads,
                                                  ss->learn_done == 0};
            quads += (unsigned long long)(npx / 4);
        } else if (e == cudaSuccess) {
            e = launch_learn_accum(fr, 1, npx, s->d_S, s->d_Q, s->d_vmin, s->d_vmax, ss->learn_done == 0,
                                   s->st, v->cs);
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            status = HMI_ERR_DEVICE;
        }
    }
    if (status == HMI_OK && nitems > 0 &&
        (cudaMemcpyAsync(v->d_items, v->h_items[buf], sizeof(LearnItem) * nitems, cudaMemcpyHostToDevice, v->cs) !=
             cudaSuccess ||
         launch_learn_batch(v->d_items, nitems, quads, v->cs) != cudaSuccess)) {
        (void)cudaGetLastError();
        status = HMI_ERR_DEVICE;
    }
    for (int i = 0; i < n && status == HMI_OK; ++i) {
        if (!take[i].f.host || !take[i].learning) continue;
        SrvStream *ss = take[i].ss;
        hmi_stream *s = ss->s;
        const uint8_t *fr = take[i].src ? take[i].src : s->d_frame;
        cudaError_t e = cudaSuccess;
        if (s->L.mix_k) {   // the mixture learns the same frame
            if (ss->learn_done == 0) e = enqueue_mix_reset(s, v->cs);
            if (e == cudaSuccess)
                e = launch_mix_learn(fr, 1, (uint32_t)ss->learn_done, s->w, s->h, s->ds.mix, v->cs);
        }
        if (e == cudaSuccess && ss->learn_done + 1 == ss->learn_n) e = enqueue_band(s, ss->learn_n, v->cs);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            status = HMI_ERR_DEVICE;
            break;
        }
        if (++ss->learn_done == ss->learn_n) {
            s->learned = 1;
            s->n_learn = ss->learn_n;
        }
        rec.learning += 1;
    }
    if (status == HMI_OK && any_active) {
        const int slot = acquire_slot(b);
        TickIO *io = b->h_io + (size_t)slot * n;
        for (int i = 0; i < n; ++i) {
            hmi_stream *s = b->s[i];
            TickIO &t = io[b->pos[i]];
            t.mask = nullptr;
            t.ptr_out = v->d_ptrs[buf] + i;
            t.src = nullptr;
            if (take[i].f.host && !take[i].learning) {
                s->used = true;
                t.frame = s->d_frame;
                t.frame_pitch = s->L.fpitch;
                if (take[i].src) {
                    t.src = take[i].src;
                    t.frame = s->arena + s->L.frame_ph[slot % kPhases];
                }
            } else {
                t.frame = nullptr;
                t.frame_pitch = 0;
            }
        }
        status = run_tick(b, slot, v->cs, false);
        if (status == HMI_OK &&
            (cudaMemcpyAsync(v->h_ptrs[buf], v->d_ptrs[buf], sizeof(hmi_pointer) * n, cudaMemcpyDeviceToHost, v->cs) != cudaSuccess ||
             cudaMemcpyAsync(v->h_err[buf], b->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, v->cs) != cudaSuccess ||
             cudaMemsetAsync(b->d_err, 0, sizeof(uint32_t), v->cs) != cudaSuccess)) {
            (void)cudaGetLastError();
            status = HMI_ERR_DEVICE;
        }
    }
    // whatever was enqueued has finished with the round's host frames (read
    // by copies or by the luma pass) when the event has completed; they are
    // given back when the round is posted
    if (cudaEventRecord(v->ev[buf], v->cs) != cudaSuccess) {
        (void)cudaGetLastError();
        status = HMI_ERR_DEVICE;
    }
    rec.issued_ns = now_ns();
    rec.streams = n;
    hmi_server::Flight F;
    F.take = std::move(take);
    F.ids = v->plan_ids;
    F.rec = rec;
    F.any_active = any_active;
    F.status = status;
    F.buf = buf;
    v->flights.push_back(std::move(F));
    v->next_buf ^= 1;
    return true;
}

// Post the oldest round in flight: wait for its device work, then hand its
// results (and its pooled host frames) back.
void complete_round(hmi_server *v)
{
    NvtxRange range("hmi server round: post");
    hmi_server::Flight F = std::move(v->flights.front());
    v->flights.pop_front();
    int status = F.status;
    if (cudaEventSynchronize(v->ev[F.buf]) != cudaSuccess) {
        (void)cudaGetLastError();
        status = HMI_ERR_DEVICE;
    }
    if (status == HMI_OK && F.any_active && *v->h_err[F.buf])
        status = (*v->h_err[F.buf] & kErrBounds) ? HMI_ERR_DEVICE : HMI_ERR_DEVICE_TIMEOUT;
    *v->h_err[F.buf] = 0;
    const uint64_t t_done = now_ns();
    hmi_server_round &rec = F.rec;
    rec.done_ns = t_done;
    std::unique_lock<std::mutex> lk(v->mu);
    v->ticks += 1;
    for (int i = 0; i < (int)F.take.size(); ++i) {
        const SrvFrame &f = F.take[i].f;
        if (!f.host) continue;
        hmi_server_result r;
        memset(&r, 0, sizeof(r));
        r.stream_id = F.ids[i];
        r.status = status;
        r.tag = f.tag;
        r.submit_ns = f.submit_ns;
        r.done_ns = t_done;
        if (status == HMI_OK && F.take[i].learning) {
            r.status = HMI_LEARNING;
            r.pointer = empty_pointer();
        } else if (status == HMI_OK) {
            r.pointer = v->h_ptrs[F.buf][i];
        }
        v->done.push_back(r);
        if (f.owned) v->pool[f.bytes].push_back(const_cast<uint8_t *>(f.host));
        v->frames += 1;
        if (!F.take[i].learning) rec.frames += 1;
    }
    log_round(v, rec);
    lk.unlock();
    v->done_cv.notify_all();
}


void server_loop(hmi_server *v)
{
    cudaSetDevice(v->dev);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(v->mu);
            if (v->stop) break;
        }
        // post the rounds whose device work has finished
        while (!v->flights.empty() && cudaEventQuery(v->ev[v->flights.front().buf]) == cudaSuccess)
            complete_round(v);
        (void)cudaGetLastError();   // a query of unfinished work reports cudaErrorNotReady
        const bool issued = v->flights.size() < 2 && server_issue(v);
        if (issued) continue;
        if (!v->flights.empty()) {
            complete_round(v);   // nothing new to issue: wait for the device
            continue;
        }
        std::unique_lock<std::mutex> lk(v->mu);
        if (v->stop) break;
        v->work_cv.wait_for(lk, std::chrono::microseconds(500));
    }
    drain_rounds(v);
}

}  // namespace

extern "C" {

uint64_t hmi_server_now_ns(void) { return now_ns(); }

hmi_server *hmi_server_create(size_t device_budget_bytes, int max_queue)
{
    if (max_queue < 1 || max_queue > 64) {
        fail(HMI_ERR_INVALID_ARG);
        return nullptr;
    }
    hmi_server *v = new (std::nothrow) hmi_server();
    if (!v) {
        fail(HMI_ERR_NO_MEMORY);
        return nullptr;
    }
    v->budget = device_budget_bytes;
    v->max_queue = max_queue;
    bool ok = cudaGetDevice(&v->dev) == cudaSuccess &&
              cudaStreamCreateWithFlags(&v->cs, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; ok && k < 2; ++k)
        ok = cudaEventCreateWithFlags(&v->ev[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaMallocHost(&v->h_err[k], sizeof(uint32_t)) == cudaSuccess;
    if (!ok) {
        (void)cudaGetLastError();
        for (int k = 0; k < 2; ++k) {
            if (v->ev[k]) cudaEventDestroy(v->ev[k]);
            if (v->h_err[k]) cudaFreeHost(v->h_err[k]);
        }
        if (v->cs) cudaStreamDestroy(v->cs);
        delete v;
        fail(HMI_ERR_DEVICE);
        return nullptr;
    }
    *v->h_err[0] = *v->h_err[1] = 0;
    // Map the stream-arena pool up to the budget (at most a quarter of the free
    // device memory) now, so that admitting a burst of streams later only
    // sub-allocates; the pool keeps freed memory while any stream lives.
    size_t free_b = 0, total_b = 0;
    cudaMemPool_t pool = arena_pool(v->dev);
    if (pool && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const size_t want = std::min(device_budget_bytes, free_b / 4);
        void *p = nullptr;
        if (want > 0 && cudaMallocFromPoolAsync(&p, want, pool, v->cs) == cudaSuccess) {
            cudaFreeAsync(p, v->cs);
            cudaStreamSynchronize(v->cs);
        }
    }
    (void)cudaGetLastError();
    v->worker = std::thread(server_loop, v);
    return v;
}

void hmi_server_destroy(hmi_server *v)
{
    if (!v) return;
    {
        std::lock_guard<std::mutex> lk(v->mu);
        v->stop = true;
    }
    v->work_cv.notify_all();
    if (v->worker.joinable()) v->worker.join();
    cudaSetDevice(v->dev);
    batch_free(v->plan);
    for (auto &kv : v->streams) {
        for (auto &f : kv.second.q)
            if (f.owned) cudaFreeHost(const_cast<uint8_t *>(f.host));
        hmi_destroy_stream(kv.second.s);
    }
    for (auto &kv : v->pool)
        for (auto *p : kv.second) cudaFreeHost(p);
    for (int k = 0; k < 2; ++k) {
        cudaFreeHost(v->h_ptrs[k]);
        cudaFree(v->d_ptrs[k]);
        cudaFreeHost(v->h_items[k]);
        cudaFreeHost(v->h_err[k]);
        if (v->ev[k]) cudaEventDestroy(v->ev[k]);
    }
    cudaFree(v->d_items);
    if (v->cs) cudaStreamDestroy(v->cs);
    delete v;
}

int hmi_server_admit(hmi_server *v, int w, int h, const hmi_params *p, const uint8_t *learn_frames,
                     int n, int *stream_id)
{
    if (!v || !stream_id || n < 1 || n > 65535) return fail(HMI_ERR_INVALID_ARG);
    const size_t bytes = hmi_stream_device_bytes(w, h, p);
    if (bytes == 0) return fail(HMI_ERR_INVALID_ARG);
    {
        std::lock_guard<std::mutex> lk(v->mu);
        if (v->used + bytes > v->budget) return fail(HMI_ERR_NO_MEMORY);
        v->used += bytes;   // reserved while the stream is set up
    }
    if (!learn_frames) {
        // online learning: a reservation only; the dispatcher creates the
        // stream at its next round, and frames may be queued meanwhile
        std::lock_guard<std::mutex> lk(v->mu);
        const int id = v->next_id++;
        SrvStream &ss = v->streams[id];
        ss.w = w;
        ss.h = h;
        if (p) ss.p = *p;
        else hmi_default_params(&ss.p);
        ss.bytes = bytes;
        ss.pending = true;
        ss.learn_n = n;
        *stream_id = id;
        v->work_cv.notify_all();
        return HMI_OK;
    }
    HMI_CUDA(cudaSetDevice(v->dev));
    hmi_stream *s = hmi_create_stream(w, h, p);
    int st = s ? HMI_OK : g_last_error;
    if (s) st = learn_background(s, learn_frames, n);
    if (st != HMI_OK) {
        if (s) hmi_destroy_stream(s);
        std::lock_guard<std::mutex> lk(v->mu);
        v->used -= bytes;
        return fail(st);
    }
    std::lock_guard<std::mutex> lk(v->mu);
    const int id = v->next_id++;
    SrvStream &ss = v->streams[id];
    ss.s = s;
    ss.w = w;
    ss.h = h;
    ss.p = s->p;
    ss.bytes = bytes;
    v->dirty = true;
    *stream_id = id;
    return HMI_OK;
}

int hmi_server_release(hmi_server *v, int stream_id)
{
    if (!v) return fail(HMI_ERR_INVALID_ARG);
    std::lock_guard<std::mutex> lk(v->mu);
    auto it = v->streams.find(stream_id);
    if (it == v->streams.end() || it->second.releasing) return fail(HMI_ERR_INVALID_ARG);
    it->second.releasing = true;
    v->work_cv.notify_all();
    return HMI_OK;
}

static int server_enqueue(hmi_server *v, int stream_id, const uint8_t *frame, uint64_t tag, bool copy)
{
    if (!v || !frame) return fail(HMI_ERR_INVALID_ARG);
    size_t bytes;
    {
        std::lock_guard<std::mutex> lk(v->mu);
        auto it = v->streams.find(stream_id);
        if (it == v->streams.end() || it->second.releasing) return fail(HMI_ERR_INVALID_ARG);
        if ((int)it->second.q.size() >= v->max_queue) return fail(HMI_ERR_NO_MEMORY);
        bytes = 3 * (size_t)it->second.w * it->second.h;
    }
    SrvFrame f;
    f.bytes = bytes;
    f.tag = tag;
    f.submit_ns = now_ns();
    f.owned = copy;
    if (copy) {
        uint8_t *buf;
        {
            std::lock_guard<std::mutex> lk(v->mu);
            buf = pool_get(v, bytes);
        }
        if (!buf) return fail(HMI_ERR_NO_MEMORY);
        memcpy(buf, frame, bytes);
        f.host = buf;
    } else {
        f.host = frame;
    }
    {
        std::lock_guard<std::mutex> lk(v->mu);
        auto it = v->streams.find(stream_id);
        if (it == v->streams.end() || it->second.releasing) {
            if (copy) v->pool[bytes].push_back(const_cast<uint8_t *>(f.host));
            return fail(HMI_ERR_INVALID_ARG);
        }
        it->second.q.push_back(f);
    }
    v->work_cv.notify_all();
    return HMI_OK;
}

int hmi_server_submit(hmi_server *v, int stream_id, const uint8_t *frame, uint64_t tag)
{
    return server_enqueue(v, stream_id, frame, tag, true);
}

int hmi_server_submit_ref(hmi_server *v, int stream_id, const uint8_t *frame, uint64_t tag)
{
    return server_enqueue(v, stream_id, frame, tag, false);
}

int hmi_server_poll(hmi_server *v, hmi_server_result *out, int max_results, int wait_us)
{
    if (!v || !out || max_results < 1) return fail(HMI_ERR_INVALID_ARG);
    std::unique_lock<std::mutex> lk(v->mu);
    if (v->done.empty() && wait_us > 0)
        v->done_cv.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !v->done.empty(); });
    int k = 0;
    while (k < max_results && !v->done.empty()) {
        out[k++] = v->done.front();
        v->done.pop_front();
    }
    return k;
}

int hmi_server_rounds(hmi_server *v, hmi_server_round *out, int max_rounds)
{
    if (!v || !out || max_rounds < 1) return fail(HMI_ERR_INVALID_ARG);
    std::lock_guard<std::mutex> lk(v->mu);
    const uint64_t have = std::min<uint64_t>(v->rounds_written, v->rounds.size());
    const uint64_t k = std::min<uint64_t>(have, (uint64_t)max_rounds);
    for (uint64_t i = 0; i < k; ++i) {
        const uint64_t r = v->rounds_written - k + i;   // oldest of the last k first
        out[i] = v->rounds[r % kRoundLog];
    }
    return (int)k;
}

int hmi_server_stats(hmi_server *v, size_t *bytes_admitted, uint64_t *ticks, uint64_t *frames)
{
    if (!v) return fail(HMI_ERR_INVALID_ARG);
    std::lock_guard<std::mutex> lk(v->mu);
    if (bytes_admitted) *bytes_admitted = v->used;
    if (ticks) *ticks = v->ticks;
    if (frames) *frames = v->frames;
    return HMI_OK;
}

}  // extern "C"

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int hmi_last_error(void) { return g_last_error; }

const char *hmi_status_string(int status)
{
    switch (status) {
    case HMI_OK: return "ok";
    case HMI_ERR_INVALID_ARG: return "invalid argument";
    case HMI_ERR_NOT_LEARNED: return "background not learned";
    case HMI_ERR_NO_MEMORY: return "out of memory or admission refused";
    case HMI_ERR_DEVICE: return "CUDA error";
    case HMI_ERR_DEVICE_TIMEOUT: return "device-side bounded wait or loop gave up";
    default: return "unknown status";
    }
}

int hmi_default_params(hmi_params *p)
{
    if (!p) return fail(HMI_ERR_INVALID_ARG);
    memset(p, 0, sizeof(*p));
    p->gain_min_q16 = 32768;
    p->gain_max_q16 = 131072;
    p->min_area = 50;
    p->hue_lo = 1472;
    p->hue_hi = 256;
    p->click_window = 30;
    p->gray_tol = 15;
    p->bg_margin = 2;
    p->bg_k_num = 5;
    p->bg_k_den = 2;
    p->open_iters = 1;
    p->close_iters = 1;
    p->click_on_pct = 80;
    p->click_off_pct = 90;
    p->mix_k = 3;
    p->mix_bg_pct = 70;
    p->mix_sigma0 = 15;
    p->mix_sigma_min = 2;
    p->mix_rate_n = 256;
    return HMI_OK;
}

size_t hmi_stream_device_bytes(int w, int h, const hmi_params *p)
{
    hmi_params d;
    hmi_default_params(&d);
    const hmi_params &pp = p ? *p : d;
    if (w < 1 || h < 1 || w > kMaxDim || h > kMaxDim || !params_valid(pp)) return 0;
    return make_layout(w, h, pp).total;
}

hmi_stream *hmi_create_stream(int w, int h, const hmi_params *p)
{
    return create_stream_on(w, h, p, nullptr);
}

void hmi_destroy_stream(hmi_stream *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        if (g_cache && std::find(g_cache->s.begin(), g_cache->s.end(), s) != g_cache->s.end()) {
            batch_free(g_cache);
            g_cache = nullptr;
        }
    }
    cudaSetDevice(s->dev);
    batch_free(s->self);
    cudaDeviceSynchronize();   // no work of any stream may still use the state
    release_arena(s);
    delete s;
}

int hmi_learn_background(hmi_stream *s, const uint8_t *frames, int n)
{
    const int st = learn_background(s, frames, n);
    // the single-frame launch plan is made now rather than by the first
    // hmi_process_frame (best effort: that call makes it otherwise)
    if (st == HMI_OK && !self_plan(s)) (void)cudaGetLastError();
    return st;
}

int learn_background(hmi_stream *s, const uint8_t *frames, int n)
{
    NvtxRange range("hmi learn background");
    if (!s || !frames || n < 1 || n > 65535) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(s->dev));
    const long long npx = (long long)s->w * s->h;
    const size_t fbytes = (size_t)npx * 3;
    if (s->used) HMI_CUDA(cudaDeviceSynchronize());   // no tick of this stream may be in flight
    // reset the learning luma total
    HMI_CUDA(cudaMemsetAsync(&s->st->learn_luma, 0, sizeof(unsigned long long), s->cs));
    HMI_CUDA(enqueue_mix_reset(s, s->cs));
    if (is_device_ptr(frames)) {
        HMI_CUDA(launch_learn_accum(frames, n, npx, s->d_S, s->d_Q, s->d_vmin, s->d_vmax, 1, s->st, s->cs));
        if (s->L.mix_k) HMI_CUDA(launch_mix_learn(frames, n, 0u, s->w, s->h, s->ds.mix, s->cs));
    } else {
        // host frames: stream through a bounded staging buffer
        const int per = (int)std::max<size_t>(1, std::min<size_t>((size_t)n, (256u << 20) / fbytes));
        uint8_t *stage = nullptr;   // stream-ordered: no device-wide synchronisation
        if (cudaMallocAsync(reinterpret_cast<void **>(&stage), fbytes * per, s->cs) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(HMI_ERR_NO_MEMORY);
        }
        int status = HMI_OK;
        for (int i = 0; i < n && status == HMI_OK; i += per) {
            const int k = std::min(per, n - i);
            if (cudaMemcpyAsync(stage, frames + (size_t)i * fbytes, fbytes * k, cudaMemcpyHostToDevice, s->cs) != cudaSuccess ||
                launch_learn_accum(stage, k, npx, s->d_S, s->d_Q, s->d_vmin, s->d_vmax, i == 0, s->st, s->cs) != cudaSuccess ||
                (s->L.mix_k && launch_mix_learn(stage, k, (uint32_t)i, s->w, s->h, s->ds.mix, s->cs) != cudaSuccess) ||
                cudaStreamSynchronize(s->cs) != cudaSuccess)
                status = cuda_fail(cudaErrorUnknown);
        }
        cudaFreeAsync(stage, s->cs);
        if (status != HMI_OK) return status;
    }
    HMI_CUDA(enqueue_band(s, n, s->cs));
    HMI_CUDA(cudaStreamSynchronize(s->cs));
    s->learned = 1;
    s->n_learn = n;
    return HMI_OK;
}

int hmi_process_frame(hmi_stream *s, const uint8_t *frame, uint8_t *mask_out, hmi_pointer *pointer_out)
{
    if (!s || !frame) return fail(HMI_ERR_INVALID_ARG);
    uint8_t *const masks[1] = {mask_out};
    if (!self_plan(s)) return g_last_error;
    return batch_sync(s->self, &frame, masks, pointer_out);
}

int hmi_process_frame_async(hmi_stream *s, const uint8_t *frame, uint8_t *mask_out,
                            hmi_pointer *pointer_out, void *cuda_stream)
{
    if (!s || !frame) return fail(HMI_ERR_INVALID_ARG);
    uint8_t *const masks[1] = {mask_out};
    if (!self_plan(s)) return g_last_error;
    return batch_async(s->self, &frame, masks, pointer_out, cuda_stream, 0);
}

hmi_batch *hmi_batch_create(hmi_stream *const *s, int n)
{
    return streams_ok(s, n) ? batch_new(s, n, default_groups(s, n, kDefaultTuning)) : batch_new(s, n, 1);
}

int hmi_batch_set_groups(hmi_batch *b, int groups) { return batch_set_groups(b, groups); }

int hmi_batch_set_loop_limit(hmi_batch *b, uint32_t limit)
{
    if (!b) return fail(HMI_ERR_INVALID_ARG);
    b->loop_limit = limit;
    return batch_retune(b, b->tune);
}

int hmi_batch_get_groups(const hmi_batch *b)
{
    if (!b) return fail(HMI_ERR_INVALID_ARG);
    return (int)b->groups.size();
}

int hmi_batch_set_tuning(hmi_batch *b, const hmi_tuning *t)
{
    if (!b || !t) return fail(HMI_ERR_INVALID_ARG);
    return batch_retune(b, *t);
}

int hmi_batch_get_tuning(const hmi_batch *b, hmi_tuning *t)
{
    if (!b || !t) return fail(HMI_ERR_INVALID_ARG);
    *t = b->tune;
    if (t->groups == 0) t->groups = (int32_t)b->groups.size();
    return HMI_OK;
}

int hmi_batch_autotune(hmi_batch *b, const uint8_t *const *frames, int ticks, int pipelined,
                       hmi_tuning *best, double *best_tick_us)
{
    return batch_autotune(b, frames, ticks, pipelined != 0, best, best_tick_us);
}

void hmi_batch_destroy(hmi_batch *b) { batch_free(b); }

int hmi_batch_process(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
                      hmi_pointer *ptrs)
{
    return batch_sync(b, frames, masks, ptrs);
}

int hmi_batch_process_async(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
                            hmi_pointer *ptrs, void *cuda_stream, int use_graph)
{
    return batch_async(b, frames, masks, ptrs, cuda_stream, use_graph);
}

int hmi_batch_process_pipelined(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
                                hmi_pointer *ptrs, void *cuda_stream, int use_graph)
{
    return batch_pipelined(b, frames, masks, ptrs, cuda_stream, use_graph);
}

int hmi_batch_flush(hmi_batch *b, void *cuda_stream)
{
    if (!b) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(b->dev));
    return flush_pending(b, reinterpret_cast<cudaStream_t>(cuda_stream));
}

int hmi_process_batch(hmi_stream *const *s, int n, const uint8_t *const *frames,
                      uint8_t *const *masks, hmi_pointer *ptrs)
{
    if (!s || n < 1 || n > kMaxBatch || !frames) return fail(HMI_ERR_INVALID_ARG);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (!g_cache || g_cache->n != n || !std::equal(g_cache->s.begin(), g_cache->s.end(), s)) {
        batch_free(g_cache);
        g_cache = batch_new(s, n, streams_ok(s, n) ? default_groups(s, n, kDefaultTuning) : 1);
        if (!g_cache) return g_last_error;
    }
    return batch_sync(g_cache, frames, masks, ptrs);
}

int hmi_batch_profile(hmi_batch *b, int max_ticks)
{
    if (!b || max_ticks < 0 || max_ticks > 1000000) return fail(HMI_ERR_INVALID_ARG);
    if (max_ticks > 0 && b->groups.size() != 1) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(b->dev));
    const int fs = flush_pending(b, b->cs);
    if (fs != HMI_OK) return fs;
    HMI_CUDA(cudaDeviceSynchronize());
    for (auto e : b->prof_ev) cudaEventDestroy(e);
    b->prof_ev.assign((size_t)(kTickKernels + 1) * max_ticks, nullptr);
    for (auto &e : b->prof_ev) HMI_CUDA(cudaEventCreate(&e));
    b->prof_max = max_ticks;
    b->prof_used = 0;
    return HMI_OK;
}

int hmi_batch_profile_kernels(hmi_batch *b, int *ticks, double *ms, int n_kernels)
{
    if (!b || !ticks || !ms || n_kernels < 1 || n_kernels > HMI_TICK_KERNELS) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(b->dev));
    for (int k = 0; k < n_kernels; ++k) ms[k] = 0.0;
    for (int i = 0; i < b->prof_used; ++i) {
        const cudaEvent_t *ev = b->prof_ev.data() + (size_t)(kTickKernels + 1) * i;
        HMI_CUDA(cudaEventSynchronize(ev[kTickKernels]));
        for (int k = 0; k < n_kernels; ++k) {
            float t = 0.f;
            HMI_CUDA(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
            ms[k] += t;
        }
    }
    *ticks = b->prof_used;
    return HMI_OK;
}

int hmi_batch_profile_read(hmi_batch *b, int *ticks, double *total_ms)
{
    if (!b || !ticks || !total_ms) return fail(HMI_ERR_INVALID_ARG);
    double ms[HMI_TICK_KERNELS];
    const int st = hmi_batch_profile_kernels(b, ticks, ms, HMI_TICK_KERNELS);
    if (st != HMI_OK) return st;
    *total_ms = b->groups[0].bd.fused ? ms[0] : ms[1];   // the per-pixel HBM pass
    return HMI_OK;
}

int hmi_get_background_stats(const hmi_stream *s, float *mean, float *std)
{
    if (!s) return fail(HMI_ERR_INVALID_ARG);
    if (!s->learned) return fail(HMI_ERR_NOT_LEARNED);
    if (!mean && !std) return HMI_OK;
    HMI_CUDA(cudaSetDevice(s->dev));
    const long long count = (long long)s->w * s->h * 3;
    const size_t bytes = (size_t)count * sizeof(float);
    float *dm = nullptr, *dd = nullptr;
    const bool mdev = mean && is_device_ptr(mean), sdev = std && is_device_ptr(std);
    if (mean && !mdev && cudaMalloc(&dm, bytes) != cudaSuccess) return fail(HMI_ERR_NO_MEMORY);
    if (std && !sdev && cudaMalloc(&dd, bytes) != cudaSuccess) {
        cudaFree(dm);
        return fail(HMI_ERR_NO_MEMORY);
    }
    cudaError_t e = launch_stats(s->d_S, s->d_Q, s->n_learn, count, mean ? (mdev ? mean : dm) : nullptr,
                                 std ? (sdev ? std : dd) : nullptr, s->cs);
    if (e == cudaSuccess && dm) e = cudaMemcpyAsync(mean, dm, bytes, cudaMemcpyDeviceToHost, s->cs);
    if (e == cudaSuccess && dd) e = cudaMemcpyAsync(std, dd, bytes, cudaMemcpyDeviceToHost, s->cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cs);
    cudaFree(dm);
    cudaFree(dd);
    if (e != cudaSuccess) return cuda_fail(e);
    return HMI_OK;
}

int hmi_get_labels(const hmi_stream *s, int32_t *labels)
{
    if (!s || !labels) return fail(HMI_ERR_INVALID_ARG);
    if (!s->learned) return fail(HMI_ERR_NOT_LEARNED);
    HMI_CUDA(cudaSetDevice(s->dev));
    HMI_CUDA(cudaDeviceSynchronize());   // the last tick may have run on any stream
    const size_t bytes = (size_t)s->w * s->h * sizeof(int32_t);
    const bool dev = is_device_ptr(labels);
    int32_t *d = labels;
    if (!dev && cudaMalloc(&d, bytes) != cudaSuccess) return fail(HMI_ERR_NO_MEMORY);
    cudaError_t e = launch_labels(s->d_ds, s->ds, d, s->cs);
    if (e == cudaSuccess && !dev) e = cudaMemcpyAsync(labels, d, bytes, cudaMemcpyDeviceToHost, s->cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->cs);
    if (!dev) cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e);
    return HMI_OK;
}

int hmi_set_interface(hmi_stream *s, const hmi_interface *ui)
{
    if (!s || !ui || ui->nzones < 0 || ui->nzones > HMI_MAX_ZONES || ui->wheel_r_in < 0 ||
        ui->wheel_r_in > ui->wheel_r_out || ui->wheel_r_out > 65535 || ui->dead_zone < 0 ||
        ui->dead_zone > 2048)
        return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(s->dev));
    HMI_CUDA(cudaDeviceSynchronize());   // no tick of the stream may be reading it
    HMI_CUDA(cudaMemcpy(s->arena + s->L.ui, ui, sizeof(hmi_interface), cudaMemcpyHostToDevice));
    return HMI_OK;
}

int hmi_get_event(const hmi_stream *s, hmi_event *out)
{
    if (!s || !out) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(s->dev));
    HMI_CUDA(cudaDeviceSynchronize());   // the last tick may have run on any stream
    HMI_CUDA(cudaMemcpy(out, &s->st->event, sizeof(hmi_event), cudaMemcpyDefault));
    return HMI_OK;
}

int hmi_get_band(const hmi_stream *s, uint8_t *lo, uint8_t *hi)
{
    if (!s || !lo || !hi) return fail(HMI_ERR_INVALID_ARG);
    if (!s->learned) return fail(HMI_ERR_NOT_LEARNED);
    HMI_CUDA(cudaSetDevice(s->dev));
    HMI_CUDA(cudaDeviceSynchronize());   // the last tick may have run on any stream
    const size_t row = 3 * (size_t)s->w;
    HMI_CUDA(cudaMemcpy2D(lo, row, s->arena + s->L.lo, s->L.fpitch, row, s->h, cudaMemcpyDefault));
    HMI_CUDA(cudaMemcpy2D(hi, row, s->arena + s->L.hi, s->L.fpitch, row, s->h, cudaMemcpyDefault));
    return HMI_OK;
}

int hmi_get_mixture(const hmi_stream *s, uint16_t *out)
{
    if (!s || !out || !s->L.mix_k) return fail(HMI_ERR_INVALID_ARG);
    if (!s->learned) return fail(HMI_ERR_NOT_LEARNED);
    HMI_CUDA(cudaSetDevice(s->dev));
    HMI_CUDA(cudaDeviceSynchronize());   // the last tick may have run on any stream
    const int F = 6 * s->L.mix_k;
    std::vector<uint16_t> tiles(s->L.mbytes / 2), dense((size_t)F * s->w * s->h);
    HMI_CUDA(cudaMemcpy(tiles.data(), s->arena + s->L.mix, s->L.mbytes, cudaMemcpyDeviceToHost));
    const size_t plane = (size_t)s->w * s->h;
    for (int y = 0; y < s->h; ++y)
        for (int x = 0; x < s->w; ++x) {
            const size_t t = mix_tile(s->ds.mix, x, y) + (x & 31);
            for (int f = 0; f < F; ++f) dense[f * plane + (size_t)y * s->w + x] = tiles[t + 32 * f];
        }
    HMI_CUDA(cudaMemcpy(out, dense.data(), dense.size() * 2, cudaMemcpyDefault));
    return HMI_OK;
}

int hmi_export_background(const hmi_stream *s, uint32_t *S, uint32_t *Q, uint8_t *vmin,
                          uint8_t *vmax, uint8_t *lo, uint8_t *hi, uint64_t *syref, int *n)
{
    if (!s) return fail(HMI_ERR_INVALID_ARG);
    if (!s->learned) return fail(HMI_ERR_NOT_LEARNED);
    HMI_CUDA(cudaSetDevice(s->dev));
    HMI_CUDA(cudaDeviceSynchronize());
    const size_t cnt = (size_t)s->w * s->h * 3;
    if (S) HMI_CUDA(cudaMemcpy(S, s->d_S, cnt * 4, cudaMemcpyDefault));
    if (Q) HMI_CUDA(cudaMemcpy(Q, s->d_Q, cnt * 4, cudaMemcpyDefault));
    if (vmin) HMI_CUDA(cudaMemcpy(vmin, s->d_vmin, cnt, cudaMemcpyDefault));
    if (vmax) HMI_CUDA(cudaMemcpy(vmax, s->d_vmax, cnt, cudaMemcpyDefault));
    if (lo) HMI_CUDA(cudaMemcpy2D(lo, 3 * (size_t)s->w, s->arena + s->L.lo, s->L.fpitch, 3 * (size_t)s->w, s->h, cudaMemcpyDefault));
    if (hi) HMI_CUDA(cudaMemcpy2D(hi, 3 * (size_t)s->w, s->arena + s->L.hi, s->L.fpitch, 3 * (size_t)s->w, s->h, cudaMemcpyDefault));
    if (syref) HMI_CUDA(cudaMemcpy(syref, &s->st->syref, sizeof(uint64_t), cudaMemcpyDefault));
    if (n) *n = s->n_learn;
    return HMI_OK;
}

int hmi_import_background(hmi_stream *s, const uint32_t *S, const uint32_t *Q, const uint8_t *vmin,
                          const uint8_t *vmax, int n, uint64_t syref)
{
    if (!s || !S || !Q || !vmin || !vmax || n < 1 || n > 65535) return fail(HMI_ERR_INVALID_ARG);
    if (syref > (uint64_t)255 * s->w * s->h) return fail(HMI_ERR_INVALID_ARG);
    if (s->L.mix_k) return fail(HMI_ERR_INVALID_ARG);   // a mixture is learned from frames only
    HMI_CUDA(cudaSetDevice(s->dev));
    HMI_CUDA(cudaDeviceSynchronize());
    const size_t cnt = (size_t)s->w * s->h * 3;
    HMI_CUDA(cudaMemcpy(s->d_S, S, cnt * 4, cudaMemcpyDefault));
    HMI_CUDA(cudaMemcpy(s->d_Q, Q, cnt * 4, cudaMemcpyDefault));
    HMI_CUDA(cudaMemcpy(s->d_vmin, vmin, cnt, cudaMemcpyDefault));
    HMI_CUDA(cudaMemcpy(s->d_vmax, vmax, cnt, cudaMemcpyDefault));
    const unsigned long long tot = (unsigned long long)syref * (unsigned long long)n;
    HMI_CUDA(cudaMemcpy(&s->st->learn_luma, &tot, sizeof(tot), cudaMemcpyHostToDevice));
    HMI_CUDA(enqueue_band(s, n, s->cs));
    HMI_CUDA(cudaStreamSynchronize(s->cs));
    s->learned = 1;
    s->n_learn = n;
    return HMI_OK;
}

int hmi_get_last_gain(const hmi_stream *s, uint32_t *gain_q16)
{
    if (!s || !gain_q16) return fail(HMI_ERR_INVALID_ARG);
    HMI_CUDA(cudaSetDevice(s->dev));
    HMI_CUDA(cudaDeviceSynchronize());
    HMI_CUDA(cudaMemcpy(gain_q16, &s->st->gain, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return HMI_OK;
}

}  // extern "C"
