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
// exported C functions.  The server (hmi_server_*) is in hmi_server.cu; the
// structures both files use are in hmi_host.h.
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

#include "hmi_host.h"
#include "hmi_queue.h"

using namespace hmi;

namespace {
thread_local int g_last_error = HMI_OK;
}  // namespace

int hmi::fail(int status)
{
    g_last_error = status;
    return status;
}

int hmi::cuda_fail(cudaError_t e)
{
    (void)cudaGetLastError();
    (void)e;
    return fail(HMI_ERR_DEVICE);
}

// Thread-local status of the last failed call, for the other translation units.
int hmi::set_error(int status) { return fail(status); }

namespace {


// Default launch shape (hmi_tuning): 16-px chunks per CTA piece of the
// per-pixel kernels (512 = 8192 px), luma CTAs per SM (0 = as many as fit),
// skin-test and block-component CTAs per SM, stream groups (0 = by the
// streams, see default_groups), stages of a pipelined tick, the persistent
// tick off (the chain of kernels measured faster on the 64-stream batch), its
// queue lag chosen from the grid, 512 threads per stream merge.
constexpr hmi_tuning kDefaultTuning = {512, 0, 8, 8, 0, 2, 0, 0, 0};


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

}  // namespace

cudaMemPool_t hmi::arena_pool(int dev)
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

namespace {

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

}  // namespace

void hmi::plan_free(hmi_batch *b)
{
    plan_free_graphs(b);
    for (auto &g : b->groups) group_destroy(g);
    b->groups.clear();
    if (b->plan) cudaFree(b->plan);
    b->plan = nullptr;
    b->plan_cap = 0;
}

int hmi::batch_free(hmi_batch *b)
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

namespace {

// Build the launch plan with `ng` stream groups: streams are dealt to groups
// by pixel count (largest first, to the least-loaded group); each group gets
// its own descriptor array, prefix tables, work pieces, counters and
// component list, and its own branch stream.
}  // namespace

int hmi::plan_build(hmi_batch *b, int ng)
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
        // persistent tick (fused 1): work queue and per-stream progress;
        // fused 2: the cooperative per-pixel stage
        int fused = 0;
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
        const bool band_only = !t.any_mix && t.uniform_halo >= 0;
        t.fused = (b->tune.fused == 1 && band_only && t.uniform_halo <= kTickMaxHalo)     ? 1
                  : (b->tune.fused == 2 && band_only && t.uniform_halo <= kStripMaxHalo) ? 2
                                                                                        : 0;
        if (t.fused == 1) {
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
             (t.fused != 1 ||
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
        bd.fused = t.fused;
        const bool queue = t.fused == 1;
        bd.items = queue ? reinterpret_cast<const int4 *>(A + t.o_items) : nullptr;
        bd.nitems = queue ? (int)t.items.size() : 0;
        bd.sync = queue ? reinterpret_cast<TickSync *>(A + t.o_sync) : nullptr;
        bd.tick_head = queue ? reinterpret_cast<uint32_t *>(A + t.o_head) : nullptr;
        bd.tick_exit = queue ? bd.tick_head + 1 : nullptr;
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

namespace {

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
}  // namespace

int hmi::default_groups(hmi_stream *const *s, int n, const hmi_tuning &t)
{
    bool fusable = t.fused != 0;
    for (int i = 0; i < n && fusable; ++i)
        fusable = s[i]->L.mix_k == 0 && 2 * (s[i]->p.open_iters + s[i]->p.close_iters) <= kTickMaxHalo;
    return fusable ? 1 : std::min(2, n);
}


hmi_batch *hmi::batch_new(hmi_stream *const *s, int n, int ngroups)
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

namespace {

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
}  // namespace

int hmi::flush_pending(hmi_batch *b, cudaStream_t cs)
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

namespace {

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

}  // namespace

int hmi::acquire_slot(hmi_batch *b)
{
    const int slot = b->next;
    b->next = (b->next + 1) % kRing;
    if (b->slot_used[slot]) {
        cudaError_t e = cudaEventSynchronize(b->slot_ev[slot]);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return slot;
}


int hmi::run_tick(hmi_batch *b, int slot, cudaStream_t cs, bool use_graph)
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


bool hmi::all_learned(hmi_batch *b)
{
    for (auto s : b->s)
        if (!s->learned) return false;
    return true;
}

namespace {

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

}  // namespace

int hmi::batch_async(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
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


int hmi::batch_pipelined(hmi_batch *b, const uint8_t *const *frames, uint8_t *const *masks,
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

namespace {
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
}  // namespace

hmi_stream *hmi::create_stream_on(int w, int h, const hmi_params *p, cudaStream_t order)
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

namespace {

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
}  // namespace

int hmi::batch_replan(hmi_batch *b, hmi_stream *const *s, int n, int ngroups)
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

namespace {

// An empty Gaussian mixture (every plane zero: no component), before its
// learning frames.
}  // namespace

cudaError_t hmi::enqueue_mix_reset(hmi_stream *s, cudaStream_t cs)
{
    if (!s->L.mix_k) return cudaSuccess;
    return cudaMemsetAsync(s->arena + s->L.mix, 0, s->L.mbytes, cs);
}

namespace {

// Band of a stream from its learned sums after n frames (Sec. 3.1 (i)), in
// the padded row layout; the padding bytes are zeroed first.
}  // namespace

cudaError_t hmi::enqueue_band(hmi_stream *s, int n, cudaStream_t cs)
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
