// hmi_server.cu -- the serving loop of the C ABI (hmi_server_*): admission of
// camera streams by a device-memory budget, resident per-stream state, online
// learning from a stream's first frames, and continuous batching by a
// dispatcher thread that issues one tick over the admitted streams per round
// while the previous round is still on the device (Sec. 2 running step, per
// stream; the batching and serving layers are this library's own).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "hmi_host.h"

namespace {

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
    std::vector<SrvFrame> more;     // further queued learning frames of a learning stream
};

// Learning frames a learning stream may give one round: its queue drains this
// many times faster while it learns (a round processes at most one frame of a
// stream that already runs), so a burst of streams joining at once does not
// leave them behind their arrivals.
constexpr int kLearnPerRound = 4;

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
                // a learning stream's later learning frames join the round too
                // (learn_done is this thread's own state)
                int more = st.s ? std::min(kLearnPerRound - 1, st.learn_n - st.learn_done - 1) : 0;
                for (; more > 0 && !st.q.empty(); --more) {
                    take[i].more.push_back(st.q.front());
                    st.q.pop_front();
                }
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
        const size_t per = sizeof(LearnItem) * (size_t)cap * kLearnPerRound;   // a table per layer
        if (cudaMallocHost(&v->h_items[0], per) == cudaSuccess && cudaMallocHost(&v->h_items[1], per) == cudaSuccess &&
            cudaMalloc(&v->d_items, per) == cudaSuccess)
            v->item_cap = cap;
        else
            status = HMI_ERR_NO_MEMORY;
    }
    // Learning frames in layers: layer 0 holds each learning stream's frame of
    // this round, layer k its k-th further learning frame; one batched launch
    // per layer, so that a stream's frames add to its sums one after the
    // other.  A layer's table has its own host and device region (the copies
    // of earlier layers may not have run yet).
    for (int layer = 0; layer < kLearnPerRound && status == HMI_OK; ++layer) {
        LearnItem *items = v->h_items[buf] + (size_t)layer * v->item_cap;
        LearnItem *d_items = v->d_items + (size_t)layer * v->item_cap;
        int nitems = 0, in_layer = 0;
        unsigned long long quads = 0;
        for (int i = 0; i < n && status == HMI_OK; ++i) {
            if (!take[i].f.host || !take[i].learning || (int)take[i].more.size() < layer) continue;
            SrvStream *ss = take[i].ss;
            hmi_stream *s = ss->s;
            const long long npx = (long long)s->w * s->h;
            const uint8_t *fr = take[i].src ? take[i].src : s->d_frame;
            cudaError_t e = cudaSuccess;
            if (layer > 0) {   // a pinned frame is read in place, others go to the frame buffer
                const SrvFrame &m = take[i].more[layer - 1];
                cudaPointerAttributes at;
                fr = nullptr;
                if (npx % 4 == 0 && cudaPointerGetAttributes(&at, m.host) == cudaSuccess &&
                    at.type == cudaMemoryTypeHost && at.devicePointer != nullptr &&
                    (reinterpret_cast<uintptr_t>(at.devicePointer) & 3u) == 0)
                    fr = static_cast<const uint8_t *>(at.devicePointer);
                (void)cudaGetLastError();
                if (!fr) {
                    fr = s->d_frame;   // free again: the layers before have been enqueued
                    e = cudaMemcpyAsync(s->d_frame, m.host, m.bytes, cudaMemcpyHostToDevice, v->cs);
                }
            }
            if (e == cudaSuccess && layer == 0 && ss->learn_done == 0)
                e = cudaMemsetAsync(&s->st->learn_luma, 0, sizeof(unsigned long long), v->cs);
            if (e == cudaSuccess && npx % 4 == 0 && (reinterpret_cast<uintptr_t>(fr) & 3u) == 0) {
                items[nitems++] = LearnItem{fr, s->d_S, s->d_Q, s->d_vmin, s->d_vmax, s->st, quads,
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
            ++in_layer;
        }
        if (in_layer == 0) break;
        if (status == HMI_OK && nitems > 0 &&
            (cudaMemcpyAsync(d_items, items, sizeof(LearnItem) * nitems, cudaMemcpyHostToDevice, v->cs) !=
                 cudaSuccess ||
             launch_learn_batch(d_items, nitems, quads, v->cs) != cudaSuccess)) {
            (void)cudaGetLastError();
            status = HMI_ERR_DEVICE;
        }
        for (int i = 0; i < n && status == HMI_OK; ++i) {
            if (!take[i].f.host || !take[i].learning || (int)take[i].more.size() < layer) continue;
            SrvStream *ss = take[i].ss;
            hmi_stream *s = ss->s;
            cudaError_t e = cudaSuccess;
            if (s->L.mix_k) {   // the mixture learns the same frame
                const uint8_t *fr = layer == 0 ? (take[i].src ? take[i].src : s->d_frame) : nullptr;
                if (layer > 0) {
                    cudaPointerAttributes at;
                    const SrvFrame &m = take[i].more[layer - 1];
                    if (cudaPointerGetAttributes(&at, m.host) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                        at.devicePointer != nullptr &&
                        (reinterpret_cast<uintptr_t>(at.devicePointer) & 3u) == 0 && ((long long)s->w * s->h) % 4 == 0)
                        fr = static_cast<const uint8_t *>(at.devicePointer);
                    (void)cudaGetLastError();
                    if (!fr) fr = s->d_frame;   // copied there above
                }
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
        for (const SrvFrame &m : F.take[i].more) {   // the stream's further learning frames
            r.tag = m.tag;
            r.submit_ns = m.submit_ns;
            v->done.push_back(r);
            if (m.owned) v->pool[m.bytes].push_back(const_cast<uint8_t *>(m.host));
            v->frames += 1;
        }
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
    int st = s ? HMI_OK : hmi_last_error();
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
