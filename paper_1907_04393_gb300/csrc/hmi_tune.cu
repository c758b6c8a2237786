// hmi_tune.cu -- launch shapes of a plan (hmi_tuning): validity, re-planning
// with a new shape, and the autotuner, which times whole ticks of the caller's
// frames for each candidate shape on the plan's own streams (stream state
// saved and restored around the search) and keeps the fastest.  The axes are
// the tick form (the chain of kernels, the persistent tick or the cooperative
// per-pixel stage), the piece size of the per-pixel kernels, CTAs per SM of
// the luma, skin and block kernels, the threads of a stream's merge CTA, and
// the pipeline depth or stream groups; the form and the piece size are
// searched together, the others one at a time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <utility>
#include <vector>

#include "hmi_host.h"

bool hmi::tuning_ok(const hmi_tuning &t)
{
    return t.piece_chunks >= 32 && t.piece_chunks <= 65536 && t.piece_chunks % 32 == 0 &&
           t.luma_ctas_per_sm >= 0 && t.luma_ctas_per_sm <= 32 && t.skin_ctas_per_sm >= 1 &&
           t.skin_ctas_per_sm <= 32 && t.cc_ctas_per_sm >= 1 && t.cc_ctas_per_sm <= 32 &&
           t.groups >= 0 && t.groups <= 64 && t.pipeline_depth >= 2 && t.pipeline_depth <= kPhases &&
           (t.fused >= 0 && t.fused <= 2) && t.queue_lag >= 0 && t.queue_lag <= (1 << 20) &&
           (t.merge_threads == 0 || t.merge_threads == 256 || t.merge_threads == 512 ||
            t.merge_threads == 1024);
}

// Apply a launch shape: the plan is re-made with the device idle.
int hmi::batch_retune(hmi_batch *b, const hmi_tuning &t)
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
// pointers not written), after untimed ticks that build the graph of every
// per-tick slot (a slot's graph is made on its first use; timing that would
// rank shapes by graph instantiation, not by their ticks).
namespace {

int time_ticks(hmi_batch *b, const uint8_t *const *frames, int ticks, bool pipelined, double *us)
{
    auto one = [&]() {
        return pipelined ? batch_pipelined(b, frames, nullptr, nullptr, b->cs, 1)
                         : batch_async(b, frames, nullptr, nullptr, b->cs, 1);
    };
    for (int i = 0; i < kRing + 3; ++i) {
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

}  // namespace

int hmi::batch_autotune(hmi_batch *b, const uint8_t *const *frames, int ticks, bool pipelined,
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
    // the tick form and the piece size together (each form has its own best
    // piece size: a form ranked at another form's piece size can lose to it
    // there and win at its own), then the other parameters one at a time
    const hmi_tuning base = cur;
    for (int32_t f : {0, 1, 2}) {
        for (int32_t p : {128, 256, 512, 1024, 2048}) {
            if (st != HMI_OK || (f == cur.fused && p == cur.piece_chunks)) continue;
            hmi_tuning cand = base;
            cand.fused = f;
            cand.piece_chunks = p;
            double us = 0.0;
            st = batch_retune(b, cand);
            if (st == HMI_OK) st = time_ticks(b, frames, ticks, pipelined, &us);
            if (st == HMI_OK && us < cur_us) {
                cur = cand;
                cur_us = us;
            }
        }
    }
    struct Axis {
        int32_t hmi_tuning::*field;
        std::vector<int32_t> values;
    };
    std::vector<Axis> axes = {{&hmi_tuning::luma_ctas_per_sm, {0, 2, 3, 4, 6}},
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

