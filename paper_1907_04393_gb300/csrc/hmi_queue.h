// hmi_queue.h -- the work queue of a persistent tick (host code, also built
// by the CPU tests): the per-stream progress record the kernel keeps, the kinds
// of work item and the planner that puts the items in order.
#pragma once

#include <stdint.h>
#include <vector_types.h>

#include <algorithm>
#include <vector>

namespace hmi {

// Per-stream progress of a persistent tick (hmi_tick.cu), in the plan's
// buffer: the planner writes the item counts; the counters and the stage go
// back to zero by the end of every tick.
struct TickSync {
    uint32_t nl, nc, nm;          // luma, classify and strips items of the stream
    uint32_t l, c, m;             // items of each kind finished this tick
    uint32_t stage;               // 0 luma; 1 gain ready; 2 raw bits complete (back to 0 after the strips)
    uint32_t pad;
};

// Work items of a persistent tick: int4 (kind << 24 | stream, begin, end, 0),
// chunk ranges for luma and classify items, strip ranges (kStripRows x 30 words,
// row-major over the stream's strips) for strips items.
enum : int { kItemLuma = 0, kItemClassify = 1, kItemStrips = 2 };
constexpr int kKinds = 3;
constexpr int kStripRows = 16;     // rows of a morphology strip (a divisor of 32)
constexpr int kStripsPerItem = 8;  // strips per strips item (one per warp)

inline int4 queue_item(int kind, int stream, int begin, int end)
{
    int4 e;
    e.x = (kind << 24) | stream;
    e.y = begin;
    e.z = end;
    e.w = 0;
    return e;
}

// Work queue of a persistent tick (hmi_tick.cu) over m streams with the given
// 16-px chunk and morphology strip counts, and each stream's item counts.  Per
// stream the items come in the order luma, classify, strips; a kind becomes
// eligible `lag` queue positions after the stream's last item of the kind
// before (so that, with at most lag items in flight, nobody waits and the
// frame read by the luma items is still in L2 for the classify items).
// Eligible later kinds go first; then luma items, largest streams first;
// once those run out, the rest in order.
inline std::vector<int4> tick_queue(const std::vector<int> &chunks, const std::vector<int> &strips, int piece,
                                    long long lag, std::vector<TickSync> *sync)
{
    const int m = (int)chunks.size();
    std::vector<int> ord(m);
    for (int i = 0; i < m; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return chunks[x] > chunks[y]; });
    sync->assign(m, TickSync{});
    std::vector<int4> seq[kKinds];   // per kind, streams in queue order
    for (int k : ord) {
        TickSync &Y = (*sync)[k];
        for (int c = 0; c < chunks[k]; c += piece) {
            seq[kItemLuma].push_back(queue_item(kItemLuma, k, c, std::min(chunks[k], c + piece)));
            seq[kItemClassify].push_back(queue_item(kItemClassify, k, c, std::min(chunks[k], c + piece)));
            ++Y.nl;
            ++Y.nc;
        }
        for (int q = 0; q < strips[k]; q += kStripsPerItem) {
            seq[kItemStrips].push_back(queue_item(kItemStrips, k, q, std::min(strips[k], q + kStripsPerItem)));
            ++Y.nm;
        }
    }
    size_t next[kKinds] = {0, 0, 0};
    std::vector<long long> left[kKinds], last[kKinds];
    for (int kind = 0; kind < kKinds; ++kind) {
        left[kind].assign(m, 0);
        last[kind].assign(m, -(1ll << 40));
        for (const int4 &e : seq[kind]) ++left[kind][e.x & 0xffffff];
    }
    const size_t total = seq[0].size() + seq[1].size() + seq[2].size();
    std::vector<int4> out;
    out.reserve(total);
    auto eligible = [&](int kind) {
        if (next[kind] >= seq[kind].size()) return false;
        if (kind == kItemLuma) return true;
        const int k = seq[kind][next[kind]].x & 0xffffff;
        return left[kind - 1][k] == 0 && (long long)out.size() - last[kind - 1][k] >= lag;
    };
    while (out.size() < total) {
        int kind = -1;
        for (int c : {kItemStrips, kItemClassify, kItemLuma})
            if (eligible(c)) {
                kind = c;
                break;
            }
        if (kind < 0)   // the tail: whatever comes next in order
            for (int c : {kItemClassify, kItemStrips})
                if (next[c] < seq[c].size()) {
                    kind = c;
                    break;
                }
        const int4 e = seq[kind][next[kind]++];
        const int k = e.x & 0xffffff;
        --left[kind][k];
        last[kind][k] = (long long)out.size();
        out.push_back(e);
    }
    return out;
}

}  // namespace hmi
