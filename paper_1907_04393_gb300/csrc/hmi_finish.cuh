// hmi_finish.cuh -- the last step of a frame (Mouse module, Sec. 2: the binary
// image's hand zone becomes a pointer with a position and a click state),
// shared by the finishing kernel of a tick (hmi_cc.cu) and the persistent tick
// kernel (hmi_tick.cu): union-find over the block components that touch
// across block borders (8-connected; the root of every set is its component
// with the smallest key, the smallest pixel index, so the larger-key root is
// hooked under the smaller), the statistics of non-roots added into their
// roots, the largest root (ties: smaller label) or the tracked one, the
// pointer, the click state machine and the Interface module's event.  Every
// retry loop is bounded; overruns set an error flag in the stream state.
#pragma once

#include "hmi_ccfill.cuh"
#include "hmi_internal.cuh"

namespace hmi {

__device__ __forceinline__ uint32_t ld_parent(const uint32_t *parent, uint32_t i)
{
    return __ldcg(parent + i);
}

__device__ __forceinline__ uint32_t find_root(const uint32_t *parent, uint32_t x, uint32_t *err,
                                              uint32_t limit = kLoopLimit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        const uint32_t p = ld_parent(parent, x);
        if (p == x) return x;
        x = p;
    }
    atomicOr(err, kErrFindLoop);
    return x;
}

__device__ __forceinline__ void unite(uint32_t *parent, const Comp *comp, uint32_t a, uint32_t b,
                                      uint32_t *err, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        a = find_root(parent, a, err, limit);
        b = find_root(parent, b, err, limit);
        if (a == b) return;
        // hook the root with the larger key under the root with the smaller key
        if (comp[a].key < comp[b].key) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(parent + a, a, b) == a) return;
    }
    atomicOr(err, kErrUnionLoop);
}

// Unions of block `lb`'s components with those of one neighbour block that
// touch them across the shared border (8-connected).  dir 0: right,
// 1: down, 2: down-right corner, 3: down-left corner.
__device__ __forceinline__ void merge_dir(const DevStream &D, uint32_t lb, int dir, uint32_t *err,
                                          uint32_t limit)
{
    const int nw = D.nwords;
    const int by = (int)lb / nw, bx = (int)lb - by * nw;
    const bool has_r = bx + 1 < nw, has_d = by + 1 < D.bh, has_l = bx > 0;
    uint32_t nb;
    if (dir == 0) {
        if (!has_r) return;
        nb = lb + 1;
    } else if (dir == 1) {
        if (!has_d) return;
        nb = lb + nw;
    } else if (dir == 2) {
        if (!(has_d && has_r)) return;
        nb = lb + nw + 1;
    } else {
        if (!(has_d && has_l)) return;
        nb = lb + nw - 1;
    }
    const uint32_t cnt = D.count[lb];
    const uint32_t cn = D.count[nb];
    if (cn == 0) return;
    for (uint32_t j = 0; j < cnt; ++j) {
        const uint32_t id = lb * kSlots + j;
        const Comp &A = D.comp[id];
        const uint32_t edge = (dir == 0) ? A.right : A.bot;
        if (edge == 0u) continue;
        if (dir == 2 && !(edge >> 31)) continue;
        if (dir == 3 && !(edge & 1u)) continue;
        for (uint32_t i = 0; i < cn; ++i) {
            const Comp &B = D.comp[nb * kSlots + i];
            bool touch;
            if (dir == 0) {
                const uint32_t L = B.left;
                touch = (edge & (L | (L << 1) | (L >> 1))) != 0u;
            } else if (dir == 1) {
                const uint32_t T = B.top;
                touch = (edge & (T | (T << 1) | (T >> 1))) != 0u;
            } else if (dir == 2) {
                touch = (B.top & 1u) != 0u;
            } else {
                touch = (B.top >> 31) != 0u;
            }
            if (touch) unite(D.parent, D.comp, id, nb * kSlots + i, err, limit);
        }
    }
}

// Non-root components of block lb add their statistics into their roots.
__device__ __forceinline__ void resolve_block(const DevStream &D, uint32_t lb, uint32_t *err,
                                              uint32_t limit)
{
    const uint32_t cnt = D.count[lb];
    for (uint32_t j = 0; j < cnt; ++j) {
        const uint32_t id = lb * kSlots + j;
        const uint32_t r = find_root(D.parent, id, err, limit);
        if (r == id) continue;
        const Comp &A = D.comp[id];
        Comp &R = D.comp[r];
        atomicAdd(&R.area, A.area);
        atomicAdd(&R.sx, A.sx);
        atomicAdd(&R.sy, A.sy);
        atomicMin(&R.x0, A.x0);
        atomicMin(&R.y0, A.y0);
        atomicMax(&R.x1, A.x1);
        atomicMax(&R.y1, A.y1);
    }
}

// The Interface module's event (Sec. 2) and the driving wheel (Sec. 4) from
// the frame's pointer point (px, py), valid or not; see hmi_interface.
__device__ __forceinline__ int32_t diamond_angle(long long dx, long long dy)
{
    const long long u = dx, v = -dy;
    if (u == 0 && v == 0) return 0;
    if (u >= 0 && v > 0) return (int32_t)(1024 * u / (u + v));
    if (u > 0 && v <= 0) return (int32_t)(1024 + 1024 * (-v) / (u - v));
    if (u <= 0 && v < 0) return (int32_t)(2048 + 1024 * (-u) / (-u - v));
    return (int32_t)(3072 + 1024 * v / (v - u));
}

__device__ __forceinline__ void interface_event(const DevStream &D, bool valid, int32_t px, int32_t py, int32_t click,
                                int32_t frame, hmi_event *out)
{
    hmi_event E;
    E.zone = -1;
    E.event = -1;
    E.on_wheel = E.steer = E.left = E.right = E.throttle = 0;
    E.frame = frame;
    const hmi_interface &U = *D.ui;
    if (valid) {
        for (int z = 0; z < U.nzones && z < HMI_MAX_ZONES; ++z) {
            const hmi_zone &Z = U.zones[z];
            if (px >= Z.x0 && px <= Z.x1 && py >= Z.y0 && py <= Z.y1) {
                E.zone = z;
                E.event = Z.event;
                break;
            }
        }
        if (U.wheel_on) {
            const long long dx = (long long)px - U.wheel_cx, dy = (long long)py - U.wheel_cy;
            const long long d2 = dx * dx + dy * dy;
            const long long r0 = U.wheel_r_in, r1 = U.wheel_r_out;
            if (d2 >= r0 * r0 && d2 <= r1 * r1) {
                const int32_t a = diamond_angle(dx, dy);
                E.on_wheel = 1;
                E.steer = a > 2048 ? a - 4096 : a;
                E.left = E.steer < -U.dead_zone;
                E.right = E.steer > U.dead_zone;
                E.throttle = click != 0;
            }
        }
    }
    *out = E;
}

// Pointer of one stream from its largest component's statistics (has == 0:
// no foreground), then the click state machine: A_ref = max area of the last
// click_window valid frames; a valid frame sets the click when
// 100*area < on*A_ref and clears it when 100*area > off*A_ref (no history yet:
// no click) and is then appended; an invalid frame changes nothing.
__device__ __forceinline__ void finalize_pointer(const DevStream &D, const TickIO &io, bool has, uint32_t area,
                                 uint32_t key, unsigned long long sx, unsigned long long sy,
                                 int x0, int y0, int x1, int y1, const uint32_t *hist_copy = nullptr)
{
    StreamState *st = D.st;
    hmi_pointer P;
    if (!has) {
        P.valid = 0; P.area = 0; P.label = -1;
        P.x0 = P.y0 = P.x1 = P.y1 = -1;
        P.x = -1.0f; P.y = -1.0f;
    } else {
        P.area = area;
        P.label = (int32_t)key;
        P.valid = area >= D.min_area ? 1 : 0;
        P.x = (float)((double)sx / (double)area);
        P.y = (float)((double)sy / (double)area);
        P.x0 = x0; P.y0 = y0; P.x1 = x1; P.y1 = y1;
    }
    if (P.valid) {   // the tracked point follows the valid pointer
        st->track_valid = 1;
        st->track_x = (int32_t)((2ull * sx + area) / (2ull * area));
        st->track_y = (int32_t)((2ull * sy + area) / (2ull * area));
    }
    if (P.valid) {
        const int win = D.click_window;
        if (st->hist_count == 0) {
            st->click = 0;
        } else {
            unsigned long long aref = 0;
            const uint32_t *hs = hist_copy ? hist_copy : D.hist;
            for (int i = 0; i < st->hist_count; ++i) {
                const uint32_t a = hs[(st->hist_head + i) % win];
                if (a > aref) aref = a;
            }
            const unsigned long long a100 = 100ull * P.area;
            if (a100 < (unsigned long long)D.click_on * aref) st->click = 1;
            else if (a100 > (unsigned long long)D.click_off * aref) st->click = 0;
        }
        if (win > 0) {
            if (st->hist_count < win) {
                D.hist[(st->hist_head + st->hist_count) % win] = P.area;
                st->hist_count += 1;
            } else {
                D.hist[st->hist_head] = P.area;
                st->hist_head = (st->hist_head + 1) % win;
            }
        }
    }
    P.click = st->click;
    for (int k = 0; k < 3; ++k)   // the phase whose bit mask holds this frame, for the labels
        if (D.bits == D.bits_p[k]) st->last_phase = (uint32_t)k;
    interface_event(D, P.valid != 0, st->track_x, st->track_y, P.click, st->frames + 1, &st->event);
    st->last = P;
    st->frames += 1;
    st->best = 0ull;
    if (io.ptr_out != nullptr) *io.ptr_out = P;
}

// Pointer from the packed argmax (area, ~key) over the global records.
__device__ __forceinline__ void finalize_stream(const DevStream &D, const TickIO &io, unsigned long long best)
{
    if (best == 0ull) {
        finalize_pointer(D, io, false, 0, 0, 0, 0, 0, 0, 0, 0);
        return;
    }
    const uint32_t area = (uint32_t)(best >> 32);
    const uint32_t key = 0xffffffffu - (uint32_t)(best & 0xffffffffull);
    const uint32_t y = key / (uint32_t)D.w, x = key - y * (uint32_t)D.w;
    const uint32_t blk = (y / kBlock) * (uint32_t)D.nwords + x / kWordPx;
    const uint32_t cnt = D.count[blk];
    for (uint32_t j = 0; j < cnt; ++j) {
        const Comp &C = D.comp[blk * kSlots + j];
        if (C.key == key) {
            finalize_pointer(D, io, true, area, key, __ldcg(&C.sx), __ldcg(&C.sy), __ldcg(&C.x0),
                             __ldcg(&C.y0), __ldcg(&C.x1), __ldcg(&C.y1));
            return;
        }
    }
    atomicOr(&D.st->err, kErrRoot);
    finalize_pointer(D, io, false, 0, 0, 0, 0, 0, 0, 0, 0);
}

// One CTA per stream.  The blocks that hold components are listed in
// ascending order in shared memory and their component records copied there;
// the border merge (union-find with atomicCAS on shared parents, larger key
// hooked under the smaller), the resolve of non-roots into roots, and the
// argmax on (area, ~key) then all run in shared memory between CTA barriers,
// with no grid-wide wait.  Final roots are written back to the global parent
// array for the on-demand labels.  A stream with more than ACT non-empty
// blocks or REC components runs the same steps on the global arrays.
template <int NT, int ACT, int REC>
struct FinishSmem {
    Comp rec[REC];
    uint32_t hist[1024];         // click history (click_window <= 1024)
    uint32_t parent[REC];
    uint32_t act[ACT];           // non-empty blocks, ascending
    uint32_t rbase[ACT + 1];     // first record of each listed block
    uint32_t wsum[NT / 32];
    uint32_t nact, nrec, pick;
    unsigned long long best;     // packed (area, ~key) of the largest root
    uint32_t tdist;              // tracking: least box distance to the tracked point
    unsigned long long tbest;    // tracking: packed (area, ~key) among the nearest
    bool overflow;
};

// L1 distance from point (tx, ty) to the box [x0, x1] x [y0, y1] (0 inside).
__device__ __forceinline__ uint32_t box_dist(int tx, int ty, int x0, int y0, int x1, int y1)
{
    const int dx = max(0, max(x0 - tx, tx - x1));
    const int dy = max(0, max(y0 - ty, ty - y1));
    return (uint32_t)(dx + dy);
}

__device__ __forceinline__ bool tracking(const DevStream &D)
{
    return D.track_max_dist > 0 && D.st->track_valid;
}

// Root of x with path halving (every visited node is re-pointed to its
// grandparent, always an ancestor, so concurrent unions stay correct).
// At most `limit` steps (a path is never longer than the records); running
// out sets kErrFindLoop in *err.
__device__ __forceinline__ uint32_t sm_find(uint32_t *parent, uint32_t x, uint32_t limit, uint32_t *err)
{
    for (uint32_t it = 0; it < limit; ++it) {
        const uint32_t p = parent[x];
        if (p == x) return x;
        const uint32_t gp = parent[p];
        if (gp != p) parent[x] = gp;
        x = gp;
    }
    atomicOr(err, kErrFindLoop);
    return x;
}

__device__ __forceinline__ void sm_unite(uint32_t *parent, const Comp *rec, uint32_t a, uint32_t b,
                                         uint32_t limit, uint32_t *err)
{
    for (uint32_t it = 0; it < limit; ++it) {
        a = sm_find(parent, a, limit, err);
        b = sm_find(parent, b, limit, err);
        if (a == b) return;
        if (rec[a].key < rec[b].key) {
            const uint32_t t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(parent + a, a, b) == a) return;
    }
    atomicOr(err, kErrUnionLoop);
}

// index of block blk in the ascending list act[0..n), or -1
__device__ __forceinline__ int act_index(const uint32_t *act, uint32_t n, uint32_t blk)
{
    int lo = 0, hi = (int)n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (act[mid] < blk) lo = mid + 1; else hi = mid;
    }
    return (lo < (int)n && act[lo] == blk) ? lo : -1;
}

__device__ __forceinline__ void finish_global(const DevStream &D, const TickIO &io,
                                              unsigned long long *best, uint32_t *tdist,
                                              unsigned long long *tbest, uint32_t limit)
{
    uint32_t *err = &D.st->err;
    const uint32_t nblk = (uint32_t)D.bh * (uint32_t)D.nwords;
    for (uint32_t it = threadIdx.x; it < 4 * nblk; it += blockDim.x) {
        const uint32_t lb = it >> 2;
        if (D.count[lb] != 0u) merge_dir(D, lb, (int)(it & 3), err, limit);
    }
    __syncthreads();
    for (uint32_t lb = threadIdx.x; lb < nblk; lb += blockDim.x) resolve_block(D, lb, err, limit);
    __syncthreads();
    for (uint32_t lb = threadIdx.x; lb < nblk; lb += blockDim.x) {
        const uint32_t cnt = D.count[lb];
        for (uint32_t j = 0; j < cnt; ++j) {
            const uint32_t id = lb * kSlots + j;
            if (ld_parent(D.parent, id) != id) continue;
            const Comp &C = D.comp[id];
            const unsigned long long packed = ((unsigned long long)__ldcg(&C.area) << 32) |
                                              (unsigned long long)(0xffffffffu - C.key);
            atomicMax(best, packed);
        }
    }
    __syncthreads();
    if (tracking(D)) {   // the root nearest the tracked point (same rule as the shared path)
        const int tx = D.st->track_x, ty = D.st->track_y;
        for (int pass = 0; pass < 2; ++pass) {
            for (uint32_t lb = threadIdx.x; lb < nblk; lb += blockDim.x) {
                const uint32_t cnt = D.count[lb];
                for (uint32_t j = 0; j < cnt; ++j) {
                    const uint32_t id = lb * kSlots + j;
                    if (ld_parent(D.parent, id) != id) continue;
                    const Comp &C = D.comp[id];
                    const uint32_t area = __ldcg(&C.area);
                    if (area < D.min_area) continue;
                    const uint32_t d = box_dist(tx, ty, __ldcg(&C.x0), __ldcg(&C.y0), __ldcg(&C.x1), __ldcg(&C.y1));
                    if (d > (uint32_t)D.track_max_dist) continue;
                    if (pass == 0) atomicMin(tdist, d);
                    else if (d == *tdist)
                        atomicMax(tbest, ((unsigned long long)area << 32) | (unsigned long long)(0xffffffffu - C.key));
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) finalize_stream(D, io, *tbest ? *tbest : *best);
}

// The finish of one stream by a CTA of NT threads (ACT listed blocks and REC
// records at most in shared memory; beyond them the global path).  Stream
// errors are ORed into *batch_err; every union-find loop takes at most
// `limit` steps.
template <int NT, int ACT, int REC>
__device__ __forceinline__ void finish_stream(const DevStream &D, const TickIO &io,
                                              FinishSmem<NT, ACT, REC> &S, uint32_t *batch_err,
                                              uint32_t limit)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t nblk = (uint32_t)D.bh * (uint32_t)D.nwords;
    uint32_t *err = &D.st->err;
    if (tid == 0) {
        S.nact = 0;
        S.nrec = 0;
        S.best = 0;
        S.tdist = 0xffffffffu;
        S.tbest = 0;
        S.overflow = false;
        S.pick = 0xffffffffu;
    }
    for (int i = tid; i < D.click_window; i += blockDim.x) S.hist[i] = D.hist[i];
    __syncthreads();
    // ordered list of non-empty blocks and their record offsets
    for (uint32_t base = 0; base < nblk; base += blockDim.x) {
        const uint32_t blk = base + tid;
        const uint32_t cnt = blk < nblk ? D.count[blk] : 0u;
        const unsigned m = __ballot_sync(kFull, cnt != 0u);
        if (lane == 0) S.wsum[wid] = (uint32_t)__popc(m);
        __syncthreads();
        uint32_t off = S.nact;
        for (int i = 0; i < wid; ++i) off += S.wsum[i];
        const uint32_t pos = off + (uint32_t)__popc(m & ((1u << lane) - 1u));
        if (cnt != 0u && pos < (uint32_t)ACT) {
            S.act[pos] = blk;
            S.rbase[pos] = cnt;   // counts for now, offsets below
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t t = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += S.wsum[i];
            S.nact += t;
        }
        __syncthreads();
    }
    if (S.nact > (uint32_t)ACT) {
        if (tid == 0) S.overflow = true;
    } else {
        // exclusive scan of the listed blocks' counts, ACT / NT per thread
        constexpr int kPer = ACT / NT;
        const uint32_t na0 = S.nact;
        uint32_t v[kPer], run = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t i = (uint32_t)tid * kPer + q;
            v[q] = i < na0 ? S.rbase[i] : 0u;
            run += v[q];
        }
        uint32_t incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        __syncthreads();
        if (lane == 31) S.wsum[wid] = incl;
        __syncthreads();
        uint32_t off = incl - run;
        for (int i = 0; i < wid; ++i) off += S.wsum[i];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const uint32_t i = (uint32_t)tid * kPer + q;
            if (i < na0) S.rbase[i] = off;
            off += v[q];
        }
        if (tid == NT - 1) {
            S.rbase[na0] = off;
            S.nrec = off;
            if (off > (uint32_t)REC) S.overflow = true;
        }
    }
    __syncthreads();
    if (S.overflow) {
        finish_global(D, io, &S.best, &S.tdist, &S.tbest, limit);
        if (tid == 0) {   // this frame's errors are reported once, through the batch
            const uint32_t e = D.st->err;
            if (e) {
                atomicOr(batch_err, e);
                atomicAnd(&D.st->err, ~e);   // flags raised meanwhile stay for the next report
            }
        }
        return;
    }
    const uint32_t na = S.nact, nr = S.nrec;
    // copy the records
    for (uint32_t r = tid; r < nr; r += blockDim.x) {
        int lo = 0, hi = (int)na - 1;   // last i with rbase[i] <= r
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (S.rbase[mid] <= r) lo = mid; else hi = mid - 1;
        }
        const uint32_t gid = S.act[lo] * kSlots + (r - S.rbase[lo]);
        const uint4 *src = reinterpret_cast<const uint4 *>(D.comp + gid);
        uint4 *dst = reinterpret_cast<uint4 *>(S.rec + r);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = src[q];
        S.parent[r] = r;
    }
    __syncthreads();
    // border merge: item = (listed block, direction)
    const int nw = D.nwords;
    for (uint32_t it = tid; it < 4 * na; it += blockDim.x) {
        const uint32_t i = it >> 2, dir = it & 3;
        const uint32_t lb = S.act[i];
        const int by = (int)lb / nw, bx = (int)lb - by * nw;
        int nbb;
        if (dir == 0) nbb = (bx + 1 < nw) ? (int)lb + 1 : -1;
        else if (dir == 1) nbb = (by + 1 < D.bh) ? (int)lb + nw : -1;
        else if (dir == 2) nbb = (by + 1 < D.bh && bx + 1 < nw) ? (int)lb + nw + 1 : -1;
        else nbb = (by + 1 < D.bh && bx > 0) ? (int)lb + nw - 1 : -1;
        if (nbb < 0) continue;
        const int ni = act_index(S.act, na, (uint32_t)nbb);
        if (ni < 0) continue;
        for (uint32_t a = S.rbase[i]; a < S.rbase[i + 1]; ++a) {
            const uint32_t edge = (dir == 0) ? S.rec[a].right : S.rec[a].bot;
            if (edge == 0u) continue;
            if (dir == 2 && !(edge >> 31)) continue;
            if (dir == 3 && !(edge & 1u)) continue;
            for (uint32_t c = S.rbase[ni]; c < S.rbase[ni + 1]; ++c) {
                bool touch;
                if (dir == 0) {
                    const uint32_t L = S.rec[c].left;
                    touch = (edge & (L | (L << 1) | (L >> 1))) != 0u;
                } else if (dir == 1) {
                    const uint32_t T = S.rec[c].top;
                    touch = (edge & (T | (T << 1) | (T >> 1))) != 0u;
                } else if (dir == 2) {
                    touch = (S.rec[c].top & 1u) != 0u;
                } else {
                    touch = (S.rec[c].top >> 31) != 0u;
                }
                if (touch) sm_unite(S.parent, S.rec, a, c, limit, err);
            }
        }
    }
    __syncthreads();
    for (uint32_t r = tid; r < nr; r += blockDim.x) S.parent[r] = sm_find(S.parent, r, limit, err);
    __syncthreads();
    // resolve: non-roots into roots, aggregated per warp and root (a block
    // record's sums are below 2^23 and at most 32 are combined, so the
    // per-warp sums fit in 32 bits); final roots back to the global parents
    for (uint32_t base = 0; base < nr; base += blockDim.x) {
        const uint32_t r = base + tid;
        const bool valid = r < nr;
        const uint32_t root = valid ? S.parent[r] : 0xffffffffu;
        const bool contrib = valid && root != r;
        if (valid) {
            int lo = 0, hi = (int)na - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (S.rbase[mid] <= r) lo = mid; else hi = mid - 1;
            }
            int lo2 = 0, hi2 = (int)na - 1;
            while (lo2 < hi2) {
                const int mid = (lo2 + hi2 + 1) >> 1;
                if (S.rbase[mid] <= root) lo2 = mid; else hi2 = mid - 1;
            }
            D.parent[S.act[lo] * kSlots + (r - S.rbase[lo])] = S.act[lo2] * kSlots + (root - S.rbase[lo2]);
        }
        const uint32_t key = contrib ? root : 0xfffffffeu;
        const unsigned grp = __match_any_sync(kFull, key);
        if (contrib) {
            const Comp &A = S.rec[r];
            const uint32_t area = __reduce_add_sync(grp, A.area);
            const uint32_t sx = __reduce_add_sync(grp, (uint32_t)A.sx);
            const uint32_t sy = __reduce_add_sync(grp, (uint32_t)A.sy);
            const uint32_t x0 = __reduce_min_sync(grp, (uint32_t)A.x0);
            const uint32_t y0 = __reduce_min_sync(grp, (uint32_t)A.y0);
            const uint32_t x1 = __reduce_max_sync(grp, (uint32_t)A.x1);
            const uint32_t y1 = __reduce_max_sync(grp, (uint32_t)A.y1);
            if (lane == __ffs(grp) - 1) {
                Comp &R = S.rec[root];
                atomicAdd(&R.area, area);
                atomicAdd(&R.sx, (unsigned long long)sx);
                atomicAdd(&R.sy, (unsigned long long)sy);
                atomicMin(&R.x0, (int)x0);
                atomicMin(&R.y0, (int)y0);
                atomicMax(&R.x1, (int)x1);
                atomicMax(&R.y1, (int)y1);
            }
        }
    }
    __syncthreads();
    for (uint32_t r = tid; r < nr; r += blockDim.x) {
        if (S.parent[r] != r) continue;
        const unsigned long long packed = ((unsigned long long)S.rec[r].area << 32) |
                                          (unsigned long long)(0xffffffffu - S.rec[r].key);
        atomicMax(&S.best, packed);
    }
    __syncthreads();
    if (tracking(D)) {   // Sec. 2 tracking: the root nearest the tracked point
        const int tx = D.st->track_x, ty = D.st->track_y;
        for (int pass = 0; pass < 2; ++pass) {
            for (uint32_t r = tid; r < nr; r += blockDim.x) {
                if (S.parent[r] != r || S.rec[r].area < D.min_area) continue;
                const Comp &C = S.rec[r];
                const uint32_t d = box_dist(tx, ty, C.x0, C.y0, C.x1, C.y1);
                if (d > (uint32_t)D.track_max_dist) continue;
                if (pass == 0) atomicMin(&S.tdist, d);
                else if (d == S.tdist)
                    atomicMax(&S.tbest, ((unsigned long long)C.area << 32) | (unsigned long long)(0xffffffffu - C.key));
            }
            __syncthreads();
        }
    }
    const unsigned long long best = S.tbest ? S.tbest : S.best;
    for (uint32_t r = tid; r < nr; r += blockDim.x) {
        if (S.parent[r] == r && best != 0ull &&
            S.rec[r].key == 0xffffffffu - (uint32_t)(best & 0xffffffffull))
            S.pick = r;
    }
    __syncthreads();
    if (tid == 0) {
        if (best != 0ull && S.pick >= nr) atomicOr(err, kErrRoot);   // no root with the best key
        if (best == 0ull || S.pick >= nr) {
            finalize_pointer(D, io, false, 0, 0, 0, 0, 0, 0, 0, 0);
        } else {
            const Comp &C = S.rec[S.pick];
            finalize_pointer(D, io, true, C.area, C.key, C.sx, C.sy, C.x0, C.y0, C.x1, C.y1, S.hist);
        }
        const uint32_t e = D.st->err;   // this frame's errors are reported once, through the batch
        if (e) {
            atomicOr(batch_err, e);
            atomicAnd(&D.st->err, ~e);   // flags raised meanwhile stay for the next report
        }
    }
}

}  // namespace hmi
