// hmi_cc.cu -- connected components across 32x32 blocks and the pointer
// (Mouse module, Sec. 2: the binary image's hand zone becomes a pointer with a
// position and a click state).
//   k_merge    union-find over the block components that touch across block
//              borders (8-connected); the root of every set is its component
//              with the smallest key (smallest pixel index), by hooking the
//              root with the larger key under the one with the smaller key
//   k_resolve  adds every non-root's statistics into its root
//   k_pointer  largest root (ties: smaller label) per stream, then the last
//              CTA writes every stream's pointer and steps its click state
//   k_labels   per-pixel labels on demand (label = root key), same component
//              enumeration as the tick's block pass
// Every retry loop is bounded; overruns set an error flag in the stream state.
#include "hmi_ccfill.cuh"
#include "hmi_internal.cuh"

namespace hmi {

__device__ __forceinline__ uint32_t ld_parent(const uint32_t *parent, uint32_t i)
{
    return __ldcg(parent + i);
}

__device__ __forceinline__ uint32_t find_root(const uint32_t *parent, uint32_t x, uint32_t *err)
{
    for (uint32_t it = 0; it < kLoopLimit; ++it) {
        const uint32_t p = ld_parent(parent, x);
        if (p == x) return x;
        x = p;
    }
    atomicOr(err, kErrFindLoop);
    return x;
}

__device__ void unite(uint32_t *parent, const Comp *comp, uint32_t a, uint32_t b, uint32_t *err)
{
    for (uint32_t it = 0; it < kLoopLimit; ++it) {
        a = find_root(parent, a, err);
        b = find_root(parent, b, err);
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
__device__ void merge_dir(const DevStream &D, uint32_t lb, int dir, uint32_t *err)
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
            if (touch) unite(D.parent, D.comp, id, nb * kSlots + i, err);
        }
    }
}

// Non-root components of block lb add their statistics into their roots.
__device__ void resolve_block(const DevStream &D, uint32_t lb, uint32_t *err)
{
    const uint32_t cnt = D.count[lb];
    for (uint32_t j = 0; j < cnt; ++j) {
        const uint32_t id = lb * kSlots + j;
        const uint32_t r = find_root(D.parent, id, err);
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

// Pointer of one stream from its packed argmax, then the click state machine:
// A_ref = max area of the last click_window valid frames; a valid frame sets
// the click when 100*area < on*A_ref and clears it when 100*area > off*A_ref
// (no history yet: no click) and is then appended; an invalid frame changes
// nothing.
__device__ void finalize_stream(const DevStream &D, const TickIO &io)
{
    StreamState *st = D.st;
    const unsigned long long best = *(volatile unsigned long long *)&st->best;
    hmi_pointer P;
    if (best == 0ull) {
        P.valid = 0; P.area = 0; P.label = -1;
        P.x0 = P.y0 = P.x1 = P.y1 = -1;
        P.x = -1.0f; P.y = -1.0f;
    } else {
        const uint32_t area = (uint32_t)(best >> 32);
        const uint32_t key = 0xffffffffu - (uint32_t)(best & 0xffffffffull);
        const uint32_t y = key / (uint32_t)D.w, x = key - y * (uint32_t)D.w;
        const uint32_t blk = (y / kBlock) * (uint32_t)D.nwords + x / kWordPx;
        const uint32_t cnt = D.count[blk];
        uint32_t r = 0xffffffffu;
        for (uint32_t j = 0; j < cnt; ++j)
            if (D.comp[blk * kSlots + j].key == key) { r = blk * kSlots + j; break; }
        if (r == 0xffffffffu) {
            atomicOr(&st->err, kErrRoot);
            P.valid = 0; P.area = 0; P.label = -1;
            P.x0 = P.y0 = P.x1 = P.y1 = -1;
            P.x = -1.0f; P.y = -1.0f;
        } else {
            const Comp &C = D.comp[r];
            P.area = area;
            P.label = (int32_t)key;
            P.valid = area >= D.min_area ? 1 : 0;
            P.x = (float)((double)C.sx / (double)area);
            P.y = (float)((double)C.sy / (double)area);
            P.x0 = C.x0; P.y0 = C.y0; P.x1 = C.x1; P.y1 = C.y1;
        }
    }
    if (P.valid) {
        const int win = D.click_window;
        if (st->hist_count == 0) {
            st->click = 0;
        } else {
            unsigned long long aref = 0;
            for (int i = 0; i < st->hist_count; ++i) {
                const uint32_t a = D.hist[(st->hist_head + i) % win];
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
    st->last = P;
    st->frames += 1;
    st->best = 0ull;
    if (io.ptr_out != nullptr) *io.ptr_out = P;
}

// One CTA per stream: the blocks that hold components are compacted into
// shared memory, then (separated by CTA barriers, no grid-wide wait) their
// borders are merged, non-roots are added into their roots, the largest root
// is chosen with a shared 64-bit atomicMax on (area, ~key), and thread 0
// writes the pointer and steps the click state.
constexpr int kFinishThreads = 512;
constexpr int kActCap = 4096;

__global__ void __launch_bounds__(kFinishThreads) k_finish(BatchDev b)
{
    __shared__ uint32_t act[kActCap];
    __shared__ uint32_t nact;
    __shared__ unsigned long long best;
    const int tid = threadIdx.x;
    const DevStream &D = b.ds[blockIdx.x];
    const TickIO io = b.io[blockIdx.x];
    uint32_t *err = &D.st->err;
    const uint32_t nblk = (uint32_t)D.bh * (uint32_t)D.nwords;
    if (tid == 0) {
        nact = 0;
        best = 0;
    }
    __syncthreads();
    for (uint32_t base = 0; base < nblk; base += blockDim.x) {
        const uint32_t blk = base + tid;
        const bool a = blk < nblk && D.count[blk] != 0u;
        const unsigned m = __ballot_sync(kFull, a);
        uint32_t pos = 0;
        if ((tid & 31) == 0 && m) pos = atomicAdd(&nact, (uint32_t)__popc(m));
        pos = __shfl_sync(kFull, pos, 0) + (uint32_t)__popc(m & ((1u << (tid & 31)) - 1u));
        if (a && pos < kActCap) act[pos] = blk;
    }
    __syncthreads();
    const uint32_t na = nact;
    const bool fits = na <= (uint32_t)kActCap;
    const uint32_t nitems = fits ? na : nblk;
    for (uint32_t it = tid; it < 4 * nitems; it += blockDim.x) {
        const uint32_t lb = fits ? act[it >> 2] : (it >> 2);
        if (!fits && D.count[lb] == 0u) continue;
        merge_dir(D, lb, (int)(it & 3), err);
    }
    __syncthreads();
    for (uint32_t it = tid; it < nitems; it += blockDim.x) resolve_block(D, fits ? act[it] : it, err);
    __syncthreads();
    for (uint32_t it = tid; it < nitems; it += blockDim.x) {
        const uint32_t lb = fits ? act[it] : it;
        const uint32_t cnt = D.count[lb];
        for (uint32_t j = 0; j < cnt; ++j) {
            const uint32_t id = lb * kSlots + j;
            if (ld_parent(D.parent, id) != id) continue;
            const Comp &C = D.comp[id];
            const unsigned long long packed = ((unsigned long long)__ldcg(&C.area) << 32) |
                                              (unsigned long long)(0xffffffffu - C.key);
            atomicMax(&best, packed);
        }
    }
    __syncthreads();
    if (tid == 0) {
        D.st->best = best;
        finalize_stream(D, io);
        const uint32_t e = D.st->err;
        if (e) atomicOr(b.err, e);
    }
}

// Labels of one stream: warp per 32x32 block.
__global__ void __launch_bounds__(kThreads) k_labels(const DevStream *dsp, int32_t *labels)
{
    const DevStream &D = *dsp;
    const int lane = threadIdx.x & 31;
    const int blk = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nblk = D.bh * D.nwords;
    if (blk >= nblk) return;   // warp-uniform
    const int by = blk / D.nwords, bx = blk - by * D.nwords;
    const int y = by * kBlock + lane, xb = bx * kWordPx;
    const int npx = min(kWordPx, D.w - xb);
    uint32_t m = D.bits[(long long)y * D.nwords + bx];
    int32_t *row = labels + (long long)y * D.w + xb;
    if (y < D.h)
        for (int i = 0; i < npx; ++i) row[i] = -1;
    uint32_t *err = &D.st->err;
    int j = 0;
    while (__any_sync(kFull, m != 0u)) {
        int r0, c0;
        const uint32_t c = cc_extract_first(m, lane, &r0, &c0);
        m &= ~c;
        int32_t lab = -1;
        if (lane == 0 && j < kSlots) {
            const uint32_t root = find_root(D.parent, (uint32_t)blk * kSlots + (uint32_t)j, err);
            lab = (int32_t)D.comp[root].key;
        }
        lab = __shfl_sync(kFull, lab, 0);
        if (y < D.h)
            for (int i = 0; i < npx; ++i)
                if ((c >> i) & 1u) row[i] = lab;
        ++j;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_finish(const BatchDev &b, cudaStream_t cs)
{
    k_finish<<<b.n, kFinishThreads, 0, cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_labels(const DevStream *ds_dev, const DevStream &ds, int32_t *labels,
                          cudaStream_t cs)
{
    const long long nblk = (long long)ds.bh * ds.nwords;
    const unsigned grid = (unsigned)((nblk * 32 + kThreads - 1) / kThreads);
    k_labels<<<grid, kThreads, 0, cs>>>(ds_dev, labels);
    return cudaGetLastError();
}

}  // namespace hmi
