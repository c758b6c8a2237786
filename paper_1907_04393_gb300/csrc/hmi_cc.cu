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

// Stream of CC block g (flattened over the batch) and the block's local index.
__device__ __forceinline__ int block_stream(const BatchDev &b, uint32_t g, uint32_t *local)
{
    int lo = 0, hi = b.n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (b.block_prefix[mid] <= g) lo = mid; else hi = mid;
    }
    *local = g - b.block_prefix[lo];
    return lo;
}

__global__ void __launch_bounds__(kThreads) k_merge(BatchDev b)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= b.total_blocks) return;
    uint32_t lb;
    const DevStream &D = b.ds[block_stream(b, g, &lb)];
    const uint32_t cnt = D.count[lb];
    if (cnt == 0) return;
    const int nw = D.nwords;
    const int by = (int)lb / nw, bx = (int)lb - by * nw;
    const bool has_r = bx + 1 < nw, has_d = by + 1 < D.bh, has_l = bx > 0;
    const uint32_t nb_r = lb + 1, nb_d = lb + nw, nb_dr = lb + nw + 1, nb_dl = lb + nw - 1;
    const uint32_t c_r = has_r ? D.count[nb_r] : 0u;
    const uint32_t c_d = has_d ? D.count[nb_d] : 0u;
    const uint32_t c_dr = (has_d && has_r) ? D.count[nb_dr] : 0u;
    const uint32_t c_dl = (has_d && has_l) ? D.count[nb_dl] : 0u;
    uint32_t *err = &D.st->err;
    for (uint32_t j = 0; j < cnt; ++j) {
        const uint32_t id = lb * kSlots + j;
        const Comp &A = D.comp[id];
        const uint32_t ar = A.right, ab = A.bot;
        if (ar) {
            for (uint32_t i = 0; i < c_r; ++i) {
                const uint32_t L = D.comp[nb_r * kSlots + i].left;
                if (ar & (L | (L << 1) | (L >> 1))) unite(D.parent, D.comp, id, nb_r * kSlots + i, err);
            }
        }
        if (ab) {
            for (uint32_t i = 0; i < c_d; ++i) {
                const uint32_t T = D.comp[nb_d * kSlots + i].top;
                if (ab & (T | (T << 1) | (T >> 1))) unite(D.parent, D.comp, id, nb_d * kSlots + i, err);
            }
            if (ab >> 31) {
                for (uint32_t i = 0; i < c_dr; ++i)
                    if (D.comp[nb_dr * kSlots + i].top & 1u) unite(D.parent, D.comp, id, nb_dr * kSlots + i, err);
            }
            if (ab & 1u) {
                for (uint32_t i = 0; i < c_dl; ++i)
                    if (D.comp[nb_dl * kSlots + i].top >> 31) unite(D.parent, D.comp, id, nb_dl * kSlots + i, err);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_resolve(BatchDev b)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= b.total_blocks) return;
    uint32_t lb;
    const DevStream &D = b.ds[block_stream(b, g, &lb)];
    const uint32_t cnt = D.count[lb];
    uint32_t *err = &D.st->err;
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

__global__ void __launch_bounds__(kThreads) k_pointer(BatchDev b)
{
    __shared__ bool is_last;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < b.total_blocks) {
        uint32_t lb;
        const DevStream &D = b.ds[block_stream(b, g, &lb)];
        const uint32_t cnt = D.count[lb];
        for (uint32_t j = 0; j < cnt; ++j) {
            const uint32_t id = lb * kSlots + j;
            if (ld_parent(D.parent, id) != id) continue;
            const Comp &C = D.comp[id];
            const unsigned long long packed = ((unsigned long long)__ldcg(&C.area) << 32) |
                                              (unsigned long long)(0xffffffffu - C.key);
            atomicMax(&D.st->best, packed);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(&b.done[1], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int s = threadIdx.x; s < b.n; s += blockDim.x) {
        finalize_stream(b.ds[s], b.io[s]);
        const uint32_t e = b.ds[s].st->err;
        if (e) atomicOr(b.err, e);
    }
    if (threadIdx.x == 0) b.done[1] = 0;
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
static unsigned blocks_grid(const BatchDev &b)
{
    return (b.total_blocks + kThreads - 1) / kThreads;
}

cudaError_t launch_merge(const BatchDev &b, cudaStream_t cs)
{
    k_merge<<<blocks_grid(b), kThreads, 0, cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_resolve(const BatchDev &b, cudaStream_t cs)
{
    k_resolve<<<blocks_grid(b), kThreads, 0, cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_pointer(const BatchDev &b, cudaStream_t cs)
{
    k_pointer<<<blocks_grid(b), kThreads, 0, cs>>>(b);
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
