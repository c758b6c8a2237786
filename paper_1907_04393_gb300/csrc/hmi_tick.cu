// hmi_tick.cu -- the per-pixel work of every band-test stream of a batch in
// one persistent launch per tick.
//
// The launch's CTAs take work items from a queue, in order, with one atomic
// counter.  Per stream there are three kinds of item, each kind depending only
// on the stream's items of the kind before it:
//   luma      a chunk range: the frame's integer luma sum (Sec. 2 brightness
//             correction, Sec. 3.2 luminosity filter); the last luma item of
//             the stream turns the sum into the Q16 gain and opens the stream
//   classify  a chunk range: gain, background band test (Sec. 3.1 (i)), gray
//             and hue tests (Sec. 3.1 (ii), (iii)) of the out-of-band pixels
//             and their AND, as raw mask bits
//   strips    up to eight strips of 16 rows: opening and closing (Sec. 3.1
//             erosion and dilation) in registers, the mask bits and 0/1 mask
//             bytes, and the list of 32x32 blocks holding foreground
// The blocks' components and their merge into the pointer (Mouse module,
// Sec. 2) follow in the tick's last two kernels, which a pipelined tick runs
// beside the next tick's persistent launch.
// A stream's counter of finished items of one kind releases the next kind
// (bounded waits; a wait that runs out sets an error flag and lets the item
// go on, so the tick always ends).  The planner orders the queue so that a
// stream's classify items come well after its luma items: by then the gain is
// ready and the frame, read once from HBM by the luma pass, is still in L2.
// No item waits for an item later in the queue, and every dequeued item runs
// on a resident CTA, so the launch cannot deadlock whatever the grid size.
//
// Integer and bit work bound by HBM bandwidth and issue rate; nothing here is
// a dense contraction, so no tensor-core path is used.
#include <algorithm>

#include "hmi_ccfill.cuh"
#include "hmi_internal.cuh"
#include "hmi_pixel.cuh"

namespace hmi {

constexpr int kTickWarps = kThreads / 32;
constexpr uint32_t kErrWait = 16u;

struct TickSmem {
    SkinSmem skin[kTickWarps];
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Frame words re-read by a classify item: coherent at L2 (a pinned host frame
// is stored into the staging frame by this launch's luma items), last use.
__device__ __forceinline__ void load48_cg(const uint8_t *src, uint64_t pol, uint32_t (&w)[12])
{
    const uint4 *q = reinterpret_cast<const uint4 *>(src);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint4 r;
        asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                     : "l"(q + k), "l"(pol));
        w[4 * k] = r.x; w[4 * k + 1] = r.y; w[4 * k + 2] = r.z; w[4 * k + 3] = r.w;
    }
}

// Frame words read by a luma item: default L2 priority, so that they are
// still there when the stream's classify items read them again.
__device__ __forceinline__ void load48_keep(const uint8_t *src, uint32_t (&w)[12])
{
    const uint4 *q = reinterpret_cast<const uint4 *>(src);
    const uint4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
}

// Thread 0 of a CTA: wait until the stream's stage reaches `want`, polling at
// most `limit` times (with sleeps, about a second at the default limit).
__device__ __forceinline__ void wait_stage(const uint32_t *stage, uint32_t want, uint32_t limit,
                                           uint32_t *err)
{
    for (uint32_t it = 0; it < limit; ++it) {
        if (ld_acquire(stage) >= want) return;
        __nanosleep(it < 64 ? 64 : 256);
    }
    atomicOr(err, kErrWait);
}

// Thread 0, after every thread of the CTA has fenced its writes: count one
// finished item of the kind counted by *done (n in all); the last one resets
// the count and moves the stream to stage `next`.  Returns true for the last.
__device__ __forceinline__ bool finish_item(uint32_t *done, uint32_t n, uint32_t *stage, uint32_t next)
{
    const uint32_t old = atomicAdd(done, 1u);
    if (old + 1u != n) return false;
    __threadfence();
    *done = 0u;
    __threadfence();
    st_release(stage, next);
    return true;
}

// ---------------------------------------------------------------------------
// luma item
// ---------------------------------------------------------------------------
constexpr int kLumaPerThread = 2;

__device__ __forceinline__ void item_luma(const BatchDev &b, int s, int c0, int c1,
                                          unsigned long long *red)
{
    const int tid = threadIdx.x;
    const DevStream &D = b.ds[s];
    const TickIO io = b.io[s];
    const int w = D.w, cpr = 2 * D.nwords;
    const uint32_t magic = D.cpr_magic;
    unsigned long long acc = 0;
    for (int u = c0 + tid; u < c1; u += kLumaPerThread * kThreads) {
        uint32_t f[kLumaPerThread][12];
        int npx[kLumaPerThread];
#pragma unroll
        for (int q = 0; q < kLumaPerThread; ++q) {
            const int uu = u + q * kThreads;
            npx[q] = 0;
            if (uu < c1) {
                const int y = chunk_row((uint32_t)uu, magic), x0 = (uu - y * cpr) * kChunkPx;
                if (x0 < w) {
                    npx[q] = min(kChunkPx, w - x0);
                    if (io.src) {   // a pinned host frame: w is a multiple of 16, rows dense
                        load48_host(io.src + (long long)y * 3 * w + 3 * x0, f[q]);
                        store48(const_cast<uint8_t *>(io.frame) + (long long)y * io.frame_pitch + 3 * x0, f[q]);
                    } else {
                        load48_keep(io.frame + (long long)y * io.frame_pitch + 3 * x0, f[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kLumaPerThread; ++q)
            if (npx[q] > 0) acc += (npx[q] == kChunkPx) ? luma_sum16(f[q]) : luma_sum_n(f[q], npx[q]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < kTickWarps; ++i) t += red[i];
        StreamState *st = D.st;
        atomicAdd(&st->sy, t);
        __threadfence();
        TickSync &Y = b.sync[s];
        const uint32_t old = atomicAdd(&Y.l, 1u);
        if (old + 1u == Y.nl) {   // the stream's whole luma sum is in: its gain
            __threadfence();
            const unsigned long long sy = *(volatile unsigned long long *)&st->sy;
            const unsigned long long syref = st->syref;
            unsigned long long g = (sy == 0) ? 65536ull : ((syref << 16) + sy / 2) / sy;
            if (g < D.gain_min) g = D.gain_min;
            if (g > D.gain_max) g = D.gain_max;
            st->gain = (uint32_t)g;
            st->gain_p[b.phase] = (uint32_t)g;
            st->sy = 0;
            st->lframes += 1;
            st->lframe_p[b.phase] = st->lframes;
            Y.l = 0u;
            __threadfence();
            st_release(&Y.stage, 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// classify item
// ---------------------------------------------------------------------------
__device__ __forceinline__ void item_classify(const BatchDev &b, int s, int c0, int c1, TickSmem &sm,
                                              uint8_t *table)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevStream &D = b.ds[s];
    const TickIO io = b.io[s];
    TickSync &Y = b.sync[s];
    if (tid == 0) wait_stage(&Y.stage, 1u, b.loop_limit, &D.st->err);
    __syncthreads();
    const uint32_t g = __ldcg(&D.st->gain_p[b.phase]);
    fill_table(table, g);
    __syncthreads();
    const uint64_t once = policy_evict_first();
    const int w = D.w, cpr = 2 * D.nwords, fpitch = D.fpitch;
    uint32_t *raw = D.raw[b.phase];
    SkinSmem &S = sm.skin[warp];
    // warp-uniform loop, so that chunk pairs can combine with a shuffle
    for (int base = c0 + (tid & ~31); base < c1; base += kThreads) {
        const int u = base + lane;
        uint32_t bits = 0;
        uint32_t f[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) f[k] = 0u;
        int y = 0, j = 0;
        if (u < c1) {
            y = chunk_row((uint32_t)u, D.cpr_magic);
            j = u - y * cpr;
            const int x0 = j * kChunkPx;
            if (x0 < w) {
                uint32_t l[12], h[12];
                load48_cg(io.frame + (long long)y * io.frame_pitch + 3 * x0, once, f);
                load48(D.lo + (long long)y * fpitch + 3 * x0, once, l);
                load48(D.hi + (long long)y * fpitch + 3 * x0, once, h);
                bits = band_outside16(f, l, h, TableCorr{table});
                const int npx = w - x0;
                if (npx < kChunkPx) bits &= (1u << npx) - 1u;
            }
        }
        bits &= ~skin_fail_warp(bits, f, D, table, S, lane);
        const uint32_t other = __shfl_xor_sync(kFull, bits, 1);
        if (u < c1 && (u & 1) == 0 && HMI_IN_BOUNDS(y < D.bh * kBlock && (j >> 1) < D.nwords, &D.st->err))
            raw[(long long)y * D.nwords + (j >> 1)] = bits | (other << 16);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) finish_item(&Y.c, Y.nc, &Y.stage, 2u);
}

// ---------------------------------------------------------------------------
// strips item
// ---------------------------------------------------------------------------
template <int HR>
__device__ __forceinline__ void item_strips_hr(const BatchDev &b, int s, int k0, int k1)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = k0 + warp;
    if (k >= k1) return;   // warp-uniform
    const DevStream &D = b.ds[s];
    const int ty = k / D.strips_x, tx = k - ty * D.strips_x;
    morph_strip<HR>(D, b.io[s], ty, tx, lane, s, b.cc_count, b.cc_list, b.total_blocks, D.raw[b.phase]);
}

__device__ __forceinline__ void item_strips(const BatchDev &b, int s, int k0, int k1)
{
    const int tid = threadIdx.x;
    const DevStream &D = b.ds[s];
    TickSync &Y = b.sync[s];
    if (tid == 0) wait_stage(&Y.stage, 2u, b.loop_limit, &D.st->err);
    __syncthreads();
    (void)ld_acquire(&Y.stage);   // every thread: raw bits of other CTAs are visible
    switch (b.uniform_halo) {   // the planner keeps halos above kTickMaxHalo in the chain
    case 0: item_strips_hr<0>(b, s, k0, k1); break;
    case 2: item_strips_hr<2>(b, s, k0, k1); break;
    default: item_strips_hr<4>(b, s, k0, k1); break;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) finish_item(&Y.m, Y.nm, &Y.stage, 0u);   // the stream is ready for the next tick
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 3) k_tick(BatchDev b)
{
    extern __shared__ __align__(16) unsigned char tick_smem[];
    TickSmem &sm = *reinterpret_cast<TickSmem *>(tick_smem);
    __shared__ unsigned long long red[kTickWarps];
    __shared__ uint8_t table[256];   // corrected values of a classify item's frame
    __shared__ int s_next;
    const int tid = threadIdx.x;
    if (tid == 0) s_next = (int)atomicAdd(b.tick_head, 1u);
    __syncthreads();
    int cur = s_next;
    while (cur < b.nitems) {
        __syncthreads();                                    // every thread has read s_next
        if (tid == 0) s_next = (int)atomicAdd(b.tick_head, 1u);   // the next item, fetched early
        const int4 e = b.items[cur];
        const int kind = e.x >> 24, s = e.x & 0xffffff;
        if (b.io[s].frame != nullptr) {                     // CTA-uniform: no frame, no work
            switch (kind) {
            case kItemLuma: item_luma(b, s, e.y, e.z, red); break;
            case kItemClassify: item_classify(b, s, e.y, e.z, sm, table); break;
            default: item_strips(b, s, e.y, e.z); break;
            }
        }
        __syncthreads();
        cur = s_next;
    }
    // the last CTA out resets the queue for the next tick
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(b.tick_exit, 1u) == gridDim.x - 1u) {
            *b.tick_head = 0u;
            *b.tick_exit = 0u;
        }
    }
}

int tick_ctas_per_sm(int requested)
{
    static int fit[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (fit[dev] == 0) {
        int n = 0;
        if (cudaFuncSetAttribute(k_tick, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(TickSmem)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tick, kThreads, sizeof(TickSmem)) != cudaSuccess ||
            n < 1) {
            (void)cudaGetLastError();
            n = 1;
        }
        fit[dev] = n;
    }
    return requested > 0 ? std::min(requested, fit[dev]) : fit[dev];
}

cudaError_t launch_tick(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    const int per = tick_ctas_per_sm(b.luma_ctas_per_sm);
    const int grid = std::max(1, std::min(b.nitems, num_sms * per));
    k_tick<<<grid, kThreads, sizeof(TickSmem), cs>>>(b);
    return cudaGetLastError();
}

}  // namespace hmi
