// hmi_frame.cu -- per-pixel kernels of a tick:
//   k_luma        frame luma sum per stream; the last CTA turns the sums into the
//                 brightness gains (Sec. 2 brightness correction,
//                 Sec. 3.2 luminosity filter)
//   k_classify    gain and background band test (Sec. 3.1 (i)) of every pixel,
//                 then the gray and hue tests (Sec. 3.1 (ii), (iii)) of its
//                 out-of-band pixels and the AND (the merging step), one bit
//                 per pixel
//   k_skin        the gray and hue tests of the pixels that the mixture
//                 background queued (bg_model 1 streams)
//   k_morph_strip opening/closing on the bit mask (Sec. 3.1 erosion and
//                 dilation) in registers, the 0/1 mask bytes, and the list
//                 of 32x32 blocks holding foreground
//   k_block_cc    8-connected components of each listed block with their
//                 statistics (Mouse module, Sec. 2)
//   k_morph_cc    generic form of the last two for mixed morphology settings
//   k_stage       k_luma, k_classify and k_morph_strip as the three phases of
//                 one cooperative launch, separated by grid barriers (the
//                 same Sec. 2, 3.1 and 3.2 steps, one launch ramp and tail)
// All are integer/bit work, bound by HBM bandwidth, issue rate or latency;
// nothing here is a dense contraction, so no tensor-core path is used.
#include <algorithm>

#include "hmi_ccfill.cuh"
#include "hmi_internal.cuh"
#include "hmi_pixel.cuh"

namespace hmi {

// ---------------------------------------------------------------------------
// k_luma: one resident wave of CTAs, each over a contiguous range of pieces.
// Consecutive pieces of one stream are walked as a single chunk range, with
// kLumaChunks chunks per thread in flight before the sums; the partial sum is
// flushed (one atomic per CTA) when the stream changes.
// ---------------------------------------------------------------------------
constexpr int kLumaChunks = 2;

__global__ void __launch_bounds__(kThreads, 5) k_luma(BatchDev b)
{
    __shared__ unsigned long long red[kThreads / 32];
    __shared__ bool is_last;
    const int tid = threadIdx.x;
    const uint64_t keep = policy_evict_first();
    const int p0 = (int)(((long long)b.npieces * blockIdx.x) / gridDim.x);
    const int p1 = (int)(((long long)b.npieces * (blockIdx.x + 1)) / gridDim.x);
    for (int pc = p0; pc < p1;) {
        const int4 first = b.pieces[pc];
        int c1 = first.z, pn = pc + 1;
        while (pn < p1) {
            const int4 nx = b.pieces[pn];
            if (nx.x != first.x || nx.y != c1) break;
            c1 = nx.z;
            ++pn;
        }
        pc = pn;
        const DevStream &D = b.ds[first.x];
        const TickIO io = b.io[first.x];
        if (io.frame == nullptr) continue;   // no frame for this stream this tick (CTA-uniform)
        const int w = D.w, cpr = 2 * D.nwords;
        const uint32_t magic = D.cpr_magic;
        unsigned long long acc = 0;
        for (int u = first.y + tid; u < c1; u += kLumaChunks * blockDim.x) {
            uint32_t f[kLumaChunks][12];
            int npx[kLumaChunks];
#pragma unroll
            for (int q = 0; q < kLumaChunks; ++q) {
                const int uu = u + q * (int)blockDim.x;
                npx[q] = 0;
                if (uu < c1) {
                    const int y = chunk_row((uint32_t)uu, magic), x0 = (uu - y * cpr) * kChunkPx;
                    if (x0 < w && HMI_IN_BOUNDS(y < D.h && 3LL * (x0 + kChunkPx) <= io.frame_pitch, &D.st->err)) {
                        npx[q] = min(kChunkPx, w - x0);
                        if (io.src) {   // a pinned host frame: w is a multiple of 16, rows dense
                            load48_host(io.src + (long long)y * 3 * w + 3 * x0, f[q]);
                            store48(const_cast<uint8_t *>(io.frame) + (long long)y * io.frame_pitch + 3 * x0, f[q]);
                        } else {
                            load48(io.frame + (long long)y * io.frame_pitch + 3 * x0, keep, f[q]);
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kLumaChunks; ++q)
                acc += (npx[q] == kChunkPx) ? luma_sum16(f[q]) : luma_sum_n(f[q], npx[q]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if ((tid & 31) == 0) red[tid >> 5] = acc;
        __syncthreads();
        if (tid == 0) {
            unsigned long long t = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
            atomicAdd(&D.st->sy, t);
        }
        __syncthreads();
    }
    // the last CTA to finish computes every stream's gain
    __threadfence();
    if (tid == 0) is_last = (atomicAdd(&b.done[0], 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int s = tid; s < b.n; s += blockDim.x) {
        if (b.io[s].frame == nullptr) continue;
        const DevStream &D = b.ds[s];
        StreamState *st = D.st;
        unsigned long long sy = *(volatile unsigned long long *)&st->sy;
        unsigned long long syref = st->syref;
        unsigned long long g = (sy == 0) ? 65536ull : ((syref << 16) + sy / 2) / sy;
        if (g < D.gain_min) g = D.gain_min;
        if (g > D.gain_max) g = D.gain_max;
        st->gain = (uint32_t)g;
        st->gain_p[b.phase] = (uint32_t)g;
        st->sy = 0;
        st->lframes += 1;
        st->lframe_p[b.phase] = st->lframes;   // read by later kernels of this tick only
    }
    if (tid == 0) b.done[0] = 0;
}

// ---------------------------------------------------------------------------
// k_classify
// ---------------------------------------------------------------------------
// One thread per 16-pixel chunk: the background test on all 16 pixels; the
// warp then lists its out-of-band pixels (a few percent: the hand, camera
// noise) in shared memory and its lanes share the gray and hue tests of that
// list, so that the raw mask word stored is the AND of the three tests.
__global__ void __launch_bounds__(kThreads, 4) k_classify(BatchDev b)
{
    __shared__ uint8_t table[256];
    __shared__ SkinSmem skin[kThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    const uint64_t once = policy_evict_first();
    for (int pc = blockIdx.x; pc < b.npieces; pc += gridDim.x) {
        const int4 piece = b.pieces[pc];
        const DevStream &D = b.ds[piece.x];
        const TickIO io = b.io[piece.x];
        if (io.frame == nullptr || D.mix.K != 0) continue;   // no frame this tick, or a mixture stream
        const uint32_t g = D.st->gain_p[b.phase];
        __syncthreads();   // the previous piece is done with the table
        fill_table(table, g);
        __syncthreads();
        const int w = D.w, cpr = 2 * D.nwords, fpitch = D.fpitch;
        const uint8_t *lo = D.lo, *hi = D.hi;
        uint32_t *raw = D.raw[b.phase];
        // warp-uniform loop so that chunk pairs can combine with a shuffle
        for (int base = piece.y + (tid & ~31); base < piece.z; base += blockDim.x) {
            const int u = base + lane;
            uint32_t bits = 0;
            uint32_t f[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) f[k] = 0u;
            int y = 0, j = 0;
            if (u < piece.z) {
                y = chunk_row((uint32_t)u, D.cpr_magic);
                j = u - y * cpr;
                const int x0 = j * kChunkPx;
                if (x0 < w && HMI_IN_BOUNDS(y < D.h && 3LL * (x0 + kChunkPx) <= io.frame_pitch &&
                                                3 * (x0 + kChunkPx) <= fpitch, &D.st->err)) {
                    uint32_t l[12], h[12];
                    load48(io.frame + (long long)y * io.frame_pitch + 3 * x0, once, f);
                    load48(lo + (long long)y * fpitch + 3 * x0, once, l);
                    load48(hi + (long long)y * fpitch + 3 * x0, once, h);
                    bits = band_outside16(f, l, h, TableCorr{table});
                    const int npx = w - x0;
                    if (npx < kChunkPx) bits &= (1u << npx) - 1u;
                }
            }
            // gray and hue tests of the warp's out-of-band pixels, then the AND
            bits &= ~skin_fail_warp(bits, f, D, table, skin[tid >> 5], lane);
            const uint32_t other = __shfl_xor_sync(kFull, bits, 1);
            if (u < piece.z && (u & 1) == 0 &&
                HMI_IN_BOUNDS(y < D.bh * kBlock && (j >> 1) < D.nwords, &D.st->err))
                raw[(long long)y * D.nwords + (j >> 1)] = bits | (other << 16);
        }
    }
}

// One thread per queued chunk: gray and hue tests on its out-of-band pixels;
// the pixels that fail are cleared from the raw mask word.
__global__ void __launch_bounds__(kThreads) k_skin(BatchDev b)
{
    const uint32_t n = *(volatile uint32_t *)b.skin_count;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += gridDim.x * blockDim.x) {
        const uint2 e = b.skin_list[it];
        const int sidx = (int)(e.x >> 16);
        const uint32_t bits = e.x & 0xffffu;
        const int u = (int)e.y;
        const DevStream &D = b.ds[sidx];
        const TickIO io = b.io[sidx];
        const uint32_t g = D.st->gain_p[b.phase];
        const int cpr = 2 * D.nwords;
        const int y = chunk_row((uint32_t)u, D.cpr_magic), j = u - y * cpr;
        const uint8_t *row = io.frame + (long long)y * io.frame_pitch + 3 * j * kChunkPx;
        uint32_t fail = 0;
        if (__popc(bits) > 4) {
            uint32_t f[12];
            const uint4 *q = reinterpret_cast<const uint4 *>(row);
            const uint4 a = __ldg(q), c = __ldg(q + 1), d = __ldg(q + 2);
            f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w;
            f[4] = c.x; f[5] = c.y; f[6] = c.z; f[7] = c.w;
            f[8] = d.x; f[9] = d.y; f[10] = d.z; f[11] = d.w;
#pragma unroll
            for (int k = 0; k < kChunkPx; ++k) {
                if (!((bits >> k) & 1u)) continue;
                if (!skin_rgb(byte_of(f, 3 * k), byte_of(f, 3 * k + 1), byte_of(f, 3 * k + 2), D, g))
                    fail |= 1u << k;
            }
        } else {
            for (uint32_t todo = bits; todo; todo &= todo - 1u) {
                const int k = __ffs(todo) - 1;
                const uint8_t *px = row + 3 * k;
                if (!skin_rgb(__ldg(px), __ldg(px + 1), __ldg(px + 2), D, g)) fail |= 1u << k;
            }
        }
        if (fail) atomicAnd(D.raw[b.phase] + (long long)y * D.nwords + (j >> 1), ~(fail << (16 * (j & 1))));
    }
}

// ---------------------------------------------------------------------------
// k_relearn: re-learning sums (Sec. 3.3, part of the learning restarted).
// In a window frame of a stream, every background pixel (all three gain-
// corrected channels inside the band: the test of k_classify) adds its
// corrected values to the stream's sums.  One thread per 16-px chunk, four
// pixels (12 values) at a time: value sums as 3 x 8 B (uint16), squares as
// 3 x 16 B, min and max as 3 x 4 B each, counts as 4 B.
// ---------------------------------------------------------------------------
template <int P>
__device__ __forceinline__ bool px_in_band(const uint32_t (&f)[12], const uint32_t (&l)[12],
                                           const uint32_t (&h)[12], uint32_t g)
{
    return in_band<3 * P>(f, l, h, g) & in_band<3 * P + 1>(f, l, h, g) & in_band<3 * P + 2>(f, l, h, g);
}

template <int K>
__device__ __forceinline__ uint32_t corrected(const uint32_t (&f)[12], uint32_t g)
{
    return (uint32_t)corr(__byte_perm(f[K >> 2], 0u, 0x4440u | (K & 3)), g);
}

// One value (index k of the group's 12) of a background pixel into the sums.
template <int KK, int k>
__device__ __forceinline__ void relearn_value(const uint32_t (&f)[12], uint32_t g, bool in,
                                              uint32_t (&S)[6], uint32_t (&Q)[12],
                                              uint32_t (&mn)[3], uint32_t (&mx)[3])
{
    const uint32_t v = corrected<KK>(f, g);
    const uint32_t sh = 8u * (k & 3);
    if (in) {
        S[k >> 1] += v << (16 * (k & 1));
        Q[k] += v * v;
        mn[k >> 2] = __vminu4(mn[k >> 2], (v << sh) | ~(0xffu << sh));
        mx[k >> 2] = __vmaxu4(mx[k >> 2], v << sh);
    }
}

template <int GQ>
__device__ __forceinline__ void relearn_quad(const DevStream &D, long long q0, int npx,
                                             const uint32_t (&f)[12], const uint32_t (&l)[12],
                                             const uint32_t (&h)[12], uint32_t g)
{
    if (4 * GQ >= npx) return;
    const bool in0 = px_in_band<4 * GQ>(f, l, h, g) && 4 * GQ < npx;
    const bool in1 = px_in_band<4 * GQ + 1>(f, l, h, g) && 4 * GQ + 1 < npx;
    const bool in2 = px_in_band<4 * GQ + 2>(f, l, h, g) && 4 * GQ + 2 < npx;
    const bool in3 = px_in_band<4 * GQ + 3>(f, l, h, g) && 4 * GQ + 3 < npx;
    if (!(in0 | in1 | in2 | in3)) return;
    const long long q = q0 + 4 * GQ;   // first pixel of the group, a multiple of 4
    uint2 *pS = reinterpret_cast<uint2 *>(D.rS + 3 * q);
    uint4 *pQ = reinterpret_cast<uint4 *>(D.rQ + 3 * q);
    uint32_t *pmn = reinterpret_cast<uint32_t *>(D.rmin + 3 * q);
    uint32_t *pmx = reinterpret_cast<uint32_t *>(D.rmax + 3 * q);
    uint32_t *pc = reinterpret_cast<uint32_t *>(D.rcnt + q);
    uint32_t S[6], Q[12], mn[3], mx[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const uint2 a = pS[i];
        const uint4 b = pQ[i];
        S[2 * i] = a.x;
        S[2 * i + 1] = a.y;
        Q[4 * i] = b.x;
        Q[4 * i + 1] = b.y;
        Q[4 * i + 2] = b.z;
        Q[4 * i + 3] = b.w;
        mn[i] = pmn[i];
        mx[i] = pmx[i];
    }
    relearn_value<12 * GQ + 0, 0>(f, g, in0, S, Q, mn, mx);
    relearn_value<12 * GQ + 1, 1>(f, g, in0, S, Q, mn, mx);
    relearn_value<12 * GQ + 2, 2>(f, g, in0, S, Q, mn, mx);
    relearn_value<12 * GQ + 3, 3>(f, g, in1, S, Q, mn, mx);
    relearn_value<12 * GQ + 4, 4>(f, g, in1, S, Q, mn, mx);
    relearn_value<12 * GQ + 5, 5>(f, g, in1, S, Q, mn, mx);
    relearn_value<12 * GQ + 6, 6>(f, g, in2, S, Q, mn, mx);
    relearn_value<12 * GQ + 7, 7>(f, g, in2, S, Q, mn, mx);
    relearn_value<12 * GQ + 8, 8>(f, g, in2, S, Q, mn, mx);
    relearn_value<12 * GQ + 9, 9>(f, g, in3, S, Q, mn, mx);
    relearn_value<12 * GQ + 10, 10>(f, g, in3, S, Q, mn, mx);
    relearn_value<12 * GQ + 11, 11>(f, g, in3, S, Q, mn, mx);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        pS[i] = make_uint2(S[2 * i], S[2 * i + 1]);
        pQ[i] = make_uint4(Q[4 * i], Q[4 * i + 1], Q[4 * i + 2], Q[4 * i + 3]);
        pmn[i] = mn[i];
        pmx[i] = mx[i];
    }
    *pc += (uint32_t)in0 | ((uint32_t)in1 << 8) | ((uint32_t)in2 << 16) | ((uint32_t)in3 << 24);
}

__global__ void __launch_bounds__(kThreads) k_relearn(BatchDev b)
{
    const uint64_t once = policy_evict_first();
    for (int pc = blockIdx.x; pc < b.npieces; pc += gridDim.x) {
        const int4 piece = b.pieces[pc];
        const DevStream &D = b.ds[piece.x];
        const TickIO io = b.io[piece.x];
        if (io.frame == nullptr || D.relearn_frames == 0) continue;
        if (!relearn_window(D.st->lframe_p[b.phase], D.relearn_period, D.relearn_frames)) continue;
        const uint32_t g = D.st->gain_p[b.phase];
        const int w = D.w, cpr = 2 * D.nwords, fpitch = D.fpitch;
        for (int u = piece.y + threadIdx.x; u < piece.z; u += blockDim.x) {
            const int y = chunk_row((uint32_t)u, D.cpr_magic), x0 = (u - y * cpr) * kChunkPx;
            if (x0 >= w) continue;
            uint32_t f[12], l[12], h[12];
            load48(io.frame + (long long)y * io.frame_pitch + 3 * x0, once, f);
            load48(D.lo + (long long)y * fpitch + 3 * x0, once, l);
            load48(D.hi + (long long)y * fpitch + 3 * x0, once, h);
            const int npx = min(kChunkPx, w - x0);
            const long long q0 = (long long)y * D.rpitch + x0;
            relearn_quad<0>(D, q0, npx, f, l, h, g);
            relearn_quad<1>(D, q0, npx, f, l, h, g);
            relearn_quad<2>(D, q0, npx, f, l, h, g);
            relearn_quad<3>(D, q0, npx, f, l, h, g);
        }
    }
}

template <int HR>
__global__ void __launch_bounds__(kStripWarps * 32, 5) k_morph_strip(BatchDev b)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t strip = blockIdx.x * kStripWarps + warp;
    if (strip >= b.total_strips) return;   // warp-uniform
    int lo = 0, hi = b.n;                   // largest s with strip_prefix[s] <= strip
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (b.strip_prefix[mid] <= strip) lo = mid; else hi = mid;
    }
    const DevStream &D = b.ds[lo];
    const TickIO io = b.io[lo];
    if (io.frame == nullptr) return;       // no frame for this stream this tick
    const int ls = (int)(strip - b.strip_prefix[lo]);
    const int ty = ls / D.strips_x, tx = ls - ty * D.strips_x;
    morph_strip<HR>(D, io, ty, tx, lane, lo, b.cc_count, b.cc_list, b.total_blocks, D.raw[b.phase]);
}

// ---------------------------------------------------------------------------
// k_stage (hmi_tuning.fused = 2): the per-pixel stage of a tick in one
// cooperative launch, whose CTAs are all resident at once: the luma sums of
// every piece, a grid barrier, the gain (each CTA forms it from the stream's
// complete sum) with the band, gray and hue tests of every piece, a second
// grid barrier, then the morphology strips.  Three phases in one launch
// instead of three launches: one ramp and one tail, which is what dominates
// a tick of one small stream.  Frame and raw-bit reads after a barrier go
// through L2 (other CTAs of the launch wrote them).  Every barrier wait is
// bounded (by kLoopLimit steps, not by a plan's lowered loop limit: a barrier
// that let CTAs through early would leave a stream's luma sum to the next
// tick); a wait that runs out flags the batch's error word and goes on.
// ---------------------------------------------------------------------------
constexpr uint32_t kErrStageWait = 16u;

__device__ __forceinline__ void load48_l2(const uint8_t *src, uint64_t pol, uint32_t (&w)[12])
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

// Every CTA of the launch arrives; thread 0 then waits (bounded) until
// `target` arrivals are counted at *ctr.
__device__ __forceinline__ void stage_barrier(uint32_t *ctr, uint32_t target, uint32_t limit, uint32_t *err)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        for (uint32_t it = 0;; ++it) {
            uint32_t v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (it >= limit) {
                atomicOr(err, kErrStageWait);
                break;
            }
            __nanosleep(it < 16 ? 32 : 128);
        }
    }
    __syncthreads();
}

// Q16 gain of a stream from its complete luma sum (the luma pass's formula).
__device__ __forceinline__ uint32_t stream_gain(const DevStream &D)
{
    const unsigned long long sy = __ldcg(&D.st->sy);
    const unsigned long long syref = D.st->syref;
    unsigned long long g = (sy == 0) ? 65536ull : ((syref << 16) + sy / 2) / sy;
    if (g < D.gain_min) g = D.gain_min;
    if (g > D.gain_max) g = D.gain_max;
    return (uint32_t)g;
}

template <int HR>
__global__ void __launch_bounds__(kThreads, 2) k_stage(BatchDev b)
{
    __shared__ unsigned long long red[kThreads / 32];
    __shared__ uint8_t table[256];
    __shared__ SkinSmem skin[kThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint64_t pol = policy_evict_first();
    const uint32_t limit = kLoopLimit;

    // 1. luma sums, a piece at a time
    for (int pc = blockIdx.x; pc < b.npieces; pc += gridDim.x) {
        const int4 piece = b.pieces[pc];
        const DevStream &D = b.ds[piece.x];
        const TickIO io = b.io[piece.x];
        if (io.frame == nullptr) continue;   // CTA-uniform
        const int w = D.w, cpr = 2 * D.nwords;
        unsigned long long acc = 0;
        for (int u = piece.y + tid; u < piece.z; u += kLumaChunks * kThreads) {
            uint32_t f[kLumaChunks][12];
            int npx[kLumaChunks];
#pragma unroll
            for (int q = 0; q < kLumaChunks; ++q) {
                const int uu = u + q * kThreads;
                npx[q] = 0;
                if (uu < piece.z) {
                    const int y = chunk_row((uint32_t)uu, D.cpr_magic), x0 = (uu - y * cpr) * kChunkPx;
                    if (x0 < w && HMI_IN_BOUNDS(y < D.h && 3LL * (x0 + kChunkPx) <= io.frame_pitch, &D.st->err)) {
                        npx[q] = min(kChunkPx, w - x0);
                        if (io.src) {   // a pinned host frame: w is a multiple of 16, rows dense
                            load48_host(io.src + (long long)y * 3 * w + 3 * x0, f[q]);
                            store48(const_cast<uint8_t *>(io.frame) + (long long)y * io.frame_pitch + 3 * x0, f[q]);
                        } else {
                            load48(io.frame + (long long)y * io.frame_pitch + 3 * x0, pol, f[q]);
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kLumaChunks; ++q)
                if (npx[q] > 0) acc += (npx[q] == kChunkPx) ? luma_sum16(f[q]) : luma_sum_n(f[q], npx[q]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (tid == 0) {
            unsigned long long t = 0;
            for (int i = 0; i < kThreads / 32; ++i) t += red[i];
            atomicAdd(&D.st->sy, t);
        }
        __syncthreads();
    }
    stage_barrier(b.done + 2, gridDim.x, limit, b.err);

    // 2. gain, band test, gray and hue tests, AND: raw mask bits
    for (int pc = blockIdx.x; pc < b.npieces; pc += gridDim.x) {
        const int4 piece = b.pieces[pc];
        const DevStream &D = b.ds[piece.x];
        const TickIO io = b.io[piece.x];
        if (io.frame == nullptr) continue;   // CTA-uniform
        const uint32_t g = stream_gain(D);
        __syncthreads();   // the previous piece is done with the table
        fill_table(table, g);
        __syncthreads();
        const int w = D.w, cpr = 2 * D.nwords, fpitch = D.fpitch;
        uint32_t *raw = D.raw[b.phase];
        for (int base = piece.y + (tid & ~31); base < piece.z; base += kThreads) {   // warp-uniform
            const int u = base + lane;
            uint32_t bits = 0;
            uint32_t f[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) f[k] = 0u;
            int y = 0, j = 0;
            if (u < piece.z) {
                y = chunk_row((uint32_t)u, D.cpr_magic);
                j = u - y * cpr;
                const int x0 = j * kChunkPx;
                if (x0 < w && HMI_IN_BOUNDS(y < D.h && 3LL * (x0 + kChunkPx) <= io.frame_pitch &&
                                                3 * (x0 + kChunkPx) <= fpitch, &D.st->err)) {
                    uint32_t l[12], h[12];
                    load48_l2(io.frame + (long long)y * io.frame_pitch + 3 * x0, pol, f);
                    load48(D.lo + (long long)y * fpitch + 3 * x0, pol, l);
                    load48(D.hi + (long long)y * fpitch + 3 * x0, pol, h);
                    bits = band_outside16(f, l, h, TableCorr{table});
                    const int npx = w - x0;
                    if (npx < kChunkPx) bits &= (1u << npx) - 1u;
                }
            }
            bits &= ~skin_fail_warp(bits, f, D, table, skin[warp], lane);
            const uint32_t other = __shfl_xor_sync(kFull, bits, 1);
            if (u < piece.z && (u & 1) == 0 &&
                HMI_IN_BOUNDS(y < D.bh * kBlock && (j >> 1) < D.nwords, &D.st->err))
                raw[(long long)y * D.nwords + (j >> 1)] = bits | (other << 16);
        }
    }
    stage_barrier(b.done + 2, 2u * gridDim.x, limit, b.err);

    // every luma sum has been read: the gains into the streams' state
    if (blockIdx.x == 0) {
        for (int s = tid; s < b.n; s += kThreads) {
            if (b.io[s].frame == nullptr) continue;
            const DevStream &D = b.ds[s];
            StreamState *st = D.st;
            const uint32_t g = stream_gain(D);
            st->gain = g;
            st->gain_p[b.phase] = g;
            st->sy = 0;
            st->lframes += 1;
            st->lframe_p[b.phase] = st->lframes;
        }
    }

    // 3. opening and closing of the raw bits, strip by strip (a warp each)
    for (uint32_t strip = blockIdx.x * (kThreads / 32) + warp; strip < b.total_strips;
         strip += gridDim.x * (kThreads / 32)) {   // warp-uniform
        int lo = 0, hi = b.n;                   // largest s with strip_prefix[s] <= strip
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (b.strip_prefix[mid] <= strip) lo = mid; else hi = mid;
        }
        const DevStream &D = b.ds[lo];
        const TickIO io = b.io[lo];
        if (io.frame == nullptr) continue;
        const int ls = (int)(strip - b.strip_prefix[lo]);
        const int ty = ls / D.strips_x, tx = ls - ty * D.strips_x;
        morph_strip<HR>(D, io, ty, tx, lane, lo, b.cc_count, b.cc_list, b.total_blocks, D.raw[b.phase]);
    }

    // the last CTA out resets the barrier counter for the next tick
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(b.done + 3, 1u) == gridDim.x - 1u) {
            b.done[2] = 0u;
            b.done[3] = 0u;
        }
    }
}

// k_block_cc: one warp per listed non-empty 32x32 block (any stream of the
// batch): its 8-connected components and their statistics; its flag is
// cleared for the next tick.
constexpr int kBlockCcWarps = 8;

__global__ void __launch_bounds__(kBlockCcWarps * 32) k_block_cc(BatchDev b)
{
    const int lane = threadIdx.x & 31;
    const uint32_t n = *(volatile uint32_t *)b.cc_count;
    for (uint32_t it = blockIdx.x * kBlockCcWarps + (threadIdx.x >> 5); it < n;
         it += gridDim.x * kBlockCcWarps) {
        const uint2 e = b.cc_list[it];
        if (!HMI_IN_BOUNDS(e.x < (uint32_t)b.n, b.err)) continue;   // warp-uniform
        const DevStream &D = b.ds[e.x];
        const int by = (int)e.y / D.nwords, bx = (int)e.y - by * D.nwords;
        const uint32_t m = __ldcg(D.bits + (long long)(by * kBlock + lane) * D.nwords + bx);
        if (lane == 0) D.flag[e.y] = 0u;
        emit_block_components(D, m, lane, (int)e.y, bx * kWordPx, by * kBlock);
    }
}

// ---------------------------------------------------------------------------
// k_morph_cc: one CTA per tile of 32 rows x kMorphTW words.
// ---------------------------------------------------------------------------
constexpr int kMR = kMorphRows + 2 * kMaxHalo;   // buffer rows
constexpr int kMW = kMorphTW + 2;                // buffer words (one halo word each side)

struct MorphGeo {
    int y0, k0, HR, R, h, w, nwords;
    uint32_t lastmask;
    __device__ uint32_t valid(int r, int k) const
    {
        const int y = y0 - HR + r, kw = k0 - 1 + k;
        if (y < 0 || y >= h || kw < 0 || kw >= nwords) return 0u;
        return (kw == nwords - 1) ? lastmask : 0xffffffffu;
    }
};

__global__ void __launch_bounds__(kThreads) k_morph_cc(BatchDev b)
{
    __shared__ uint32_t buf[2][kMR][kMW];
    __shared__ int s_sh;
    const int tid = threadIdx.x;
    const unsigned tile = blockIdx.x;
    if (tid == 0) {
        int lo = 0, hi = b.n;   // largest s with tile_prefix[s] <= tile
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (b.tile_prefix[mid] <= tile) lo = mid; else hi = mid;
        }
        s_sh = lo;
    }
    __syncthreads();
    const int s = s_sh;
    const DevStream &D = b.ds[s];
    const TickIO io = b.io[s];
    if (io.frame == nullptr) return;       // CTA-uniform: no frame this tick
    const int lt = (int)(tile - b.tile_prefix[s]);
    const int ty = lt / D.tiles_x, tx = lt - ty * D.tiles_x;
    MorphGeo G;
    G.HR = 2 * (D.open_iters + D.close_iters);
    G.R = kMorphRows + 2 * G.HR;
    G.y0 = ty * kMorphRows;
    G.k0 = tx * kMorphTW;
    G.h = D.h;
    G.w = D.w;
    G.nwords = D.nwords;
    G.lastmask = (D.w & 31) ? ((1u << (D.w & 31)) - 1u) : 0xffffffffu;
    const int ncell = G.R * kMW;

    for (int i = tid; i < ncell; i += blockDim.x) {
        const int r = i / kMW, k = i - r * kMW;
        const int y = G.y0 - G.HR + r, kw = G.k0 - 1 + k;
        buf[0][r][k] = (y >= 0 && y < G.h && kw >= 0 && kw < G.nwords) ? D.raw[b.phase][(long long)y * G.nwords + kw] : 0u;
    }
    __syncthreads();

    // open_iters x (erode, dilate), then close_iters x (dilate, erode);
    // out-of-image pixels are neutral for each operator
    const int nops = 2 * (D.open_iters + D.close_iters);
    int cur = 0;
    for (int op = 0; op < nops; ++op) {
        const bool ero = (op < 2 * D.open_iters) ? ((op & 1) == 0) : (((op - 2 * D.open_iters) & 1) == 1);
        for (int i = tid; i < ncell; i += blockDim.x) {
            const int r = i / kMW, k = i - r * kMW;
            uint32_t acc = ero ? 0xffffffffu : 0u;
#pragma unroll
            for (int dr = -1; dr <= 1; ++dr) {
                const int rr = r + dr;
                uint32_t v[3];
#pragma unroll
                for (int dk = -1; dk <= 1; ++dk) {
                    const int kk = k + dk;
                    uint32_t x;
                    if (rr < 0 || rr >= G.R || kk < 0 || kk >= kMW) {
                        x = ero ? 0xffffffffu : 0u;
                    } else {
                        const uint32_t vm = G.valid(rr, kk);
                        const uint32_t raw = buf[cur][rr][kk];
                        x = ero ? (raw | ~vm) : (raw & vm);
                    }
                    v[dk + 1] = x;
                }
                if (ero) {
                    acc &= v[1] & ((v[1] << 1) | (v[0] >> 31)) & ((v[1] >> 1) | (v[2] << 31));
                } else {
                    acc |= v[1] | (v[1] << 1) | (v[0] >> 31) | (v[1] >> 1) | (v[2] << 31);
                }
            }
            buf[cur ^ 1][r][k] = acc;
        }
        __syncthreads();
        cur ^= 1;
    }

    // final bits of the tile interior: global bit mask, mask bytes, and a
    // copy in the other buffer for the component pass
    uint32_t (*fin)[kMW] = buf[cur ^ 1];
    for (int i = tid; i < kMorphRows * kMorphTW; i += blockDim.x) {
        const int r = i / kMorphTW, k = i - r * kMorphTW;
        const int rb = G.HR + r, kb = 1 + k;
        const uint32_t v = buf[cur][rb][kb] & G.valid(rb, kb);
        fin[r][k] = v;
        const int y = G.y0 + r, kw = G.k0 + k;
        if (kw < G.nwords) {
            D.bits[(long long)y * G.nwords + kw] = v;
            if (io.mask != nullptr && y < G.h) {
                uint8_t *dst = io.mask + (long long)y * G.w + kw * kWordPx;
                const int npx = min(kWordPx, G.w - kw * kWordPx);
                if (npx == kWordPx && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
                    uint32_t q[8];
#pragma unroll
                    for (int n4 = 0; n4 < 8; ++n4) q[n4] = (((v >> (4 * n4)) & 0xfu) * 0x00204081u) & 0x01010101u;
                    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
                    __stcs(d4, make_uint4(q[0], q[1], q[2], q[3]));
                    __stcs(d4 + 1, make_uint4(q[4], q[5], q[6], q[7]));
                } else {
                    for (int x = 0; x < npx; ++x) dst[x] = (uint8_t)((v >> x) & 1u);
                }
            }
        }
    }
    __syncthreads();

    // 8-connected components of each 32x32 block of the tile (one warp each)
    const int wid = tid >> 5, lane = tid & 31;
    for (int k = wid; k < kMorphTW; k += blockDim.x >> 5) {
        const int kw = G.k0 + k;
        if (kw >= G.nwords) continue;
        emit_block_components(D, fin[lane][k], lane, ty * G.nwords + kw, kw * kWordPx, G.y0);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_for_pieces(int npieces)
{
    return npieces > 0 ? npieces : 1;
}

// CTAs of `kernel` that fit on one SM at once (queried once per device).
template <typename K>
static int resident_ctas(K kernel, int threads, int *cache)
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, 0) != cudaSuccess || n < 1) {
            (void)cudaGetLastError();
            n = 1;
        }
        cache[dev] = n;
    }
    return cache[dev];
}

cudaError_t launch_luma(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    static int per_sm[64];
    const int fit = resident_ctas(k_luma, kThreads, per_sm);
    const int per = b.luma_ctas_per_sm > 0 ? std::min(b.luma_ctas_per_sm, fit) : fit;
    const int grid = std::max(1, std::min(b.npieces, num_sms * per));
    k_luma<<<grid, kThreads, 0, cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_classify(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    (void)num_sms;   // one CTA per piece: CTAs of the tail kernels of the previous
    if (!b.any_band) return cudaSuccess;   // tick find SMs as pieces finish
    k_classify<<<grid_for_pieces(b.npieces), kThreads, 0, cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_relearn(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    (void)num_sms;
    if (!b.relearn) return cudaSuccess;
    k_relearn<<<grid_for_pieces(b.npieces), kThreads, 0, cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_skin(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    if (!b.any_mix) return cudaSuccess;   // band streams are tested in k_classify
    k_skin<<<num_sms * std::max(1, b.skin_ctas_per_sm), kThreads, 0, cs>>>(b);
    return cudaGetLastError();
}

static bool strip_path(const BatchDev &b)
{
    return b.uniform_halo >= 0 && b.uniform_halo <= kStripMaxHalo;
}

cudaError_t launch_morph(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    (void)num_sms;
    if (strip_path(b)) {
        const unsigned grid = (b.total_strips + kStripWarps - 1) / kStripWarps;
        switch (b.uniform_halo) {
        case 0: k_morph_strip<0><<<grid, kStripWarps * 32, 0, cs>>>(b); break;
        case 2: k_morph_strip<2><<<grid, kStripWarps * 32, 0, cs>>>(b); break;
        case 4: k_morph_strip<4><<<grid, kStripWarps * 32, 0, cs>>>(b); break;
        case 6: k_morph_strip<6><<<grid, kStripWarps * 32, 0, cs>>>(b); break;
        default: k_morph_strip<8><<<grid, kStripWarps * 32, 0, cs>>>(b); break;
        }
    } else {
        k_morph_cc<<<b.total_tiles, kThreads, 0, cs>>>(b);
    }
    return cudaGetLastError();
}

// The cooperative per-pixel stage: as many CTAs as are resident at once (or
// as there are pieces or strip groups, if fewer), launched so that the CUDA
// driver guarantees they all run together.
template <int HR>
static cudaError_t launch_stage_hr(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    static int fit[64];
    const int per_fit = resident_ctas(k_stage<HR>, kThreads, fit);
    const int per = b.luma_ctas_per_sm > 0 ? std::min(b.luma_ctas_per_sm, per_fit) : per_fit;
    const long long work = std::max<long long>(b.npieces, ((long long)b.total_strips + 7) / 8);
    const int grid = (int)std::max<long long>(1, std::min<long long>((long long)num_sms * per, work));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = cs;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_stage<HR>, b);
}

static cudaError_t launch_stage(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    switch (b.uniform_halo) {   // the plan keeps this form to halos of the strip path
    case 0: return launch_stage_hr<0>(b, cs, num_sms);
    case 2: return launch_stage_hr<2>(b, cs, num_sms);
    case 4: return launch_stage_hr<4>(b, cs, num_sms);
    case 6: return launch_stage_hr<6>(b, cs, num_sms);
    default: return launch_stage_hr<8>(b, cs, num_sms);
    }
}

cudaError_t launch_block_cc(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    if (!strip_path(b)) return cudaSuccess;   // k_morph_cc labels its blocks itself
    const unsigned g2 = std::min<unsigned>((b.total_blocks + kBlockCcWarps - 1) / kBlockCcWarps,
                                           (unsigned)num_sms * (unsigned)std::max(1, b.cc_ctas_per_sm));
    k_block_cc<<<std::max(g2, 1u), kBlockCcWarps * 32, 0, cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_tick_kernel(int k, const BatchDev &b, cudaStream_t cs, int num_sms)
{
    if (b.fused == 2) {   // one cooperative launch does kernels 0, 1, 5 and 6
        switch (k) {
        case 0: return launch_stage(b, cs, num_sms);
        case 3: return launch_relearn(b, cs, num_sms);
        case 4: return launch_relearn_band(b, cs, num_sms);
        case 7: return launch_block_cc(b, cs, num_sms);
        case 8: return launch_finish(b, cs);
        default: return cudaSuccess;
        }
    }
    if (b.fused) {   // one persistent launch does the per-pixel work of kernels 0, 1, 5 and 6
        switch (k) {
        case 0: return launch_tick(b, cs, num_sms);
        case 3: return launch_relearn(b, cs, num_sms);
        case 4: return launch_relearn_band(b, cs, num_sms);
        case 7: return launch_block_cc(b, cs, num_sms);
        case 8: return launch_finish(b, cs);
        default: return cudaSuccess;
        }
    }
    switch (k) {
    case 0: return launch_luma(b, cs, num_sms);
    case 1: return launch_classify(b, cs, num_sms);
    case 2: return launch_mix(b, cs, num_sms);
    case 3: return launch_relearn(b, cs, num_sms);
    case 4: return launch_relearn_band(b, cs, num_sms);
    case 5: return launch_skin(b, cs, num_sms);
    case 6: return launch_morph(b, cs, num_sms);
    case 7: return launch_block_cc(b, cs, num_sms);
    default: return launch_finish(b, cs);
    }
}

}  // namespace hmi
