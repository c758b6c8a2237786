// hmi_pixel.cuh -- per-pixel device helpers shared by the kernels of a tick
// (hmi_frame.cu) and the persistent tick kernel (hmi_tick.cu): vector loads of
// frame and band chunks with L2 eviction hints, the integer luma of the
// brightness correction (Sec. 2, Sec. 3.2), the background band test
// (Sec. 3.1 (i)), the gray and hue tests (Sec. 3.1 (ii), (iii)) and the
// component enumeration of a 32x32 block (Mouse module, Sec. 2).
#pragma once

#include <stdint.h>

#include "hmi_band.h"
#include "hmi_ccfill.cuh"
#include "hmi_internal.cuh"

namespace hmi {

// L2 eviction policy of the per-pixel streams: every frame, band and mask read
// is evict-first.  (Keeping the luma pass's frame evict-last for the band test
// made the luma pass ~15 % slower and the pipelined tick ~3 % slower: the next
// tick's frame then competes for L2 with the band stream.)
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint4 ld_hint(const uint4 *ptr, uint64_t pol)
{
    uint4 r;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(ptr), "l"(pol));
    return r;
}

__device__ __forceinline__ void load48(const uint8_t *src, uint64_t pol, uint32_t (&w)[12])
{
    const uint4 *q = reinterpret_cast<const uint4 *>(src);
    const uint4 a = ld_hint(q, pol), b = ld_hint(q + 1, pol), c = ld_hint(q + 2, pol);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    w[8] = c.x; w[9] = c.y; w[10] = c.z; w[11] = c.w;
}

// 48 bytes of a pinned host frame (read once over the host link, through the
// non-coherent path, no L2 policy), and their store into the staging frame.
__device__ __forceinline__ void load48_host(const uint8_t *src, uint32_t (&w)[12])
{
    const uint4 *q = reinterpret_cast<const uint4 *>(src);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint4 r;
        asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(q + k));
        w[4 * k] = r.x; w[4 * k + 1] = r.y; w[4 * k + 2] = r.z; w[4 * k + 3] = r.w;
    }
}

__device__ __forceinline__ void store48(uint8_t *dst, const uint32_t (&w)[12])
{
    uint4 *q = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int k = 0; k < 3; ++k) q[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
}

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[12], int b)
{
    return __byte_perm(w[b >> 2], 0u, 0x4440u | (uint32_t)(b & 3));
}

// Integer BT.601 luma, (77 R + 150 G + 29 B + 128) >> 8.
__device__ __forceinline__ uint32_t luma8(uint32_t r, uint32_t g, uint32_t b)
{
    return (77u * r + 150u * g + 29u * b + 128u) >> 8;
}

// Sum of luma8 over 16 pixels (48 bytes): each pixel's 3 bytes are gathered
// into one word with a byte permute, then one 4-way byte dot product with
// (77, 150, 29, 0) plus 128, shifted per pixel.
__device__ __forceinline__ uint32_t luma_sum16(const uint32_t (&f)[12])
{
    constexpr uint32_t kW = 77u | (150u << 8) | (29u << 16);
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kChunkPx; ++k) {
        const int b = 3 * k, wi = b >> 2, o = b & 3;
        // bytes b, b+1, b+2 of the 48 (they span at most two words)
        const uint32_t lo = f[wi], hi = (wi + 1 < 12) ? f[wi + 1] : 0u;
        const uint32_t px = __byte_perm(lo, hi, (uint32_t)(o | ((o + 1) << 4) | ((o + 2) << 8) | (0x7 << 12)) & 0x7777u);
        sum += __dp4a(px & 0x00ffffffu, kW, 128u) >> 8;
    }
    return sum;
}

__device__ __forceinline__ uint32_t luma_sum_n(const uint32_t (&f)[12], int npx)
{
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < kChunkPx; ++k) {
        const uint32_t v = luma8(byte_of(f, 3 * k), byte_of(f, 3 * k + 1), byte_of(f, 3 * k + 2));
        sum += (k < npx) ? v : 0u;
    }
    return sum;
}

// ---------------------------------------------------------------------------
// Gain correction, band test, gray and hue tests
// ---------------------------------------------------------------------------
// Gain-corrected channel: c' = min(255, (c g + 2^15) >> 16).
__device__ __forceinline__ int corr(uint32_t c, uint32_t g)
{
    return (int)min((c * g + 32768u) >> 16, 255u);
}

// Background test of one pixel (Sec. 3.1 (i)): 1 iff some gain-corrected
// channel lies outside the learned band [lo, hi].  Compared in the scaled
// domain: with Y = min(c g + 2^15, 255 * 2^16 + 2^15),
//   c' >= lo  <=>  Y >= lo << 16      and      c' <= hi  <=>  Y <= (hi << 16) | 0xffff,
// where byte permutes place lo / hi straight into bits 16..23.
template <int K>
__device__ __forceinline__ bool in_band(const uint32_t (&f)[12], const uint32_t (&l)[12],
                                        const uint32_t (&h)[12], uint32_t g)
{
    constexpr int W = K >> 2, B = K & 3;
    const uint32_t c = __byte_perm(f[W], 0u, 0x4440u | B);
    const uint32_t y = min(c * g + 32768u, 255u * 65536u + 32768u);
    const uint32_t lo16 = __byte_perm(l[W], 0u, 0x4044u | (B << 8));
    const uint32_t hi16 = __byte_perm(h[W], 0x0000ffffu, 0x6054u | (B << 8));
    return (y >= lo16) & (y <= hi16);
}

template <int k>
__device__ __forceinline__ uint32_t outside_band(const uint32_t (&f)[12], const uint32_t (&l)[12],
                                                 const uint32_t (&h)[12], uint32_t g)
{
    const bool in = in_band<3 * k>(f, l, h, g) & in_band<3 * k + 1>(f, l, h, g) &
                    in_band<3 * k + 2>(f, l, h, g);
    return in ? 0u : (1u << k);
}

template <int k>
__device__ __forceinline__ uint32_t outside_bits(const uint32_t (&f)[12], const uint32_t (&l)[12],
                                                 const uint32_t (&h)[12], uint32_t g)
{
    if constexpr (k == 0) {
        return outside_band<0>(f, l, h, g);
    } else {
        return outside_band<k>(f, l, h, g) | outside_bits<k - 1>(f, l, h, g);
    }
}

// The frame's table of corrected values (shared memory) as the word
// correction of the packed band test (hmi_band.h).
struct TableCorr {
    const uint8_t *t;
    __device__ __forceinline__ uint32_t operator()(uint32_t w) const { return corrected_word(w, t); }
};

// Fill the CTA's table of corrected values for gain g (blockDim.x >= 256);
// the caller synchronises before and after.
__device__ __forceinline__ void fill_table(uint8_t *table, uint32_t g)
{
    if (threadIdx.x < 256) table[threadIdx.x] = (uint8_t)corrected_value(threadIdx.x, g);
}

// Gray and hue tests of one pixel (Sec. 3.1 (ii), (iii)) on the corrected
// values: not gray (max - min >= S) and hue inside the arc.  The hue test
// compares N = 512 (t + d) + d against d-scaled interval ends, which equals
// testing h = base - 256 + floor(N / 2d) without a division.
__device__ __forceinline__ bool skin_corrected(int r, int g, int b, const DevStream &D)
{
    const int mx = max(r, max(g, b));
    const int mn = min(r, min(g, b));
    const int d = mx - mn;
    int t, sec;
    if (r == mx) {
        t = g - b; sec = 0;
    } else if (g == mx) {
        t = b - r; sec = 1;
    } else {
        t = r - g; sec = 2;
    }
    const int N = 512 * (t + d) + d;
    const bool hue = ((N >= d * D.hueA[sec][0]) & (N < d * D.hueB[sec][0])) |
                     ((N >= d * D.hueA[sec][1]) & (N < d * D.hueB[sec][1]));
    return (d > 0) & (d >= D.gray_tol) & hue;
}

__device__ __forceinline__ bool skin_rgb(uint32_t r0, uint32_t g0, uint32_t b0, const DevStream &D,
                                         uint32_t gain)
{
    return skin_corrected(corr(r0, gain), corr(g0, gain), corr(b0, gain), D);
}

// ---------------------------------------------------------------------------
// Block components: one warp, lane r holds row r of the 32x32 block `blk`
// (columns xb.., rows yb..).  Components are enumerated in raster order of
// their first pixel and written to the block's record slots with their area,
// coordinate sums, box, smallest pixel index and border pixels.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void emit_block_components(const DevStream &D, uint32_t m, int lane,
                                                      int blk, int xb, int yb)
{
    if (!HMI_IN_BOUNDS((uint32_t)blk < (uint32_t)(D.bh * D.nwords), &D.st->err)) return;   // warp-uniform
    Comp *out = D.comp + (long long)blk * kSlots;
    uint32_t *parent = D.parent + (long long)blk * kSlots;
    int ncomp = 0;
    while (__any_sync(kFull, m != 0u)) {
        int r0, c0;
        const uint32_t c = cc_extract_first(m, lane, &r0, &c0);
        m &= ~c;
        const uint32_t pc = (uint32_t)__popc(c);
        const uint32_t area = __reduce_add_sync(kFull, pc);
        const uint32_t sx = __reduce_add_sync(kFull, pc * (uint32_t)xb + bit_index_sum(c));
        const uint32_t sy = __reduce_add_sync(kFull, pc * (uint32_t)(yb + lane));
        const unsigned rows = __ballot_sync(kFull, c != 0u);
        const uint32_t xmin = __reduce_min_sync(kFull, c ? (uint32_t)(__ffs(c) - 1) : 32u);
        const uint32_t xmax = __reduce_max_sync(kFull, c ? (uint32_t)(31 - __clz(c)) : 0u);
        const uint32_t top = __shfl_sync(kFull, c, 0);
        const uint32_t bot = __shfl_sync(kFull, c, 31);
        const uint32_t left = __ballot_sync(kFull, c & 1u);
        const uint32_t right = __ballot_sync(kFull, c >> 31);
        if (ncomp < kSlots) {
            uint32_t *o = reinterpret_cast<uint32_t *>(out + ncomp);
            uint32_t val = 0;
            switch (lane) {
            case 0: val = (uint32_t)(yb + r0) * (uint32_t)D.w + (uint32_t)(xb + c0); break;
            case 1: val = area; break;
            case 2: val = sx; break;
            case 4: val = sy; break;
            case 6: val = (uint32_t)xb + xmin; break;
            case 7: val = (uint32_t)(yb + __ffs(rows) - 1); break;
            case 8: val = (uint32_t)xb + xmax; break;
            case 9: val = (uint32_t)(yb + 31 - __clz(rows)); break;
            case 10: val = top; break;
            case 11: val = bot; break;
            case 12: val = left; break;
            case 13: val = right; break;
            default: val = 0; break;
            }
            if (lane < 16) o[lane] = val;
            if (lane == 0) parent[ncomp] = (uint32_t)ncomp + (uint32_t)blk * kSlots;
        }
        ++ncomp;
    }
    if (lane == 0) {
        if (ncomp > kSlots) atomicOr(&D.st->err, kErrSlots);
        D.count[blk] = (uint32_t)min(ncomp, kSlots);
    }
}

struct __align__(16) SkinSmem {   // per warp: the classify item's gray / hue queue
    uint32_t f[32][12];           // frame words of the lanes' chunks
    uint16_t list[32 * kChunkPx]; // queued pixels: lane << 4 | pixel
    uint32_t fail[32];            // pixels of each lane's chunk that fail
};

// Gray and hue tests of a warp's out-of-band pixels, on corrected values from
// the frame's table.  When the candidates are spread over the lanes (camera
// noise: a pixel or two per chunk), each lane tests its own; when a few lanes
// hold most of them (the hand), the warp lists them (lane << 4 | pixel) in
// shared memory and every lane takes pixels in turn, so that a chunk with
// many candidate pixels does not stall the warp behind one lane.  Returns this
// lane's pixels that fail.
__device__ __forceinline__ uint32_t skin_fail_warp(uint32_t bits, const uint32_t (&f)[12],
                                                   const DevStream &D, const uint8_t *table,
                                                   SkinSmem &S, int lane)
{
    const uint32_t cnt = (uint32_t)__popc(bits);
    const uint32_t total = __reduce_add_sync(kFull, cnt);
    if (total == 0u) return 0u;
    const uint32_t most = __reduce_max_sync(kFull, cnt);
    if (bits) {
        uint4 *dst = reinterpret_cast<uint4 *>(S.f[lane]);
        dst[0] = make_uint4(f[0], f[1], f[2], f[3]);
        dst[1] = make_uint4(f[4], f[5], f[6], f[7]);
        dst[2] = make_uint4(f[8], f[9], f[10], f[11]);
    }
    if (most <= (total + 31u) / 32u + 1u) {   // warp-uniform: each lane its own pixels
        const uint8_t *row = reinterpret_cast<const uint8_t *>(S.f[lane]);
        uint32_t fail = 0;
        for (uint32_t m = bits; m; m &= m - 1u) {
            const int k = __ffs(m) - 1;
            const uint8_t *px = row + 3 * k;
            if (!skin_corrected(table[px[0]], table[px[1]], table[px[2]], D)) fail |= 1u << k;
        }
        __syncwarp();   // S.f is free again
        return fail;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t pos = incl - cnt;
    for (uint32_t m = bits; m; m &= m - 1u)
        if (HMI_IN_BOUNDS(pos < 32u * kChunkPx, &D.st->err))
            S.list[pos++] = (uint16_t)((lane << 4) | (__ffs(m) - 1));
    S.fail[lane] = 0u;
    __syncwarp();
    for (uint32_t i = (uint32_t)lane; i < total; i += 32u) {
        const uint32_t e = S.list[i];
        const int ln = (int)(e >> 4), k = (int)(e & 15u);
        const uint8_t *px = reinterpret_cast<const uint8_t *>(S.f[ln]) + 3 * k;
        if (!skin_corrected(table[px[0]], table[px[1]], table[px[2]], D)) atomicOr(&S.fail[ln], 1u << k);
    }
    __syncwarp();
    const uint32_t fail = S.fail[lane];
    __syncwarp();
    return fail;
}

// ---------------------------------------------------------------------------
// k_morph_strip: one warp per strip of kStripRows output rows x 30 words (960 px),
// lane j = word column (lanes 0 and 31 are the left/right halo words), rows
// (32 + 2*HR with HR = 2*(open+close) halo rows) held in registers.  Each
// operator neutralises out-of-image pixels (1 for erosion, 0 for dilation),
// forms the horizontal 3-pixel AND/OR with the neighbour lanes' words, then
// the vertical 3-row AND/OR.  Garbage from the strip's own edges moves one
// pixel per operator and never reaches the interior (HR rows, 32 - HR bits).
// ---------------------------------------------------------------------------
constexpr int kStripWords = 30;
constexpr int kStripWarps = 4;


// One 3x3 erosion (ERO) or dilation of the strip's R rows of one word column
// (lane), out-of-image pixels made neutral first when the strip touches an
// image edge.  A compile-time operator, so that each row step is one
// expression; the caller's loop over operators stays a loop, which keeps the
// kernel small enough for the instruction cache.
template <bool ERO, int R>
__device__ __forceinline__ void morph_pass(uint32_t (&v)[R], bool edge, int rlo, int rhi, uint32_t wmask)
{
    if (edge) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t vm = (r >= rlo && r < rhi) ? wmask : 0u;
            v[r] = ERO ? (v[r] | ~vm) : (v[r] & vm);
        }
    }
    uint32_t prev = 0, cur = 0;
#pragma unroll
    for (int r = 0; r <= R; ++r) {
        uint32_t nxt = cur;
        if (r < R) {
            const uint32_t x = v[r];
            const uint32_t L = __shfl_up_sync(kFull, x, 1);
            const uint32_t Rt = __shfl_down_sync(kFull, x, 1);
            nxt = ERO ? (x & ((x << 1) | (L >> 31)) & ((x >> 1) | (Rt << 31)))
                      : (x | (x << 1) | (L >> 31) | (x >> 1) | (Rt << 31));
        }
        if (r == 1) {
            v[0] = ERO ? (cur & nxt) : (cur | nxt);
        } else if (r >= 2) {
            v[r - 1] = ERO ? (prev & cur & nxt) : (prev | cur | nxt);
        }
        prev = cur;
        cur = nxt;
    }
}

template <int HR>
__device__ __forceinline__ void morph_strip(const DevStream &D, const TickIO &io, int ty, int tx,
                                            int lane, int sidx, uint32_t *cc_count, uint2 *cc_list,
                                            uint32_t cc_cap, const uint32_t *raw)
{
    constexpr int R = kStripRows + 2 * HR;
    const int w = D.w, h = D.h, nwords = D.nwords;
    const int kw = tx * kStripWords - 1 + lane;
    const bool col_ok = kw >= 0 && kw < nwords;
    const uint32_t wmask = !col_ok ? 0u : ((kw == nwords - 1 && (w & 31)) ? ((1u << (w & 31)) - 1u) : 0xffffffffu);
    const int y0 = ty * kStripRows;
    const int ybase = y0 - HR;
    const int rlo = max(0, -ybase), rhi = min(R, h - ybase);   // rows inside the image
    uint32_t v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = ybase + r;
        // at L2: in the persistent tick the raw bits come from other CTAs of the launch
        v[r] = (col_ok && r >= rlo && r < rhi) ? __ldcg(raw + (long long)y * nwords + kw) : 0u;
    }
    // strips away from every image edge need no neutral out-of-image pixels
    const bool edge = rlo > 0 || rhi < R || __any_sync(kFull, wmask != 0xffffffffu);
    // open_iters x (erode, dilate), then close_iters x (dilate, erode)
    const int open2 = 2 * D.open_iters;
#pragma unroll 1
    for (int op = 0; op < HR; ++op) {   // HR == 2 (open + close) operators
        const bool ero = (op < open2) ? ((op & 1) == 0) : (((op - open2) & 1) == 1);
        if (ero) morph_pass<true>(v, edge, rlo, rhi, wmask);
        else morph_pass<false>(v, edge, rlo, rhi, wmask);
    }
    // interior: global bit mask and mask bytes
    const bool interior = lane >= 1 && lane <= kStripWords && col_ok;
    if (!interior) return;
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < kStripRows; ++i) {
        const int r = HR + i, y = y0 + i;
        const uint32_t fin = v[r] & ((r >= rlo && r < rhi) ? wmask : 0u);
        any |= fin;
        if (!HMI_IN_BOUNDS(y < D.bh * kBlock, &D.st->err)) break;
        D.bits[(long long)y * nwords + kw] = fin;
        if (io.mask != nullptr && y < h) {
            uint8_t *dst = io.mask + (long long)y * w + kw * kWordPx;
            const int npx = min(kWordPx, w - kw * kWordPx);
            if (npx == kWordPx && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
                uint32_t q[8];
#pragma unroll
                for (int n4 = 0; n4 < 8; ++n4) q[n4] = (((fin >> (4 * n4)) & 0xfu) * 0x00204081u) & 0x01010101u;
                uint4 *d4 = reinterpret_cast<uint4 *>(dst);
                __stcs(d4, make_uint4(q[0], q[1], q[2], q[3]));
                __stcs(d4 + 1, make_uint4(q[4], q[5], q[6], q[7]));
            } else {
                for (int x = 0; x < npx; ++x) dst[x] = (uint8_t)((fin >> x) & 1u);
            }
        }
    }
    // the 32x32 block of this word: the upper strip of a block clears its
    // count; the first strip to find pixels in it lists it for k_block_cc
    const uint32_t blk = (uint32_t)((y0 / kBlock) * nwords + kw);
    if (!HMI_IN_BOUNDS(blk < (uint32_t)(D.bh * nwords), &D.st->err)) return;
    if ((y0 % kBlock) == 0) D.count[blk] = 0u;   // the top strip of the block
    if (any != 0u && atomicOr(D.flag + blk, 1u) == 0u) {
        const uint32_t slot = atomicAdd(cc_count, 1u);
        if (HMI_IN_BOUNDS(slot < cc_cap, &D.st->err)) cc_list[slot] = make_uint2((uint32_t)sidx, blk);
    }
}

}  // namespace hmi
