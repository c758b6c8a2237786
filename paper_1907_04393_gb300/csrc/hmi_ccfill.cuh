// hmi_ccfill.cuh -- warp-level 8-connected component enumeration of one
// 32x32 block of mask bits (one 32-bit word per row, lane r holds row r,
// bit i = column i).  Used by the fused morphology/labelling kernel and by the
// on-demand label export, so that both enumerate components in the same order.
#pragma once

#include <stdint.h>

namespace hmi {

constexpr unsigned kFull = 0xffffffffu;

// Propagate the bits of g towards higher bit indices through runs of p
// (logarithmic occluded fill; g must be a subset of p).
__device__ __forceinline__ uint32_t fill_up(uint32_t g, uint32_t p)
{
    g |= p & (g << 1);
    p &= p << 1;
    g |= p & (g << 2);
    p &= p << 2;
    g |= p & (g << 4);
    p &= p << 4;
    g |= p & (g << 8);
    p &= p << 8;
    g |= p & (g << 16);
    return g;
}

__device__ __forceinline__ uint32_t fill_down(uint32_t g, uint32_t p)
{
    g |= p & (g >> 1);
    p &= p >> 1;
    g |= p & (g >> 2);
    p &= p >> 2;
    g |= p & (g >> 4);
    p &= p >> 4;
    g |= p & (g >> 8);
    p &= p >> 8;
    g |= p & (g >> 16);
    return g;
}

// Whole horizontal runs of m that contain a bit of c.
__device__ __forceinline__ uint32_t run_fill(uint32_t c, uint32_t m)
{
    return fill_up(c, m) | fill_down(c, m);
}

// Propagate the bits of g along the columns (lane r -> r+1 -> ...) through
// vertical runs of p, and the other way (lane r -> r-1 -> ...); logarithmic
// fills across lanes with shuffles.  g must be a subset of p.
__device__ __forceinline__ uint32_t col_fill(uint32_t g, uint32_t p, int lane)
{
    uint32_t gd = g, pd = p, gu = g, pu = p;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        uint32_t a = __shfl_up_sync(kFull, gd, s), b = __shfl_up_sync(kFull, pd, s);
        if (lane < s) a = b = 0u;
        gd |= pd & a;
        pd &= b;
        uint32_t c = __shfl_down_sync(kFull, gu, s), d = __shfl_down_sync(kFull, pu, s);
        if (lane >= 32 - s) c = d = 0u;
        gu |= pu & c;
        pu &= d;
    }
    return gd | gu;
}

// Extract the component of the first remaining pixel in raster order
// (lowest row, then lowest column) from the per-lane row words m.
// Returns this lane's row of the component; *seed_row / *seed_col give the
// seed, which is the component's smallest pixel index inside the block.
// Each round grows the set by whole horizontal runs, whole vertical runs, and
// the 8-neighbours in the rows above and below, until a round adds nothing;
// the fixed point is closed under every 8-neighbour step, so it is the whole
// component.  A round that does not stop adds at least one pixel, so the loop
// ends within 1024 rounds (a convex blob takes about three).
__device__ __forceinline__ uint32_t cc_extract_first(uint32_t m, int lane, int *seed_row,
                                                     int *seed_col)
{
    unsigned rows = __ballot_sync(kFull, m != 0u);
    int r0 = __ffs(rows) - 1;
    uint32_t mr0 = __shfl_sync(kFull, m, r0);
    int b0 = __ffs(mr0) - 1;
    *seed_row = r0;
    *seed_col = b0;
    uint32_t c = (lane == r0) ? (1u << b0) : 0u;
    for (int it = 0; it < 1100; ++it) {
        c = run_fill(c, m);
        c = col_fill(c, m, lane);
        uint32_t d = c | (c << 1) | (c >> 1);
        uint32_t up = __shfl_up_sync(kFull, d, 1);
        uint32_t dn = __shfl_down_sync(kFull, d, 1);
        if (lane == 0) up = 0u;
        if (lane == 31) dn = 0u;
        uint32_t nc = c | ((up | dn) & m);
        bool grew = __any_sync(kFull, nc != c);
        c = nc;
        if (!grew) break;
    }
    return c;
}

// Sum over the set bits of c of their bit index (0..31).
__device__ __forceinline__ uint32_t bit_index_sum(uint32_t c)
{
    return (uint32_t)__popc(c & 0xAAAAAAAAu) + 2u * (uint32_t)__popc(c & 0xCCCCCCCCu) +
           4u * (uint32_t)__popc(c & 0xF0F0F0F0u) + 8u * (uint32_t)__popc(c & 0xFF00FF00u) +
           16u * (uint32_t)__popc(c & 0xFFFF0000u);
}

}  // namespace hmi
