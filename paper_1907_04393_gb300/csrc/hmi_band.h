// hmi_band.h -- the background band test (Sec. 3.1 (i)) of 16 pixels at once
// on packed bytes.  Host and device code: the CPU tests build it with g++ and
// check it against the per-channel definition.
//
// A pixel is background iff each of its gain-corrected channels c' lies in the
// learned band [lo, hi] of that pixel and channel.  The corrected values come
// from a per-frame table c' = min(255, (c g + 2^15) >> 16) of the 256 byte
// values (shared memory on the device), so that the per-channel work is one
// table read; the comparisons then run on four channels per 32-bit word
// (SWAR), and the three channels of a pixel are gathered with byte permutes.
// A 16-px chunk is 48 bytes = 12 words, in the frame's RGB-interleaved order;
// lo and hi have the same layout, so word i of the frame lines up with word i
// of lo and hi.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define HMI_HD __host__ __device__ __forceinline__
#else
#define HMI_HD inline
#endif

namespace hmi {

// Byte permute: result byte j is byte s_j (nibble j of s, 0..7) of the pair
// (a = bytes 0..3, b = bytes 4..7).
HMI_HD uint32_t bperm(uint32_t a, uint32_t b, uint32_t s)
{
#if defined(__CUDA_ARCH__)
    return __byte_perm(a, b, s);
#else
    const uint64_t ab = (uint64_t)a | ((uint64_t)b << 32);
    uint32_t r = 0;
    for (int j = 0; j < 4; ++j) r |= (uint32_t)((ab >> (8 * ((s >> (4 * j)) & 7u))) & 0xffu) << (8 * j);
    return r;
#endif
}

// Per byte (bit 7 of each byte, the other bits 0): x >= y as unsigned bytes.
// (x | 0x80) - (y & 0x7f) stays within each byte (1..255), and its bit 7 is
// (x & 0x7f) >= (y & 0x7f); that decides when the top bits of x and y agree,
// and the top bits decide when they differ.
HMI_HD uint32_t swar_ge(uint32_t x, uint32_t y)
{
    const uint32_t d = (x | 0x80808080u) - (y & 0x7f7f7f7fu);
    return ((x & ~y) | (~(x ^ y) & d)) & 0x80808080u;
}

// Per byte (bit 7): lo <= c <= hi.
HMI_HD uint32_t swar_in_band(uint32_t c, uint32_t lo, uint32_t hi)
{
    return swar_ge(c, lo) & swar_ge(hi, c);
}

// Out-of-band bits of a 16-px chunk (bit k = pixel k) from its 12 frame words
// and the band words; corr(word) gives the word of the four corrected values.
// Group q (pixels 4q..4q+3) uses words 3q..3q+2; the R, G and B bytes of its
// pixels sit at bytes (0, 3, 6, 9), (1, 4, 7, 10), (2, 5, 8, 11) of those 12.
template <class Corr>
HMI_HD uint32_t band_outside16(const uint32_t (&f)[12], const uint32_t (&lo)[12], const uint32_t (&hi)[12],
                               const Corr &corr)
{
    uint32_t in16 = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t w0 = swar_in_band(corr(f[3 * q]), lo[3 * q], hi[3 * q]);
        const uint32_t w1 = swar_in_band(corr(f[3 * q + 1]), lo[3 * q + 1], hi[3 * q + 1]);
        const uint32_t w2 = swar_in_band(corr(f[3 * q + 2]), lo[3 * q + 2], hi[3 * q + 2]);
        const uint32_t r = bperm(bperm(w0, w1, 0x0630u), w2, 0x5210u);   // w0.b0 w0.b3 w1.b2 w2.b1
        const uint32_t g = bperm(bperm(w0, w1, 0x0741u), w2, 0x6210u);   // w0.b1 w1.b0 w1.b3 w2.b2
        const uint32_t b = bperm(bperm(w0, w1, 0x0052u), w2, 0x7410u);   // w0.b2 w1.b1 w2.b0 w2.b3
        const uint32_t p = r & g & b;   // bit 7 of byte j: pixel 4q + j in the band
        // bit 7 of byte j moves to bit 28 + j (the other partial products stay
        // below bit 24 or above bit 31)
        in16 |= ((p * 0x00204081u) >> 28) << (4 * q);
    }
    return ~in16 & 0xffffu;
}

// The word of the corrected values of four bytes through a 256-entry table.
HMI_HD uint32_t corrected_word(uint32_t w, const uint8_t *table)
{
    return (uint32_t)table[w & 0xffu] + (uint32_t)table[(w >> 8) & 0xffu] * 0x100u +
           (uint32_t)table[(w >> 16) & 0xffu] * 0x10000u + (uint32_t)table[w >> 24] * 0x1000000u;
}

// The per-frame table of corrected values.
HMI_HD uint32_t corrected_value(uint32_t c, uint32_t g)
{
    const uint32_t v = (c * g + 32768u) >> 16;
    return v < 255u ? v : 255u;
}

}  // namespace hmi
