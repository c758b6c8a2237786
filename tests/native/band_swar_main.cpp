// Checks the packed-byte band test (csrc/hmi_band.h) against the
// per-channel definition: (1) every (c, lo, hi) byte triple in every byte
// lane of a word, (2) random 16-pixel chunks at random gains, against a plain
// per-pixel loop.  Prints "ok" or the first mismatch; exit status 0 / 1.
#include <cstdint>
#include <cstdio>

#include "hmi_band.h"

static uint64_t g_state = 0x1907043930ull;
static uint32_t rnd()
{
    g_state += 0x9e3779b97f4a7c15ull;   // splitmix64
    uint64_t z = g_state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return (uint32_t)((z ^ (z >> 31)) >> 16);
}

int main()
{
    using namespace hmi;
    for (uint32_t c = 0; c < 256; ++c)
        for (uint32_t lo = 0; lo < 256; ++lo)
            for (uint32_t hi = 0; hi < 256; ++hi) {
                const int lane = (int)((c + lo + hi) & 3u);
                const uint32_t other = rnd(), sh = 8u * (uint32_t)lane, m = ~(0xffu << sh);
                const uint32_t w = swar_in_band((other & m) | (c << sh), (rnd() & m) | (lo << sh),
                                                (rnd() & m) | (hi << sh));
                const uint32_t want = (lo <= c && c <= hi) ? 1u : 0u;
                if (((w >> (sh + 7)) & 1u) != want || (w & ~0x80808080u) != 0u) {
                    std::printf("swar mismatch c=%u lo=%u hi=%u lane=%d\n", c, lo, hi, lane);
                    return 1;
                }
            }
    for (int it = 0; it < 2000000; ++it) {
        uint32_t g;
        switch (it % 8) {
        case 0: g = 65536u; break;
        case 1: g = 32768u; break;
        case 2: g = 131072u; break;
        default: g = 32768u + rnd() % 98305u; break;
        }
        uint8_t f[48], lo[48], hi[48];
        for (int k = 0; k < 48; ++k) {
            f[k] = (uint8_t)rnd();
            const uint32_t a = rnd() & 0xffu, b = rnd() & 0xffu;
            // bands near the corrected value, so that both outcomes occur
            const uint32_t cv = corrected_value(f[k], g);
            const uint32_t l = (it & 1) ? (a < b ? a : b) : (cv > (a & 7u) ? cv - (a & 7u) : 0u);
            const uint32_t h = (it & 1) ? (a < b ? b : a) : (cv + (b & 7u) < 255u ? cv + (b & 7u) : 255u);
            lo[k] = (uint8_t)((rnd() % 23u == 0u) ? h : l);   // now and then lo > hi
            hi[k] = (uint8_t)h;
        }
        uint32_t fw[12], lw[12], hw[12];
        for (int i = 0; i < 12; ++i) {
            fw[i] = lw[i] = hw[i] = 0;
            for (int j = 0; j < 4; ++j) {
                fw[i] |= (uint32_t)f[4 * i + j] << (8 * j);
                lw[i] |= (uint32_t)lo[4 * i + j] << (8 * j);
                hw[i] |= (uint32_t)hi[4 * i + j] << (8 * j);
            }
        }
        uint8_t table[256];
        for (uint32_t v = 0; v < 256; ++v) table[v] = (uint8_t)corrected_value(v, g);
        uint32_t want = 0;
        for (int k = 0; k < 16; ++k) {
            bool in = true;
            for (int ch = 0; ch < 3; ++ch) {
                const int b = 3 * k + ch;
                const uint32_t v = (f[b] * g + 32768u) >> 16;
                const uint32_t cp = v > 255u ? 255u : v;
                in = in && lo[b] <= cp && cp <= hi[b];
            }
            if (!in) want |= 1u << k;
        }
        const uint32_t got = band_outside16(fw, lw, hw, [&](uint32_t w) { return corrected_word(w, table); });
        if (got != want) {
            std::printf("chunk mismatch it=%d g=%u got=%04x want=%04x\n", it, g, got, want);
            return 1;
        }
    }
    std::printf("ok\n");
    return 0;
}
