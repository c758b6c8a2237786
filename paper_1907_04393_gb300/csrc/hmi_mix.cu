// hmi_mix.cu -- Gaussian mixture background (Sec. 2: the FIZI module learns
// the background with advanced machine learning; Sec. 3.3 cites Lee's adaptive
// Gaussian mixture learning), a variant of the band of Sec. 3.1 (i):
//   k_mix        per tick: brightness-corrected value of every pixel of the
//                mixture streams, the mixture's background test (the raw bit
//                and the skin queue, exactly as k_classify leaves them for the
//                band) and the update of its components
//   k_mix_learn  the same update over learning frames (no test, gain 1)
// Per pixel and frame t, with K components in fitness order, each a weight W
// (Q15), a mean per channel M (Q8), one variance V (Q4) and a match count C:
//   match     the first non-empty component with
//             kd^2 sum_c (256 x_c - M_c)^2 <= kn^2 V 4096
//   test      background iff it matched component j and the weights before j
//             sum to at most T percent of all weights
//   update    matched: C + 1, r = min(C, N), M += (256 x - M) / r,
//             V += (D / 3 - V) / r (D the squared distance in Q4), V clamped
//             to [Vmin, 65535]; none matched: the last component restarts at
//             x (V0, C = 1, W = 0); then every W moves by (32768 or 0 - W) / m,
//             m = min(t, N); divisions round half away from zero
//   order     stable re-sort: non-empty first, by W / sqrt(V) descending
// All integer, so the result is exact.  Bound by HBM: 12 K bytes of state read
// and written per pixel plus the frame.
#include <algorithm>

#include "hmi_ccfill.cuh"
#include "hmi_internal.cuh"

namespace hmi {

template <int K>
struct MixPx {
    uint32_t w[K], m[K][3], v[K], c[K];
};

// round(a / m), halves away from zero, for a >= 0 and 2 a + m < 2^32.
__device__ __forceinline__ uint32_t udiv_round(uint32_t a, uint32_t m)
{
    return (2u * a + m) / (2u * m);
}

__device__ __forceinline__ int32_t sdiv_round(int32_t a, uint32_t m)
{
    const uint32_t q = udiv_round((uint32_t)(a < 0 ? -a : a), m);
    return a < 0 ? -(int32_t)q : (int32_t)q;
}

// Component a + 1 goes before component a iff it is strictly fitter.
template <int K>
__device__ __forceinline__ void order_pair(MixPx<K> &s, int a)
{
    const bool ca = s.c[a] != 0u, cb = s.c[a + 1] != 0u;
    // W <= 32768, so W^2 fits 32 bits and W^2 V fits 48
    const unsigned long long lhs = (unsigned long long)(s.w[a + 1] * s.w[a + 1]) * s.v[a];
    const unsigned long long rhs = (unsigned long long)(s.w[a] * s.w[a]) * s.v[a + 1];
    if (cb && (!ca || lhs > rhs)) {
        uint32_t t;
        t = s.w[a]; s.w[a] = s.w[a + 1]; s.w[a + 1] = t;
        t = s.v[a]; s.v[a] = s.v[a + 1]; s.v[a + 1] = t;
        t = s.c[a]; s.c[a] = s.c[a + 1]; s.c[a + 1] = t;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            t = s.m[a][ch]; s.m[a][ch] = s.m[a + 1][ch]; s.m[a + 1][ch] = t;
        }
    }
}

// One frame of one pixel: x the (corrected) value, t the frame's number.
// Returns whether the pixel is background (meaningful when classify).
template <int K>
__device__ __forceinline__ bool mix_step(MixPx<K> &s, uint32_t x0, uint32_t x1, uint32_t x2,
                                         uint32_t t, const MixView &G, bool classify)
{
    const int32_t X0 = (int32_t)(256u * x0), X1 = (int32_t)(256u * x1), X2 = (int32_t)(256u * x2);
    int j = -1;
    int32_t e0 = 0, e1 = 0, e2 = 0;
    unsigned long long d2 = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int32_t a0 = X0 - (int32_t)s.m[k][0], a1 = X1 - (int32_t)s.m[k][1],
                      a2 = X2 - (int32_t)s.m[k][2];
        const uint32_t b0 = (uint32_t)abs(a0), b1 = (uint32_t)abs(a1), b2 = (uint32_t)abs(a2);
        // each |a| <= 65280, so each square fits 32 bits
        const unsigned long long q = (unsigned long long)(b0 * b0) + (b1 * b1) + (unsigned long long)(b2 * b2);
        const bool hit = s.c[k] != 0u && (unsigned long long)G.lam_a * q <= (unsigned long long)G.lam_b * s.v[k];
        if (hit && j < 0) {
            j = k;
            e0 = a0;
            e1 = a1;
            e2 = a2;
            d2 = q;
        }
    }
    bool background = false;
    if (classify) {
        uint32_t total = 0, before = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            total += s.w[k];
            if (k < j) before += s.w[k];
        }
        background = j >= 0 && 100u * before <= (uint32_t)G.bg_pct * total;
    }
    const uint32_t mt = min(t, (uint32_t)G.rate_n);
    int jj = j;
    if (j < 0) {
        jj = K - 1;
        s.m[K - 1][0] = (uint32_t)X0;
        s.m[K - 1][1] = (uint32_t)X1;
        s.m[K - 1][2] = (uint32_t)X2;
        s.v[K - 1] = G.v_init;
        s.c[K - 1] = 1u;
        s.w[K - 1] = 0u;
    } else {
        // D / 3 in Q4: round(d2 / (3 * 4096)), d2 < 2^34
        const int32_t target = (int32_t)((2ull * d2 + 12288ull) / 24576ull);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k != j) continue;
            s.c[k] = min(s.c[k] + 1u, 65535u);
            const uint32_t r = min(s.c[k], (uint32_t)G.rate_n);
            s.m[k][0] = (uint32_t)((int32_t)s.m[k][0] + sdiv_round(e0, r));
            s.m[k][1] = (uint32_t)((int32_t)s.m[k][1] + sdiv_round(e1, r));
            s.m[k][2] = (uint32_t)((int32_t)s.m[k][2] + sdiv_round(e2, r));
            const int32_t v = (int32_t)s.v[k] + sdiv_round(target - (int32_t)s.v[k], r);
            s.v[k] = (uint32_t)min(max(v, (int32_t)G.v_min), 65535);
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
        s.w[k] = (k == jj) ? s.w[k] + udiv_round(32768u - s.w[k], mt) : s.w[k] - udiv_round(s.w[k], mt);
    // stable bubble network: K - 1 passes of adjacent pairs
#pragma unroll
    for (int pass = 0; pass < K - 1; ++pass) {
#pragma unroll
        for (int a = 0; a + 1 < K - pass; ++a) order_pair<K>(s, a);
    }
    return background;
}

// Field f of component k in the plane order W[k], M[k][c], V[k], C[k].
template <int K>
__device__ __forceinline__ uint32_t &field(MixPx<K> &s, int p)
{
    if (p < K) return s.w[p];
    if (p < 4 * K) return s.m[(p - K) / 3][(p - K) % 3];
    if (p < 5 * K) return s.v[p - 4 * K];
    return s.c[p - 5 * K];
}

// ---------------------------------------------------------------------------
// k_mix: one lane per pixel, so that every plane access of a warp is 64
// contiguous bytes and a warp's 32 pixels (two 16-px chunks of one row) are
// exactly one raw mask word (a ballot).
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void mix_piece(const BatchDev &b, const int4 piece, const DevStream &D,
                                          const TickIO &io, uint32_t g, uint32_t t)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int cpr = 2 * D.nwords, w = D.w;
    const MixView G = D.mix;
    uint32_t *raw = D.raw[b.phase];
    // pieces start at even chunks, so `base` is the first chunk of a word
    for (int base = piece.y + 2 * warp; base < piece.z; base += 2 * nwarp) {
        const int u = base + (lane >> 4);
        bool fg = false;
        int y = 0, j = 0;
        if (u < piece.z) {
            y = chunk_row((uint32_t)u, D.cpr_magic);
            j = u - y * cpr;
            const int x = j * kChunkPx + (lane & 15);
            if (x < w) {
                const uint8_t *px = io.frame + (long long)y * io.frame_pitch + 3 * x;
                uint16_t *P = G.planes + (size_t)y * G.pitch + x;
                MixPx<K> s;
#pragma unroll
                for (int p = 0; p < 6 * K; ++p) field<K>(s, p) = P[(size_t)p * G.plane];
                const uint32_t c0 = min((px[0] * g + 32768u) >> 16, 255u);
                const uint32_t c1 = min((px[1] * g + 32768u) >> 16, 255u);
                const uint32_t c2 = min((px[2] * g + 32768u) >> 16, 255u);
                fg = !mix_step<K>(s, c0, c1, c2, t, G, true);
#pragma unroll
                for (int p = 0; p < 6 * K; ++p) P[(size_t)p * G.plane] = (uint16_t)field<K>(s, p);
            }
        }
        const uint32_t word = __ballot_sync(kFull, fg);
        if (lane == 0 && u < piece.z) raw[(long long)y * D.nwords + (j >> 1)] = word;
        const uint32_t cb = (word >> (lane & 16)) & 0xffffu;   // this lane's chunk
        const bool lead = (lane & 15) == 0 && u < piece.z && cb != 0u;
        const unsigned want = __ballot_sync(kFull, lead);
        if (want) {
            uint32_t slot0 = 0;
            if (lane == __ffs(want) - 1) slot0 = atomicAdd(b.skin_count, (uint32_t)__popc(want));
            slot0 = __shfl_sync(kFull, slot0, __ffs(want) - 1);
            if (lead) {
                const uint32_t slot = slot0 + (uint32_t)__popc(want & ((1u << lane) - 1u));
                b.skin_list[slot] = make_uint2(((uint32_t)piece.x << 16) | cb, (uint32_t)u);
            }
        }
    }
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_mix(BatchDev b)
{
    for (int pc = blockIdx.x; pc < b.npieces; pc += gridDim.x) {
        const int4 piece = b.pieces[pc];
        const DevStream &D = b.ds[piece.x];
        const TickIO io = b.io[piece.x];
        if (io.frame == nullptr || D.mix.K != K) continue;   // CTA-uniform
        const uint32_t g = D.st->gain_p[b.phase];
        const uint32_t t = D.st->nlearn + D.st->lframe_p[b.phase];
        mix_piece<K>(b, piece, D, io, g, t);
    }
}

// ---------------------------------------------------------------------------
// k_mix_learn: one thread per pixel over nf dense frames, the state kept in
// registers between frames.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void mix_learn_px(const uint8_t *frames, int nf, uint32_t t0, long long npx,
                                             long long p, int x, int y, const MixView &G)
{
    uint16_t *P = G.planes + (size_t)y * G.pitch + x;
    MixPx<K> s;
#pragma unroll
    for (int f = 0; f < 6 * K; ++f) field<K>(s, f) = P[(size_t)f * G.plane];
    for (int i = 0; i < nf; ++i) {
        const uint8_t *px = frames + (long long)i * npx * 3 + 3 * p;
        mix_step<K>(s, px[0], px[1], px[2], t0 + (uint32_t)i + 1u, G, false);
    }
#pragma unroll
    for (int f = 0; f < 6 * K; ++f) P[(size_t)f * G.plane] = (uint16_t)field<K>(s, f);
}

__global__ void __launch_bounds__(kThreads) k_mix_learn(const uint8_t *frames, int nf, uint32_t t0, int w,
                                                        int h, MixView G)
{
    const long long npx = (long long)w * h;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx;
         p += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(p / w), x = (int)(p - (long long)y * w);
        switch (G.K) {
        case 1: mix_learn_px<1>(frames, nf, t0, npx, p, x, y, G); break;
        case 2: mix_learn_px<2>(frames, nf, t0, npx, p, x, y, G); break;
        case 3: mix_learn_px<3>(frames, nf, t0, npx, p, x, y, G); break;
        default: mix_learn_px<4>(frames, nf, t0, npx, p, x, y, G); break;
        }
    }
}

// One kernel per component count present in the batch (bit K of any_mix).
cudaError_t launch_mix(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    (void)num_sms;
    const unsigned grid = b.npieces > 0 ? (unsigned)b.npieces : 1u;
    if (b.any_mix & 2) k_mix<1><<<grid, kThreads, 0, cs>>>(b);
    if (b.any_mix & 4) k_mix<2><<<grid, kThreads, 0, cs>>>(b);
    if (b.any_mix & 8) k_mix<3><<<grid, kThreads, 0, cs>>>(b);
    if (b.any_mix & 16) k_mix<4><<<grid, kThreads, 0, cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_mix_learn(const uint8_t *frames, int nf, uint32_t t0, int w, int h, const MixView &mix,
                             cudaStream_t cs)
{
    if (mix.K < 1 || mix.K > 4 || nf < 1) return cudaErrorInvalidValue;
    const long long npx = (long long)w * h;
    const unsigned grid = (unsigned)std::min<long long>((npx + kThreads - 1) / kThreads, 1ll << 16);
    k_mix_learn<<<grid, kThreads, 0, cs>>>(frames, nf, t0, w, h, mix);
    return cudaGetLastError();
}

}  // namespace hmi
