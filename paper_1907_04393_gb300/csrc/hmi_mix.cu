// hmi_mix.cu -- Gaussian mixture background (Sec. 2: FIZI's background is
// learned with advanced machine learning; Sec. 3.3 cites Lee's adaptive
// Gaussian mixture learning), a variant of the band of Sec. 3.1 (i):
//   k_mix        per tick: brightness-corrected value of every pixel of the
//                mixture streams, the mixture's background test (the raw bit
//                and the skin queue, exactly as k_classify leaves them for the
//                band) and the update of its components
//   k_mix_learn  the same update over learning frames (no test, gain 1)
// Per pixel and frame t, with K components in fitness order, each a weight W
// (Q15), a mean per channel M (Q8), one variance V (Q4) and a match count C:
//   match     the first non-empty component with
//             kd^2 sum_c (256 x_c - M_c)^2 <= 3 kn^2 V 4096 (mean squared
//             channel deviation within (kn / kd)^2 V)
//   test      background iff it matched component j and the weights before j
//             sum to at most T percent of all weights
//   update    matched: C + 1, r = min(C, N), M += (256 x - M) / r,
//             V += (D / 3 - V) / r (D the squared distance in Q4), V clamped
//             to [Vmin, 65535]; none matched: the last component restarts at
//             x (V0, C = 1, W = 0); then every W moves by (32768 or 0 - W) / m,
//             m = min(t, N); divisions round half away from zero
//   order     stable re-sort: non-empty first, by W / sqrt(V) descending
// All integer, so the result is exact.  Bound by HBM and instruction issue:
// 12 K bytes of state read and written per pixel plus the frame, and a few
// hundred integer instructions per pixel.
#include <algorithm>

#include "hmi_ccfill.cuh"
#include "hmi_internal.cuh"

namespace hmi {

template <int K>
struct MixPx {
    uint32_t w[K], m[K][3], v[K], c[K];
};

// Every numerator below stays under 2^22, as recip40 requires: 2 |a| + m
// with |a| <= 1,040,400 (a variance step) and m <= 65535.
// round(a / m), halves away from zero: floor((2 a + m) / 2 m), for a >= 0,
// with rm = recip40(2 m) (one multiply) or by a plain division.
__device__ __forceinline__ uint32_t udiv_round(uint32_t a, uint32_t m, unsigned long long rm)
{
    return (uint32_t)(((unsigned long long)(2u * a + m) * rm) >> 40);
}

__device__ __forceinline__ uint32_t udiv_round_plain(uint32_t a, uint32_t m)
{
    return (2u * a + m) / (2u * m);
}

__device__ __forceinline__ int32_t sdiv_round(int32_t a, uint32_t m, unsigned long long rm)
{
    const uint32_t q = udiv_round((uint32_t)(a < 0 ? -a : a), m, rm);
    return a < 0 ? -(int32_t)q : (int32_t)q;
}

__device__ __forceinline__ int32_t sdiv_round_plain(int32_t a, uint32_t m)
{
    const uint32_t q = udiv_round_plain((uint32_t)(a < 0 ? -a : a), m);
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
// rmt: recip40(2 min(t, N)), the weights' divisor for this frame.
template <int K>
__device__ __forceinline__ bool mix_step(MixPx<K> &s, uint32_t x0, uint32_t x1, uint32_t x2,
                                         uint32_t t, unsigned long long rmt, const MixView &G,
                                         bool classify)
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
    // the component this frame updates: the matched one, or the last one
    // replaced by a new component at x; gathered once, updated, put back
    const int jj = j < 0 ? K - 1 : j;
    uint32_t m0 = s.m[K - 1][0], m1 = s.m[K - 1][1], m2 = s.m[K - 1][2], v = s.v[K - 1], c = s.c[K - 1];
#pragma unroll
    for (int k = 0; k < K - 1; ++k)
        if (k == jj) {
            m0 = s.m[k][0];
            m1 = s.m[k][1];
            m2 = s.m[k][2];
            v = s.v[k];
            c = s.c[k];
        }
    if (j < 0) {
        m0 = (uint32_t)X0;
        m1 = (uint32_t)X1;
        m2 = (uint32_t)X2;
        v = G.v_init;
        c = 1u;
    } else {
        // D / 3 in Q4: round(d2 / (3 * 4096)), d2 < 2^34
        const int32_t target = (int32_t)((2ull * d2 + 12288ull) / 24576ull);
        c = min(c + 1u, 65535u);
        const uint32_t r = min(c, (uint32_t)G.rate_n);
        const int32_t dv = target - (int32_t)v;
        int32_t q0, q1, q2, qv;
        if (r == (uint32_t)G.rate_n) {   // the steady state: the stream's reciprocal
            q0 = sdiv_round(e0, r, G.recip_n);
            q1 = sdiv_round(e1, r, G.recip_n);
            q2 = sdiv_round(e2, r, G.recip_n);
            qv = sdiv_round(dv, r, G.recip_n);
        } else {                         // a young component: plain divisions
            q0 = sdiv_round_plain(e0, r);
            q1 = sdiv_round_plain(e1, r);
            q2 = sdiv_round_plain(e2, r);
            qv = sdiv_round_plain(dv, r);
        }
        m0 = (uint32_t)((int32_t)m0 + q0);
        m1 = (uint32_t)((int32_t)m1 + q1);
        m2 = (uint32_t)((int32_t)m2 + q2);
        v = (uint32_t)min(max((int32_t)v + qv, (int32_t)G.v_min), 65535);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const bool mine = k == jj;
        if (mine) {
            s.m[k][0] = m0;
            s.m[k][1] = m1;
            s.m[k][2] = m2;
            s.v[k] = v;
            s.c[k] = c;
        }
        // toward 32768 for the updated component (a new one starts at 0),
        // toward 0 for the others: one rounded division each
        const uint32_t w0 = (mine && j < 0) ? 0u : s.w[k];
        const uint32_t q = udiv_round(mine ? 32768u - w0 : w0, mt, rmt);
        s.w[k] = mine ? w0 + q : w0 - q;
    }
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
// k_mix: a warp per 32-pixel tile (one mask word, one lane per pixel).  The
// tile's state block (6 K fields x 64 bytes, contiguous) and its frame bytes
// are staged in shared memory by cp.async, one tile ahead, so that each
// warp's next loads are in flight while it computes; results go straight
// back to global memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp16(void *dst, const void *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int K>
struct MixStage {
    static constexpr int kTile = 6 * K * 64;     // state bytes of a tile
    static constexpr int kBytes = kTile + 96;    // + the frame bytes of 32 pixels
};

// Row and first pixel of word wd (the chunk pair 2 wd, 2 wd + 1) of a stream.
__device__ __forceinline__ void word_pos(const DevStream &D, int wd, int &y, int &x0)
{
    const int u = 2 * wd;
    y = chunk_row((uint32_t)u, D.cpr_magic);
    x0 = (u - y * 2 * D.nwords) * kChunkPx;
}

template <int K>
__device__ __forceinline__ void stage_word(const DevStream &D, const TickIO &io, int wd, uint8_t *dst, int lane)
{
    int y, x0;
    word_pos(D, wd, y, x0);
    const uint8_t *tile = reinterpret_cast<const uint8_t *>(D.mix.planes + mix_tile(D.mix, x0, y));
    // frame bytes of the tile's valid pixels, rounded up to whole 16-pixel
    // chunks (inside the row: the staging pitch and direct frames' widths are
    // multiples of 16 pixels)
    const int nf = 3 * ((min(32, D.w - x0) + 15) >> 4);   // 16-byte pieces: 3 or 6
    const uint8_t *fr = io.frame + (long long)y * io.frame_pitch + 3 * x0;
    constexpr int nt = MixStage<K>::kTile / 16;
    for (int c = lane; c < nt + nf; c += 32) {
        if (c < nt) cp16(dst + 16 * c, tile + 16 * c);
        else cp16(dst + MixStage<K>::kTile + 16 * (c - nt), fr + 16 * (c - nt));
    }
}

template <int K>
__device__ __forceinline__ void mix_piece(const BatchDev &b, const int4 piece, const DevStream &D,
                                          const TickIO &io, uint32_t g, uint32_t t,
                                          uint8_t (*stage)[MixStage<K>::kBytes])
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int w = D.w;
    const MixView G = D.mix;
    uint32_t *raw = D.raw[b.phase];
    const uint32_t mt = min(t, (uint32_t)G.rate_n);
    const unsigned long long rmt = mt == (uint32_t)G.rate_n ? G.recip_n : recip40(2u * mt);
    // pieces start and end at even chunks: words [piece.y / 2, piece.z / 2)
    const int w1 = piece.z >> 1;
    int wd = (piece.y >> 1) + warp, st = 0;
    if (wd < w1) stage_word<K>(D, io, wd, stage[0], lane);
    cp_commit();
    for (; wd < w1; wd += nwarp) {
        if (wd + nwarp < w1) stage_word<K>(D, io, wd + nwarp, stage[st ^ 1], lane);
        cp_commit();
        cp_wait<1>();      // this lane's copies of word wd have landed
        __syncwarp();      // and every other lane's
        int y, x0;
        word_pos(D, wd, y, x0);
        const int x = x0 + lane;
        bool fg = false;
        if (x < w) {
            const uint16_t *S = reinterpret_cast<const uint16_t *>(stage[st]) + lane;
            const uint8_t *px = stage[st] + MixStage<K>::kTile + 3 * lane;
            MixPx<K> s;
#pragma unroll
            for (int p = 0; p < 6 * K; ++p) field<K>(s, p) = S[32 * p];
            const uint32_t c0 = min((px[0] * g + 32768u) >> 16, 255u);
            const uint32_t c1 = min((px[1] * g + 32768u) >> 16, 255u);
            const uint32_t c2 = min((px[2] * g + 32768u) >> 16, 255u);
            fg = !mix_step<K>(s, c0, c1, c2, t, rmt, G, true);
            uint16_t *P = G.planes + mix_tile(G, x0, y) + lane;
#pragma unroll
            for (int p = 0; p < 6 * K; ++p) P[32 * p] = (uint16_t)field<K>(s, p);
        }
        __syncwarp();      // the stage is read before it is refilled
        st ^= 1;
        const uint32_t word = __ballot_sync(kFull, fg);
        if (lane == 0) raw[(long long)y * D.nwords + (x0 >> 5)] = word;
        const uint32_t cb = (word >> (lane & 16)) & 0xffffu;   // this lane's chunk
        const bool lead = (lane & 15) == 0 && cb != 0u;
        const unsigned want = __ballot_sync(kFull, lead);
        if (want) {
            uint32_t slot0 = 0;
            if (lane == __ffs(want) - 1) slot0 = atomicAdd(b.skin_count, (uint32_t)__popc(want));
            slot0 = __shfl_sync(kFull, slot0, __ffs(want) - 1);
            if (lead) {
                const uint32_t slot = slot0 + (uint32_t)__popc(want & ((1u << lane) - 1u));
                b.skin_list[slot] = make_uint2(((uint32_t)piece.x << 16) | cb, (uint32_t)(2 * wd + (lane >> 4)));
            }
        }
    }
    cp_wait<0>();
}

template <int K>
__global__ void __launch_bounds__(kThreads) k_mix(BatchDev b)
{
    __shared__ __align__(16) uint8_t stage[kThreads / 32][2][MixStage<K>::kBytes];
    const int warp = threadIdx.x >> 5;
    for (int pc = blockIdx.x; pc < b.npieces; pc += gridDim.x) {
        const int4 piece = b.pieces[pc];
        const DevStream &D = b.ds[piece.x];
        const TickIO io = b.io[piece.x];
        if (io.frame == nullptr || D.mix.K != K) continue;   // CTA-uniform
        const uint32_t g = D.st->gain_p[b.phase];
        const uint32_t t = D.st->nlearn + D.st->lframe_p[b.phase];
        mix_piece<K>(b, piece, D, io, g, t, stage[warp]);
    }
}

// ---------------------------------------------------------------------------
// k_mix_learn: one thread per pixel over up to kLearnFrames dense frames, the
// state kept in registers between frames; the frames' weight divisors are
// computed once per CTA.
// ---------------------------------------------------------------------------
constexpr int kLearnFrames = 64;

template <int K>
__global__ void __launch_bounds__(kThreads) k_mix_learn(const uint8_t *frames, int nf, uint32_t t0, int w,
                                                        int h, MixView G)
{
    __shared__ unsigned long long rmt[kLearnFrames];
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const uint32_t mt = min(t0 + (uint32_t)i + 1u, (uint32_t)G.rate_n);
        rmt[i] = mt == (uint32_t)G.rate_n ? G.recip_n : recip40(2u * mt);
    }
    __syncthreads();
    const long long npx = (long long)w * h;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < npx;
         p += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(p / w), x = (int)(p - (long long)y * w);
        uint16_t *P = G.planes + mix_tile(G, x, y) + (x & 31);
        MixPx<K> s;
#pragma unroll
        for (int f = 0; f < 6 * K; ++f) field<K>(s, f) = P[32 * f];
        for (int i = 0; i < nf; ++i) {
            const uint8_t *px = frames + (long long)i * npx * 3 + 3 * p;
            mix_step<K>(s, px[0], px[1], px[2], t0 + (uint32_t)i + 1u, rmt[i], G, false);
        }
#pragma unroll
        for (int f = 0; f < 6 * K; ++f) P[32 * f] = (uint16_t)field<K>(s, f);
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
    for (int i = 0; i < nf; i += kLearnFrames) {
        const int k = std::min(kLearnFrames, nf - i);
        const uint8_t *f = frames + (size_t)i * (size_t)npx * 3;
        const uint32_t t = t0 + (uint32_t)i;
        switch (mix.K) {
        case 1: k_mix_learn<1><<<grid, kThreads, 0, cs>>>(f, k, t, w, h, mix); break;
        case 2: k_mix_learn<2><<<grid, kThreads, 0, cs>>>(f, k, t, w, h, mix); break;
        case 3: k_mix_learn<3><<<grid, kThreads, 0, cs>>>(f, k, t, w, h, mix); break;
        default: k_mix_learn<4><<<grid, kThreads, 0, cs>>>(f, k, t, w, h, mix); break;
        }
    }
    return cudaGetLastError();
}

}  // namespace hmi
