// hmi_learn.cu -- background learning (Sec. 2: FIZI's background is learned
// before the hand enters; Sec. 3.1 (i): per-pixel minimum and
// maximum taken during that learning; Sec. 3.3: Gaussian background models).
//   k_learn_accum  exact per pixel-channel sums S = sum v, Q = sum v^2 and the
//                  min / max over a chunk of frames, plus the frames' luma total
//                  (k_learn_accum4: the same, four pixels per thread, vectorised)
//   k_learn_band   band [lo, hi] = [min(vmin, L_k) - delta, max(vmax, H_k) + delta]
//                  clamped to bytes, with L_k / H_k the exact integer edges of
//                  mu -/+ k sigma; written in the padded row layout the
//                  per-pixel kernel reads
//   k_stats        FP32 mean S/n and std sqrt((n Q - S^2) / n^2), one correctly
//                  rounded IEEE operation per step
#include "hmi_internal.cuh"

namespace hmi {

__global__ void __launch_bounds__(kThreads) k_learn_accum(const uint8_t *__restrict__ frames,
                                                          int nf, long long npx,
                                                          uint32_t *S, uint32_t *Q,
                                                          uint8_t *vmin, uint8_t *vmax,
                                                          int first, StreamState *st)
{
    __shared__ unsigned long long red[kThreads / 32];
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long luma = 0;
    if (p < npx) {
        uint32_t s[3], q[3], mn[3], mx[3];
        for (int c = 0; c < 3; ++c) {
            s[c] = first ? 0u : S[3 * p + c];
            q[c] = first ? 0u : Q[3 * p + c];
            mn[c] = first ? 255u : vmin[3 * p + c];
            mx[c] = first ? 0u : vmax[3 * p + c];
        }
        for (int i = 0; i < nf; ++i) {
            const uint8_t *f = frames + ((long long)i * npx + p) * 3;
            const uint32_t v0 = f[0], v1 = f[1], v2 = f[2];
            const uint32_t v[3] = {v0, v1, v2};
            for (int c = 0; c < 3; ++c) {
                s[c] += v[c];
                q[c] += v[c] * v[c];
                mn[c] = min(mn[c], v[c]);
                mx[c] = max(mx[c], v[c]);
            }
            luma += (77u * v0 + 150u * v1 + 29u * v2 + 128u) >> 8;
        }
        for (int c = 0; c < 3; ++c) {
            S[3 * p + c] = s[c];
            Q[3 * p + c] = q[c];
            vmin[3 * p + c] = (uint8_t)mn[c];
            vmax[3 * p + c] = (uint8_t)mx[c];
        }
    }
    for (int o = 16; o > 0; o >>= 1) luma += __shfl_xor_sync(0xffffffffu, luma, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = luma;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        if (t) atomicAdd(&st->learn_luma, t);
    }
}

// Same sums, four pixels (twelve channel values) per thread: the frame bytes,
// min and max as three 32-bit words each (byte-wise min / max on packed
// bytes), S and Q as three 128-bit words each.  Needs npx % 4 == 0, frames
// 4-byte aligned and S, Q 16-byte aligned.  Returns the frames' luma total
// over the four pixels.  Frame i is at frame0 + i * fstride.
__device__ __forceinline__ unsigned long long learn_quad(const uint8_t *frame0, long long fstride, int nf,
                                                         long long quad, uint32_t *S, uint32_t *Q,
                                                         uint8_t *vmin, uint8_t *vmax, int first)
{
    unsigned long long luma = 0;
    uint4 *S4 = reinterpret_cast<uint4 *>(S) + 3 * quad;
    uint4 *Q4 = reinterpret_cast<uint4 *>(Q) + 3 * quad;
    uint32_t *mn4 = reinterpret_cast<uint32_t *>(vmin) + 3 * quad;
    uint32_t *mx4 = reinterpret_cast<uint32_t *>(vmax) + 3 * quad;
    uint32_t s[12], q[12], mn[3], mx[3];
    if (first) {
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] = q[k] = 0u;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            mn[k] = 0xffffffffu;
            mx[k] = 0u;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint4 a = S4[k], b = Q4[k];
            s[4 * k] = a.x; s[4 * k + 1] = a.y; s[4 * k + 2] = a.z; s[4 * k + 3] = a.w;
            q[4 * k] = b.x; q[4 * k + 1] = b.y; q[4 * k + 2] = b.z; q[4 * k + 3] = b.w;
            mn[k] = mn4[k];
            mx[k] = mx4[k];
        }
    }
    for (int i = 0; i < nf; ++i) {
        const uint32_t *f = reinterpret_cast<const uint32_t *>(frame0 + (long long)i * fstride) + 3 * quad;
        uint32_t wv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            wv[k] = __ldg(f + k);
            mn[k] = __vminu4(mn[k], wv[k]);
            mx[k] = __vmaxu4(mx[k], wv[k]);
        }
        uint32_t v[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            v[k] = (wv[k >> 2] >> (8 * (k & 3))) & 0xffu;
            s[k] += v[k];
            q[k] += v[k] * v[k];
        }
#pragma unroll
        for (int px = 0; px < 4; ++px)
            luma += (77u * v[3 * px] + 150u * v[3 * px + 1] + 29u * v[3 * px + 2] + 128u) >> 8;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        S4[k] = make_uint4(s[4 * k], s[4 * k + 1], s[4 * k + 2], s[4 * k + 3]);
        Q4[k] = make_uint4(q[4 * k], q[4 * k + 1], q[4 * k + 2], q[4 * k + 3]);
        mn4[k] = mn[k];
        mx4[k] = mx[k];
    }
    return luma;
}

__global__ void __launch_bounds__(kThreads) k_learn_accum4(const uint8_t *__restrict__ frames,
                                                           int nf, long long npx,
                                                           uint32_t *S, uint32_t *Q,
                                                           uint8_t *vmin, uint8_t *vmax,
                                                           int first, StreamState *st)
{
    __shared__ unsigned long long red[kThreads / 32];
    const long long quad = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long luma = 0;
    if (quad < npx / 4) luma = learn_quad(frames, npx * 3, nf, quad, S, Q, vmin, vmax, first);
    for (int o = 16; o > 0; o >>= 1) luma += __shfl_xor_sync(0xffffffffu, luma, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = luma;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        if (t) atomicAdd(&st->learn_luma, t);
    }
}

// One learning frame of each of several streams in one launch (a server round
// whose new streams are all learning at once): item e covers quads [quad0,
// quad0 + npx / 4) of the launch.  A warp whose lanes all belong to one item
// adds its luma total with one atomic, a warp across items lane by lane.
__global__ void __launch_bounds__(kThreads) k_learn_batch(const LearnItem *items, int nitems,
                                                          unsigned long long total)
{
    const unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    int e = -1;
    unsigned long long luma = 0;
    if (g < total) {
        int lo = 0, hi = nitems - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].quad0 <= g) lo = mid;
            else hi = mid - 1;
        }
        e = lo;
        const LearnItem it = items[e];
        luma = learn_quad(it.frame, 0, 1, (long long)(g - it.quad0), it.S, it.Q, it.vmin, it.vmax, it.first);
    }
    const int e0 = __shfl_sync(0xffffffffu, e, 0);
    if (__all_sync(0xffffffffu, e == e0)) {
        for (int o = 16; o > 0; o >>= 1) luma += __shfl_xor_sync(0xffffffffu, luma, o);
        if ((threadIdx.x & 31) == 0 && e0 >= 0 && luma) atomicAdd(&items[e0].st->learn_luma, luma);
    } else if (e >= 0 && luma) {
        atomicAdd(&items[e].st->learn_luma, luma);
    }
}

// Band edge predicate P(L): n L <= S and kd^2 (S - n L)^2 >= kn^2 D (low side).
__device__ __forceinline__ bool low_ok(long long L, long long s, long long n, long long kd2,
                                       long long knD)
{
    const long long gap = s - n * L;
    return gap >= 0 && kd2 * gap * gap >= knD;
}

__device__ __forceinline__ bool high_ok(long long H, long long s, long long n, long long kd2,
                                        long long knD)
{
    const long long gap = n * H - s;
    return gap >= 0 && kd2 * gap * gap >= knD;
}

// Band of one pixel-channel from its sums over n frames: [min(vmin, L_k) -
// delta, max(vmax, H_k) + delta] clamped to bytes, L_k / H_k the exact integer
// edges of mu -/+ k sigma with k = kn / kd.
__device__ __forceinline__ void band_of(long long s, long long q, long long nn, int kn, int kd, int delta,
                                        int vmin, int vmax, uint8_t *lo, uint8_t *hi)
{
    const long long D = nn * q - s * s;
    const long long kd2 = (long long)kd * kd, knD = (long long)kn * kn * D;
    // L' = max(L_k, -1) and H' = min(H_k, 256) give the same clamped band as
    // the unbounded edges; the predicates are monotone, so start from a
    // floating estimate and step to the exact edge.  The estimate is FP32
    // (FP64 is slow on this part) and lands within a step of the edge, so the
    // predicates are only evaluated next to it, where kd^2 gap^2 stays near
    // kn^2 D, below 2^63 for n <= 65535 and 8-bit k.
    const float ksig = (float)kn / (float)kd * sqrtf(__ll2float_rn(D)) / (float)nn;
    const float mu = __ll2float_rn(s) / (float)nn;
    const long long lmax = s / nn;   // largest L with n L <= S
    long long L = (long long)floorf(mu - ksig);
    L = max(-1ll, min(L, lmax));
    while (L + 1 <= lmax && low_ok(L + 1, s, nn, kd2, knD)) ++L;
    while (L > -1 && !low_ok(L, s, nn, kd2, knD)) --L;
    const long long hmin = (s + nn - 1) / nn;   // smallest H with n H >= S
    long long H = (long long)ceilf(mu + ksig);
    H = min(256ll, max(H, hmin));
    while (H - 1 >= hmin && high_ok(H - 1, s, nn, kd2, knD)) --H;
    while (H < 256 && !high_ok(H, s, nn, kd2, knD)) ++H;
    long long a = min((long long)vmin, L) - delta;
    long long b = max((long long)vmax, H) + delta;
    *lo = (uint8_t)max(0ll, min(255ll, a));
    *hi = (uint8_t)max(0ll, min(255ll, b));
}

__global__ void __launch_bounds__(kThreads) k_learn_band(const uint32_t *S, const uint32_t *Q,
                                                         const uint8_t *vmin, const uint8_t *vmax,
                                                         int n, int kn, int kd, int delta, int w,
                                                         int h, int fpitch, uint8_t *lo,
                                                         uint8_t *hi, StreamState *st)
{
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j == 0) {
        st->syref = st->learn_luma / (unsigned long long)n;
        st->sy = 0;
        st->best = 0;
        st->click = 0;
        st->hist_count = 0;
        st->hist_head = 0;
        st->frames = 0;
        st->lframes = 0;
        st->track_valid = 0;
        st->nlearn = (uint32_t)n;
        st->err = 0;
    }
    const long long count = (long long)w * h * 3;
    if (j >= count) return;
    const long long pxi = j / 3, c = j - pxi * 3;
    const long long y = pxi / w, x = pxi - y * w;
    const long long o = y * fpitch + 3 * x + c;
    band_of(S[j], Q[j], n, kn, kd, delta, vmin[j], vmax[j], lo + o, hi + o);
}

// k_relearn_band: after the last frame of a re-learning window, every pixel
// counted at least relearn_min times gets the band of its re-learning sums
// (n = its count), and every pixel's sums restart.  One thread per 16-px
// chunk of the streams whose window ends this tick.
__global__ void __launch_bounds__(kThreads) k_relearn_band(BatchDev b)
{
    for (int pc = blockIdx.x; pc < b.npieces; pc += gridDim.x) {
        const int4 piece = b.pieces[pc];
        const DevStream &D = b.ds[piece.x];
        if (b.io[piece.x].frame == nullptr || D.relearn_frames == 0) continue;
        const uint32_t f = D.st->lframe_p[b.phase];
        if (!relearn_window(f, D.relearn_period, D.relearn_frames) || f % (uint32_t)D.relearn_period != 0)
            continue;
        const int w = D.w, cpr = 2 * D.nwords;
        for (int u = piece.y + threadIdx.x; u < piece.z; u += blockDim.x) {
            const int y = chunk_row((uint32_t)u, D.cpr_magic), x0 = (u - y * cpr) * kChunkPx;
            for (int k = 0; k < kChunkPx && x0 + k < w; ++k) {
                const long long q = (long long)y * D.rpitch + x0 + k;
                const int n = D.rcnt[q];
                const long long o = (long long)y * D.fpitch + 3LL * (x0 + k);
                for (int ch = 0; ch < 3; ++ch) {
                    const long long j = 3 * q + ch;
                    if (n >= D.relearn_min && n > 0)
                        band_of(D.rS[j], D.rQ[j], n, D.bg_kn, D.bg_kd, D.bg_delta, D.rmin[j], D.rmax[j],
                                D.lo + o + ch, D.hi + o + ch);
                    D.rS[j] = 0;
                    D.rQ[j] = 0;
                    D.rmin[j] = 255;
                    D.rmax[j] = 0;
                }
                D.rcnt[q] = 0;
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_stats(const uint32_t *S, const uint32_t *Q, int n,
                                                    long long count, float *mean, float *stdv)
{
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const long long s = S[j];
    const long long num = (long long)n * (long long)Q[j] - s * s;
    const long long nn = (long long)n * (long long)n;
    if (mean) mean[j] = __int2float_rn((int)s) / __int2float_rn(n);
    if (stdv) stdv[j] = sqrtf(__ll2float_rn(num) / __ll2float_rn(nn));
}

cudaError_t launch_learn_accum(const uint8_t *frames, int nf, long long npx, uint32_t *S,
                               uint32_t *Q, uint8_t *vmin, uint8_t *vmax, int first,
                               StreamState *st, cudaStream_t cs)
{
    const bool vec = (npx % 4) == 0 && (reinterpret_cast<uintptr_t>(frames) & 3u) == 0 &&
                     (reinterpret_cast<uintptr_t>(S) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(Q) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(vmin) & 3u) == 0 &&
                     (reinterpret_cast<uintptr_t>(vmax) & 3u) == 0;
    if (vec) {
        const unsigned grid = (unsigned)((npx / 4 + kThreads - 1) / kThreads);
        k_learn_accum4<<<grid, kThreads, 0, cs>>>(frames, nf, npx, S, Q, vmin, vmax, first, st);
    } else {
        const unsigned grid = (unsigned)((npx + kThreads - 1) / kThreads);
        k_learn_accum<<<grid, kThreads, 0, cs>>>(frames, nf, npx, S, Q, vmin, vmax, first, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_learn_batch(const LearnItem *items, int nitems, unsigned long long total_quads,
                               cudaStream_t cs)
{
    if (nitems < 1 || total_quads == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((total_quads + kThreads - 1) / kThreads);
    k_learn_batch<<<grid, kThreads, 0, cs>>>(items, nitems, total_quads);
    return cudaGetLastError();
}

cudaError_t launch_learn_band(const uint32_t *S, const uint32_t *Q, const uint8_t *vmin,
                              const uint8_t *vmax, int n, int kn, int kd, int delta, int w,
                              int h, int fpitch, uint8_t *lo, uint8_t *hi, StreamState *st,
                              cudaStream_t cs)
{
    const long long count = (long long)w * h * 3;
    const unsigned grid = (unsigned)((count + kThreads - 1) / kThreads);
    k_learn_band<<<grid, kThreads, 0, cs>>>(S, Q, vmin, vmax, n, kn, kd, delta, w, h, fpitch,
                                            lo, hi, st);
    return cudaGetLastError();
}

cudaError_t launch_relearn_band(const BatchDev &b, cudaStream_t cs, int num_sms)
{
    (void)num_sms;
    if (!b.relearn) return cudaSuccess;
    k_relearn_band<<<b.npieces > 0 ? b.npieces : 1, kThreads, 0, cs>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_stats(const uint32_t *S, const uint32_t *Q, int n, long long count,
                         float *mean, float *stdv, cudaStream_t cs)
{
    const unsigned grid = (unsigned)((count + kThreads - 1) / kThreads);
    k_stats<<<grid, kThreads, 0, cs>>>(S, Q, n, count, mean, stdv);
    return cudaGetLastError();
}

}  // namespace hmi
