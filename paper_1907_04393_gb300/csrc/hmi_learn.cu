// hmi_learn.cu -- background learning (Sec. 2: the FIZI module learns the
// background without the user; Sec. 3.1 (i): minimum and maximum values learned
// in the initialisation step; Sec. 3.3: Gaussian background models).
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
// 4-byte aligned and S, Q 16-byte aligned.
__global__ void __launch_bounds__(kThreads) k_learn_accum4(const uint8_t *__restrict__ frames,
                                                           int nf, long long npx,
                                                           uint32_t *S, uint32_t *Q,
                                                           uint8_t *vmin, uint8_t *vmax,
                                                           int first, StreamState *st)
{
    __shared__ unsigned long long red[kThreads / 32];
    const long long quad = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long luma = 0;
    if (quad < npx / 4) {
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
            const uint32_t *f = reinterpret_cast<const uint32_t *>(frames + (long long)i * npx * 3) + 3 * quad;
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
        st->err = 0;
    }
    const long long count = (long long)w * h * 3;
    if (j >= count) return;
    const long long s = S[j], nn = n;
    const long long D = nn * (long long)Q[j] - s * s;
    const long long kd2 = (long long)kd * kd, knD = (long long)kn * kn * D;
    // L' = max(L_k, -1) and H' = min(H_k, 256) give the same clamped band as
    // the unbounded edges; the predicates are monotone, so start from a
    // floating estimate and step to the exact edge.  The estimate is FP32
    // (FP64 is slow on this part) and lands within a step of the edge, so the
    // predicates are only evaluated next to it, where kd^2 gap^2 stays near
    // kn^2 D, below 2^63 for n <= 65535 and 8-bit k.
    const float ksig = (float)kn / (float)kd * sqrtf(__ll2float_rn(D)) / (float)n;
    const float mu = __ll2float_rn(s) / (float)n;
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
    long long a = min((long long)vmin[j], L) - delta;
    long long b = max((long long)vmax[j], H) + delta;
    a = max(0ll, min(255ll, a));
    b = max(0ll, min(255ll, b));
    const long long pxi = j / 3, c = j - pxi * 3;
    const long long y = pxi / w, x = pxi - y * w;
    const long long o = y * fpitch + 3 * x + c;
    lo[o] = (uint8_t)a;
    hi[o] = (uint8_t)b;
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

cudaError_t launch_stats(const uint32_t *S, const uint32_t *Q, int n, long long count,
                         float *mean, float *stdv, cudaStream_t cs)
{
    const unsigned grid = (unsigned)((count + kThreads - 1) / kThreads);
    k_stats<<<grid, kThreads, 0, cs>>>(S, Q, n, count, mean, stdv);
    return cudaGetLastError();
}

}  // namespace hmi
