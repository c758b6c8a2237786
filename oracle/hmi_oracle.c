/*
 * hmi_oracle.c -- plain, slow, single-threaded CPU oracle of the per-frame
 * hand-isolation path of Magoules & Zou, "GPU Accelerated Contactless Human
 * Machine Interface for Driving Car" (arXiv 1907.04393).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline arm may load this library.  The product path (the
 * CUDA library and its Python binding) never calls it and shares no code,
 * header, table or helper with it.
 *
 * Every function states the passage of the paper it follows.  Where the paper
 * is silent, garbled or self-contradictory, the reading taken is written next
 * to the code as "Reading:".  All arithmetic on the per-pixel path is integer;
 * the only floating point values are the background mean/std and the pointer
 * centroid, each computed from exact integers with one correctly rounded IEEE
 * operation per step (compile with -ffp-contract=off so that no FMA changes
 * a rounding).
 *
 * Data layouts (all packed, no padding):
 *   frame      : H*W*3 bytes, RGB interleaved, pixel p = y*W + x at bytes 3p..3p+2
 *   per-channel: arrays of H*W*3 entries indexed like the frame bytes
 *   mask       : H*W bytes, 0 or 1
 *   labels     : H*W int32, -1 for background
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Pointer record (the Mouse module's output: position + click state).       */
/* Same field order as the library's public struct; defined independently.  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t valid, click;
    float x, y;
    uint32_t area;
    int32_t x0, y0, x1, y1;
    int32_t label;
} orc_pointer;

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }

/* ======================================================================== */
/* Step L -- background learning (Sec. 2: FIZI's background is learned       */
/* before the hand enters; Sec. 3.1 (i): per-pixel minimum and                */
/* maximum taken during that learning; Sec. 3.3 cites Gaussian background     */
/* models for the learning).                                                 */
/* ======================================================================== */

/* Per pixel-channel sums over n user-free frames: S = sum v, Q = sum v^2,
 * and the literal min / max of Sec. 3.1 (i).  Exact in uint32 for n <= 65535. */
void orc_learn_stats(const uint8_t *frames, int n, int w, int h,
                     uint32_t *S, uint32_t *Q, uint8_t *vmin, uint8_t *vmax)
{
    size_t count = (size_t)w * (size_t)h * 3u;
    for (size_t j = 0; j < count; ++j) {
        S[j] = 0; Q[j] = 0; vmin[j] = 255; vmax[j] = 0;
    }
    for (int i = 0; i < n; ++i) {
        const uint8_t *f = frames + (size_t)i * count;
        for (size_t j = 0; j < count; ++j) {
            uint32_t v = f[j];
            S[j] += v;
            Q[j] += v * v;
            if (v < vmin[j]) vmin[j] = (uint8_t)v;
            if (v > vmax[j]) vmax[j] = (uint8_t)v;
        }
    }
}

/* FP32 mean and standard deviation of the learned Gaussian per channel:
 *   mu    = (float)S / (float)n
 *   sigma = sqrtf( (float)(n*Q - S^2) / (float)(n*n) )
 * The int64 numerator and n*n are converted with C's correctly rounded
 * integer-to-float conversion. */
void orc_learn_meanstd(const uint32_t *S, const uint32_t *Q, int n, size_t count,
                       float *mean, float *stdv)
{
    for (size_t j = 0; j < count; ++j) {
        int64_t s = S[j], q = Q[j];
        int64_t num = (int64_t)n * q - s * s;
        int64_t nn = (int64_t)n * (int64_t)n;
        mean[j] = (float)s / (float)n;
        stdv[j] = sqrtf((float)num / (float)nn);
    }
}

/* Gaussian band edges, exact in integers.  With D = n*Q - S^2 and k = kn/kd:
 *   L_k = largest integer L with  n*L <= S  and  kd^2 (S - n L)^2 >= kn^2 D
 *         (i.e. L <= mu - k sigma)
 *   H_k = smallest integer H with n*H >= S  and  kd^2 (n H - S)^2 >= kn^2 D
 *         (i.e. H >= mu + k sigma)
 * Written as plain searches that step away from the mean until the condition
 * holds.  Reading: the paper names min/max only; the k-sigma widening follows
 * the Gaussian background models the paper cites for the learning step. */
int64_t orc_band_low(uint32_t S, uint32_t Q, int n, int kn, int kd)
{
    int64_t s = S, D = (int64_t)n * (int64_t)Q - s * s;
    int64_t L = s / n;                         /* largest L with n L <= S */
    for (;;) {
        int64_t gap = s - (int64_t)n * L;      /* >= 0 */
        if ((int64_t)kd * kd * gap * gap >= (int64_t)kn * kn * D) return L;
        --L;
    }
}

int64_t orc_band_high(uint32_t S, uint32_t Q, int n, int kn, int kd)
{
    int64_t s = S, D = (int64_t)n * (int64_t)Q - s * s;
    int64_t H = (s + n - 1) / n;               /* smallest H with n H >= S */
    for (;;) {
        int64_t gap = (int64_t)n * H - s;      /* >= 0 */
        if ((int64_t)kd * kd * gap * gap >= (int64_t)kn * kn * D) return H;
        ++H;
    }
}

/* Band used by the background test: the paper's literal [min, max] widened to
 * cover [mu - k sigma, mu + k sigma] and by a margin delta, clamped to bytes:
 *   lo = clamp(min(vmin, L_k) - delta, 0, 255)
 *   hi = clamp(max(vmax, H_k) + delta, 0, 255)
 * k = 0, delta = 0 gives the paper-literal band [vmin, vmax]. */
void orc_learn_band(const uint32_t *S, const uint32_t *Q,
                    const uint8_t *vmin, const uint8_t *vmax,
                    int n, size_t count, int kn, int kd, int delta,
                    uint8_t *lo, uint8_t *hi)
{
    for (size_t j = 0; j < count; ++j) {
        int64_t L = orc_band_low(S[j], Q[j], n, kn, kd);
        int64_t H = orc_band_high(S[j], Q[j], n, kn, kd);
        int64_t a = (L < vmin[j] ? L : vmin[j]) - delta;
        int64_t b = (H > vmax[j] ? H : vmax[j]) + delta;
        if (a < 0) a = 0;
        if (a > 255) a = 255;
        if (b < 0) b = 0;
        if (b > 255) b = 255;
        lo[j] = (uint8_t)a;
        hi[j] = (uint8_t)b;
    }
}

/* ======================================================================== */
/* Re-learning, Sec. 3.3: as the lighting drifts, part of the learning is    */
/* restarted from time to time.                                               */
/* Reading: with a period of P frames and a window of the last R of them,     */
/* every frame of a window adds the gain-corrected values of the pixels that  */
/* its background test classified as background (all three channels inside  */
/* the current band) to per-pixel re-learning sums S', Q', min', max' and a   */
/* count; after the window's last frame, every pixel counted at least         */
/* `min_cnt` times gets the band of those sums with n = its count (the same  */
/* formula as the initial band), the others keep theirs, and all sums are     */
/* reset.  Frames are counted from 1 after learning; frame f belongs to a     */
/* window iff (f - 1) mod P >= P - R, and ends it iff f mod P == 0.           */
/* ======================================================================== */

void orc_relearn_reset(size_t npx, uint32_t *S2, uint32_t *Q2, uint8_t *vmin2, uint8_t *vmax2,
                       uint8_t *cnt)
{
    for (size_t j = 0; j < npx * 3; ++j) {
        S2[j] = 0;
        Q2[j] = 0;
        vmin2[j] = 255;
        vmax2[j] = 0;
    }
    for (size_t p = 0; p < npx; ++p) cnt[p] = 0;
}

/* c: gain-corrected frame (npx x 3). */
void orc_relearn_accumulate(const uint8_t *c, const uint8_t *lo, const uint8_t *hi, size_t npx,
                            uint32_t *S2, uint32_t *Q2, uint8_t *vmin2, uint8_t *vmax2,
                            uint8_t *cnt)
{
    for (size_t p = 0; p < npx; ++p) {
        int background = 1;
        for (int k = 0; k < 3; ++k)
            if (c[3 * p + k] < lo[3 * p + k] || c[3 * p + k] > hi[3 * p + k]) background = 0;
        if (!background) continue;
        cnt[p] += 1;
        for (int k = 0; k < 3; ++k) {
            const uint32_t v = c[3 * p + k];
            S2[3 * p + k] += v;
            Q2[3 * p + k] += v * v;
            if (v < vmin2[3 * p + k]) vmin2[3 * p + k] = (uint8_t)v;
            if (v > vmax2[3 * p + k]) vmax2[3 * p + k] = (uint8_t)v;
        }
    }
}

void orc_relearn_apply(uint32_t *S2, uint32_t *Q2, uint8_t *vmin2, uint8_t *vmax2, uint8_t *cnt,
                       size_t npx, int min_cnt, int kn, int kd, int delta, uint8_t *lo, uint8_t *hi)
{
    for (size_t p = 0; p < npx; ++p) {
        const int n = cnt[p];
        if (n >= min_cnt && n > 0) {
            for (int k = 0; k < 3; ++k) {
                const size_t j = 3 * p + k;
                int64_t L = orc_band_low(S2[j], Q2[j], n, kn, kd);
                int64_t H = orc_band_high(S2[j], Q2[j], n, kn, kd);
                int64_t a = (L < vmin2[j] ? L : vmin2[j]) - delta;
                int64_t b = (H > vmax2[j] ? H : vmax2[j]) + delta;
                lo[j] = (uint8_t)(a < 0 ? 0 : (a > 255 ? 255 : a));
                hi[j] = (uint8_t)(b < 0 ? 0 : (b > 255 ? 255 : b));
            }
        }
    }
    orc_relearn_reset(npx, S2, Q2, vmin2, vmax2, cnt);
}

int orc_relearn_in_window(long long f, int period, int frames)
{
    return period > 0 && frames > 0 && (int)((f - 1) % period) >= period - frames;
}

/* ======================================================================== */
/* Mixture-of-Gaussians background (Sec. 2: FIZI's background is learned     */
/* with advanced machine learning; Sec. 3.3 cites Lee's adaptive              */
/* Gaussian mixture learning for it).  A variant of the learning (step L) and */
/* of the background test (step 2); the other steps are unchanged.            */
/* Reading, all integer, per pixel: K components kept in fitness order, each  */
/* a weight W (Q15), a mean per channel M (Q8), one variance V shared by the  */
/* three channels (Q4: level^2 * 16) and a match count C (C = 0: empty).  For */
/* the value x (3 bytes) of frame t, t counted from 1 over the learning and   */
/* then the running frames:                                                  */
/*  1. match: the first non-empty component with                             */
/*       ld^2 * sum_ch (256 x - M)^2 <= 3 * ln^2 * V * 4096                   */
/*     (the mean squared channel deviation at most lambda^2 V, lambda =      */
/*     ln / ld: within lambda standard deviations, read per channel as the   */
/*     band reads k; the joint distance with lambda = 2.5 would reject a     */
/*     tenth of pure-noise background pixels, the chi-square tail with 3     */
/*     degrees of freedom);                                                   */
/*  2. decision (running frames only, on the model before this frame): the   */
/*     pixel is background iff it matched component j and the weights of the */
/*     components before j sum to at most T percent of all weights (the      */
/*     fittest components that first exceed T are the background, after      */
/*     Stauffer and Grimson);                                                 */
/*  3. update with Lee's per-component rates: a matched component's count    */
/*     grows by one, and with r = min(C, N) its mean moves by (256 x - M) / r */
/*     and its variance by (D / 3 - V) / r, D the squared distance of step 1  */
/*     in Q4 (V clamped to [Vmin, 65535]); with no match the last component   */
/*     becomes a new one at x (M = 256 x, V = V0, C = 1, W = 0).  Then, with  */
/*     m = min(t, N), every weight moves by (32768 [matched or new] or 0      */
/*     [others] - W) / m.  Every division rounds half away from zero; the     */
/*     1/r and 1/m schedules make early estimates plain averages, and         */
/*     1/N is the learning rate alpha once enough frames are seen;            */
/*  4. the components are stably re-sorted: non-empty ones first, by        */
/*     W / sqrt(V), largest first (a before b iff W_a^2 V_b > W_b^2 V_a       */
/*     strictly), empty ones last.                                            */
/* State layout: planes of npx entries, W[k], M[k][ch], V[k], C[k] in this    */
/* order, k in storage (fitness) order.                                      */
/* ======================================================================== */

/* round(a / m) for m > 0, halves away from zero */
static int64_t div_round(int64_t a, int64_t m)
{
    const int64_t q = (2 * (a < 0 ? -a : a) + m) / (2 * m);
    return a < 0 ? -q : q;
}

void orc_mixture_step(uint16_t *W, uint16_t *M, uint16_t *V, uint16_t *C, size_t npx, int K,
                      const uint8_t *x, uint32_t t, int rate_n, int bg_pct, int ln, int ld,
                      uint32_t v_init, uint32_t v_min, uint8_t *fg1)
{
    const int64_t mt = (int64_t)(t < (uint32_t)rate_n ? t : (uint32_t)rate_n);
    for (size_t p = 0; p < npx; ++p) {
        const uint8_t *px = x + 3 * p;
        int j = -1;
        int64_t e[3] = {0, 0, 0};
        int64_t d2 = 0;
        for (int k = 0; k < K && j < 0; ++k) {
            if (C[k * npx + p] == 0) continue;
            int64_t dk[3], s2 = 0;
            for (int ch = 0; ch < 3; ++ch) {
                dk[ch] = 256 * (int64_t)px[ch] - (int64_t)M[(3 * k + ch) * npx + p];
                s2 += dk[ch] * dk[ch];
            }
            if ((int64_t)ld * ld * s2 <= 3 * (int64_t)ln * ln * (int64_t)V[k * npx + p] * 4096) {
                j = k;
                for (int ch = 0; ch < 3; ++ch) e[ch] = dk[ch];
                d2 = s2;
            }
        }
        if (fg1) {
            int64_t total = 0, before = 0;
            for (int k = 0; k < K; ++k) {
                total += W[k * npx + p];
                if (k < j) before += W[k * npx + p];
            }
            const int background = (j >= 0) && (100 * before <= (int64_t)bg_pct * total);
            fg1[p] = (uint8_t)!background;
        }
        if (j >= 0) {
            uint16_t *c = &C[j * npx + p];
            if (*c < 65535) *c += 1;
            const int64_t r = *c < rate_n ? *c : rate_n;
            for (int ch = 0; ch < 3; ++ch) {
                uint16_t *m = &M[(3 * j + ch) * npx + p];
                *m = (uint16_t)(*m + div_round(e[ch], r));
            }
            const int64_t target = div_round(d2, 3 * 4096);
            int64_t v = V[j * npx + p];
            v += div_round(target - v, r);
            if (v < (int64_t)v_min) v = v_min;
            if (v > 65535) v = 65535;
            V[j * npx + p] = (uint16_t)v;
        } else {
            j = K - 1;
            for (int ch = 0; ch < 3; ++ch) M[(3 * j + ch) * npx + p] = (uint16_t)(256 * px[ch]);
            V[j * npx + p] = (uint16_t)v_init;
            C[j * npx + p] = 1;
            W[j * npx + p] = 0;
        }
        for (int k = 0; k < K; ++k) {
            const int64_t w = W[k * npx + p];
            W[k * npx + p] = (uint16_t)(w + div_round((k == j ? 32768 : 0) - w, mt));
        }
        /* stable insertion sort, fittest first */
        for (int a = 1; a < K; ++a) {
            for (int b = a; b > 0; --b) {
                const uint64_t wb = W[b * npx + p], wp = W[(b - 1) * npx + p];
                const uint64_t vb = V[b * npx + p], vp = V[(b - 1) * npx + p];
                const int cb = C[b * npx + p] > 0, cp = C[(b - 1) * npx + p] > 0;
                const int fitter = cb && (!cp || wb * wb * vp > wp * wp * vb);
                if (!fitter) break;
                uint16_t tmp;
#define ORC_SWAP(arr, i0, i1) (tmp = arr[(i0)], arr[(i0)] = arr[(i1)], arr[(i1)] = tmp)
                ORC_SWAP(W, b * npx + p, (b - 1) * npx + p);
                ORC_SWAP(V, b * npx + p, (b - 1) * npx + p);
                ORC_SWAP(C, b * npx + p, (b - 1) * npx + p);
                for (int ch = 0; ch < 3; ++ch) ORC_SWAP(M, (3 * b + ch) * npx + p, (3 * (b - 1) + ch) * npx + p);
#undef ORC_SWAP
            }
        }
    }
}

/* Learning of the mixture: the update of every learning frame in order,     */
/* from an empty model (all planes zero), with t = 1..n.                     */
void orc_mixture_learn(const uint8_t *frames, int n, size_t npx, int K, uint16_t *W, uint16_t *M,
                       uint16_t *V, uint16_t *C, int rate_n, int ln, int ld, uint32_t v_init,
                       uint32_t v_min)
{
    memset(W, 0, sizeof(uint16_t) * npx * K);
    memset(M, 0, sizeof(uint16_t) * npx * K * 3);
    memset(V, 0, sizeof(uint16_t) * npx * K);
    memset(C, 0, sizeof(uint16_t) * npx * K);
    for (int f = 0; f < n; ++f)
        orc_mixture_step(W, M, V, C, npx, K, frames + (size_t)f * npx * 3, (uint32_t)(f + 1), rate_n,
                         100, ln, ld, v_init, v_min, NULL);
}

/* ======================================================================== */
/* Step 1 -- brightness correction (Sec. 2: the running step corrects the    */
/* brightness; Sec. 3.2: a filter acts on the luminosity component).          */
/* Reading: the frame is rescaled so that its total luma equals the mean      */
/* total luma of the learning frames.  A uniform RGB scale leaves hue          */
/* unchanged and moves luminosity, which is what the filter must do.          */
/* ======================================================================== */

/* Integer BT.601 luma of one pixel: (77 R + 150 G + 29 B + 128) >> 8. */
static uint32_t luma8(const uint8_t *p)
{
    return (77u * p[0] + 150u * p[1] + 29u * p[2] + 128u) >> 8;
}

/* SY = sum of luma8 over the frame. */
uint64_t orc_luma_sum(const uint8_t *frame, size_t npx)
{
    uint64_t sy = 0;
    for (size_t p = 0; p < npx; ++p) sy += luma8(frame + 3 * p);
    return sy;
}

/* Reference luma of the learned background: floor(sum_i SY(F_i) / n). */
uint64_t orc_ref_luma(const uint8_t *frames, int n, size_t npx)
{
    uint64_t tot = 0;
    for (int i = 0; i < n; ++i) tot += orc_luma_sum(frames + (size_t)i * npx * 3u, npx);
    return tot / (uint64_t)n;
}

/* Gain in Q16: round(SYref / SY), clamped to [gmin, gmax].  A black frame
 * (SY = 0) gets unit gain before the clamp. */
uint32_t orc_gain(uint64_t sy, uint64_t syref, uint32_t gmin, uint32_t gmax)
{
    uint64_t g = (sy == 0) ? 65536u : ((syref << 16) + sy / 2) / sy;
    if (g < gmin) g = gmin;
    if (g > gmax) g = gmax;
    return (uint32_t)g;
}

/* c' = min(255, (c * g + 2^15) >> 16) on every byte of the frame. */
void orc_apply_gain(const uint8_t *frame, size_t nbytes, uint32_t g, uint8_t *out)
{
    for (size_t j = 0; j < nbytes; ++j) {
        uint64_t c = ((uint64_t)frame[j] * g + 32768u) >> 16;
        out[j] = (uint8_t)(c > 255 ? 255 : c);
    }
}

/* ======================================================================== */
/* Steps 2-3 -- the three thresholded images of Sec. 3.1 and their AND.       */
/* ======================================================================== */

/* Integer hue, 1536 units per turn (256 per 60 degrees), of an RGB triple;
 * -1 when max == min (hue undefined).  HSV and HSL share this hue, so the
 * HSV of Sec. 3.1 (iii) item and the HSL of its text agree.
 * The sector is chosen by the first maximum in the order R, G, B; within a
 * sector the hexagonal hue is base + 256 * t / d, rounded half up:
 *   h = base - 256 + floor((512 (t + d) + d) / (2 d)),  wrapped to [0,1536). */
int orc_hue(int r, int g, int b)
{
    int mx = imax(r, imax(g, b)), mn = imin(r, imin(g, b));
    int d = mx - mn, base, t;
    if (d == 0) return -1;
    if (r == mx)      { base = 0;    t = g - b; }
    else if (g == mx) { base = 512;  t = b - r; }
    else              { base = 1024; t = r - g; }
    int h = base - 256 + (512 * (t + d) + d) / (2 * d);
    if (h < 0) h += 1536;
    if (h >= 1536) h -= 1536;
    return h;
}

/* Integer hue of every pixel of a frame (-1 where undefined). */
void orc_hue_map(const uint8_t *c, size_t npx, int16_t *out)
{
    for (size_t p = 0; p < npx; ++p) out[p] = (int16_t)orc_hue(c[3 * p], c[3 * p + 1], c[3 * p + 2]);
}

/* Hue inside the closed arc [a1, a2] taken modulo one turn (Sec. 3.1 (iii):
 * the skin hue lies between alpha1 and alpha2 modulo 2 pi): a1 > a2 means the
 * arc wraps through 0. */
static int in_arc(int h, int a1, int a2)
{
    return (a1 <= a2) ? (h >= a1 && h <= a2) : (h >= a1 || h <= a2);
}

/* Per-pixel masks on the gain-corrected frame c (H*W*3 bytes):
 *   fg1 (Sec. 3.1 (i))  : 1 iff some channel lies outside [lo_c, hi_c].
 *       Reading: the printed formula keeps pixels between min and max,
 *       which contradicts the text above it (pixels inside the range are the
 *       background and are dropped);
 *       the sentence is taken, with inclusive bounds.
 *   fg2 (Sec. 3.1 (ii)) : 1 iff max(c) - min(c) >= S (gray pixels removed).
 *       Reading: the printed formula has no comparison; the text
 *       (pixels whose channel spread is below a tolerance S are dropped) is
 *       taken.
 *   fg3 (Sec. 3.1 (iii)): 1 iff the hue is defined and inside the arc.
 *   raw = fg1 AND fg2 AND fg3 (the merging step of Sec. 3.1).
 * Any of the output pointers may be NULL. */
void orc_fg(const uint8_t *c, const uint8_t *lo, const uint8_t *hi, size_t npx,
            int gray_tol, int hue_lo, int hue_hi,
            uint8_t *fg1, uint8_t *fg2, uint8_t *fg3, uint8_t *raw)
{
    for (size_t p = 0; p < npx; ++p) {
        const uint8_t *px = c + 3 * p;
        int outside = 0;
        for (int k = 0; k < 3; ++k) {
            if (px[k] < lo[3 * p + k] || px[k] > hi[3 * p + k]) outside = 1;
        }
        int mx = imax(px[0], imax(px[1], px[2]));
        int mn = imin(px[0], imin(px[1], px[2]));
        int notgray = (mx - mn) >= gray_tol;
        int h = orc_hue(px[0], px[1], px[2]);
        int skin = (h >= 0) && in_arc(h, hue_lo, hue_hi);
        if (fg1) fg1[p] = (uint8_t)outside;
        if (fg2) fg2[p] = (uint8_t)notgray;
        if (fg3) fg3[p] = (uint8_t)skin;
        if (raw) raw[p] = (uint8_t)(outside && notgray && skin);
    }
}

/* ======================================================================== */
/* Step 4 -- morphology, Sec. 3.1: erosion and dilation clean away small     */
/* spurious blobs and join nearby regions.                                    */
/* Reading: 3x3 square element; opening (erode then dilate) open_iters times,  */
/* then closing (dilate then erode) close_iters times; pixels outside the      */
/* image are neutral (ignored) for both operators.                             */
/* ======================================================================== */

void orc_erode(const uint8_t *in, int w, int h, uint8_t *out)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int v = 1;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                    if (!in[(size_t)yy * w + xx]) v = 0;
                }
            out[(size_t)y * w + x] = (uint8_t)v;
        }
}

void orc_dilate(const uint8_t *in, int w, int h, uint8_t *out)
{
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            int v = 0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                    if (in[(size_t)yy * w + xx]) v = 1;
                }
            out[(size_t)y * w + x] = (uint8_t)v;
        }
}

void orc_morph(const uint8_t *raw, int w, int h, int open_iters, int close_iters,
               uint8_t *out)
{
    size_t npx = (size_t)w * (size_t)h;
    uint8_t *tmp = (uint8_t *)malloc(npx ? npx : 1);
    memcpy(out, raw, npx);
    for (int i = 0; i < open_iters; ++i) {
        orc_erode(out, w, h, tmp);
        orc_dilate(tmp, w, h, out);
    }
    for (int i = 0; i < close_iters; ++i) {
        orc_dilate(out, w, h, tmp);
        orc_erode(tmp, w, h, out);
    }
    free(tmp);
}

/* ======================================================================== */
/* Step 5a -- connected components (Sec. 2 Mouse module: it follows the      */
/* hand's region of the binary image).                                        */
/* Reading: 8-connectivity; every component is labelled with the smallest     */
/* linear index y*W + x of its pixels; background is -1.  Plain flood fill:   */
/* scanning in raster order, the first unlabelled foreground pixel of a       */
/* component is its smallest index.  Returns the number of components.       */
/* ======================================================================== */
int orc_label(const uint8_t *mask, int w, int h, int32_t *labels)
{
    size_t npx = (size_t)w * (size_t)h;
    int32_t *queue = (int32_t *)malloc((npx ? npx : 1) * sizeof(int32_t));
    int ncomp = 0;
    for (size_t p = 0; p < npx; ++p) labels[p] = -1;
    for (size_t p = 0; p < npx; ++p) {
        if (!mask[p] || labels[p] >= 0) continue;
        size_t head = 0, tail = 0;
        labels[p] = (int32_t)p;
        queue[tail++] = (int32_t)p;
        while (head < tail) {
            int32_t q = queue[head++];
            int qy = q / w, qx = q % w;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int yy = qy + dy, xx = qx + dx;
                    if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                    size_t r = (size_t)yy * w + xx;
                    if (mask[r] && labels[r] < 0) {
                        labels[r] = (int32_t)p;
                        queue[tail++] = (int32_t)r;
                    }
                }
        }
        ++ncomp;
    }
    free(queue);
    return ncomp;
}

/* ======================================================================== */
/* Step 5b -- pointer (Sec. 2: the Mouse module turns the hand zone into a   */
/* pointer, whose movement and clicked / not-clicked state the Interface     */
/* reads).                                                                    */
/* Reading: the hand is the largest component (ties: smaller label); the      */
/* pointer is its centroid with pixel centres at integer coordinates, and its */
/* inclusive bounding box; valid iff area >= min_area.  With no component:    */
/* valid 0, area 0, label -1, box -1, x = y = -1.                             */
/* ======================================================================== */
/* Pointer (Sec. 2 Mouse module) from a label image.  Reading: the hand is the
 * largest component (ties: the smaller label).  With tracking (Sec. 2: the
 * Mouse module "tracks" the hand zone; max_dist > 0) and a tracked point from
 * an earlier valid frame (track[0] != 0, point track[1], track[2]), the hand is
 * instead the component of at least min_area pixels whose bounding box is
 * nearest that point, the distance being max(0, x0 - tx, tx - x1) +
 * max(0, y0 - ty, ty - y1) and at most max_dist (ties: the larger area, then
 * the smaller label); with no such component, the largest.  A valid pointer
 * then moves the tracked point to its rounded centroid,
 * floor((2 sum + area) / (2 area)) per axis.  track may be NULL (no tracking). */
void orc_pointer_select(const int32_t *labels, int w, int h, uint32_t min_area, int max_dist,
                        int32_t *track, orc_pointer *out)
{
    size_t npx = (size_t)w * (size_t)h;
    /* per-label accumulators, indexed by the label (= a pixel index) */
    uint32_t *area = (uint32_t *)calloc(npx ? npx : 1, sizeof(uint32_t));
    uint64_t *sx = (uint64_t *)calloc(npx ? npx : 1, sizeof(uint64_t));
    uint64_t *sy = (uint64_t *)calloc(npx ? npx : 1, sizeof(uint64_t));
    int32_t *bx0 = (int32_t *)malloc((npx ? npx : 1) * sizeof(int32_t));
    int32_t *by0 = (int32_t *)malloc((npx ? npx : 1) * sizeof(int32_t));
    int32_t *bx1 = (int32_t *)malloc((npx ? npx : 1) * sizeof(int32_t));
    int32_t *by1 = (int32_t *)malloc((npx ? npx : 1) * sizeof(int32_t));
    for (size_t p = 0; p < npx; ++p) {
        int32_t l = labels[p];
        if (l < 0) continue;
        int y = (int)(p / (size_t)w), x = (int)(p % (size_t)w);
        if (area[l] == 0) { bx0[l] = x; bx1[l] = x; by0[l] = y; by1[l] = y; }
        area[l] += 1;
        sx[l] += (uint64_t)x;
        sy[l] += (uint64_t)y;
        if (x < bx0[l]) bx0[l] = x;
        if (x > bx1[l]) bx1[l] = x;
        if (y < by0[l]) by0[l] = y;
        if (y > by1[l]) by1[l] = y;
    }
    int32_t best = -1;
    for (size_t l = 0; l < npx; ++l) {
        if (area[l] == 0) continue;
        if (best < 0 || area[l] > area[best]) best = (int32_t)l;  /* ascending l: ties keep the smaller */
    }
    if (track && max_dist > 0 && track[0]) {
        int32_t tb = -1;
        long long tbd = 0;
        for (size_t l = 0; l < npx; ++l) {
            if (area[l] == 0 || area[l] < min_area) continue;
            long long dx = 0, dy = 0;
            if (track[1] < bx0[l]) dx = bx0[l] - track[1];
            if (track[1] > bx1[l]) dx = track[1] - bx1[l];
            if (track[2] < by0[l]) dy = by0[l] - track[2];
            if (track[2] > by1[l]) dy = track[2] - by1[l];
            const long long d = dx + dy;
            if (d > max_dist) continue;
            /* ascending l: equal distance and area keep the smaller label */
            if (tb < 0 || d < tbd || (d == tbd && area[l] > area[tb])) { tb = (int32_t)l; tbd = d; }
        }
        if (tb >= 0) best = tb;
    }
    memset(out, 0, sizeof(*out));
    if (best < 0) {
        out->valid = 0; out->area = 0; out->label = -1;
        out->x0 = out->y0 = out->x1 = out->y1 = -1;
        out->x = -1.0f; out->y = -1.0f;
    } else {
        out->area = area[best];
        out->label = best;
        out->valid = area[best] >= min_area;
        out->x = (float)((double)sx[best] / (double)area[best]);
        out->y = (float)((double)sy[best] / (double)area[best]);
        out->x0 = bx0[best]; out->y0 = by0[best];
        out->x1 = bx1[best]; out->y1 = by1[best];
        if (track && out->valid) {
            track[0] = 1;
            track[1] = (int32_t)((2 * sx[best] + area[best]) / (2 * (uint64_t)area[best]));
            track[2] = (int32_t)((2 * sy[best] + area[best]) / (2 * (uint64_t)area[best]));
        }
    }
    free(area); free(sx); free(sy); free(bx0); free(by0); free(bx1); free(by1);
}

void orc_pointer_from_labels(const int32_t *labels, int w, int h, uint32_t min_area,
                             orc_pointer *out)
{
    orc_pointer_select(labels, w, h, min_area, 0, NULL, out);
}

/* Click state machine of one stream (reading of the pointer's clicked / not-clicked state).
 * hist holds the areas of the last `window` valid frames, oldest first
 * (hist_count entries).  For a valid frame, A_ref = max(hist):
 *   click := 1 if 100*area < on_pct  * A_ref
 *   click := 0 if 100*area > off_pct * A_ref   (otherwise unchanged)
 *   no history yet => click := 0
 * then the area is appended (dropping the oldest beyond `window`).
 * An invalid frame changes nothing.  Writes the state into out->click. */
void orc_click_update(int32_t *click, uint32_t *hist, int32_t *hist_count, int window,
                      int on_pct, int off_pct, orc_pointer *out)
{
    if (out->valid) {
        if (*hist_count == 0) {
            *click = 0;
        } else {
            uint64_t aref = 0;
            for (int i = 0; i < *hist_count; ++i) if (hist[i] > aref) aref = hist[i];
            uint64_t a100 = 100u * (uint64_t)out->area;
            if (a100 < (uint64_t)on_pct * aref) *click = 1;
            else if (a100 > (uint64_t)off_pct * aref) *click = 0;
        }
        if (window > 0) {
            if (*hist_count == window) {
                memmove(hist, hist + 1, (size_t)(window - 1) * sizeof(uint32_t));
                hist[window - 1] = out->area;
            } else {
                hist[(*hist_count)++] = out->area;
            }
        }
    }
    out->click = *click;
}

/* A stream's mixture as the whole-path function takes it: the planes of      */
/* orc_mixture_step, the number t of the frame being processed and the        */
/* parameters.                                                                */
typedef struct {
    uint16_t *W, *M, *V, *C;
    int K;
    uint32_t t;
    int rate_n, bg_pct, ln, ld;
    uint32_t v_init, v_min;
} orc_mixture;

/* ======================================================================== */
/* One frame through the whole path (Sec. 2 running step):                    */
/* brightness -> three masks -> AND -> morphology -> components -> pointer.  */
/* mask_out / labels_out may be NULL.  mix NULL: the band test with lo / hi;  */
/* else the mixture's test on the frame number mix->t, then its update.       */
/* ======================================================================== */
void orc_process_frame_bg(const uint8_t *frame, int w, int h,
                       const uint8_t *lo, const uint8_t *hi, const orc_mixture *mix, uint64_t syref,
                       int gray_tol, int hue_lo, int hue_hi,
                       int open_iters, int close_iters,
                       uint32_t gain_min, uint32_t gain_max, uint32_t min_area,
                       int on_pct, int off_pct, int window,
                       int track_max_dist, int32_t *track,
                       int32_t *click, uint32_t *hist, int32_t *hist_count,
                       uint8_t *mask_out, int32_t *labels_out, orc_pointer *pointer_out,
                       uint32_t *gain_out)
{
    size_t npx = (size_t)w * (size_t)h;
    uint8_t *c = (uint8_t *)malloc(npx * 3 + 1);
    uint8_t *raw = (uint8_t *)malloc(npx + 1);
    uint8_t *mask = (uint8_t *)malloc(npx + 1);
    int32_t *labels = (int32_t *)malloc((npx + 1) * sizeof(int32_t));
    uint64_t sy = orc_luma_sum(frame, npx);
    uint32_t g = orc_gain(sy, syref, gain_min, gain_max);
    orc_apply_gain(frame, npx * 3, g, c);
    if (mix) {
        /* background test by the mixture (on the model before this frame), */
        /* then its update; the gray and hue tests as for the band            */
        uint8_t *fg1 = (uint8_t *)malloc(npx + 1);
        uint8_t *fg2 = (uint8_t *)malloc(npx + 1);
        uint8_t *fg3 = (uint8_t *)malloc(npx + 1);
        orc_mixture_step(mix->W, mix->M, mix->V, mix->C, npx, mix->K, c, mix->t, mix->rate_n,
                         mix->bg_pct, mix->ln, mix->ld, mix->v_init, mix->v_min, fg1);
        orc_fg(c, c, c, npx, gray_tol, hue_lo, hue_hi, NULL, fg2, fg3, NULL);
        for (size_t p = 0; p < npx; ++p) raw[p] = (uint8_t)(fg1[p] && fg2[p] && fg3[p]);
        free(fg1); free(fg2); free(fg3);
    } else {
        orc_fg(c, lo, hi, npx, gray_tol, hue_lo, hue_hi, NULL, NULL, NULL, raw);
    }
    orc_morph(raw, w, h, open_iters, close_iters, mask);
    orc_label(mask, w, h, labels);
    orc_pointer_select(labels, w, h, min_area, track_max_dist, track, pointer_out);
    orc_click_update(click, hist, hist_count, window, on_pct, off_pct, pointer_out);
    if (mask_out) memcpy(mask_out, mask, npx);
    if (labels_out) memcpy(labels_out, labels, npx * sizeof(int32_t));
    if (gain_out) *gain_out = g;
    free(c); free(raw); free(mask); free(labels);
}

void orc_process_frame(const uint8_t *frame, int w, int h,
                       const uint8_t *lo, const uint8_t *hi, uint64_t syref,
                       int gray_tol, int hue_lo, int hue_hi,
                       int open_iters, int close_iters,
                       uint32_t gain_min, uint32_t gain_max, uint32_t min_area,
                       int on_pct, int off_pct, int window,
                       int track_max_dist, int32_t *track,
                       int32_t *click, uint32_t *hist, int32_t *hist_count,
                       uint8_t *mask_out, int32_t *labels_out, orc_pointer *pointer_out,
                       uint32_t *gain_out)
{
    orc_process_frame_bg(frame, w, h, lo, hi, NULL, syref, gray_tol, hue_lo, hue_hi, open_iters,
                         close_iters, gain_min, gain_max, min_area, on_pct, off_pct, window,
                         track_max_dist, track, click, hist, hist_count, mask_out, labels_out,
                         pointer_out, gain_out);
}

/* ======================================================================== */
/* Interface module (Sec. 2: fed by the Mouse module, it finds which         */
/* interface zone holds the pointer; each zone maps to an event)             */
/* and the driving application (Sec. 4: rotating the hand about a virtual     */
/* wheel steers left or right; the speed is the third control).              */
/* Reading, headless and integer: the pointer point is the rounded centroid   */
/* of a valid pointer (floor((2 sum + area) / (2 area)) per axis); the zone   */
/* is the first listed inclusive rectangle that contains it; the point is on  */
/* the wheel when r_in^2 <= dx^2 + dy^2 <= r_out^2 around the wheel centre;   */
/* its angle is the "diamond" pseudo-angle, 4096 units per turn, 0 at the     */
/* top, growing clockwise (1024 per quadrant: 1024 u / (u + v) in the first,  */
/* u = dx, v = -dy, and likewise in the others, floor division); steer is     */
/* that angle in (-2048, 2048]; left and right are steer beyond the dead      */
/* zone, and throttle is the click state (the closed hand), all three only    */
/* on the wheel.                                                              */
/* ======================================================================== */
int32_t orc_diamond_angle(int64_t dx, int64_t dy)
{
    const int64_t u = dx, v = -dy;
    if (u == 0 && v == 0) return 0;
    if (u >= 0 && v > 0) return (int32_t)(1024 * u / (u + v));
    if (u > 0 && v <= 0) return (int32_t)(1024 + 1024 * (-v) / (u - v));
    if (u <= 0 && v < 0) return (int32_t)(2048 + 1024 * (-u) / (-u - v));
    return (int32_t)(3072 + 1024 * v / (v - u));
}

/* valid, (px, py): the pointer point; zones: nzones x (x0, y0, x1, y1, event);
 * wheel: (on, cx, cy, r_in, r_out, dead_zone).
 * out: (zone, event, on_wheel, steer, left, right, throttle). */
void orc_interface_event(int valid, int32_t px, int32_t py, int click, const int32_t *zones,
                         int nzones, const int32_t *wheel, int32_t *out)
{
    for (int k = 0; k < 7; ++k) out[k] = 0;
    out[0] = -1;
    out[1] = -1;
    if (!valid) return;
    for (int z = 0; z < nzones; ++z) {
        const int32_t *Z = zones + 5 * z;
        if (px >= Z[0] && px <= Z[2] && py >= Z[1] && py <= Z[3]) {
            out[0] = z;
            out[1] = Z[4];
            break;
        }
    }
    if (!wheel[0]) return;
    const int64_t dx = (int64_t)px - wheel[1], dy = (int64_t)py - wheel[2];
    const int64_t d2 = dx * dx + dy * dy;
    const int64_t r0 = wheel[3], r1 = wheel[4];
    if (d2 < r0 * r0 || d2 > r1 * r1) return;
    int32_t a = orc_diamond_angle(dx, dy);
    int32_t steer = a > 2048 ? a - 4096 : a;
    out[2] = 1;
    out[3] = steer;
    out[4] = steer < -wheel[5];
    out[5] = steer > wheel[5];
    out[6] = click != 0;
}
