/*
 * gen.c -- seeded synthetic camera frames shaped like the workloads of the
 * contactless interface of arXiv 1907.04393 (a camera watching a static scene
 * in which a hand moves, with brightness changes; Sec. 2 and Sec. 3.2).
 *
 * This module only makes input bytes.  It holds none of the method's
 * arithmetic (no brightness correction, thresholds, morphology or labelling)
 * and is the one piece of code that both the CUDA path's tests and the CPU
 * oracle consume.
 *
 * Determinism: every random number is a pure function of (seed, frame,
 * pixel, channel) through a counter-based splitmix64 hash, so the bytes do not
 * depend on thread count or evaluation order.  Gaussian variates use a scaled
 * sum of four uniforms (Irwin-Hall), which needs no transcendental function.
 *
 * Scene recipe (per configuration `cfg` 1..5 and stream index `s`):
 *   background  smooth gradient R = 40 + 100 x/W, G = 60 + 120 y/H,
 *               B = 200 - 80 x/W (+ per-stream offsets in batched configs)
 *               plus i.i.d. N(0, sigma) camera noise per channel and frame
 *   skin        per pixel and frame Y ~ U[80,200], Cb ~ N(110,4),
 *               Cr ~ N(150,4), converted with full-range BT.601 to RGB
 *   hand        filled ellipse with full axes 40x60 at 320x240, scaled by
 *               W/320, centre on a Lissajous path
 *               x = W/2 + 0.35 W sin(2 pi (t + px)/97),
 *               y = H/2 + 0.35 H sin(2 pi (t + py)/61 + pi/4)
 *   brightness  a global multiply on RGB, applied last, then round + clamp
 * Per configuration:
 *   1  320x240, sigma 3, brightness 1 + 0.1 sin(2 pi t/60)
 *   2  640x480, sigma 3, static face ellipse 90x120 (also in the learning
 *      frames), brightness ramp 0.7 -> 1.3 over 300 frames, salt and pepper
 *      on 0.5 % of pixels (run frames), hand area x1.3 (open) / x0.7 (closed)
 *      alternating every 20 frames
 *   3  1920x1080, sigma 5, two hands (second at 0.7x axes), gradient drift
 *      +1 level per 50 frames, brightness 1 + 0.15 sin(2 pi 2 t/30)
 *   4  64 streams: 32/16/12/4 at 320x240/640x480/1280x720/1920x1080
 *   5  256 streams: the same mix times four
 * Streams of configs 4 and 5 draw their own gradient offsets, path phases
 * and brightness phase from their seed.  Learning frames contain no hand,
 * no salt and pepper and unit brightness.
 */
#include <stdint.h>
#include <math.h>
#include <string.h>

#define PI_D 3.14159265358979323846

static uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* uniform double in [0, 1) from (key, counter) */
static double u01(uint64_t key, uint64_t ctr)
{
    return (double)(mix64(key ^ mix64(ctr)) >> 11) * (1.0 / 9007199254740992.0);
}

/* approximately standard normal: (sum of 4 uniforms - 2) * sqrt(3) */
static double nrm(uint64_t key, uint64_t ctr)
{
    double s = u01(key, 4 * ctr) + u01(key, 4 * ctr + 1) + u01(key, 4 * ctr + 2) +
               u01(key, 4 * ctr + 3);
    return (s - 2.0) * 1.7320508075688772;
}

static int clamp255(double v)
{
    double r = floor(v + 0.5);
    if (r < 0) return 0;
    if (r > 255) return 255;
    return (int)r;
}

int synth_num_streams(int cfg)
{
    if (cfg == 4) return 64;
    if (cfg == 5) return 256;
    if (cfg >= 1 && cfg <= 3) return 1;
    return 0;
}

/* Resolution of stream s of configuration cfg; returns 0 on success. */
int synth_shape(int cfg, int s, int *w, int *h)
{
    static const int W[4] = {320, 640, 1280, 1920}, H[4] = {240, 480, 720, 1080};
    int k;
    if (cfg == 1) k = 0;
    else if (cfg == 2) k = 1;
    else if (cfg == 3) k = 3;
    else if (cfg == 4 || cfg == 5) {
        int m = (cfg == 4) ? 1 : 4;
        if (s < 0 || s >= 64 * m) return -1;
        if (s < 32 * m) k = 0;
        else if (s < 48 * m) k = 1;
        else if (s < 60 * m) k = 2;
        else k = 3;
    } else return -1;
    if (cfg <= 3 && s != 0) return -1;
    *w = W[k];
    *h = H[k];
    return 0;
}

typedef struct {
    int w, h, cfg, s;
    uint64_t seed;
    double sigma;
    double off[3];      /* gradient offsets */
    double phx, phy;    /* Lissajous phases (frames) */
    double phb;         /* brightness phase (frames) */
} scene;

static int scene_init(scene *sc, int cfg, int s)
{
    memset(sc, 0, sizeof(*sc));
    if (synth_shape(cfg, s, &sc->w, &sc->h)) return -1;
    sc->cfg = cfg;
    sc->s = s;
    sc->seed = 1907043930ull + 1000ull * (uint64_t)cfg + (uint64_t)s;
    sc->sigma = (cfg == 3) ? 5.0 : 3.0;
    if (cfg >= 4) {
        uint64_t k = mix64(sc->seed ^ 0x5eedull);
        for (int c = 0; c < 3; ++c) sc->off[c] = -15.0 + 30.0 * u01(k, (uint64_t)c);
        sc->phx = 97.0 * u01(k, 3);
        sc->phy = 61.0 * u01(k, 4);
        sc->phb = 60.0 * u01(k, 5);
    }
    return 0;
}

/* Ellipses present in run frame t: centre, semi-axes.  Returns the count. */
static int hands(const scene *sc, int t, double e[][4], int *open_state)
{
    double sc_w = (double)sc->w / 320.0;
    double a = 20.0 * sc_w, b = 30.0 * sc_w;
    double cx = sc->w / 2.0 + 0.35 * sc->w * sin(2.0 * PI_D * (t + sc->phx) / 97.0);
    double cy = sc->h / 2.0 + 0.35 * sc->h * sin(2.0 * PI_D * (t + sc->phy) / 61.0 + PI_D / 4.0);
    int open = 1;
    if (sc->cfg == 2) {
        open = ((t / 20) % 2) == 0;
        double f = open ? sqrt(1.3) : sqrt(0.7);
        a *= f;
        b *= f;
    }
    if (open_state) *open_state = open;
    e[0][0] = cx; e[0][1] = cy; e[0][2] = a; e[0][3] = b;
    if (sc->cfg == 3) {
        double cx2 = sc->w / 2.0 - 0.3 * sc->w * sin(2.0 * PI_D * (t + 40.0) / 89.0);
        double cy2 = sc->h / 2.0 + 0.3 * sc->h * sin(2.0 * PI_D * (t + 10.0) / 67.0);
        e[1][0] = cx2; e[1][1] = cy2; e[1][2] = 0.7 * a; e[1][3] = 0.7 * b;
        return 2;
    }
    return 1;
}

static double brightness(const scene *sc, int t)
{
    switch (sc->cfg) {
    case 1: return 1.0 + 0.1 * sin(2.0 * PI_D * t / 60.0);
    case 2: return 0.7 + 0.6 * (double)t / 299.0;
    case 3: return 1.0 + 0.15 * sin(2.0 * PI_D * 2.0 * t / 30.0);
    default: return 1.0 + 0.1 * sin(2.0 * PI_D * (t + sc->phb) / 60.0);
    }
}

static int inside(double x, double y, const double e[4])
{
    double u = (x - e[0]) / e[2], v = (y - e[1]) / e[3];
    return u * u + v * v <= 1.0;
}

static void skin_rgb(uint64_t key, uint64_t ctr, double rgb[3])
{
    double Y = 80.0 + 120.0 * u01(key, 3 * ctr);
    double Cb = 110.0 + 4.0 * nrm(key, 3 * ctr + 1);
    double Cr = 150.0 + 4.0 * nrm(key, 3 * ctr + 2);
    rgb[0] = Y + 1.402 * (Cr - 128.0);
    rgb[1] = Y - 0.344136 * (Cb - 128.0) - 0.714136 * (Cr - 128.0);
    rgb[2] = Y + 1.772 * (Cb - 128.0);
}

/* Frame t of stream s of configuration cfg into out (H*W*3 bytes, packed RGB).
 * learn != 0 gives learning frame t (no user); learn == 0 gives run frame t. */
int synth_frame(int cfg, int s, int t, int learn, uint8_t *out)
{
    scene sc;
    if (scene_init(&sc, cfg, s)) return -1;
    const int w = sc.w, h = sc.h;
    double e[2][4];
    int nh = learn ? 0 : hands(&sc, t, e, NULL);
    double br = learn ? 1.0 : brightness(&sc, t);
    double drift = (!learn && cfg == 3) ? (double)(t / 50) : 0.0;
    /* face ellipse of configuration 2: 90x120 full axes, static */
    double face[4] = {0.22 * w, 0.32 * h, 45.0, 60.0};
    uint64_t frame_id = (learn ? 0x100000ull : 0x200000ull) + (uint64_t)t;
    uint64_t knoise = mix64(sc.seed ^ (frame_id << 20) ^ 0xA1ull);
    uint64_t kskin = mix64(sc.seed ^ (frame_id << 20) ^ 0xB2ull);
    uint64_t ksalt = mix64(sc.seed ^ (frame_id << 20) ^ 0xC3ull);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y) {
        for (int x = 0; x < w; ++x) {
            uint64_t p = (uint64_t)y * (uint64_t)w + (uint64_t)x;
            double rgb[3];
            int skin = 0;
            for (int k = 0; k < nh; ++k) skin |= inside(x, y, e[k]);
            if (cfg == 2 && inside(x, y, face)) skin = 1;
            if (skin) {
                skin_rgb(kskin, p, rgb);
            } else {
                rgb[0] = 40.0 + 100.0 * x / w + sc.off[0] + drift;
                rgb[1] = 60.0 + 120.0 * y / h + sc.off[1] + drift;
                rgb[2] = 200.0 - 80.0 * x / w + sc.off[2] + drift;
                for (int c = 0; c < 3; ++c) rgb[c] += sc.sigma * nrm(knoise, 3 * p + (uint64_t)c);
            }
            uint8_t *o = out + 3 * p;
            for (int c = 0; c < 3; ++c) o[c] = (uint8_t)clamp255(rgb[c] * br);
            if (!learn && cfg == 2 && u01(ksalt, 2 * p) < 0.005) {
                uint8_t v = u01(ksalt, 2 * p + 1) < 0.5 ? 0 : 255;
                o[0] = o[1] = o[2] = v;
            }
        }
    }
    return 0;
}

/* Ground truth of run frame t: up to 2 ellipses (cx, cy, a, b) and the open
 * state of the hand.  Returns the number of hands, or -1. */
int synth_truth(int cfg, int s, int t, double *ellipses, int *open_state)
{
    scene sc;
    if (scene_init(&sc, cfg, s)) return -1;
    double e[2][4];
    int n = hands(&sc, t, e, open_state);
    for (int k = 0; k < n; ++k) for (int j = 0; j < 4; ++j) ellipses[4 * k + j] = e[k][j];
    return n;
}

/* Brightness multiplier of run frame t (ground truth for tests). */
double synth_brightness(int cfg, int s, int t)
{
    scene sc;
    if (scene_init(&sc, cfg, s)) return -1.0;
    return brightness(&sc, t);
}
