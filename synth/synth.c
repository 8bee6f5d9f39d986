/*
 * Seeded synthetic electron-micrograph series.
 *
 * Stand-in for the UHV-HRTEM aluminium-oxidation frames of the paper's
 * experiments (Section "Electron microscopy data"), which are not available:
 * a square lattice of Gaussian atom columns plus a few large low-contrast
 * blobs (so that coarse pyramid levels keep structure), moved per frame by a
 * random-walk translation and a smooth sinusoidal distortion, sampled at
 * pixel centres, optionally under Poisson shot noise.
 *
 * This module is an input producer only: it contains none of the
 * registration method's arithmetic (no interpolation, no NCC, no FE
 * operators).  Random numbers come from a counter-based generator (the
 * published SplitMix64 finaliser, Steele/Lea/Flood 2014) keyed by
 * (seed, stream, frame, index), so every value is independent of the order
 * in which frames or pixels are produced.
 *
 * Frame model.  Frame k at pixel position y = (col, row) shows the specimen
 * at lattice coordinate z = y + d_k(y), with
 *   d_k(y) = t_k + sum_m a_{k,m} (sin(2 pi nu_m y_1 / W + th_m),
 *                                  sin(2 pi nu_m y_0 / W + th'_m)),
 *   a_{k,m} = A sin(2 pi k / P_m + psi_m),  t_0 = 0,  t_k = t_{k-1} + sd * N(0, I).
 * The exact deformation registering frame k to frame 0 (f_k o phi_{0,k} = f_0)
 * is the solution of phi = x + d_0(x) - d_k(phi); it is returned in pixels
 * as phi(x) - x when requested (fixed-point iteration in double precision).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_PI 3.14159265358979323846

typedef struct synth_params {
    uint64_t seed;
    int32_t n_frames;
    int32_t side;            /* frame side in pixels */
    double spacing;          /* lattice spacing, px */
    double sigma;            /* atom column Gaussian sigma, px */
    double peak;             /* expected counts at an atom centre */
    double background;       /* relative background level */
    double blob_amp;         /* relative amplitude of the large blobs */
    int32_t n_blobs;
    int32_t noise;           /* 1: Poisson counts, 0: expected intensity */
    double drift_sd;         /* random-walk step sd, px per frame */
    double dist_amp;         /* sinusoidal distortion amplitude A, px */
    double dist_period[2];   /* P_m in frames */
    double dist_freq[2];     /* nu_m in cycles per frame width */
    const double *drift_override; /* optional n_frames x 2 translations t_k (px) */
} synth_params;

/* ---- counter-based random numbers ------------------------------------ */
static uint64_t sm64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t rkey(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b)
{
    return sm64(sm64(sm64(sm64(seed) ^ (stream * 0x632BE59BD9B4E019ull)) ^ a) ^ (b * 0xD1B54A32D192ED03ull));
}

/* uniform in the open interval (0, 1) */
static double unif(uint64_t h) { return ((double)(h >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

static double gauss(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b)
{
    double u1 = unif(rkey(seed, stream, a, 2 * b));
    double u2 = unif(rkey(seed, stream, a, 2 * b + 1));
    return sqrt(-2.0 * log(u1)) * cos(2.0 * SYN_PI * u2);
}

/* Poisson(lam) by inversion of the CDF with one uniform. */
static double poisson(double lam, double u)
{
    if (lam <= 0.0) return 0.0;
    double p = exp(-lam), F = p;
    int k = 0;
    while (u > F && k < 1000) {
        k++;
        p *= lam / k;
        F += p;
    }
    return (double)k;
}

/* ---- series geometry -------------------------------------------------- */
typedef struct {
    double ox, oy;                  /* lattice origin */
    int nb;
    double bx[16], by[16], br[16], ba[16];
    double th[2], thp[2], psi[2];   /* distortion phases */
} series_geom;

static void make_geom(const synth_params *p, series_geom *g)
{
    uint64_t s = p->seed;
    g->ox = p->spacing * unif(rkey(s, 10, 0, 0));
    g->oy = p->spacing * unif(rkey(s, 10, 0, 1));
    g->nb = p->n_blobs < 16 ? p->n_blobs : 16;
    for (int b = 0; b < g->nb; b++) {
        g->bx[b] = p->side * unif(rkey(s, 11, b, 0));
        g->by[b] = p->side * unif(rkey(s, 11, b, 1));
        g->br[b] = p->side * (1.0 / 16.0 + (1.0 / 6.0 - 1.0 / 16.0) * unif(rkey(s, 11, b, 2)));
        g->ba[b] = 0.5 + 0.5 * unif(rkey(s, 11, b, 3));
    }
    for (int m = 0; m < 2; m++) {
        g->th[m] = 2.0 * SYN_PI * unif(rkey(s, 12, m, 0));
        g->thp[m] = 2.0 * SYN_PI * unif(rkey(s, 12, m, 1));
        g->psi[m] = 2.0 * SYN_PI * unif(rkey(s, 12, m, 2));
    }
}

/* translations t_k of all frames */
static void make_drift(const synth_params *p, double *t)
{
    if (p->drift_override) {
        memcpy(t, p->drift_override, sizeof(double) * 2 * p->n_frames);
        return;
    }
    t[0] = 0.0;
    t[1] = 0.0;
    for (int k = 1; k < p->n_frames; k++) {
        t[2 * k] = t[2 * k - 2] + p->drift_sd * gauss(p->seed, 13, k, 0);
        t[2 * k + 1] = t[2 * k - 1] + p->drift_sd * gauss(p->seed, 13, k, 1);
    }
}

/* frame displacement d_k(y) in px */
static void disp(const synth_params *p, const series_geom *g, const double *t, int k,
                 double y0, double y1, double *d0, double *d1)
{
    double a0 = t[2 * k], a1 = t[2 * k + 1];
    double W = (double)p->side;
    for (int m = 0; m < 2; m++) {
        if (p->dist_amp == 0.0) break;
        double amp = p->dist_amp * sin(2.0 * SYN_PI * k / p->dist_period[m] + g->psi[m]);
        a0 += amp * sin(2.0 * SYN_PI * p->dist_freq[m] * y1 / W + g->th[m]);
        a1 += amp * sin(2.0 * SYN_PI * p->dist_freq[m] * y0 / W + g->thp[m]);
    }
    *d0 = a0;
    *d1 = a1;
}

/* specimen intensity (expected counts) at lattice coordinate z */
static double intensity(const synth_params *p, const series_geom *g, double z0, double z1)
{
    double a = p->spacing, s2 = 2.0 * p->sigma * p->sigma;
    double i0 = floor((z0 - g->ox) / a + 0.5), i1 = floor((z1 - g->oy) / a + 0.5);
    double lat = 0.0;
    for (int di = -1; di <= 1; di++)
        for (int dj = -1; dj <= 1; dj++) {
            double c0 = g->ox + (i0 + di) * a, c1 = g->oy + (i1 + dj) * a;
            double r2 = (z0 - c0) * (z0 - c0) + (z1 - c1) * (z1 - c1);
            lat += exp(-r2 / s2);
        }
    double blob = 0.0;
    for (int b = 0; b < g->nb; b++) {
        double r2 = (z0 - g->bx[b]) * (z0 - g->bx[b]) + (z1 - g->by[b]) * (z1 - g->by[b]);
        blob += g->ba[b] * exp(-r2 / (2.0 * g->br[b] * g->br[b]));
    }
    return p->peak * (p->background + p->blob_amp * blob + lat) / (1.0 + p->background + p->blob_amp);
}

/*
 * frames: n_frames x side x side float32 (row-major, row = y_1, col = y_0).
 * gt (nullable): n_frames x 2 x side x side float64, phi_{0,k}(x) - x in px
 *   (channel 0 = column / x_0, channel 1 = row / x_1).
 * drift (nullable): n_frames x 2 translations t_k actually used.
 * Returns 0 on success.
 */
int synth_series(const synth_params *p, float *frames, double *gt, double *drift)
{
    if (!p || p->n_frames <= 0 || p->side <= 0 || !frames) return 1;
    series_geom g;
    make_geom(p, &g);
    double *t = (double *)malloc(sizeof(double) * 2 * p->n_frames);
    if (!t) return 2;
    make_drift(p, t);
    const int S = p->side;
    const long long rows = (long long)p->n_frames * S;
#pragma omp parallel for schedule(static)
    for (long long kr = 0; kr < rows; kr++) {
        int k = (int)(kr / S), r = (int)(kr % S);
        for (int c = 0; c < S; c++) {
            double d0, d1;
            disp(p, &g, t, k, (double)c, (double)r, &d0, &d1);
            double lam = intensity(p, &g, c + d0, r + d1);
            double v = lam;
            if (p->noise) v = poisson(lam, unif(rkey(p->seed, 20 + (uint64_t)k, (uint64_t)r, (uint64_t)c)));
            frames[((long long)k * S + r) * S + c] = (float)v;
            if (gt) {
                double e0, e1;
                disp(p, &g, t, 0, (double)c, (double)r, &e0, &e1);
                /* phi = x + d_0(x) - d_k(phi), by fixed-point iteration */
                double f0 = c + e0 - t[2 * k];
                double f1 = r + e1 - t[2 * k + 1];
                for (int it = 0; it < 200; it++) {
                    double q0, q1;
                    disp(p, &g, t, k, f0, f1, &q0, &q1);
                    double n0 = c + e0 - q0, n1 = r + e1 - q1;
                    double ch = fabs(n0 - f0) + fabs(n1 - f1);
                    f0 = n0;
                    f1 = n1;
                    if (ch < 1e-13) break;
                }
                long long base = (long long)k * 2 * S * S;
                gt[base + (long long)r * S + c] = f0 - c;
                gt[base + (long long)S * S + (long long)r * S + c] = f1 - r;
            }
        }
    }
    if (drift) memcpy(drift, t, sizeof(double) * 2 * p->n_frames);
    free(t);
    return 0;
}
