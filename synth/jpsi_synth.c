/*
 * Seeded synthetic CBM-MUCH-like events: hit coordinates in SoA FP32 and
 * per-(event, station, layer) hit counts.  This module is an INPUT GENERATOR
 * only.  It is shared by the test oracle and the GPU path and therefore holds
 * none of the selection arithmetic (no fits, no cuts, no chaining).
 *
 * What it models (paper Sec. 2 and Sec. 3.1):
 *   - stations of three detector layers 10 cm apart (Sec. 2), the layer z
 *     being written into every hit (Sec. 3.2: hits carry x, y, z);
 *   - background hits in an annulus around the uninstrumented beam hole
 *     (Sec. 3.1, Fig. 2 right), radius 15 cm < r < 0.4 z, either uniform in
 *     area or with an area density falling as 1/r^2;
 *   - signal muons as straight lines from the target (0,0,0) (Sec. 3.1),
 *     slopes uniform in (-0.35, 0.35), Gaussian smear sigma per coordinate.
 *
 * Determinism.  Every event draws from its own streams, so any sub-range of a
 * workload is generated identically on its own, and multithreading never
 * changes the output.  Only +, -, *, / and sqrt (all correctly rounded in IEEE
 * double) are used; log and exp are evaluated by the series below instead of
 * the C library, so x86-64 and aarch64 hosts produce identical bytes.  Build
 * with -ffp-contract=off.
 *
 * Random numbers:
 *   SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom
 *   number generators", OOPSLA 2014) seeds
 *   xoshiro256** (D. Blackman, S. Vigna, "Scrambled linear pseudorandom
 *   number generators", ACM TOMS 2021).
 *   Normal deviates: Marsaglia's polar method.  Directions in the transverse
 *   plane: rejection sampling in the unit disc.  Poisson counts: Knuth's
 *   multiplication method on chunks of mean <= 25 (a sum of independent
 *   Poisson variables is Poisson with the summed mean).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYNTH_MAX_STATIONS 16

typedef struct {
    int32_t n_stations;
    int32_t radial;        /* 0: uniform in area, 1: area density ~ 1/r^2 */
    int32_t bg_mode;       /* 0: Poisson(bg_lambda) per layer;
                              1: per-event lambda_e = clip(exp(ln_median + ln_sigma*N(0,1)), lam_min, lam_max),
                                 per-layer count = clip(Poisson(lambda_e), count_min, count_max) */
    int32_t count_min, count_max;
    double station_z[SYNTH_MAX_STATIONS];
    double layer_dz;       /* layers at z_s - dz, z_s, z_s + dz */
    double bg_lambda;
    double ln_median, ln_sigma, lam_min, lam_max;
    double r_min;          /* inner radius of the annulus, cm */
    double r_max_frac;     /* outer radius = r_max_frac * z_layer */
    double p_two_mu, p_one_mu;
    double slope_max;      /* |tx|,|ty| < slope_max */
    double sigma;          /* hit smear of signal hits, cm */
} jpsi_synth_cfg;

/* ---------------------------------------------------------------- RNG */

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
#define SM64_GAMMA 0x9e3779b97f4a7c15ULL

typedef struct { uint64_t s[4]; } xo_t;

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t xo_next(xo_t *r) {
    uint64_t *s = r->s;
    const uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* Stream for (seed, event, purpose): four consecutive SplitMix64 outputs
 * starting from a state that mixes all three keys. */
static void xo_init(xo_t *r, uint64_t seed, uint64_t event, uint64_t purpose) {
    uint64_t st = sm64_mix(seed + SM64_GAMMA) ^ sm64_mix((event << 2 | purpose) * SM64_GAMMA + 0x632be59bd9b4e019ULL);
    for (int i = 0; i < 4; ++i) {
        st += SM64_GAMMA;
        r->s[i] = sm64_mix(st);
    }
    if (!(r->s[0] | r->s[1] | r->s[2] | r->s[3])) r->s[0] = 1; /* never the all-zero state */
}

static inline double u01(xo_t *r) { return (double)(xo_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0, n) by multiply-shift (bias < n / 2^64) */
static inline uint64_t uint_below(xo_t *r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)xo_next(r) * n) >> 64);
}

/* --------------------------------------- deterministic log / exp (double) */

static const double LN2 = 0.69314718055994530942;

/* ln(x) for finite x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)),
 * ln m = 2 atanh(t), t = (m-1)/(m+1), |t| < 0.172, series to t^31. */
static double g_log(double x) {
    int e;
    double m = frexp(x, &e);
    if (m < 0.70710678118654752440) {
        m *= 2.0;
        e -= 1;
    }
    const double t = (m - 1.0) / (m + 1.0);
    const double t2 = t * t;
    double sum = 0.0;
    double p = t;
    for (int n = 1; n <= 31; n += 2) {
        sum += p / (double)n;
        p *= t2;
    }
    return (double)e * LN2 + 2.0 * sum;
}

/* exp(x): x = k ln2 + r, |r| <= ln2/2 (plus rounding), Taylor to degree 24. */
static double g_exp(double x) {
    if (x < -740.0) return 0.0;
    if (x > 709.0) return HUGE_VAL;
    const double k = floor(x / LN2 + 0.5);
    const double r = x - k * LN2;
    double term = 1.0, sum = 1.0;
    for (int n = 1; n <= 24; ++n) {
        term = term * r / (double)n;
        sum += term;
    }
    return ldexp(sum, (int)k);
}

/* ----------------------------------------------------------- samplers */

static double normal01(xo_t *r) {
    for (;;) {
        const double u = 2.0 * u01(r) - 1.0;
        const double v = 2.0 * u01(r) - 1.0;
        const double s = u * u + v * v;
        if (s >= 1.0 || s == 0.0) continue;
        return u * sqrt(-2.0 * g_log(s) / s);
    }
}

static void unit_direction(xo_t *r, double *c, double *s) {
    for (;;) {
        const double u = 2.0 * u01(r) - 1.0;
        const double v = 2.0 * u01(r) - 1.0;
        const double q = u * u + v * v;
        if (q > 1.0 || q < 1e-12) continue;
        const double inv = 1.0 / sqrt(q);
        *c = u * inv;
        *s = v * inv;
        return;
    }
}

static int64_t poisson(xo_t *r, double lam) {
    if (!(lam > 0.0)) return 0;
    int64_t chunks = (int64_t)ceil(lam / 25.0);
    if (chunks < 1) chunks = 1;
    const double lc = lam / (double)chunks;
    const double L = g_exp(-lc);
    int64_t total = 0;
    for (int64_t c = 0; c < chunks; ++c) {
        int64_t k = 0;
        double p = 1.0;
        do {
            ++k;
            p *= u01(r);
        } while (p > L);
        total += k - 1;
    }
    return total;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ------------------------------------------------------ event structure */

typedef struct {
    int n_mu;
    double tx[2], ty[2];
    int32_t bg[SYNTH_MAX_STATIONS * 3];
} event_plan;

/* Stream "A" (purpose 0): signal content and per-layer background counts. */
static void plan_event(const jpsi_synth_cfg *cfg, uint64_t seed, int64_t e, event_plan *pl) {
    xo_t r;
    xo_init(&r, seed, (uint64_t)e, 0);
    const double u = u01(&r);
    pl->n_mu = u < cfg->p_two_mu ? 2 : (u < cfg->p_two_mu + cfg->p_one_mu ? 1 : 0);
    for (int m = 0; m < 2; ++m) {
        pl->tx[m] = (2.0 * u01(&r) - 1.0) * cfg->slope_max;
        pl->ty[m] = (2.0 * u01(&r) - 1.0) * cfg->slope_max;
    }
    double lam = cfg->bg_lambda;
    if (cfg->bg_mode == 1) lam = clampd(g_exp(g_log(cfg->ln_median) + cfg->ln_sigma * normal01(&r)), cfg->lam_min, cfg->lam_max);
    const int nl = cfg->n_stations * 3;
    for (int l = 0; l < nl; ++l) {
        int64_t n = poisson(&r, lam);
        if (cfg->bg_mode == 1) {
            if (n < cfg->count_min) n = cfg->count_min;
            if (n > cfg->count_max) n = cfg->count_max;
        }
        pl->bg[l] = (int32_t)n;
    }
}

/* Stream "B" (purpose 1): positions and the in-layer shuffle. */
static void fill_event(const jpsi_synth_cfg *cfg, uint64_t seed, int64_t e, const event_plan *pl, const int64_t *off,
                       float *x, float *y, float *z, int8_t *truth) {
    xo_t r;
    xo_init(&r, seed, (uint64_t)e, 1);
    const int nl = cfg->n_stations * 3;
    for (int l = 0; l < nl; ++l) {
        const int s = l / 3, k = l % 3;
        const double zl = cfg->station_z[s] + (double)(k - 1) * cfg->layer_dz;
        const float zf = (float)zl;
        const int64_t b = off[l];
        const int64_t n = off[l + 1] - off[l];
        int64_t h = 0;
        for (int m = 0; m < pl->n_mu; ++m, ++h) {
            const double gx = normal01(&r), gy = normal01(&r);
            x[b + h] = (float)(pl->tx[m] * zl + cfg->sigma * gx);
            y[b + h] = (float)(pl->ty[m] * zl + cfg->sigma * gy);
            z[b + h] = zf;
            if (truth) truth[b + h] = (int8_t)(m + 1);
        }
        const double R = cfg->r_max_frac * zl;
        const double r0 = cfg->r_min;
        const double lratio = g_log(R / r0);
        for (; h < n; ++h) {
            double c, sn;
            unit_direction(&r, &c, &sn);
            const double U = u01(&r);
            const double rad = cfg->radial == 1 ? r0 * g_exp(U * lratio) : sqrt(r0 * r0 + U * (R * R - r0 * r0));
            x[b + h] = (float)(rad * c);
            y[b + h] = (float)(rad * sn);
            z[b + h] = zf;
            if (truth) truth[b + h] = 0;
        }
        /* Fisher-Yates shuffle of the layer (all arrays together) */
        for (int64_t i = n - 1; i > 0; --i) {
            const int64_t j = (int64_t)uint_below(&r, (uint64_t)(i + 1));
            float t;
            t = x[b + i]; x[b + i] = x[b + j]; x[b + j] = t;
            t = y[b + i]; y[b + i] = y[b + j]; y[b + j] = t;
            if (truth) {
                int8_t q = truth[b + i];
                truth[b + i] = truth[b + j];
                truth[b + j] = q;
            }
        }
    }
}

/* ---------------------------------------------------------- threading */

typedef struct {
    const jpsi_synth_cfg *cfg;
    uint64_t seed;
    int64_t e0, n_ev;
    int32_t *counts;
    const int64_t *offsets;
    float *x, *y, *z;
    int8_t *truth;
    int64_t next;          /* shared work counter */
    pthread_mutex_t mu;
    int phase;             /* 0 counts, 1 fill */
} job_t;

#define CHUNK 1024

static void *worker(void *arg) {
    job_t *j = (job_t *)arg;
    const int nl = j->cfg->n_stations * 3;
    for (;;) {
        pthread_mutex_lock(&j->mu);
        const int64_t a = j->next;
        j->next += CHUNK;
        pthread_mutex_unlock(&j->mu);
        if (a >= j->n_ev) break;
        const int64_t b = a + CHUNK < j->n_ev ? a + CHUNK : j->n_ev;
        for (int64_t i = a; i < b; ++i) {
            event_plan pl;
            plan_event(j->cfg, j->seed, j->e0 + i, &pl);
            if (j->phase == 0) {
                for (int l = 0; l < nl; ++l) j->counts[i * nl + l] = pl.bg[l] + pl.n_mu;
            } else {
                fill_event(j->cfg, j->seed, j->e0 + i, &pl, j->offsets + i * nl, j->x, j->y, j->z, j->truth);
            }
        }
    }
    return NULL;
}

static int run_job(job_t *j, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    j->next = 0;
    pthread_mutex_init(&j->mu, NULL);
    int started = 0;
    for (int t = 1; t < n_threads; ++t) {
        if (pthread_create(&th[t], NULL, worker, j) != 0) break;
        ++started;
    }
    worker(j);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&j->mu);
    return 0;
}

static int cfg_ok(const jpsi_synth_cfg *cfg) {
    return cfg && cfg->n_stations >= 1 && cfg->n_stations <= SYNTH_MAX_STATIONS;
}

/* Per-layer hit counts of events [e0, e0+n_ev): counts[(e-e0)*S*3 + s*3 + l]. */
int jpsi_synth_counts(const jpsi_synth_cfg *cfg, uint64_t seed, int64_t e0, int64_t n_ev, int32_t *counts, int n_threads) {
    if (!cfg_ok(cfg) || n_ev < 0 || (n_ev > 0 && !counts)) return 1;
    job_t j;
    memset(&j, 0, sizeof j);
    j.cfg = cfg; j.seed = seed; j.e0 = e0; j.n_ev = n_ev; j.counts = counts; j.phase = 0;
    return run_job(&j, n_threads);
}

/* Hits of events [e0, e0+n_ev) at the CSR positions `offsets` (int64, n_ev*S*3+1
 * entries, offsets[0] = 0) that jpsi_synth_counts' counts imply. */
int jpsi_synth_fill(const jpsi_synth_cfg *cfg, uint64_t seed, int64_t e0, int64_t n_ev, const int64_t *offsets,
                    float *x, float *y, float *z, int8_t *truth, int n_threads) {
    if (!cfg_ok(cfg) || n_ev < 0 || (n_ev > 0 && (!offsets || !x || !y || !z))) return 1;
    job_t j;
    memset(&j, 0, sizeof j);
    j.cfg = cfg; j.seed = seed; j.e0 = e0; j.n_ev = n_ev; j.offsets = offsets;
    j.x = x; j.y = y; j.z = z; j.truth = truth; j.phase = 1;
    return run_job(&j, n_threads);
}

/* Exposed for the generator's own tests (accuracy of the series). */
double jpsi_synth_log(double x) { return g_log(x); }
double jpsi_synth_exp(double x) { return g_exp(x); }
uint64_t jpsi_synth_xoshiro_first(uint64_t s0, uint64_t s1, uint64_t s2, uint64_t s3, int n, uint64_t *out) {
    xo_t r = {{s0, s1, s2, s3}};
    for (int i = 0; i < n; ++i) out[i] = xo_next(&r);
    return n > 0 ? out[n - 1] : 0;
}
uint64_t jpsi_synth_splitmix_mix(uint64_t z) { return sm64_mix(z); }
