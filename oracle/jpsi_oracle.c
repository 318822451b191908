/*
 * TEST INFRASTRUCTURE ONLY -- the oracle.  Plain C reference of the
 * first-level J/psi event selection of Singhal, Chattopadhyay and Friese,
 * "Investigation of heterogeneous computing platforms for real-time data
 * analysis in the CBM experiment" (arXiv:1810.11966).  Only tests, the smoke
 * check and the benchmark's CPU-baseline leg call it.  It shares no code with
 * the GPU library.
 *
 * Method (Sec. 3.2, the three numbered steps):
 *   1. form every triplet of hits of a station, one hit from each of its three
 *      layers (the paper: the trigger station, i.e. the last one, Sec. 2);
 *   2. fit the triplet together with the vertex (0,0) by straight lines
 *      x = m0 z and y = m1 z, and reject it if the mean square deviation per
 *      degree of freedom exceeds a threshold in either plane (step 2b);
 *   3. select the event if at least two triplets pass.
 *
 * Readings where the paper is silent (each is a parameter or stated here):
 *   - the fit is unweighted least squares through the origin; with three
 *     hits and one slope ndf = 2 and "MSD per dof <= T" is S <= ndf*T with
 *     S the summed squared residual, evaluated as S <= fl32(ndf*T);
 *   - "above a threshold" rejects, so equality passes; both planes must pass;
 *   - precision is FP32 with every operation rounded to nearest in the order
 *     written below (no contraction, no flush-to-zero): the reference result.
 *     jpsi_oracle_run(fp64=1) evaluates the same formulas in double for the
 *     precision audit;
 *   - CHAIN mode (an extension beyond the paper, which uses the trigger
 *     station alone): every station is processed; a passing trigger triplet T
 *     is a track candidate iff each other station holds a passing triplet t
 *     whose three hits, taken against T's slopes (no refit), have a summed
 *     squared residual <= the same thresholds in both planes.  PAPER mode: the
 *     candidates are the passing trigger triplets (step 3 as printed);
 *   - "at least two triplets" (step 3) counts any candidates by default; with
 *     distinct_hits = 1 it needs min_candidates candidates (at most 2) no two
 *     of which share a hit: two candidates share a hit when they use the same
 *     hit of the same trigger-station layer (one hit, one particle).  Track
 *     counts stay the number of candidates.
 *
 * The pair early-out (brute = 0) skips (i, j) when
 *     |u_i/z_i - u_j/z_j| > (sqrt(C)(1+1e-5) + 1e-3) (1/z_i + 1/z_j)
 *                            + 1e-6 (|u_i/z_i| + |u_j/z_j|)
 * in either plane, evaluated in double, and applies the same test to (i, k)
 * and (j, k).  It never removes a passing triplet: if the FP32 residuals r_k
 * of a fit with slope m satisfy sum r_k^2 <= C, then every hit obeys
 * |u_k/z_k - m| <= (|r_k|(1+2eps) + eps |m z_k|) / z_k with |r_k| <= sqrt(C)
 * (1+2eps), eps = 2^-24; subtracting the relations of two hits gives a bound
 * below the one tested (the 1e-3 cm and 1e-6 relative terms dominate the
 * rounding terms, including the underflow of squares when C = 0).  The tests
 * check brute == pruned on random and adversarial events.
 */
#include "jpsi_oracle.h"

#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs float expressions evaluated in float (FLT_EVAL_METHOD == 0)"
#endif

#define JO_MAX_STATIONS 64

/* ------------------------------------------------------------------ P1 */

float jpsi_oracle_cut(int32_t ndf, float t) { return (float)ndf * t; }

/* One plane of step 2: slope of u = m z through the origin and the summed
 * squared residual, FP32, in exactly this order. */
static inline float fit_plane32(const float u[3], const float zz[3], float szz, float *m_out) {
    const float suz = (u[0] * zz[0] + u[1] * zz[1]) + u[2] * zz[2];
    const float m = suz / szz;
    const float r0 = u[0] - m * zz[0];
    const float r1 = u[1] - m * zz[1];
    const float r2 = u[2] - m * zz[2];
    *m_out = m;
    return (r0 * r0 + r1 * r1) + r2 * r2;
}

int jpsi_oracle_triplet(const float xs[3], const float ys[3], const float zs[3], float c_xz, float c_yz, float *m_x,
                        float *m_y, float *s_x, float *s_y) {
    const float szz = (zs[0] * zs[0] + zs[1] * zs[1]) + zs[2] * zs[2];
    float mx, my;
    const float sx = fit_plane32(xs, zs, szz, &mx);
    const float sy = fit_plane32(ys, zs, szz, &my);
    if (m_x) *m_x = mx;
    if (m_y) *m_y = my;
    if (s_x) *s_x = sx;
    if (s_y) *s_y = sy;
    return (sx <= c_xz) && (sy <= c_yz); /* ordered compares: NaN fails */
}

static inline double fit_plane64(const double u[3], const double zz[3], double szz, double *m_out) {
    const double suz = (u[0] * zz[0] + u[1] * zz[1]) + u[2] * zz[2];
    const double m = suz / szz;
    const double r0 = u[0] - m * zz[0];
    const double r1 = u[1] - m * zz[1];
    const double r2 = u[2] - m * zz[2];
    *m_out = m;
    return (r0 * r0 + r1 * r1) + r2 * r2;
}

int jpsi_oracle_triplet64(const float xs[3], const float ys[3], const float zs[3], double c_xz, double c_yz, double *m_x,
                          double *m_y, double *s_x, double *s_y) {
    const double X[3] = {xs[0], xs[1], xs[2]}, Y[3] = {ys[0], ys[1], ys[2]}, Z[3] = {zs[0], zs[1], zs[2]};
    const double szz = (Z[0] * Z[0] + Z[1] * Z[1]) + Z[2] * Z[2];
    double mx, my;
    const double sx = fit_plane64(X, Z, szz, &mx);
    const double sy = fit_plane64(Y, Z, szz, &my);
    if (m_x) *m_x = mx;
    if (m_y) *m_y = my;
    if (s_x) *s_x = sx;
    if (s_y) *s_y = sy;
    return (sx <= c_xz) && (sy <= c_yz);
}

/* ----------------------------------------------------- P2 (CHAIN mode) */

/* Residuals of the three hits of t against the trigger slope m (no refit). */
static inline float chain_plane32(const float u[3], const float zz[3], float m) {
    const float r0 = u[0] - m * zz[0];
    const float r1 = u[1] - m * zz[1];
    const float r2 = u[2] - m * zz[2];
    return (r0 * r0 + r1 * r1) + r2 * r2;
}

static inline double chain_plane64(const double u[3], const double zz[3], double m) {
    const double r0 = u[0] - m * zz[0];
    const double r1 = u[1] - m * zz[1];
    const double r2 = u[2] - m * zz[2];
    return (r0 * r0 + r1 * r1) + r2 * r2;
}

/* ------------------------------------------------------ per-event work */

typedef struct {
    int32_t i, j, k;   /* layer-local hit indices */
    int32_t hi, hj, hk;/* batch hit indices */
    double mx, my;     /* fitted slopes (the FP32 values, exactly, in FP32 mode) */
    int cand;          /* a candidate (trigger station only) */
} trip_t;

typedef struct {
    trip_t *v;
    int64_t n, cap;
} tripvec;

static int tv_push(tripvec *tv, const trip_t *t) {
    if (tv->n == tv->cap) {
        const int64_t nc = tv->cap ? tv->cap * 2 : 64;
        trip_t *nv = (trip_t *)realloc(tv->v, (size_t)nc * sizeof(trip_t));
        if (!nv) return 0;
        tv->v = nv;
        tv->cap = nc;
    }
    tv->v[tv->n++] = *t;
    return 1;
}

typedef struct {
    int32_t *v;
    int64_t n, cap;
} i32vec;

static int iv_push3(i32vec *iv, int32_t a, int32_t b, int32_t c) {
    if (iv->n + 3 > iv->cap) {
        int64_t nc = iv->cap ? iv->cap * 2 : 3 * 256;
        while (nc < iv->n + 3) nc *= 2;
        int32_t *nv = (int32_t *)realloc(iv->v, (size_t)nc * sizeof(int32_t));
        if (!nv) return 0;
        iv->v = nv;
        iv->cap = nc;
    }
    iv->v[iv->n++] = a;
    iv->v[iv->n++] = b;
    iv->v[iv->n++] = c;
    return 1;
}

typedef struct {
    /* shared, read-only */
    const jo_params *p;
    const float *x, *y, *z;
    const int32_t *off;
    float cx, cy;       /* FP32 thresholds */
    double cx64, cy64;  /* FP64 thresholds (same real value as ndf*T in double) */
    double kx, ky;      /* early-out slope factors */
    int brute, fp64, want_trip;
    int32_t *unit_counts;   /* [n_events*S] */
    int32_t *track_counts;  /* [n_events] */
    uint8_t *disjoint;      /* [n_events]: two candidates share no hit (distinct_hits) */
    /* per thread */
    int64_t e_begin, e_end;
    tripvec per_station[JO_MAX_STATIONS];
    i32vec out;         /* emitted triplets of this thread, event order */
    double *ux, *uy, *iz;   /* per-hit u/z and 1/z for the early-out, one station */
    int64_t hcap;
    int status;
} worker_t;

static int pair_may_pass(const worker_t *w, int64_t a, int64_t b) {
    /* a, b: station-local indices into ux/uy/iz */
    const double s = w->iz[a] + w->iz[b];
    const double dx = fabs(w->ux[a] - w->ux[b]);
    const double dy = fabs(w->uy[a] - w->uy[b]);
    const double bx = w->kx * s + 1e-6 * (fabs(w->ux[a]) + fabs(w->ux[b])) + 1e-300;
    const double by = w->ky * s + 1e-6 * (fabs(w->uy[a]) + fabs(w->uy[b])) + 1e-300;
    return !(dx > bx) && !(dy > by); /* NaN never prunes */
}

/* Step 1 and 2 for one station of one event: every passing triplet, in
 * (i, j, k) lexicographic order. */
static int process_station(worker_t *w, int64_t e, int s, tripvec *tv) {
    const int S = w->p->n_stations;
    const int32_t *o = w->off + ((int64_t)e * S + s) * 3;
    const int64_t b0 = o[0], b1 = o[1], b2 = o[2], b3 = o[3];
    const int64_t n0 = b1 - b0, n1 = b2 - b1, n2 = b3 - b2;
    tv->n = 0;
    for (int64_t h = b0; h < b3; ++h)
        if (w->z[h] <= 0.0f) return JO_EINVAL;
    if (n0 == 0 || n1 == 0 || n2 == 0) return JO_OK;
    if (!w->brute) {
        const int64_t nh = b3 - b0;
        if (nh > w->hcap) {
            free(w->ux);
            free(w->uy);
            free(w->iz);
            w->ux = (double *)malloc((size_t)nh * sizeof(double));
            w->uy = (double *)malloc((size_t)nh * sizeof(double));
            w->iz = (double *)malloc((size_t)nh * sizeof(double));
            if (!w->ux || !w->uy || !w->iz) return JO_ENOMEM;
            w->hcap = nh;
        }
        for (int64_t h = 0; h < nh; ++h) {
            const double zz = (double)w->z[b0 + h];
            w->ux[h] = (double)w->x[b0 + h] / zz;
            w->uy[h] = (double)w->y[b0 + h] / zz;
            w->iz[h] = 1.0 / zz;
        }
    }
    for (int64_t i = 0; i < n0; ++i) {
        for (int64_t j = 0; j < n1; ++j) {
            if (!w->brute && !pair_may_pass(w, i, n0 + j)) continue;
            for (int64_t k = 0; k < n2; ++k) {
                if (!w->brute && (!pair_may_pass(w, i, n0 + n1 + k) || !pair_may_pass(w, n0 + j, n0 + n1 + k)))
                    continue;
                const int64_t hi = b0 + i, hj = b1 + j, hk = b2 + k;
                const float xs[3] = {w->x[hi], w->x[hj], w->x[hk]};
                const float ys[3] = {w->y[hi], w->y[hj], w->y[hk]};
                const float zs[3] = {w->z[hi], w->z[hj], w->z[hk]};
                trip_t t;
                int pass;
                if (w->fp64) {
                    double mx, my;
                    pass = jpsi_oracle_triplet64(xs, ys, zs, w->cx64, w->cy64, &mx, &my, NULL, NULL);
                    t.mx = mx;
                    t.my = my;
                } else {
                    float mx, my;
                    pass = jpsi_oracle_triplet(xs, ys, zs, w->cx, w->cy, &mx, &my, NULL, NULL);
                    t.mx = mx;
                    t.my = my;
                }
                if (!pass) continue;
                t.i = (int32_t)i; t.j = (int32_t)j; t.k = (int32_t)k;
                t.hi = (int32_t)hi; t.hj = (int32_t)hj; t.hk = (int32_t)hk;
                if (!tv_push(tv, &t)) return JO_ENOMEM;
            }
        }
    }
    return JO_OK;
}

/* CHAIN-mode compatibility of station triplet t with trigger triplet T. */
static int compatible(const worker_t *w, const trip_t *T, const trip_t *t) {
    const float xs[3] = {w->x[t->hi], w->x[t->hj], w->x[t->hk]};
    const float ys[3] = {w->y[t->hi], w->y[t->hj], w->y[t->hk]};
    const float zs[3] = {w->z[t->hi], w->z[t->hj], w->z[t->hk]};
    if (w->fp64) {
        const double X[3] = {xs[0], xs[1], xs[2]}, Y[3] = {ys[0], ys[1], ys[2]}, Z[3] = {zs[0], zs[1], zs[2]};
        return (chain_plane64(X, Z, T->mx) <= w->cx64) && (chain_plane64(Y, Z, T->my) <= w->cy64);
    }
    return (chain_plane32(xs, zs, (float)T->mx) <= w->cx) && (chain_plane32(ys, zs, (float)T->my) <= w->cy);
}

static int process_event(worker_t *w, int64_t e) {
    const jo_params *p = w->p;
    const int S = p->n_stations, trig = p->trigger_station;
    for (int s = 0; s < S; ++s) {
        w->per_station[s].n = 0;
        if (p->mode == JO_MODE_PAPER && s != trig) continue;
        const int rc = process_station(w, e, s, &w->per_station[s]);
        if (rc != JO_OK) return rc;
    }
    /* step 3 (PAPER) or chaining (CHAIN): a candidate is a passing trigger
     * triplet (PAPER) or one compatible with every other station (CHAIN) */
    const tripvec *T = &w->per_station[trig];
    int64_t n_cand = 0;
    for (int64_t a = 0; a < T->n; ++a) {
        int ok = 1;
        if (p->mode == JO_MODE_CHAIN) {
            for (int s = 0; s < S && ok; ++s) {
                if (s == trig) continue;
                const tripvec *ts = &w->per_station[s];
                int found = 0;
                for (int64_t b = 0; b < ts->n && !found; ++b) found = compatible(w, &T->v[a], &ts->v[b]);
                ok = found;
            }
        }
        T->v[a].cand = ok;
        n_cand += ok;
    }
    w->track_counts[e] = n_cand > INT32_MAX ? INT32_MAX : (int32_t)n_cand;
    if (w->disjoint) {
        /* two candidates with no hit in common (same layer, same index) */
        int found = 0;
        for (int64_t a = 0; a < T->n && !found; ++a) {
            if (!T->v[a].cand) continue;
            for (int64_t b = a + 1; b < T->n && !found; ++b)
                found = T->v[b].cand && T->v[a].i != T->v[b].i && T->v[a].j != T->v[b].j && T->v[a].k != T->v[b].k;
        }
        w->disjoint[e] = (uint8_t)found;
    }
    for (int s = 0; s < S; ++s) {
        const tripvec *ts = &w->per_station[s];
        if (ts->n > INT32_MAX) return JO_EINVAL;
        w->unit_counts[e * S + s] = (int32_t)ts->n;
        if (w->want_trip)
            for (int64_t b = 0; b < ts->n; ++b)
                if (!iv_push3(&w->out, ts->v[b].i, ts->v[b].j, ts->v[b].k)) return JO_ENOMEM;
    }
    return JO_OK;
}

static void *worker_main(void *arg) {
    worker_t *w = (worker_t *)arg;
    w->status = JO_OK;
    for (int64_t e = w->e_begin; e < w->e_end; ++e) {
        const int rc = process_event(w, e);
        if (rc != JO_OK) {
            w->status = rc;
            break;
        }
    }
    return NULL;
}

static int params_ok(const jo_params *p) {
    if (!p) return 0;
    if (p->n_stations < 1 || p->n_stations > JO_MAX_STATIONS) return 0;
    if (p->trigger_station < 0 || p->trigger_station >= p->n_stations) return 0;
    if (p->mode != JO_MODE_PAPER && p->mode != JO_MODE_CHAIN) return 0;
    if (p->ndf < 1 || p->min_candidates < 0) return 0;
    if (p->distinct_hits != 0 && (p->distinct_hits != 1 || p->min_candidates > 2)) return 0;
    if (!(p->t_xz >= 0.0f) || !(p->t_yz >= 0.0f) || isinf(p->t_xz) || isinf(p->t_yz)) return 0;
    return 1;
}

int jpsi_oracle_run(const jo_params *p, int64_t n_events, int64_t n_hits, const float *x, const float *y,
                    const float *z, const int32_t *offsets, uint32_t *accept_bits, int32_t *track_counts,
                    int64_t *trip_off, int32_t *triplets, int64_t trip_capacity, int64_t *trip_needed,
                    int32_t *unit_counts, int n_threads, int brute, int fp64) {
    if (!params_ok(p) || n_events < 0 || n_hits < 0 || n_hits >= ((int64_t)1 << 31)) return JO_EINVAL;
    const int S = p->n_stations;
    if (n_events > (((int64_t)1 << 31) - 2) / (3 * S)) return JO_EINVAL;
    if (n_events > 0 && !offsets) return JO_EINVAL;
    if (n_hits > 0 && (!x || !y || !z)) return JO_EINVAL;
    if (n_events == 0) {
        if (offsets && offsets[0] != n_hits) return JO_EINVAL;
        if (!offsets && n_hits != 0) return JO_EINVAL;
        if (trip_off) trip_off[0] = 0;
        if (trip_needed) *trip_needed = 0;
        return JO_OK;
    }
    const int64_t n_off = n_events * S * 3 + 1;
    if (offsets[0] != 0 || offsets[n_off - 1] != n_hits) return JO_EINVAL;
    for (int64_t i = 1; i < n_off; ++i)
        if (offsets[i] < offsets[i - 1]) return JO_EINVAL;

    const int64_t n_units = n_events * S;
    int32_t *uc = unit_counts ? unit_counts : (int32_t *)malloc((size_t)n_units * sizeof(int32_t));
    int32_t *tc = track_counts ? track_counts : (int32_t *)malloc((size_t)n_events * sizeof(int32_t));
    uint8_t *dj = p->distinct_hits ? (uint8_t *)calloc((size_t)n_events, 1) : NULL;
    if (!uc || !tc || (p->distinct_hits && !dj)) {
        if (!unit_counts) free(uc);
        if (!track_counts) free(tc);
        free(dj);
        return JO_ENOMEM;
    }
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (n_threads > n_events) n_threads = (int)n_events;

    worker_t *ws = (worker_t *)calloc((size_t)n_threads, sizeof(worker_t));
    pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
    int rc = JO_OK;
    if (!ws || !th) rc = JO_ENOMEM;
    if (rc == JO_OK) {
        const float cx = jpsi_oracle_cut(p->ndf, p->t_xz), cy = jpsi_oracle_cut(p->ndf, p->t_yz);
        for (int t = 0; t < n_threads; ++t) {
            worker_t *w = &ws[t];
            w->p = p; w->x = x; w->y = y; w->z = z; w->off = offsets;
            w->cx = cx; w->cy = cy;
            w->cx64 = (double)p->ndf * (double)p->t_xz;
            w->cy64 = (double)p->ndf * (double)p->t_yz;
            w->kx = sqrt(fmax((double)cx, w->cx64)) * (1.0 + 1e-5) + 1e-3;
            w->ky = sqrt(fmax((double)cy, w->cy64)) * (1.0 + 1e-5) + 1e-3;
            w->brute = brute; w->fp64 = fp64;
            w->want_trip = triplets != NULL;
            w->unit_counts = uc; w->track_counts = tc; w->disjoint = dj;
            w->e_begin = n_events * t / n_threads;
            w->e_end = n_events * (t + 1) / n_threads;
        }
        int started = 0;
        for (int t = 1; t < n_threads; ++t) {
            if (pthread_create(&th[t], NULL, worker_main, &ws[t]) != 0) break;
            ++started;
        }
        worker_main(&ws[0]);
        for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
        for (int t = started + 1; t < n_threads; ++t) worker_main(&ws[t]); /* threads that failed to start */
        for (int t = 0; t < n_threads && rc == JO_OK; ++t) rc = ws[t].status;
    }
    if (rc == JO_OK) {
        int64_t total = 0;
        if (trip_off) trip_off[0] = 0;
        for (int64_t u = 0; u < n_units; ++u) {
            total += uc[u];
            if (trip_off) trip_off[u + 1] = total;
        }
        if (trip_needed) *trip_needed = total;
        if (accept_bits) {
            memset(accept_bits, 0, (size_t)((n_events + 31) / 32) * sizeof(uint32_t));
            for (int64_t e = 0; e < n_events; ++e)
                if (p->distinct_hits && p->min_candidates == 2 ? dj[e] : tc[e] >= p->min_candidates)
                    accept_bits[e >> 5] |= 1u << (e & 31);
        }
        if (triplets) {
            if (total > trip_capacity) {
                rc = JO_ECAPACITY;
            } else {
                int64_t pos = 0;
                for (int t = 0; t < n_threads; ++t) {
                    memcpy(triplets + pos, ws[t].out.v, (size_t)ws[t].out.n * sizeof(int32_t));
                    pos += ws[t].out.n;
                }
            }
        }
    }
    if (ws)
        for (int t = 0; t < n_threads; ++t) {
            for (int s = 0; s < JO_MAX_STATIONS; ++s) free(ws[t].per_station[s].v);
            free(ws[t].out.v);
            free(ws[t].ux);
            free(ws[t].uy);
            free(ws[t].iz);
        }
    free(ws);
    free(th);
    free(dj);
    if (!unit_counts) free(uc);
    if (!track_counts) free(tc);
    return rc;
}

/* ------------------------------------------- free-streaming timeslices */
/* See jpsi_oracle.h: hits carry times, windows replace events, a triplet
 * must be coincident (max t <= fl32(min t + dt)) and belongs to the window
 * of its earliest hit.  Written for clarity: binary searches give each
 * layer's time range, then every triple in the ranges is tested. */

/* First index i in [lo, hi) with t[i] >= v (t sorted). */
static int64_t t_lower(const float *t, int64_t lo, int64_t hi, float v) {
    while (lo < hi) {
        const int64_t m = lo + (hi - lo) / 2;
        if (t[m] < v) lo = m + 1; else hi = m;
    }
    return lo;
}

/* First index i in [lo, hi) with t[i] > v. */
static int64_t t_upper(const float *t, int64_t lo, int64_t hi, float v) {
    while (lo < hi) {
        const int64_t m = lo + (hi - lo) / 2;
        if (t[m] <= v) lo = m + 1; else hi = m;
    }
    return lo;
}

typedef struct {
    int32_t i, j, k;       /* indices within the layer groups */
    int64_t hi, hj, hk;    /* timeslice hit indices */
    float mx, my;          /* fitted slopes */
    float tmin, tmax;      /* earliest and latest hit time */
} strip_t;

typedef struct {
    strip_t *v;
    int64_t n, cap;
} stripvec;

static int sv_push(stripvec *sv, const strip_t *e) {
    if (sv->n == sv->cap) {
        const int64_t nc = sv->cap ? sv->cap * 2 : 64;
        strip_t *nv = (strip_t *)realloc(sv->v, (size_t)nc * sizeof(strip_t));
        if (!nv) return 0;
        sv->v = nv;
        sv->cap = nc;
    }
    sv->v[sv->n++] = *e;
    return 1;
}

/* Coincident passing triplets of station s with every hit time in [lo, hi];
 * when own_end is not NULL only those with earliest time < *own_end. */
static int stream_station(const jo_params *p, const float *x, const float *y, const float *z, const float *t,
                          const int32_t *off, float dt, int s, float lo, float hi, const float *own_end,
                          stripvec *out) {
    const float cx = jpsi_oracle_cut(p->ndf, p->t_xz), cy = jpsi_oracle_cut(p->ndf, p->t_yz);
    int64_t a[3], b[3];
    out->n = 0;
    for (int l = 0; l < 3; ++l) {
        a[l] = t_lower(t, off[3 * s + l], off[3 * s + l + 1], lo);
        b[l] = t_upper(t, a[l], off[3 * s + l + 1], hi);
        if (a[l] >= b[l]) return JO_OK;
    }
    for (int64_t h0 = a[0]; h0 < b[0]; ++h0)
        for (int64_t h1 = a[1]; h1 < b[1]; ++h1)
            for (int64_t h2 = a[2]; h2 < b[2]; ++h2) {
                const float t0 = t[h0], t1 = t[h1], t2 = t[h2];
                const float tmin = fminf(fminf(t0, t1), t2), tmax = fmaxf(fmaxf(t0, t1), t2);
                if (!(tmax <= tmin + dt)) continue; /* not coincident */
                if (own_end && !(tmin < *own_end)) continue; /* earliest hit in a later window */
                const float xs[3] = {x[h0], x[h1], x[h2]};
                const float ys[3] = {y[h0], y[h1], y[h2]};
                const float zs[3] = {z[h0], z[h1], z[h2]};
                strip_t e;
                if (!jpsi_oracle_triplet(xs, ys, zs, cx, cy, &e.mx, &e.my, NULL, NULL)) continue;
                e.i = (int32_t)(h0 - off[3 * s]);
                e.j = (int32_t)(h1 - off[3 * s + 1]);
                e.k = (int32_t)(h2 - off[3 * s + 2]);
                e.hi = h0; e.hj = h1; e.hk = h2;
                e.tmin = tmin; e.tmax = tmax;
                if (!sv_push(out, &e)) return JO_ENOMEM;
            }
    return JO_OK;
}

int jpsi_oracle_stream(const jo_params *p, const jo_stream *sp, int64_t n_hits, const float *x, const float *y,
                       const float *z, const float *t, const int32_t *offsets, uint32_t *accept_bits,
                       int32_t *track_counts, int64_t *trip_off, int32_t *triplets, int64_t trip_capacity,
                       int64_t *trip_needed, int32_t *unit_counts) {
    if (!params_ok(p) || p->distinct_hits || !sp || sp->n_windows < 0 || !(sp->dt >= 0.0f) || isinf(sp->dt))
        return JO_EINVAL;
    const int S = p->n_stations, K = sp->n_windows, trig = p->trigger_station;
    const int chain = p->mode == JO_MODE_CHAIN && S > 1;
    if (n_hits < 0 || n_hits >= ((int64_t)1 << 31) || !offsets) return JO_EINVAL;
    if (n_hits > 0 && (!x || !y || !z || !t)) return JO_EINVAL;
    if (K > 0 && !sp->bounds) return JO_EINVAL;
    for (int k = 0; k <= K && K > 0; ++k) {
        if (isnan(sp->bounds[k]) || isinf(sp->bounds[k])) return JO_EINVAL;
        if (k > 0 && !(sp->bounds[k] > sp->bounds[k - 1])) return JO_EINVAL;
    }
    if (offsets[0] != 0 || offsets[3 * S] != n_hits) return JO_EINVAL;
    for (int g = 0; g < 3 * S; ++g) {
        if (offsets[g + 1] < offsets[g]) return JO_EINVAL;
        for (int64_t h = offsets[g]; h < offsets[g + 1]; ++h) {
            if (isnan(t[h]) || (h > offsets[g] && !(t[h] >= t[h - 1]))) return JO_EINVAL; /* sorted, no NaN */
            const int s = g / 3;
            if ((p->mode == JO_MODE_CHAIN || s == trig) && z[h] <= 0.0f) return JO_EINVAL;
        }
    }
    const float cx = jpsi_oracle_cut(p->ndf, p->t_xz), cy = jpsi_oracle_cut(p->ndf, p->t_yz);
    stripvec per[JO_MAX_STATIONS], other;
    memset(per, 0, sizeof(per));
    memset(&other, 0, sizeof(other));
    int rc = JO_OK;
    int64_t total = 0, pos = 0;
    if (trip_off) trip_off[0] = 0;
    if (accept_bits) memset(accept_bits, 0, (size_t)((K + 31) / 32) * sizeof(uint32_t));
    for (int k = 0; k < K && rc == JO_OK; ++k) {
        const float lo = sp->bounds[k], own_end = sp->bounds[k + 1], hi = sp->bounds[k + 1] + sp->dt;
        for (int s = 0; s < S && rc == JO_OK; ++s) {
            per[s].n = 0;
            if (p->mode == JO_MODE_PAPER && s != trig) continue;
            rc = stream_station(p, x, y, z, t, offsets, sp->dt, s, lo, hi, &own_end, &per[s]);
        }
        if (rc != JO_OK) break;
        int64_t n_cand = 0;
        for (int64_t a = 0; a < per[trig].n && rc == JO_OK; ++a) {
            const strip_t *T = &per[trig].v[a];
            int ok = 1;
            for (int s = 0; s < S && ok && chain; ++s) {
                if (s == trig) continue;
                /* hits of a coincident partner lie in [max_T - dt, fl32(min_T + dt)]
                 * (searched with a margin below: the exact tests decide) */
                double lod = (double)T->tmax - (double)sp->dt;
                lod -= 1e-6 * (fabs((double)T->tmax) + (double)sp->dt) + 1e-30;
                const float lo_s = nextafterf((float)lod, -INFINITY), hi_s = T->tmin + sp->dt;
                rc = stream_station(p, x, y, z, t, offsets, sp->dt, s, lo_s, hi_s, NULL, &other);
                if (rc != JO_OK) break;
                int found = 0;
                for (int64_t b2 = 0; b2 < other.n && !found; ++b2) {
                    const strip_t *u = &other.v[b2];
                    const float mn = fminf(T->tmin, u->tmin), mx = fmaxf(T->tmax, u->tmax);
                    if (!(mx <= mn + sp->dt)) continue; /* the six hits not coincident */
                    const float xs[3] = {x[u->hi], x[u->hj], x[u->hk]};
                    const float ys[3] = {y[u->hi], y[u->hj], y[u->hk]};
                    const float zs[3] = {z[u->hi], z[u->hj], z[u->hk]};
                    found = (chain_plane32(xs, zs, T->mx) <= cx) && (chain_plane32(ys, zs, T->my) <= cy);
                }
                ok = found;
            }
            n_cand += ok;
        }
        if (rc != JO_OK) break;
        if (track_counts) track_counts[k] = n_cand > INT32_MAX ? INT32_MAX : (int32_t)n_cand;
        if (accept_bits && n_cand >= p->min_candidates) accept_bits[k >> 5] |= 1u << (k & 31);
        for (int s = 0; s < S; ++s) {
            if (unit_counts) unit_counts[(int64_t)k * S + s] = (int32_t)per[s].n;
            total += per[s].n;
            if (trip_off) trip_off[(int64_t)k * S + s + 1] = total;
            if (triplets && total <= trip_capacity)
                for (int64_t b2 = 0; b2 < per[s].n; ++b2) {
                    triplets[3 * pos] = per[s].v[b2].i;
                    triplets[3 * pos + 1] = per[s].v[b2].j;
                    triplets[3 * pos + 2] = per[s].v[b2].k;
                    ++pos;
                }
        }
    }
    for (int s = 0; s < JO_MAX_STATIONS; ++s) free(per[s].v);
    free(other.v);
    if (rc != JO_OK) return rc;
    if (trip_needed) *trip_needed = total;
    if (triplets && total > trip_capacity) return JO_ECAPACITY;
    return JO_OK;
}
