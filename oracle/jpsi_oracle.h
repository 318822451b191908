/*
 * TEST INFRASTRUCTURE ONLY.  Plain single-threaded-per-event C reference of
 * the first-level J/psi event selection (paper Sec. 3.2).  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may call it; the product
 * path never does.  It shares no code, header or constant with the GPU
 * library.
 */
#ifndef JPSI_ORACLE_H
#define JPSI_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { JO_OK = 0, JO_EINVAL = 1, JO_ENOMEM = 2, JO_ECAPACITY = 3 };
enum { JO_MODE_PAPER = 0, JO_MODE_CHAIN = 1 };

typedef struct {
    int32_t n_stations;      /* stations per event (three layers each) */
    int32_t trigger_station; /* the last station is the trigger station (Sec. 2) */
    int32_t mode;            /* JO_MODE_PAPER: trigger station only (Sec. 3.2);
                                JO_MODE_CHAIN: every station + chaining */
    int32_t ndf;             /* degrees of freedom of the fit (2: three hits, one slope) */
    int32_t min_candidates;  /* accept if #candidates >= this (2, Sec. 3.2 step 3) */
    float t_xz, t_yz;        /* MSD-per-dof thresholds (Sec. 3.2 step 2b), cm^2 */
    int32_t distinct_hits;   /* 0: step 3 counts any candidates; 1: the event needs
                                min_candidates (<= 2) candidates no two of which share
                                a hit of the trigger station */
} jo_params;

/*
 * Runs the selection over a host batch.
 *   x, y, z      : float32 [n_hits]
 *   offsets      : int32 [n_events*n_stations*3 + 1], offsets[0] = 0,
 *                  non-decreasing, offsets[last] = n_hits; hits of layer l of
 *                  station s of event e are [offsets[(e*S+s)*3+l], ...+1).
 * Outputs (host, caller-owned; any may be NULL except where noted):
 *   accept_bits  : uint32 [(n_events+31)/32], bit e%32 of word e/32
 *   track_counts : int32 [n_events]
 *   trip_off     : int64 [n_events*S + 1] exclusive scan of per-unit counts
 *   triplets     : int32 [3*trip_capacity] layer-local (i,j,k), canonical
 *                  (i, j, k) lexicographic order inside each unit
 *   trip_needed  : total passing triplets (always written when non-NULL)
 *   unit_counts  : int32 [n_events*S] passing triplets per unit (may be NULL)
 * fp64 = 1 evaluates the same predicates in double from the same float inputs
 * (precision audit); brute = 1 disables the pair early-out.
 * Returns JO_OK, JO_EINVAL (bad offsets, z <= 0 in a processed hit, bad
 * params), JO_ENOMEM, or JO_ECAPACITY (triplets requested and capacity too
 * small: counts and accept bits are still complete, triplets unwritten).
 */
int jpsi_oracle_run(const jo_params *p, int64_t n_events, int64_t n_hits, const float *x, const float *y,
                    const float *z, const int32_t *offsets, uint32_t *accept_bits, int32_t *track_counts,
                    int64_t *trip_off, int32_t *triplets, int64_t trip_capacity, int64_t *trip_needed,
                    int32_t *unit_counts, int n_threads, int brute, int fp64);

/*
 * Free-streaming selection (an extension; the paper's Outlook, Sec. 8, only
 * says that free-streaming data need hit times and event building).  One
 * timeslice of hits with times t (ns, float32), grouped per (station, layer):
 * offsets [n_stations*3 + 1], each group sorted by t (non-decreasing, no
 * NaN).  Windows k = 0 .. n_windows-1 are [bounds[k], bounds[k+1]) (bounds
 * strictly increasing, finite).  A triplet (one hit per layer of a station)
 * is coincident when max t <= fl32(min t + dt); it belongs to the window
 * that holds its earliest time.  Passing triplets of window k at station s
 * are its coincident triplets that pass P1; in CHAIN mode a passing trigger
 * triplet T of window k is a candidate when every other station holds a
 * passing coincident triplet t (anywhere in the timeslice) compatible with T (P2) whose
 * six hits together are coincident.  Window k is accepted when it holds at
 * least min_candidates candidates.  Outputs as for jpsi_oracle_run with
 * windows in place of events; triplet rows are indices into the timeslice's
 * layer groups.  distinct_hits must be 0.
 */
typedef struct {
    int32_t n_windows;
    float dt;             /* coincidence width, ns, >= 0 */
    const float *bounds;  /* [n_windows + 1] window starts and the last end */
} jo_stream;

int jpsi_oracle_stream(const jo_params *p, const jo_stream *sp, int64_t n_hits, const float *x, const float *y,
                       const float *z, const float *t, const int32_t *offsets, uint32_t *accept_bits,
                       int32_t *track_counts, int64_t *trip_off, int32_t *triplets, int64_t trip_capacity,
                       int64_t *trip_needed, int32_t *unit_counts);

/* P1 on one triplet (hits k = 0,1,2 from layers 0,1,2): returns 1 if it
 * passes both planes; writes the fitted slopes. */
int jpsi_oracle_triplet(const float xs[3], const float ys[3], const float zs[3], float c_xz, float c_yz,
                        float *m_x, float *m_y, float *s_x, float *s_y);

/* FP64 counterpart of jpsi_oracle_triplet. */
int jpsi_oracle_triplet64(const float xs[3], const float ys[3], const float zs[3], double c_xz, double c_yz,
                          double *m_x, double *m_y, double *s_x, double *s_y);

/* Threshold on the summed squared residual: fl32(ndf * t). */
float jpsi_oracle_cut(int32_t ndf, float t);

#ifdef __cplusplus
}
#endif
#endif
