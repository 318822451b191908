/*
 * libjpsi -- GB300 (sm_103a) first-level J/psi event selection in the CBM
 * muon chambers, after V. Singhal, S. Chattopadhyay, V. Friese,
 * "Investigation of heterogeneous computing platforms for real-time data
 * analysis in the CBM experiment", arXiv:1810.11966.
 *
 * The operation (Sec. 3.2, steps 1-3): for every event, form all triplets of
 * hits of a station with one hit from each of its three layers; fit each
 * triplet together with the event vertex (0, 0) by straight lines x = m0 z and
 * y = m1 z; reject the triplet if its mean square deviation per degree of
 * freedom exceeds a threshold in either plane; select the event if at least
 * two candidates remain.
 *
 *   JPSI_MODE_PAPER  exactly the paper: the trigger station (the last one,
 *                    Sec. 2) only; candidates = passing trigger triplets.
 *   JPSI_MODE_CHAIN  an extension: triplets are formed in every station, and a
 *                    passing trigger triplet T is a track candidate iff every
 *                    other station holds a passing triplet whose three hits,
 *                    taken against T's fitted slopes (no refit), have a summed
 *                    squared residual within the same thresholds in both
 *                    planes.  With one station it equals PAPER.
 *
 * Arithmetic (the reference result).  FP32, every operation rounded to
 * nearest in this order, no contraction, no flush-to-zero:
 *     Szz = (z0*z0 + z1*z1) + z2*z2,  Suz = (u0*z0 + u1*z1) + u2*z2,
 *     m = Suz / Szz,  r_k = u_k - m*z_k,  S_u = (r0*r0 + r1*r1) + r2*r2,
 *     pass = S_x <= C_xz && S_y <= C_yz,   C = fl32(ndf * t).
 * "MSD per dof <= t" is read as S <= ndf * t (equality passes; NaN fails).
 *
 * Data layout (all device memory, caller-owned unless stated):
 *   x, y, z   float32 [n_hits], structure of arrays, in cm.
 *   offsets   int32 [n_events * n_stations * 3 + 1]: hits of layer l of station
 *             s of event e are [offsets[(e*S+s)*3+l], offsets[(e*S+s)*3+l+1]);
 *             offsets[0] = 0, non-decreasing, offsets[last] = n_hits.
 *             Layer 0 is the most upstream layer of its station.
 *   n_hits < 2^31; every z of a hit that the mode reads must not be <= 0
 *   (NaN and +Inf coordinates are legal and never pass).
 *   z_layer   optional float32 [n_stations * 3], used when z is NULL: every
 *             hit of layer l of station s lies at z = z_layer[s*3 + l] (the
 *             detector layers are planes at fixed z, Sec. 2).  The library
 *             fills a per-hit z array from it before the selection, so results
 *             equal those of a per-hit z array holding the same values, and a
 *             host run moves 8 instead of 12 bytes per hit.  It lives in the
 *             same kind of memory as the call's other inputs.
 *             jpsi_select_noalloc does not take it (z must be given).
 *
 * Outputs (device memory, caller-owned; any pointer may be NULL = not wanted,
 * except that triplets need trip_off):
 *   accept_bits   uint32 [(n_events+31)/32]; bit (e & 31) of word e >> 5 is
 *                 set iff event e has >= min_candidates candidates.
 *   track_counts  int32 [n_events]: candidates per event.
 *   trip_off      int64 [n_events*S + 1]: exclusive scan of the passing-triplet
 *                 counts per unit u = e*S + s (CHAIN: every station; PAPER:
 *                 the trigger station, other units 0).
 *   triplets      int32 [3 * trip_capacity]: (i, j, k) layer-local hit indices
 *                 of every passing triplet, unit u at rows [trip_off[u],
 *                 trip_off[u+1]); order inside a unit is unspecified.
 *   trip_needed   set to the total number of passing triplets.
 *
 * Errors: every call returns a status; nothing throws across the ABI.  On
 * JPSI_ECAPACITY the counts, trip_off and accept bits are complete and
 * trip_needed holds the size to retry with; triplets are unspecified.  On
 * JPSI_EINVAL / JPSI_ECUDA outputs are unspecified.  Device waits inside the
 * library are bounded and surface as JPSI_ETIMEOUT.
 *
 * Threads: a context is used by one host thread at a time (JPSI_EBUSY
 * otherwise).  Runs are synchronous with respect to the given stream: the
 * call returns after the stream has completed the work.
 */
#ifndef JPSI_H
#define JPSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    JPSI_OK = 0,
    JPSI_EINVAL = 1,    /* malformed arguments, offsets or z <= 0 */
    JPSI_ENOMEM = 2,    /* device/host allocation failed or exceeds the budget */
    JPSI_ECAPACITY = 3, /* triplet buffer too small; see trip_needed */
    JPSI_ECUDA = 4,     /* a CUDA call failed */
    JPSI_ETIMEOUT = 5,  /* a bounded wait ran out */
    JPSI_EBUSY = 6      /* context in use by another call */
} jpsi_status;

typedef enum { JPSI_MODE_PAPER = 0, JPSI_MODE_CHAIN = 1 } jpsi_mode;

/* Selection parameters (Sec. 3.2).  Defaults of the paper: ndf = 2 (three
 * hits, one slope), min_candidates = 2, trigger_station = n_stations - 1,
 * t_xz = 0.03 and t_yz = 0.025 cm^2 (step 2b).
 * distinct_hits = 1 reads step 3's "at least two triplets" as candidates
 * that share no hit: the event is accepted only if it holds min_candidates
 * (at most 2) candidates no two of which use the same hit of a
 * trigger-station layer.  track_counts stay the number of candidates. */
typedef struct {
    int32_t n_stations;      /* 1 .. 16 */
    int32_t trigger_station; /* 0 .. n_stations-1 */
    int32_t mode;            /* jpsi_mode */
    int32_t ndf;             /* >= 1 */
    int32_t min_candidates;  /* >= 0 (<= 2 with distinct_hits) */
    float t_xz, t_yz;        /* >= 0, finite */
    int32_t distinct_hits;   /* 0 (default) or 1 */
} jpsi_params;

typedef struct {
    int64_t n_events;
    int64_t n_hits;
    const float *x, *y, *z; /* z may be NULL when z_layer is given */
    const int32_t *offsets;
    const float *z_layer;   /* optional per-layer geometry, see above */
} jpsi_batch;

typedef struct {
    uint32_t *accept_bits;
    int32_t *track_counts;
    int64_t *trip_off;
    int32_t *triplets;
    int64_t trip_capacity; /* rows of 3 int32 */
    int64_t trip_needed;   /* out */
} jpsi_outputs;

typedef struct jpsi_ctx jpsi_ctx;

/* Creates a context on `device`.  hbm_budget bounds the bytes of device
 * scratch the context may hold (0 = 8 GiB).  The context owns its scratch
 * (per-unit counts, scan buffers, work queues, graphs, serving slots).  The
 * paper's CUDA program allocates device memory for every batch before it
 * copies the events over (Sec. 5.3); a context keeps that memory across
 * runs instead.  JPSI_EINVAL for bad parameters or device number, JPSI_ECUDA
 * without a usable device, JPSI_ENOMEM if its control blocks cannot be
 * allocated; *out is NULL unless JPSI_OK. */
jpsi_status jpsi_create(const jpsi_params *params, int device, size_t hbm_budget, jpsi_ctx **out);

/* Releases everything the context owns (it first stops serving and waits
 * for the device).  NULL is ignored.  No counterpart in the paper. */
void jpsi_destroy(jpsi_ctx *ctx);

/* One-launch form: Sec. 5.3's kernel with one thread per event, recast as a
 * static grid with one warp per event, plus a static grid with one block per
 * event for the events too large for a warp's shared-memory tile (the block
 * of an event the warp finished returns at once).  No event lists, work
 * queues or graphs: the baseline the batched form is measured against.
 * `batch` and `out` point to device memory.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream). */
jpsi_status jpsi_run_plain(jpsi_ctx *ctx, const jpsi_batch *batch, jpsi_outputs *out, void *cuda_stream);

/* Batched form of Sec. 3.2 steps 1-3 over a batch of events (the paper
 * times batches of 10^3 to 8*10^4 events per kernel, Table 1): persistent
 * kernels over atomic work queues, events split between warp tiles, the
 * block tile and the unpruned kernel by their size (jpsi_tuning), the phases
 * replayed from captured CUDA graphs.  `batch` and `out` point to device
 * memory; `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 * Same contract and bit-identical results as jpsi_run_plain. */
jpsi_status jpsi_run(jpsi_ctx *ctx, const jpsi_batch *batch, jpsi_outputs *out, void *cuda_stream);

/* jpsi_run on HOST memory: `batch` and `out` point to host buffers (pinned
 * for full speed).  The library copies inputs into device buffers it keeps
 * resident, runs, and copies the outputs back before returning; Sec. 5.3
 * copies the events to the GPU and the selected events back, and Table 1
 * reports that transfer beside the kernel time.  Batches of at least 131,072
 * events in CHAIN mode are copied in chunks while earlier chunks are counted
 * (the paper notes that the transfer can be overlapped with computation); in
 * PAPER mode, pinned inputs are read in place and only the trigger station
 * crosses the link (the paper's host-side trigger filtering, Sec. 5.3).
 * Errors as for jpsi_run. */
jpsi_status jpsi_run_host(jpsi_ctx *ctx, const jpsi_batch *batch, jpsi_outputs *out, void *cuda_stream);

/* Free-streaming selection: an extension.  The paper's Outlook (Sec. 8)
 * notes that CBM's data acquisition will deliver free-streaming data, hits
 * with times and no event association, so that hit times and event building
 * have to enter the selection; it gives no rule.  This library's rule:
 *   - a timeslice holds hits x, y, z, t (t in ns) grouped per (station,
 *     layer): offsets [n_stations*3 + 1], hits of layer l of station s at
 *     [offsets[s*3+l], offsets[s*3+l+1]), each group sorted by t
 *     (non-decreasing, no NaN); z may be NULL with z_layer [n_stations*3];
 *   - window k (0 .. n_windows-1) is [bounds[k], bounds[k+1]) (bounds
 *     finite and strictly increasing);
 *   - a triplet counts only when its hits are coincident, max t <=
 *     fl32(min t + dt), and it belongs to the window holding its earliest
 *     time, so a triplet across a boundary counts once;
 *   - CHAIN: a passing trigger triplet T of window k is a candidate when
 *     every other station holds a passing coincident triplet (anywhere in
 *     the timeslice) compatible with T whose six hits together are
 *     coincident.
 * Outputs as for jpsi_run with windows in place of events; a triplet row
 * (i, j, k) of unit w*S + s names hits offsets[3s] + i, offsets[3s+1] + j,
 * offsets[3s+2] + k of the timeslice.  All pointers are device memory.  The
 * library builds one event per window on the device (its hits within the
 * window's time range) and keeps that copy in its scratch, so the budget
 * must hold about 16 bytes per hit of the windows' ranges.  JPSI_EINVAL for a
 * malformed timeslice (the time order, NaN times, z <= 0 and the bounds are
 * checked on the device), for distinct_hits = 1, and when the windows'
 * ranges hold 2^31 hits or more (split the timeslice).  jpsi_run_stream runs
 * the batched form, jpsi_run_stream_plain the one-launch form; both give the
 * same results. */
typedef struct {
    int64_t n_hits;
    const float *x, *y, *z, *t;
    const int32_t *offsets;   /* [n_stations * 3 + 1] */
    const float *z_layer;     /* optional, as in jpsi_batch */
    int64_t n_windows;
    const float *bounds;      /* [n_windows + 1] */
    float dt;                 /* coincidence width, ns: finite, >= 0 */
} jpsi_timeslice;
jpsi_status jpsi_run_stream(jpsi_ctx *ctx, const jpsi_timeslice *ts, jpsi_outputs *out, void *cuda_stream);
jpsi_status jpsi_run_stream_plain(jpsi_ctx *ctx, const jpsi_timeslice *ts, jpsi_outputs *out, void *cuda_stream);

/* How a context maps the work onto the GPU.  The paper has no counterpart
 * (its one kernel has one thread per event, Sec. 5.3); none of these knobs
 * changes a result.
 *   light_wpb          warps per block of the small warp-tile kernel: 2, 4 or 8.
 *   light_grab         events a persistent warp takes per atomic grab: 1 .. 64.
 *   small_layer_cap    most hits in any layer of a processed station for an
 *                      event to stay on the small warp tile: 1 .. 192.
 *   medium_layer_cap   the same for the medium warp tile: 1 .. 384; events
 *                      beyond both go to the block tile (or, past its limits,
 *                      to the unpruned kernel).
 *   heavy_ctas_per_sm  persistent block-tile CTAs per SM: 0 = as many as fit,
 *                      else 1 .. that many.
 *   record_cap         triplet rows the counting pass may record for the
 *                      scatter: -1 = as needed within the budget, 0 = none
 *                      (rows are then written by a second enumeration),
 *                      > 0 = at most that many.
 * jpsi_set_tuning returns JPSI_EINVAL for a value out of range and then
 * changes nothing. */
typedef struct {
    int32_t light_wpb;
    int32_t light_grab;
    int32_t small_layer_cap;
    int32_t medium_layer_cap;
    int32_t heavy_ctas_per_sm;
    int32_t reserved; /* 0 */
    int64_t record_cap;
} jpsi_tuning;
jpsi_status jpsi_get_tuning(const jpsi_ctx *ctx, jpsi_tuning *out);
jpsi_status jpsi_set_tuning(jpsi_ctx *ctx, const jpsi_tuning *tuning);

/* Picks the batched form's tuning (warps per block and events per grab of the
 * small warp tile, the small and medium tiles' layer cutoffs, block-tile CTAs
 * per SM) by timing candidates on `sample` (device memory) and keeps the
 * fastest in the context; record_cap is left as it is.  No counterpart in
 * the paper.  Results do not depend on the choice.  If no candidate ran, the
 * previous tuning is kept and the first failed run's status is returned.
 * JPSI_EBUSY while serving (the slots' graphs are fixed). */
jpsi_status jpsi_autotune(jpsi_ctx *ctx, const jpsi_batch *sample);

/* ------------------------------------------------------------ serving
 * Continuous batching of timeslices; no counterpart in the paper, whose
 * Outlook (Sec. 8) only anticipates a free-streaming data flow.
 * jpsi_serve_start reserves `n_slots`
 * resident slots whose device buffers fit `slot_hits` hits, `slot_events`
 * events and `slot_triplets` triplets each, within the context's budget.
 * jpsi_serve_submit hands one batch to a free slot, which runs it on its own
 * stream (the call blocks while all slots are busy: back-pressure, nothing is
 * dropped).  The batch's arrays and the outputs may each be in host memory or
 * in device memory of the context's device.  When all of them are in device
 * memory of that device the slot reads and writes them in place, as jpsi_run
 * does; otherwise it copies the batch into its resident buffers and the
 * outputs back into `out` (the copies follow the pointers).  They must stay
 * valid until jpsi_serve_wait returns for the ticket.  Each result is
 * identical to jpsi_run on the same batch alone (the order of rows inside a
 * unit is unspecified, as for jpsi_run). */
jpsi_status jpsi_serve_start(jpsi_ctx *ctx, int n_slots, int64_t slot_events, int64_t slot_hits,
                             int64_t slot_triplets);
jpsi_status jpsi_serve_submit(jpsi_ctx *ctx, const jpsi_batch *batch, jpsi_outputs *out, uint64_t *ticket);
/* Waits at most timeout_ms (< 0: no limit) for `ticket`; on completion writes
 * the run's status and its latency (submit -> outputs in host memory). */
jpsi_status jpsi_serve_wait(jpsi_ctx *ctx, uint64_t ticket, int timeout_ms, jpsi_status *result,
                            double *latency_s);
jpsi_status jpsi_serve_stop(jpsi_ctx *ctx);

/* Host-side fault injection, for tests of the error paths (no counterpart in
 * the paper).  Nothing is injected on the GPU: the library only behaves as if
 * a host call had failed.
 *   JPSI_FAULT_ALLOC  the context's next `count` device allocations fail as
 *                     cudaMalloc would; the call that needed one returns
 *                     JPSI_ENOMEM and the context stays usable.
 *   JPSI_FAULT_RUN    the next `count` runs of serving slots fail with
 *                     JPSI_ECUDA before anything is copied or launched.  A
 *                     slot repeats a run that failed with anything but
 *                     JPSI_EINVAL or JPSI_ECAPACITY once, and reports the
 *                     second attempt's status: one injected failure is
 *                     absorbed, two are reported.
 * count = 0 clears the kind; count < 0 or an unknown kind: JPSI_EINVAL. */
enum { JPSI_FAULT_ALLOC = 1, JPSI_FAULT_RUN = 2 };
jpsi_status jpsi_inject_fault(jpsi_ctx *ctx, int kind, int count);

/* Device-time accounting of runs, for roofline measurements (the paper times
 * its kernel and the transfers separately, Table 1).  While enabled,
 * each run records CUDA events on its stream around its phases: the
 * warp-per-event counting kernel (light_ms), the rest of the counting phase
 * (block-per-event kernel, accept bits, scan: count_rest_ms) and the
 * triplet-writing phase (emit_ms).  Enabling resets the totals.  The last
 * two int fields report the batched form's current launch shape (warps per
 * block and events per grab of the warp-per-event kernel, as chosen by
 * jpsi_autotune or the defaults 4 and 2).  window_ms: free-streaming runs'
 * event building (window ranges, their scan, the gather of the window
 * batch, and the mapping of triplet rows back to the timeslice). */
typedef struct {
    int64_t runs;
    int64_t kernel_launches; /* kernels of this library launched by those runs */
    double light_ms, count_rest_ms, emit_ms;
    int32_t light_wpb, light_grab;
    double window_ms;
} jpsi_timing;
jpsi_status jpsi_timing_enable(jpsi_ctx *ctx, int enable);
jpsi_status jpsi_timing_get(jpsi_ctx *ctx, jpsi_timing *out);

/* ------------------------------------------------- allocation-free counting
 * The paper has no counterpart to this entry point; it serves callers that
 * must not allocate device memory while they run: for example a trigger
 * process that reserves all of its GPU memory at start-up so that no
 * cudaMalloc (which can synchronise the device and take milliseconds) ever
 * lands in its latency budget, a plug-in running inside another program's
 * event loop whose memory is owned by that program's allocator, or code that
 * must not call cudaMalloc/cudaFree between its own stream operations.
 *
 * Counts passing triplets per unit and track candidates per event, exactly
 * as jpsi_run does, without a context and without allocating: no cudaMalloc,
 * cudaFree, host pinning or allocating library call.  Its only scratch is one
 * file-scope device array of about 3.4 MB (job descriptor, control block and
 * per-event bookkeeping for at most 262,144 events) that every GPU which loads
 * the library holds until the process exits.
 *   batch          device memory as for jpsi_run; n_events <= 262,144, else
 *                  JPSI_EINVAL before anything runs.
 *   track_counts   int32 [n_events] device, caller-owned (accept an event iff
 *                  track_counts[e] >= min_candidates).
 *   unit_counts    int32 [n_events * n_stations] device, caller-owned: passing
 *                  triplets per unit (the counts jpsi_run scans into trip_off).
 * Only events that fit the warp tiles (192 hits per layer, 384 per station, at
 * most 32 passing trigger triplets in CHAIN mode, finite pruning bounds) are
 * handled; a batch holding any other event returns JPSI_EINVAL (use jpsi_run).
 * distinct_hits = 1 is not supported here (JPSI_EINVAL): it changes accept
 * bits only, which this entry point does not return.
 * The call is synchronous on `cuda_stream`.  The first call on a device looks
 * up the array's device address for that device (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents (each call clears what must start at
 * zero), so calls that overlap on the GPU (other streams, other threads) race:
 * serialise them. */
jpsi_status jpsi_select_noalloc(const jpsi_params *params, const jpsi_batch *batch, int32_t *track_counts,
                                int32_t *unit_counts, void *cuda_stream);

/* Static description of a status code (no counterpart in the paper). */
const char *jpsi_strerror(jpsi_status status);

/* Detail of the last error seen on this context (empty if none; no
 * counterpart in the paper). */
const char *jpsi_last_error(const jpsi_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* JPSI_H */
