// Internal interface between the C-ABI layer (jpsi_api.cu) and the kernels
// (jpsi_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace jpsi {

constexpr int kMaxStations = 16;

// Status bits written by kernels into Ctrl::status.
enum : int32_t {
    kStInvalid = 1,        // malformed offsets or z <= 0
    kStEmitMismatch = 2,   // emit pass found a different count than the count pass (internal error)
    kStNoScratch = 4,      // a triplet index did not fit the scratch entry format
    kStNoPool = 8,         // distinct_hits: the candidates' hits found no room in the trigger pool
    kStBounds = 16,        // checked build: a store with an index outside its array was skipped
};

// Checked build.  Compiled with -DJPSI_CHECKED=1 (libjpsi_checked.so, which
// the tests run the parity suite on; the stand-in for a device memory
// checker), every store whose index comes from data, a scan or a counter
// tests the index against its array's extent first: JPSI_IN(ctrl, ok) is
// `ok`, and a false `ok` skips the store and sets kStBounds in the run's
// status word, which fails the run with JPSI_ECUDA.  In the normal build
// JPSI_IN is `true` and the test disappears.
#if defined(JPSI_CHECKED) && JPSI_CHECKED
#define JPSI_IN(ctrl, ok) ((ok) || (atomicOr(&(ctrl)->status, (int32_t)kStBounds), false))
#else
#define JPSI_IN(ctrl, ok) true
#endif

// Layer-local indices (i, j, k) of a trigger triplet, 21 bits each.
__host__ __device__ inline unsigned long long pack_ijk(int i, int j, int k) {
    return (unsigned long long)i | ((unsigned long long)j << 21) | ((unsigned long long)k << 42);
}
// Do two packed triplets use no common hit (each layer's index differs)?
__host__ __device__ inline bool ijk_disjoint(unsigned long long a, unsigned long long b) {
    const unsigned long long d = a ^ b, m = (1ull << 21) - 1;
    return (d & m) && ((d >> 21) & m) && ((d >> 42) & m);
}

// A passing triplet recorded by the counting pass: unit, rank inside the
// unit, (i, j, k) packed 20 bits each, and in bits 60-62 the class of the
// path that wrote it, which must match the path that finally owned the event.
struct TripEntry {
    int32_t unit;
    int32_t rank;
    unsigned long long ijk;
};
constexpr int kTagShift = 60;
constexpr int32_t kPackLimit = 1 << 20;

// Event classes (Job::ev_class).
enum : uint8_t { kClsLight = 0, kClsHeavy = 1, kClsInvalid = 2, kClsGeneric = 3, kClsMedium = 4 };

// Device-resident control block of one run (zeroed before each run).  The
// three event lists grow over the whole run: a run counted chunk by chunk
// appends every chunk's events behind the previous chunk's, and each
// counting pass takes the list entries from its *_begin on (the emit pass
// over the whole batch starts them at 0 again).
struct Ctrl {
    int32_t status;
    int32_t n_medium;             // events sent to the medium warp kernel
    int32_t n_heavy;              // events sent to the block-tile kernel
    int32_t n_generic;            // events sent to the unpruned block kernel
    int32_t m_begin;              // first medium / block-tile / unpruned list entry
    int32_t h_begin;              //   of the current pass (same order as the
    int32_t g_begin;              //   three counts above)
    int32_t pad_;
    // persistent work counters: small, medium, heavy, generic (count); same
    // (emit); [8] per-station units of the block-tile path (count)
    unsigned long long work[10];
    unsigned long long tpool_n;   // trigger slopes placed in the pool
    int64_t trip_total;           // copy of trip_off[n_units]
    unsigned long long scratch_n; // triplet entries appended by the counting pass
};

// Everything a run's kernels read.  Kernels take it by value (a
// __grid_constant__ parameter); a captured graph gets the current job
// written into its kernel nodes before each replay.
struct Job {
    const float* x;
    const float* y;
    const float* z;
    const int32_t* off;
    int64_t n_events;             // events of the whole batch
    int64_t n_hits;
    int64_t ev_begin, ev_count;   // events the warp kernels take from the batch (all by default)
    int32_t S, trig, mode, minc;
    int32_t distinct;             // distinct_hits: accept bits from dpair when minc == 2
    // free-streaming windows (events are time windows built from a
    // timeslice): a triplet counts when coincident, max t <= fl32(min t + dt),
    // and owned by its window, wb[e] <= min t < wb[e + 1]; CHAIN partners
    // must be coincident with the trigger triplet
    int32_t stream;
    float dt;
    const float* t;               // [n_hits] hit times (stream)
    const float* wb;              // [n_events + 1] window bounds (stream)
    float cx, cy, K;
    int32_t grab;                 // events per atomic grab (persistent light kernel)
    int32_t cap_small, cap_medium;// most hits per layer on the small / medium warp tile (<= the tile's own)
    int32_t persistent;           // warp kernels: persistent warps (1) or one warp per event (0)
    int32_t plain;                // one-launch form: no event lists (events carry their class only)
    int32_t host_hits;            // x, y, z, off are pinned host memory read over the link: no L2 prefetch
    int32_t* unit_counts;         // [n_events*S]
    int32_t* track_counts;        // [n_events]
    uint8_t* ev_class;            // [n_events]: kCls*
    int32_t* mlist;               // [n_events] events for the medium warp kernel
    int32_t* hlist;               // [n_events] events for the block-tile kernel
    int32_t* glist;               // [n_events] events for the unpruned block kernel
    float2* tlist;                // [heavy blocks * tlist_cap] trigger slopes (block-tile kernel)
    uint8_t* talive;              // [heavy blocks * tlist_cap]
    int32_t tlist_cap;
    float2* tpool;                // [tpool_cap] trigger slopes of block-tile events split by station
    uint8_t* tpool_alive;         // [tpool_cap]
    int64_t tpool_cap;
    int2* hT;                     // [n_events] per block-tile list entry: pool start, slope count or state
    uint8_t* dpair;               // [n_events] distinct_hits: two candidates share no hit
    unsigned long long* tlist_ijk;// [heavy blocks * tlist_cap] distinct_hits: candidates' packed hits
    unsigned long long* tpool_ijk;// [tpool_cap] distinct_hits
    uint32_t* accept_bits;        // may be null
    int64_t* trip_off;            // [n_units + 1]
    int64_t* block_sums;          // scan scratch
    int32_t* triplets;            // may be null
    int64_t trip_cap;             // rows the triplet buffer holds
    TripEntry* tscr;              // counting-pass triplet entries (null: not recorded)
    int64_t tscr_cap;
    Ctrl* ctrl;
};

struct LaunchCfg {
    int light_wpb = 4;            // warps per block of the warp-per-event kernel
    int light_blocks = 0;         // persistent grid (0 = static, one warp per event)
    int medium_blocks = 0;        // grid of the medium warp kernel (4 warps per block)
    int generic_threads = 256;
    int generic_blocks = 0;       // grid of the unpruned block kernel
    int heavy_blocks = 0;         // grid of the block-tile kernel
    int scan_blocks = 0;
};

// Launchers (jpsi_kernels.cu), declared for both builds of that file: the
// event kernels (jpsi::basek) and those of free-streaming windows
// (jpsi::streamk).  All asynchronous on `st`.
//   launch_light_count, launch_count_rest: the counting phase = the small
//     warp kernel (1 launch), then the rest (medium tile, block tiles,
//     unpruned kernel, accept bits, scan: 10 launches).
//   launch_count_lists, launch_count_tail: the rest split in two, for counting
//     a batch chunk by chunk (6 + 4 launches).
//   launch_scatter: the counting pass's triplet entries to trip_off[unit] + rank.
//   launch_emit_phase: the fallback when the entries overflowed; the
//     enumeration kernels write rows at trip_off (4 launches).
//   launch_plain_*: the one-launch form (no lists, queues or graphs): the
//     static warp grid (1), then the static block grid and the tail (1 + 4);
//     its emit fallback is the two static grids again (2).
//   launch_expand_z: per-hit z of events [ev0, ev1) from a per-layer table.
#define JPSI_DECLARE_LAUNCHERS                                                                                  \
    cudaError_t launch_light_count(const Job& j, int64_t n_events, const LaunchCfg& lc, bool persistent,    \
                                   cudaStream_t st);                                                          \
    cudaError_t launch_count_rest(const Job& j, const LaunchCfg& lc, cudaStream_t st);                        \
    cudaError_t launch_count_lists(const Job& j, const LaunchCfg& lc, cudaStream_t st);                       \
    cudaError_t launch_count_tail(const Job& j, const LaunchCfg& lc, cudaStream_t st);                        \
    cudaError_t launch_scatter(const Job& j, const LaunchCfg& lc, cudaStream_t st);                           \
    cudaError_t launch_emit_phase(const Job& j, int64_t n_events, const LaunchCfg& lc, bool persistent,     \
                                  cudaStream_t st);                                                           \
    cudaError_t launch_plain_light(const Job& j, const LaunchCfg& lc, cudaStream_t st);                       \
    cudaError_t launch_plain_rest(const Job& j, const LaunchCfg& lc, cudaStream_t st);                        \
    cudaError_t launch_plain_emit(const Job& j, const LaunchCfg& lc, cudaStream_t st);                        \
    cudaError_t launch_expand_z(const int32_t* off, const float* z_layer, float* z, int64_t ev0, int64_t ev1, \
                                int S, int64_t n_hits, int n_sm, cudaStream_t st);                            \
    size_t light_smem_bytes(int wpb);                                                                         \
    int light_max_blocks_per_sm(int wpb);                                                                     \
    int generic_max_blocks_per_sm(int threads);                                                               \
    int heavy_max_blocks_per_sm();                                                                            \
    int medium_max_blocks_per_sm();                                                                           \
    size_t heavy_smem_bytes();                                                                                \
    const void* light_count_kernel_ptr();

namespace basek {
JPSI_DECLARE_LAUNCHERS
}
namespace streamk {
JPSI_DECLARE_LAUNCHERS
}

// Event building for free-streaming timeslices: window k becomes event k
// whose layer group g holds the timeslice hits of group g in a time range
// (the trigger station: [b_k, fl32(b_k+1 + dt)]; the other stations of CHAIN
// mode from a margin below b_k - dt to the same end; PAPER mode's other
// stations: none).
struct WinJob {
    const float *x, *y, *z, *t;
    const float* z_layer;  // per-group z when z is null
    const int32_t* off;    // [3S + 1] timeslice layer groups (checked on the host)
    const float* wb;       // [K + 1] window bounds
    int64_t n_hits, K;
    int32_t S, trig, chain;
    float dt;
    int32_t* wlo;          // [K*3S] first timeslice hit of each range
    int32_t* wcnt;         // [K*3S] hits of each range
    int64_t* woff;         // [K*3S + 1] exclusive scan of wcnt
    int64_t* block_sums;   // scan scratch
    int32_t* off_out;      // [K*3S + 1] the window batch's offsets
    float *xo, *yo, *zo, *to;  // [total] the window batch's hits
    Ctrl* ctrl;            // status (kStInvalid) and trip_total = the window batch's hits
    int n_sm;
};
namespace streamk {
//   launch_window_ranges: validates the timeslice (times sorted per group, no
//     NaN; z > 0 where read; bounds finite and increasing), finds each
//     window's ranges and scans their sizes (4 launches).
//   launch_window_gather: the window batch's offsets and hits (1 launch).
//   launch_window_rows: triplet rows from window-batch indices to timeslice
//     layer-group indices (1 launch).
cudaError_t launch_window_ranges(const WinJob& w, cudaStream_t st);
cudaError_t launch_window_gather(const WinJob& w, cudaStream_t st);
cudaError_t launch_window_rows(const WinJob& w, const int64_t* trip_off, int32_t* triplets, cudaStream_t st);
}  // namespace streamk
constexpr int kLaunchesWindows = 6;
constexpr int kLaunchesLight = 1, kLaunchesRest = 10, kLaunchesEmit = 4;
constexpr int kLaunchesScatter = 1;
constexpr int kLaunchesPlainLight = 1, kLaunchesPlainRest = 5, kLaunchesPlainEmit = 2;
constexpr int kHeavyTCap = 1 << 15;  // trigger triplets per event on the block-tile path


}  // namespace jpsi
