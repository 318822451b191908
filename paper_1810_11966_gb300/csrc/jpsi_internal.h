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
};

// A passing triplet recorded by the counting pass: unit, rank inside the
// unit, and (i, j, k) packed 21 bits each; bit 63 marks entries written by
// the block-per-event kernel.
struct TripEntry {
    int32_t unit;
    int32_t rank;
    unsigned long long ijk;
};
constexpr unsigned long long kFromGeneric = 1ull << 63;
constexpr int32_t kPackLimit = 1 << 21;

// Device-resident control block of one run (zeroed before each run).
struct Ctrl {
    int32_t status;
    int32_t n_generic;            // events sent to the block-per-event kernel
    unsigned long long work[4];   // persistent work counters: light count, generic count, light emit, generic emit
    int64_t trip_total;           // copy of trip_off[n_units]
    unsigned long long scratch_n; // triplet entries appended by the counting pass
};

// Everything a run's kernels read; lives in device memory so a captured
// graph can be replayed for any batch after the host rewrites it.
struct Job {
    const float* x;
    const float* y;
    const float* z;
    const int32_t* off;
    int64_t n_events;
    int64_t n_hits;
    int32_t S, trig, mode, minc;
    float cx, cy, K;
    int32_t grab;                 // events per atomic grab (persistent light kernel)
    int32_t* unit_counts;         // [n_events*S]
    int32_t* track_counts;        // [n_events]
    uint8_t* ev_class;            // [n_events]: 0 light, 1 block-per-event
    int32_t* glist;               // [n_events] events for the block-per-event kernel
    uint32_t* accept_bits;        // may be null
    int64_t* trip_off;            // [n_units + 1]
    int64_t* block_sums;          // scan scratch
    int32_t* triplets;            // may be null
    TripEntry* tscr;              // counting-pass triplet entries (null: not recorded)
    int64_t tscr_cap;
    Ctrl* ctrl;
};

struct LaunchCfg {
    int light_wpb = 4;            // warps per block of the warp-per-event kernel
    int light_blocks = 0;         // persistent grid (0 = static, one warp per event)
    int generic_threads = 256;
    int generic_blocks = 0;       // grid of the block-per-event kernel
    int scan_blocks = 0;
};

// Launchers (jpsi_kernels.cu).  All asynchronous on `st`.
// Count phase = light kernel, then the rest (block-per-event kernel, accept
// bits, scan).  Kernel launches per call: 1 and 5.
cudaError_t launch_light_count(const Job* djob, int64_t n_events, const LaunchCfg& lc, bool persistent,
                               cudaStream_t st);
cudaError_t launch_count_rest(const Job* djob, const LaunchCfg& lc, cudaStream_t st);
constexpr int kLaunchesLight = 1, kLaunchesRest = 5, kLaunchesEmit = 2;
// Places the counting pass's triplet entries at trip_off[unit] + rank.
cudaError_t launch_scatter(const Job* djob, const LaunchCfg& lc, cudaStream_t st);
constexpr int kLaunchesScatter = 1;
// Emit phase (fallback when the entries overflowed): light emit kernel and
// block-per-event emit kernel re-enumerate the units.
cudaError_t launch_emit_phase(const Job* djob, int64_t n_events, const LaunchCfg& lc, bool persistent,
                              cudaStream_t st);
size_t light_smem_bytes(int wpb);
int light_max_blocks_per_sm(int wpb);
int generic_max_blocks_per_sm(int threads);
const void* light_count_kernel_ptr();

}  // namespace jpsi
