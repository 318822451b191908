// C-ABI of libjpsi (include/jpsi.h): contexts, scratch management, the
// plain and batched run forms, host-buffer runs, the autotuner and the
// continuous-batching serving loop.  All device work is in jpsi_kernels.cu.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <deque>
#include <initializer_list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "jpsi.h"
#include "jpsi_internal.h"

using namespace jpsi;
using namespace jpsi::basek;  // the event kernels; stream runs take jpsi::streamk's launchers

namespace {

// NVTX range around a host call (header-only NVTX: a no-op unless a profiler
// such as Nsight Systems is attached)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

constexpr size_t kDefaultBudget = (size_t)8 << 30;
// what a run of the checked build reports when one of its kernels skipped a
// store outside its array (the normal build never sets the bit)
constexpr const char* kBoundsMsg = "checked build: a store outside its array was skipped";
constexpr int kMaxChunks = 8;            // jpsi_run_host pipelines copies and counting in up to 8 chunks
constexpr int64_t kChunkMinEvents = 65536;

// Trigger-slope pool of the block-tile path for a batch of `ne` events (an
// event whose slopes find no room runs all its stations on one block).
int64_t tpool_entries(int64_t ne) { return std::min<int64_t>(std::max<int64_t>(ne * 64, 1 << 16), 1 << 24); }

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct HostBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// One captured phase of the batched form: the graph (kept for its kernel
// node handles), its executable form and each kernel node's launch shape,
// re-applied with the current job before every replay.
struct Graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> nodes;
    std::vector<cudaKernelNodeParams> params;
};

// Per-run state: job, control block, graphs.  The serving loop owns one per
// slot; plain runs use the context's own.
struct RunState {
    Job job{};                // the current run's job (passed to every kernel by value)
    Ctrl* d_ctrl = nullptr;
    Ctrl* h_ctrl = nullptr;   // pinned
    DevBuf unit_counts, track_counts, ev_class, mlist, hlist, glist, block_sums, trip_off, tscr, tlist, talive;
    DevBuf tpool, tpool_alive, hT;
    DevBuf dpair, tlist_ijk, tpool_ijk;  // distinct_hits
    DevBuf zfill, ztab;  // per-hit z filled from a batch's z_layer table; the table on the device
    int64_t tscr_want = (int64_t)1 << 22;  // entries; grows after an overflow
    Graph g_light, g_rest, g_emit, g_scatter;
    int g_cfg_id = -1;
    bool g_stream = false;  // the graphs hold the free-streaming kernels
    cudaEvent_t ev[9] = {};  // timing marks: light start/end, rest end, emit start/end; window build and rows
    cudaEvent_t chunk_ev[kMaxChunks] = {};  // hit chunks copied (pipelined host run)
};

struct Slot {
    RunState rs;
    DevBuf x, y, z, off, accept, tracks, trip_off, triplets;
    int64_t cap_events = 0, cap_hits = 0, cap_trip = 0;
    cudaStream_t stream = nullptr;
    // current request
    jpsi_batch batch{};
    jpsi_outputs* out = nullptr;
    uint64_t ticket = 0;
    std::chrono::steady_clock::time_point t_submit;
    bool busy = false;
};

struct Done {
    jpsi_status st;
    double latency;
};

// The launchers of one build of the kernels: the event kernels or those of
// free-streaming windows (time tests compiled in).
struct Launchers {
    bool stream;
    decltype(&basek::launch_light_count) light_count;
    decltype(&basek::launch_count_rest) count_rest;
    decltype(&basek::launch_emit_phase) emit_phase;
    decltype(&basek::launch_scatter) scatter;
    decltype(&basek::launch_plain_light) plain_light;
    decltype(&basek::launch_plain_rest) plain_rest;
    decltype(&basek::launch_plain_emit) plain_emit;
};
const Launchers kEventL{false, basek::launch_light_count, basek::launch_count_rest, basek::launch_emit_phase,
                        basek::launch_scatter, basek::launch_plain_light, basek::launch_plain_rest,
                        basek::launch_plain_emit};
// Time inputs of a run over free-streaming windows (device pointers).
struct StreamJob {
    const float* t;   // [window-batch hits]
    const float* wb;  // [n_windows + 1]
    float dt;
};

const Launchers kStreamL{true, streamk::launch_light_count, streamk::launch_count_rest, streamk::launch_emit_phase,
                         streamk::launch_scatter, streamk::launch_plain_light, streamk::launch_plain_rest,
                         streamk::launch_plain_emit};

}  // namespace

struct jpsi_ctx {
    jpsi_params p{};
    int device = 0;
    size_t budget = 0;
    size_t used = 0;
    int n_sm = 0;
    bool pageable_ok = false;
    float cx = 0, cy = 0, K = 0;
    LaunchCfg plain_cfg, batch_cfg;
    jpsi_tuning tune{4, 2, 192, 384, 0, 0, -1};
    int cfg_id = 0;  // bumps when the launch shape changes (graphs re-captured)
    cudaStream_t cap_stream = nullptr;
    cudaStream_t copy_stream = nullptr;  // host-to-device copies of jpsi_run_host
    RunState rs;
    // device copies for jpsi_run_host
    DevBuf hx, hy, hz, hoff, hacc, htc, htoff, htrip;
    // window batch of a free-streaming run: ranges, their scan, offsets, hits
    DevBuf wlo, wcnt, woff, wbs, woff32, wx, wy, wz, wt;
    std::string last_error;
    std::mutex err_mu, cap_mu, alloc_mu;
    std::atomic<bool> timing{false};
    jpsi_timing tm{};
    std::atomic<bool> busy{false};
    // serving
    std::mutex mu;
    std::condition_variable cv;
    std::vector<Slot*> slots;
    std::vector<std::thread> workers;
    std::deque<int> free_slots;
    std::map<uint64_t, Done> done;
    uint64_t next_ticket = 1;
    bool serving = false, stopping = false;
    std::vector<std::condition_variable*> slot_cv;
    // host-side fault injection (jpsi_inject_fault)
    std::atomic<int> fault_alloc{0}, fault_run{0};
};

namespace {

struct BusyGuard {
    jpsi_ctx* c;
    bool ok;
    explicit BusyGuard(jpsi_ctx* ctx) : c(ctx) {
        bool expected = false;
        ok = c->busy.compare_exchange_strong(expected, true);
    }
    ~BusyGuard() {
        if (ok) c->busy.store(false);
    }
};

jpsi_status fail(jpsi_ctx* c, jpsi_status st, const std::string& msg) {
    if (c) {
        std::lock_guard<std::mutex> lk(c->err_mu);
        c->last_error = msg;
    }
    return st;
}

jpsi_status cuda_fail(jpsi_ctx* c, cudaError_t e, const char* where) {
    return fail(c, JPSI_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Takes one injected fault of a kind, if any is left.
bool take_fault(std::atomic<int>& left) {
    int v = left.load();
    while (v > 0)
        if (left.compare_exchange_weak(v, v - 1)) return true;
    return false;
}

// Grows a device buffer within the context budget (contents not kept).
jpsi_status ensure(jpsi_ctx* c, DevBuf& b, size_t bytes, const char* what) {
    if (bytes <= b.bytes) return JPSI_OK;
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    const size_t nb = std::max(bytes, b.bytes + b.bytes / 4);
    const size_t extra = nb - b.bytes;
    if (c->used + extra > c->budget)
        return fail(c, JPSI_ENOMEM, std::string("scratch for ") + what + " exceeds the device budget");
    if (take_fault(c->fault_alloc)) return fail(c, JPSI_ENOMEM, std::string("injected allocation failure for ") + what);
    void* p = nullptr;
    if (cudaMalloc(&p, nb) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, JPSI_ENOMEM, std::string("cudaMalloc failed for ") + what);
    }
    if (b.p) cudaFree(b.p);
    c->used = c->used - b.bytes + nb;
    b.p = p;
    b.bytes = nb;
    return JPSI_OK;
}

void release(jpsi_ctx* c, DevBuf& b) {
    std::lock_guard<std::mutex> lk(c->alloc_mu);
    if (b.p) cudaFree(b.p);
    c->used -= b.bytes;
    b = DevBuf{};
}

jpsi_status params_ok(const jpsi_params* p) {
    if (!p) return JPSI_EINVAL;
    if (p->n_stations < 1 || p->n_stations > kMaxStations) return JPSI_EINVAL;
    if (p->trigger_station < 0 || p->trigger_station >= p->n_stations) return JPSI_EINVAL;
    if (p->mode != JPSI_MODE_PAPER && p->mode != JPSI_MODE_CHAIN) return JPSI_EINVAL;
    if (p->ndf < 1 || p->min_candidates < 0) return JPSI_EINVAL;
    if (p->distinct_hits != 0 && (p->distinct_hits != 1 || p->min_candidates > 2)) return JPSI_EINVAL;
    if (!(p->t_xz >= 0.0f) || !(p->t_yz >= 0.0f) || std::isinf(p->t_xz) || std::isinf(p->t_yz)) return JPSI_EINVAL;
    return JPSI_OK;
}

// Pruning factor: sqrt(max C) (1 + 1e-4) + 1e-20, rounded up to float.
float pruning_K(float cx, float cy) {
    const double k = std::sqrt((double)std::max(cx, cy)) * (1.0 + 1e-4) + 1e-20;
    float f = (float)k;
    if ((double)f < k) f = std::nextafter(f, INFINITY);
    return f;
}

bool device_accessible(jpsi_ctx* c, const void* p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return c->pageable_ok;
    }
    if (a.type == cudaMemoryTypeDevice) return a.device == c->device;
    if (a.type == cudaMemoryTypeManaged || a.type == cudaMemoryTypeHost) return true;
    return c->pageable_ok;
}

jpsi_status check_batch(jpsi_ctx* c, const jpsi_batch* b, const jpsi_outputs* o, bool device_ptrs) {
    if (!b || !o) return fail(c, JPSI_EINVAL, "null batch or outputs");
    const int64_t S = c->p.n_stations;
    if (b->n_events < 0 || b->n_hits < 0) return fail(c, JPSI_EINVAL, "negative sizes");
    if (b->n_hits >= ((int64_t)1 << 31)) return fail(c, JPSI_EINVAL, "n_hits must be < 2^31");
    if (b->n_events > (((int64_t)1 << 31) - 2) / (3 * S)) return fail(c, JPSI_EINVAL, "too many events for int32 offsets");
    if (b->n_events == 0 && b->n_hits != 0) return fail(c, JPSI_EINVAL, "hits without events");
    if (b->n_events > 0 && !b->offsets) return fail(c, JPSI_EINVAL, "offsets missing");
    if (b->n_hits > 0 && (!b->x || !b->y || (!b->z && !b->z_layer))) return fail(c, JPSI_EINVAL, "hit arrays missing");
    if (o->triplets && !o->trip_off) return fail(c, JPSI_EINVAL, "triplets need trip_off");
    if (o->trip_capacity < 0) return fail(c, JPSI_EINVAL, "negative triplet capacity");
    if (device_ptrs) {
        const void* ptrs[] = {b->x, b->y, b->z, b->offsets, b->z_layer, o->accept_bits, o->track_counts, o->trip_off,
                              o->triplets};
        for (const void* p : ptrs)
            if (!device_accessible(c, p)) return fail(c, JPSI_EINVAL, "pointer is not device-accessible");
    }
    return JPSI_OK;
}

// Prepares scratch and the job descriptor of a run.
jpsi_status prepare(jpsi_ctx* c, RunState& rs, const jpsi_batch* b, jpsi_outputs* o, bool host_hits,
                    bool stream = false) {
    const int64_t S = c->p.n_stations;
    const int64_t ne = b->n_events, nu = ne * S;
    jpsi_status st;
    if ((st = ensure(c, rs.unit_counts, (size_t)std::max<int64_t>(nu, 1) * 4, "unit counts")) != JPSI_OK) return st;
    if ((st = ensure(c, rs.ev_class, (size_t)std::max<int64_t>(ne, 1), "event classes")) != JPSI_OK) return st;
    if ((st = ensure(c, rs.mlist, (size_t)std::max<int64_t>(ne, 1) * 4, "event list")) != JPSI_OK) return st;
    if ((st = ensure(c, rs.hlist, (size_t)std::max<int64_t>(ne, 1) * 4, "event list")) != JPSI_OK) return st;
    if ((st = ensure(c, rs.glist, (size_t)std::max<int64_t>(ne, 1) * 4, "event list")) != JPSI_OK) return st;
    const size_t tl = (size_t)std::max(c->batch_cfg.heavy_blocks, c->plain_cfg.heavy_blocks) * kHeavyTCap;
    if ((st = ensure(c, rs.tlist, tl * sizeof(float2), "trigger lists")) != JPSI_OK) return st;
    if ((st = ensure(c, rs.talive, tl, "trigger lists")) != JPSI_OK) return st;
    const int64_t tp = tpool_entries(ne);
    if ((st = ensure(c, rs.tpool, (size_t)tp * sizeof(float2), "trigger pool")) != JPSI_OK) return st;
    if ((st = ensure(c, rs.tpool_alive, (size_t)tp, "trigger pool")) != JPSI_OK) return st;
    if ((st = ensure(c, rs.hT, (size_t)std::max<int64_t>(ne, 1) * sizeof(int2), "event list")) != JPSI_OK) return st;
    // distinct_hits: the candidates' packed hits; free-streaming windows: the
    // trigger triplets' (earliest, latest) times, in the same arrays
    if (c->p.distinct_hits && (st = ensure(c, rs.dpair, (size_t)std::max<int64_t>(ne, 1), "disjoint flags")) != JPSI_OK)
        return st;
    if ((c->p.distinct_hits || stream) &&
        ((st = ensure(c, rs.tlist_ijk, tl * sizeof(unsigned long long), "trigger lists")) != JPSI_OK ||
         (st = ensure(c, rs.tpool_ijk, (size_t)tp * sizeof(unsigned long long), "trigger pool")) != JPSI_OK))
        return st;
    static_assert(sizeof(float2) == sizeof(unsigned long long), "times share the packed-hit arrays");
    const int64_t ntiles = (nu + 4095) / 4096 + 1;
    if ((st = ensure(c, rs.block_sums, (size_t)ntiles * 8, "scan")) != JPSI_OK) return st;
    if (!o->track_counts && (st = ensure(c, rs.track_counts, (size_t)std::max<int64_t>(ne, 1) * 4, "track counts")))
        return st;
    if (!o->trip_off && (st = ensure(c, rs.trip_off, (size_t)(nu + 1) * 8, "triplet offsets"))) return st;
    Job& j = rs.job;
    j = Job{};
    j.x = b->x;
    j.y = b->y;
    j.z = b->z;
    j.off = b->offsets;
    j.n_events = ne;
    j.n_hits = b->n_hits;
    j.ev_begin = 0;
    j.ev_count = ne;
    j.S = c->p.n_stations;
    j.trig = c->p.trigger_station;
    j.mode = c->p.mode;
    j.minc = c->p.min_candidates;
    j.distinct = c->p.distinct_hits;
    j.dpair = (uint8_t*)rs.dpair.p;
    j.tlist_ijk = (unsigned long long*)rs.tlist_ijk.p;
    j.tpool_ijk = (unsigned long long*)rs.tpool_ijk.p;
    j.cx = c->cx;
    j.cy = c->cy;
    j.K = c->K;
    j.grab = c->tune.light_grab;
    j.cap_small = c->tune.small_layer_cap;
    j.cap_medium = c->tune.medium_layer_cap;
    j.host_hits = host_hits ? 1 : 0;
    j.unit_counts = (int32_t*)rs.unit_counts.p;
    j.track_counts = o->track_counts ? o->track_counts : (int32_t*)rs.track_counts.p;
    j.ev_class = (uint8_t*)rs.ev_class.p;
    j.mlist = (int32_t*)rs.mlist.p;
    j.hlist = (int32_t*)rs.hlist.p;
    j.glist = (int32_t*)rs.glist.p;
    j.tlist = (float2*)rs.tlist.p;
    j.talive = (uint8_t*)rs.talive.p;
    j.tlist_cap = kHeavyTCap;
    j.tpool = (float2*)rs.tpool.p;
    j.tpool_alive = (uint8_t*)rs.tpool_alive.p;
    j.tpool_cap = (int64_t)std::min(rs.tpool.bytes / sizeof(float2), rs.tpool_alive.bytes);
    if (c->p.distinct_hits || stream)
        j.tpool_cap = std::min<int64_t>(j.tpool_cap, (int64_t)(rs.tpool_ijk.bytes / sizeof(unsigned long long)));
    j.hT = (int2*)rs.hT.p;
    j.accept_bits = o->accept_bits;
    j.trip_off = o->trip_off ? o->trip_off : (int64_t*)rs.trip_off.p;
    j.block_sums = (int64_t*)rs.block_sums.p;
    j.triplets = o->triplets;
    j.trip_cap = o->triplets ? o->trip_capacity : 0;
    j.tscr = nullptr;
    j.tscr_cap = 0;
    if (o->triplets && c->tune.record_cap != 0) {
        // entries of the counting pass; without room for them the triplets are
        // written by re-enumeration instead (same result, slower).  Entries
        // also come from paths that later hand their event on, so the record
        // may need a little more than the run's triplets.
        const int64_t cap = std::max<int64_t>(o->trip_capacity, 1);
        int64_t n_want = std::min<int64_t>(rs.tscr_want, cap + cap / 4 + 4096);
        if (c->tune.record_cap > 0) n_want = std::min<int64_t>(n_want, c->tune.record_cap);
        const size_t want = (size_t)n_want * sizeof(TripEntry);
        const bool fits = want <= rs.tscr.bytes || c->used + (want - rs.tscr.bytes) <= c->budget;
        if (fits && ensure(c, rs.tscr, want, "triplet entries") == JPSI_OK) {
            j.tscr = (TripEntry*)rs.tscr.p;
            j.tscr_cap = (int64_t)std::min<size_t>(rs.tscr.bytes / sizeof(TripEntry), (size_t)n_want);
        }
    }
    j.ctrl = rs.d_ctrl;
    return JPSI_OK;
}

jpsi_status state_init(jpsi_ctx* c, RunState& rs) {
    if (cudaMalloc(&rs.d_ctrl, sizeof(Ctrl)) != cudaSuccess || cudaMallocHost(&rs.h_ctrl, sizeof(Ctrl)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, JPSI_ENOMEM, "control block allocation failed");
    }
    rs.job = Job{};
    memset(rs.h_ctrl, 0, sizeof(Ctrl));
    for (cudaEvent_t& e : rs.ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(c, JPSI_ECUDA, "event creation failed");
    return JPSI_OK;
}

void destroy_graphs(RunState& rs) {
    Graph* gs[] = {&rs.g_light, &rs.g_rest, &rs.g_emit, &rs.g_scatter};
    for (Graph* g : gs) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->g) cudaGraphDestroy(g->g);
        *g = Graph{};
    }
}

void state_free(jpsi_ctx* c, RunState& rs) {
    destroy_graphs(rs);
    for (cudaEvent_t& e : rs.chunk_ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    for (cudaEvent_t& e : rs.ev) {
        if (e) cudaEventDestroy(e);
        e = nullptr;
    }
    if (rs.d_ctrl) cudaFree(rs.d_ctrl);
    if (rs.h_ctrl) cudaFreeHost(rs.h_ctrl);
    rs.d_ctrl = nullptr;
    rs.h_ctrl = nullptr;
    release(c, rs.unit_counts);
    release(c, rs.track_counts);
    release(c, rs.ev_class);
    release(c, rs.mlist);
    release(c, rs.hlist);
    release(c, rs.glist);
    release(c, rs.tlist);
    release(c, rs.talive);
    release(c, rs.tpool);
    release(c, rs.tpool_alive);
    release(c, rs.hT);
    release(c, rs.dpair);
    release(c, rs.tlist_ijk);
    release(c, rs.tpool_ijk);
    release(c, rs.zfill);
    release(c, rs.ztab);
    release(c, rs.block_sums);
    release(c, rs.trip_off);
    release(c, rs.tscr);
}

// Captures the count and emit phases of the batched form into graphs (with
// the current job; graph_launch writes each run's job into their nodes).
jpsi_status capture_graphs(jpsi_ctx* c, RunState& rs, const Launchers& L = kEventL) {
    if (rs.g_light.exec && rs.g_cfg_id == c->cfg_id && rs.g_stream == L.stream) return JPSI_OK;
    std::lock_guard<std::mutex> cap_lock(c->cap_mu);
    destroy_graphs(rs);
    for (int phase = 0; phase < 4; ++phase) {
        Graph& G = phase == 0 ? rs.g_light : phase == 1 ? rs.g_rest : phase == 2 ? rs.g_emit : rs.g_scatter;
        cudaError_t e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
        cudaError_t le = phase == 0   ? L.light_count(rs.job, 0, c->batch_cfg, true, c->cap_stream)
                         : phase == 1 ? L.count_rest(rs.job, c->batch_cfg, c->cap_stream)
                         : phase == 2 ? L.emit_phase(rs.job, 0, c->batch_cfg, true, c->cap_stream)
                                      : L.scatter(rs.job, c->batch_cfg, c->cap_stream);
        e = cudaStreamEndCapture(c->cap_stream, &G.g);
        if (le != cudaSuccess) return cuda_fail(c, le, "graph capture launch");
        if (e != cudaSuccess) return cuda_fail(c, e, "graph end capture");
        size_t n = 0;
        if ((e = cudaGraphGetNodes(G.g, nullptr, &n)) != cudaSuccess) return cuda_fail(c, e, "graph nodes");
        std::vector<cudaGraphNode_t> all(n);
        if (n && (e = cudaGraphGetNodes(G.g, all.data(), &n)) != cudaSuccess) return cuda_fail(c, e, "graph nodes");
        for (cudaGraphNode_t node : all) {
            cudaGraphNodeType t;
            if ((e = cudaGraphNodeGetType(node, &t)) != cudaSuccess) return cuda_fail(c, e, "graph node type");
            if (t != cudaGraphNodeTypeKernel) continue;
            cudaKernelNodeParams kp{};
            if ((e = cudaGraphKernelNodeGetParams(node, &kp)) != cudaSuccess) return cuda_fail(c, e, "graph node");
            G.nodes.push_back(node);
            G.params.push_back(kp);
        }
        if ((e = cudaGraphInstantiate(&G.exec, G.g, 0)) != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    }
    rs.g_cfg_id = c->cfg_id;
    rs.g_stream = L.stream;
    return JPSI_OK;
}

// Replays a captured phase for `job`: every kernel node of the graph takes
// the job as its only parameter (warp kernels in their persistent form).
cudaError_t graph_launch(Graph& G, const Job& job, cudaStream_t st) {
    Job j = job;
    j.persistent = 1;
    void* args[] = {&j};
    for (size_t i = 0; i < G.nodes.size(); ++i) {
        cudaKernelNodeParams kp = G.params[i];
        kp.kernelParams = args;
        kp.extra = nullptr;
        const cudaError_t e = cudaGraphExecKernelNodeSetParams(G.exec, G.nodes[i], &kp);
        if (e != cudaSuccess) return e;
    }
    return cudaGraphLaunch(G.exec, st);
}

// Accumulates per-phase device times of a finished run (events already complete).
void add_timing(jpsi_ctx* c, RunState& rs, int launches, bool emitted) {
    if (!c->timing.load()) return;
    float a = 0, b = 0, d = 0;
    cudaEventElapsedTime(&a, rs.ev[0], rs.ev[1]);
    cudaEventElapsedTime(&b, rs.ev[1], rs.ev[2]);
    if (emitted) cudaEventElapsedTime(&d, rs.ev[3], rs.ev[4]);
    std::lock_guard<std::mutex> lk(c->err_mu);
    c->tm.runs += 1;
    c->tm.kernel_launches += launches;
    c->tm.light_ms += a;
    c->tm.count_rest_ms += b;
    c->tm.emit_ms += d;
}

// The common run: count phase, status/capacity check, emit phase.
jpsi_status run_device(jpsi_ctx* c, RunState& rs, const jpsi_batch* b, jpsi_outputs* o, cudaStream_t st,
                       bool batched, bool host_hits = false, const Launchers& L = kEventL,
                       const StreamJob* sj = nullptr) {
    jpsi_status s;
    jpsi_batch bz;
    if (!b->z && b->n_hits > 0) {
        // per-hit z from the batch's geometry table (device memory)
        if ((s = ensure(c, rs.zfill, (size_t)b->n_hits * 4, "hits z")) != JPSI_OK) return s;
        const cudaError_t e = launch_expand_z(b->offsets, b->z_layer, (float*)rs.zfill.p, 0, b->n_events,
                                              c->p.n_stations, b->n_hits, c->n_sm, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "z from geometry");
        bz = *b;
        bz.z = (const float*)rs.zfill.p;
        b = &bz;
    }
    if ((s = prepare(c, rs, b, o, host_hits, sj != nullptr)) != JPSI_OK) return s;
    if (sj) {  // free-streaming windows: the time tests' inputs
        rs.job.stream = 1;
        rs.job.dt = sj->dt;
        rs.job.t = sj->t;
        rs.job.wb = sj->wb;
    }
    const int64_t ne = b->n_events;
    cudaError_t e;
    if ((e = cudaMemsetAsync(rs.d_ctrl, 0, sizeof(Ctrl), st)) != cudaSuccess) return cuda_fail(c, e, "ctrl reset");
    if (c->p.distinct_hits && ne > 0 && (e = cudaMemsetAsync(rs.dpair.p, 0, (size_t)ne, st)) != cudaSuccess)
        return cuda_fail(c, e, "flag reset");
    const bool timing = c->timing.load();
    if (batched && (s = capture_graphs(c, rs, L)) != JPSI_OK) return s;
    if (timing) cudaEventRecord(rs.ev[0], st);
    e = batched ? graph_launch(rs.g_light, rs.job, st) : L.plain_light(rs.job, c->plain_cfg, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "light count");
    if (timing) cudaEventRecord(rs.ev[1], st);
    e = batched ? graph_launch(rs.g_rest, rs.job, st) : L.plain_rest(rs.job, c->plain_cfg, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "count rest");
    if (timing) cudaEventRecord(rs.ev[2], st);
    int launches = batched ? kLaunchesLight + kLaunchesRest : kLaunchesPlainLight + kLaunchesPlainRest;
    if ((e = cudaMemcpyAsync(rs.h_ctrl, rs.d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(c, e, "ctrl readback");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "count phase");
    const Ctrl ctl = *rs.h_ctrl;
    if (ctl.status & kStBounds) return fail(c, JPSI_ECUDA, kBoundsMsg);
    if (ctl.status & kStInvalid) return fail(c, JPSI_EINVAL, "malformed offsets or a hit with z <= 0");
    if (ctl.status & kStNoPool) return fail(c, JPSI_ENOMEM, "distinct_hits: candidates exceed the trigger pool");
    o->trip_needed = ctl.trip_total;
    if (!o->triplets) {
        add_timing(c, rs, launches, false);
        return JPSI_OK;
    }
    if (ctl.trip_total > o->trip_capacity)
        return fail(c, JPSI_ECAPACITY, "triplet capacity " + std::to_string(o->trip_capacity) + " < needed " +
                                           std::to_string(ctl.trip_total));
    if (ctl.trip_total == 0) {
        add_timing(c, rs, launches, false);
        return JPSI_OK;
    }
    // triplet rows: scatter the recorded entries, or re-enumerate when they
    // did not fit (then record more next time, within the budget)
    const bool scattered = rs.job.tscr && !(ctl.status & kStNoScratch) &&
                           ctl.scratch_n <= (unsigned long long)rs.job.tscr_cap;
    if (!scattered && rs.job.tscr && !(ctl.status & kStNoScratch))
        rs.tscr_want = std::max<int64_t>(rs.tscr_want, (int64_t)(ctl.scratch_n + ctl.scratch_n / 4));
    if (timing) cudaEventRecord(rs.ev[3], st);
    if (scattered)
        e = batched ? graph_launch(rs.g_scatter, rs.job, st) : L.scatter(rs.job, c->plain_cfg, st);
    else
        e = batched ? graph_launch(rs.g_emit, rs.job, st) : L.plain_emit(rs.job, c->plain_cfg, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "emit");
    if (timing) cudaEventRecord(rs.ev[4], st);
    launches += scattered ? kLaunchesScatter : batched ? kLaunchesEmit : kLaunchesPlainEmit;
    if ((e = cudaMemcpyAsync(rs.h_ctrl, rs.d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(c, e, "ctrl readback");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "emit phase");
    if (rs.h_ctrl->status & kStBounds) return fail(c, JPSI_ECUDA, kBoundsMsg);
    if (rs.h_ctrl->status & kStEmitMismatch) return fail(c, JPSI_ECUDA, "internal: emit pass count mismatch");
    add_timing(c, rs, launches, true);
    return JPSI_OK;
}

// Launch grids of the batched form from the context's tuning.
void apply_tuning(jpsi_ctx* c) {
    const int wpb = c->tune.light_wpb;
    const int lb = std::max(1, light_max_blocks_per_sm(wpb));
    const int gb = std::max(1, generic_max_blocks_per_sm(256));
    const int hmax = std::max(1, heavy_max_blocks_per_sm());
    const int hb = c->tune.heavy_ctas_per_sm > 0 ? std::min(c->tune.heavy_ctas_per_sm, hmax) : hmax;
    const int mb = std::max(1, medium_max_blocks_per_sm());
    c->batch_cfg.light_wpb = wpb;
    c->batch_cfg.light_blocks = c->n_sm * lb;
    c->batch_cfg.generic_threads = 256;
    c->batch_cfg.generic_blocks = c->n_sm * gb;
    c->batch_cfg.heavy_blocks = c->n_sm * hb;
    c->batch_cfg.medium_blocks = c->n_sm * mb;
    c->batch_cfg.scan_blocks = c->n_sm * 2;
    c->plain_cfg = c->batch_cfg;
    c->plain_cfg.light_wpb = 4;
    c->plain_cfg.light_blocks = 0;
    ++c->cfg_id;
}

// Copies a batch into device buffers `x, y, z, off`: from host memory, or
// (serving) from device memory of the context's device; the direction of each
// copy follows from the pointer (unified addressing).
jpsi_status upload(jpsi_ctx* c, const jpsi_batch* hb, DevBuf& x, DevBuf& y, DevBuf& z, DevBuf& off, DevBuf& ztab,
                   jpsi_batch* db, cudaStream_t st) {
    const int64_t S = c->p.n_stations;
    const size_t hb_bytes = (size_t)hb->n_hits * 4;
    const size_t ob = (size_t)(hb->n_events * 3 * S + 1) * 4;
    jpsi_status s;
    if ((s = ensure(c, x, std::max<size_t>(hb_bytes, 4), "hits x")) || (s = ensure(c, y, std::max<size_t>(hb_bytes, 4), "hits y")) ||
        (s = ensure(c, z, std::max<size_t>(hb_bytes, 4), "hits z")) || (s = ensure(c, off, ob, "offsets")))
        return s;
    cudaError_t e = cudaSuccess;
    if (hb_bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(x.p, hb->x, hb_bytes, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(y.p, hb->y, hb_bytes, cudaMemcpyDefault, st);
        if (e == cudaSuccess && hb->z) e = cudaMemcpyAsync(z.p, hb->z, hb_bytes, cudaMemcpyDefault, st);
    }
    if (e == cudaSuccess && hb->n_events > 0) e = cudaMemcpyAsync(off.p, hb->offsets, ob, cudaMemcpyDefault, st);
    if (e == cudaSuccess && !hb->z && hb_bytes) {
        // per-hit z filled on the device from the geometry table
        if ((s = ensure(c, ztab, (size_t)S * 3 * 4, "z table")) != JPSI_OK) return s;
        e = cudaMemcpyAsync(ztab.p, hb->z_layer, (size_t)S * 3 * 4, cudaMemcpyDefault, st);
        if (e == cudaSuccess)
            e = launch_expand_z((const int32_t*)off.p, (const float*)ztab.p, (float*)z.p, 0, hb->n_events, (int)S,
                                hb->n_hits, c->n_sm, st);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "input upload");
    *db = *hb;
    db->x = (const float*)x.p;
    db->y = (const float*)y.p;
    db->z = (const float*)z.p;
    db->offsets = (const int32_t*)off.p;
    return JPSI_OK;
}

// Device addresses of a host batch whose arrays are all pinned (page-locked
// and mapped into the device's address space); false when one is not.
bool map_host_batch(const jpsi_batch* hb, jpsi_batch* db) {
    *db = *hb;
    if (hb->n_hits > 0 && !hb->z) return false;  // z from a table: uploaded and filled instead
    const void* hp[4] = {hb->x, hb->y, hb->z, hb->offsets};
    const void* dp[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; ++k) {
        if (!hp[k]) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, hp[k]) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
        dp[k] = a.devicePointer;
    }
    db->x = (const float*)dp[0];
    db->y = (const float*)dp[1];
    db->z = (const float*)dp[2];
    db->offsets = (const int32_t*)dp[3];
    return true;
}

// jpsi_run on host buffers with the given device buffers.  With `mapped`
// (the batch's pinned arrays at their device addresses) the kernels read the
// hits over the host link instead of from an uploaded copy.
jpsi_status run_host_with(jpsi_ctx* c, RunState& rs, const jpsi_batch* hb, jpsi_outputs* ho, DevBuf& x, DevBuf& y,
                          DevBuf& z, DevBuf& off, DevBuf& acc, DevBuf& tc, DevBuf& toff, DevBuf& trip,
                          int64_t trip_cap_dev, cudaStream_t st, const jpsi_batch* mapped = nullptr) {
    jpsi_batch db;
    jpsi_status s = JPSI_OK;
    if (mapped)
        db = *mapped;
    else if ((s = upload(c, hb, x, y, z, off, rs.ztab, &db, st)) != JPSI_OK)
        return s;
    const int64_t ne = hb->n_events, nu = ne * c->p.n_stations;
    jpsi_outputs dout{};
    if (ho->accept_bits) {
        if ((s = ensure(c, acc, (size_t)std::max<int64_t>((ne + 31) / 32, 1) * 4, "accept bits"))) return s;
        dout.accept_bits = (uint32_t*)acc.p;
    }
    if (ho->track_counts) {
        if ((s = ensure(c, tc, (size_t)std::max<int64_t>(ne, 1) * 4, "track counts"))) return s;
        dout.track_counts = (int32_t*)tc.p;
    }
    if (ho->trip_off || ho->triplets) {
        if ((s = ensure(c, toff, (size_t)(nu + 1) * 8, "triplet offsets"))) return s;
        dout.trip_off = (int64_t*)toff.p;
    }
    if (ho->triplets) {
        const int64_t cap = trip_cap_dev >= 0 ? std::min(trip_cap_dev, ho->trip_capacity) : ho->trip_capacity;
        if ((s = ensure(c, trip, (size_t)std::max<int64_t>(cap, 1) * 12, "triplets"))) return s;
        dout.triplets = (int32_t*)trip.p;
        dout.trip_capacity = cap;
    }
    s = run_device(c, rs, &db, &dout, st, true, mapped != nullptr);
    ho->trip_needed = dout.trip_needed;
    if (s != JPSI_OK && s != JPSI_ECAPACITY) return s;
    cudaError_t e = cudaSuccess;
    // outputs to host memory, or (serving) to device memory
    if (ho->accept_bits && ne > 0)
        e = cudaMemcpyAsync(ho->accept_bits, acc.p, (size_t)((ne + 31) / 32) * 4, cudaMemcpyDefault, st);
    if (e == cudaSuccess && ho->track_counts && ne > 0)
        e = cudaMemcpyAsync(ho->track_counts, tc.p, (size_t)ne * 4, cudaMemcpyDefault, st);
    if (e == cudaSuccess && ho->trip_off)
        e = cudaMemcpyAsync(ho->trip_off, toff.p, (size_t)(nu + 1) * 8, cudaMemcpyDefault, st);
    if (e == cudaSuccess && ho->triplets && s == JPSI_OK && dout.trip_needed > 0)
        e = cudaMemcpyAsync(ho->triplets, trip.p, (size_t)dout.trip_needed * 12, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "output download");
    return s;
}

// Between the chunks of a pipelined counting pass: the work counters start
// again, and the next chunk's list entries start where this chunk's end (its
// events are appended behind them, so the lists end up covering the batch).
cudaError_t next_pass_lists(RunState& rs, cudaStream_t st) {
    static_assert(offsetof(Ctrl, m_begin) == offsetof(Ctrl, n_medium) + 3 * sizeof(int32_t), "list fields");
    cudaError_t e = cudaMemsetAsync(rs.d_ctrl->work, 0, sizeof(rs.d_ctrl->work), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&rs.d_ctrl->m_begin, &rs.d_ctrl->n_medium, 3 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    return e;
}

// jpsi_run_host for large batches: the hits go to the device chunk by chunk
// on the copy stream while the warp kernels count the chunks that have
// arrived (events [ev_begin, ev_begin + ev_count) of the batch); accept bits,
// scan and triplet rows then run once over the whole batch.  Returns
// JPSI_EBUSY (nothing done) when the batch is better run in one piece.
jpsi_status run_host_pipelined(jpsi_ctx* c, RunState& rs, const jpsi_batch* hb, jpsi_outputs* ho, cudaStream_t st) {
    const int64_t S = c->p.n_stations, ne = hb->n_events, nu = ne * S, S3 = 3 * S;
    const int nch = (int)std::min<int64_t>(kMaxChunks, ne / kChunkMinEvents);
    if (nch < 2 || !c->copy_stream) return JPSI_EBUSY;
    int64_t cs = (ne + nch - 1) / nch;
    cs = (cs + 31) / 32 * 32;  // whole accept-bit words per chunk
    const int32_t* hoff = hb->offsets;
    for (int64_t e = 0; e <= ne; e += cs) {  // chunk boundaries must be usable as copy ranges
        const int64_t b = hoff[std::min(e, ne) * S3];
        if (b < 0 || b > hb->n_hits) return JPSI_EBUSY;
    }
    if (hoff[ne * S3] != hb->n_hits) return JPSI_EBUSY;
    jpsi_status s;
    if (!rs.chunk_ev[0]) {
        for (cudaEvent_t& e : rs.chunk_ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(c, JPSI_ECUDA, "events");
    }
    const size_t hbytes = (size_t)hb->n_hits * 4, obytes = (size_t)(ne * S3 + 1) * 4;
    if ((s = ensure(c, c->hx, std::max<size_t>(hbytes, 4), "hits x")) || (s = ensure(c, c->hy, std::max<size_t>(hbytes, 4), "hits y")) ||
        (s = ensure(c, c->hz, std::max<size_t>(hbytes, 4), "hits z")) || (s = ensure(c, c->hoff, obytes, "offsets")))
        return s;
    jpsi_batch db = *hb;
    db.x = (const float*)c->hx.p;
    db.y = (const float*)c->hy.p;
    db.z = (const float*)c->hz.p;
    db.offsets = (const int32_t*)c->hoff.p;
    jpsi_outputs dout{};
    if (ho->accept_bits) {
        if ((s = ensure(c, c->hacc, (size_t)((ne + 31) / 32) * 4, "accept bits"))) return s;
        dout.accept_bits = (uint32_t*)c->hacc.p;
    }
    if (ho->track_counts) {
        if ((s = ensure(c, c->htc, (size_t)ne * 4, "track counts"))) return s;
        dout.track_counts = (int32_t*)c->htc.p;
    }
    if (ho->trip_off || ho->triplets) {
        if ((s = ensure(c, c->htoff, (size_t)(nu + 1) * 8, "triplet offsets"))) return s;
        dout.trip_off = (int64_t*)c->htoff.p;
    }
    if (ho->triplets) {
        if ((s = ensure(c, c->htrip, (size_t)std::max<int64_t>(ho->trip_capacity, 1) * 12, "triplets"))) return s;
        dout.triplets = (int32_t*)c->htrip.p;
        dout.trip_capacity = ho->trip_capacity;
    }
    if ((s = prepare(c, rs, &db, &dout, false)) != JPSI_OK) return s;
    const Job& all = rs.job;  // the whole batch (accept bits, scan, rows)
    const bool ztable = !hb->z;  // z filled per chunk from the geometry table
    if (ztable && (s = ensure(c, rs.ztab, (size_t)S * 3 * 4, "z table")) != JPSI_OK) return s;
    cudaError_t e = cudaMemcpyAsync(c->hoff.p, hoff, obytes, cudaMemcpyHostToDevice, c->copy_stream);
    if (e == cudaSuccess && ztable)
        e = cudaMemcpyAsync(rs.ztab.p, hb->z_layer, (size_t)S * 3 * 4, cudaMemcpyHostToDevice, c->copy_stream);
    int k = 0;
    for (int64_t e0 = 0; e0 < ne && e == cudaSuccess; e0 += cs, ++k) {
        const int64_t e1 = std::min(ne, e0 + cs);
        const int64_t h0 = hoff[e0 * S3], h1 = hoff[e1 * S3];
        const size_t nb = (size_t)(h1 - h0) * 4;
        if (nb) {
            e = cudaMemcpyAsync((float*)c->hx.p + h0, hb->x + h0, nb, cudaMemcpyHostToDevice, c->copy_stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync((float*)c->hy.p + h0, hb->y + h0, nb, cudaMemcpyHostToDevice, c->copy_stream);
            if (e == cudaSuccess && !ztable)
                e = cudaMemcpyAsync((float*)c->hz.p + h0, hb->z + h0, nb, cudaMemcpyHostToDevice, c->copy_stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(rs.chunk_ev[k], c->copy_stream);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "chunk upload");
    if ((e = cudaMemsetAsync(rs.d_ctrl, 0, sizeof(Ctrl), st)) != cudaSuccess) return cuda_fail(c, e, "ctrl reset");
    if (c->p.distinct_hits && (e = cudaMemsetAsync(rs.dpair.p, 0, (size_t)ne, st)) != cudaSuccess)
        return cuda_fail(c, e, "flag reset");
    k = 0;
    for (int64_t e0 = 0; e0 < ne; e0 += cs, ++k) {
        const int64_t e1 = std::min(ne, e0 + cs);
        Job jk = all;  // the chunk's events
        jk.ev_begin = e0;
        jk.ev_count = e1 - e0;
        if ((e = cudaStreamWaitEvent(st, rs.chunk_ev[k], 0)) != cudaSuccess ||
            (ztable && (e = launch_expand_z((const int32_t*)c->hoff.p, (const float*)rs.ztab.p, (float*)c->hz.p, e0,
                                            e1, (int)S, hb->n_hits, c->n_sm, st)) != cudaSuccess) ||
            (k > 0 && (e = next_pass_lists(rs, st)) != cudaSuccess) ||
            (e = launch_light_count(jk, e1 - e0, c->batch_cfg, true, st)) != cudaSuccess ||
            (e = launch_count_lists(jk, c->batch_cfg, st)) != cudaSuccess)
            return cuda_fail(c, e, "chunk count");
    }
    if ((e = launch_count_tail(all, c->batch_cfg, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(rs.h_ctrl, rs.d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(c, e, "count phase");
    const Ctrl ctl = *rs.h_ctrl;
    if (ctl.status & kStBounds) return fail(c, JPSI_ECUDA, kBoundsMsg);
    if (ctl.status & kStInvalid) return fail(c, JPSI_EINVAL, "malformed offsets or a hit with z <= 0");
    if (ctl.status & kStNoPool) return fail(c, JPSI_ENOMEM, "distinct_hits: candidates exceed the trigger pool");
    ho->trip_needed = ctl.trip_total;
    s = JPSI_OK;
    if (ho->triplets && ctl.trip_total > ho->trip_capacity) {
        s = fail(c, JPSI_ECAPACITY, "triplet capacity " + std::to_string(ho->trip_capacity) + " < needed " +
                                        std::to_string(ctl.trip_total));
    } else if (ho->triplets && ctl.trip_total > 0) {
        const bool scattered = all.tscr && !(ctl.status & kStNoScratch) &&
                               ctl.scratch_n <= (unsigned long long)all.tscr_cap;
        if (!scattered && all.tscr && !(ctl.status & kStNoScratch))
            rs.tscr_want = std::max<int64_t>(rs.tscr_want, (int64_t)(ctl.scratch_n + ctl.scratch_n / 4));
        if (!scattered) e = cudaMemsetAsync(&rs.d_ctrl->m_begin, 0, 3 * sizeof(int32_t), st);  // every chunk's events
        if (e == cudaSuccess)
            e = scattered ? launch_scatter(all, c->batch_cfg, st) : launch_emit_phase(all, ne, c->batch_cfg, true, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rs.h_ctrl, rs.d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(c, e, "emit");
        if (rs.h_ctrl->status & kStBounds) return fail(c, JPSI_ECUDA, kBoundsMsg);
        if (rs.h_ctrl->status & kStEmitMismatch) return fail(c, JPSI_ECUDA, "internal: emit pass count mismatch");
    }
    e = cudaSuccess;
    if (ho->accept_bits) e = cudaMemcpyAsync(ho->accept_bits, c->hacc.p, (size_t)((ne + 31) / 32) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ho->track_counts)
        e = cudaMemcpyAsync(ho->track_counts, c->htc.p, (size_t)ne * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ho->trip_off)
        e = cudaMemcpyAsync(ho->trip_off, c->htoff.p, (size_t)(nu + 1) * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ho->triplets && s == JPSI_OK && ctl.trip_total > 0)
        e = cudaMemcpyAsync(ho->triplets, c->htrip.p, (size_t)ctl.trip_total * 12, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "output download");
    return s;
}

// A free-streaming timeslice: windows become the events of a window batch
// (ranges found and gathered on the device), the selection runs with the
// time tests compiled in, and the triplet rows are moved back to timeslice
// group indices.
jpsi_status run_stream(jpsi_ctx* c, const jpsi_timeslice* ts, jpsi_outputs* o, cudaStream_t st, bool batched) {
    if (!ts || !o) return fail(c, JPSI_EINVAL, "null timeslice or outputs");
    if (c->p.distinct_hits) return fail(c, JPSI_EINVAL, "distinct_hits is not defined for free-streaming windows");
    const int64_t S = c->p.n_stations, S3 = 3 * S, K = ts->n_windows;
    if (ts->n_hits < 0 || K < 0) return fail(c, JPSI_EINVAL, "negative sizes");
    if (ts->n_hits >= ((int64_t)1 << 31)) return fail(c, JPSI_EINVAL, "n_hits must be < 2^31");
    if (K > (((int64_t)1 << 31) - 2) / S3) return fail(c, JPSI_EINVAL, "too many windows for int32 offsets");
    if (!(ts->dt >= 0.0f) || std::isinf(ts->dt)) return fail(c, JPSI_EINVAL, "dt must be finite and >= 0");
    if (!ts->offsets || (K > 0 && !ts->bounds)) return fail(c, JPSI_EINVAL, "offsets or bounds missing");
    if (ts->n_hits > 0 && (!ts->x || !ts->y || !ts->t || (!ts->z && !ts->z_layer)))
        return fail(c, JPSI_EINVAL, "hit arrays missing");
    if (o->triplets && !o->trip_off) return fail(c, JPSI_EINVAL, "triplets need trip_off");
    if (o->trip_capacity < 0) return fail(c, JPSI_EINVAL, "negative triplet capacity");
    const void* ptrs[] = {ts->x, ts->y, ts->z, ts->t, ts->offsets, ts->z_layer, ts->bounds, o->accept_bits,
                          o->track_counts, o->trip_off, o->triplets};
    for (const void* p : ptrs)
        if (!device_accessible(c, p)) return fail(c, JPSI_EINVAL, "pointer is not device-accessible");
    // the 3S+1 group offsets are checked here: the range search reads them
    int32_t hoff[3 * kMaxStations + 1];
    cudaError_t e = cudaMemcpyAsync(hoff, ts->offsets, (size_t)(S3 + 1) * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "offsets readback");
    if (hoff[0] != 0 || hoff[S3] != ts->n_hits) return fail(c, JPSI_EINVAL, "malformed offsets");
    for (int g = 0; g < S3; ++g)
        if (hoff[g + 1] < hoff[g]) return fail(c, JPSI_EINVAL, "malformed offsets");
    const int64_t n = K * S3;
    jpsi_status s;
    if ((s = ensure(c, c->wlo, (size_t)std::max<int64_t>(n, 1) * 4, "window ranges")) ||
        (s = ensure(c, c->wcnt, (size_t)std::max<int64_t>(n, 1) * 4, "window ranges")) ||
        (s = ensure(c, c->woff, (size_t)(n + 1) * 8, "window ranges")) ||
        (s = ensure(c, c->wbs, (size_t)((n + 4095) / 4096 + 1) * 8, "scan")) ||
        (s = ensure(c, c->woff32, (size_t)(n + 1) * 4, "window offsets")))
        return s;
    RunState& rs = c->rs;
    WinJob w{};
    w.x = ts->x;
    w.y = ts->y;
    w.z = ts->z;
    w.t = ts->t;
    w.z_layer = ts->z_layer;
    w.off = ts->offsets;
    w.wb = ts->bounds;
    w.n_hits = ts->n_hits;
    w.K = K;
    w.S = (int32_t)S;
    w.trig = c->p.trigger_station;
    w.chain = c->p.mode == JPSI_MODE_CHAIN && S > 1;
    w.dt = ts->dt;
    w.wlo = (int32_t*)c->wlo.p;
    w.wcnt = (int32_t*)c->wcnt.p;
    w.woff = (int64_t*)c->woff.p;
    w.block_sums = (int64_t*)c->wbs.p;
    w.off_out = (int32_t*)c->woff32.p;
    w.ctrl = rs.d_ctrl;
    w.n_sm = c->n_sm;
    const bool timing = c->timing.load();
    if ((e = cudaMemsetAsync(rs.d_ctrl, 0, sizeof(Ctrl), st)) != cudaSuccess) return cuda_fail(c, e, "ctrl reset");
    if (timing) cudaEventRecord(rs.ev[5], st);
    if ((e = streamk::launch_window_ranges(w, st)) != cudaSuccess) return cuda_fail(c, e, "window ranges");
    if ((e = cudaMemcpyAsync(rs.h_ctrl, rs.d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(c, e, "ctrl readback");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "window ranges");
    if (rs.h_ctrl->status & kStInvalid)
        return fail(c, JPSI_EINVAL, "malformed timeslice: unsorted or NaN times, z <= 0, or bounds not increasing");
    const int64_t total = rs.h_ctrl->trip_total;
    if (total >= ((int64_t)1 << 31))
        return fail(c, JPSI_EINVAL, "the windows' hit ranges hold 2^31 hits or more: split the timeslice");
    const size_t hb = (size_t)std::max<int64_t>(total, 1) * 4;
    if ((s = ensure(c, c->wx, hb, "window hits")) || (s = ensure(c, c->wy, hb, "window hits")) ||
        (s = ensure(c, c->wz, hb, "window hits")) || (s = ensure(c, c->wt, hb, "window hits")))
        return s;
    w.xo = (float*)c->wx.p;
    w.yo = (float*)c->wy.p;
    w.zo = (float*)c->wz.p;
    w.to = (float*)c->wt.p;
    if ((e = streamk::launch_window_gather(w, st)) != cudaSuccess) return cuda_fail(c, e, "window gather");
    if (timing) cudaEventRecord(rs.ev[6], st);
    jpsi_batch wbat{};
    wbat.n_events = K;
    wbat.n_hits = total;
    wbat.x = w.xo;
    wbat.y = w.yo;
    wbat.z = w.zo;
    wbat.offsets = w.off_out;
    const StreamJob sj{w.to, ts->bounds, ts->dt};
    s = run_device(c, rs, &wbat, o, st, batched, false, kStreamL, &sj);
    if (s != JPSI_OK) return s;
    int launches = kLaunchesWindows;
    const bool rows = o->triplets && o->trip_needed > 0;
    if (rows) {
        if (timing) cudaEventRecord(rs.ev[7], st);
        if ((e = streamk::launch_window_rows(w, o->trip_off, o->triplets, st)) != cudaSuccess)
            return cuda_fail(c, e, "window rows");
        if (timing) cudaEventRecord(rs.ev[8], st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(c, e, "window rows");
        ++launches;
    }
    if (timing) {
        float a = 0, b = 0;
        cudaEventElapsedTime(&a, rs.ev[5], rs.ev[6]);
        if (rows) cudaEventElapsedTime(&b, rs.ev[7], rs.ev[8]);
        std::lock_guard<std::mutex> lk(c->err_mu);
        c->tm.kernel_launches += launches;
        c->tm.window_ms += a + b;
    }
    return JPSI_OK;
}

}  // namespace

// ===================================================================== ABI

extern "C" {

const char* jpsi_strerror(jpsi_status s) {
    switch (s) {
        case JPSI_OK: return "ok";
        case JPSI_EINVAL: return "invalid argument or input";
        case JPSI_ENOMEM: return "out of memory or over the device budget";
        case JPSI_ECAPACITY: return "triplet buffer too small";
        case JPSI_ECUDA: return "CUDA error";
        case JPSI_ETIMEOUT: return "timed out";
        case JPSI_EBUSY: return "context busy";
    }
    return "unknown status";
}

const char* jpsi_last_error(const jpsi_ctx* c) { return c ? c->last_error.c_str() : ""; }


jpsi_status jpsi_create(const jpsi_params* params, int device, size_t hbm_budget, jpsi_ctx** out) {
    if (!out) return JPSI_EINVAL;
    *out = nullptr;
    if (params_ok(params) != JPSI_OK) return JPSI_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ndev == 0 ? JPSI_ECUDA : JPSI_EINVAL;
    }
    if (cudaSetDevice(device) != cudaSuccess) return JPSI_ECUDA;
    jpsi_ctx* c = new (std::nothrow) jpsi_ctx;
    if (!c) return JPSI_ENOMEM;
    c->p = *params;
    c->device = device;
    c->budget = hbm_budget ? hbm_budget : kDefaultBudget;
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    int pma = 0;
    cudaDeviceGetAttribute(&pma, cudaDevAttrPageableMemoryAccess, device);
    c->pageable_ok = pma != 0;
    c->cx = (float)params->ndf * params->t_xz;
    c->cy = (float)params->ndf * params->t_yz;
    c->K = pruning_K(c->cx, c->cy);
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
        jpsi_destroy(c);
        return JPSI_ECUDA;
    }
    if (state_init(c, c->rs) != JPSI_OK) {
        jpsi_destroy(c);
        return JPSI_ENOMEM;
    }
    apply_tuning(c);
    *out = c;
    return JPSI_OK;
}

jpsi_status jpsi_serve_stop(jpsi_ctx* c);

void jpsi_destroy(jpsi_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    jpsi_serve_stop(c);
    cudaDeviceSynchronize();
    state_free(c, c->rs);
    DevBuf* bufs[] = {&c->hx,  &c->hy,   &c->hz,  &c->hoff, &c->hacc, &c->htc, &c->htoff, &c->htrip, &c->wlo,
                      &c->wcnt, &c->woff, &c->wbs, &c->woff32, &c->wx, &c->wy, &c->wz,   &c->wt};
    for (DevBuf* b : bufs) release(c, *b);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    delete c;
}

jpsi_status jpsi_run_plain(jpsi_ctx* c, const jpsi_batch* b, jpsi_outputs* o, void* stream) {
    if (!c) return JPSI_EINVAL;
    Range r("jpsi_run_plain");
    BusyGuard g(c);
    if (!g.ok) return fail(c, JPSI_EBUSY, "context in use");
    cudaSetDevice(c->device);
    c->last_error.clear();
    jpsi_status s = check_batch(c, b, o, true);
    if (s != JPSI_OK) return s;
    return run_device(c, c->rs, b, o, (cudaStream_t)stream, false);
}

jpsi_status jpsi_run(jpsi_ctx* c, const jpsi_batch* b, jpsi_outputs* o, void* stream) {
    if (!c) return JPSI_EINVAL;
    Range r("jpsi_run");
    BusyGuard g(c);
    if (!g.ok) return fail(c, JPSI_EBUSY, "context in use");
    cudaSetDevice(c->device);
    c->last_error.clear();
    jpsi_status s = check_batch(c, b, o, true);
    if (s != JPSI_OK) return s;
    return run_device(c, c->rs, b, o, (cudaStream_t)stream, true);
}

jpsi_status jpsi_run_stream(jpsi_ctx* c, const jpsi_timeslice* ts, jpsi_outputs* o, void* stream) {
    if (!c) return JPSI_EINVAL;
    Range r("jpsi_run_stream");
    BusyGuard g(c);
    if (!g.ok) return fail(c, JPSI_EBUSY, "context in use");
    cudaSetDevice(c->device);
    c->last_error.clear();
    return run_stream(c, ts, o, (cudaStream_t)stream, true);
}

jpsi_status jpsi_run_stream_plain(jpsi_ctx* c, const jpsi_timeslice* ts, jpsi_outputs* o, void* stream) {
    if (!c) return JPSI_EINVAL;
    Range r("jpsi_run_stream_plain");
    BusyGuard g(c);
    if (!g.ok) return fail(c, JPSI_EBUSY, "context in use");
    cudaSetDevice(c->device);
    c->last_error.clear();
    return run_stream(c, ts, o, (cudaStream_t)stream, false);
}

jpsi_status jpsi_run_host(jpsi_ctx* c, const jpsi_batch* b, jpsi_outputs* o, void* stream) {
    if (!c) return JPSI_EINVAL;
    Range r("jpsi_run_host");
    BusyGuard g(c);
    if (!g.ok) return fail(c, JPSI_EBUSY, "context in use");
    cudaSetDevice(c->device);
    c->last_error.clear();
    jpsi_status s = check_batch(c, b, o, false);
    if (s != JPSI_OK) return s;
    if (c->p.mode == JPSI_MODE_PAPER && c->p.n_stations > 1) {
        // PAPER mode reads only the trigger station: from pinned buffers the
        // kernels fetch just that station over the host link instead of
        // copying every station first (the paper's host-side trigger
        // filtering, Sec. 5.3, without a host-side gather)
        jpsi_batch mb;
        if (map_host_batch(b, &mb))
            return run_host_with(c, c->rs, b, o, c->hx, c->hy, c->hz, c->hoff, c->hacc, c->htc, c->htoff, c->htrip,
                                 -1, (cudaStream_t)stream, &mb);
    }
    s = run_host_pipelined(c, c->rs, b, o, (cudaStream_t)stream);
    if (s != JPSI_EBUSY) return s;
    return run_host_with(c, c->rs, b, o, c->hx, c->hy, c->hz, c->hoff, c->hacc, c->htc, c->htoff, c->htrip, -1,
                         (cudaStream_t)stream);
}

jpsi_status jpsi_inject_fault(jpsi_ctx* c, int kind, int count) {
    if (!c || count < 0) return JPSI_EINVAL;
    if (kind == JPSI_FAULT_ALLOC)
        c->fault_alloc.store(count);
    else if (kind == JPSI_FAULT_RUN)
        c->fault_run.store(count);
    else
        return JPSI_EINVAL;
    return JPSI_OK;
}

jpsi_status jpsi_timing_enable(jpsi_ctx* c, int enable) {
    if (!c) return JPSI_EINVAL;
    std::lock_guard<std::mutex> lk(c->err_mu);
    c->tm = jpsi_timing{};
    c->timing.store(enable != 0);
    return JPSI_OK;
}

jpsi_status jpsi_timing_get(jpsi_ctx* c, jpsi_timing* out) {
    if (!c || !out) return JPSI_EINVAL;
    std::lock_guard<std::mutex> lk(c->err_mu);
    *out = c->tm;
    out->light_wpb = c->batch_cfg.light_wpb;
    out->light_grab = c->tune.light_grab;
    return JPSI_OK;
}

jpsi_status jpsi_get_tuning(const jpsi_ctx* c, jpsi_tuning* out) {
    if (!c || !out) return JPSI_EINVAL;
    *out = c->tune;
    return JPSI_OK;
}

jpsi_status jpsi_set_tuning(jpsi_ctx* c, const jpsi_tuning* t) {
    if (!c || !t) return JPSI_EINVAL;
    BusyGuard g(c);
    if (!g.ok) return fail(c, JPSI_EBUSY, "context in use");
    if (c->serving) return fail(c, JPSI_EBUSY, "tuning is fixed while serving");
    cudaSetDevice(c->device);
    const bool ok = (t->light_wpb == 2 || t->light_wpb == 4 || t->light_wpb == 8) && t->light_grab >= 1 &&
                    t->light_grab <= 64 && t->small_layer_cap >= 1 && t->small_layer_cap <= 192 &&
                    t->medium_layer_cap >= 1 && t->medium_layer_cap <= 384 && t->heavy_ctas_per_sm >= 0 &&
                    t->heavy_ctas_per_sm <= heavy_max_blocks_per_sm() && t->reserved == 0 && t->record_cap >= -1;
    if (!ok) return fail(c, JPSI_EINVAL, "tuning value out of range");
    c->tune = *t;
    apply_tuning(c);
    return JPSI_OK;
}

jpsi_status jpsi_autotune(jpsi_ctx* c, const jpsi_batch* sample) {
    if (!c) return JPSI_EINVAL;
    Range r("jpsi_autotune");
    BusyGuard g(c);
    if (!g.ok) return fail(c, JPSI_EBUSY, "context in use");
    if (c->serving) return fail(c, JPSI_EBUSY, "tuning is fixed while serving");
    cudaSetDevice(c->device);
    c->last_error.clear();
    jpsi_outputs o{};
    jpsi_status s = check_batch(c, sample, &o, true);
    if (s != JPSI_OK) return s;
    DevBuf acc;
    if ((s = ensure(c, acc, (size_t)std::max<int64_t>((sample->n_events + 31) / 32, 1) * 4, "autotune"))) return s;
    o.accept_bits = (uint32_t*)acc.p;
    cudaStream_t st = c->cap_stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        release(c, acc);
        return fail(c, JPSI_ECUDA, "event creation failed");
    }
    const jpsi_tuning start = c->tune;
    jpsi_tuning best = start;
    float best_ms = INFINITY;
    jpsi_status first_err = JPSI_OK;
    // device time of three runs of the sample after one warm-up run (graph
    // capture, scratch growth); false if a run failed
    auto trial = [&](const jpsi_tuning& t) {
        c->tune = t;
        apply_tuning(c);
        float tot = 0;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, st);
            const jpsi_status r = run_device(c, c->rs, sample, &o, st, true);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            if (r != JPSI_OK) {
                if (first_err == JPSI_OK) first_err = r;
                return;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;
        }
        if (tot < best_ms) {
            best_ms = tot;
            best = t;
        }
    };
    // one dimension at a time, each from the best shape so far
    for (int w : {2, 4, 8}) {
        if (light_max_blocks_per_sm(w) < 1) continue;
        for (int gr : {1, 2, 4, 8}) {
            jpsi_tuning t = best;
            t.light_wpb = w;
            t.light_grab = gr;
            trial(t);
        }
    }
    if (best_ms < INFINITY) {
        const jpsi_tuning b1 = best;
        for (int cap : {96, 128, 160, 192}) {
            jpsi_tuning t = b1;
            t.small_layer_cap = cap;
            if (cap != b1.small_layer_cap) trial(t);
        }
        const jpsi_tuning b2 = best;
        for (int cap : {256, 320, 384}) {
            jpsi_tuning t = b2;
            t.medium_layer_cap = cap;
            if (cap != b2.medium_layer_cap) trial(t);
        }
        const jpsi_tuning b3 = best;
        const int hmax = heavy_max_blocks_per_sm();
        for (int h = 1; h <= hmax; ++h) {
            jpsi_tuning t = b3;
            t.heavy_ctas_per_sm = h;
            if (h != (b3.heavy_ctas_per_sm > 0 ? b3.heavy_ctas_per_sm : hmax)) trial(t);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release(c, acc);
    const bool any = best_ms < INFINITY;
    c->tune = any ? best : start;
    apply_tuning(c);
    if (!any) return fail(c, first_err != JPSI_OK ? first_err : JPSI_ECUDA, "autotune: no candidate ran");
    return JPSI_OK;
}

// ------------------------------------------------------------- serving

// True when every non-null pointer is device memory of `device`.
static bool all_on_device(std::initializer_list<const void*> ps, int device) {
    for (const void* p : ps) {
        if (!p) continue;
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (a.type != cudaMemoryTypeDevice || a.device != device) return false;
    }
    return true;
}

static void slot_worker(jpsi_ctx* c, int si) {
    cudaSetDevice(c->device);
    Slot* sl = c->slots[si];
    std::unique_lock<std::mutex> lk(c->mu);
    for (;;) {
        c->slot_cv[si]->wait(lk, [&] { return c->stopping || sl->busy; });
        if (!sl->busy && c->stopping) return;
        jpsi_batch b = sl->batch;
        jpsi_outputs* o = sl->out;
        lk.unlock();
        Range r("jpsi_serve slot run");
        // a batch and outputs that are all in this device's memory are used
        // in place, as jpsi_run uses them; otherwise the slot's own buffers
        // take copies
        const bool in_place = all_on_device(
            {b.x, b.y, b.z, b.offsets, o->accept_bits, o->track_counts, o->trip_off, o->triplets}, c->device);
        auto run_once = [&]() -> jpsi_status {
            if (take_fault(c->fault_run)) return fail(c, JPSI_ECUDA, "injected run failure");
            if (in_place) return run_device(c, sl->rs, &b, o, sl->stream, true);
            return run_host_with(c, sl->rs, &b, o, sl->x, sl->y, sl->z, sl->off, sl->accept, sl->tracks,
                                 sl->trip_off, sl->triplets, sl->cap_trip, sl->stream);
        };
        jpsi_status s = run_once();
        // one more attempt after a failure that is not the request's own
        // fault (an invalid batch or too small an output buffer fails again)
        if (s != JPSI_OK && s != JPSI_EINVAL && s != JPSI_ECAPACITY) s = run_once();
        const double lat =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - sl->t_submit).count();
        lk.lock();
        c->done[sl->ticket] = Done{s, lat};
        sl->busy = false;
        c->free_slots.push_back(si);
        c->cv.notify_all();
    }
}

jpsi_status jpsi_serve_start(jpsi_ctx* c, int n_slots, int64_t slot_events, int64_t slot_hits,
                             int64_t slot_triplets) {
    if (!c || n_slots < 1 || n_slots > 64 || slot_events < 0 || slot_hits < 0 || slot_triplets < 0)
        return JPSI_EINVAL;
    BusyGuard g(c);
    if (!g.ok) return fail(c, JPSI_EBUSY, "context in use");
    cudaSetDevice(c->device);
    if (c->serving) return fail(c, JPSI_EINVAL, "serving already started");
    if (slot_hits >= ((int64_t)1 << 31)) return fail(c, JPSI_EINVAL, "slot_hits must be < 2^31");
    const int64_t S = c->p.n_stations;
    jpsi_status s = JPSI_OK;
    for (int i = 0; i < n_slots && s == JPSI_OK; ++i) {
        Slot* sl = new Slot;
        c->slots.push_back(sl);
        c->slot_cv.push_back(new std::condition_variable);
        sl->cap_events = slot_events;
        sl->cap_hits = slot_hits;
        sl->cap_trip = slot_triplets;
        if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess) {
            s = fail(c, JPSI_ECUDA, "stream creation");
            break;
        }
        if ((s = state_init(c, sl->rs)) != JPSI_OK) break;
        const int64_t ne = std::max<int64_t>(slot_events, 1), nu = ne * S;
        const size_t hb = (size_t)std::max<int64_t>(slot_hits, 1) * 4;
        // reserve everything up front: admission is by free slots within the budget
        if ((s = ensure(c, sl->x, hb, "slot hits")) || (s = ensure(c, sl->y, hb, "slot hits")) ||
            (s = ensure(c, sl->z, hb, "slot hits")) || (s = ensure(c, sl->off, (size_t)(ne * 3 * S + 1) * 4, "slot offsets")) ||
            (s = ensure(c, sl->accept, (size_t)((ne + 31) / 32) * 4, "slot accept")) ||
            (s = ensure(c, sl->tracks, (size_t)ne * 4, "slot tracks")) ||
            (s = ensure(c, sl->trip_off, (size_t)(nu + 1) * 8, "slot trip_off")) ||
            (s = ensure(c, sl->triplets, (size_t)std::max<int64_t>(slot_triplets, 1) * 12, "slot triplets")) ||
            (s = ensure(c, sl->rs.unit_counts, (size_t)nu * 4, "slot unit counts")) ||
            (s = ensure(c, sl->rs.ev_class, (size_t)ne, "slot classes")) ||
            (s = ensure(c, sl->rs.track_counts, (size_t)ne * 4, "slot track scratch")) ||
            (s = ensure(c, sl->rs.trip_off, (size_t)(nu + 1) * 8, "slot offsets scratch")) ||
            (s = ensure(c, sl->rs.mlist, (size_t)ne * 4, "slot list")) ||
            (s = ensure(c, sl->rs.hlist, (size_t)ne * 4, "slot list")) ||
            (s = ensure(c, sl->rs.glist, (size_t)ne * 4, "slot list")) ||
            (s = ensure(c, sl->rs.tlist, (size_t)c->batch_cfg.heavy_blocks * kHeavyTCap * sizeof(float2), "slot trigger lists")) ||
            (s = ensure(c, sl->rs.talive, (size_t)c->batch_cfg.heavy_blocks * kHeavyTCap, "slot trigger lists")) ||
            (s = ensure(c, sl->rs.tpool, (size_t)tpool_entries(ne) * sizeof(float2), "slot trigger pool")) ||
            (s = ensure(c, sl->rs.tpool_alive, (size_t)tpool_entries(ne), "slot trigger pool")) ||
            (s = ensure(c, sl->rs.hT, (size_t)ne * sizeof(int2), "slot list")) ||
            (s = ensure(c, sl->rs.block_sums, (size_t)((nu + 4095) / 4096 + 1) * 8, "slot scan")))
            break;
        // graphs are captured with the context's launch shape
        if ((s = capture_graphs(c, sl->rs)) != JPSI_OK) break;
        c->free_slots.push_back(i);
    }
    if (s != JPSI_OK) {
        c->serving = true;  // let stop() tear down what exists
        jpsi_serve_stop(c);
        return s;
    }
    c->stopping = false;
    c->serving = true;
    for (int i = 0; i < n_slots; ++i) c->workers.emplace_back(slot_worker, c, i);
    return JPSI_OK;
}

jpsi_status jpsi_serve_submit(jpsi_ctx* c, const jpsi_batch* hb, jpsi_outputs* ho, uint64_t* ticket) {
    if (!c || !hb || !ho || !ticket) return JPSI_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    std::unique_lock<std::mutex> lk(c->mu);
    if (!c->serving || c->stopping) return JPSI_EINVAL;
    if (hb->n_events < 0 || hb->n_hits < 0 || (hb->n_events > 0 && !hb->offsets) ||
        (hb->n_hits > 0 && (!hb->x || !hb->y || !hb->z)) || (ho->triplets && !ho->trip_off))
        return JPSI_EINVAL;
    const Slot* s0 = c->slots[0];
    if (hb->n_events > s0->cap_events || hb->n_hits > s0->cap_hits) return JPSI_EINVAL;
    // back-pressure: block until a slot frees up
    c->cv.wait(lk, [&] { return !c->free_slots.empty() || c->stopping; });
    if (c->stopping) return JPSI_EINVAL;
    const int si = c->free_slots.front();
    c->free_slots.pop_front();
    Slot* sl = c->slots[si];
    sl->batch = *hb;
    sl->out = ho;
    sl->ticket = c->next_ticket++;
    sl->t_submit = t0;
    sl->busy = true;
    *ticket = sl->ticket;
    c->slot_cv[si]->notify_one();
    return JPSI_OK;
}

jpsi_status jpsi_serve_wait(jpsi_ctx* c, uint64_t ticket, int timeout_ms, jpsi_status* result, double* latency_s) {
    if (!c) return JPSI_EINVAL;
    std::unique_lock<std::mutex> lk(c->mu);
    auto ready = [&] { return c->done.count(ticket) != 0; };
    if (timeout_ms < 0)
        c->cv.wait(lk, ready);
    else if (!c->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return JPSI_ETIMEOUT;
    const Done d = c->done[ticket];
    c->done.erase(ticket);
    if (result) *result = d.st;
    if (latency_s) *latency_s = d.latency;
    return JPSI_OK;
}

jpsi_status jpsi_serve_stop(jpsi_ctx* c) {
    if (!c) return JPSI_EINVAL;
    {
        std::unique_lock<std::mutex> lk(c->mu);
        if (!c->serving) return JPSI_OK;
        // finish what was admitted
        c->cv.wait(lk, [&] {
            for (Slot* s : c->slots)
                if (s->busy) return false;
            return true;
        });
        c->stopping = true;
        for (auto* cv : c->slot_cv) cv->notify_all();
        c->cv.notify_all();
    }
    for (auto& t : c->workers) t.join();
    c->workers.clear();
    for (Slot* sl : c->slots) {
        if (sl->stream) cudaStreamSynchronize(sl->stream);
        state_free(c, sl->rs);
        DevBuf* bufs[] = {&sl->x, &sl->y, &sl->z, &sl->off, &sl->accept, &sl->tracks, &sl->trip_off, &sl->triplets};
        for (DevBuf* b : bufs) release(c, *b);
        if (sl->stream) cudaStreamDestroy(sl->stream);
        delete sl;
    }
    c->slots.clear();
    for (auto* cv : c->slot_cv) delete cv;
    c->slot_cv.clear();
    c->free_slots.clear();
    c->done.clear();
    c->serving = false;
    c->stopping = false;
    return JPSI_OK;
}

}  // extern "C"
