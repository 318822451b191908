// Kernels of the J/psi first-level selection (arXiv:1810.11966, Sec. 3.2) on
// sm_103a.  Work unit: one event (on the block tile in CHAIN mode, one of its
// stations).  Four paths, chosen per event, give bit-identical results:
//
//   k_light    one warp per event.  Each station's hits are staged from HBM
//              (coalesced loads into registers) into a per-warp shared tile
//              sorted into cells (row = bin of s_y, column = bin of s_x; the
//              small tile has one row of 128 columns).  Pairs (L0, L1) whose
//              slopes are close enough to belong to a passing triplet are
//              found by 32 lanes walking the candidate windows of 32 L0 hits,
//              compacted into a pair queue with ballot/popc, and drained
//              against the L2 hits in the meet of both windows (their items
//              spread evenly over the lanes);
//              every surviving triple gets the exact FP32 fit (P1).  CHAIN
//              mode keeps the passing trigger triplets' slopes in the tile
//              and searches the other stations' tiles for compatible
//              triplets (P2).  Limits: 192 hits per layer, 384 per station,
//              32 passing trigger triplets.
//   k_medium   the block-tile code on 2-warp blocks (384 hits per layer, 960
//              per station, 16 x 32 cells) for the events k_light passes on.
//   k_heavy, k_heavy_units, k_heavy_final
//              8-warp blocks on the block tile (2048 hits per layer, 5632 per
//              station, 32 x 64 cells), the warps taking L0 rounds and
//              trigger-slope searches from a shared counter.  k_sort_heavy
//              orders these events largest first; k_heavy runs each one's
//              trigger station and, in CHAIN mode, hands the other stations
//              to k_heavy_units (one block per station, trigger slopes in a
//              batch-wide pool) and k_heavy_final (alive slopes left per
//              event).
//   k_generic  one block per event, unpruned where the pruning bound is not
//              finite (extreme coordinates) and no size limit: reads hits
//              straight from global memory.
//   k_accept   accept bits from track counts (ballot per 32 events).
//   k_scan*    exclusive scan of per-unit counts into int64 trip_off.
//   k_scatter  moves the triplets recorded by the counting pass to their rows
//              trip_off[unit] + rank; when the record overflowed, the emit
//              variants of the enumeration kernels re-enumerate instead.
//
// Every kernel takes the run's Job by value (a __grid_constant__ parameter).
// Pruning only skips triples that provably fail P1 (see jpsi_device.cuh), and
// P1/P2 are the same correctly rounded FP32 expressions everywhere.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "jpsi.h"
#include "jpsi_device.cuh"
#include "jpsi_internal.h"

// The file is compiled twice: JPSI_STREAM = 0 gives the event kernels
// (namespace jpsi::basek), JPSI_STREAM = 1 the same kernels with the time
// tests of free-streaming windows (jpsi::streamk); `if constexpr (kStream)`
// keeps those tests, and their registers, out of the event build.
#ifndef JPSI_STREAM
#define JPSI_STREAM 0
#endif
namespace jpsi {
#if JPSI_STREAM
namespace streamk {
#else
namespace basek {
#endif

constexpr bool kStream = JPSI_STREAM != 0;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kQCap = 128;                // pair queue entries per warp
constexpr int kWalkCells = 512;           // tiles of at most this many cells per layer walk pair windows per lane

// warp path: tile shape per variant.  A layer's hits are sorted into
// NY x NX cells: row = bin of s_y, column = bin of s_x (row-major), so the
// cells of a slope window are one run of positions per row.  The small tile
// uses one row (NY = 1): at about 100 hits per layer a second row, or a 16 x
// 16 grid, saves fewer candidate tests than its extra staging, window work
// and registers cost.
constexpr int kTCap = 64;                 // passing trigger triplets per event (CHAIN)
template <int RMAX_, int HCAP_, int NX_, int NY_, uint8_t CLS_, int WPB_, int TCAP_ = kTCap>
struct WCfg {
    static constexpr int RMAX = RMAX_;              // hits per lane per layer
    static constexpr int LAYER_CAP = 32 * RMAX_;    // hits per layer
    static constexpr int HCAP = HCAP_;              // hits per station tile
    static constexpr int NX = NX_, NY = NY_;        // slope bins per layer in s_x, s_y
    static constexpr int NC = NX_ * NY_;            // cells per layer
    static constexpr uint8_t CLS = CLS_;            // event class of this path
    static constexpr int WPB = WPB_;                // warps per block (medium: fixed)
    static constexpr int TCAP = TCAP_;              // passing trigger triplets kept (CHAIN)
};
// the small tile: 192 hits per layer, 384 per station, one row of 128 cells
// (a pair window of the 10^6-event workload holds 4.0 candidates instead of
// 5.0 with 64 cells: 5 % less time), 32 passing trigger triplets kept
using SmallCfg = WCfg<6, 384, 128, 1, kClsLight, 0, 32>;
// the size limits of the medium tile (a 2-warp block tile, MedBCfg below)
using MediumCfg = WCfg<12, 960, 32, 16, kClsMedium, 4>;  // 384 hits/layer, 960/station

// block-tile paths: a block of THREADS threads stages a station (each thread
// up to RMAX hits per layer) into NY x NX cells per layer, and its warps
// share the station's enumeration rounds and trigger-slope searches
template <int THREADS_, int RMAX_, int HCAP_, int NX_, int NY_, uint8_t CLS_>
struct BCfg {
    static constexpr int THREADS = THREADS_, WARPS = THREADS_ / 32;
    static constexpr int RMAX = RMAX_;                   // hits per thread per layer
    static constexpr int LAYER_CAP = THREADS_ * RMAX_;   // hits per layer
    static constexpr int HCAP = HCAP_;                   // hits per station tile
    static constexpr int NX = NX_, NY = NY_, NC = NX_ * NY_;
    static constexpr uint8_t CLS = CLS_;                 // event class of this path
};
// the block tile proper: 8 warps, 2048 hits per layer, 5632 per station, 32 x 64 cells
using HeavyCfg = BCfg<256, 8, 5632, 64, 32, kClsHeavy>;
// the medium tile: 2 warps, 384 hits per layer, 960 per station, 16 x 32 cells
using MedBCfg = BCfg<64, 6, 960, 32, 16, kClsMedium>;
constexpr int kHThreads = HeavyCfg::THREADS;
constexpr int kHLayerCap = HeavyCfg::LAYER_CAP;
constexpr int kHHCap = HeavyCfg::HCAP;

struct LayerMeta {
    float lox, scx, loy, scy;  // cell map: column = bin of s_x, row = bin of s_y
    float bmax;                // largest pruning bound b of the layer
    float rmax, smax;          // largest r ~ 1/z and |s_x| + |s_y| (pair bounds)
    int32_t base;              // global index of the layer's first hit
    int32_t pbase;             // tile position of the layer's first stored hit
    int32_t nlive;             // stored hits (finite coordinates)
};

// One station staged in shared memory: hit slopes (s_x, s_y) and layer-local
// indices, sorted by layer then cell; cell starts and per-layer metadata.
template <int NX_, int NY_>
struct TileView {
    static constexpr int NX = NX_, NY = NY_, NC = NX_ * NY_;
    float2* P;
    uint16_t* idx;
    uint16_t* bst;  // [3 * NC + 1] tile positions: layer l, cell k at l * NC + k
    LayerMeta* meta;
};

template <class Cfg>
struct WarpTile {
    float2 P[Cfg::HCAP];
    uint16_t idx[Cfg::HCAP];
    union alignas(16) {
        uint32_t queue[kQCap];  // pair queue (enumeration)
        uint32_t cnt[Cfg::NC];  // cell counts of the layer being staged
    };
    float2 T[Cfg::TCAP];        // trigger triplet slopes
    union {
        unsigned long long Tijk[Cfg::TCAP];  // their packed hits (distinct_hits)
        float2 Tt[Cfg::TCAP];                // or their (min t, max t) (free-streaming windows)
    };
    uint8_t alive[Cfg::TCAP];
    alignas(8) uint16_t bst[3 * Cfg::NC + 1];  // cell starts
    LayerMeta meta[3];
    static_assert(Cfg::NC <= kQCap, "cell counts share the pair queue's memory");
};

template <class B>
struct BlockSmem {
    float2 P[B::HCAP];
    uint16_t idx[B::HCAP];
    uint32_t queue[B::WARPS][kQCap];
    alignas(4) uint16_t bst[3 * B::NC + 1];  // cell starts (cell counts while a layer is staged)
    LayerMeta meta[3];
    int32_t off[3 * kMaxStations + 1];
    int32_t wsum[B::WARPS];
    int red_i[B::WARPS][2];
    int red_k[B::WARPS][7];
    unsigned long long s_pool;
    long long s_item;
    int s_gi, s_rank, s_nT, s_cand, s_hx, s_hy, s_next;
};
using HeavySmem = BlockSmem<HeavyCfg>;

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// distinct_hits: do the candidates ijk[0, n) (those with alive set, when
// alive is given) hold two that use no common hit?  The warp walks the pair
// matrix in 32 x 32 tiles (candidate b of a tile comes by shuffle) and stops
// at the first tile with such a pair; warp-uniform result.  Block version:
// the warps take the rows of tiles in turn and stop at a block-shared flag.
__device__ __forceinline__ bool pair_tile_rows(const unsigned long long* ijk, const uint8_t* alive, int n, int a0,
                                               int lane) {
    const int a = a0 + lane;
    const bool va = a < n && (!alive || alive[a]);
    const unsigned long long ca = va ? ijk[a] : 0ull;
    for (int b0 = a0; b0 < n; b0 += 32) {
        const int b = b0 + lane;
        const bool vb = b < n && (!alive || alive[b]);
        const unsigned long long cb = vb ? ijk[b] : 0ull;
        bool f = false;
        for (int q = 0; q < 32; ++q) {
            const unsigned long long cq = __shfl_sync(0xffffffffu, cb, q);
            const bool vq = __shfl_sync(0xffffffffu, vb, q);
            f |= va & vq & (b0 + q > a) && ijk_disjoint(ca, cq);
        }
        if (__any_sync(0xffffffffu, f)) return true;
    }
    return false;
}

__device__ bool warp_disjoint_pair(const unsigned long long* ijk, const uint8_t* alive, int n, int lane) {
    for (int a0 = 0; a0 < n; a0 += 32)
        if (pair_tile_rows(ijk, alive, n, a0, lane)) return true;
    return false;
}

// All threads of the block call it; sh_flag is block-shared scratch.
template <int THREADS>
__device__ bool block_disjoint_pair(const unsigned long long* ijk, const uint8_t* alive, int n, int* sh_flag) {
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (threadIdx.x == 0) *sh_flag = 0;
    __syncthreads();
    for (int a0 = 32 * wp; a0 < n; a0 += THREADS) {
        if (__any_sync(0xffffffffu, *(volatile int*)sh_flag)) break;  // warp-uniform
        if (pair_tile_rows(ijk, alive, n, a0, lane)) {
            if (lane == 0) *(volatile int*)sh_flag = 1;
            break;
        }
    }
    return __syncthreads_or(*(volatile int*)sh_flag);
}

// Min/max of non-NaN floats through the integer reduction unit: the map is
// strictly increasing on floats ordered by value.
__device__ __forceinline__ int f2key(float f) {
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float key2f(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }
__device__ __forceinline__ float warp_min(float v) { return key2f(__reduce_min_sync(kFull, f2key(v))); }
__device__ __forceinline__ float warp_max(float v) { return key2f(__reduce_max_sync(kFull, f2key(v))); }

__device__ __forceinline__ int warp_incl_scan(int v, int lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += o;
    }
    return v;
}

// Index of the lane whose exclusive prefix `excl` is the last one <= it
// (excl non-decreasing over the lanes): binary lifting over shuffles.
__device__ __forceinline__ int owner_lane(int excl, int it) {
    int o = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int ex = __shfl_sync(kFull, excl, o + s);
        o += (ex <= it) ? s : 0;
    }
    return o;
}

// Pulls the hit lines [h0, h1) of x, y, z into L2 (addresses stay inside the
// arrays: the first line starts at or after index h0 & ~31 >= 0).
__device__ __forceinline__ void prefetch_hits_l2(const Job& j, int32_t h0, int32_t h1, int lane) {
    for (int32_t a = (h0 & ~31) + 32 * lane; a < h1; a += 32 * 32) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(j.x + a));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(j.y + a));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(j.z + a));
    }
}

__device__ __forceinline__ int station_of(int si, int trig) { return si == 0 ? trig : (si - 1 < trig ? si - 1 : si); }

// Free-streaming windows: are the times a, b, c coincident (max t <=
// fl32(min t + dt))?  Also returns min and max.
__device__ __forceinline__ bool coincident3(float a, float b, float c, float dt, float& tmin, float& tmax) {
    tmin = fminf(fminf(a, b), c);
    tmax = fmaxf(fmaxf(a, b), c);
    return tmax <= __fadd_rn(tmin, dt);
}

// A partner triplet with times (pmin, pmax) of a trigger triplet with times
// T = (min, max): itself coincident, and the six hits together.
__device__ __forceinline__ bool partner_coincident(float pmin, float pmax, float2 T, float dt) {
    return pmax <= __fadd_rn(pmin, dt) && fmaxf(pmax, T.y) <= __fadd_rn(fminf(pmin, T.x), dt);
}

// ------------------------------------------------------- event offsets

// The (3S+1) offsets of one event live in two registers per lane.
struct EvOff {
    int32_t a, b;
};

__device__ __forceinline__ int32_t off_get(const EvOff& o, int idx) {  // idx warp-uniform
    return idx < 32 ? __shfl_sync(kFull, o.a, idx) : __shfl_sync(kFull, o.b, idx - 32);
}

// Loads and checks the event's CSR span: non-decreasing, first >= 0 (== 0
// for event 0), last <= n_hits (== n_hits for the last event).
__device__ bool warp_load_offsets(const Job& j, int64_t e, int lane, EvOff& o) {
    const int S3 = j.S * 3;
    const int32_t* base = j.off + e * S3;
    o.a = lane <= S3 ? __ldg(base + lane) : 0;
    o.b = 32 + lane <= S3 ? __ldg(base + 32 + lane) : 0;
    int32_t na = __shfl_down_sync(kFull, o.a, 1);
    const int32_t b0 = __shfl_sync(kFull, o.b, 0);
    if (lane == 31) na = b0;
    const int32_t nb = __shfl_down_sync(kFull, o.b, 1);
    bool bad = (lane < S3 && na < o.a) || (32 + lane < S3 && nb < o.b);
    const int32_t first = off_get(o, 0), last = off_get(o, S3);
    if (lane == 0) {
        if (first < 0 || (e == 0 && first != 0)) bad = true;
        if ((int64_t)last > j.n_hits || (e == j.n_events - 1 && (int64_t)last != j.n_hits)) bad = true;
    }
    return !__any_sync(kFull, bad);
}

// ------------------------------------------------------- warp staging

// Cell histogram of the layer being staged on a block tile, kept in place in
// the layer's own cell-start array: two 16-bit counters per 32-bit word (a
// count never exceeds the layer's hit capacity, < 2^16, so no carry crosses
// into the neighbour).  Returns the hit's rank in its cell.  (The warp tile
// counts with 32-bit counters in its pair queue's memory instead.)
__device__ __forceinline__ int cell_count_add(uint16_t* cnt, int cell) {
    uint32_t* wd = reinterpret_cast<uint32_t*>(cnt) + (cell >> 1);
    const int sh = (cell & 1) << 4;
    return (int)((atomicAdd(wd, 1u << sh) >> sh) & 0xffffu);
}

// Stages one layer into the warp tile.  Returns 0, or 1 (z <= 0), or 2 (a
// hit whose pruning bound is not finite).  Hits are counted into cells with
// shared-memory atomics on 32-bit counters that share the pair queue's
// memory (the queue is empty between stations; the order inside a cell is
// not fixed, and results do not depend on it) and written sorted by cell.
template <class Cfg>
__device__ int stage_layer_warp(const Job& j, WarpTile<Cfg>& w, int l, int32_t base, int32_t n, int32_t pbase,
                                int lane, int& nlive) {
    constexpr int R = Cfg::RMAX, NX = Cfg::NX, NY = Cfg::NY, NC = Cfg::NC, CPL = NC / 32;  // cells per lane
    static_assert(NC % 128 == 0, "cells per layer: four 32-bit counters (16 bytes) per lane");
    float sx[R], sy[R];
    int key[R];  // cell << 16 | rank in the cell once binned; -1: not stored
    float lox = INFINITY, hix = -INFINITY, loy = INFINITY, hiy = -INFINITY, bmax = 0.0f, rmax = 0.0f, smax = 0.0f;
    bool bad = false;
    uint16_t* bst = w.bst + l * NC;  // the end of layer l is the start of layer l + 1
#pragma unroll
    for (int q = 0; q < CPL / 4; ++q) reinterpret_cast<uint4*>(w.cnt)[CPL / 4 * lane + q] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        key[r] = -1;
        sx[r] = sy[r] = 0.0f;
    }
    // fast path: lanes past the end re-read the layer's last hit (a real hit,
    // harmless in min/max; it is not stored)
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (32 * r >= n) break;  // warp-uniform
        const int h = lane + 32 * r;
        const bool in = h < n;
        const int hc = in ? h : n - 1;
        const HitFast p = hit_fast(__ldg(j.x + base + hc), __ldg(j.y + base + hc), __ldg(j.z + base + hc), j.K);
        bad |= !p.ok;
        key[r] = in ? 0 : -1;
        sx[r] = p.sx;
        sy[r] = p.sy;
        lox = fminf(lox, p.sx);
        hix = fmaxf(hix, p.sx);
        if constexpr (NY > 1) {
            loy = fminf(loy, p.sy);
            hiy = fmaxf(hiy, p.sy);
        }
        bmax = fmaxf(bmax, p.b);
        rmax = fmaxf(rmax, p.r);
        smax = fmaxf(smax, p.l1);
    }
    if (__any_sync(kFull, bad)) {
        // some hit has an odd coordinate: classify every hit exactly
        bool zbad = false, wild = false;
        lox = loy = INFINITY;
        hix = hiy = -INFINITY;
        bmax = rmax = smax = 0.0f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (32 * r >= n) break;
            const int h = lane + 32 * r;
            const bool in = h < n;
            const int hc = in ? h : n - 1;
            const HitPrep p = hit_prep(__ldg(j.x + base + hc), __ldg(j.y + base + hc), __ldg(j.z + base + hc), j.K);
            zbad |= in & p.zbad;
            wild |= in & p.wild;
            const bool live = in & p.live & !p.wild;
            key[r] = live ? 0 : -1;
            lox = live ? fminf(lox, p.sx) : lox;
            hix = live ? fmaxf(hix, p.sx) : hix;
            if constexpr (NY > 1) {
                loy = live ? fminf(loy, p.sy) : loy;
                hiy = live ? fmaxf(hiy, p.sy) : hiy;
            }
            bmax = live ? fmaxf(bmax, p.b) : bmax;
            rmax = live ? fmaxf(rmax, p.r) : rmax;
            smax = live ? fmaxf(smax, p.l1) : smax;
        }
        if (__any_sync(kFull, zbad)) return 1;
        if (__any_sync(kFull, wild)) return 2;
    }
    lox = warp_min(lox);
    hix = warp_max(hix);
    if constexpr (NY > 1) {
        loy = warp_min(loy);
        hiy = warp_max(hiy);
    }
    // the bounds and their parts are finite and >= 0 here: their bit patterns
    // order like the values
    bmax = __int_as_float(__reduce_max_sync(kFull, __float_as_int(bmax)));
    rmax = __int_as_float(__reduce_max_sync(kFull, __float_as_int(rmax)));
    smax = __int_as_float(__reduce_max_sync(kFull, __float_as_int(smax)));
    const float scx = bin_scale(lox, hix, NX), scy = NY > 1 ? bin_scale(loy, hiy, NY) : 0.0f;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (32 * r >= n) break;
        if (key[r] >= 0) {
            const int row = NY > 1 ? slope_bin<NY>(sy[r], loy, scy) : 0;
            const int cell = row * NX + slope_bin<NX>(sx[r], lox, scx);
            key[r] = JPSI_IN(j.ctrl, cell >= 0 && cell < NC) ? (cell << 16) | (int)atomicAdd(&w.cnt[cell], 1u) : -1;
        }
    }
    __syncwarp();
    // exclusive scan of the NC cell counts, NC/32 consecutive cells per lane
    int cs[CPL];
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < CPL / 4; ++q) {
        const uint4 c4 = reinterpret_cast<const uint4*>(w.cnt)[CPL / 4 * lane + q];
        cs[4 * q] = (int)c4.x;
        cs[4 * q + 1] = (int)c4.y;
        cs[4 * q + 2] = (int)c4.z;
        cs[4 * q + 3] = (int)c4.w;
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) cnt += cs[q];
    const int incl = warp_incl_scan(cnt, lane);
    const int total = __shfl_sync(kFull, incl, 31);
    int run = pbase + incl - cnt;
#pragma unroll
    for (int q = 0; q < CPL / 4; ++q) {  // four 16-bit starts per 8-byte store
        const uint32_t s0 = (uint32_t)run, s1 = s0 + cs[4 * q], s2 = s1 + cs[4 * q + 1], s3 = s2 + cs[4 * q + 2];
        reinterpret_cast<uint2*>(bst)[CPL / 4 * lane + q] = make_uint2((s0 & 0xffffu) | (s1 << 16), (s2 & 0xffffu) | (s3 << 16));
        run = (int)s3 + cs[4 * q + 3];
    }
    if (lane == 31) bst[NC] = (uint16_t)(pbase + total);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (32 * r >= n) break;
        if (key[r] >= 0) {
            const int pos = bst[key[r] >> 16] + (key[r] & 0xffff);
            if (JPSI_IN(j.ctrl, pos >= 0 && pos < Cfg::HCAP)) {
                w.P[pos] = make_float2(sx[r], sy[r]);
                w.idx[pos] = (uint16_t)(lane + 32 * r);
            }
        }
    }
    if (lane == 0) {
        LayerMeta m;
        m.lox = lox;
        m.scx = scx;
        m.loy = loy;
        m.scy = scy;
        m.bmax = bmax;
        m.rmax = rmax;
        m.smax = smax;
        m.base = base;
        m.pbase = pbase;
        m.nlive = total;
        w.meta[l] = m;
    }
    __syncwarp();
    nlive = total;
    return 0;
}

template <class Cfg>
__device__ int stage_station_warp(const Job& j, WarpTile<Cfg>& w, int lane, const EvOff& o, int s) {
    int pbase = 0;
    for (int l = 0; l < 3; ++l) {
        const int32_t b = off_get(o, s * 3 + l), e = off_get(o, s * 3 + l + 1);
        int nl = 0;
        const int st = stage_layer_warp<Cfg>(j, w, l, b, e - b, pbase, lane, nl);
        if (st) return st;
        pbase += nl;
    }
    return 0;
}

// ------------------------------------------------------ block staging

// Block version of the staging (block-tile paths).
template <class B>
__device__ int stage_layer_block(const Job& j, BlockSmem<B>& sm, int l, int32_t base, int32_t n, int32_t pbase,
                                 int& nlive) {
    constexpr int CPT = B::NC / B::THREADS;  // cells per thread
    static_assert(B::NC % B::THREADS == 0, "cells per layer");
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    float sx[B::RMAX], sy[B::RMAX];
    int key[B::RMAX];  // cell << 16 | rank in the cell once binned; -1: not stored
    static_assert(CPT % 2 == 0, "two 16-bit cell counters per word");
    float lox = INFINITY, hix = -INFINITY, loy = INFINITY, hiy = -INFINITY, bmax = 0.0f, rmax = 0.0f, smax = 0.0f;
    bool zbad = false, wild = false;
    uint16_t* bst = sm.bst + l * B::NC;  // the end of layer l is the start of layer l + 1
#pragma unroll
    for (int q = 0; q < CPT / 2; ++q) reinterpret_cast<uint32_t*>(bst)[CPT / 2 * tid + q] = 0;
#pragma unroll
    for (int r = 0; r < B::RMAX; ++r) {
        key[r] = -1;
        sx[r] = sy[r] = 0.0f;
    }
#pragma unroll
    for (int r = 0; r < B::RMAX; ++r) {
        if (B::THREADS * r >= n) break;  // block-uniform
        const int h = tid + B::THREADS * r;
        const bool in = h < n;
        const int hc = in ? h : n - 1;
        const HitPrep p = hit_prep(__ldg(j.x + base + hc), __ldg(j.y + base + hc), __ldg(j.z + base + hc), j.K);
        zbad |= in & p.zbad;
        wild |= in & p.wild;
        const bool live = in & p.live & !p.wild;
        key[r] = live ? 0 : -1;
        sx[r] = p.sx;
        sy[r] = p.sy;
        lox = live ? fminf(lox, p.sx) : lox;
        hix = live ? fmaxf(hix, p.sx) : hix;
        loy = live ? fminf(loy, p.sy) : loy;
        hiy = live ? fmaxf(hiy, p.sy) : hiy;
        bmax = live ? fmaxf(bmax, p.b) : bmax;
        rmax = live ? fmaxf(rmax, p.r) : rmax;
        smax = live ? fmaxf(smax, p.l1) : smax;
    }
    // block-wide ranges, bounds and flags: a warp reduction of order-
    // preserving integer keys (the bounds and their parts are >= 0, so their
    // bit patterns already order like the values), one slot per warp, then
    // each warp reduces the slots itself
    int kv[7] = {f2key(lox), -f2key(hix), f2key(loy), -f2key(hiy), -__float_as_int(bmax), -__float_as_int(rmax),
                 -__float_as_int(smax)};  // minima (maxima negated; keys of finite values never overflow)
#pragma unroll
    for (int q = 0; q < 7; ++q) kv[q] = __reduce_min_sync(kFull, kv[q]);
    const int fz = __any_sync(kFull, zbad), fw = __any_sync(kFull, wild);
    if (lane == 0) {
#pragma unroll
        for (int q = 0; q < 7; ++q) sm.red_k[wp][q] = kv[q];
        sm.red_i[wp][0] = fz;
        sm.red_i[wp][1] = fw;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 7; ++q) kv[q] = __reduce_min_sync(kFull, lane < B::WARPS ? sm.red_k[lane][q] : INT_MAX);
    const int anyz = __any_sync(kFull, lane < B::WARPS && sm.red_i[lane][0]);
    const int anyw = __any_sync(kFull, lane < B::WARPS && sm.red_i[lane][1]);
    lox = key2f(kv[0]);
    hix = key2f(-kv[1]);
    loy = key2f(kv[2]);
    hiy = key2f(-kv[3]);
    bmax = __int_as_float(-kv[4]);
    rmax = __int_as_float(-kv[5]);
    smax = __int_as_float(-kv[6]);
    // (red_k / red_i are written again only in the next layer, behind the
    // three barriers below)
    if (anyz) return 1;
    if (anyw) return 2;
    const float scx = bin_scale(lox, hix, B::NX), scy = bin_scale(loy, hiy, B::NY);
#pragma unroll
    for (int r = 0; r < B::RMAX; ++r) {
        if (B::THREADS * r >= n) break;
        if (key[r] >= 0) {
            const int cell = slope_bin<B::NY>(sy[r], loy, scy) * B::NX + slope_bin<B::NX>(sx[r], lox, scx);
            key[r] = JPSI_IN(j.ctrl, cell >= 0 && cell < B::NC) ? (cell << 16) | cell_count_add(bst, cell) : -1;
        }
    }
    __syncthreads();
    // block exclusive scan of the cell counts, CPT consecutive cells per thread
    int cs[CPT];
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        cs[q] = (int)bst[CPT * tid + q];
        cnt += cs[q];
    }
    const int incl = warp_incl_scan(cnt, lane);
    if (lane == 31) sm.wsum[wp] = incl;
    __syncthreads();
    int woff = 0, total = 0;
    if constexpr (B::WARPS > 2) {  // the warps' offsets by a scan over the lanes
        const int ws = lane < B::WARPS ? sm.wsum[lane] : 0;
        const int wi = warp_incl_scan(ws, lane);
        woff = __shfl_sync(kFull, wi - ws, wp);
        total = __shfl_sync(kFull, wi, B::WARPS - 1);
    } else {
#pragma unroll
        for (int q = 0; q < B::WARPS; ++q) {
            woff += q < wp ? sm.wsum[q] : 0;
            total += sm.wsum[q];
        }
    }
    int run = pbase + woff + incl - cnt;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        bst[CPT * tid + q] = (uint16_t)run;
        run += cs[q];
    }
    if (tid == B::THREADS - 1) bst[B::NC] = (uint16_t)(pbase + total);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < B::RMAX; ++r) {
        if (B::THREADS * r >= n) break;
        if (key[r] >= 0) {
            const int pos = bst[key[r] >> 16] + (key[r] & 0xffff);
            if (JPSI_IN(j.ctrl, pos >= 0 && pos < B::HCAP)) {
                sm.P[pos] = make_float2(sx[r], sy[r]);
                sm.idx[pos] = (uint16_t)(tid + B::THREADS * r);
            }
        }
    }
    if (tid == 0) {
        LayerMeta m;
        m.lox = lox;
        m.scx = scx;
        m.loy = loy;
        m.scy = scy;
        m.bmax = bmax;
        m.rmax = rmax;
        m.smax = smax;
        m.base = base;
        m.pbase = pbase;
        m.nlive = total;
        sm.meta[l] = m;
    }
    // no barrier here: the next layer works on its own cells and tile
    // positions, and the caller synchronises before the tile is read
    nlive = total;
    return 0;
}

// Cell window of a query: columns [x0, x1] around c_x +- W_x, rows [y0, y1]
// around c_y +- W_y, each padded as in query_bins.  An intersection of
// windows may be empty (x0 > x1 or y0 > y1).
struct Win {
    int x0, x1, y0, y1;
};

template <class TV>
__device__ __forceinline__ Win cell_window(const TV& t, int l, float cx, float cy, float Wx, float Wy) {
    const LayerMeta& m = t.meta[l];
    Win w;
    query_bins<TV::NX>(cx, Wx, m.lox, m.scx, w.x0, w.x1);
    if constexpr (TV::NY > 1) {
        query_bins<TV::NY>(cy, Wy, m.loy, m.scy, w.y0, w.y1);
    } else {
        w.y0 = w.y1 = 0;
    }
    return w;
}

__device__ __forceinline__ Win win_meet(const Win& a, const Win& b) {
    return Win{max(a.x0, b.x0), min(a.x1, b.x1), max(a.y0, b.y0), min(a.y1, b.y1)};
}

// Tile positions of window w in layer l as two runs: its first row
// [a, a + n0), and the positions from its second row's first column to its
// last row's last column [a2, a2 + n1) (every cell in between included, a
// superset when the window spans more than two rows; empty for one row).
template <class TV>
__device__ __forceinline__ void win_runs(const TV& t, int l, const Win& w, int& a, int& n0, int& a2, int& n1) {
    a = n0 = a2 = n1 = 0;
    if (w.x0 > w.x1 || w.y0 > w.y1) return;
    const uint16_t* b = t.bst + l * TV::NC;
    a = b[w.y0 * TV::NX + w.x0];
    n0 = b[w.y0 * TV::NX + w.x1 + 1] - a;
    if (w.y1 > w.y0) {
        a2 = b[(w.y0 + 1) * TV::NX + w.x0];
        n1 = b[w.y1 * TV::NX + w.x1 + 1] - a2;
    }
}

// ---------------------------------------------------------- enumeration

// Pair bound of the staged layers a and b (pair_bound in jpsi_device.cuh).
template <class TV>
__device__ __forceinline__ float layer_pair_bound(const TV& t, int a, int b, float K) {
    const LayerMeta &ma = t.meta[a], &mb = t.meta[b];
    return pair_bound(ma.rmax, ma.smax, mb.rmax, mb.smax, K);
}

// Where passing trigger triplets' slopes go (CHAIN mode, trigger station).
// Warp path: a warp-local count; block path: a block-shared counter.
struct TSink {
    bool on;
    float2* T;
    int cap;
    int* sh_n;  // block-shared counter, or null
    int n;      // warp-local counter when sh_n is null
    bool norec = false;  // a repeated enumeration: record no triplet entries
    unsigned long long* ijk = nullptr;  // distinct_hits: the triplets' packed hits beside T
    float2* tt = nullptr;               // free-streaming windows: their (min t, max t) beside T
};

// Items of up to 32 lanes laid end to end: lane i owns items [excl, excl +
// n0 + n1), the first n0 at tile positions a.., the others at a2.. (runs of
// win_runs).  An item's owner is found by owner_lane over excl.
struct Runs {
    int excl, total;    // this lane's first item; items of the warp
    int sa, split, sb;  // item it of this lane sits at (it < split ? sa : sb) + it
    bool two;           // some lane has a second run (warp-uniform)
};

template <int NY>
__device__ __forceinline__ Runs runs_scan(int a, int n0, int a2, int n1, int lane) {
    Runs r;
    const int len = n0 + n1;
    const int incl = warp_incl_scan(len, lane);
    r.total = __shfl_sync(kFull, incl, 31);
    r.excl = incl - len;
    r.sa = a - r.excl;
    r.split = r.excl + n0;
    r.sb = a2 - r.split;
    r.two = NY > 1 && __any_sync(kFull, n1 > 0);  // one-row tiles never have a second run
    return r;
}

// Tile position of item `it`, owned by lane o (all lanes call it).
template <int NY>
__device__ __forceinline__ int runs_pos(const Runs& r, int o, int it) {
    const int pa = __shfl_sync(kFull, r.sa, o) + it;
    if (NY == 1 || !r.two) return pa;
    const int sp = __shfl_sync(kFull, r.split, o), pb = __shfl_sync(kFull, r.sb, o) + it;
    return it < sp ? pa : pb;
}

// Position of the k-th (0-based) set bit of m (binary lifting over the
// counts of lower bits; k < popc(m)).
__device__ __forceinline__ int nth_set_bit(unsigned m, int k) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1)
        if (__popc(m & ((1u << (pos + s)) - 1u)) <= k) pos += s;
    return pos;
}

// Triples that passed both pair tests and wait for their exact fit (block
// paths): lane l < m holds one, as tile positions i | j << 16 and k.  The
// fits (and the global loads of their hits) then run 32 at a time.
struct Pending {
    uint32_t pair = 0;
    int k = 0;
    int m = 0;
};

// P1 on the triples of the lanes with `has` (tile positions pi, pj, pk) and
// what follows from a pass: the triplet's rank in its unit (warp-local on
// the warp path, from a block-shared counter on the block path), its row
// (emit pass), its slopes for the trigger sink (CHAIN) and its entry in the
// scatter record.  All lanes call it.
template <bool EMIT, class TV>
__device__ __forceinline__ void fit_and_record(const Job& j, const TV& t, int lane, const Cuts& c, bool has, int pi,
                                               int pj, int pk, TSink& ts, int32_t* rows, int limit, int64_t unit,
                                               int* sh_rank, int tag, int& count) {
    bool ok = false;
    float mx = 0.f, my = 0.f;
    float2 tt = make_float2(0.f, 0.f);
    int ii = 0, jj = 0, kk = 0;
    if (has) {
        const int32_t base0 = t.meta[0].base, base1 = t.meta[1].base, base2 = t.meta[2].base;
        ii = t.idx[pi];
        jj = t.idx[pj];
        kk = t.idx[pk];
        const float xs[3] = {__ldg(j.x + base0 + ii), __ldg(j.x + base1 + jj), __ldg(j.x + base2 + kk)};
        const float ys[3] = {__ldg(j.y + base0 + ii), __ldg(j.y + base1 + jj), __ldg(j.y + base2 + kk)};
        const float zs[3] = {__ldg(j.z + base0 + ii), __ldg(j.z + base1 + jj), __ldg(j.z + base2 + kk)};
        ok = fit_pass(xs, ys, zs, c, mx, my);
        if constexpr (kStream) {  // coincident, and owned by this window
            const int64_t e = unit / j.S;
            ok = ok && coincident3(__ldg(j.t + base0 + ii), __ldg(j.t + base1 + jj), __ldg(j.t + base2 + kk), j.dt,
                                   tt.x, tt.y) &&
                 tt.x >= __ldg(j.wb + e) && tt.x < __ldg(j.wb + e + 1);
        }
    }
    const unsigned mask = __ballot_sync(kFull, ok);
    if (mask) {
        const int rk = __popc(mask & lanemask_lt()), np = __popc(mask);
        int base = count;
        if (sh_rank) {
            int b = 0;
            if (lane == 0) b = atomicAdd(sh_rank, np);
            base = __shfl_sync(kFull, b, 0);
        }
        if (EMIT && ok && base + rk < limit &&  // never past the unit's rows
            JPSI_IN(j.ctrl, (rows - j.triplets) / 3 + base + rk < j.trip_cap)) {
            int32_t* r = rows + 3 * (int64_t)(base + rk);
            r[0] = ii;
            r[1] = jj;
            r[2] = kk;
        }
        if (ts.on) {
            int tb = ts.n;
            if (ts.sh_n) {
                int b = 0;
                if (lane == 0) b = atomicAdd(ts.sh_n, np);
                tb = __shfl_sync(kFull, b, 0);
            } else {
                ts.n += np;
            }
            if (ok && tb + rk < ts.cap) {
                ts.T[tb + rk] = make_float2(mx, my);
                if (ts.ijk) ts.ijk[tb + rk] = pack_ijk(ii, jj, kk);
                if (ts.tt) ts.tt[tb + rk] = tt;
            }
        }
        if (!EMIT && j.tscr && !ts.norec) {  // record for the scatter pass
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(&j.ctrl->scratch_n, (unsigned long long)np);
            b = __shfl_sync(kFull, b, 0) + rk;
            if (ok && b < (unsigned long long)j.tscr_cap) {
                TripEntry te;
                te.unit = (int32_t)unit;
                te.rank = base + rk;
                te.ijk = (unsigned long long)ii | ((unsigned long long)jj << 20) | ((unsigned long long)kk << 40) |
                         ((unsigned long long)tag << kTagShift);
                j.tscr[b] = te;
            }
        }
        count += np;
    }
}

// Drains a pair queue: every (i, j) against the L2 hits in the meet of both
// cell windows.  The (pair, k) items of up to 32 pairs are spread evenly over
// the lanes (a warp prefix sum over the window sizes; each lane finds the
// pair owning its item by binary lifting).  Items that pass both pair tests
// get the exact fit at once (COMPACT false: the warp tile, where a station
// has about one such item) or join the pending triples of `pd` first
// (COMPACT true: the block paths), so that the global loads of the fits
// run for 32 triples at a time.
template <bool EMIT, bool COMPACT, class TV>
__device__ void drain(const Job& j, const TV& t, const uint32_t* queue, int lane, const Cuts& c, int qn,
                      TSink& ts, int32_t* rows, int limit, int64_t unit, int* sh_rank, int tag, int& count,
                      Pending& pd) {
    const float B02 = layer_pair_bound(t, 0, 2, c.K), B12 = layer_pair_bound(t, 1, 2, c.K);
    for (int q0 = 0; q0 < qn; q0 += 32) {
        const int q = q0 + lane;
        uint32_t en = 0;
        int a = 0, m0 = 0, a2 = 0, m1 = 0;
        if (q < qn) {
            en = queue[q];
            const float2 Pi = t.P[en & 0xffffu], Pj = t.P[en >> 16];
            const Win w = win_meet(cell_window(t, 2, Pi.x, Pi.y, B02, B02), cell_window(t, 2, Pj.x, Pj.y, B12, B12));
            win_runs(t, 2, w, a, m0, a2, m1);
        }
        const Runs rr = runs_scan<TV::NY>(a, m0, a2, m1, lane);
        const int total = rr.total;
        for (int it0 = 0; it0 < total; it0 += 32) {
            const int it = it0 + lane;
            const int o = owner_lane(rr.excl, it);
            const uint32_t eo = __shfl_sync(kFull, en, o);
            const int ko = runs_pos<TV::NY>(rr, o, it);
            const bool in = it < total;
            const int ko_c = in ? ko : (int)(eo >> 16);
            const float2 Pi = t.P[eo & 0xffffu], Pj = t.P[eo >> 16], Pk = t.P[ko_c];
            const bool cand = in & pair_ok(Pi.x, Pi.y, Pk.x, Pk.y, B02) & pair_ok(Pj.x, Pj.y, Pk.x, Pk.y, B12);
            if constexpr (!COMPACT) {
                fit_and_record<EMIT>(j, t, lane, c, cand, (int)(eo & 0xffffu), (int)(eo >> 16), ko_c, ts, rows, limit,
                                     unit, sh_rank, tag, count);
            } else {
                unsigned mask = __ballot_sync(kFull, cand);
                while (mask) {  // warp-uniform: candidates of rank r go to lane pd.m + r
                    const int np = __popc(mask), take = min(np, 32 - pd.m);
                    const int r = lane - pd.m;
                    const int src = nth_set_bit(mask, min(max(r, 0), np - 1));
                    const uint32_t vp = __shfl_sync(kFull, eo, src);
                    const int vk = __shfl_sync(kFull, ko_c, src);
                    if (r >= 0 && r < take) {
                        pd.pair = vp;
                        pd.k = vk;
                    }
                    pd.m += take;
                    mask = take == np ? 0u : mask & ~((1u << nth_set_bit(mask, take)) - 1u);
                    if (pd.m == 32) {
                        fit_and_record<EMIT>(j, t, lane, c, true, (int)(pd.pair & 0xffffu), (int)(pd.pair >> 16),
                                             pd.k, ts, rows, limit, unit, sh_rank, tag, count);
                        pd.m = 0;
                    }
                }
            }
        }
    }
    __syncwarp();
}

// The pending triples of a block-path warp, at the end of its station.
template <bool EMIT, class TV>
__device__ __forceinline__ void flush_pending(const Job& j, const TV& t, int lane, const Cuts& c, TSink& ts,
                                              int32_t* rows, int limit, int64_t unit, int* sh_rank, int tag,
                                              int& count, Pending& pd) {
    if (pd.m > 0)
        fit_and_record<EMIT>(j, t, lane, c, lane < pd.m, (int)(pd.pair & 0xffffu), (int)(pd.pair >> 16), pd.k, ts,
                             rows, limit, unit, sh_rank, tag, count);
    pd.m = 0;
}

template <class TV>
__device__ bool road_warp(const Job& j, const TV& t, const Cuts& c, float mx, float my, float2 Tt, int lane);

// CHAIN-mode trigger slopes a block searches for while it enumerates a
// station (block path): item n_rounds + i of the block-shared counter is
// slope i; a slope with no compatible triplet in the station loses its flag.
struct RoadItems {
    const float2* T;
    uint8_t* alive;
    int n;
    const float2* Tt = nullptr;  // free-streaming windows: the slopes' (min t, max t)
};

// All passing triplets of the staged station (Sec. 3.2 steps 1-2) found by
// this warp: rounds of 32 L0 hits (all of them, or those this warp takes
// from a block-shared counter when the warps of a block share a station).
// On the small and medium tiles each lane walks its own hit's L1 window; on
// the block tile each hit's window (its runs of cells) is spread over the
// lanes so every lane tests one candidate pair per step.  Pairs that may
// belong to a passing triplet are queued and drained against L2.
template <bool EMIT, bool SHARED, class TV>
__device__ int enum_station(const Job& j, const TV& t, uint32_t* queue, int lane, const Cuts& c,
                            TSink& ts, int32_t* rows, int limit, int64_t unit, int* sh_rank, int tag, int* sh_next,
                            const RoadItems* rd = nullptr) {
    const int n0 = t.meta[0].nlive, n1 = t.meta[1].nlive, n2 = t.meta[2].nlive;
    if (n0 == 0 || n1 == 0 || n2 == 0) return 0;
    const int n_rounds = (n0 + 31) >> 5;
    const int p0 = t.meta[0].pbase;
    const float B01 = layer_pair_bound(t, 0, 1, c.K);
    int qn = 0, count = 0;
    Pending pd;
    // rounds of 32 L0 hits: in order on the warp path; on the block path each
    // warp takes the next one from a block-shared counter
    auto next_round = [&]() {
        int g = 0;
        if (lane == 0) g = atomicAdd(sh_next, 1);
        return 32 * __shfl_sync(kFull, g, 0);
    };
    int i0 = 0;
    if constexpr (SHARED) {
        i0 = next_round();
        // items past the rounds: trigger slopes to search for (CHAIN)
        while (rd && i0 >= n0 && (i0 >> 5) - n_rounds < rd->n) {
            const int ti = (i0 >> 5) - n_rounds;
            if (rd->alive[ti]) {
                const float2 m = rd->T[ti];
                const bool found = road_warp(j, t, c, m.x, m.y, rd->Tt ? rd->Tt[ti] : make_float2(0.f, 0.f), lane);
                if (lane == 0 && !found) rd->alive[ti] = 0;
            }
            i0 = next_round();
        }
    }
    for (; i0 < n0;) {
        const bool has = i0 + lane < n0;
        const float2 Pi = t.P[p0 + (has ? i0 + lane : 0)];
        int a = 0, m0 = 0, a2 = 0, m1 = 0;
        if (has) win_runs(t, 1, cell_window(t, 1, Pi.x, Pi.y, B01, B01), a, m0, a2, m1);
        if constexpr (TV::NC <= kWalkCells) {
            // small and medium tiles: each lane walks its own hit's window
            // (both runs), as long as the warp's longest.  The 32 L0 hits of
            // a round are neighbours in the cell order, so their windows are
            // alike, and a step costs a load, the test and a vote instead of
            // the balanced step's owner search: 8 % less kernel time on the
            // 10^6-event workload (about 3 candidates per window), 3 % on the
            // medium tile.  The block tile's wider windows keep balanced steps.
            const int len = m0 + m1;
            const int nmax = __reduce_max_sync(kFull, len);
            for (int k = 0; k < nmax; ++k) {
                const bool in = k < len;
                const int pj = k < m0 ? a + k : a2 + (k - m0);
                const float2 Pj = t.P[in ? pj : p0];
                const bool pass = in & pair_ok(Pi.x, Pi.y, Pj.x, Pj.y, B01);
                const unsigned mask = __ballot_sync(kFull, pass);
                if (mask) {
                    const int qi = qn + __popc(mask & lanemask_lt());
                    if (pass && JPSI_IN(j.ctrl, qi < kQCap)) queue[qi] = (uint32_t)(p0 + i0 + lane) | ((uint32_t)pj << 16);
                    qn += __popc(mask);
                    if (qn > kQCap - 32) {
                        __syncwarp();
                        drain<EMIT, SHARED>(j, t, queue, lane, c, qn, ts, rows, limit, unit, sh_rank, tag, count, pd);
                        qn = 0;
                    }
                }
            }
        } else {
            const Runs rr = runs_scan<TV::NY>(a, m0, a2, m1, lane);
            const int total = rr.total;
            for (int it0 = 0; it0 < total; it0 += 32) {
                const int it = it0 + lane;
                const int o = owner_lane(rr.excl, it);
                const int pj = runs_pos<TV::NY>(rr, o, it);
                const bool in = it < total;
                const float2 Po = t.P[p0 + i0 + o];
                const float2 Pj = t.P[in ? pj : p0];
                const bool pass = in & pair_ok(Po.x, Po.y, Pj.x, Pj.y, B01);
                const unsigned mask = __ballot_sync(kFull, pass);
                if (mask) {
                    const int qi = qn + __popc(mask & lanemask_lt());
                    if (pass && JPSI_IN(j.ctrl, qi < kQCap))
                        queue[qi] = (uint32_t)(p0 + i0 + o) | ((uint32_t)pj << 16);
                    qn += __popc(mask);
                    if (qn > kQCap - 32) {
                        __syncwarp();
                        drain<EMIT, SHARED>(j, t, queue, lane, c, qn, ts, rows, limit, unit, sh_rank, tag, count, pd);
                        qn = 0;
                    }
                }
            }
        }
        if constexpr (SHARED) {
            i0 = next_round();
            while (rd && i0 >= n0 && (i0 >> 5) - n_rounds < rd->n) {
                const int ti = (i0 >> 5) - n_rounds;
                if (rd->alive[ti]) {
                    const float2 m = rd->T[ti];
                    const bool found = road_warp(j, t, c, m.x, m.y, rd->Tt ? rd->Tt[ti] : make_float2(0.f, 0.f), lane);
                    if (lane == 0 && !found) rd->alive[ti] = 0;
                }
                i0 = next_round();
            }
        } else {
            i0 += 32;
        }
    }
    __syncwarp();
    drain<EMIT, SHARED>(j, t, queue, lane, c, qn, ts, rows, limit, unit, sh_rank, tag, count, pd);
    if constexpr (SHARED) flush_pending<EMIT>(j, t, lane, c, ts, rows, limit, unit, sh_rank, tag, count, pd);
    return count;
}

// Tile positions of a cell window, row by row: the first row's run [a, e)
// is given; windows of more than one row continue on the next rows (each
// row's columns [x0, x1] are one run of positions).
template <int NX, int NY>
struct WinIter {
    int p, end, row, y1, x0, x1;
    const uint16_t* bs;
    __device__ __forceinline__ WinIter(int a, int e, const uint16_t* b, const Win& w) : p(a), end(e) {
        if constexpr (NY > 1) {
            bs = b;
            row = w.y0;
            y1 = w.y1;
            x0 = w.x0;
            x1 = w.x1;
            settle();
        }
    }
    __device__ __forceinline__ void settle() {
        if constexpr (NY > 1) {
            while (p >= end && row < y1) {
                ++row;
                p = bs[row * NX + x0];
                end = bs[row * NX + x1 + 1];
            }
        }
    }
    __device__ __forceinline__ bool valid() const { return p < end; }
    __device__ __forceinline__ void next() {
        ++p;
        settle();
    }
};

// Does the staged station hold a passing triplet compatible with the
// trigger slopes (mx, my)?  Per-thread search through each layer's cells
// inside the tube, row by row.
template <class TV>
__device__ bool road(const Job& j, const TV& t, const Cuts& c, float mx, float my, float2 Tt) {
    Win w[3];
    int a[3], e[3];  // first-row runs
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const float b = t.meta[l].bmax;
        w[l] = cell_window(t, l, mx, my, __fadd_rn(b, __fmul_rn(2.0f * kKappa, fabsf(mx))),
                           __fadd_rn(b, __fmul_rn(2.0f * kKappa, fabsf(my))));
        const uint16_t* bs = t.bst + l * TV::NC;
        a[l] = bs[w[l].y0 * TV::NX + w[l].x0];
        e[l] = bs[w[l].y0 * TV::NX + w[l].x1 + 1];
    }
    const uint16_t *bs0 = t.bst, *bs1 = t.bst + TV::NC, *bs2 = t.bst + 2 * TV::NC;
    const int32_t base0 = t.meta[0].base, base1 = t.meta[1].base, base2 = t.meta[2].base;
    const float b0 = t.meta[0].bmax, b1 = t.meta[1].bmax, b2 = t.meta[2].bmax;
    for (WinIter<TV::NX, TV::NY> i0(a[0], e[0], bs0, w[0]); i0.valid(); i0.next()) {
        const int p0 = i0.p;
        const float2 P0 = t.P[p0];
        if (!tube_ok(P0.x, P0.y, b0, mx, my)) continue;
        const int h0 = base0 + t.idx[p0];
        const float x0 = __ldg(j.x + h0), y0 = __ldg(j.y + h0), z0 = __ldg(j.z + h0);
        if (!tube_pass(x0, y0, z0, mx, my, c)) continue;
        for (WinIter<TV::NX, TV::NY> i1(a[1], e[1], bs1, w[1]); i1.valid(); i1.next()) {
            const int p1 = i1.p;
            const float2 P1 = t.P[p1];
            if (!tube_ok(P1.x, P1.y, b1, mx, my)) continue;
            const int h1 = base1 + t.idx[p1];
            const float x1 = __ldg(j.x + h1), y1 = __ldg(j.y + h1), z1 = __ldg(j.z + h1);
            if (!tube_pass(x1, y1, z1, mx, my, c)) continue;
            for (WinIter<TV::NX, TV::NY> i2(a[2], e[2], bs2, w[2]); i2.valid(); i2.next()) {
                const int p2 = i2.p;
                const float2 P2 = t.P[p2];
                if (!tube_ok(P2.x, P2.y, b2, mx, my)) continue;
                const int h2 = base2 + t.idx[p2];
                const float xs[3] = {x0, x1, __ldg(j.x + h2)};
                const float ys[3] = {y0, y1, __ldg(j.y + h2)};
                const float zs[3] = {z0, z1, __ldg(j.z + h2)};
                float fx, fy;
                if (fit_pass(xs, ys, zs, c, fx, fy) && chain_pass(xs, ys, zs, mx, my, c)) {
                    if constexpr (!kStream) return true;
                    float pmin, pmax;
                    coincident3(__ldg(j.t + h0), __ldg(j.t + h1), __ldg(j.t + h2), j.dt, pmin, pmax);
                    if (partner_coincident(pmin, pmax, Tt, j.dt)) return true;
                }
            }
        }
    }
    return false;
}

// Warp-cooperative road(): the 32 lanes search together for one trigger
// slope (mx, my warp-uniform).  For each layer they test the tube on the
// window's tile positions, row by row, 32 at a time, and keep the hits that
// pass tube_pass: the k-th kept hit of layer l sits in lane k's registers.
// Every combination of one kept hit per layer then gets P1 and P2.  A layer
// with more than 32 kept hits hands the slope to road() on one lane (no such
// limit).  Same answer as road(), warp-uniform.
template <class TV>
__device__ bool road_warp(const Job& j, const TV& t, const Cuts& c, float mx, float my, float2 Tt, int lane) {
    float hx[3] = {0.f, 0.f, 0.f}, hy[3] = {0.f, 0.f, 0.f}, hz[3] = {0.f, 0.f, 0.f}, ht[3] = {0.f, 0.f, 0.f};
    int nk[3] = {0, 0, 0};
    bool over = false;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        const float b = t.meta[l].bmax;
        const Win w = cell_window(t, l, mx, my, __fadd_rn(b, __fmul_rn(2.0f * kKappa, fabsf(mx))),
                                  __fadd_rn(b, __fmul_rn(2.0f * kKappa, fabsf(my))));
        const uint16_t* bs = t.bst + l * TV::NC;
        const int32_t base = t.meta[l].base;
        for (int row = w.y0; row <= w.y1 && !over; ++row) {
            const int a = bs[row * TV::NX + w.x0], e = bs[row * TV::NX + w.x1 + 1];
            for (int p0 = a; p0 < e; p0 += 32) {
                const int p = p0 + lane;
                bool keep = false;
                float x = 0.f, y = 0.f, z = 0.f, tm = 0.f;
                if (p < e) {
                    const float2 P = t.P[p];
                    if (tube_ok(P.x, P.y, b, mx, my)) {
                        const int h = base + t.idx[p];
                        x = __ldg(j.x + h);
                        y = __ldg(j.y + h);
                        z = __ldg(j.z + h);
                        if constexpr (kStream) tm = __ldg(j.t + h);
                        keep = tube_pass(x, y, z, mx, my, c);
                    }
                }
                unsigned m = __ballot_sync(kFull, keep);
                if (nk[l] + __popc(m) > 32) {
                    over = true;
                    break;
                }
                while (m) {  // the kept hits go to lanes nk, nk + 1, ...
                    const int src = __ffs(m) - 1;
                    m &= m - 1;
                    const float vx = __shfl_sync(kFull, x, src), vy = __shfl_sync(kFull, y, src),
                                vz = __shfl_sync(kFull, z, src), vt = __shfl_sync(kFull, tm, src);
                    if (lane == nk[l]) {
                        hx[l] = vx;
                        hy[l] = vy;
                        hz[l] = vz;
                        ht[l] = vt;
                    }
                    ++nk[l];
                }
            }
        }
        if (over) break;
        if (nk[l] == 0) return false;
    }
    if (over) {
        bool f = false;
        if (lane == 0) f = road(j, t, c, mx, my, Tt);
        return __shfl_sync(kFull, f, 0);
    }
    const int n01 = nk[0] * nk[1], total = n01 * nk[2];
    for (int it0 = 0; it0 < total; it0 += 32) {
        const int it = min(it0 + lane, total - 1);
        const int i2 = it / n01, r = it - i2 * n01, i1 = r / nk[0], i0 = r - i1 * nk[0];
        const float xs[3] = {__shfl_sync(kFull, hx[0], i0), __shfl_sync(kFull, hx[1], i1),
                             __shfl_sync(kFull, hx[2], i2)};
        const float ys[3] = {__shfl_sync(kFull, hy[0], i0), __shfl_sync(kFull, hy[1], i1),
                             __shfl_sync(kFull, hy[2], i2)};
        const float zs[3] = {__shfl_sync(kFull, hz[0], i0), __shfl_sync(kFull, hz[1], i1),
                             __shfl_sync(kFull, hz[2], i2)};
        float fx, fy;
        bool ok = fit_pass(xs, ys, zs, c, fx, fy) && chain_pass(xs, ys, zs, mx, my, c);
        if constexpr (kStream) {
            float pmin, pmax;
            coincident3(__shfl_sync(kFull, ht[0], i0), __shfl_sync(kFull, ht[1], i1), __shfl_sync(kFull, ht[2], i2),
                        j.dt, pmin, pmax);
            ok = ok && partner_coincident(pmin, pmax, Tt, j.dt);
        }
        if (__any_sync(kFull, ok)) return true;
    }
    return false;
}

// ------------------------------------------------------------ warp path

__device__ __forceinline__ void push_event(const Job& j, int64_t e, uint8_t cls) {
    j.ev_class[e] = cls;
    if (j.plain) return;  // the one-launch form's block kernel finds the event by its class
    if (cls == kClsMedium) {
        const int gi = atomicAdd(&j.ctrl->n_medium, 1);
        if (JPSI_IN(j.ctrl, gi < j.n_events)) j.mlist[gi] = (int32_t)e;
    } else if (cls == kClsHeavy) {
        const int gi = atomicAdd(&j.ctrl->n_heavy, 1);
        if (JPSI_IN(j.ctrl, gi < j.n_events)) j.hlist[gi] = (int32_t)e;
    } else {
        const int gi = atomicAdd(&j.ctrl->n_generic, 1);
        if (JPSI_IN(j.ctrl, gi < j.n_events)) j.glist[gi] = (int32_t)e;
    }
}

// Does an event fit a warp tile of this shape (processed stations only)?
// The tile's layer capacity may be lowered at run time (Job::cap_small,
// cap_medium: a tuning choice, results do not depend on it).
template <class Cfg>
__device__ __forceinline__ bool fits_warp(const Job& j, const EvOff& o, int nproc) {
    const int cap = min(Cfg::LAYER_CAP, Cfg::CLS == kClsLight ? j.cap_small : j.cap_medium);
    bool fits = true;
    for (int si = 0; si < nproc; ++si) {
        const int s = station_of(si, j.trig);
        const int32_t o0 = off_get(o, 3 * s), o1 = off_get(o, 3 * s + 1), o2 = off_get(o, 3 * s + 2),
                      o3 = off_get(o, 3 * s + 3);
        if (o1 - o0 > cap || o2 - o1 > cap || o3 - o2 > cap || o3 - o0 > Cfg::HCAP) fits = false;
    }
    return fits;
}

template <class Cfg>
__device__ void light_event_count(const Job& j, WarpTile<Cfg>& w, int lane, const Cuts& c, int64_t e) {
    using TV = TileView<Cfg::NX, Cfg::NY>;
    constexpr bool kSmall = Cfg::CLS == kClsLight;
    EvOff o;
    const int S = j.S;
    const bool valid = warp_load_offsets(j, e, lane, o);
    if (kSmall && !valid) {
        if (lane == 0) {
            atomicOr(&j.ctrl->status, kStInvalid);
            j.ev_class[e] = kClsInvalid;
        }
        return;
    }
    const bool chain = j.mode == 1 && S > 1;
    const int nproc = j.mode == 1 ? S : 1;
    if (!fits_warp<Cfg>(j, o, nproc)) {
        // all lanes take part in the shuffles of the size check
        const bool to_medium = kSmall && !j.plain && fits_warp<MediumCfg>(j, o, nproc);
        if (lane == 0) push_event(j, e, to_medium ? kClsMedium : kClsHeavy);
        return;
    }
    {  // the first station's lines start towards L2 now; each station then
       // prefetches the next (prefetching all of them evicted some lines
       // before use: 17 % more DRAM reads, against 4 % for one ahead)
        const int s0 = station_of(0, j.trig);
        if (!j.host_hits) prefetch_hits_l2(j, off_get(o, 3 * s0), off_get(o, 3 * s0 + 3), lane);
    }
    const TV t{w.P, w.idx, w.bst, w.meta};
    TSink ts{false, w.T, Cfg::TCAP, nullptr, 0};
    ts.ijk = j.distinct ? w.Tijk : nullptr;
    ts.tt = kStream ? w.Tt : nullptr;
    int trig_count = 0;
    for (int si = 0; si < nproc; ++si) {
        const int s = station_of(si, j.trig);
        if (si + 1 < nproc && !j.host_hits) {
            const int sn = station_of(si + 1, j.trig);
            prefetch_hits_l2(j, off_get(o, 3 * sn), off_get(o, 3 * sn + 3), lane);
        }
        const int st = stage_station_warp<Cfg>(j, w, lane, o, s);
        if (st == 1) {
            if (lane == 0) {
                atomicOr(&j.ctrl->status, kStInvalid);
                j.ev_class[e] = kClsInvalid;
            }
            return;
        }
        if (st == 2) {
            if (lane == 0) push_event(j, e, kClsGeneric);
            return;
        }
        ts.on = (chain || j.distinct) && s == j.trig;  // the trigger triplets: CHAIN slopes, candidates' hits
        const int cnt = enum_station<false, false>(j, t, w.queue, lane, c, ts, nullptr, 0, e * S + s, nullptr, Cfg::CLS,
                                            nullptr);
        if (ts.on) {
            if (ts.n > Cfg::TCAP) {
                if (lane == 0) push_event(j, e, kClsHeavy);
                return;
            }
            for (int i = lane; i < ts.n; i += 32) w.alive[i] = 1;
            __syncwarp();
            ts.on = false;
        }
        if (s == j.trig) trig_count = cnt;
        if (lane == 0) j.unit_counts[e * S + s] = cnt;
        if (chain && s != j.trig && ts.n > 0) {
            // one trigger slope per lane (a warp tile holds few; measured
            // faster here than the warp-cooperative search of the block tile)
            for (int ti = lane; ti < ts.n; ti += 32)
                if (w.alive[ti]) {
                    const float2 m = w.T[ti];
                    if (!road(j, t, c, m.x, m.y, kStream ? w.Tt[ti] : make_float2(0.f, 0.f))) w.alive[ti] = 0;
                }
            __syncwarp();
        }
    }
    if (j.mode == 0 && lane < S && lane != j.trig) j.unit_counts[e * S + lane] = 0;
    int tc = trig_count;
    if (chain) {
        int a = 0;
        for (int ti = lane; ti < ts.n; ti += 32) a += w.alive[ti];
        tc = __reduce_add_sync(kFull, a);
    }
    if (j.distinct) {  // ts.n is warp-uniform
        const bool f = ts.n >= 2 && warp_disjoint_pair(w.Tijk, chain ? w.alive : nullptr, ts.n, lane);
        if (lane == 0) j.dpair[e] = f;
    }
    if (lane == 0) {
        j.track_counts[e] = tc;
        j.ev_class[e] = Cfg::CLS;
    }
}

template <class Cfg>
__device__ void light_event_emit(const Job& j, WarpTile<Cfg>& w, int lane, const Cuts& c, int64_t e) {
    using TV = TileView<Cfg::NX, Cfg::NY>;
    if (j.ev_class[e] != Cfg::CLS) return;
    const int S = j.S;
    const int nproc = j.mode == 1 ? S : 1;
    bool any = false;
    for (int si = 0; si < nproc; ++si) any |= j.unit_counts[e * S + station_of(si, j.trig)] != 0;
    if (!any) return;
    EvOff o;
    warp_load_offsets(j, e, lane, o);
    const TV t{w.P, w.idx, w.bst, w.meta};
    TSink ts{false, nullptr, 0, nullptr, 0};
    for (int si = 0; si < nproc; ++si) {
        const int s = station_of(si, j.trig);
        const int64_t u = e * S + s;
        const int cnt = j.unit_counts[u];
        if (cnt == 0) continue;
        if (stage_station_warp<Cfg>(j, w, lane, o, s) != 0) {
            if (lane == 0) atomicOr(&j.ctrl->status, kStEmitMismatch);
            return;
        }
        const int got = enum_station<true, false>(j, t, w.queue, lane, c, ts, j.triplets + 3 * j.trip_off[u], cnt, u,
                                           nullptr, Cfg::CLS, nullptr);
        if (got != cnt && lane == 0) atomicOr(&j.ctrl->status, kStEmitMismatch);
    }
}

template <bool EMIT, class Cfg>
__device__ __forceinline__ void light_event(const Job& j, WarpTile<Cfg>& w, int lane, const Cuts& c, int64_t e) {
    if (EMIT)
        light_event_emit<Cfg>(j, w, lane, c, e);
    else
        light_event_count<Cfg>(j, w, lane, c, e);
}

// Small warp tiles: every event of the batch (statically one warp per event,
// or persistent warps grabbing `grab` events at a time).
// 56 registers: nine 4-warp blocks (36 warps) fit an SM by registers (the
// 5.3 KB warp tiles would allow ten); measured faster than 64 registers with
// eight blocks, despite some spills.
template <bool EMIT>
__global__ void __maxnreg__(56) k_light(const __grid_constant__ Job j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    WarpTile<SmallCfg>& w = reinterpret_cast<WarpTile<SmallCfg>*>(smem_raw)[wi];
    const Cuts c{j.cx, j.cy, j.K};
    if (j.persistent) {
        unsigned long long* ctr = &j.ctrl->work[EMIT ? 4 : 0];
        const long long e_end = j.ev_begin + j.ev_count;
        for (;;) {
            long long e0 = 0;
            if (lane == 0) e0 = (long long)atomicAdd(ctr, (unsigned long long)j.grab);
            e0 = j.ev_begin + __shfl_sync(kFull, e0, 0);
            if (e0 >= e_end) break;
            const long long e1 = min(e0 + (long long)j.grab, e_end);
            for (long long e = e0; e < e1; ++e) light_event<EMIT, SmallCfg>(j, w, lane, c, e);
        }
    } else {
        const long long e = j.ev_begin + (long long)blockIdx.x * (blockDim.x >> 5) + wi;
        if (e < j.ev_begin + j.ev_count) light_event<EMIT, SmallCfg>(j, w, lane, c, e);
    }
}

// ------------------------------------------------------ block-tile path

// Stages station s of the event whose offsets are in sm.off.  Returns 0, 1
// (z <= 0) or 2 (not prunable).
template <class B>
__device__ int stage_station_block(const Job& j, BlockSmem<B>& sm, int s) {
    int pbase = 0;
    for (int l = 0; l < 3; ++l) {
        const int32_t b = sm.off[3 * s + l], e = sm.off[3 * s + l + 1];
        int nl = 0;
        const int st = stage_layer_block(j, sm, l, b, e - b, pbase, nl);
        if (st) return st;
        pbase += nl;
    }
    return 0;
}

template <class B>
__device__ __forceinline__ void load_event_offsets(const Job& j, BlockSmem<B>& sm, int64_t e) {
    const int S3 = 3 * j.S;
    for (int i = threadIdx.x; i <= S3; i += B::THREADS) sm.off[i] = j.off[e * S3 + i];
    __syncthreads();
}

// Job::hT[gi].y of a block-tile event: >= 0, its stations run on separate
// blocks with that many trigger slopes in the pool from hT[gi].x on; or
constexpr int kHTOwned = -1;  // its first block does (did) all of it
constexpr int kHTMoved = -2;  // it went to the unpruned kernel

// Hands an event from the block-tile path to the unpruned kernel, once (the
// per-station blocks of one event may all find a reason).
__device__ __forceinline__ void heavy_to_generic(const Job& j, int gi, int64_t e) {
    if (atomicExch(&j.hT[gi].y, kHTMoved) != kHTMoved) push_event(j, e, kClsGeneric);
}

// One station of a block-tile event: staging, the triplet search of the
// station (Sec. 3.2 steps 1-2) and, in CHAIN mode, the trigger slopes in
// T[0, nT) that find no compatible triplet here lose their alive flag.
// Counting pass: writes the unit count (also returned in cnt); returns false
// when the event left the path (then nothing else may be done for it).
// Emit pass: writes rows.  Block-uniform arguments; all threads call it.
// Who hands an event on when a station cannot be pruned: gi >= 0 is the
// event's block-tile list entry (its state in Job::hT);
constexpr int kGiPlain = -1;  // the one-launch form: the same block goes on unpruned
constexpr int kGiOwn = -2;    // a block that owns the whole event: to the unpruned list

// Pulls the hit lines of station s of the event in sm.off into L2 (block
// version of prefetch_hits_l2; addresses stay inside [o[0] & ~31, o[3])).
template <class B>
__device__ __forceinline__ void prefetch_station_block(const Job& j, const BlockSmem<B>& sm, int s) {
    if (j.host_hits) return;
    const int32_t h0 = sm.off[3 * s], h1 = sm.off[3 * s + 3];
    for (int32_t a = (h0 & ~31) + 32 * (int)threadIdx.x; a < h1; a += 32 * B::THREADS) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(j.x + a));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(j.y + a));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(j.z + a));
    }
}

// s_next: the station this block stages next (-1: none), whose lines start
// towards L2 now; the station's own lines too, so that its second and third
// layers arrive while the first is staged.
template <bool EMIT, class B>
__device__ bool heavy_unit(const Job& j, BlockSmem<B>& sm, const Cuts& c, int gi, int64_t e, int s, TSink& ts,
                           const float2* T, uint8_t* alive, int nT, int& cnt, int s_next = -1,
                           const float2* Tt = nullptr) {
    using TV = TileView<B::NX, B::NY>;
    const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
    const int64_t u = e * j.S + s;
    const int cnt_expected = EMIT ? j.unit_counts[u] : 0;
    prefetch_station_block(j, sm, s);
    if (s_next >= 0) prefetch_station_block(j, sm, s_next);
    const int st = stage_station_block(j, sm, s);
    if (st != 0) {
        if (tid == 0) {
            if (EMIT) {
                atomicOr(&j.ctrl->status, kStEmitMismatch);
            } else if (st == 1) {
                atomicOr(&j.ctrl->status, kStInvalid);
                j.ev_class[e] = kClsInvalid;
            } else if (gi == kGiPlain) {
                j.ev_class[e] = kClsGeneric;
            } else if (gi == kGiOwn) {
                push_event(j, e, kClsGeneric);
            } else {
                heavy_to_generic(j, gi, e);
            }
        }
        return false;
    }
    if (tid == 0) {
        sm.s_rank = 0;
        sm.s_next = 0;
    }
    __syncthreads();
    int32_t* rows = EMIT ? j.triplets + 3 * j.trip_off[u] : nullptr;
    // the station's trigger-slope searches run on the warps beside its
    // enumeration rounds (both only read the staged tile)
    const bool empty = sm.meta[0].nlive == 0 || sm.meta[1].nlive == 0 || sm.meta[2].nlive == 0;
    const RoadItems rd{T, alive, EMIT || empty ? 0 : nT, Tt};
    enum_station<EMIT, true>(j, TV{sm.P, sm.idx, sm.bst, sm.meta}, sm.queue[wp], lane, c, ts, rows,
                       cnt_expected, u, &sm.s_rank, B::CLS, &sm.s_next, &rd);
    __syncthreads();
    cnt = sm.s_rank;
    if (EMIT) {
        if (tid == 0 && cnt != cnt_expected) atomicOr(&j.ctrl->status, kStEmitMismatch);
        return true;
    }
    if (tid == 0) j.unit_counts[u] = cnt;
    if (empty)  // no triplet at all in this station: no slope finds one
        for (int ti = tid; ti < nT; ti += B::THREADS) alive[ti] = 0;
    return true;
}

// Counting pass of one block-tile event (list index gi).  The trigger
// station comes first; in CHAIN mode its passing triplets' slopes go to the
// block's own list, and then, when the trigger-slope pool has room, to the
// pool: the other stations are then left to k_heavy_units (one block per
// station) and k_heavy_final.  Otherwise this block does them itself.  The
// event may move on to the unpruned kernel (too large, extreme coordinates
// or too many trigger triplets for the block's list).
__device__ void heavy_event(const Job& j, HeavySmem& sm, const Cuts& c, int gi, int64_t e) {
    const int tid = threadIdx.x, lane = tid & 31;
    const int S = j.S;
    const bool chain = j.mode == 1 && S > 1;
    const int nproc = j.mode == 1 ? S : 1;
    if (tid == 0) {
        sm.s_nT = 0;
        j.hT[gi] = make_int2(0, kHTOwned);
    }
    load_event_offsets(j, sm, e);
    bool fits = true;
    for (int si = 0; si < nproc; ++si) {
        const int32_t* o = sm.off + 3 * station_of(si, j.trig);
        if (o[1] - o[0] > kHLayerCap || o[2] - o[1] > kHLayerCap || o[3] - o[2] > kHLayerCap || o[3] - o[0] > kHHCap)
            fits = false;
    }
    if (!fits) {
        if (tid == 0) heavy_to_generic(j, gi, e);
        return;
    }
    float2* T = j.tlist + (int64_t)blockIdx.x * j.tlist_cap;
    uint8_t* alive = j.talive + (int64_t)blockIdx.x * j.tlist_cap;
    unsigned long long* ijk = j.distinct ? j.tlist_ijk + (int64_t)blockIdx.x * j.tlist_cap : nullptr;
    // free-streaming windows: the slopes' times in the same per-block storage
    float2* tt = kStream ? reinterpret_cast<float2*>(j.tlist_ijk + (int64_t)blockIdx.x * j.tlist_cap) : nullptr;
    int trig_count = 0, nT = 0;
    for (int si = 0; si < nproc; ++si) {
        const int s = station_of(si, j.trig);
        TSink ts{(chain || j.distinct) && si == 0, T, j.tlist_cap, &sm.s_nT, 0};
        ts.ijk = ijk;
        ts.tt = tt;
        int cnt = 0;
        const int sn = si + 1 < nproc ? station_of(si + 1, j.trig) : -1;
        if (!heavy_unit<false>(j, sm, c, gi, e, s, ts, T, alive, si == 0 ? 0 : nT, cnt, sn, tt)) return;
        if (si > 0) {
            __syncthreads();
            continue;
        }
        trig_count = cnt;
        nT = sm.s_nT;
        if (nT > j.tlist_cap) {
            if (tid == 0) heavy_to_generic(j, gi, e);
            return;
        }
        if (!chain) {
            if (j.distinct) {  // PAPER: every passing trigger triplet is a candidate
                const bool f = nT >= 2 && block_disjoint_pair<kHThreads>(ijk, nullptr, nT, &sm.s_hx);
                if (tid == 0) j.dpair[e] = f;
            }
            break;
        }
        if (tid == 0) sm.s_pool = nT > 0 ? atomicAdd(&j.ctrl->tpool_n, (unsigned long long)nT) : 0ull;
        __syncthreads();
        const unsigned long long pb = sm.s_pool;
        if (pb + (unsigned long long)nT <= (unsigned long long)j.tpool_cap) {
            for (int i = tid; i < nT; i += kHThreads) {
                j.tpool[pb + i] = T[i];
                j.tpool_alive[pb + i] = 1;
                if (ijk) j.tpool_ijk[pb + i] = ijk[i];
                if (tt) reinterpret_cast<float2*>(j.tpool_ijk)[pb + i] = tt[i];
            }
            if (tid == 0) j.hT[gi] = make_int2((int)pb, nT);
            return;
        }
        for (int i = tid; i < nT; i += kHThreads) alive[i] = 1;
        __syncthreads();
    }
    int tc = trig_count;
    if (chain) {
        if (tid == 0) sm.s_cand = 0;
        __syncthreads();
        int a = 0;
        for (int ti = tid; ti < nT; ti += kHThreads) a += alive[ti];
        a = __reduce_add_sync(kFull, a);
        if (lane == 0 && a) atomicAdd(&sm.s_cand, a);
        __syncthreads();
        tc = sm.s_cand;
        if (j.distinct) {
            const bool f = nT >= 2 && block_disjoint_pair<kHThreads>(ijk, alive, nT, &sm.s_hx);
            if (tid == 0) j.dpair[e] = f;
        }
    }
    if (tid == 0) {
        if (j.mode == 0)
            for (int s = 0; s < S; ++s)
                if (s != j.trig) j.unit_counts[e * S + s] = 0;
        j.track_counts[e] = tc;
    }
}

// Medium tile: 2-warp blocks take the events of the medium list, one at a
// time, and run every station of their event: the trigger station first (in
// CHAIN mode its passing triplets' slopes, at most kTCap, stay in shared
// memory), then the others, whose enumeration rounds share the warps with
// the searches for those slopes.  An event with more trigger slopes goes on
// to the block tile; one with extreme coordinates to the unpruned kernel.
struct MediumSmem {
    BlockSmem<MedBCfg> b;
    float2 T[kTCap];
    union {
        unsigned long long Tijk[kTCap];  // their packed hits (distinct_hits)
        float2 Tt[kTCap];                // or their (min t, max t) (free-streaming windows)
    };
    uint8_t alive[kTCap];
};

template <bool EMIT>
__device__ void medium_event(const Job& j, MediumSmem& ms, const Cuts& c, int64_t e) {
    BlockSmem<MedBCfg>& sm = ms.b;
    const int tid = threadIdx.x, lane = tid & 31;
    const int S = j.S;
    const bool chain = j.mode == 1 && S > 1;
    const int nproc = j.mode == 1 ? S : 1;
    load_event_offsets(j, sm, e);
    if (EMIT) {
        for (int si = 0; si < nproc; ++si) {
            const int s = station_of(si, j.trig);
            if (j.unit_counts[e * S + s] == 0) continue;
            TSink ts{false, nullptr, 0, nullptr, 0};
            int cnt = 0;
            heavy_unit<true>(j, sm, c, kGiOwn, e, s, ts, nullptr, nullptr, 0, cnt,
                             si + 1 < nproc ? station_of(si + 1, j.trig) : -1);
            __syncthreads();
        }
        return;
    }
    int trig_count = 0, nT = 0;
    for (int si = 0; si < nproc; ++si) {
        const int s = station_of(si, j.trig);
        if (tid == 0) sm.s_nT = 0;
        __syncthreads();
        TSink ts{(chain || j.distinct) && si == 0, ms.T, kTCap, &sm.s_nT, 0};
        ts.ijk = j.distinct ? ms.Tijk : nullptr;
        ts.tt = kStream ? ms.Tt : nullptr;
        int cnt = 0;
        const int sn = si + 1 < nproc ? station_of(si + 1, j.trig) : -1;
        if (!heavy_unit<false>(j, sm, c, kGiOwn, e, s, ts, ms.T, ms.alive, si == 0 ? 0 : nT, cnt, sn,
                               kStream ? ms.Tt : nullptr))
            return;
        __syncthreads();
        if (si > 0) continue;
        trig_count = cnt;
        nT = sm.s_nT;
        if (nT > kTCap) {  // more trigger slopes than this tile keeps
            if (tid == 0) push_event(j, e, kClsHeavy);
            return;
        }
        if (!chain) break;
        for (int i = tid; i < nT; i += MedBCfg::THREADS) ms.alive[i] = 1;
        __syncthreads();
    }
    int tc = trig_count;
    if (chain) {
        if (tid == 0) sm.s_cand = 0;
        __syncthreads();
        int a = 0;
        for (int ti = tid; ti < nT; ti += MedBCfg::THREADS) a += ms.alive[ti];
        a = __reduce_add_sync(kFull, a);
        if (lane == 0 && a) atomicAdd(&sm.s_cand, a);
        __syncthreads();
        tc = sm.s_cand;
    }
    if (j.distinct) {
        const bool f = nT >= 2 && block_disjoint_pair<MedBCfg::THREADS>(ms.Tijk, chain ? ms.alive : nullptr, nT,
                                                                         &sm.s_hx);
        if (tid == 0) j.dpair[e] = f;
    }
    if (tid == 0) {
        if (j.mode == 0)
            for (int s = 0; s < S; ++s)
                if (s != j.trig) j.unit_counts[e * S + s] = 0;
        j.track_counts[e] = tc;
    }
}

template <bool EMIT>
__global__ void __launch_bounds__(MedBCfg::THREADS, 14) k_medium(const __grid_constant__ Job j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MediumSmem& ms = *reinterpret_cast<MediumSmem*>(smem_raw);
    const Cuts c{j.cx, j.cy, j.K};
    const int n_med = *(volatile int32_t*)&j.ctrl->n_medium, m0 = *(volatile int32_t*)&j.ctrl->m_begin;
    unsigned long long* ctr = &j.ctrl->work[EMIT ? 5 : 1];
    for (;;) {
        if (threadIdx.x == 0) ms.b.s_gi = m0 + (int)atomicAdd(ctr, 1ull);
        __syncthreads();
        const int gi = ms.b.s_gi;
        __syncthreads();
        if (gi >= n_med) break;
        const int64_t e = j.mlist[gi];
        if (!EMIT || j.ev_class[e] == kClsMedium) medium_event<EMIT>(j, ms, c, e);
        __syncthreads();
    }
}

// Orders the block-tile list by decreasing event size (hits), so the
// persistent blocks take the largest events first and the smaller ones fill
// in behind them.  One block, bitonic sort in shared memory; lists longer
// than kSortCap keep their order (they have enough events to balance).
constexpr int kSortCap = 4096;
__global__ void __launch_bounds__(1024) k_sort_heavy(const __grid_constant__ Job j) {
    __shared__ unsigned long long key[kSortCap];  // hits << 32 | event
    const int h0 = *(volatile int32_t*)&j.ctrl->h_begin;
    const int n = *(volatile int32_t*)&j.ctrl->n_heavy - h0;
    int32_t* list = j.hlist + h0;
    if (n < 2 || n > kSortCap) return;
    int m = 2;
    while (m < n) m <<= 1;
    const int64_t S3 = 3 * j.S;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        unsigned long long k = 0;  // padding sorts last
        if (i < n) {
            const int32_t e = list[i];
            const int64_t hits = j.off[(e + 1) * S3] - j.off[e * S3];
            k = ((unsigned long long)hits << 32) | (uint32_t)e;
        }
        key[i] = k;
    }
    __syncthreads();
    for (int size = 2; size <= m; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int p = i ^ stride;
                if (p > i) {
                    const unsigned long long a = key[i], b = key[p];
                    const bool down = (i & size) == 0;  // this run ends up decreasing
                    if (down ? a < b : a > b) {
                        key[i] = b;
                        key[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) list[i] = (int32_t)(uint32_t)key[i];
}

// Counting pass: persistent blocks take block-tile events from the list.
__global__ void __launch_bounds__(kHThreads, 3) k_heavy(const __grid_constant__ Job j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HeavySmem& sm = *reinterpret_cast<HeavySmem*>(smem_raw);
    const Cuts c{j.cx, j.cy, j.K};
    const int n_heavy = *(volatile int32_t*)&j.ctrl->n_heavy, h0 = *(volatile int32_t*)&j.ctrl->h_begin;
    for (;;) {
        if (threadIdx.x == 0) sm.s_gi = h0 + (int)atomicAdd(&j.ctrl->work[2], 1ull);
        __syncthreads();
        const int gi = sm.s_gi;
        __syncthreads();
        if (gi >= n_heavy) break;
        heavy_event(j, sm, c, gi, j.hlist[gi]);
        __syncthreads();
    }
}

// One block per (event, station) unit of the block-tile path.  Counting pass
// (CHAIN): the non-trigger stations of events whose trigger slopes went to
// the pool.  Emit pass: every processed station with triplets.
template <bool EMIT>
__global__ void __launch_bounds__(kHThreads, 3) k_heavy_units(const __grid_constant__ Job j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HeavySmem& sm = *reinterpret_cast<HeavySmem*>(smem_raw);
    const int S = j.S;
    if (!EMIT && (j.mode != 1 || S < 2)) return;
    const int per = EMIT ? (j.mode == 1 ? S : 1) : S - 1;  // units per event
    const Cuts c{j.cx, j.cy, j.K};
    const int h0 = *(volatile int32_t*)&j.ctrl->h_begin;
    const long long n_items = (long long)(*(volatile int32_t*)&j.ctrl->n_heavy - h0) * per;
    for (;;) {
        // thread 0 takes an item and decides (the state it reads may change
        // under other blocks; the block must act on one reading)
        if (threadIdx.x == 0) {
            long long k = (long long)atomicAdd(&j.ctrl->work[EMIT ? 6 : 8], 1ull);
            int hx = 0, hy = 0;
            if (k < n_items) {
                const int gi = h0 + (int)(k / per);
                const int64_t e = j.hlist[gi];
                const int s = station_of((int)(k % per) + (EMIT ? 0 : 1), j.trig);
                bool skip = j.ev_class[e] != kClsHeavy;
                if (EMIT) {
                    skip |= j.unit_counts[e * S + s] == 0;
                } else {
                    const int2 h = j.hT[gi];
                    hx = h.x;
                    hy = h.y;
                    skip |= hy < 0;  // finished by its first block, or moved on
                }
                if (skip) k = -1;
            }
            sm.s_item = k;
            sm.s_hx = hx;
            sm.s_hy = hy;
        }
        __syncthreads();
        const long long k = sm.s_item;
        const int hx = sm.s_hx, hy = sm.s_hy;
        __syncthreads();
        if (k >= n_items) break;
        if (k < 0) continue;
        const int gi = h0 + (int)(k / per);
        const int64_t e = j.hlist[gi];
        const int s = station_of((int)(k % per) + (EMIT ? 0 : 1), j.trig);
        load_event_offsets(j, sm, e);
        TSink ts{false, nullptr, 0, nullptr, 0};
        int cnt = 0;
        heavy_unit<EMIT>(j, sm, c, gi, e, s, ts, j.tpool + hx, j.tpool_alive + hx, hy, cnt, -1,
                         kStream ? reinterpret_cast<const float2*>(j.tpool_ijk) + hx : nullptr);
        __syncthreads();
    }
}

// CHAIN track counts of the events whose stations ran on separate blocks:
// the trigger slopes still alive after every station (one warp per event).
__global__ void k_heavy_final(const __grid_constant__ Job j) {
    if (j.mode != 1 || j.S < 2) return;
    const int n_heavy = *(volatile int32_t*)&j.ctrl->n_heavy, h0 = *(volatile int32_t*)&j.ctrl->h_begin;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int gi = h0 + ((blockIdx.x * blockDim.x + threadIdx.x) >> 5); gi < n_heavy; gi += nw) {
        const int2 h = j.hT[gi];
        const int64_t e = j.hlist[gi];
        if (h.y < 0 || j.ev_class[e] != kClsHeavy) continue;
        int a = 0;
        for (int t = lane; t < h.y; t += 32) a += j.tpool_alive[h.x + t];
        a = __reduce_add_sync(kFull, a);
        if (lane == 0) j.track_counts[e] = a;
        if (j.distinct) {
            const bool f = a >= 2 && warp_disjoint_pair(j.tpool_ijk + h.x, j.tpool_alive + h.x, h.y, lane);
            if (lane == 0) j.dpair[e] = f;
        }
    }
}

// --------------------------------------------------- unpruned block path

struct GHit {
    float x, y, z;
    HitPrep p;
};

__device__ __forceinline__ GHit ghit(const Job& j, int64_t h) {
    GHit g;
    g.x = __ldg(j.x + h);
    g.y = __ldg(j.y + h);
    g.z = __ldg(j.z + h);
    g.p = hit_prep(g.x, g.y, g.z, j.K);
    return g;
}

// Brute-force P2 search over every hit of every other station.
__device__ bool road_global(const Job& j, const int32_t* soff, const Cuts& c, float mx, float my, float2 Tt) {
    for (int s = 0; s < j.S; ++s) {
        if (s == j.trig) continue;
        const int32_t* o = soff + 3 * s;
        bool found = false;
        for (int32_t h0 = o[0]; h0 < o[1] && !found; ++h0) {
            const float x0 = __ldg(j.x + h0), y0 = __ldg(j.y + h0), z0 = __ldg(j.z + h0);
            if (!tube_pass(x0, y0, z0, mx, my, c)) continue;
            for (int32_t h1 = o[1]; h1 < o[2] && !found; ++h1) {
                const float x1 = __ldg(j.x + h1), y1 = __ldg(j.y + h1), z1 = __ldg(j.z + h1);
                if (!tube_pass(x1, y1, z1, mx, my, c)) continue;
                for (int32_t h2 = o[2]; h2 < o[3] && !found; ++h2) {
                    const float xs[3] = {x0, x1, __ldg(j.x + h2)};
                    const float ys[3] = {y0, y1, __ldg(j.y + h2)};
                    const float zs[3] = {z0, z1, __ldg(j.z + h2)};
                    if (!tube_pass(xs[2], ys[2], zs[2], mx, my, c)) continue;
                    float fx, fy;
                    found = fit_pass(xs, ys, zs, c, fx, fy) && chain_pass(xs, ys, zs, mx, my, c);
                    if (kStream && found) {
                        float pmin, pmax;
                        coincident3(__ldg(j.t + h0), __ldg(j.t + h1), __ldg(j.t + h2), j.dt, pmin, pmax);
                        found = partner_coincident(pmin, pmax, Tt, j.dt);
                    }
                }
            }
        }
        if (!found) return false;
    }
    return true;
}

// Shared scratch of the unpruned search of one event (from the caller).
struct GenShared {
    int32_t* soff;  // [3 * kMaxStations + 1] the event's offsets
    int* s_count;
    int* s_cand;
    int* s_bad;
    unsigned long long* s_pool;
};

constexpr int kGenThreads = 256;  // block size of the unpruned search (both callers)

// distinct_hits on the unpruned path: a second pass over the trigger
// station writes the packed hits of the event's candidates (passing
// triplets; in CHAIN mode those with a compatible triplet in every other
// station) to out[0, cap), ranked by the block-shared counter.
__device__ void generic_candidates(const Job& j, const int32_t* soff, const Cuts& c, unsigned long long* out, int cap,
                                   int* s_rank) {
    const int32_t* o = soff + 3 * j.trig;
    const bool chain = j.mode == 1 && j.S > 1;
    const int64_t n0 = o[1] - o[0], n1 = o[2] - o[1], n2 = o[3] - o[2];
    const int64_t npairs = n0 * n1;
    for (int64_t p = threadIdx.x; p < npairs; p += blockDim.x) {
        const int64_t i = p / n1, jx = p - i * n1;
        const GHit hi = ghit(j, o[0] + i), hj = ghit(j, o[1] + jx);
        if (!hi.p.live || !hj.p.live) continue;
        if (!hi.p.wild && !hj.p.wild && !pair_ok(hi.p.sx, hi.p.sy, hj.p.sx, hj.p.sy, __fadd_rn(hi.p.b, hj.p.b)))
            continue;
        for (int64_t k = 0; k < n2; ++k) {
            const GHit hk = ghit(j, o[2] + k);
            if (!hk.p.live) continue;
            if (!hk.p.wild) {
                if (!hi.p.wild && !pair_ok(hi.p.sx, hi.p.sy, hk.p.sx, hk.p.sy, __fadd_rn(hi.p.b, hk.p.b))) continue;
                if (!hj.p.wild && !pair_ok(hj.p.sx, hj.p.sy, hk.p.sx, hk.p.sy, __fadd_rn(hj.p.b, hk.p.b))) continue;
            }
            const float xs[3] = {hi.x, hj.x, hk.x}, ys[3] = {hi.y, hj.y, hk.y}, zs[3] = {hi.z, hj.z, hk.z};
            float mx, my;
            if (!fit_pass(xs, ys, zs, c, mx, my)) continue;
            if (chain && !road_global(j, soff, c, mx, my, make_float2(0.f, 0.f))) continue;  // (no streams here)
            const int r = atomicAdd(s_rank, 1);
            if (r < cap) out[r] = pack_ijk((int)i, (int)jx, (int)k);
        }
    }
}

// The unpruned search of one event by one block: any size, any coordinates
// (pruning only where the per-hit bound is finite).  Counting pass: unit
// counts, track count and recorded entries; emit pass: rows.  All threads of
// the block call it.
template <bool EMIT>
__device__ void generic_event(const Job& j, int64_t e, const GenShared& g) {
    const Cuts c{j.cx, j.cy, j.K};
    const int S = j.S, S3 = 3 * S;
    const bool chain = j.mode == 1 && S > 1;
    const int nproc = j.mode == 1 ? S : 1;
    int32_t* soff = g.soff;
    __syncthreads();  // earlier users of the shared scratch are done
    for (int i = threadIdx.x; i <= S3; i += blockDim.x) soff[i] = j.off[e * S3 + i];
    if (threadIdx.x == 0) *g.s_cand = 0;
    __syncthreads();
    int trig_count = 0;
    bool bad_event = false;
    for (int si = 0; si < nproc && !bad_event; ++si) {
        const int s = station_of(si, j.trig);
        const int64_t u = e * S + s;
        const int32_t* o = soff + 3 * s;
        if (EMIT && j.unit_counts[u] == 0) continue;
        if (threadIdx.x == 0) {
            *g.s_count = 0;
            *g.s_bad = 0;
        }
        __syncthreads();
        if (!EMIT) {
            for (int32_t h = o[0] + threadIdx.x; h < o[3]; h += blockDim.x)
                if (__ldg(j.z + h) <= 0.0f) *g.s_bad = 1;
            __syncthreads();
            if (*g.s_bad) {
                if (threadIdx.x == 0) {
                    atomicOr(&j.ctrl->status, kStInvalid);
                    j.ev_class[e] = kClsInvalid;
                }
                bad_event = true;
                break;
            }
        }
        const int64_t n0 = o[1] - o[0], n1 = o[2] - o[1], n2 = o[3] - o[2];
        const int64_t npairs = n0 * n1;
        int32_t* rows = EMIT ? j.triplets + 3 * j.trip_off[u] : nullptr;
        const int ulimit = EMIT ? j.unit_counts[u] : 0;
        int local = 0;
        const bool collect = !EMIT && chain && s == j.trig;
        for (int64_t p = threadIdx.x; p < npairs; p += blockDim.x) {
            const int64_t i = p / n1, jx = p - i * n1;
            const GHit hi = ghit(j, o[0] + i), hj = ghit(j, o[1] + jx);
            if (!hi.p.live || !hj.p.live) continue;
            if (!hi.p.wild && !hj.p.wild && !pair_ok(hi.p.sx, hi.p.sy, hj.p.sx, hj.p.sy, __fadd_rn(hi.p.b, hj.p.b)))
                continue;
            for (int64_t k = 0; k < n2; ++k) {
                const GHit hk = ghit(j, o[2] + k);
                if (!hk.p.live) continue;
                if (!hk.p.wild) {
                    if (!hi.p.wild && !pair_ok(hi.p.sx, hi.p.sy, hk.p.sx, hk.p.sy, __fadd_rn(hi.p.b, hk.p.b)))
                        continue;
                    if (!hj.p.wild && !pair_ok(hj.p.sx, hj.p.sy, hk.p.sx, hk.p.sy, __fadd_rn(hj.p.b, hk.p.b)))
                        continue;
                }
                const float xs[3] = {hi.x, hj.x, hk.x}, ys[3] = {hi.y, hj.y, hk.y}, zs[3] = {hi.z, hj.z, hk.z};
                float mx, my;
                if (!fit_pass(xs, ys, zs, c, mx, my)) continue;
                float2 Tt = make_float2(0.f, 0.f);
                if constexpr (kStream) {  // coincident and owned by this window
                    const bool co = coincident3(__ldg(j.t + o[0] + i), __ldg(j.t + o[1] + jx), __ldg(j.t + o[2] + k), j.dt,
                                                Tt.x, Tt.y);
                    if (!(co && Tt.x >= __ldg(j.wb + e) && Tt.x < __ldg(j.wb + e + 1))) continue;
                }
                ++local;
                if (!EMIT && j.tscr) {
                    const int rk = atomicAdd(g.s_count, 1);
                    if (i >= kPackLimit || jx >= kPackLimit || k >= kPackLimit) {
                        atomicOr(&j.ctrl->status, kStNoScratch);
                    } else {
                        const unsigned long long b = atomicAdd(&j.ctrl->scratch_n, 1ull);
                        if (b < (unsigned long long)j.tscr_cap) {
                            TripEntry te;
                            te.unit = (int32_t)u;
                            te.rank = rk;
                            te.ijk = (unsigned long long)i | ((unsigned long long)jx << 20) |
                                     ((unsigned long long)k << 40) | ((unsigned long long)kClsGeneric << kTagShift);
                            j.tscr[b] = te;
                        }
                    }
                }
                if (EMIT) {
                    const int pos = atomicAdd(g.s_count, 1);
                    if (pos < ulimit &&  // never past the unit's rows
                        JPSI_IN(j.ctrl, (rows - j.triplets) / 3 + pos < j.trip_cap)) {
                        int32_t* r = rows + 3 * (int64_t)pos;
                        r[0] = (int32_t)i;
                        r[1] = (int32_t)jx;
                        r[2] = (int32_t)k;
                    }
                }
                if (collect && road_global(j, soff, c, mx, my, Tt)) atomicAdd(g.s_cand, 1);
            }
        }
        if (!EMIT && !j.tscr && local) atomicAdd(g.s_count, local);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (EMIT) {
                if (*g.s_count != j.unit_counts[u]) atomicOr(&j.ctrl->status, kStEmitMismatch);
            } else {
                j.unit_counts[u] = *g.s_count;
            }
        }
        if (s == j.trig) trig_count = *g.s_count;
        __syncthreads();
    }
    if (!EMIT && !bad_event && threadIdx.x == 0) {
        if (j.mode == 0)
            for (int s = 0; s < S; ++s)
                if (s != j.trig) j.unit_counts[e * S + s] = 0;
        j.track_counts[e] = chain ? *g.s_cand : trig_count;
    }
    if (!EMIT && !bad_event && j.distinct) {  // block-uniform
        const int nc = chain ? *g.s_cand : trig_count;
        bool f = false;
        if (nc >= 2) {
            __syncthreads();
            if (threadIdx.x == 0) {
                *g.s_pool = atomicAdd(&j.ctrl->tpool_n, (unsigned long long)nc);
                *g.s_count = 0;
            }
            __syncthreads();
            const unsigned long long pb = *g.s_pool;
            if (pb + (unsigned long long)nc <= (unsigned long long)j.tpool_cap) {
                generic_candidates(j, soff, c, j.tpool_ijk + pb, nc, g.s_count);
                __syncthreads();
                f = block_disjoint_pair<kGenThreads>(j.tpool_ijk + pb, nullptr, nc, g.s_bad);
            } else if (threadIdx.x == 0) {
                atomicOr(&j.ctrl->status, kStNoPool);
            }
        }
        if (threadIdx.x == 0) j.dpair[e] = f;
    }
    __syncthreads();
}

// Persistent blocks take the events of the unpruned list.
template <bool EMIT>
__global__ void __launch_bounds__(kGenThreads) k_generic(const __grid_constant__ Job j) {
    __shared__ int32_t soff[3 * kMaxStations + 1];
    __shared__ int s_gi, s_count, s_cand, s_bad;
    __shared__ unsigned long long s_pool;
    const int n_gen = *(volatile int32_t*)&j.ctrl->n_generic, g0 = *(volatile int32_t*)&j.ctrl->g_begin;
    for (;;) {
        if (threadIdx.x == 0) s_gi = g0 + (int)atomicAdd(&j.ctrl->work[EMIT ? 7 : 3], 1ull);
        __syncthreads();
        const int gi = s_gi;
        if (gi >= n_gen) break;
        const int64_t e = j.glist[gi];
        if (!EMIT || j.ev_class[e] == kClsGeneric)
            generic_event<EMIT>(j, e, GenShared{soff, &s_count, &s_cand, &s_bad, &s_pool});
        __syncthreads();
    }
}

// ------------------------------------------------- one-launch form, blocks

// The one-launch form (jpsi_run_plain) has no event lists, queues, sort,
// pool hand-off or graphs: a static grid of one warp per event (k_light with
// Job::plain), then a static grid of one block per event (below).  A block
// whose event the warp finished returns at once; the others run the whole
// event here: every station on the block tile, or the unpruned search when
// the event does not fit the tile or has extreme coordinates.
constexpr int kPlainTCap = 128;  // trigger slopes kept in shared memory (more: the pool)

struct PlainSmem {
    HeavySmem h;
    float2 T[kPlainTCap];
    uint8_t alive[kPlainTCap];
};

// One block-tile event of the one-launch form.  Returns true when the event
// must go on to the unpruned search (its class is then kClsGeneric).
template <bool EMIT>
__device__ bool plain_block_event(const Job& j, PlainSmem& ps, int64_t e) {
    HeavySmem& sm = ps.h;
    const int tid = threadIdx.x, lane = tid & 31;
    const int S = j.S;
    const bool chain = j.mode == 1 && S > 1;
    const int nproc = j.mode == 1 ? S : 1;
    const Cuts c{j.cx, j.cy, j.K};
    load_event_offsets(j, sm, e);
    if (EMIT) {
        for (int si = 0; si < nproc; ++si) {
            const int s = station_of(si, j.trig);
            if (j.unit_counts[e * S + s] == 0) continue;
            TSink ts{false, nullptr, 0, nullptr, 0};
            int cnt = 0;
            heavy_unit<true>(j, sm, c, kGiPlain, e, s, ts, nullptr, nullptr, 0, cnt,
                             si + 1 < nproc ? station_of(si + 1, j.trig) : -1);
            __syncthreads();
        }
        return false;
    }
    bool fits = true;
    for (int si = 0; si < nproc; ++si) {
        const int32_t* o = sm.off + 3 * station_of(si, j.trig);
        if (o[1] - o[0] > kHLayerCap || o[2] - o[1] > kHLayerCap || o[3] - o[2] > kHLayerCap || o[3] - o[0] > kHHCap)
            fits = false;
    }
    if (!fits) {
        if (tid == 0) j.ev_class[e] = kClsGeneric;
        return true;
    }
    float2* T = ps.T;
    uint8_t* alive = ps.alive;
    unsigned long long* ijk = nullptr;  // distinct_hits: the candidates' packed hits (in the pool)
    float2* tt = nullptr;               // free-streaming windows: the slopes' times (in the pool)
    int trig_count = 0, nT = 0;
    for (int si = 0; si < nproc; ++si) {
        const int s = station_of(si, j.trig);
        if (tid == 0) sm.s_nT = 0;
        __syncthreads();
        TSink ts{(chain || j.distinct) && si == 0, T, kPlainTCap, &sm.s_nT, 0};
        int cnt = 0;
        const int sn = si + 1 < nproc ? station_of(si + 1, j.trig) : -1;
        if (!heavy_unit<false>(j, sm, c, kGiPlain, e, s, ts, T, alive, si == 0 ? 0 : nT, cnt, sn, tt)) {
            __syncthreads();
            return j.ev_class[e] == kClsGeneric;
        }
        __syncthreads();
        if (si > 0) continue;
        trig_count = cnt;
        if (!chain && !j.distinct) break;
        nT = sm.s_nT;
        if (nT > kPlainTCap || (j.distinct && nT >= 2) || (kStream && chain && nT > 0)) {
            // more slopes than the block keeps, or (distinct_hits) the
            // candidates' hits or (free-streaming windows) the slopes' times
            // wanted: room in the batch's pool, and the trigger station once
            // more (same count, nothing recorded)
            if (tid == 0) sm.s_pool = atomicAdd(&j.ctrl->tpool_n, (unsigned long long)nT);
            __syncthreads();
            const unsigned long long pb = sm.s_pool;
            if (pb + (unsigned long long)nT > (unsigned long long)j.tpool_cap) {
                if (tid == 0) j.ev_class[e] = kClsGeneric;
                return true;
            }
            T = j.tpool + pb;
            alive = j.tpool_alive + pb;
            if (j.distinct) ijk = j.tpool_ijk + pb;
            if constexpr (kStream) tt = reinterpret_cast<float2*>(j.tpool_ijk) + pb;
            if (tid == 0) sm.s_nT = 0;
            __syncthreads();
            TSink ts2{true, T, nT, &sm.s_nT, 0};
            ts2.norec = true;
            ts2.ijk = ijk;
            ts2.tt = tt;
            if (!heavy_unit<false>(j, sm, c, kGiPlain, e, s, ts2, nullptr, nullptr, 0, cnt)) {
                __syncthreads();
                return j.ev_class[e] == kClsGeneric;
            }
            __syncthreads();
        }
        if (!chain) {  // PAPER with distinct_hits: every passing trigger triplet is a candidate
            const bool f = nT >= 2 && block_disjoint_pair<kHThreads>(ijk, nullptr, nT, &sm.s_hx);
            if (tid == 0) j.dpair[e] = f;
            break;
        }
        for (int i = tid; i < nT; i += kHThreads) alive[i] = 1;
        __syncthreads();
    }
    int tc = trig_count;
    if (chain) {
        if (tid == 0) sm.s_cand = 0;
        __syncthreads();
        int a = 0;
        for (int ti = tid; ti < nT; ti += kHThreads) a += alive[ti];
        a = __reduce_add_sync(kFull, a);
        if (lane == 0 && a) atomicAdd(&sm.s_cand, a);
        __syncthreads();
        tc = sm.s_cand;
        if (j.distinct) {
            const bool f = nT >= 2 && block_disjoint_pair<kHThreads>(ijk, alive, nT, &sm.s_hx);
            if (tid == 0) j.dpair[e] = f;
        }
    }
    if (tid == 0) {
        if (j.mode == 0)
            for (int s = 0; s < S; ++s)
                if (s != j.trig) j.unit_counts[e * S + s] = 0;
        j.track_counts[e] = tc;
    }
    return false;
}

template <bool EMIT>
__global__ void __launch_bounds__(kHThreads, 3) k_plain_block(const __grid_constant__ Job j) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PlainSmem& ps = *reinterpret_cast<PlainSmem*>(smem_raw);
    const int64_t e = j.ev_begin + blockIdx.x;
    if (e >= j.ev_begin + j.ev_count) return;
    const uint8_t cls = j.ev_class[e];
    bool generic = cls == kClsGeneric;
    if (cls == kClsHeavy) generic = plain_block_event<EMIT>(j, ps, e);
    if (generic) generic_event<EMIT>(j, e, GenShared{ps.h.off, &ps.h.s_rank, &ps.h.s_cand, &ps.h.s_next, &ps.h.s_pool});
}

// -------------------------------------------------------- accept bits

__global__ void k_accept(const __grid_constant__ Job j) {
    if (!j.accept_bits) return;
    const int64_t nwords = (j.n_events + 31) / 32;
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); w < nwords; w += wstride) {
        const int64_t e = w * 32 + lane;
        // distinct_hits with min_candidates 2: two candidates sharing no hit
        const bool v = e < j.n_events && (j.distinct && j.minc == 2 ? j.dpair[e] != 0 : j.track_counts[e] >= j.minc);
        const unsigned bits = __ballot_sync(kFull, v);
        if (lane == 0) j.accept_bits[w] = bits;
    }
}

// --------------------------------------------------------------- scan

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t& total) {
    // sh: kScanThreads/32 + 1 entries
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t o = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += o;
    }
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int64_t s = lane < nw ? sh[lane] : 0;
        int64_t si = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t o = __shfl_up_sync(kFull, si, d);
            if (lane >= d) si += o;
        }
        if (lane < nw) sh[lane] = si - s;
        if (lane == 31) sh[32] = si;
    }
    __syncthreads();
    const int64_t r = sh[w] + incl - v;
    total = sh[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const __grid_constant__ Job j) {
    __shared__ int64_t sh[33];
    const int64_t n = j.n_events * j.S;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int64_t v = 0;
        const int64_t b = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q)
            if (b + q < n) v += j.unit_counts[b + q];
        int64_t total;
        block_excl_scan(v, sh, total);
        if (threadIdx.x == 0) j.block_sums[tile] = total;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(const __grid_constant__ Job j) {
    __shared__ int64_t sh[33];
    const int64_t n = j.n_events * j.S;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += kScanThreads) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = i < ntiles ? j.block_sums[i] : 0;
        int64_t total;
        const int64_t ex = block_excl_scan(v, sh, total);
        if (i < ntiles) j.block_sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) {
        j.trip_off[n] = carry;
        j.ctrl->trip_total = carry;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const __grid_constant__ Job j) {
    __shared__ int64_t sh[33];
    const int64_t n = j.n_events * j.S;
    const int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t b = tile * kScanTile + (int64_t)threadIdx.x * kScanItems;
        int32_t v[kScanItems];
        int64_t sum = 0;
#pragma unroll
        for (int q = 0; q < kScanItems; ++q) {
            v[q] = b + q < n ? j.unit_counts[b + q] : 0;
            sum += v[q];
        }
        int64_t total;
        int64_t run = block_excl_scan(sum, sh, total) + j.block_sums[tile];
#pragma unroll
        for (int q = 0; q < kScanItems; ++q)
            if (b + q < n) {
                j.trip_off[b + q] = run;
                run += v[q];
            }
    }
}

// ------------------------------------------------------ triplet scatter

// Moves each recorded triplet to its row trip_off[unit] + rank.  Entries
// written by a path that did not keep the event (it moved on to the next
// path part-way) are dropped; the final path recorded the event again.
__global__ void k_scatter(const __grid_constant__ Job j) {
    const unsigned long long n = j.ctrl->scratch_n;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        const TripEntry te = j.tscr[q];
        const int64_t e = te.unit / j.S;
        const unsigned tag = (unsigned)((te.ijk >> kTagShift) & 7u);
        if (j.ev_class[e] != tag) continue;
        const int64_t row = j.trip_off[te.unit] + te.rank;
        if (!JPSI_IN(j.ctrl, row >= 0 && row < j.trip_cap)) continue;
        int32_t* r = j.triplets + 3 * row;
        r[0] = (int32_t)(te.ijk & 0xfffffu);
        r[1] = (int32_t)((te.ijk >> 20) & 0xfffffu);
        r[2] = (int32_t)((te.ijk >> 40) & 0xfffffu);
    }
}

// ------------------------------------------------- per-layer z geometry

// Per-hit z from a detector geometry table (every hit of layer l of station s
// at z_layer[s*3 + l]) for events [ev0, ev1): blocks take events in turn;
// each hit finds its layer among the event's 3S+1 offsets by binary search.
// Writes stay inside [0, n_hits) whatever the offsets hold (malformed offsets
// fail the selection afterwards), and the table index stays below 3S.
__global__ void __launch_bounds__(256) k_expand_z(const int32_t* __restrict__ off,
                                                  const float* __restrict__ z_layer, float* __restrict__ z,
                                                  int64_t ev0, int64_t ev1, int S, int64_t n_hits) {
    __shared__ int32_t so[3 * kMaxStations + 1];
    const int S3 = 3 * S;
    for (int64_t e = ev0 + blockIdx.x; e < ev1; e += gridDim.x) {
        __syncthreads();
        for (int i = threadIdx.x; i <= S3; i += blockDim.x) so[i] = off[e * S3 + i];
        __syncthreads();
        const int64_t h0 = max((int64_t)so[0], (int64_t)0), h1 = min((int64_t)so[S3], n_hits);
        for (int64_t h = h0 + threadIdx.x; h < h1; h += blockDim.x) {
            int q = 0;  // last layer q < S3 with so[q] <= h
#pragma unroll
            for (int step = 32; step > 0; step >>= 1)
                if (q + step < S3 && so[q + step] <= h) q += step;
            z[h] = z_layer[q];
        }
    }
}

// ------------------------------------------------------------ launchers

size_t light_smem_bytes(int wpb) { return (size_t)wpb * sizeof(WarpTile<SmallCfg>); }
static size_t medium_smem_bytes() { return sizeof(MediumSmem); }
size_t heavy_smem_bytes() { return sizeof(HeavySmem); }
static size_t plain_smem_bytes() { return sizeof(PlainSmem); }

// Kernel attributes are per device: set once for each device a context or a
// call runs on (serving threads may get here at the same time).
static std::mutex g_attr_mu;
static uint64_t g_attr_done = 0;  // bit d: device d done (devices >= 64: every call)

static cudaError_t ensure_attrs() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    const uint64_t bit = dev < 64 ? (uint64_t)1 << dev : 0;
    if (g_attr_done & bit) return cudaSuccess;
    const int maxw = 8;
    e = cudaFuncSetAttribute(k_light<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)light_smem_bytes(maxw));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_light<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)light_smem_bytes(maxw));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_medium<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)medium_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_medium<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)medium_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)heavy_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_heavy_units<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)heavy_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_heavy_units<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)heavy_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_plain_block<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)plain_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_plain_block<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)plain_smem_bytes());
    if (e == cudaSuccess) g_attr_done |= bit;
    return e;
}

int light_max_blocks_per_sm(int wpb) {
    if (ensure_attrs() != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_light<false>, wpb * 32, light_smem_bytes(wpb)) !=
        cudaSuccess)
        return 0;
    return nb;
}

int heavy_max_blocks_per_sm() {
    if (ensure_attrs() != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_heavy, kHThreads, heavy_smem_bytes()) !=
        cudaSuccess)
        return 0;
    return nb;
}

int medium_max_blocks_per_sm() {
    if (ensure_attrs() != cudaSuccess) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_medium<false>, MedBCfg::THREADS, medium_smem_bytes()) !=
        cudaSuccess)
        return 0;
    return nb;
}

int generic_max_blocks_per_sm(int threads) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_generic<false>, threads, 0) != cudaSuccess) return 0;
    return nb;
}

const void* light_count_kernel_ptr() { return (const void*)k_light<false>; }

// Kernels take the job by value (a __grid_constant__ parameter), so every
// field read is a constant-bank operand rather than a load.
cudaError_t launch_light_count(const Job& job, int64_t n_events, const LaunchCfg& lc, bool persistent,
                               cudaStream_t st) {
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    const int wpb = lc.light_wpb;
    const size_t smem = light_smem_bytes(wpb);
    Job j = job;
    j.persistent = persistent ? 1 : 0;
    const int64_t nb = persistent ? lc.light_blocks : std::max<int64_t>((n_events + wpb - 1) / wpb, 1);
    k_light<false><<<(unsigned)nb, wpb * 32, smem, st>>>(j);
    return cudaGetLastError();
}

cudaError_t launch_count_lists(const Job& j, const LaunchCfg& lc, cudaStream_t st) {
    k_medium<false><<<lc.medium_blocks, MedBCfg::THREADS, medium_smem_bytes(), st>>>(j);
    k_sort_heavy<<<1, 1024, 0, st>>>(j);
    k_heavy<<<lc.heavy_blocks, kHThreads, heavy_smem_bytes(), st>>>(j);
    k_heavy_units<false><<<lc.heavy_blocks, kHThreads, heavy_smem_bytes(), st>>>(j);
    k_heavy_final<<<lc.scan_blocks, 256, 0, st>>>(j);
    k_generic<false><<<lc.generic_blocks, kGenThreads, 0, st>>>(j);
    return cudaGetLastError();
}

cudaError_t launch_count_tail(const Job& j, const LaunchCfg& lc, cudaStream_t st) {
    k_accept<<<lc.scan_blocks, 256, 0, st>>>(j);
    k_scan_reduce<<<lc.scan_blocks, kScanThreads, 0, st>>>(j);
    k_scan_top<<<1, kScanThreads, 0, st>>>(j);
    k_scan_down<<<lc.scan_blocks, kScanThreads, 0, st>>>(j);
    return cudaGetLastError();
}

cudaError_t launch_count_rest(const Job& j, const LaunchCfg& lc, cudaStream_t st) {
    const cudaError_t e = launch_count_lists(j, lc, st);
    return e != cudaSuccess ? e : launch_count_tail(j, lc, st);
}

cudaError_t launch_expand_z(const int32_t* off, const float* z_layer, float* z, int64_t ev0, int64_t ev1, int S,
                            int64_t n_hits, int n_sm, cudaStream_t st) {
    if (ev1 <= ev0) return cudaSuccess;
    const int64_t grid = std::min<int64_t>(ev1 - ev0, (int64_t)n_sm * 8);
    k_expand_z<<<(unsigned)grid, 256, 0, st>>>(off, z_layer, z, ev0, ev1, S, n_hits);
    return cudaGetLastError();
}

// One-launch form: the static warp grid, then the static block grid and the
// tail (accept bits, scan); its emit phase is the same two grids.
static cudaError_t launch_plain_grids(const Job& job, bool emit, bool warps, bool blocks, const LaunchCfg& lc,
                                      cudaStream_t st) {
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    Job j = job;
    j.persistent = 0;
    j.plain = 1;
    const int wpb = lc.light_wpb;
    const int64_t n = j.ev_count;
    if (warps) {
        const int64_t nb = std::max<int64_t>((n + wpb - 1) / wpb, 1);
        if (emit)
            k_light<true><<<(unsigned)nb, wpb * 32, light_smem_bytes(wpb), st>>>(j);
        else
            k_light<false><<<(unsigned)nb, wpb * 32, light_smem_bytes(wpb), st>>>(j);
    }
    if (blocks) {
        const unsigned nb = (unsigned)std::max<int64_t>(n, 1);
        if (emit)
            k_plain_block<true><<<nb, kHThreads, plain_smem_bytes(), st>>>(j);
        else
            k_plain_block<false><<<nb, kHThreads, plain_smem_bytes(), st>>>(j);
    }
    return cudaGetLastError();
}

cudaError_t launch_plain_light(const Job& j, const LaunchCfg& lc, cudaStream_t st) {
    return launch_plain_grids(j, false, true, false, lc, st);
}

cudaError_t launch_plain_rest(const Job& j, const LaunchCfg& lc, cudaStream_t st) {
    const cudaError_t e = launch_plain_grids(j, false, false, true, lc, st);
    return e != cudaSuccess ? e : launch_count_tail(j, lc, st);
}

cudaError_t launch_plain_emit(const Job& j, const LaunchCfg& lc, cudaStream_t st) {
    return launch_plain_grids(j, true, true, true, lc, st);
}

cudaError_t launch_scatter(const Job& j, const LaunchCfg& lc, cudaStream_t st) {
    k_scatter<<<lc.scan_blocks, 256, 0, st>>>(j);
    return cudaGetLastError();
}

cudaError_t launch_emit_phase(const Job& job, int64_t n_events, const LaunchCfg& lc, bool persistent,
                              cudaStream_t st) {
    cudaError_t e = ensure_attrs();
    if (e != cudaSuccess) return e;
    const int wpb = lc.light_wpb;
    const size_t smem = light_smem_bytes(wpb);
    Job j = job;
    j.persistent = persistent ? 1 : 0;
    const int64_t nb = persistent ? lc.light_blocks : std::max<int64_t>((n_events + wpb - 1) / wpb, 1);
    k_light<true><<<(unsigned)nb, wpb * 32, smem, st>>>(j);
    k_medium<true><<<lc.medium_blocks, MedBCfg::THREADS, medium_smem_bytes(), st>>>(j);
    k_heavy_units<true><<<lc.heavy_blocks, kHThreads, heavy_smem_bytes(), st>>>(j);
    k_generic<true><<<lc.generic_blocks, kGenThreads, 0, st>>>(j);
    return cudaGetLastError();
}

#if JPSI_STREAM
// ------------------------------------------- free-streaming event building
//
// A timeslice's hits are grouped by (station, layer), each group sorted by
// time.  Window k = [b_k, b_k+1) becomes event k of a window batch: group g
// of event k holds the group-g hits whose times lie in the window's range
// (the trigger station: [b_k, fl32(b_k+1 + dt)], which holds every triplet
// owned by the window; the other stations of CHAIN mode from a margin below
// b_k - dt to the same end, which holds every partner that can be coincident
// with such a triplet).  The selection kernels of this build then apply the
// time tests themselves; the rows they write index the window batch and are
// moved back to timeslice group indices at the end.

// Last group q < S3 with so[q] <= h (so: the 3S+1 offsets, non-decreasing).
__device__ __forceinline__ int group_of(const int32_t* so, int S3, int64_t h) {
    int q = 0;
#pragma unroll
    for (int step = 32; step > 0; step >>= 1)
        if (q + step < S3 && so[q + step] <= h) q += step;
    return q;
}

// First index in [lo, hi) whose time is >= v (> v with STRICT); stays in
// [lo, hi] whatever the times hold.
template <bool STRICT>
__device__ __forceinline__ int64_t t_search(const float* __restrict__ t, int64_t lo, int64_t hi, float v) {
    while (lo < hi) {
        const int64_t m = lo + ((hi - lo) >> 1);
        const float tm = __ldg(t + m);
        if (STRICT ? tm <= v : tm < v)
            lo = m + 1;
        else
            hi = m;
    }
    return lo;
}

// The timeslice's own checks: times sorted within each group and not NaN,
// z > 0 for every hit of a station the mode reads, window bounds finite and
// strictly increasing.  Sets kStInvalid.
__global__ void __launch_bounds__(256) k_win_check(const __grid_constant__ WinJob w) {
    __shared__ int32_t so[3 * kMaxStations + 1];
    const int S3 = 3 * w.S;
    for (int i = threadIdx.x; i <= S3; i += blockDim.x) so[i] = w.off[i];
    __syncthreads();
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x, g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t h = g0; h < w.n_hits; h += stride) {
        const int g = group_of(so, S3, h);
        const float th = __ldg(w.t + h);
        if (isnan(th) || (h > so[g] && !(th >= __ldg(w.t + h - 1)))) bad = true;
        if (w.z && (w.chain || g / 3 == w.trig) && __ldg(w.z + h) <= 0.f) bad = true;
    }
    for (int64_t k = g0; w.K > 0 && k <= w.K; k += stride) {  // no windows: bounds may be null
        const float b = __ldg(w.wb + k);
        if (!isfinite(b) || (k > 0 && !(b > __ldg(w.wb + k - 1)))) bad = true;
    }
    if (!w.z && blockIdx.x == 0 && threadIdx.x < S3) {
        const int g = threadIdx.x;
        if (so[g + 1] > so[g] && (w.chain || g / 3 == w.trig) && __ldg(w.z_layer + g) <= 0.f) bad = true;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&w.ctrl->status, kStInvalid);
}

// Each (window, group) range: first hit and size.
__global__ void __launch_bounds__(256) k_win_ranges(const __grid_constant__ WinJob w) {
    __shared__ int32_t so[3 * kMaxStations + 1];
    const int S3 = 3 * w.S;
    for (int i = threadIdx.x; i <= S3; i += blockDim.x) so[i] = w.off[i];
    __syncthreads();
    const int64_t n = w.K * S3, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
        const int64_t k = q / S3;
        const int g = (int)(q - k * S3), s = g / 3;
        int64_t lo = so[g], hi = so[g];
        if (s == w.trig || w.chain) {
            const float b0 = __ldg(w.wb + k), end = __fadd_rn(__ldg(w.wb + k + 1), w.dt);
            float from = b0;
            if (s != w.trig) {
                // a partner's hits are no earlier than (latest trigger-triplet
                // time) - dt, less one rounding of the sum: a margin of 1e-6
                // relative covers it, the exact tests decide
                double lod = (double)b0 - (double)w.dt;
                lod -= 1e-6 * (fabs((double)b0) + (double)w.dt) + 1e-30;
                from = nextafterf(__double2float_rn(lod), -INFINITY);
            }
            lo = t_search<false>(w.t, so[g], so[g + 1], from);
            hi = t_search<true>(w.t, lo, so[g + 1], end);
        }
        w.wlo[q] = (int32_t)lo;
        w.wcnt[q] = (int32_t)(hi - lo);
    }
}

// The window batch: its offsets (from the scan) and its hits, one warp per
// (window, group) range.
__global__ void __launch_bounds__(256) k_win_gather(const __grid_constant__ WinJob w) {
    const int S3 = 3 * w.S;
    const int64_t n = w.K * S3;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < n; q += nwarps) {
        const int64_t dst = w.woff[q];
        const int64_t src = w.wlo[q];
        const int cnt = w.wcnt[q];
        if (lane == 0) w.off_out[q] = (int32_t)dst;
        if (cnt == 0) continue;  // (a timeslice without hits may come without z and z_layer)
        const float zl = w.z ? 0.f : __ldg(w.z_layer + (int)(q % S3));
        for (int i = lane; i < cnt; i += 32) {
            w.xo[dst + i] = __ldg(w.x + src + i);
            w.yo[dst + i] = __ldg(w.y + src + i);
            w.zo[dst + i] = w.z ? __ldg(w.z + src + i) : zl;
            w.to[dst + i] = __ldg(w.t + src + i);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) w.off_out[n] = (int32_t)w.woff[n];
}

// Triplet rows of unit (k, s): window-batch layer indices plus the start of
// the window's range in the timeslice group, less the group's start.
__global__ void __launch_bounds__(256) k_win_rows(const __grid_constant__ WinJob w, const int64_t* trip_off,
                                                  int32_t* tr) {
    const int64_t nu = w.K * w.S;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < nu; u += nwarps) {
        const int64_t a = trip_off[u], b = trip_off[u + 1];
        if (a == b) continue;
        const int64_t k = u / w.S;
        const int s = (int)(u - k * w.S);
        const int64_t q = k * 3 * w.S + 3 * s;
        const int32_t d0 = w.wlo[q] - __ldg(w.off + 3 * s), d1 = w.wlo[q + 1] - __ldg(w.off + 3 * s + 1),
                      d2 = w.wlo[q + 2] - __ldg(w.off + 3 * s + 2);
        for (int64_t r = a + lane; r < b; r += 32) {
            tr[3 * r] += d0;
            tr[3 * r + 1] += d1;
            tr[3 * r + 2] += d2;
        }
    }
}

static unsigned win_grid(int64_t threads, int n_sm) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, (int64_t)n_sm * 8));
}

cudaError_t launch_window_ranges(const WinJob& w, cudaStream_t st) {
    const int64_t n = w.K * 3 * w.S;
    k_win_check<<<win_grid(std::max(w.n_hits, w.K + 1), w.n_sm), 256, 0, st>>>(w);
    k_win_ranges<<<win_grid(n, w.n_sm), 256, 0, st>>>(w);
    // the sizes' scan, with the scan kernels of the selection reading a job
    // whose "units" are the (window, group) ranges
    Job j{};
    j.n_events = w.K;
    j.S = 3 * w.S;
    j.unit_counts = w.wcnt;
    j.block_sums = w.block_sums;
    j.trip_off = w.woff;
    j.ctrl = w.ctrl;
    k_scan_reduce<<<w.n_sm * 2, kScanThreads, 0, st>>>(j);
    k_scan_top<<<1, kScanThreads, 0, st>>>(j);
    k_scan_down<<<w.n_sm * 2, kScanThreads, 0, st>>>(j);
    return cudaGetLastError();
}

cudaError_t launch_window_gather(const WinJob& w, cudaStream_t st) {
    k_win_gather<<<win_grid(w.K * 3 * w.S * 32, w.n_sm), 256, 0, st>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_window_rows(const WinJob& w, const int64_t* trip_off, int32_t* triplets, cudaStream_t st) {
    k_win_rows<<<win_grid(w.K * w.S * 32, w.n_sm), 256, 0, st>>>(w, trip_off, triplets);
    return cudaGetLastError();
}
#endif  // JPSI_STREAM

}  // namespace basek / streamk
}  // namespace jpsi

#if !JPSI_STREAM
// ======================================================================
// Allocation-free counting entry point (jpsi_select_noalloc, include/jpsi.h).
//
// For callers that may not allocate device memory at run time.  Its only
// scratch is the file-scope array below: the control block, one class byte
// per event and the three per-event lists of the warp kernel, for at most
// kNoAllocMaxEvents events (the job itself is a kernel parameter).  Every GPU that loads the
// library holds the array until the process exits.  Host code must not use
// the array's name as a device address: each device's address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
// ======================================================================
namespace jpsi {

constexpr int64_t kNoAllocMaxEvents = (int64_t)1 << 18;  // 262,144 events per call
constexpr size_t kNoAllocCtrlOff = 0;
constexpr size_t kNoAllocClassOff = 512;
constexpr size_t kNoAllocListOff = kNoAllocClassOff + (size_t)kNoAllocMaxEvents;
constexpr size_t kNoAllocBytes = kNoAllocListOff + 3 * sizeof(int32_t) * (size_t)kNoAllocMaxEvents;
static_assert(sizeof(Ctrl) <= kNoAllocClassOff - kNoAllocCtrlOff, "control block slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static unsigned char* g_noalloc_dev[kNoAllocMaxDevices];  // device address of the array, per device

// Device address of the scratch array on `dev` (the current device).
static cudaError_t noalloc_scratch(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_dev[dev]) {
        void* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_dev[dev] = static_cast<unsigned char*>(ptr);
    }
    *out = g_noalloc_dev[dev];
    return cudaSuccess;
}

}  // namespace jpsi

extern "C" jpsi_status jpsi_select_noalloc(const jpsi_params* p, const jpsi_batch* b, int32_t* track_counts,
                                           int32_t* unit_counts, void* cuda_stream) {
    using namespace jpsi;
    using namespace jpsi::basek;
    if (!p || !b) return JPSI_EINVAL;
    if (p->n_stations < 1 || p->n_stations > kMaxStations || p->trigger_station < 0 ||
        p->trigger_station >= p->n_stations || (p->mode != JPSI_MODE_PAPER && p->mode != JPSI_MODE_CHAIN) ||
        p->ndf < 1 || p->min_candidates < 0 || !(p->t_xz >= 0.0f) || !(p->t_yz >= 0.0f) ||
        std::isinf(p->t_xz) || std::isinf(p->t_yz) || p->distinct_hits != 0)
        return JPSI_EINVAL;  // (distinct_hits changes accept bits only, which this entry point does not return)
    if (b->n_events < 0 || b->n_events > kNoAllocMaxEvents) return JPSI_EINVAL;  // beyond the static scratch
    if (b->n_hits < 0 || b->n_hits >= ((int64_t)1 << 31) || (b->n_events == 0 && b->n_hits != 0)) return JPSI_EINVAL;
    if (b->n_events == 0) return JPSI_OK;
    if (!b->offsets || (b->n_hits > 0 && (!b->x || !b->y || !b->z)) || !track_counts || !unit_counts)
        return JPSI_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return JPSI_ECUDA;
    unsigned char* base = nullptr;
    if (noalloc_scratch(dev, &base) != cudaSuccess) return JPSI_ECUDA;
    Ctrl* dctrl = reinterpret_cast<Ctrl*>(base + kNoAllocCtrlOff);
    Job j{};
    j.x = b->x;
    j.y = b->y;
    j.z = b->z;
    j.off = b->offsets;
    j.n_events = b->n_events;
    j.n_hits = b->n_hits;
    j.ev_begin = 0;
    j.ev_count = b->n_events;
    j.S = p->n_stations;
    j.trig = p->trigger_station;
    j.mode = p->mode;
    j.minc = p->min_candidates;
    j.cx = (float)p->ndf * p->t_xz;
    j.cy = (float)p->ndf * p->t_yz;
    {  // pruning slope factor sqrt(max C)(1 + 1e-4) + 1e-20, rounded up (as for contexts)
        const double kk = std::sqrt((double)std::max(j.cx, j.cy)) * (1.0 + 1e-4) + 1e-20;
        float f = (float)kk;
        if ((double)f < kk) f = std::nextafter(f, INFINITY);
        j.K = f;
    }
    j.grab = 2;
    j.cap_small = SmallCfg::LAYER_CAP;
    j.cap_medium = MediumCfg::LAYER_CAP;
    j.persistent = 1;
    j.unit_counts = unit_counts;
    j.track_counts = track_counts;
    j.ev_class = base + kNoAllocClassOff;
    int32_t* lists = reinterpret_cast<int32_t*>(base + kNoAllocListOff);
    j.mlist = lists;
    j.hlist = lists + kNoAllocMaxEvents;
    j.glist = lists + 2 * kNoAllocMaxEvents;
    j.ctrl = dctrl;  // tlist, accept bits, offsets, triplets and entries stay null: the warp kernel alone runs
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return JPSI_ECUDA;
    const int wpb = 4;
    const int per_sm = light_max_blocks_per_sm(wpb);
    if (per_sm < 1) return JPSI_ECUDA;
    if (cudaMemsetAsync(dctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return JPSI_ECUDA;  // counters start at zero
    k_light<false><<<n_sm * per_sm, 32 * wpb, light_smem_bytes(wpb), st>>>(j);
    if (cudaGetLastError() != cudaSuccess) return JPSI_ECUDA;
    Ctrl ctl{};
    if (cudaMemcpyAsync(&ctl, dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess) return JPSI_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return JPSI_ECUDA;
    if (ctl.status & kStBounds) return JPSI_ECUDA;  // (checked build only)
    if (ctl.status & kStInvalid) return JPSI_EINVAL;
    // an event beyond the warp tile (or with extreme coordinates) needs the
    // other kernels and their scratch: not available here
    if (ctl.n_medium + ctl.n_heavy + ctl.n_generic > 0) return JPSI_EINVAL;
    return JPSI_OK;
}
#endif  // !JPSI_STREAM
