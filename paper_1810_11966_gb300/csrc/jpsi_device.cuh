// Device-side arithmetic of the J/psi triplet selection (arXiv:1810.11966,
// Sec. 3.2) and the conservative pruning it runs behind.
//
// Exact part (decides results): P1, the fit of a triplet with the vertex by
// u = m z in both planes and the cut on the summed squared residual, and P2,
// the CHAIN-mode compatibility of a station triplet with a trigger slope.
// Both use __fmul_rn / __fadd_rn / __fsub_rn / __fdiv_rn so that nothing is
// contracted into an FMA and every step rounds to nearest in the order below.
//
// Pruning part (only skips work): per hit, s_u = u * r with r ~ 1/z from the
// hardware reciprocal approximation (rcp.approx.ftz.f32; a relative error of
// a few 2^-23 at most, used only for normal z in [2^-126, 2^126)), and a bound
//     b = K * r + kappa * (|s_x| + |s_y|) + tau,
//     K = sqrt(max C)(1 + 1e-4) + 1e-20 (rounded up), kappa = 2^-17, tau = 1e-37.
// If a triplet passes P1 with slope m, each hit obeys
//     |u_k/z_k - m| <= (|r_k|(1+2eps) + eps |m z_k|) / z_k,  |r_k| <= sqrt(C)(1+2eps) + 2^-74
// (eps = 2^-24; the 2^-74 covers squares that underflow).  Subtracting the
// relations of two hits and adding the error of s (< 2^-20 |s|) gives
//     |s_i - s_j| <= b_i (1 - 5e-5) + b_j (1 - 5e-5),
// so the FP32 test |fl(s_i - s_j)| <= fl(b_i + b_j) never rejects a pair that
// belongs to a passing triplet (K's 1e-4 slack covers the error of r, kappa
// the relative errors of s and eps |m|).  The tiles keep one bound per layer,
// B_l = max of b over the layer's stored hits, and test against
// fl(B_l + B_l') >= fl(b_i + b_j) (rounding is monotone); the hits of a
// detector layer share its z, so B_l is b up to the small kappa term.  Hits with a non-finite coordinate
// cannot pass P1 at all (Szz, Suz or a residual becomes Inf/NaN) and are
// dropped; hits with finite coordinates but z outside [2^-126, 2^126) or a
// non-finite s or b send their event to the unpruned path.
#pragma once
#include <cstdint>

namespace jpsi {

constexpr float kKappa = 7.62939453125e-06f;    // 2^-17
constexpr float kPad = 9.5367431640625e-07f;     // 2^-20, query padding
constexpr float kTau = 1e-37f;

struct Cuts {
    float cx, cy;  // thresholds on S_x, S_y: fl32(ndf * t)
    float K;       // pruning slope factor (see above)
};

// ---------------------------------------------------------------- P1 / P2

// Szz = (z0*z0 + z1*z1) + z2*z2
__device__ __forceinline__ float sum_sq3(float a, float b, float c) {
    return __fadd_rn(__fadd_rn(__fmul_rn(a, a), __fmul_rn(b, b)), __fmul_rn(c, c));
}

// (u0*z0 + u1*z1) + u2*z2
__device__ __forceinline__ float dot3(float u0, float u1, float u2, float z0, float z1, float z2) {
    return __fadd_rn(__fadd_rn(__fmul_rn(u0, z0), __fmul_rn(u1, z1)), __fmul_rn(u2, z2));
}

// (r0*r0 + r1*r1) + r2*r2 with r_k = u_k - m*z_k
__device__ __forceinline__ float resid3(float u0, float u1, float u2, float z0, float z1, float z2, float m) {
    const float r0 = __fsub_rn(u0, __fmul_rn(m, z0));
    const float r1 = __fsub_rn(u1, __fmul_rn(m, z1));
    const float r2 = __fsub_rn(u2, __fmul_rn(m, z2));
    return sum_sq3(r0, r1, r2);
}

// P1: Sec. 3.2 step 2 on hits k = 0,1,2 of layers 0,1,2.
__device__ __forceinline__ bool fit_pass(const float x[3], const float y[3], const float z[3], const Cuts& c,
                                         float& mx, float& my) {
    const float szz = sum_sq3(z[0], z[1], z[2]);
    mx = __fdiv_rn(dot3(x[0], x[1], x[2], z[0], z[1], z[2]), szz);
    my = __fdiv_rn(dot3(y[0], y[1], y[2], z[0], z[1], z[2]), szz);
    const float sx = resid3(x[0], x[1], x[2], z[0], z[1], z[2], mx);
    const float sy = resid3(y[0], y[1], y[2], z[0], z[1], z[2], my);
    return (sx <= c.cx) && (sy <= c.cy);  // ordered: NaN fails
}

// P2: residuals of a station triplet against a trigger slope, no refit.
__device__ __forceinline__ bool chain_pass(const float x[3], const float y[3], const float z[3], float mx, float my,
                                           const Cuts& c) {
    return (resid3(x[0], x[1], x[2], z[0], z[1], z[2], mx) <= c.cx) &&
           (resid3(y[0], y[1], y[2], z[0], z[1], z[2], my) <= c.cy);
}

// Necessary condition of P2 for one hit: S >= fl(r_k^2) for every k because
// the partial sums of non-negative terms never round below a term.
__device__ __forceinline__ bool tube_pass(float x, float y, float z, float mx, float my, const Cuts& c) {
    const float rx = __fsub_rn(x, __fmul_rn(mx, z));
    const float ry = __fsub_rn(y, __fmul_rn(my, z));
    return (__fmul_rn(rx, rx) <= c.cx) && (__fmul_rn(ry, ry) <= c.cy);
}

// ------------------------------------------------------------- pruning

struct HitPrep {
    float sx, sy, b;
    float r, l1;  // r ~ 1/z and |s_x| + |s_y| (the parts of b the pair bound uses)
    bool live;  // all coordinates finite (else the hit can never pass)
    bool wild;  // live but s or b not finite: no pruning for its event
    bool zbad;  // z <= 0: invalid input
};

__device__ __forceinline__ HitPrep hit_prep(float x, float y, float z, float K) {
    HitPrep h;
    h.zbad = z <= 0.0f;
    h.live = (fabsf(x) < INFINITY) & (fabsf(y) < INFINITY) & (fabsf(z) < INFINITY);
    float iz;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(iz) : "f"(z));
    h.sx = __fmul_rn(x, iz);
    h.sy = __fmul_rn(y, iz);
    h.r = iz;
    h.l1 = __fadd_rn(fabsf(h.sx), fabsf(h.sy));
    h.b = __fadd_rn(__fadd_rn(__fmul_rn(K, iz), __fmul_rn(kKappa, h.l1)), kTau);
    // b finite implies s_x, s_y finite (b >= kappa |s|)
    h.wild = h.live & !((z >= 1.17549435e-38f) & (z < 8.50705917e+37f) & (h.b < INFINITY));
    return h;
}

// Fast staging path: slopes and bound without the per-hit classification.
// ok is exactly live && !wild && !zbad of hit_prep: z in the normal range
// [2^-126, 2^126) excludes z <= 0, NaN and Inf, and a finite b implies finite
// s_x, s_y, hence finite x, y.
struct HitFast {
    float sx, sy, b;
    float r, l1;  // as in HitPrep
    bool ok;
};

__device__ __forceinline__ HitFast hit_fast(float x, float y, float z, float K) {
    HitFast h;
    float iz;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(iz) : "f"(z));
    h.sx = __fmul_rn(x, iz);
    h.sy = __fmul_rn(y, iz);
    h.r = iz;
    h.l1 = __fadd_rn(fabsf(h.sx), fabsf(h.sy));
    h.b = __fadd_rn(__fadd_rn(__fmul_rn(K, iz), __fmul_rn(kKappa, h.l1)), kTau);
    h.ok = (z >= 1.17549435e-38f) & (z < 8.50705917e+37f) & (h.b < INFINITY);
    return h;
}

// Pair bound of two layers, tighter than b_i + b_j.  For a triplet passing P1
// the computed residuals of two of its hits satisfy r_i^2 + r_j^2 <= C (1 +
// 4 eps) + 2^-148 (S <= C, and the partial sums of non-negative terms never
// round below their parts), so with the per-hit relation above and
// Cauchy-Schwarz
//     |s_i - s_j| <= (1 + 2 eps)(|r_i|/z_i + |r_j|/z_j) + 2 eps |m|
//                 <= (1 + 2 eps)(sqrt(C)(1 + 2 eps) + 2^-74) sqrt(1/z_i^2 + 1/z_j^2) + 2 eps |m|,
// against sqrt(C)(1/z_i + 1/z_j) for b_i + b_j: a factor sqrt(2) at equal z.
// With R_l the largest r ~ 1/z (1/z <= r (1 + 2^-21)) and S_l the largest
// |s_x| + |s_y| of the stored hits of layer l,
//     B_ab = K sqrt(R_a^2 + R_b^2) + kappa (S_a + S_b) + 2 tau
// exceeds that for every pair of hits of layers a and b, by the argument for
// b: K's relative slack 1e-4 covers the factors above and the rounding of
// the squares, sum, root, product and sums here (a few 2^-24 each), its
// 1e-20 covers 2^-74, and the kappa terms cover 2 eps |m| and the errors of
// s.  When max(R_a, R_b) lies outside [2^-60, 2^60] (squares that could
// overflow or lose the smaller term to underflow) R_a + R_b, which is never
// below sqrt(R_a^2 + R_b^2), takes the root's place.
__device__ __forceinline__ float pair_bound(float ra, float sa, float rb, float sb, float K) {
    const float rm = fmaxf(ra, rb);
    const float q = (rm >= 8.67361737988403547e-19f && rm <= 1.15292150460684698e+18f)
                        ? __fsqrt_rn(__fadd_rn(__fmul_rn(ra, ra), __fmul_rn(rb, rb)))
                        : __fadd_rn(ra, rb);
    return __fadd_rn(__fadd_rn(__fmul_rn(K, q), __fmul_rn(kKappa, __fadd_rn(sa, sb))), 2.0f * kTau);
}

// May hits i and j belong to one passing triplet?  (never false for such a
// pair when bb >= fl(b_i + b_j), or bb >= the pair bound of their layers)
__device__ __forceinline__ bool pair_ok(float sxi, float syi, float sxj, float syj, float bb) {
    return (fabsf(__fsub_rn(sxi, sxj)) <= bb) & (fabsf(__fsub_rn(syi, syj)) <= bb);
}

// May a hit pass the tube of trigger slope (mx, my)?  From tube_pass:
// |s - m| <= b (1 - 5e-5) + 2^-21 |m| for a passing hit; the test allows
// b + 2^-16 |m|.
__device__ __forceinline__ bool tube_ok(float sx, float sy, float b, float mx, float my) {
    const float wx = __fadd_rn(b, __fmul_rn(2.0f * kKappa, fabsf(mx)));
    const float wy = __fadd_rn(b, __fmul_rn(2.0f * kKappa, fabsf(my)));
    return (fabsf(__fsub_rn(sx, mx)) <= wx) & (fabsf(__fsub_rn(sy, my)) <= wy);
}

// Slope bins of one layer: bin(v) = clamp(floor((v - lo) * inv_w), 0, NB-1),
// non-decreasing in v (each step is a monotone rounding), so a value range
// maps to a contiguous bin range.
template <int NB>
__device__ __forceinline__ int slope_bin(float v, float lo, float inv_w) {
    // floor to int saturates out-of-range values and maps NaN to 0
    const int t = __float2int_rd(__fmul_rn(__fsub_rn(v, lo), inv_w));
    return min(max(t, 0), NB - 1);
}

// Scale of a layer's bin map, about nb / (hi - lo) from the hardware
// reciprocal: any finite scale >= 0 gives monotone bins, and queries use the
// stored value, so it need not be rounded correctly.  0 when the range is
// empty or the scale is not finite (every value then falls in bin 0).
__device__ __forceinline__ float bin_scale(float lo, float hi, int nb) {
    if (!(hi > lo)) return 0.0f;
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__fsub_rn(hi, lo)));
    const float s = __fmul_rn((float)nb, r);
    return s < INFINITY ? s : 0.0f;
}

// Bins that contain every stored value v with |v - c| <= W (1 + 2^-20):
// the half-width is padded by 2^-18 W + 2^-20 |c|, which exceeds the rounding
// of c -/+ W'' (<= eps (|c| + W'')).
template <int NB>
__device__ __forceinline__ void query_bins(float c, float W, float lo, float inv_w, int& b0, int& b1) {
    const float Wp = __fadd_rn(__fadd_rn(__fmul_rn(W, 1.000003814697265625f), __fmul_rn(kPad, fabsf(c))), kTau);
    b0 = slope_bin<NB>(__fsub_rn(c, Wp), lo, inv_w);
    b1 = slope_bin<NB>(__fadd_rn(c, Wp), lo, inv_w);
}

}  // namespace jpsi
