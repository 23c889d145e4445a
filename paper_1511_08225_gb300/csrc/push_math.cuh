// push_math.cuh -- per-particle arithmetic of the SLPIC step (device code).
//
// Velocity push (Appendix A, Eq. slpicIntegrationV).  E is frozen over the
// step, so the velocity moves along the straight line v = u + a tau with
// dtau/dt = beta(|v|).  Write w for the component of v along a and D for
// |v_perp|^2 (unchanged).  Then dw/dt = |a| beta(sqrt(w^2 + D)), i.e.
//
//     int_{w_start}^{w_end} dw / beta(sqrt(w^2 + D)) = |a| dt.          (*)
//
// 1/beta is 1 in the slow band |v| <= v0 (Heaviside) and sqrt(w^2+D')/v0 in
// a fast piece (D' = D for Heaviside, D + v0^2 for the relativistic beta),
// whose integral has the closed form
//
//     F(w) = (w sqrt(w^2+D') + D' asinh(w / sqrt(D'))) / 2.
//
// Most particles need no iteration (push_vx_easy): plain leapfrog inside the
// band, or the 6th-order series reversion of (*) when the step is small
// against the speed.  The rest walk the pieces the line crosses (fast w < 0,
// slow band, fast w > 0), spending the budget |a| dt of (*), and solve the
// last piece for w_end (push_vx_walk): by the series, or by Newton from a
// one-sided bound (the piece integrand is convex for w > 0, concave for
// w < 0, so Newton converges monotonically).  Differences of F are formed
// without cancellation (see seg_integral), and w_end itself is returned, so
// the new velocity keeps full FP32 precision even when |a| dt << |v|.
//
// Quantised deposit: the bit-exact rule declared with slpic_charge_raw in
// slpic.h; every FP32 operation uses an explicit round-to-nearest intrinsic
// so that no multiply-add is fused.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "slpic.h"

namespace slpic {

// beta(|v|) of Sec. II, Eqs. (heavisideBeta)/(relativisticBeta), in the
// exact FP32 operation order of the quantised deposit rule.
__device__ __forceinline__ float beta_q(int kind, float vx, float vy, float vz, float v0)
{
    if (kind == SLPIC_BETA_ONE)
        return 1.0f;
    float s2 = __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz));
    if (kind == SLPIC_BETA_HEAVISIDE) {
        float r = __fsqrt_rn(s2);
        return (r <= v0) ? 1.0f : __fdiv_rn(v0, r);
    }
    return __fdiv_rn(v0, __fsqrt_rn(__fadd_rn(s2, __fmul_rn(v0, v0))));
}

// rint(x) (round to nearest, ties to even) for 0 <= x < 2^41 as two 32-bit words,
// value = hi 2^32 + lo, in FP32 and 32-bit operations (a float -> int64 conversion
// would run on the FP64 pipe, which is narrow on this GPU):
//   hf = floor(x 2^-32): the scaling by a power of two is exact, and hf is an integer
//        below 2^9; the bits of hf + 2^23 (exact: the float spacing there is 1) minus
//        those of 2^23 are hi;
//   x - hf 2^32 is exact in FP32 (below 2^32 it is x; above, x and hf 2^32 are both
//        multiples of the ulp of x and the difference is below 2^32, so it has at most
//        24 significant bits) and lies in [0, 2^32); converted to an unsigned integer
//        with ties to even it is lo, because rint(a + n) = rint(a) + n for an even
//        integer n = hf 2^32.
// Checked against llrintf for every float in [0, 2^41) on the CPU.
__device__ __forceinline__ void rint_split(float x, unsigned &lo, unsigned &hi)
{
    const float hf = floorf(__fmul_rn(x, 0x1p-32f));
    hi = __float_as_uint(__fadd_rn(hf, 8388608.0f)) - 0x4B000000u;
    lo = __float2uint_rn(__fmaf_rn(-hf, 4294967296.0f, x));
}

// The same value as one unsigned 64-bit integer.
__device__ __forceinline__ unsigned long long rint_u64(float x)
{
    unsigned lo, hi;
    rint_split(x, lo, hi);
    return ((unsigned long long)hi << 32) | lo;
}

// qT = rint(beta 2^40), qR = rint((beta*offset) 2^40); node c gets qL = qT - qR,
// node c+1 gets qR; each as two 32-bit words (value = hi 2^32 + lo).
__device__ __forceinline__ void quantise_split(float beta, float offset, unsigned &qLlo,
                                               unsigned &qLhi, unsigned &qRlo, unsigned &qRhi)
{
    const float two40 = 1099511627776.0f;
    unsigned tlo, thi;
    rint_split(__fmul_rn(__fmul_rn(beta, offset), two40), qRlo, qRhi);
    rint_split(__fmul_rn(beta, two40), tlo, thi);
    qLlo = tlo - qRlo;
    qLhi = thi - qRhi - (tlo < qRlo ? 1u : 0u);
}

// The same as 64-bit integers.
__device__ __forceinline__ void quantise(float beta, float offset, unsigned long long &qL,
                                         unsigned long long &qR)
{
    unsigned llo, lhi, rlo, rhi;
    quantise_split(beta, offset, llo, lhi, rlo, rhi);
    qL = ((unsigned long long)lhi << 32) | llo;
    qR = ((unsigned long long)rhi << 32) | rlo;
}

// int_{wa}^{wa+d} sqrt(w^2 + D) dw for a segment that does not cross w = 0
// (d >= 0, wb = wa + d, ra/rb the speeds at the ends).  From F above:
//   wb rb - wa ra = (d/2) [(ra+rb) + (wa+wb)^2/(ra+rb)]
//   asinh(wb/sqrt(D)) - asinh(wa/sqrt(D)) = asinh(d (wa+wb) / (wb ra + wa rb))
// (the second by the asinh subtraction identity); with wa, wb of one sign
// every sum here adds like-signed terms, so nothing cancels.
__device__ __forceinline__ float seg_integral(float wa, float ra, float d, float wb, float rb,
                                              float D)
{
    if (d <= 0.0f)
        return 0.0f;
    // the quotients by a reciprocal approximation (__fdividef, within 2 ulp): the
    // walk's root is then within a few ulp, far inside the push's error bar
    float S = ra + rb;
    float sum = wa + wb;
    float t1 = 0.25f * d * (S + __fdividef(sum * sum, S));
    float t2 = 0.0f;
    if (D > 0.0f) {
        float den = wb * ra + wa * rb;
        t2 = 0.5f * D * asinhf(__fdividef(d * sum, den));
    }
    return t1 + t2;
}

// Series reversion of int_{wa}^{wa+d} sqrt(w^2 + D) dw = y about wa.  With
// ra = sqrt(wa^2 + D), om = wa/ra and k = y/ra^2 (so D/ra^2 = 1 - om^2),
//   d / ra = k (1 + b2 k + b3 k^2 + ... + b6 k^5) + O(k^7),
// the b_i below (derived symbolically; b2..b4 by hand).  Against the exact root
// (40-digit arithmetic, om in [-1, 1]) the truncation error is below 9.2e-7 ra at
// k = 0.12 and falls as k^7: a tenth of the push's 1e-5 |v| bar at the largest k,
// and about 2e-21 ra at the median k of the sheath's particles (about 1e-3).  The
// terms b7, b8 would take it to 3.6e-8 ra for eight more fused multiply-adds per
// particle, on the path nearly every particle takes.  The
// integrand is analytic within |w - wa| < ra, so the series holds across w = 0
// when D > 0; it must not be used across the Heaviside band edge.
constexpr float kSeriesMax = 0.12f;

__device__ __forceinline__ float series_poly(float om, float k)
{
    // b_n is even in om for odd n and om times an even polynomial for even n, so the
    // sum splits into two polynomials in k^2 whose coefficients are polynomials in
    // om^2 (the divisors folded into them):
    //   1 + b3 k^2 + b5 k^4  +  om k (d2 + d4 k^2 + d6 k^4),  b_n = om d_n.
    // Explicit fused multiply-adds: every kernel that inlines this gets the same bits.
    const float o2 = __fmul_rn(om, om);
    const float k2 = __fmul_rn(k, k);
    const float b3 = __fmaf_rn(4.0f / 6.0f, o2, -1.0f / 6.0f);
    const float b5 = __fmaf_rn(__fmaf_rn(280.0f / 120.0f, o2, -188.0f / 120.0f), o2, 13.0f / 120.0f);
    const float d4 = __fmaf_rn(-28.0f / 24.0f, o2, 13.0f / 24.0f);
    const float d6 = __fmaf_rn(__fmaf_rn(-3640.0f / 720.0f, o2, 3188.0f / 720.0f), o2, -493.0f / 720.0f);
    const float ev = __fmaf_rn(__fmaf_rn(b5, k2, b3), k2, 1.0f);
    const float od = __fmul_rn(__fmaf_rn(__fmaf_rn(d6, k2, d4), k2, -0.5f), k);
    return __fmaf_rn(om, od, ev);
}

// Solve int_{wa}^{wa+d} sqrt(w^2 + D) dw = y for d in [0, dmax], on a piece
// where w keeps the sign of wa (wa >= 0: convex; wa < 0: concave).
__device__ __forceinline__ float solve_seg(float wa, float D, float y, float dmax)
{
    float ra = sqrtf(wa * wa + D);
    float inv_ra = 1.0f / ra;
    float kap = y * inv_ra * inv_ra;  // y / ra^2
    if (kap <= kSeriesMax) {
        float d = y * inv_ra * series_poly(wa * inv_ra, kap);
        return fminf(d, dmax);
    }
    float d;
    if (wa >= 0.0f) {
        // convex piece: both y/ra and the D = 0 solution bound the root from above
        float s = sqrtf(wa * wa + 2.0f * y);
        d = fminf(y * inv_ra, 2.0f * y / (s + wa));
    } else {
        // concave piece: y/ra bounds the root from below
        d = fminf(y * inv_ra, dmax);
    }
    for (int it = 0; it < 24; ++it) {
        float wb = wa + d;
        const float r2 = wb * wb + D;  // > 0: a fast piece never reaches |v| = 0
        float rb = r2 * rsqrtf(r2);
        float f = seg_integral(wa, ra, d, wb, rb, D) - y;
        float dn = fminf(fmaxf(d - __fdividef(f, rb), 0.0f), dmax);
        bool done = fabsf(dn - d) <= 4e-7f * dn;
        d = dn;
        if (done)
            break;
    }
    return d;
}

// The general walk over the pieces of (*) for the particles push_vx_easy leaves.
// Not inlined: it is long (asinh, Newton) and rare, and inlining it at every
// call site overflows the instruction cache of the particle kernels.
static __device__ __noinline__ float push_vx_walk(int kind, float ux, float uy, float uz, float ax,
                                         float dt, float v0)
{
    if (kind == SLPIC_BETA_ONE)
        return __fadd_rn(ux, __fmul_rn(ax, dt));  // plain leapfrog: int beta dt = dt
    float A = fabsf(ax);
    if (A == 0.0f)
        return ux;
    float sg = (ax > 0.0f) ? 1.0f : -1.0f;
    float wa = sg * ux;                                      // along a
    float Dp = __fadd_rn(__fmul_rn(uy, uy), __fmul_rn(uz, uz)); // |v_perp|^2
    float rem = __fmul_rn(A, dt);                            // budget of (*)
    float v02 = v0 * v0;
    float D = Dp, lo = 0.0f, hi = 0.0f, r_lo;
    bool band = false;
    if (kind == SLPIC_BETA_HEAVISIDE) {
        float wb = __fadd_rn(wa, rem);
        // |v| is convex along the line: both ends in the band => beta = 1 all
        // step and the push is plain leapfrog, bit for bit
        if (__fadd_rn(__fmul_rn(wa, wa), Dp) <= v02 && __fadd_rn(__fmul_rn(wb, wb), Dp) <= v02)
            return sg * wb;
        if (Dp < v02) {
            band = true;
            hi = sqrtf(v02 - Dp);
            lo = -hi;
            r_lo = v0;
        } else {
            r_lo = sqrtf(Dp);
        }
    } else {
        D = Dp + v02;
        r_lo = sqrtf(D);
    }
    float w = wa;
    if (w < lo) {
        // fast piece below lo; its integrand is at least r_lo/v0
        float dist = lo - w;
        bool inside = dist * r_lo >= rem * v0;
        if (!inside) {
            float ra = sqrtf(w * w + D);
            float cost = seg_integral(w, ra, dist, lo, r_lo, D) / v0;
            if (cost >= rem) {
                inside = true;
            } else {
                rem -= cost;
                w = lo;
            }
        }
        if (inside)
            return sg * (w + solve_seg(w, D, rem * v0, dist));
    }
    if (band && w < hi) {
        float len = hi - w;
        if (len >= rem)
            return sg * (w + rem);
        rem -= len;
        w = hi;
    }
    return sg * (w + solve_seg(w, D, rem * v0, CUDART_INF_F));
}

// New vx of a 1D3V particle (E along x, so vy and vz are unchanged): the cases
// that need no iteration.  Returns false (vx untouched) for the rest, which
// push_vx handles; for every particle it accepts, push_vx gives the same bits.
//   - beta == 1, or no field;
//   - Heaviside with both ends of the step in the band |v| <= v0 (plain leapfrog);
//   - a single smooth piece of (*) with k = |a| dt v0 / |v|^2 <= kSeriesMax
//     (the series).  Without a band (relativistic beta, or |v_perp| >= v0) the
//     integrand is analytic along the whole line; with a band the step must
//     start above it, or start below it and provably end below it.
__device__ __forceinline__ bool push_vx_easy(int kind, float ux, float uy, float uz, float ax,
                                             float dt, float v0, float &vx)
{
    if (kind == SLPIC_BETA_ONE) {
        vx = __fadd_rn(ux, __fmul_rn(ax, dt));  // plain leapfrog: int beta dt = dt
        return true;
    }
    float A = fabsf(ax);
    if (A == 0.0f) {
        vx = ux;
        return true;
    }
    float sg = (ax > 0.0f) ? 1.0f : -1.0f;
    float wa = sg * ux;
    float Dp = __fadd_rn(__fmul_rn(uy, uy), __fmul_rn(uz, uz));
    float rem = __fmul_rn(A, dt);
    float v02 = v0 * v0;
    float D = Dp;
    if (kind == SLPIC_BETA_HEAVISIDE) {
        float wb = __fadd_rn(wa, rem);
        const float sa = __fadd_rn(__fmul_rn(wa, wa), Dp);  // |v|^2 at the two ends
        const float sb = __fadd_rn(__fmul_rn(wb, wb), Dp);
        // |v| is convex along the line: both ends in the band => beta = 1 all
        // step and the push is plain leapfrog, bit for bit
        if (sa <= v02 && sb <= v02) {
            vx = sg * wb;
            return true;
        }
        // Otherwise one smooth piece needs the step to stay out of the band
        // |w| < hi = sqrt(v0^2 - Dp) (none if Dp >= v0^2): start above it (w grows), or
        // start below it and end below it even at leapfrog speed (below the band
        // 1/beta = |v|/v0 >= 1, so the true end lies short of wb).  Squared, no root:
        // wa >= hi <=> wa >= 0 and sa >= v0^2;  wb <= -hi <=> wb <= 0 and sb >= v0^2.
        if (Dp < v02 && !((wa >= 0.0f && sa >= v02) || (wb <= 0.0f && sb >= v02)))
            return false;
    } else {
        D = Dp + v02;
    }
    float y = __fmul_rn(rem, v0);
    float ra2 = __fmaf_rn(wa, wa, D);
    // one reciprocal square root gives 1/ra, wa/ra and y/ra^2 (its ~2 ulp error
    // moves d, already a small correction to wa, by ~1e-7 of itself).  Here ra2 is
    // about v0^2 or more, so the flush-to-zero form needs no subnormal fix-up; a
    // subnormal ra2 would give an infinite or NaN kap, and the hard path.
    float rs;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(ra2));
    float yr = __fmul_rn(y, rs);       // y / ra
    float kap = __fmul_rn(yr, rs);     // y / ra^2
    if (!(kap <= kSeriesMax))
        return false;
    vx = sg * __fmaf_rn(yr, series_poly(__fmul_rn(wa, rs), kap), wa);
    return true;
}

// New vx, any particle: the easy cases above, else walk the pieces of (*) and
// solve the last one (series or Newton, see solve_seg).
__device__ __forceinline__ float push_vx(int kind, float ux, float uy, float uz, float ax,
                                         float dt, float v0)
{
    float vx;
    if (push_vx_easy(kind, ux, uy, uz, ax, dt, v0, vx))
        return vx;
    return push_vx_walk(kind, ux, uy, uz, ax, dt, v0);
}

// ---- counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) ---------------
__device__ __forceinline__ unsigned long long sm64_mix(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
// i-th output of SplitMix64 started from state `key`
__device__ __forceinline__ unsigned long long sm64_at(unsigned long long key,
                                                      unsigned long long i)
{
    return sm64_mix(key + (i + 1ULL) * 0x9E3779B97F4A7C15ULL);
}
__device__ __forceinline__ unsigned long long sm64_stream(unsigned long long seed,
                                                          unsigned long long step,
                                                          unsigned int species)
{
    return sm64_mix(seed ^ sm64_mix(step * 16ULL + species + 1ULL));
}
// uniform on (0, 1], 24 bits
__device__ __forceinline__ float u24(unsigned long long z)
{
    return (float)((z >> 40) + 1ULL) * (1.0f / 16777216.0f);
}

}  // namespace slpic
