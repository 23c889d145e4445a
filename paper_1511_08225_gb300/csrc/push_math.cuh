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
// The push walks the pieces the line crosses (fast w < 0, slow band, fast
// w > 0), spending the budget |a| dt of (*), and solves the last piece for
// w_end.  Differences of F are formed without cancellation (see seg_integral),
// and w_end itself is returned, so the new velocity keeps full FP32
// precision even when |a| dt << |v|.  Small steps in a fast piece use the
// series reversion of (*) to 4th order; larger ones use Newton from a
// one-sided bound (the piece integrand is convex for w > 0, concave for
// w < 0, so Newton converges monotonically).
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

// qT = rint(beta 2^40), qR = rint((beta*offset) 2^40); node c gets qT - qR,
// node c+1 gets qR.
__device__ __forceinline__ void quantise(float beta, float offset, unsigned long long &qL,
                                         unsigned long long &qR)
{
    const float two40 = 1099511627776.0f;
    long long r = __float2ll_rn(__fmul_rn(__fmul_rn(beta, offset), two40));
    long long t = __float2ll_rn(__fmul_rn(beta, two40));
    qR = (unsigned long long)r;
    qL = (unsigned long long)(t - r);
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
    float S = ra + rb;
    float sum = wa + wb;
    float t1 = 0.25f * d * (S + sum * sum / S);
    float t2 = 0.0f;
    if (D > 0.0f) {
        float den = wb * ra + wa * rb;
        t2 = 0.5f * D * asinhf(d * sum / den);
    }
    return t1 + t2;
}

// Solve int_{wa}^{wa+d} sqrt(w^2 + D) dw = y for d in [0, dmax], on a piece
// where w keeps the sign of wa (wa >= 0: convex; wa < 0: concave).
__device__ __forceinline__ float solve_seg(float wa, float D, float y, float dmax)
{
    float ra = sqrtf(wa * wa + D);
    float inv_ra = 1.0f / ra;
    float kap = y * inv_ra * inv_ra;  // y / ra^2
    if (kap <= 0.03f) {
        // d/ra = k - (om/2) k^2 + ((4om^2-1)/6) k^3 + (om(13-28om^2)/24) k^4 + O(k^5),
        // om = wa/ra: series reversion of ra d + (wa/2ra) d^2 + (D/6ra^3) d^3 - (D wa/8ra^5) d^4
        float om = wa * inv_ra;
        float om2 = om * om;
        float c2 = -0.5f * om;
        float c3 = (4.0f * om2 - 1.0f) * (1.0f / 6.0f);
        float c4 = om * (13.0f - 28.0f * om2) * (1.0f / 24.0f);
        float d = y * inv_ra * (1.0f + kap * (c2 + kap * (c3 + kap * c4)));
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
        float rb = sqrtf(wb * wb + D);
        float f = seg_integral(wa, ra, d, wb, rb, D) - y;
        float dn = fminf(fmaxf(d - f / rb, 0.0f), dmax);
        bool done = fabsf(dn - d) <= 4e-7f * dn;
        d = dn;
        if (done)
            break;
    }
    return d;
}

// New vx of a 1D3V particle (E along x, so vy and vz are unchanged).
__device__ __forceinline__ float push_vx(int kind, float ux, float uy, float uz, float ax,
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
