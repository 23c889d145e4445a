// particle_step.cuh -- advance one macroparticle by one SLPIC step (device code),
// shared by every particle kernel of the library.
#pragma once

#include "push_math.cuh"
#include "slpic_internal.cuh"

namespace slpic {

__device__ __forceinline__ void deposit_node(unsigned long long *hist, int c, int c1, float b,
                                             float off)
{
    unsigned long long qL, qR;
    quantise(b, off, qL, qR);
    atomicAdd(hist + c, qL);
    atomicAdd(hist + c1, qR);
}

// Compile-time shape of a particle loop: kKind the species' beta kind (SLPIC_BETA_*)
// and kPer whether the grid is periodic (0/1), or kAny for "read at run time".  The
// fixed forms drop the run-time tests from the hot loop; the arithmetic, and so every
// result bit, is the same.
constexpr int kAny = -1;

// Gather (Sec. II): linear interpolation of the nodal field at the particle.
template <int kPer = kAny>
__device__ __forceinline__ float gather_ax(const StepParams &p, const SpeciesDev &sp,
                                           const float *sE, int c, float d)
{
    const bool periodic = kPer == kAny ? (p.periodic != 0) : (kPer != 0);
    int c1 = c + 1;
    if (periodic && c1 == p.n_cells)
        c1 = 0;
    // explicit roundings: every kernel that inlines this gets the same bits
    float Ep = __fmaf_rn(d, sE[c1], __fmul_rn(1.0f - d, sE[c]));
    return __fmul_rn(sp.qm, Ep);
}

// The speed limit of species sp in cell c (Sec. II: v0 may vary with position).
// kProf: a per-cell profile is set (p.lam), and the limit is the FP32 product
// v0 * lam[c] rounded to nearest; otherwise the species' uniform v0.  lam: a copy of
// the profile (in shared memory) to read instead of p.lam, or null.
template <bool kProf>
__device__ __forceinline__ float v0_at(const StepParams &p, const SpeciesDev &sp, int c,
                                       const float *lam = nullptr)
{
    if (!kProf)
        return sp.v0;
    return __fmul_rn(sp.v0, lam ? lam[c] : __ldg(p.lam + c));
}

// The same where a kernel serves both cases at run time (p.lam may be null).
__device__ __forceinline__ float v0_cell(const StepParams &p, const SpeciesDev &sp, int c)
{
    return p.lam ? __fmul_rn(sp.v0, __ldg(p.lam + c)) : sp.v0;
}

// After the velocity push (new vx): x^{n+1} = x^n + beta(|v^{n+1/2}|) v^{n+1/2} dt in
// cell units, walls or wrap, and rho^{n+1} += q w beta S(x - x^{n+1}) through
// dep(c, c+1, beta, offset).  Returns false if absorbed (wall = 0 at x=0, 1 at x=L).
// v0n is the limit of the start cell (that of the push); with kProf the deposit
// takes beta with the limit of the cell the particle ends in (the same beta if it
// stayed in its cell: a warp whose particles all stay skips the second division).
template <bool kProf = false, int kKind = kAny, int kPer = kAny, typename Dep>
__device__ __forceinline__ bool move_and_deposit(const StepParams &p, const SpeciesDev &sp,
                                                 Dep &dep, int &c, float4 &q, float vx, int &wall,
                                                 float v0n, const float *lam = nullptr)
{
    const int N = p.n_cells;
    const int kind = kKind == kAny ? sp.kind : kKind;
    const bool periodic = kPer == kAny ? (p.periodic != 0) : (kPer != 0);
    float b = beta_q(kind, vx, q.z, q.w, v0n);
    float xn = __fmaf_rn(__fmul_rn(b, vx), p.dt_dx, q.x);
    float fl = floorf(xn);
    int cn = c + (int)fl;
    float dn = xn - fl;
    if (dn >= 1.0f) {  // x just below a cell edge rounded up to it
        dn = 0.0f;
        cn += 1;
    }
    if (periodic) {
        cn %= N;
        if (cn < 0)
            cn += N;
    } else if (cn < 0) {
        wall = 0;
        return false;
    } else if (cn >= N) {
        wall = 1;
        return false;
    }
    int cn1 = cn + 1;
    if (periodic && cn1 == N)
        cn1 = 0;
    if (kProf && cn != c)
        b = beta_q(kind, vx, q.z, q.w, v0_at<true>(p, sp, cn, lam));
    dep(cn, cn1, b, dn);
    c = cn;
    q.x = dn;
    q.y = vx;
    return true;
}

// int64 shared-memory histogram
struct DepositU64 {
    unsigned long long *hist;
    __device__ __forceinline__ void operator()(int c, int c1, float b, float off)
    {
        deposit_node(hist, c, c1, b, off);
    }
};

// The same integers kept as two 32-bit words per node (value = hi 2^32 + lo):
// 32-bit shared-memory atomics are native; the carry out of lo is detected from
// the old value the atomic returns and added to hi, so the sum stays exact.
struct DepositSplit32 {
    unsigned *lo, *hi;
    __device__ __forceinline__ void add(int c, unsigned vl, unsigned vh)
    {
        unsigned old = atomicAdd(lo + c, vl);
        vh += (old + vl < old) ? 1u : 0u;
        if (vh)
            atomicAdd(hi + c, vh);
    }
    __device__ __forceinline__ void operator()(int c, int c1, float b, float off)
    {
        unsigned llo, lhi, rlo, rhi;
        quantise_split(b, off, llo, lhi, rlo, rhi);
        add(c, llo, lhi);
        add(c1, rlo, rhi);
    }
};

// Push one particle (Appendix A): returns false if absorbed (wall = 0 at x=0,
// 1 at x=L).  c, q updated in place.
__device__ __forceinline__ bool advance(const StepParams &p, const SpeciesDev &sp,
                                        const float *sE, unsigned long long *hist, int &c,
                                        float4 &q, int &wall)
{
    float ax = gather_ax(p, sp, sE, c, q.x);
    // v^{n+1/2} = v^{n-1/2} + a int beta dt
    float vx = push_vx(sp.kind, q.y, q.z, q.w, ax, p.dt, sp.v0);
    DepositU64 dep{hist};
    return move_and_deposit(p, sp, dep, c, q, vx, wall, sp.v0);
}

}  // namespace slpic
