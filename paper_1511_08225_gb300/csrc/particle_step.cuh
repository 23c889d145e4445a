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

// Push one particle (Appendix A): returns false if absorbed (wall = 0 at x=0,
// 1 at x=L).  c, q updated in place.
__device__ __forceinline__ bool advance(const StepParams &p, const SpeciesDev &sp,
                                        const float *sE, unsigned long long *hist, int &c,
                                        float4 &q, int &wall)
{
    const int N = p.n_cells;
    float d = q.x;
    int c1 = c + 1;
    if (p.periodic && c1 == N)
        c1 = 0;
    // gather: linear interpolation of the nodal field (Sec. II scatter/gather)
    float Ep = (1.0f - d) * sE[c] + d * sE[c1];
    float ax = sp.qm * Ep;
    // v^{n+1/2} = v^{n-1/2} + a int beta dt
    float vx = push_vx(sp.kind, q.y, q.z, q.w, ax, p.dt, sp.v0);
    // x^{n+1} = x^n + beta(|v^{n+1/2}|) v^{n+1/2} dt, in cell units
    float b = beta_q(sp.kind, vx, q.z, q.w, sp.v0);
    float xn = d + b * vx * p.dt_dx;
    float fl = floorf(xn);
    int cn = c + (int)fl;
    float dn = xn - fl;
    if (dn >= 1.0f) {  // x just below a cell edge rounded up to it
        dn = 0.0f;
        cn += 1;
    }
    if (p.periodic) {
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
    if (p.periodic && cn1 == N)
        cn1 = 0;
    // rho^{n+1} += q w beta(|v^{n+1/2}|) S(x - x^{n+1})
    deposit_node(hist, cn, cn1, b, dn);
    c = cn;
    q.x = dn;
    q.y = vx;
    return true;
}

}  // namespace slpic
