// slpic2d.cu -- the 2D3V speed-limited PIC path behind include/slpic2d.h.
//
// Per step (Appendix A, Eq. slpicIntegration, on an nx x ny grid, periodic in x,
// absorbing plates in y):
//   k_particles2d_tiles (+ k_hard2d), or k_particles2d where its windows do not fit
//                  gather E (bilinear) -> push v (the same speed-limited solve as
//                  1D, along the direction of a) -> move -> plates/wrap -> deposit
//                  rho^{n+1} (quantised int64, bilinear) into the nodal arrays: the
//                  tile kernel through windows of the grid in shared memory, listing
//                  the pushes that need the piece walk for k_hard2d; the other by
//                  global atomics.  Absorbed particles leave holes (cell = -1) in
//                  place; every kCompact2d-th step the counting sort by cell drops
//                  them (k_particles2d packs the survivors itself on that step).
//   k_inject2d     source particles appended and deposited; k_book2d the bookkeeping.
//   k_cg2d         cooperative kernel: b from the deposits, Jacobi-PCG on the
//                  5-point system (FP64 vectors, FP64 dot products in a fixed
//                  order), then E^{n+1}; the deposits are cleared for the next step.
//
// Particle store per species, ping-pong buffers b = step & 1:
//   cell[b][i] int32 (cy*nx + cx, -1 = hole), pv[b][i] float4 {ox, oy, vx, vy},
//   vz[b][i] float  -- 24 bytes per macroparticle.
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "push_math.cuh"
#include "slpic2d.h"
#include "unet_internal.h"

namespace slpic {
void set_create_error(const std::string &msg);  // api.cu
}

namespace slpic2d {

using namespace slpic;

constexpr int kMaxS = SLPIC_MAX_SPECIES;
constexpr int kThreads = 256;
constexpr int kItems = 4;                       // particles per thread per tile
constexpr int kTile = kThreads * kItems;
constexpr int kWarps = kThreads / 32;
constexpr int kCompact2d = 16;                  // compacting step interval
constexpr int kCgThreads = 256;
constexpr int kBarGroup = 16;   // CTAs per first-level group of the grid barrier
constexpr int kBarGroups = 64;  // first-level counters (CG grids up to 1,024 CTAs)
constexpr long long kBarrierSpins = 1LL << 23;  // bounded grid-barrier wait (~1 s)
constexpr long long kMaxTimedSteps2d = 4096;    // steps recorded by the kernel timing

// A particle whose push needs the piece walk, listed by the in-place tile kernel
// for k_hard2d with what the push needs.
struct HardRec2D {
    int32_t slot, cell;  // its slot in the step's buffers; c at time level n
    float ax, ay;        // (q/m) E gathered at the particle
    float4 q;            // {ox, oy, vx, vy} at time level n (v = v^{n-1/2})
    float vz, pad[3];
};

struct Species2D {
    int32_t *cell[2];
    float4 *pv[2];
    float *vz[2];
    HardRec2D *hard;     // this step's listed particles (hard_cap records)
    long long hard_cap;
    long long capacity;
    float qm, v0, vth_src;
    int kind;
    double w, inv_w;
    double rho_unit;  // q w / dx^2 * 2^-40
};

struct State2D {
    long long step;
    unsigned long long count[kMaxS][2];   // slots in use (live + holes) per buffer
    unsigned long long holes[kMaxS][2];
    unsigned long long absorbed_step[kMaxS][2];
    long long absorbed_total[kMaxS][2];
    long long injected_total[kMaxS];
    double src_frac[kMaxS];
    unsigned long long hard_n[kMaxS];  // particles listed for k_hard2d this step
    unsigned long long iter_last;      // walked pushes of the last step, all species
    long long cg_total;
    double cg_res;
    int cg_iters;
    int error;
    unsigned bar_count, bar_gen;  // grid barrier of k_cg2d: root counter, generation
    unsigned bar_group[kBarGroups];  // first-level counters of the grid barrier
};

struct Params2D {
    int nx, ny, nn, ns;
    unsigned nx_m;  // c / nx = div_nx(c): the multiplier and shift of the round-up method
    int nx_s;
    float dt, dt_dx;
    double dx, dt64, k2;          // k2 = dx^2 / eps0
    double phi_lo, phi_hi, rtol2;  // rtol^2
    int cg_maxit;
    int src_mode, src_ref;
    float src_lo, src_len;
    double src_rate;
    unsigned long long seed;
    Species2D sp[kMaxS];
    unsigned long long *acc;  // [ns][nn] int64 deposits (two's complement)
    float2 *E;                // [nn] (Ex, Ey)
    double *phi, *r, *q;            // [nn] FP64: solution, standalone solve's rho, b
    float *fr, *fpA, *fpB, *fq, *fd;  // [nn] FP32 CG iterates, zero on the plate rows
    double *part;             // [3][grid] per-CTA partial sums
    State2D *st;
    // direct solver (SLPIC2D_SOLVER_FFT)
    int solver, log2nx;
    double2 *tw;              // [nx/2] (cos, sin)(2 pi m / nx)
    double2 *spec;            // [nn] Fourier coefficients along x, row by row
    double *inv_m;            // [nn] Thomas multipliers 1/m_j per (row j, mode k)
    double *seg_f, *seg_b;    // [nn] their products within a segment, up to / from row j
    double *rpart;            // [2 (ny+1)] per-row sums of r^2 and b^2
    int *hist, *cursor, *bsum;  // cell sort: counts per cell, then slots; block sums
};

// c / nx for 0 <= c < 2^32 and nx >= 2 without a division: Granlund and Montgomery's
// method for an invariant divisor (PLDI 1994, Fig. 4.1): with l = ceil(log2 nx) and
// m = floor(2^32 (2^l - nx) / nx) + 1 (host, make_div_nx), t = mulhi(m, c) and
// q = (t + ((c - t) >> 1)) >> (l - 1).
__device__ __forceinline__ int div_nx(const Params2D &p, int c)
{
    const unsigned n = (unsigned)c;
    const unsigned t = __umulhi(p.nx_m, n);
    return (int)((t + ((n - t) >> 1)) >> p.nx_s);
}

void make_div_nx(int nx, unsigned &m, int &s)
{
    int l = 0;
    while ((1LL << l) < nx)
        ++l;
    m = (unsigned)((((unsigned long long)1 << 32) * (unsigned long long)((1LL << l) - nx)) /
                       (unsigned long long)nx + 1ULL);
    s = l - 1;
}

// ---------------------------------------------------------------------------------
// Velocity push with a = (ax, ay, 0): the speed-limited solve of Appendix A,
// Eq. slpicIntegrationV, depends only on the component w of v along a and on
// |v_perp|, so the 1D solve (push_vx with a along +x) gives w at the end of the
// step and v changes by (w_end - w) in the direction of a.
// ---------------------------------------------------------------------------------
// kEasy: only the cases push_vx_easy solves; returns false (v untouched) for the
// rest, which need the piece walk.  Otherwise every case; returns true.
template <bool kEasy>
__device__ __forceinline__ bool push_v2_impl(int kind, float ux, float uy, float uz, float ax,
                                             float ay, float dt, float v0, float &vx, float &vy)
{
    if (kind == SLPIC_BETA_ONE) {
        vx = __fadd_rn(ux, __fmul_rn(ax, dt));
        vy = __fadd_rn(uy, __fmul_rn(ay, dt));
        return true;
    }
    // |a|, the direction of a and |v_perp| from reciprocal square roots (within a few
    // ulp; the push's bar is 1e-5 of |v|): one approximation instead of a correctly
    // rounded square root and two divisions
    const float a2 = __fadd_rn(__fmul_rn(ax, ax), __fmul_rn(ay, ay));
    if (a2 == 0.0f) {
        vx = ux;
        vy = uy;
        return true;
    }
    const float ra = rsqrtf(a2);
    const float A = __fmul_rn(a2, ra);
    const float hx = __fmul_rn(ax, ra), hy = __fmul_rn(ay, ra);
    const float wa = __fadd_rn(__fmul_rn(ux, hx), __fmul_rn(uy, hy));
    const float cr = __fsub_rn(__fmul_rn(ux, hy), __fmul_rn(uy, hx));
    const float vp2 = __fadd_rn(__fmul_rn(cr, cr), __fmul_rn(uz, uz));
    const float vp = vp2 > 0.0f ? __fmul_rn(vp2, rsqrtf(vp2)) : 0.0f;
    float we;
    if (kEasy) {
        if (!push_vx_easy(kind, wa, vp, 0.0f, A, dt, v0, we))
            return false;
    } else {
        we = push_vx(kind, wa, vp, 0.0f, A, dt, v0);
    }
    const float dw = __fsub_rn(we, wa);
    vx = __fadd_rn(ux, __fmul_rn(dw, hx));
    vy = __fadd_rn(uy, __fmul_rn(dw, hy));
    return true;
}

__device__ __forceinline__ void push_v2(int kind, float ux, float uy, float uz, float ax, float ay,
                                        float dt, float v0, float &vx, float &vy)
{
    push_v2_impl<false>(kind, ux, uy, uz, ax, ay, dt, v0, vx, vy);
}

__device__ __forceinline__ bool push_v2_easy(int kind, float ux, float uy, float uz, float ax,
                                             float ay, float dt, float v0, float &vx, float &vy)
{
    return push_v2_impl<true>(kind, ux, uy, uz, ax, ay, dt, v0, vx, vy);
}

// the 2D quantised deposit rule stated in slpic2d.h: the charges of the cell's nodes
// (x, y), (x+1, y), (x, y+1), (x+1, y+1)
__device__ __forceinline__ void quantise2d(float b, float ox, float oy, unsigned long long &q00,
                                           unsigned long long &q10, unsigned long long &q01,
                                           unsigned long long &q11)
{
    const float two40 = 1099511627776.0f;
    const float bx = __fmul_rn(b, ox), by = __fmul_rn(b, oy), bxy = __fmul_rn(bx, oy);
    const unsigned long long qT = rint_u64(__fmul_rn(b, two40));
    const unsigned long long qX = rint_u64(__fmul_rn(bx, two40));
    const unsigned long long qY = rint_u64(__fmul_rn(by, two40));
    const unsigned long long qXY = rint_u64(__fmul_rn(bxy, two40));
    q00 = qT - qX - qY + qXY;
    q10 = qX - qXY;
    q01 = qY - qXY;
    q11 = qXY;
}

__device__ __forceinline__ void deposit2d(unsigned long long *acc, int k00, int k10, int k01,
                                          int k11, float b, float ox, float oy)
{
    unsigned long long q00, q10, q01, q11;
    quantise2d(b, ox, oy, q00, q10, q01, q11);
    atomicAdd(acc + k00, q00);
    atomicAdd(acc + k10, q10);
    atomicAdd(acc + k01, q01);
    atomicAdd(acc + k11, q11);
}

// ---------------------------------------------------------------------------------
// Particle step.  COMPACT = false: slot i of the input goes to slot i of the
// output (a hole where a particle is absorbed); true: the survivors are packed
// (one global atomic per CTA tile).
// ---------------------------------------------------------------------------------
template <bool COMPACT>
__global__ void __launch_bounds__(kThreads) k_particles2d(Params2D p)
{
    __shared__ int s_cnt[kItems * kWarps];
    __shared__ unsigned long long s_base;
    __shared__ unsigned s_abs[2];
    const int s = blockIdx.y;
    const Species2D &sp = p.sp[s];
    const long long step = *(volatile long long *)&p.st->step;
    const int P = (int)(step & 1);
    const long long n = (long long)p.st->count[s][P];
    const int32_t *__restrict__ cin = sp.cell[P];
    const float4 *__restrict__ vin = sp.pv[P];
    const float *__restrict__ zin = sp.vz[P];
    int32_t *__restrict__ cout = sp.cell[P ^ 1];
    float4 *__restrict__ vout = sp.pv[P ^ 1];
    float *__restrict__ zout = sp.vz[P ^ 1];
    unsigned long long *acc = p.acc + (size_t)s * p.nn;
    const int nx = p.nx, ny = p.ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 2)
        s_abs[threadIdx.x] = 0u;
    __syncthreads();
    unsigned na0 = 0, na1 = 0;

    const long long ntiles = (n + kTile - 1) / kTile;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long base = t * kTile;
        int c[kItems];
        float4 q[kItems];
        float z[kItems];
        bool live[kItems];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const long long i = base + k * kThreads + threadIdx.x;
            live[k] = i < n;
            c[k] = -1;
            if (live[k]) {
                c[k] = __ldcs(cin + i);
                q[k] = __ldcs(vin + i);
                z[k] = __ldcs(zin + i);
            }
        }
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const bool was = live[k];
            live[k] = live[k] && c[k] >= 0;
            if (live[k]) {
                const int cy = div_nx(p, c[k]), cx = c[k] - cy * nx;
                const int cx1 = (cx + 1 == nx) ? 0 : cx + 1;
                const int k00 = cy * nx + cx, k10 = cy * nx + cx1;
                const float2 e00 = __ldg(p.E + k00), e10 = __ldg(p.E + k10);
                const float2 e01 = __ldg(p.E + k00 + nx), e11 = __ldg(p.E + k10 + nx);
                const float ox = q[k].x, oy = q[k].y;
                const float wx0 = __fsub_rn(1.0f, ox), wy0 = __fsub_rn(1.0f, oy);
                const float ex = __fadd_rn(
                    __fmul_rn(wy0, __fadd_rn(__fmul_rn(wx0, e00.x), __fmul_rn(ox, e10.x))),
                    __fmul_rn(oy, __fadd_rn(__fmul_rn(wx0, e01.x), __fmul_rn(ox, e11.x))));
                const float ey = __fadd_rn(
                    __fmul_rn(wy0, __fadd_rn(__fmul_rn(wx0, e00.y), __fmul_rn(ox, e10.y))),
                    __fmul_rn(oy, __fadd_rn(__fmul_rn(wx0, e01.y), __fmul_rn(ox, e11.y))));
                float vx, vy;
                const float axp = __fmul_rn(sp.qm, ex), ayp = __fmul_rn(sp.qm, ey);
                if (!push_v2_easy(sp.kind, q[k].z, q[k].w, z[k], axp, ayp, p.dt, sp.v0, vx, vy)) {
                    // the piece walk, here inline; counted for the diagnostics
                    namespace cg = cooperative_groups;
                    cg::coalesced_group g = cg::coalesced_threads();
                    if (g.thread_rank() == 0)
                        atomicAdd(&p.st->hard_n[s], (unsigned long long)g.size());
                    push_v2(sp.kind, q[k].z, q[k].w, z[k], axp, ayp, p.dt, sp.v0, vx, vy);
                }
                // x^{n+1} = x^n + beta(|v^{n+1/2}|) v^{n+1/2} dt, in cell units
                const float b = beta_q(sp.kind, vx, vy, z[k], sp.v0);
                const float xn = __fadd_rn(ox, __fmul_rn(__fmul_rn(b, vx), p.dt_dx));
                const float yn = __fadd_rn(oy, __fmul_rn(__fmul_rn(b, vy), p.dt_dx));
                const float fx = floorf(xn), fy = floorf(yn);
                int ncx = cx + (int)fx, ncy = cy + (int)fy;
                float dxn = __fsub_rn(xn, fx), dyn = __fsub_rn(yn, fy);
                if (dxn >= 1.0f) {
                    dxn = 0.0f;
                    ++ncx;
                }
                if (dyn >= 1.0f) {
                    dyn = 0.0f;
                    ++ncy;
                }
                if ((unsigned)ncx >= (unsigned)nx) {  // the x wrap
                    ncx %= nx;
                    if (ncx < 0)
                        ncx += nx;
                }
                if (ncy < 0) {
                    ++na0;
                    live[k] = false;
                } else if (ncy >= ny) {
                    ++na1;
                    live[k] = false;
                } else {
                    const int ncx1 = (ncx + 1 == nx) ? 0 : ncx + 1;
                    const int m00 = ncy * nx + ncx, m10 = ncy * nx + ncx1;
                    deposit2d(acc, m00, m10, m00 + nx, m10 + nx, b, dxn, dyn);
                    c[k] = m00;
                    q[k] = make_float4(dxn, dyn, vx, vy);
                }
            }
            if (!COMPACT && was) {
                const long long i = base + k * kThreads + threadIdx.x;
                if (live[k]) {
                    __stcs(cout + i, c[k]);
                    __stcs(vout + i, q[k]);
                    __stcs(zout + i, z[k]);
                } else {
                    __stcs(cout + i, -1);
                }
            }
        }
        if (COMPACT) {
            unsigned mask[kItems];
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                mask[k] = __ballot_sync(0xffffffffu, live[k]);
                if (lane == 0)
                    s_cnt[k * kWarps + warp] = __popc(mask[k]);
            }
            __syncthreads();
            if (warp == 0) {
                const int v = s_cnt[lane];
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o)
                        incl += y;
                }
                s_cnt[lane] = incl - v;
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                if (lane == 0)
                    s_base = tot ? atomicAdd(&p.st->count[s][P ^ 1], (unsigned long long)tot) : 0ULL;
            }
            __syncthreads();
            const unsigned long long ob = s_base;
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                if (live[k]) {
                    const unsigned long long o = ob + (unsigned long long)s_cnt[k * kWarps + warp] +
                                                 __popc(mask[k] & ((1u << lane) - 1u));
                    __stcs(cout + o, c[k]);
                    __stcs(vout + o, q[k]);
                    __stcs(zout + o, z[k]);
                }
            }
            __syncthreads();  // s_cnt / s_base reused by the next tile
        }
    }
    na0 = __reduce_add_sync(0xffffffffu, na0);
    na1 = __reduce_add_sync(0xffffffffu, na1);
    if (lane == 0) {
        if (na0)
            atomicAdd(&s_abs[0], na0);
        if (na1)
            atomicAdd(&s_abs[1], na1);
    }
    __syncthreads();
    if (threadIdx.x < 2 && s_abs[threadIdx.x])
        atomicAdd(&p.st->absorbed_step[s][threadIdx.x], (unsigned long long)s_abs[threadIdx.x]);
}

// The move after the push: x^{n+1} = x^n + beta v^{n+1/2} dt in cell units from
// cell (cx, cy) and offset (ox, oy), the x wrap and the plates.  Returns 0 or 1 if
// the particle crossed the plate at y = 0 or y = Ly, else -1 with its new cell and
// offset.
__device__ __forceinline__ int move2d(const Params2D &p, int cx, int cy, float ox, float oy,
                                      float vx, float vy, float b, int &ncx, int &ncy,
                                      float &dxn, float &dyn)
{
    const int nx = p.nx;
    const float xn = __fadd_rn(ox, __fmul_rn(__fmul_rn(b, vx), p.dt_dx));
    const float yn = __fadd_rn(oy, __fmul_rn(__fmul_rn(b, vy), p.dt_dx));
    const float fx = floorf(xn), fy = floorf(yn);
    ncx = cx + (int)fx;
    ncy = cy + (int)fy;
    dxn = __fsub_rn(xn, fx);
    dyn = __fsub_rn(yn, fy);
    if (dxn >= 1.0f) {
        dxn = 0.0f;
        ++ncx;
    }
    if (dyn >= 1.0f) {
        dyn = 0.0f;
        ++ncy;
    }
    if ((unsigned)ncx >= (unsigned)nx) {  // the x wrap (at most a cell, but for beta = 1)
        ncx %= nx;
        if (ncx < 0)
            ncx += nx;
    }
    if (ncy < 0)
        return 0;
    if (ncy >= p.ny)
        return 1;
    return -1;
}

// ---------------------------------------------------------------------------------
// The in-place particle step with grid tiles in shared memory (the steps between
// cell sorts).  After the sort (every kCompact2d steps) consecutive slots hold
// particles of neighbouring cells, and each particle moves at most one cell per
// step, so a chunk of kChunk2d consecutive slots touches a small box of the grid.
// One CTA per chunk at a time:
//   1. the chunk is copied into shared memory (coalesced loads), in a layout padded
//      by one entry every 64 so that the strided reads below meet no bank conflict;
//   2. the box of its cells, relative to the cell of a live particle near its
//      middle (x differences taken modulo nx, so a chunk that runs over the end of a
//      row is one box), widened by the gather's node and one cell of motion;
//   3. the window of nodes covering the box (at most kWin2d nodes) gets E copied in
//      and its deposit cleared;
//   4. each particle is gathered, pushed, moved and deposited as k_particles2d does,
//      from and into the window where its four nodes are inside it, else from E and
//      into acc in global memory.  Thread (warp w, lane l) takes the chunk's
//      particles 64 l + kPer2d w + k, so the lanes of a warp sit about a cell apart
//      and their shared-memory atomics rarely meet on a node;
//   5. the window's deposits go to acc (one atomic per nonzero node) and the chunk
//      back to its slots.
// The arithmetic per particle is that of k_particles2d (the same gathered values,
// push, move and quantised deposit), so the integer deposits and every particle are
// the same bit for bit; only where the charge is summed first differs.
// ---------------------------------------------------------------------------------
constexpr int kT2d = 512;                        // threads per CTA
constexpr int kPer2d = 4;                        // particles per thread per chunk
constexpr int kChunk2d = kT2d * kPer2d;          // 2,048 slots
constexpr int kPad2d = kChunk2d + kChunk2d / 64; // padded shared-memory entries
constexpr int kWin2d = 2048;                     // window nodes

__device__ __forceinline__ int pad2d(int i) { return i + (i >> 6); }

size_t tile2d_smem_bytes()
{
    return (size_t)kPad2d * (4 + 16 + 4) + (size_t)kWin2d * (8 + 4 + 4);
}

// 64-bit integer as two 32-bit words in shared memory (value = hi 2^32 + lo, modulo
// 2^64): the carry out of lo is detected from the old value the atomic returns
__device__ __forceinline__ void win_add(unsigned *lo, unsigned *hi, int k, unsigned long long v)
{
    const unsigned vl = (unsigned)v;
    unsigned vh = (unsigned)(v >> 32);
    const unsigned old = atomicAdd(lo + k, vl);
    vh += (old + vl < old) ? 1u : 0u;
    if (vh)
        atomicAdd(hi + k, vh);
}

__global__ void __launch_bounds__(kT2d, 2) k_particles2d_tiles(Params2D p)
{
    extern __shared__ __align__(16) unsigned char smem2d[];
    float4 *s_v = reinterpret_cast<float4 *>(smem2d);                  // [kPad2d]
    float2 *s_E = reinterpret_cast<float2 *>(s_v + kPad2d);            // [kWin2d]
    int32_t *s_c = reinterpret_cast<int32_t *>(s_E + kWin2d);          // [kPad2d]
    float *s_z = reinterpret_cast<float *>(s_c + kPad2d);              // [kPad2d]
    unsigned *s_lo = reinterpret_cast<unsigned *>(s_z + kPad2d);       // [kWin2d]
    unsigned *s_hi = s_lo + kWin2d;                                    // [kWin2d]
    __shared__ int s_ref, s_box[4];  // reference cell; min dx, -max dx, min dy, -max dy
    __shared__ unsigned s_abs[2];

    const int s = blockIdx.y;
    const Species2D &sp = p.sp[s];
    const long long step = *(volatile long long *)&p.st->step;
    const int P = (int)(step & 1);
    const long long n = (long long)p.st->count[s][P];
    const int32_t *__restrict__ cin = sp.cell[P];
    const float4 *__restrict__ vin = sp.pv[P];
    const float *__restrict__ zin = sp.vz[P];
    int32_t *__restrict__ cout = sp.cell[P ^ 1];
    float4 *__restrict__ vout = sp.pv[P ^ 1];
    float *__restrict__ zout = sp.vz[P ^ 1];
    unsigned long long *acc = p.acc + (size_t)s * p.nn;
    const int nx = p.nx, ny = p.ny;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x < 2)
        s_abs[threadIdx.x] = 0u;
    unsigned na0 = 0, na1 = 0;

    const long long nchunks = (n + kChunk2d - 1) / kChunk2d;
    for (long long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const long long base = ch * kChunk2d;
        const int cnt = (int)min((long long)kChunk2d, n - base);
        // ---- 1. the chunk into shared memory
        for (int j = threadIdx.x; j < kChunk2d; j += kT2d) {
            const int q = pad2d(j);
            if (j < cnt) {
                s_c[q] = __ldcs(cin + base + j);
                s_v[q] = __ldcs(vin + base + j);
                s_z[q] = __ldcs(zin + base + j);
            } else {
                s_c[q] = -1;
            }
        }
        if (threadIdx.x == 0) {
            s_box[0] = s_box[1] = s_box[2] = s_box[3] = INT_MAX;
            s_ref = -1;
        }
        __syncthreads();
        // ---- 2. the reference cell (a live particle at or after the middle, else
        // before it) and the box of the chunk's cells relative to it
        if (threadIdx.x == 0) {
            int r = -1;
            for (int j = cnt / 2; j < cnt && r < 0; ++j)
                r = s_c[pad2d(j)];
            for (int j = cnt / 2 - 1; j >= 0 && r < 0; --j)
                r = s_c[pad2d(j)];
            s_ref = r;
        }
        __syncthreads();
        const int ref = s_ref;
        if (ref < 0) {  // nothing live: the holes stay holes
            for (int j = threadIdx.x; j < cnt; j += kT2d)
                __stcs(cout + base + j, -1);
            __syncthreads();
            continue;
        }
        const int ry = div_nx(p, ref), rx = ref - ry * nx;
        {
            int mnx = INT_MAX, mxx = INT_MAX, mny = INT_MAX, mxy = INT_MAX;  // max as -min
            for (int k = 0; k < kPer2d; ++k) {
                const int c = s_c[pad2d(k * kT2d + threadIdx.x)];
                if (c >= 0) {
                    const int cy = div_nx(p, c);
                    int dx = c - cy * nx - rx;  // to [-nx/2, nx/2)
                    if (dx >= nx - nx / 2)
                        dx -= nx;
                    else if (dx < -(nx / 2))
                        dx += nx;
                    const int dy = cy - ry;
                    mnx = min(mnx, dx);
                    mxx = min(mxx, -dx);
                    mny = min(mny, dy);
                    mxy = min(mxy, -dy);
                }
            }
            mnx = __reduce_min_sync(0xffffffffu, mnx);
            mxx = __reduce_min_sync(0xffffffffu, mxx);
            mny = __reduce_min_sync(0xffffffffu, mny);
            mxy = __reduce_min_sync(0xffffffffu, mxy);
            if (lane == 0) {
                atomicMin(&s_box[0], mnx);
                atomicMin(&s_box[1], mxx);
                atomicMin(&s_box[2], mny);
                atomicMin(&s_box[3], mxy);
            }
        }
        __syncthreads();
        // ---- 3. the window: node columns wx0 .. wx0+ww-1 (modulo nx), rows wy0 ..
        // wy0+wh-1, covering the box widened by the gather's node and one cell of
        // motion each way (cut to kWin2d nodes; particles outside it go to global memory)
        int ww = (-s_box[1]) - s_box[0] + 4;
        int wx0 = rx + s_box[0] - 1;
        const int wy0 = max(0, ry + s_box[2] - 1);
        int wh = min(ny, ry - s_box[3] + 2) - wy0 + 1;
        if (ww >= nx) {
            ww = nx;
            wx0 = 0;
        }
        wx0 %= nx;
        if (wx0 < 0)
            wx0 += nx;
        if (ww > kWin2d / 2)
            ww = kWin2d / 2;
        if (ww * wh > kWin2d)
            wh = kWin2d / ww;
        // a warp per window row, a lane per column
        for (int iy = warp; iy < wh; iy += kT2d / 32) {
            const float2 *Er = p.E + (size_t)(wy0 + iy) * nx;
            for (int ix = lane; ix < ww; ix += 32) {
                const int gx = wx0 + ix < nx ? wx0 + ix : wx0 + ix - nx;
                const int k = iy * ww + ix;
                s_E[k] = __ldg(Er + gx);
                s_lo[k] = 0u;
                s_hi[k] = 0u;
            }
        }
        __syncthreads();
        // ---- 4. the particles, lanes of a warp 64 slots apart
#pragma unroll 1
        for (int k = 0; k < kPer2d; ++k) {
            const int j = lane * 64 + warp * kPer2d + k;
            const int q = pad2d(j);
            const int c = j < cnt ? s_c[q] : -1;
            if (c < 0)
                continue;
            const float4 pv = s_v[q];
            const float z = s_z[q];
            const int cy = div_nx(p, c), cx = c - cy * nx;
            int ix = cx - wx0;
            if (ix < 0)
                ix += nx;
            const int iy = cy - wy0;
            float2 e00, e10, e01, e11;
            if (ix <= ww - 2 && iy >= 0 && iy <= wh - 2) {
                const int k00 = iy * ww + ix;
                e00 = s_E[k00];
                e10 = s_E[k00 + 1];
                e01 = s_E[k00 + ww];
                e11 = s_E[k00 + ww + 1];
            } else {
                const int cx1 = (cx + 1 == nx) ? 0 : cx + 1;
                const int k00 = cy * nx + cx, k10 = cy * nx + cx1;
                e00 = __ldg(p.E + k00);
                e10 = __ldg(p.E + k10);
                e01 = __ldg(p.E + k00 + nx);
                e11 = __ldg(p.E + k10 + nx);
            }
            const float ox = pv.x, oy = pv.y;
            const float wx0f = __fsub_rn(1.0f, ox), wy0f = __fsub_rn(1.0f, oy);
            const float ex = __fadd_rn(
                __fmul_rn(wy0f, __fadd_rn(__fmul_rn(wx0f, e00.x), __fmul_rn(ox, e10.x))),
                __fmul_rn(oy, __fadd_rn(__fmul_rn(wx0f, e01.x), __fmul_rn(ox, e11.x))));
            const float ey = __fadd_rn(
                __fmul_rn(wy0f, __fadd_rn(__fmul_rn(wx0f, e00.y), __fmul_rn(ox, e10.y))),
                __fmul_rn(oy, __fadd_rn(__fmul_rn(wx0f, e01.y), __fmul_rn(ox, e11.y))));
            const float axp = __fmul_rn(sp.qm, ex), ayp = __fmul_rn(sp.qm, ey);
            float vx, vy;
            if (!push_v2_easy(sp.kind, pv.z, pv.w, z, axp, ayp, p.dt, sp.v0, vx, vy)) {
                // the piece walk: listed for k_hard2d, which pushes it and writes its
                // slot (pushed here once the list is full)
                namespace cg = cooperative_groups;
                cg::coalesced_group g = cg::coalesced_threads();
                unsigned long long hb = 0;
                if (g.thread_rank() == 0)
                    hb = atomicAdd(&p.st->hard_n[s], (unsigned long long)g.size());
                hb = g.shfl(hb, 0) + g.thread_rank();
                if ((long long)hb < sp.hard_cap) {
                    int4 *r = reinterpret_cast<int4 *>(sp.hard + hb);
                    r[0] = make_int4((int)(base + j), c, __float_as_int(axp), __float_as_int(ayp));
                    r[1] = make_int4(__float_as_int(pv.x), __float_as_int(pv.y),
                                     __float_as_int(pv.z), __float_as_int(pv.w));
                    r[2] = make_int4(__float_as_int(z), 0, 0, 0);
                    s_c[q] = -2;  // its slot is k_hard2d's
                    continue;
                }
                push_v2(sp.kind, pv.z, pv.w, z, axp, ayp, p.dt, sp.v0, vx, vy);
            }
            // x^{n+1} = x^n + beta(|v^{n+1/2}|) v^{n+1/2} dt, in cell units
            const float b = beta_q(sp.kind, vx, vy, z, sp.v0);
            int ncx, ncy;
            float dxn, dyn;
            const int wall = move2d(p, cx, cy, ox, oy, vx, vy, b, ncx, ncy, dxn, dyn);
            if (wall == 0) {
                ++na0;
                s_c[q] = -1;
            } else if (wall == 1) {
                ++na1;
                s_c[q] = -1;
            } else {
                unsigned long long q00, q10, q01, q11;
                quantise2d(b, dxn, dyn, q00, q10, q01, q11);
                int nix = ncx - wx0;
                if (nix < 0)
                    nix += nx;
                const int niy = ncy - wy0;
                if (nix <= ww - 2 && niy >= 0 && niy <= wh - 2) {
                    const int k00 = niy * ww + nix;
                    win_add(s_lo, s_hi, k00, q00);
                    win_add(s_lo, s_hi, k00 + 1, q10);
                    win_add(s_lo, s_hi, k00 + ww, q01);
                    win_add(s_lo, s_hi, k00 + ww + 1, q11);
                } else {
                    const int ncx1 = (ncx + 1 == nx) ? 0 : ncx + 1;
                    const int m00 = ncy * nx + ncx, m10 = ncy * nx + ncx1;
                    atomicAdd(acc + m00, q00);
                    atomicAdd(acc + m10, q10);
                    atomicAdd(acc + m00 + nx, q01);
                    atomicAdd(acc + m10 + nx, q11);
                }
                s_c[q] = ncy * nx + ncx;
                s_v[q] = make_float4(dxn, dyn, vx, vy);
            }
        }
        __syncthreads();
        // ---- 5. the window's deposits to acc, the chunk to its slots
        for (int iy = warp; iy < wh; iy += kT2d / 32) {
            unsigned long long *ar = acc + (size_t)(wy0 + iy) * nx;
            for (int ix = lane; ix < ww; ix += 32) {
                const int k = iy * ww + ix;
                const unsigned long long v = ((unsigned long long)s_hi[k] << 32) + s_lo[k];
                if (v)
                    atomicAdd(ar + (wx0 + ix < nx ? wx0 + ix : wx0 + ix - nx), v);
            }
        }
        for (int j = threadIdx.x; j < cnt; j += kT2d) {
            const int q = pad2d(j);
            const int c = s_c[q];
            if (c == -2)
                continue;  // listed for k_hard2d
            __stcs(cout + base + j, c);
            if (c >= 0) {
                __stcs(vout + base + j, s_v[q]);
                __stcs(zout + base + j, s_z[q]);
            }
        }
        __syncthreads();
    }
    na0 = __reduce_add_sync(0xffffffffu, na0);
    na1 = __reduce_add_sync(0xffffffffu, na1);
    if (lane == 0) {
        if (na0)
            atomicAdd(&s_abs[0], na0);
        if (na1)
            atomicAdd(&s_abs[1], na1);
    }
    __syncthreads();
    if (threadIdx.x < 2 && s_abs[threadIdx.x])
        atomicAdd(&p.st->absorbed_step[s][threadIdx.x], (unsigned long long)s_abs[threadIdx.x]);
}

// The particles the tile kernel listed: the full push (series or piece walk, the
// arithmetic of the inline push), the move, the plates and the deposit by global
// atomics; each writes its own slot.  The species' lists are one index space.
__global__ void __launch_bounds__(256) k_hard2d(Params2D p)
{
    __shared__ unsigned s_abs[kMaxS][2];
    if (threadIdx.x < 2 * kMaxS)
        s_abs[threadIdx.x >> 1][threadIdx.x & 1] = 0u;
    __syncthreads();
    const long long step = *(volatile long long *)&p.st->step;
    const int P = (int)(step & 1);
    long long pre[kMaxS + 1];  // registers: constant indices only
    pre[0] = 0;
#pragma unroll
    for (int s = 0; s < kMaxS; ++s) {
        const long long n = s < p.ns ? (long long)*(volatile unsigned long long *)&p.st->hard_n[s] : 0;
        pre[s + 1] = pre[s] + (s < p.ns ? min(n, p.sp[s].hard_cap) : 0);
    }
    const long long total = pre[kMaxS];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int s = 0;
        long long i0 = 0;
#pragma unroll
        for (int r = 1; r < kMaxS; ++r)
            if (t >= pre[r]) {
                s = r;
                i0 = pre[r];
            }
        const Species2D &sp = p.sp[s];
        const int4 *rec = reinterpret_cast<const int4 *>(sp.hard + (t - i0));
        const int4 r0 = __ldcs(rec), r1 = __ldcs(rec + 1), r2 = __ldcs(rec + 2);
        const int slot = r0.x, c = r0.y;
        const float ax = __int_as_float(r0.z), ay = __int_as_float(r0.w);
        const float ox = __int_as_float(r1.x), oy = __int_as_float(r1.y);
        const float ux = __int_as_float(r1.z), uy = __int_as_float(r1.w), z = __int_as_float(r2.x);
        float vx, vy;
        push_v2(sp.kind, ux, uy, z, ax, ay, p.dt, sp.v0, vx, vy);
        const float b = beta_q(sp.kind, vx, vy, z, sp.v0);
        const int cy = div_nx(p, c), cx = c - cy * p.nx;
        int ncx, ncy;
        float dxn, dyn;
        const int wall = move2d(p, cx, cy, ox, oy, vx, vy, b, ncx, ncy, dxn, dyn);
        if (wall >= 0) {
            atomicAdd(&s_abs[s][wall], 1u);
            sp.cell[P ^ 1][slot] = -1;
        } else {
            const int nx = p.nx;
            const int ncx1 = (ncx + 1 == nx) ? 0 : ncx + 1;
            const int m00 = ncy * nx + ncx, m10 = ncy * nx + ncx1;
            deposit2d(p.acc + (size_t)s * p.nn, m00, m10, m00 + nx, m10 + nx, b, dxn, dyn);
            sp.cell[P ^ 1][slot] = m00;
            sp.pv[P ^ 1][slot] = make_float4(dxn, dyn, vx, vy);
            sp.vz[P ^ 1][slot] = z;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * kMaxS) {
        const int s = threadIdx.x >> 1, w = threadIdx.x & 1;
        if (s < p.ns && s_abs[s][w])
            atomicAdd(&p.st->absorbed_step[s][w], (unsigned long long)s_abs[s][w]);
    }
}

// rho^0 from the particles of the current buffer (after a load)
__global__ void __launch_bounds__(kThreads) k_deposit2d(Params2D p)
{
    const int s = blockIdx.y;
    const Species2D &sp = p.sp[s];
    const int P = (int)(p.st->step & 1);
    const long long n = (long long)p.st->count[s][P];
    unsigned long long *acc = p.acc + (size_t)s * p.nn;
    const int nx = p.nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = sp.cell[P][i];
        if (c < 0)
            continue;
        const float4 q = sp.pv[P][i];
        const int cy = c / nx, cx = c - cy * nx;
        const int cx1 = (cx + 1 == nx) ? 0 : cx + 1;
        const int k00 = cy * nx + cx, k10 = cy * nx + cx1;
        deposit2d(acc, k00, k10, k00 + nx, k10 + nx, beta_q(sp.kind, q.z, q.w, sp.vz[P][i], sp.v0),
                  q.x, q.y);
    }
}

// ---------------------------------------------------------------------------------
// Source (the 1D volume source with its band across y, x uniform over the period)
// and the step's bookkeeping.  Particle i of species s draws
// u_j = u24(SplitMix64(key(seed, step, s), 8i + j)): y = lo + u_0 len, x = u_5 nx (cells,
// FP32), a physical Maxwellian velocity from u_1..u_4 (Box-Muller).
// ---------------------------------------------------------------------------------
// The step's source count of species s (thread s): macroparticles k to make (cut to
// the room left; cut = true if it was), the first slot and the carried fraction.
__device__ __forceinline__ void source_count2d(const Params2D &p, const State2D *st, int s, int P,
                                               int compact, long long &k, long long &base,
                                               double &frac, bool &cut)
{
    double S = 0.0;
    if (p.src_mode == SLPIC_SRC_LOSS_MATCHED) {
        const int r = p.src_ref;
        S = (double)(st->absorbed_step[r][0] + st->absorbed_step[r][1]) * p.sp[r].w;
    } else if (p.src_mode == SLPIC_SRC_RATE) {
        S = p.src_rate * p.dt64;
    }
    k = 0;
    double f = st->src_frac[s];
    if (p.src_mode != SLPIC_SRC_NONE && p.sp[s].vth_src > 0.0f) {
        f = fma(S, p.sp[s].inv_w, f);
        k = (long long)floor(f);
        f -= (double)k;
    }
    // in place: the output uses the input's slots; compacted: counted by atomics
    base = (long long)(compact ? st->count[s][P ^ 1] : st->count[s][P]);
    const long long room = p.sp[s].capacity - base;
    cut = k > room;
    if (cut)
        k = room;
    frac = f;
}

// Every CTA derives the step's counts from the same state and makes its share of the
// species' particles, taken as one index space; k_book2d then updates the state.
__global__ void __launch_bounds__(256) k_inject2d(Params2D p, int compact)
{
    __shared__ long long s_k[kMaxS], s_base[kMaxS];
    const State2D *st = p.st;
    const long long step = st->step;
    const int P = (int)(step & 1);
    const int ns = p.ns;
    if ((int)threadIdx.x < kMaxS) {
        const int s = threadIdx.x;
        long long k = 0, base = 0;
        double f;
        bool cut;
        if (s < ns)
            source_count2d(p, st, s, P, compact, k, base, f, cut);
        s_k[s] = k;
        s_base[s] = base;
    }
    __syncthreads();
    long long pre[kMaxS + 1];  // registers: constant indices only
    pre[0] = 0;
#pragma unroll
    for (int s = 0; s < kMaxS; ++s)
        pre[s + 1] = pre[s] + s_k[s];
    const long long total = pre[kMaxS];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        int s = 0;
        long long i0 = 0;
#pragma unroll
        for (int r = 1; r < kMaxS; ++r)
            if (t >= pre[r]) {
                s = r;
                i0 = pre[r];
            }
        const long long i = t - i0;
        const Species2D &sp = p.sp[s];
        const unsigned long long key = sm64_stream(p.seed, (unsigned long long)step, (unsigned)s);
        unsigned long long *acc = p.acc + (size_t)s * p.nn;
        const unsigned long long b8 = 8ULL * (unsigned long long)i;
        const float u0 = u24(sm64_at(key, b8 + 0)), u1 = u24(sm64_at(key, b8 + 1));
        const float u2 = u24(sm64_at(key, b8 + 2)), u3 = u24(sm64_at(key, b8 + 3));
        const float u4 = u24(sm64_at(key, b8 + 4)), u5 = u24(sm64_at(key, b8 + 5));
        const float yc = __fadd_rn(p.src_lo, __fmul_rn(u0, p.src_len));
        float xc = __fmul_rn(u5, (float)p.nx);
        if (xc >= (float)p.nx)
            xc = 0.0f;
        const float fx = floorf(xc), fy = floorf(yc);
        const int cx = (int)fx, cy = min(max((int)fy, 0), p.ny - 1);
        const float ox = __fsub_rn(xc, fx), oy = __fsub_rn(yc, fy);
        const float r1 = sqrtf(-2.0f * logf(u1)), r2 = sqrtf(-2.0f * logf(u3));
        float s2, c2;
        sincospif(2.0f * u2, &s2, &c2);
        const float vx = sp.vth_src * r1 * c2, vy = sp.vth_src * r1 * s2;
        const float vz = sp.vth_src * r2 * cospif(2.0f * u4);
        const long long o = s_base[s] + i;
        const int c = cy * p.nx + cx;
        sp.cell[P ^ 1][o] = c;
        sp.pv[P ^ 1][o] = make_float4(ox, oy, vx, vy);
        sp.vz[P ^ 1][o] = vz;
        const int cx1 = (cx + 1 == p.nx) ? 0 : cx + 1;
        deposit2d(acc, c, cy * p.nx + cx1, c + p.nx, cy * p.nx + cx1 + p.nx,
                  beta_q(sp.kind, vx, vy, vz, sp.v0), ox, oy);
    }
}

// The step's bookkeeping, after the source (one warp; thread s for species s, from
// the same counts as k_inject2d); the step index last.
__global__ void k_book2d(Params2D p, int compact)
{
    State2D *st = p.st;
    const long long step = st->step;
    const int P = (int)(step & 1);
    if ((int)threadIdx.x < p.ns) {
        const int s = threadIdx.x;
        long long k, base;
        double f;
        bool cut;
        source_count2d(p, st, s, P, compact, k, base, f, cut);
        if (cut)
            atomicCAS(&st->error, 0, SLPIC_ERR_CAPACITY);
        const unsigned long long a0 = st->absorbed_step[s][0], a1 = st->absorbed_step[s][1];
        st->src_frac[s] = f;
        st->holes[s][P ^ 1] = compact ? 0ULL : st->holes[s][P] + a0 + a1;
        st->count[s][P ^ 1] = (unsigned long long)(base + k);
        st->injected_total[s] += k;
        st->absorbed_total[s][0] += (long long)a0;
        st->absorbed_total[s][1] += (long long)a1;
        st->absorbed_step[s][0] = 0ULL;
        st->absorbed_step[s][1] = 0ULL;
        st->count[s][P] = 0ULL;
        st->holes[s][P] = 0ULL;
    }
    __syncwarp();
    if (threadIdx.x == 0) {
        unsigned long long it = 0;
        for (int s = 0; s < p.ns; ++s)
            it += st->hard_n[s];
        st->iter_last = it;
    }
    __syncwarp();
    if ((int)threadIdx.x < p.ns)
        st->hard_n[threadIdx.x] = 0ULL;
    if (threadIdx.x == 0)
        st->step = step + 1;
}

// ---------------------------------------------------------------------------------
// Field solve.  The unknowns are phi on rows j = 1..ny-1; with A the 5-point
// stencil times dx^2 (diagonal 4) and the plates moved to the right-hand side,
// A phi = b = (dx^2/eps0) rho + [j = 1] phi_lo + [j = ny-1] phi_hi.  Jacobi-
// preconditioned CG (M = 4 I) from the previous phi:
//   r = b - A phi, p = r/4, rz = r.r/4
//   loop: q = A p; alpha = rz / p.q; phi += alpha p; r -= alpha q;
//         stop if r.r <= rtol^2 b.b; p = r/4 + (r.r/4 / rz) p
// Each iteration is two grid-wide phases: (p, q = A p, p.q) and (phi, r, r.r), the
// new p formed on the fly from r and the previous p (two p buffers).  Dot products
// are FP64 per-CTA partial sums, added in CTA order by every CTA: the same value
// everywhere and in every run.
// ---------------------------------------------------------------------------------

// Grid barrier for a cooperative launch (all CTAs co-resident), two levels: CTAs
// arrive on the counter of their group of kBarGroup, the last of each group on the
// root counter, and the last of all advances the generation the others wait on
// (each counter is reset by its last arriver before the generation moves).  The
// wait is bounded: past kBarrierSpins polls the kernel records SLPIC_ERR_TIMEOUT
// and every CTA leaves at its next check.
__device__ __forceinline__ bool grid_sync(State2D *st)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &st->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        const unsigned grp = blockIdx.x / kBarGroup;
        const unsigned ngrp = (gridDim.x + kBarGroup - 1) / kBarGroup;
        const unsigned in_grp = min((unsigned)kBarGroup, gridDim.x - grp * kBarGroup);
        bool last = false;
        if (atomicAdd(&st->bar_group[grp], 1u) == in_grp - 1) {
            st->bar_group[grp] = 0u;
            __threadfence();
            if (atomicAdd(&st->bar_count, 1u) == ngrp - 1) {
                st->bar_count = 0u;
                __threadfence();
                atomicAdd(&st->bar_gen, 1u);
                last = true;
            }
        }
        if (!last) {
            long long spins = 0;
            while (*gen == g) {
                if (++spins > kBarrierSpins) {
                    atomicCAS(&st->error, 0, SLPIC_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        // one decision per CTA, so that its threads leave or stay together
        s_ok = *(volatile int *)&st->error != SLPIC_ERR_TIMEOUT;
    }
    __syncthreads();
    return s_ok != 0;
}

// block sum of v (FP64, fixed order), result valid in every thread
__device__ __forceinline__ double block_sum(double v, double *s_red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0)
        s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        t += s_red[w];
    return t;
}

// sum of the CTAs' partials, in CTA order
__device__ __forceinline__ double grid_total(const double *part, double *s_red)
{
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        v += __ldcg(part + b);
    // fixed assignment of CTAs to threads and a fixed tree: the same in every CTA
    return block_sum(v, s_red);
}

// Arrays written by other CTAs of the cooperative grid are read with __ldcg
// (L2, not the CTA's own L1).
__device__ __forceinline__ double stencil(const double *u, int idx, int i, int nx)
{
    const int ip = (i + 1 == nx) ? idx + 1 - nx : idx + 1;
    const int im = (i == 0) ? idx - 1 + nx : idx - 1;
    return 4.0 * __ldcg(u + idx) -
           (__ldcg(u + ip) + __ldcg(u + im) + __ldcg(u + idx - nx) + __ldcg(u + idx + nx));
}

// E = -grad phi at node idx: centred differences, one-sided on the plates, periodic
// in x.  phi is read through L2 (written by other CTAs of the same grid).
__device__ __forceinline__ void store_E(const Params2D &p, int idx)
{
    const int nx = p.nx, ny = p.ny;
    const int j = idx / nx, i = idx - j * nx;
    const int ip = (i + 1 == nx) ? idx + 1 - nx : idx + 1;
    const int im = (i == 0) ? idx - 1 + nx : idx - 1;
    const double *f = p.phi;
    const double ex = -(__ldcg(f + ip) - __ldcg(f + im)) * (0.5 / p.dx);
    double ey;
    if (j == 0)
        ey = -(__ldcg(f + idx + nx) - __ldcg(f + idx)) / p.dx;
    else if (j == ny)
        ey = -(__ldcg(f + idx) - __ldcg(f + idx - nx)) / p.dx;
    else
        ey = -(__ldcg(f + idx + nx) - __ldcg(f + idx - nx)) * (0.5 / p.dx);
    p.E[idx] = make_float2((float)ex, (float)ey);
}

// mode 0: the simulation's solve (b from the deposits, which are then cleared;
// E written).  mode 1: b from p.r's initial content as rho (slpic2d_solve_poisson).
//
// Mixed precision with reliable updates: b and the solution phi are FP64; the CG
// iterates (search direction p, correction d, residual r) are FP32, with dot
// products summed in FP64.  Whenever the FP32 recursive residual has fallen by
// kUpdateDrop since the last update (or below the target), d is added to phi in
// FP64 and r is replaced by the true residual b - A phi formed in FP64; the search
// direction carries on, so the iteration keeps the convergence of one unbroken CG
// run, unless the true residual came out more than twice the recursive one (the
// FP32 recursion had drifted), when the search direction starts afresh.  At
// 1024 x 1024 with a plasma's smooth charge the correction is as large as phi
// itself early on, which limits how far an FP32 recursion can be trusted: hence
// an update at every tenfold drop.  The solve ends when that true residual meets ||b - A phi|| <= rtol ||b||,
// the figure reported.  FP64 arithmetic, narrow on this GPU, is left to the few
// updates.
constexpr double kUpdateDrop = 1e-1;

__global__ void __launch_bounds__(kCgThreads) k_cg2d(Params2D p, int mode)
{
    __shared__ double s_red[kCgThreads / 32];
    State2D *st = p.st;
    const int nx = p.nx, ny = p.ny, nn = p.nn;
    const int first = nx, last = ny * nx;  // interior nodes [first, last)
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    double *part0 = p.part, *part1 = p.part + gridDim.x, *part2 = p.part + 2 * gridDim.x;
    double *b64 = p.q;  // right-hand side, kept for the true residuals

    // ---- b (FP64, interior rows; 0 on the plates) and ||b||^2; FP32 iterates zeroed
    double bb = 0.0;
    for (long long t = gtid; t < nn; t += gstride) {
        const int idx = (int)t;
        const int j = idx / nx;
        double rho = 0.0;
        if (mode == 0) {
            for (int s = 0; s < p.ns; ++s) {
                unsigned long long *a = p.acc + (size_t)s * nn + idx;
                rho = fma(p.sp[s].rho_unit, (double)(long long)*a, rho);
                *a = 0ULL;
            }
        } else {
            rho = p.r[idx];
        }
        double b = 0.0;
        if (idx >= first && idx < last) {
            b = p.k2 * rho;
            if (j == 1)
                b += p.phi_lo;
            if (j == ny - 1)
                b += p.phi_hi;
        }
        b64[idx] = b;
        bb = fma(b, b, bb);
        p.fr[idx] = 0.0f;
        p.fpA[idx] = 0.0f;
        p.fpB[idx] = 0.0f;
        p.fd[idx] = 0.0f;
    }
    bb = block_sum(bb, s_red);
    if (threadIdx.x == 0)
        part0[blockIdx.x] = bb;
    if (!grid_sync(st))
        return;
    double BB = grid_total(part0, s_red);
    if (BB == 0.0)
        BB = 1.0;

    int it = 0;
    double RR = 0.0;
    // true residual in FP64: r = b - A phi (A phi on the unknowns = the full stencil
    // on phi, plate rows included, plus the plate terms held in b), stored in FP32
    auto true_residual = [&]() -> bool {
        double rr = 0.0;
        for (long long t = gtid + first; t < last; t += gstride) {
            const int idx = (int)t;
            const int j = idx / nx, i = idx - j * nx;
            double ap = stencil(p.phi, idx, i, nx);
            if (j == 1)
                ap += p.phi_lo;
            if (j == ny - 1)
                ap += p.phi_hi;
            const double r = __ldcg(b64 + idx) - ap;
            p.fr[idx] = (float)r;
            rr = fma(r, r, rr);
        }
        rr = block_sum(rr, s_red);
        if (threadIdx.x == 0)
            part1[blockIdx.x] = rr;
        if (!grid_sync(st))
            return false;
        RR = grid_total(part1, s_red);
        return true;
    };
    if (!true_residual())
        return;
    bool done = RR <= p.rtol2 * BB;
    double rz = 0.25 * RR, beta = 0.0, rin = RR, rlast = RR;
    bool restart = false;
    float *pold = p.fpA, *pnew = p.fpB;
    while (!done && it < p.cg_maxit) {
        // phase 1: p = r/4 + beta p_old at the node and its neighbours, q = A p
        const float bf = (float)beta;
        double pq = 0.0;
        for (long long t = gtid + first; t < last; t += gstride) {
            const int idx = (int)t;
            const int j = idx / nx, i = idx - j * nx;
            const int ip = (i + 1 == nx) ? idx + 1 - nx : idx + 1;
            const int im = (i == 0) ? idx - 1 + nx : idx - 1;
            const float pc = fmaf(bf, __ldcg(pold + idx), 0.25f * __ldcg(p.fr + idx));
            const float pe = fmaf(bf, __ldcg(pold + ip), 0.25f * __ldcg(p.fr + ip));
            const float pw = fmaf(bf, __ldcg(pold + im), 0.25f * __ldcg(p.fr + im));
            const float pn =
                (j + 1 < ny) ? fmaf(bf, __ldcg(pold + idx + nx), 0.25f * __ldcg(p.fr + idx + nx))
                             : 0.0f;
            const float ps =
                (j > 1) ? fmaf(bf, __ldcg(pold + idx - nx), 0.25f * __ldcg(p.fr + idx - nx)) : 0.0f;
            const float qv = 4.0f * pc - (pe + pw + pn + ps);
            pnew[idx] = pc;
            p.fq[idx] = qv;
            pq = fma((double)pc, (double)qv, pq);
        }
        const double pqs = block_sum(pq, s_red);
        if (threadIdx.x == 0)
            part2[blockIdx.x] = pqs;
        if (!grid_sync(st))
            return;
        const double alpha = rz / grid_total(part2, s_red);
        const float af = (float)alpha;
        // phase 2: d += alpha p, r -= alpha q
        double r2 = 0.0;
        for (long long t = gtid + first; t < last; t += gstride) {
            const int idx = (int)t;
            p.fd[idx] = fmaf(af, pnew[idx], p.fd[idx]);
            const float r = fmaf(-af, p.fq[idx], p.fr[idx]);
            p.fr[idx] = r;
            r2 = fma((double)r, (double)r, r2);
        }
        const double r2s = block_sum(r2, s_red);
        if (threadIdx.x == 0)
            part1[blockIdx.x] = r2s;
        if (!grid_sync(st))
            return;
        rin = grid_total(part1, s_red);
        ++it;
        if (rin <= kUpdateDrop * kUpdateDrop * rlast || rin <= 0.25 * p.rtol2 * BB ||
            it >= p.cg_maxit) {
            // reliable update: phi += d in FP64, r replaced by the true residual
            for (long long t = gtid + first; t < last; t += gstride) {
                const int idx = (int)t;
                p.phi[idx] += (double)p.fd[idx];
                p.fd[idx] = 0.0f;
            }
            if (!grid_sync(st))
                return;
            if (!true_residual())
                return;
            done = RR <= p.rtol2 * BB;
            // the FP32 recursion had drifted from the truth (true residual more than
            // twice the recursive one): its search direction is stale, start afresh
            restart = RR > 4.0 * rin;
            rin = RR;
            rlast = RR;
        }
        const double rz1 = 0.25 * rin;
        beta = restart ? 0.0 : rz1 / rz;
        restart = false;
        rz = rz1;
        float *tmp = pold;
        pold = pnew;
        pnew = tmp;
    }
    // E on every node from the final phi (complete after the last barrier)
    if (mode == 0)
        for (long long t = gtid; t < nn; t += gstride)
            store_E(p, (int)t);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->cg_iters = it;
        st->cg_total += it;
        st->cg_res = sqrt(RR / BB);
        if (!done)
            atomicCAS(&st->error, 0, SLPIC_ERR_NOCONVERGE);
    }
}

// ---- the direct solver (SLPIC2D_SOLVER_FFT) -----------------------------------------
// The 5-point system A phi = b on the interior rows j = 1..ny-1 is periodic in x,
// so the discrete Fourier transform along x diagonalises its x part: mode k of row
// j obeys (4 - 2 cos(2 pi k/nx)) u_j - u_{j-1} - u_{j+1} = b^_j with u_0 = u_ny = 0
// (the plate potentials are in b).  Three passes: a forward radix-2 FFT per row
// (one CTA per row, the row in shared memory, FP64), the Thomas algorithm per mode
// (one thread per k, the multipliers tabulated at creation), the inverse FFT per
// row.  Then E and the true residual as for the CG.
constexpr int kFftThreads = 256;

// in-place radix-2 FFT of x[0..n) held in bit-reversed order; sign -1 forward,
// +1 inverse (unnormalised)
__device__ void fft_smem(double2 *x, const double2 *__restrict__ tw, int n, double sign)
{
    for (int len = 2; len <= n; len <<= 1) {
        const int half = len >> 1, step = n / len;
        __syncthreads();
        for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
            const int g = b / half, pos = b - g * half;
            const int i0 = g * len + pos, i1 = i0 + half;
            const double2 w = tw[pos * step];
            const double wr = w.x, wi = sign * w.y;
            const double2 v = x[i1];
            const double tr = wr * v.x - wi * v.y, ti = wr * v.y + wi * v.x;
            const double2 u = x[i0];
            x[i0] = make_double2(u.x + tr, u.y + ti);
            x[i1] = make_double2(u.x - tr, u.y - ti);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double block_sum_fft(double v, double *s_red)
{
    for (int off = 16; off; off >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kFftThreads / 32; ++w)
            t += s_red[w];
    __syncthreads();
    return t;
}

// forward: b of row j (from the deposits, then cleared, in mode 0; from rho in p.r
// in mode 1) into p.q, its transform into p.spec; ||b_j||^2 into rpart
__global__ void __launch_bounds__(kFftThreads) k_fft_rows(Params2D p, int mode)
{
    extern __shared__ double2 sx[];
    __shared__ double s_red[kFftThreads / 32];
    const int nx = p.nx, ny = p.ny, j = blockIdx.x + 1;
    const int shift = 32 - p.log2nx;
    double bb = 0.0;
    for (int i = threadIdx.x; i < nx; i += kFftThreads) {
        const int idx = j * nx + i;
        double rho = 0.0;
        if (mode == 0) {
            for (int s = 0; s < p.ns; ++s) {
                unsigned long long *a = p.acc + (size_t)s * p.nn + idx;
                rho = fma(p.sp[s].rho_unit, (double)(long long)*a, rho);
                *a = 0ULL;
            }
            // the plate rows' deposits are consumed here too
            if (j == 1)
                for (int s = 0; s < p.ns; ++s)
                    p.acc[(size_t)s * p.nn + i] = 0ULL;
            if (j == ny - 1)
                for (int s = 0; s < p.ns; ++s)
                    p.acc[(size_t)s * p.nn + (size_t)ny * nx + i] = 0ULL;
        } else {
            rho = p.r[idx];
        }
        double b = p.k2 * rho;
        if (j == 1)
            b += p.phi_lo;
        if (j == ny - 1)
            b += p.phi_hi;
        p.q[idx] = b;
        bb = fma(b, b, bb);
        sx[__brev((unsigned)i) >> shift] = make_double2(b, 0.0);
    }
    const double bbs = block_sum_fft(bb, s_red);
    if (threadIdx.x == 0)
        p.rpart[2 * j + 1] = bbs;
    fft_smem(sx, p.tw, nx, -1.0);
    for (int k = threadIdx.x; k < nx; k += kFftThreads)
        p.spec[(size_t)j * nx + k] = sx[k];
}

// Thomas per mode k: forward u'_j = (b^_j + u'_{j-1}) / m_j, back u_j = u'_j + u_{j+1} / m_j
// (rows 1..ny-1), the multipliers 1/m_j tabulated.  Both are first-order linear
// recurrences, so each is solved in segments of L rows side by side: every segment
// from a zero start (x~), then the value entering each segment by a short sequential
// pass over the segments' ends, then x = x~ + P x_in with P the product of the
// segment's multipliers up to the row (tabulated: seg_f forward, seg_b backward).
// A CTA takes kTriModes modes (consecutive k: coalesced rows) times kTriSegs segments.
constexpr int kTriModes = 8;
constexpr int kTriSegs = 32;

__host__ __device__ __forceinline__ int tri_seg_len(int ny)
{
    return (ny - 1 + kTriSegs - 1) / kTriSegs;
}

__global__ void __launch_bounds__(kTriModes * kTriSegs) k_tridiag_modes(Params2D p)
{
    __shared__ double2 s_end[kTriSegs][kTriModes], s_in[kTriSegs][kTriModes];
    const int nx = p.nx, ny = p.ny;
    const int kk = threadIdx.x % kTriModes, sg = threadIdx.x / kTriModes;
    const int k = blockIdx.x * kTriModes + kk;
    const bool act = k < nx;
    const int L = tri_seg_len(ny);
    const int j0 = 1 + sg * L, j1 = min(ny, j0 + L);  // this segment's rows [j0, j1)
    double2 *__restrict__ spec = p.spec;
    const double *__restrict__ invm = p.inv_m;
    const double *__restrict__ pf = p.seg_f;
    const double *__restrict__ pb = p.seg_b;
    // 1. forward, from zero
    double2 x = make_double2(0.0, 0.0);
    if (act)
        for (int j = j0; j < j1; ++j) {
            const size_t o = (size_t)j * nx + k;
            const double2 v = spec[o];
            const double m = __ldg(invm + o);
            x = make_double2((v.x + x.x) * m, (v.y + x.y) * m);
            spec[o] = x;
        }
    s_end[sg][kk] = x;
    __syncthreads();
    // 2. the forward value entering each segment (a thread per mode)
    if (sg == 0 && act) {
        double2 c = make_double2(0.0, 0.0);
        for (int t = 0; t < kTriSegs; ++t) {
            s_in[t][kk] = c;
            const int e = min(ny, 1 + (t + 1) * L) - 1;  // the segment's last row
            if (1 + t * L <= e) {
                const double f = __ldg(pf + (size_t)e * nx + k);
                c = make_double2(fma(f, c.x, s_end[t][kk].x), fma(f, c.y, s_end[t][kk].y));
            }
        }
    }
    __syncthreads();
    // 3. the forward values completed, then the backward recurrence from zero, top down
    const double2 cf = s_in[sg][kk];
    double2 u = make_double2(0.0, 0.0);
    if (act)
        for (int j = j1 - 1; j >= j0; --j) {
            const size_t o = (size_t)j * nx + k;
            const double f = __ldg(pf + o);
            const double2 v = spec[o];
            const double2 d = make_double2(fma(f, cf.x, v.x), fma(f, cf.y, v.y));
            const double m = __ldg(invm + o);
            u = make_double2(fma(u.x, m, d.x), fma(u.y, m, d.y));
            spec[o] = u;
        }
    __syncthreads();  // every thread has read s_in
    s_end[sg][kk] = u;
    __syncthreads();
    // 4. the backward value entering each segment from above
    if (sg == 0 && act) {
        double2 c = make_double2(0.0, 0.0);
        for (int t = kTriSegs - 1; t >= 0; --t) {
            s_in[t][kk] = c;
            const int b0 = 1 + t * L;  // the segment's first row
            if (b0 <= min(ny, b0 + L) - 1) {
                const double g = __ldg(pb + (size_t)b0 * nx + k);
                c = make_double2(fma(g, c.x, s_end[t][kk].x), fma(g, c.y, s_end[t][kk].y));
            }
        }
    }
    __syncthreads();
    // 5. the backward values completed
    const double2 cb = s_in[sg][kk];
    if (act)
        for (int j = j0; j < j1; ++j) {
            const size_t o = (size_t)j * nx + k;
            const double g = __ldg(pb + o);
            const double2 w = spec[o];
            spec[o] = make_double2(fma(g, cb.x, w.x), fma(g, cb.y, w.y));
        }
}

// inverse: phi of row j from its coefficients
__global__ void __launch_bounds__(kFftThreads) k_ifft_rows(Params2D p)
{
    extern __shared__ double2 sx[];
    const int nx = p.nx, j = blockIdx.x + 1;
    const int shift = 32 - p.log2nx;
    for (int k = threadIdx.x; k < nx; k += kFftThreads)
        sx[__brev((unsigned)k) >> shift] = p.spec[(size_t)j * nx + k];
    fft_smem(sx, p.tw, nx, 1.0);
    const double inv = 1.0 / nx;
    for (int i = threadIdx.x; i < nx; i += kFftThreads)
        p.phi[(size_t)j * nx + i] = sx[i].x * inv;
}

// E on every node (mode 0) and the true residual r = b - A phi per row
__global__ void __launch_bounds__(kFftThreads) k_fft_finish(Params2D p, int mode)
{
    __shared__ double s_red[kFftThreads / 32];
    const int nx = p.nx, ny = p.ny, j = blockIdx.x;  // rows 0..ny
    double rr = 0.0;
    for (int i = threadIdx.x; i < nx; i += kFftThreads) {
        const int idx = j * nx + i;
        if (mode == 0)
            store_E(p, idx);
        if (j >= 1 && j < ny) {
            const int ip = (i + 1 == nx) ? idx + 1 - nx : idx + 1;
            const int im = (i == 0) ? idx - 1 + nx : idx - 1;
            const double *f = p.phi;
            double ap = 4.0 * f[idx] - (f[ip] + f[im]);
            if (j > 1)
                ap -= f[idx - nx];
            if (j < ny - 1)
                ap -= f[idx + nx];
            const double r = p.q[idx] - ap;
            rr = fma(r, r, rr);
        }
    }
    const double rrs = block_sum_fft(rr, s_red);
    if (threadIdx.x == 0)
        p.rpart[2 * j] = (j >= 1 && j < ny) ? rrs : 0.0;
}

// the per-row sums added in a fixed order (contiguous runs of rows per thread, then
// a fixed tree: the same result every run) and the bookkeeping of a solve
__global__ void __launch_bounds__(kFftThreads) k_fft_report(Params2D p)
{
    __shared__ double s_red[kFftThreads / 32];
    const int rows = p.ny - 1, per = (rows + kFftThreads - 1) / kFftThreads;
    double r = 0.0, b = 0.0;
    for (int q = 0; q < per; ++q) {
        const int j = 1 + threadIdx.x * per + q;
        if (j < p.ny) {
            r += p.rpart[2 * j];
            b += p.rpart[2 * j + 1];
        }
    }
    const double R = block_sum_fft(r, s_red);
    const double B = block_sum_fft(b, s_red);
    if (threadIdx.x != 0)
        return;
    State2D *st = p.st;
    st->cg_iters = 0;
    st->cg_res = B > 0.0 ? sqrt(R / B) : 0.0;
    if (B > 0.0 && R > p.rtol2 * B)
        atomicCAS(&st->error, 0, SLPIC_ERR_NOCONVERGE);
}

// ---- counting sort of the particles by cell ------------------------------------------
// Particles in cell order make the gather of E and the deposit atomics of
// neighbouring threads land on neighbouring nodes.  Three passes over the live
// particles of buffer `src`: a histogram per cell (lanes of a warp in the same cell
// add once, __match_any_sync), an exclusive scan of the histogram into each cell's
// first slot, and a scatter into buffer `dst` (a slot per particle by an atomic on
// its cell's cursor, again once per warp group).  The order within a cell is
// whatever the atomics give; nothing computed depends on it.
constexpr int kScanThreads = 1024, kScanPer = 4, kScanBlock = kScanThreads * kScanPer;

__global__ void __launch_bounds__(kThreads) k_sort_count2d(Params2D p, int s, int src)
{
    const Species2D &sp = p.sp[s];
    const long long n = (long long)p.st->count[s][src];
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long base = ((long long)blockIdx.x * kThreads + threadIdx.x) & ~31LL; base < n;
         base += stride) {
        const long long i = base + lane;
        const int c = i < n ? sp.cell[src][i] : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, c);
        if (c >= 0 && lane == __ffs(grp) - 1)
            atomicAdd(&p.hist[c], __popc(grp));
    }
}

// exclusive scan of hist[0..nn) into cursor: per block of kScanBlock entries, then
// the block totals, then their offsets added
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(Params2D p)
{
    __shared__ int s_w[kScanThreads / 32];
    const long long b0 = (long long)blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
    int v[kScanPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = b0 + k < p.nn ? p.hist[b0 + k] : 0;
        sum += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = s_w[lane];
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o)
                wi += y;
        }
        s_w[lane] = wi - w;  // exclusive over warps
        if (lane == 31)
            p.bsum[blockIdx.x] = wi;
    }
    __syncthreads();
    int run = s_w[warp] + incl - sum;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (b0 + k < p.nn)
            p.cursor[b0 + k] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_top(Params2D p, int nb)
{
    __shared__ int s_carry;
    __shared__ int s_w[kScanThreads / 32];
    if (threadIdx.x == 0)
        s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int i = b0 + threadIdx.x;
        const int v = i < nb ? p.bsum[i] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            s_w[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int w = s_w[lane];
            int wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o)
                    wi += y;
            }
            s_w[lane] = wi - w;
        }
        __syncthreads();
        const int carry = s_carry;
        if (i < nb)
            p.bsum[i] = carry + s_w[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1)
            s_carry = carry + s_w[warp] + incl;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_add(Params2D p)
{
    const long long i0 = (long long)blockIdx.x * kScanBlock;
    const int add = p.bsum[blockIdx.x];
    for (int k = threadIdx.x; k < kScanBlock; k += kScanThreads)
        if (i0 + k < p.nn)
            p.cursor[i0 + k] += add;
}

// the sorted buffer's slots: the end of the last cell's run; no holes
__global__ void k_sort_count_set(Params2D p, int s, int b)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        p.st->count[s][b] = (unsigned long long)p.cursor[p.nn - 1];
        p.st->holes[s][b] = 0ULL;
    }
}

__global__ void __launch_bounds__(kThreads) k_sort_scatter2d(Params2D p, int s, int src, int dst)
{
    const Species2D &sp = p.sp[s];
    const long long n = (long long)p.st->count[s][src];
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long base = ((long long)blockIdx.x * kThreads + threadIdx.x) & ~31LL; base < n;
         base += stride) {
        const long long i = base + lane;
        const int c = i < n ? sp.cell[src][i] : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, c);
        const int leader = __ffs(grp) - 1;
        int slot = 0;
        if (c >= 0 && lane == leader)
            slot = atomicAdd(&p.cursor[c], __popc(grp));
        slot = __shfl_sync(0xffffffffu, slot, leader);
        if (c >= 0) {
            const int o = slot + __popc(grp & ((1u << lane) - 1u));
            sp.cell[dst][o] = c;
            sp.pv[dst][o] = sp.pv[src][i];
            sp.vz[dst][o] = sp.vz[src][i];
        }
    }
}

// ---- initial guess of the CG (slpic2d_set_warm_start) ------------------------------
// rho of rows 0..ny-1 as FP32 from the deposits (left in place for the CG kernel);
// row 0, a plate, is zero.  The layout is the nodal one, so the array is the
// U-Net's (H, W) = (ny, nx) input.
__global__ void __launch_bounds__(kThreads) k_rho32(Params2D p, float *__restrict__ out)
{
    const long long n = (long long)p.ny * p.nx;
    for (long long t = (long long)blockIdx.x * kThreads + threadIdx.x; t < n;
         t += (long long)gridDim.x * kThreads) {
        double rho = 0.0;
        if (t >= p.nx)
            for (int s = 0; s < p.ns; ++s)
                rho = fma(p.sp[s].rho_unit, (double)(long long)p.acc[(size_t)s * p.nn + t], rho);
        out[t] = (float)rho;
    }
}

// x = a - b (the change of the charge image since the previous step)
__global__ void __launch_bounds__(kThreads) k_sub32(const float *__restrict__ a,
                                                  const float *__restrict__ b,
                                                  float *__restrict__ x, long long n)
{
    for (long long t = (long long)blockIdx.x * kThreads + threadIdx.x; t < n;
         t += (long long)gridDim.x * kThreads)
        x[t] = a[t] - b[t];
}

// phi += y on the interior rows (the previous potential plus the predicted change)
__global__ void __launch_bounds__(kThreads) k_guess_add(Params2D p, const float *__restrict__ y)
{
    const long long first = p.nx, last = (long long)p.ny * p.nx;
    for (long long t = first + (long long)blockIdx.x * kThreads + threadIdx.x; t < last;
         t += (long long)gridDim.x * kThreads)
        p.phi[t] += (double)y[t];
}

// phi on the interior rows = the straight line between the plate potentials plus
// y (the network's guess for the zero-plate problem), or the line alone when y is
// null (the zero guess).
__global__ void __launch_bounds__(kThreads) k_guess(Params2D p, const float *__restrict__ y)
{
    const long long first = p.nx, last = (long long)p.ny * p.nx;
    for (long long t = first + (long long)blockIdx.x * kThreads + threadIdx.x; t < last;
         t += (long long)gridDim.x * kThreads) {
        const int j = (int)(t / p.nx);
        double v = p.phi_lo + (p.phi_hi - p.phi_lo) * ((double)j / p.ny);
        if (y)
            v += (double)y[t];
        p.phi[t] = v;
    }
}

}  // namespace slpic2d

// =================================================================================
// C ABI
// =================================================================================
using namespace slpic2d;

struct slpic2d_sim {
    slpic2d_config cfg{};
    cudaStream_t stream = nullptr, own_stream = nullptr;
    Params2D p{};
    int ctas = 1;     // particle-kernel CTAs per species
    int tile_ctas = 0;  // k_particles2d_tiles CTAs per species (0: not resident)
    int small_ctas = 1; // k_hard2d and k_inject2d: 2 CTAs of 256 threads per SM
    int cg_ctas = 1;  // cooperative CG grid
    bool prepared = false;
    bool timing = false;               // record events around the kernels of each step
    std::vector<cudaEvent_t> events;   // 4 per recorded step
    long long t_steps = 0;             // steps recorded since the last read
    State2D *d_state = nullptr;
    int warm_mode = SLPIC2D_WARM_PREV;  // initial guess of each step's CG
    slpic_unet_t *net = nullptr;        // SLPIC2D_WARM_UNET: borrowed network
    float *rho32 = nullptr, *guess32 = nullptr;  // its input and output (ny * nx)
    float *rho32_prev = nullptr, *drho32 = nullptr;  // SLPIC2D_WARM_UNET_DELTA
    bool have_prev_rho = false;
    std::vector<void *> allocs;
    std::string err;
};

#define CK2(h, call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return SLPIC_ERR_CUDA;                                                         \
        }                                                                                  \
    } while (0)

static int fail2(slpic2d_t *h, int code, const std::string &msg)
{
    h->err = msg;
    return code;
}

static int device_status(slpic2d_t *h)
{
    CK2(h, cudaStreamSynchronize(h->stream));
    int e = 0;
    CK2(h, cudaMemcpy(&e, &h->d_state->error, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        const char *m = e == SLPIC_ERR_CAPACITY ? "particle store full: injection truncated"
                        : e == SLPIC_ERR_NOCONVERGE ? "CG did not reach cg_rtol within cg_maxit"
                        : e == SLPIC_ERR_TIMEOUT ? "grid barrier of the CG kernel timed out"
                                                 : "device error";
        return fail2(h, e, m);
    }
    return SLPIC_OK;
}

static int launch_cg(slpic2d_t *h, int mode)
{
    Params2D p = h->p;
    void *args[] = {&p, &mode};
    CK2(h, cudaLaunchCooperativeKernel((const void *)k_cg2d, dim3(h->cg_ctas), dim3(kCgThreads),
                                       args, 0, h->stream));
    return SLPIC_OK;
}

// The initial guess of the step's CG, on the handle's stream (SLPIC2D_WARM_PREV:
// phi as the previous step left it).
static int warm_start(slpic2d_t *h)
{
    const unsigned grid = (unsigned)std::min<long long>(
        ((long long)h->p.ny * h->p.nx + kThreads - 1) / kThreads, 152LL * 8);
    if (h->warm_mode == SLPIC2D_WARM_ZERO) {
        k_guess<<<grid, kThreads, 0, h->stream>>>(h->p, nullptr);
    } else if (h->warm_mode == SLPIC2D_WARM_UNET) {
        k_rho32<<<grid, kThreads, 0, h->stream>>>(h->p, h->rho32);
        CK2(h, cudaGetLastError());
        const int rc = slpic_unet_forward_on(h->net, 1, h->rho32, h->guess32, h->stream);
        if (rc)
            return fail2(h, rc, std::string("U-Net forward: ") + slpic_unet_last_error(h->net));
        k_guess<<<grid, kThreads, 0, h->stream>>>(h->p, h->guess32);
    } else if (h->warm_mode == SLPIC2D_WARM_UNET_DELTA) {
        // phi (still the previous step's) + net(rho - rho_prev); the first step
        // after a reset has no rho_prev and starts from the previous phi alone
        k_rho32<<<grid, kThreads, 0, h->stream>>>(h->p, h->rho32);
        CK2(h, cudaGetLastError());
        if (h->have_prev_rho) {
            const long long n = (long long)h->p.ny * h->p.nx;
            k_sub32<<<grid, kThreads, 0, h->stream>>>(h->rho32, h->rho32_prev, h->drho32, n);
            const int rc = slpic_unet_forward_on(h->net, 1, h->drho32, h->guess32, h->stream);
            if (rc)
                return fail2(h, rc, std::string("U-Net forward: ") + slpic_unet_last_error(h->net));
            k_guess_add<<<grid, kThreads, 0, h->stream>>>(h->p, h->guess32);
        }
        std::swap(h->rho32, h->rho32_prev);
        h->have_prev_rho = true;
    }
    CK2(h, cudaGetLastError());
    return SLPIC_OK;
}

extern "C" int slpic2d_set_warm_start(slpic2d_t *h, int32_t mode, slpic_unet_t *net)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    if (mode != SLPIC2D_WARM_PREV && mode != SLPIC2D_WARM_ZERO && mode != SLPIC2D_WARM_UNET &&
        mode != SLPIC2D_WARM_UNET_DELTA)
        return fail2(h, SLPIC_ERR_INVALID, "unknown warm-start mode");
    const bool uses_net = mode == SLPIC2D_WARM_UNET || mode == SLPIC2D_WARM_UNET_DELTA;
    if (uses_net) {
        if (!net)
            return fail2(h, SLPIC_ERR_INVALID, "this warm-start mode needs a network");
        int H, W, nb;
        slpic_unet_shape(net, &H, &W, &nb);
        if (H != h->p.ny || W != h->p.nx)
            return fail2(h, SLPIC_ERR_INVALID, "the network's grid must be (ny, nx)");
        if (!h->rho32) {
            const size_t n = (size_t)h->p.ny * h->p.nx;
            CK2(h, cudaMalloc(&h->rho32, sizeof(float) * n));
            h->allocs.push_back(h->rho32);
            CK2(h, cudaMalloc(&h->guess32, sizeof(float) * n));
            h->allocs.push_back(h->guess32);
            CK2(h, cudaMalloc(&h->rho32_prev, sizeof(float) * n));
            h->allocs.push_back(h->rho32_prev);
            CK2(h, cudaMalloc(&h->drho32, sizeof(float) * n));
            h->allocs.push_back(h->drho32);
        }
    }
    h->warm_mode = mode;
    h->net = uses_net ? net : nullptr;
    h->have_prev_rho = false;
    return SLPIC_OK;
}

// Sort every species' particles of buffer `src` by cell into buffer `dst` (holes
// dropped, the count set to the live particles), then swap the two buffers' roles,
// so that buffer index `src` names the sorted particles.
static int sort_particles(slpic2d_t *h, int src)
{
    Params2D &p = h->p;
    const int dst = src ^ 1;
    const unsigned nblk = (unsigned)((p.nn + kScanBlock - 1) / kScanBlock);
    for (int s = 0; s < p.ns; ++s) {
        CK2(h, cudaMemsetAsync(p.hist, 0, sizeof(int) * p.nn, h->stream));
        k_sort_count2d<<<h->ctas, kThreads, 0, h->stream>>>(p, s, src);
        k_scan_blocks<<<nblk, kScanThreads, 0, h->stream>>>(p);
        k_scan_top<<<1, kScanThreads, 0, h->stream>>>(p, (int)nblk);
        k_scan_add<<<nblk, kScanThreads, 0, h->stream>>>(p);
        k_sort_scatter2d<<<h->ctas, kThreads, 0, h->stream>>>(p, s, src, dst);
        k_sort_count_set<<<1, 32, 0, h->stream>>>(p, s, src);
        CK2(h, cudaGetLastError());
        std::swap(p.sp[s].cell[src], p.sp[s].cell[dst]);
        std::swap(p.sp[s].pv[src], p.sp[s].pv[dst]);
        std::swap(p.sp[s].vz[src], p.sp[s].vz[dst]);
    }
    return SLPIC_OK;
}

// The field solve of the configured solver (mode as for k_cg2d).
static int launch_solve(slpic2d_t *h, int mode)
{
    if (h->p.solver != SLPIC2D_SOLVER_FFT)
        return launch_cg(h, mode);
    const Params2D &p = h->p;
    const size_t smem = (size_t)16 * p.nx;
    k_fft_rows<<<p.ny - 1, kFftThreads, smem, h->stream>>>(p, mode);
    k_tridiag_modes<<<(p.nx + kTriModes - 1) / kTriModes, kTriModes * kTriSegs, 0, h->stream>>>(p);
    k_ifft_rows<<<p.ny - 1, kFftThreads, smem, h->stream>>>(p);
    k_fft_finish<<<p.ny + 1, kFftThreads, 0, h->stream>>>(p, mode);
    k_fft_report<<<1, kFftThreads, 0, h->stream>>>(p);
    CK2(h, cudaGetLastError());
    return SLPIC_OK;
}

extern "C" int slpic2d_create(const slpic2d_config *c, slpic2d_t **out)
{
    if (!c || !out) {
        slpic::set_create_error("null argument");
        return SLPIC_ERR_INVALID;
    }
    std::string why;
    if (c->nx < 2 || c->ny < 2 || !(c->dx > 0) || !(c->dt > 0) || !(c->eps0 > 0))
        why = "need nx >= 2, ny >= 2, dx > 0, dt > 0, eps0 > 0";
    else if ((long long)c->nx * (c->ny + 1) > (1LL << 30))
        why = "grid too large";
    else if (c->n_species < 1 || c->n_species > SLPIC_MAX_SPECIES)
        why = "n_species out of range";
    else if (!(c->cg_rtol > 0 && c->cg_rtol < 1) || c->cg_maxit <= 0)
        why = "need 0 < cg_rtol < 1 and cg_maxit > 0";
    else if (c->solver != SLPIC2D_SOLVER_CG && c->solver != SLPIC2D_SOLVER_FFT)
        why = "unknown solver";
    else if (c->solver == SLPIC2D_SOLVER_FFT && (c->nx & (c->nx - 1) || c->nx > 8192))
        why = "the FFT solver needs nx a power of two, at most 8192";
    else if (c->src_mode < SLPIC_SRC_NONE || c->src_mode > SLPIC_SRC_RATE ||
             (c->src_mode == SLPIC_SRC_LOSS_MATCHED &&
              (c->src_ref_species < 0 || c->src_ref_species >= c->n_species)))
        why = "bad source mode or reference species";
    else if (c->src_mode != SLPIC_SRC_NONE &&
             !(c->src_lo_cells >= 0 && c->src_len_cells >= 0 &&
               c->src_lo_cells + c->src_len_cells <= c->ny))
        why = "source band outside the grid";
    for (int s = 0; why.empty() && s < c->n_species; ++s) {
        const slpic_species &sp = c->species[s];
        if (!(sp.m > 0) || !(sp.w > 0) || sp.capacity <= 0 || sp.capacity > (1LL << 31) - 1 ||
            !std::isfinite(sp.q) || sp.beta_kind < 0 || sp.beta_kind > 2 || !(sp.T_src >= 0))
            why = "species " + std::to_string(s) + ": bad parameters";
        else if (sp.beta_kind != SLPIC_BETA_ONE && !(sp.v0 > 0))
            why = "species " + std::to_string(s) + ": v0 must be > 0";
        else if (sp.beta_kind != SLPIC_BETA_ONE && c->dt * sp.v0 > c->dx) {
            slpic::set_create_error("species " + std::to_string(s) + ": dt * v0 > dx");
            return SLPIC_ERR_CFL;
        } else if (sp.beta_kind == SLPIC_BETA_ONE && c->max_speed > 0 &&
                   c->dt * c->max_speed > c->dx) {
            slpic::set_create_error("species " + std::to_string(s) + ": dt * max_speed > dx");
            return SLPIC_ERR_CFL;
        }
    }
    if (!why.empty()) {
        slpic::set_create_error(why);
        return SLPIC_ERR_INVALID;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        slpic::set_create_error("no CUDA device");
        return SLPIC_ERR_CUDA;
    }
    slpic2d_t *h = new slpic2d_t();
    h->cfg = *c;
    auto bail = [&](int code, const std::string &m) {
        slpic::set_create_error(m);
        slpic2d_destroy(h);
        return code;
    };
    auto alloc = [&](void **ptr, size_t bytes) -> bool {
        if (cudaMalloc(ptr, bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        h->allocs.push_back(*ptr);
        return true;
    };
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(SLPIC_ERR_CUDA, "stream creation failed");
    h->stream = h->own_stream;
    Params2D &p = h->p;
    p.nx = c->nx;
    make_div_nx(p.nx, p.nx_m, p.nx_s);
    p.ny = c->ny;
    p.nn = c->nx * (c->ny + 1);
    p.ns = c->n_species;
    p.dt = (float)c->dt;
    p.dt_dx = (float)(c->dt / c->dx);
    p.dx = c->dx;
    p.dt64 = c->dt;
    p.k2 = c->dx * c->dx / c->eps0;
    p.phi_lo = c->phi_lo;
    p.phi_hi = c->phi_hi;
    p.rtol2 = c->cg_rtol * c->cg_rtol;
    p.cg_maxit = c->cg_maxit;
    p.src_mode = c->src_mode;
    p.src_ref = c->src_ref_species;
    p.src_lo = (float)c->src_lo_cells;
    p.src_len = (float)c->src_len_cells;
    p.src_rate = c->src_rate;
    p.seed = c->seed;
    const size_t nn = (size_t)p.nn;
    bool ok = alloc((void **)&h->d_state, sizeof(State2D)) &&
              alloc((void **)&p.acc, sizeof(unsigned long long) * nn * p.ns) &&
              alloc((void **)&p.E, sizeof(float2) * nn) && alloc((void **)&p.phi, sizeof(double) * nn) &&
              alloc((void **)&p.r, sizeof(double) * nn) && alloc((void **)&p.q, sizeof(double) * nn) &&
              alloc((void **)&p.fr, sizeof(float) * nn) && alloc((void **)&p.fpA, sizeof(float) * nn) &&
              alloc((void **)&p.fpB, sizeof(float) * nn) && alloc((void **)&p.fq, sizeof(float) * nn) &&
              alloc((void **)&p.fd, sizeof(float) * nn);
    for (int s = 0; ok && s < p.ns; ++s) {
        const slpic_species &sp = c->species[s];
        Species2D &d = p.sp[s];
        for (int b = 0; ok && b < 2; ++b)
            ok = alloc((void **)&d.cell[b], sizeof(int32_t) * sp.capacity) &&
                 alloc((void **)&d.pv[b], sizeof(float4) * sp.capacity) &&
                 alloc((void **)&d.vz[b], sizeof(float) * sp.capacity);
        // the step's list of walked pushes: an eighth of the capacity, at least 64k
        // (slot indices are int32; beyond the list the tile kernel pushes inline)
        d.hard_cap = sp.capacity <= INT_MAX
                         ? std::min<long long>(sp.capacity, std::max<long long>(sp.capacity / 8, 65536))
                         : 0;
        if (ok && d.hard_cap)
            ok = alloc((void **)&d.hard, sizeof(HardRec2D) * d.hard_cap);
        d.capacity = sp.capacity;
        d.qm = (float)(sp.q / sp.m);
        d.v0 = (float)sp.v0;
        d.vth_src = (float)std::sqrt(sp.T_src / sp.m);
        d.kind = sp.beta_kind;
        d.w = sp.w;
        d.inv_w = 1.0 / sp.w;
        d.rho_unit = sp.q * sp.w / (c->dx * c->dx) * std::ldexp(1.0, -40);
    }
    if (!ok)
        return bail(SLPIC_ERR_OOM, "device allocation failed");
    p.st = h->d_state;
    int dev = 0, sms = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg2d, kCgThreads, 0) != cudaSuccess ||
        occ < 1)
        return bail(SLPIC_ERR_CUDA, "CG kernel occupancy query failed");
    h->cg_ctas = std::min(sms * std::min(occ, 2), kBarGroup * kBarGroups);
    h->ctas = sms * 4;
    h->small_ctas = sms * 2;
    {
        // the tile kernel: every CTA of both species resident at once
        int occ_t = 0;
        if (cudaFuncSetAttribute(k_particles2d_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile2d_smem_bytes()) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_t, k_particles2d_tiles, kT2d,
                                                          tile2d_smem_bytes()) == cudaSuccess &&
            occ_t > 0)
            h->tile_ctas = std::max(1, sms * occ_t / p.ns);
        cudaGetLastError();
    }
    if (!alloc((void **)&p.part, sizeof(double) * 3 * h->cg_ctas))
        return bail(SLPIC_ERR_OOM, "device allocation failed");
    if (!alloc((void **)&p.hist, sizeof(int) * nn) || !alloc((void **)&p.cursor, sizeof(int) * nn) ||
        !alloc((void **)&p.bsum, sizeof(int) * ((nn + kScanBlock - 1) / kScanBlock + 1)))
        return bail(SLPIC_ERR_OOM, "device allocation failed");
    p.solver = c->solver;
    if (p.solver == SLPIC2D_SOLVER_FFT) {
        // twiddles and the Thomas multipliers of every (row, mode), in FP64 on the host
        p.log2nx = 0;
        while ((1 << p.log2nx) < p.nx)
            ++p.log2nx;
        if (!alloc((void **)&p.tw, sizeof(double2) * std::max(1, p.nx / 2)) ||
            !alloc((void **)&p.spec, sizeof(double2) * nn) ||
            !alloc((void **)&p.inv_m, sizeof(double) * nn) ||
            !alloc((void **)&p.seg_f, sizeof(double) * nn) ||
            !alloc((void **)&p.seg_b, sizeof(double) * nn) ||
            !alloc((void **)&p.rpart, sizeof(double) * 2 * (p.ny + 1)))
            return bail(SLPIC_ERR_OOM, "device allocation failed");
        const double two_pi = 6.283185307179586;
        std::vector<double2> tw((size_t)std::max(1, p.nx / 2));
        for (int m = 0; m < p.nx / 2; ++m)
            tw[m] = make_double2(std::cos(two_pi * m / p.nx), std::sin(two_pi * m / p.nx));
        std::vector<double> inv_m(nn, 0.0);
        for (int k = 0; k < p.nx; ++k) {
            const double a = 4.0 - 2.0 * std::cos(two_pi * k / p.nx);
            double prev = 0.0;  // 1/m_{j-1}
            for (int j = 1; j < p.ny; ++j) {
                prev = 1.0 / (a - prev);
                inv_m[(size_t)j * p.nx + k] = prev;
            }
        }
        // products of the multipliers within each segment of rows (k_tridiag_modes)
        std::vector<double> seg_f(nn, 0.0), seg_b(nn, 0.0);
        const int L = tri_seg_len(p.ny);
        for (int k = 0; k < p.nx; ++k)
            for (int j0 = 1; j0 < p.ny; j0 += L) {
                const int j1 = std::min(p.ny, j0 + L);
                double f = 1.0, g = 1.0;
                for (int j = j0; j < j1; ++j) {
                    f *= inv_m[(size_t)j * p.nx + k];
                    seg_f[(size_t)j * p.nx + k] = f;
                }
                for (int j = j1 - 1; j >= j0; --j) {
                    g *= inv_m[(size_t)j * p.nx + k];
                    seg_b[(size_t)j * p.nx + k] = g;
                }
            }
        cudaError_t e2 = cudaMemcpy(p.tw, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice);
        if (e2 == cudaSuccess)
            e2 = cudaMemcpy(p.inv_m, inv_m.data(), sizeof(double) * nn, cudaMemcpyHostToDevice);
        if (e2 == cudaSuccess)
            e2 = cudaMemcpy(p.seg_f, seg_f.data(), sizeof(double) * nn, cudaMemcpyHostToDevice);
        if (e2 == cudaSuccess)
            e2 = cudaMemcpy(p.seg_b, seg_b.data(), sizeof(double) * nn, cudaMemcpyHostToDevice);
        const int smem = 16 * p.nx;
        if (e2 == cudaSuccess && smem > 48 * 1024)
            e2 = cudaFuncSetAttribute(k_fft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e2 == cudaSuccess && smem > 48 * 1024)
            e2 = cudaFuncSetAttribute(k_ifft_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e2 != cudaSuccess)
            return bail(SLPIC_ERR_CUDA, cudaGetErrorString(e2));
    }
    cudaError_t e = cudaMemset(h->d_state, 0, sizeof(State2D));
    if (e == cudaSuccess)
        e = cudaMemset(p.acc, 0, sizeof(unsigned long long) * nn * p.ns);
    if (e == cudaSuccess)
        e = cudaMemset(p.E, 0, sizeof(float2) * nn);
    if (e == cudaSuccess)
        e = cudaMemset(p.phi, 0, sizeof(double) * nn);
    if (e != cudaSuccess)
        return bail(SLPIC_ERR_CUDA, cudaGetErrorString(e));
    // plate rows of phi
    std::vector<double> row((size_t)p.nx, c->phi_lo);
    cudaMemcpy(p.phi, row.data(), sizeof(double) * p.nx, cudaMemcpyHostToDevice);
    std::fill(row.begin(), row.end(), c->phi_hi);
    cudaMemcpy(p.phi + (size_t)p.ny * p.nx, row.data(), sizeof(double) * p.nx,
               cudaMemcpyHostToDevice);
    if (cudaDeviceSynchronize() != cudaSuccess)
        return bail(SLPIC_ERR_CUDA, "initialisation failed");
    *out = h;
    return SLPIC_OK;
}

extern "C" int slpic2d_destroy(slpic2d_t *h)
{
    if (!h)
        return SLPIC_OK;
    if (h->own_stream)
        cudaStreamSynchronize(h->own_stream);
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    for (cudaEvent_t e : h->events)
        cudaEventDestroy(e);
    for (void *a : h->allocs)
        cudaFree(a);
    if (h->own_stream)
        cudaStreamDestroy(h->own_stream);
    delete h;
    return SLPIC_OK;
}

extern "C" const char *slpic2d_last_error(const slpic2d_t *h) { return h ? h->err.c_str() : ""; }

extern "C" int slpic2d_set_stream(slpic2d_t *h, void *stream)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    h->stream = (cudaStream_t)stream;
    return SLPIC_OK;
}

static int read_state(slpic2d_t *h, State2D &st)
{
    CK2(h, cudaStreamSynchronize(h->stream));
    CK2(h, cudaMemcpy(&st, h->d_state, sizeof(State2D), cudaMemcpyDeviceToHost));
    return SLPIC_OK;
}

extern "C" int slpic2d_load_particles(slpic2d_t *h, int s, int64_t n, const int32_t *cell,
                                      const float *offset, const float *v)
{
    if (!h || s < 0 || s >= h->p.ns || n < 0 || (n > 0 && (!cell || !offset || !v)))
        return h ? fail2(h, SLPIC_ERR_INVALID, "bad arguments") : SLPIC_ERR_INVALID;
    if (n == 0)
        return SLPIC_OK;
    const int nx = h->p.nx, ny = h->p.ny;
    for (int64_t i = 0; i < n; ++i) {
        const float ox = offset[2 * i], oy = offset[2 * i + 1];
        if (cell[i] < 0 || cell[i] >= nx * ny || !(ox >= 0.0f && ox < 1.0f) ||
            !(oy >= 0.0f && oy < 1.0f) || !std::isfinite(v[3 * i]) ||
            !std::isfinite(v[3 * i + 1]) || !std::isfinite(v[3 * i + 2]))
            return fail2(h, SLPIC_ERR_INVALID,
                         "particle " + std::to_string(i) + ": cell or offset out of range");
    }
    State2D st;
    int rc = read_state(h, st);
    if (rc)
        return rc;
    const int P = (int)(st.step & 1);
    const long long have = (long long)st.count[s][P];
    if (have + n > h->p.sp[s].capacity)
        return fail2(h, SLPIC_ERR_CAPACITY, "load exceeds the species capacity");
    std::vector<float4> pv((size_t)n);
    std::vector<float> vz((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        pv[i] = make_float4(offset[2 * i], offset[2 * i + 1], v[3 * i], v[3 * i + 1]);
        vz[i] = v[3 * i + 2];
    }
    const Species2D &d = h->p.sp[s];
    CK2(h, cudaMemcpy(d.cell[P] + have, cell, sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    CK2(h, cudaMemcpy(d.pv[P] + have, pv.data(), sizeof(float4) * n, cudaMemcpyHostToDevice));
    CK2(h, cudaMemcpy(d.vz[P] + have, vz.data(), sizeof(float) * n, cudaMemcpyHostToDevice));
    const unsigned long long cnt = (unsigned long long)(have + n);
    CK2(h, cudaMemcpy(&h->d_state->count[s][P], &cnt, sizeof(cnt), cudaMemcpyHostToDevice));
    h->prepared = false;
    return SLPIC_OK;
}

extern "C" int slpic2d_prepare(slpic2d_t *h)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    Params2D &p = h->p;
    State2D st;
    int rc = read_state(h, st);
    if (rc)
        return rc;
    if ((rc = sort_particles(h, (int)(st.step & 1))))  // the load in cell order
        return rc;
    CK2(h, cudaMemsetAsync(p.acc, 0, sizeof(unsigned long long) * p.nn * p.ns, h->stream));
    k_deposit2d<<<dim3(h->ctas, p.ns), kThreads, 0, h->stream>>>(p);
    CK2(h, cudaGetLastError());
    rc = launch_solve(h, 0);
    if (rc)
        return rc;
    h->prepared = true;
    h->have_prev_rho = false;
    return device_status(h);
}

extern "C" int slpic2d_step(slpic2d_t *h, int64_t nsteps)
{
    if (!h || nsteps < 0)
        return h ? fail2(h, SLPIC_ERR_INVALID, "nsteps < 0") : SLPIC_ERR_INVALID;
    if (!h->prepared)
        return fail2(h, SLPIC_ERR_INVALID, "slpic2d_prepare must follow a load");
    State2D st;
    int rc = read_state(h, st);
    if (rc)
        return rc;
    if (st.error)
        return device_status(h);
    long long step = st.step;
    Params2D &p = h->p;
    for (int64_t k = 0; k < nsteps; ++k, ++step) {
        // every kCompact2d-th step the particles are sorted by cell again; with the tile
        // kernel that step is in place too (the sort drops the holes), else the global
        // kernel packs the survivors first
        const bool sort = (step % kCompact2d) == kCompact2d - 1;
        const bool compact = sort && !h->tile_ctas;
        cudaEvent_t *ev = nullptr;
        if (h->timing && h->t_steps < kMaxTimedSteps2d) {
            while ((long long)h->events.size() < 4 * (h->t_steps + 1)) {
                cudaEvent_t e;
                CK2(h, cudaEventCreate(&e));
                h->events.push_back(e);
            }
            ev = &h->events[4 * h->t_steps++];
        }
        if (ev)
            CK2(h, cudaEventRecord(ev[0], h->stream));
        if (compact)
            k_particles2d<true><<<dim3(h->ctas, p.ns), kThreads, 0, h->stream>>>(p);
        else if (h->tile_ctas) {
            k_particles2d_tiles<<<dim3(h->tile_ctas, p.ns), kT2d, tile2d_smem_bytes(), h->stream>>>(p);
            k_hard2d<<<h->small_ctas, 256, 0, h->stream>>>(p);
        } else {
            k_particles2d<false><<<dim3(h->ctas, p.ns), kThreads, 0, h->stream>>>(p);
        }
        if (ev)
            CK2(h, cudaEventRecord(ev[1], h->stream));
        k_inject2d<<<h->small_ctas, 256, 0, h->stream>>>(p, compact ? 1 : 0);
        k_book2d<<<1, 32, 0, h->stream>>>(p, compact ? 1 : 0);
        CK2(h, cudaGetLastError());
        // particles by cell (sources appended; holes dropped)
        if (sort && (rc = sort_particles(h, (int)((step + 1) & 1))))
            return rc;
        if (ev)
            CK2(h, cudaEventRecord(ev[2], h->stream));
        if (h->p.solver == SLPIC2D_SOLVER_CG && (rc = warm_start(h)))
            return rc;
        rc = launch_solve(h, 0);
        if (rc)
            return rc;
        if (ev)
            CK2(h, cudaEventRecord(ev[3], h->stream));
    }
    return SLPIC_OK;
}

extern "C" int slpic2d_enable_kernel_timing(slpic2d_t *h, int on)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    h->timing = on != 0;
    h->t_steps = 0;
    return SLPIC_OK;
}

extern "C" int slpic2d_kernel_times(slpic2d_t *h, double *particle_ms, double *inject_ms,
                                    double *field_ms, int64_t *steps)
{
    if (!h || !particle_ms || !inject_ms || !field_ms || !steps)
        return h ? fail2(h, SLPIC_ERR_INVALID, "bad arguments") : SLPIC_ERR_INVALID;
    CK2(h, cudaStreamSynchronize(h->stream));
    double a = 0.0, b = 0.0, c = 0.0;
    for (long long t = 0; t < h->t_steps; ++t) {
        float x = 0.f, y = 0.f, z = 0.f;
        CK2(h, cudaEventElapsedTime(&x, h->events[4 * t], h->events[4 * t + 1]));
        CK2(h, cudaEventElapsedTime(&y, h->events[4 * t + 1], h->events[4 * t + 2]));
        CK2(h, cudaEventElapsedTime(&z, h->events[4 * t + 2], h->events[4 * t + 3]));
        a += x;
        b += y;
        c += z;
    }
    *steps = h->t_steps;
    const double n = h->t_steps ? (double)h->t_steps : 1.0;
    *particle_ms = a / n;
    *inject_ms = b / n;
    *field_ms = c / n;
    h->t_steps = 0;
    return SLPIC_OK;
}

extern "C" int slpic2d_synchronize(slpic2d_t *h)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    return device_status(h);
}

extern "C" int slpic2d_fields(slpic2d_t *h, double *rho, double *phi, float *Ex, float *Ey)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    int rc = device_status(h);
    if (rc)
        return rc;
    const Params2D &p = h->p;
    const size_t nn = (size_t)p.nn;
    if (phi)
        CK2(h, cudaMemcpy(phi, p.phi, sizeof(double) * nn, cudaMemcpyDeviceToHost));
    if (Ex || Ey) {
        std::vector<float2> e(nn);
        CK2(h, cudaMemcpy(e.data(), p.E, sizeof(float2) * nn, cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < nn; ++k) {
            if (Ex)
                Ex[k] = e[k].x;
            if (Ey)
                Ey[k] = e[k].y;
        }
    }
    if (rho) {
        // rho of the current level from the deposits of the particles now stored
        // (the consumed deposit was cleared by the solve): recomputed here
        CK2(h, cudaMemsetAsync(p.acc, 0, sizeof(unsigned long long) * nn * p.ns, h->stream));
        k_deposit2d<<<dim3(h->ctas, p.ns), kThreads, 0, h->stream>>>(p);
        CK2(h, cudaGetLastError());
        CK2(h, cudaStreamSynchronize(h->stream));
        std::vector<long long> a(nn * p.ns);
        CK2(h, cudaMemcpy(a.data(), p.acc, sizeof(long long) * nn * p.ns, cudaMemcpyDeviceToHost));
        CK2(h, cudaMemsetAsync(p.acc, 0, sizeof(unsigned long long) * nn * p.ns, h->stream));
        for (size_t k = 0; k < nn; ++k) {
            double v = 0.0;
            for (int s = 0; s < p.ns; ++s)
                v = std::fma(p.sp[s].rho_unit, (double)a[(size_t)s * nn + k], v);
            rho[k] = v;
        }
    }
    return SLPIC_OK;
}

extern "C" int slpic2d_charge_raw(slpic2d_t *h, int s, int64_t *acc)
{
    if (!h || s < 0 || s >= h->p.ns || !acc)
        return h ? fail2(h, SLPIC_ERR_INVALID, "bad arguments") : SLPIC_ERR_INVALID;
    int rc = device_status(h);
    if (rc)
        return rc;
    const Params2D &p = h->p;
    const size_t nn = (size_t)p.nn;
    CK2(h, cudaMemsetAsync(p.acc, 0, sizeof(unsigned long long) * nn * p.ns, h->stream));
    k_deposit2d<<<dim3(h->ctas, p.ns), kThreads, 0, h->stream>>>(p);
    CK2(h, cudaGetLastError());
    CK2(h, cudaStreamSynchronize(h->stream));
    CK2(h, cudaMemcpy(acc, p.acc + (size_t)s * nn, sizeof(int64_t) * nn, cudaMemcpyDeviceToHost));
    CK2(h, cudaMemsetAsync(p.acc, 0, sizeof(unsigned long long) * nn * p.ns, h->stream));
    return device_status(h);
}

extern "C" int slpic2d_particle_count(slpic2d_t *h, int s, int64_t *n)
{
    if (!h || s < 0 || s >= h->p.ns || !n)
        return h ? fail2(h, SLPIC_ERR_INVALID, "bad arguments") : SLPIC_ERR_INVALID;
    State2D st;
    int rc = read_state(h, st);
    if (rc)
        return rc;
    const int P = (int)(st.step & 1);
    *n = (int64_t)(st.count[s][P] - st.holes[s][P]);
    return SLPIC_OK;
}

extern "C" int slpic2d_get_particles(slpic2d_t *h, int s, int32_t *cell, float *offset, float *v,
                                     int64_t *n)
{
    if (!h || s < 0 || s >= h->p.ns || !n || !cell || !offset || !v)
        return h ? fail2(h, SLPIC_ERR_INVALID, "bad arguments") : SLPIC_ERR_INVALID;
    State2D st;
    int rc = read_state(h, st);
    if (rc)
        return rc;
    const int P = (int)(st.step & 1);
    const long long slots = (long long)st.count[s][P];
    const long long live = slots - (long long)st.holes[s][P];
    if (*n < live)
        return fail2(h, SLPIC_ERR_CAPACITY, "output arrays too small");
    std::vector<int32_t> c((size_t)slots);
    std::vector<float4> pv((size_t)slots);
    std::vector<float> vz((size_t)slots);
    const Species2D &d = h->p.sp[s];
    if (slots) {
        CK2(h, cudaMemcpy(c.data(), d.cell[P], sizeof(int32_t) * slots, cudaMemcpyDeviceToHost));
        CK2(h, cudaMemcpy(pv.data(), d.pv[P], sizeof(float4) * slots, cudaMemcpyDeviceToHost));
        CK2(h, cudaMemcpy(vz.data(), d.vz[P], sizeof(float) * slots, cudaMemcpyDeviceToHost));
    }
    long long k = 0;
    for (long long i = 0; i < slots; ++i) {
        if (c[i] < 0)
            continue;
        cell[k] = c[i];
        offset[2 * k] = pv[i].x;
        offset[2 * k + 1] = pv[i].y;
        v[3 * k] = pv[i].z;
        v[3 * k + 1] = pv[i].w;
        v[3 * k + 2] = vz[i];
        ++k;
    }
    *n = k;
    return SLPIC_OK;
}

extern "C" int slpic2d_diagnostics(slpic2d_t *h, slpic2d_diag *out)
{
    if (!h || !out)
        return h ? fail2(h, SLPIC_ERR_INVALID, "bad arguments") : SLPIC_ERR_INVALID;
    int rc = device_status(h);
    if (rc)
        return rc;
    State2D st;
    rc = read_state(h, st);
    if (rc)
        return rc;
    std::memset(out, 0, sizeof(*out));
    out->step = st.step;
    out->time = (double)st.step * h->cfg.dt;
    const int P = (int)(st.step & 1);
    for (int s = 0; s < h->p.ns; ++s) {
        out->count[s] = (int64_t)(st.count[s][P] - st.holes[s][P]);
        out->absorbed[s][0] = st.absorbed_total[s][0];
        out->absorbed[s][1] = st.absorbed_total[s][1];
        out->injected[s] = st.injected_total[s];
    }
    out->cg_iterations = st.cg_iters;
    out->iterative_last = (int32_t)std::min<unsigned long long>(st.iter_last, 0x7fffffffULL);
    out->cg_iterations_total = st.cg_total;
    out->cg_rel_residual = st.cg_res;
    return SLPIC_OK;
}

extern "C" int slpic2d_solve_poisson(slpic2d_t *h, const double *rho, double *phi,
                                     int32_t *iterations, double *rel_residual)
{
    if (!h || !rho || !phi)
        return h ? fail2(h, SLPIC_ERR_INVALID, "bad arguments") : SLPIC_ERR_INVALID;
    int rc = device_status(h);
    if (rc)
        return rc;
    Params2D saved = h->p;
    Params2D &p = h->p;
    const size_t nn = (size_t)p.nn;
    // private phi and rho buffers so the simulation's fields stay as they are
    double *d_phi = nullptr;
    CK2(h, cudaMalloc(&d_phi, sizeof(double) * nn));
    std::vector<double> guess(phi, phi + nn);
    for (int i = 0; i < p.nx; ++i) {
        guess[i] = p.phi_lo;
        guess[(size_t)p.ny * p.nx + i] = p.phi_hi;
    }
    cudaError_t e = cudaMemcpy(d_phi, guess.data(), sizeof(double) * nn, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p.r, rho, sizeof(double) * nn, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_phi);
        return fail2(h, SLPIC_ERR_CUDA, cudaGetErrorString(e));
    }
    p.phi = d_phi;
    rc = launch_solve(h, 1);
    h->p = saved;
    if (rc == SLPIC_OK)
        rc = device_status(h);
    if (rc == SLPIC_ERR_NOCONVERGE) {
        // a standalone solve's non-convergence is reported, not kept as the
        // simulation's error
        const int zero = 0;
        cudaMemcpy(&h->d_state->error, &zero, sizeof(int), cudaMemcpyHostToDevice);
    }
    State2D st;
    if (rc == SLPIC_OK || rc == SLPIC_ERR_NOCONVERGE) {
        if (read_state(h, st) == SLPIC_OK) {
            if (iterations)
                *iterations = st.cg_iters;
            if (rel_residual)
                *rel_residual = st.cg_res;
        }
        cudaMemcpy(phi, d_phi, sizeof(double) * nn, cudaMemcpyDeviceToHost);
    }
    cudaFree(d_phi);
    return rc;
}
