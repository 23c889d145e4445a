// kernels.cu -- the GPU kernels of one SLPIC timestep (1D3V, electrostatic).
//
//   k_particles  gather + push + move + walls + deposit + compaction   (HBM-bound)
//   k_field      source injection, Poisson solve, E, bookkeeping       (one CTA)
//   k_deposit    deposit of the current particles (after a load)
//   k_diag       reductions for slpic_diagnostics
//   k_validate   range checks of device-side particle loads
//
// Citations: Werner et al., arXiv 1511.08225, Appendix A, Eq. (slpicIntegration).
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.h"
#include "particle_step.cuh"
#include "push_math.cuh"
#include "slpic_internal.cuh"

namespace slpic {

// ---------------------------------------------------------------------------------
// Particle kernel: one launch advances every live particle of every species by one
// step.  Grid (ctas_per_species, n_species); CTA b of species s owns a contiguous
// range of tiles of the input buffer.  The whole 1D grid (E as float, the deposit
// as int64) is staged in shared memory: the gather and the deposit never touch
// global memory, so the kernel streams 20 B in and 20 B out per particle.
// Survivors are compacted into the other buffer: per tile, a ballot per warp, one
// warp scanning the (item, warp) counts, and one atomicAdd to reserve the tile's
// output range (order inside a tile is kept; tile order is not).
// ---------------------------------------------------------------------------------
constexpr int kPB = kParticleThreads;  // threads per CTA
constexpr int kPI = 4;                 // particles per thread per tile
constexpr int kPT = kPB * kPI;         // particles per tile
constexpr int kNW = kPB / 32;
static_assert(kPI * kNW == 32, "one warp scans the per-(item, warp) counts");

__global__ void __launch_bounds__(kPB, 3) k_particles(StepParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_hist = reinterpret_cast<unsigned long long *>(smem);
    float *s_E = reinterpret_cast<float *>(s_hist + p.nn);
    __shared__ int s_off[32];
    __shared__ unsigned long long s_base;
    __shared__ unsigned int s_abs[2];

    const int s = blockIdx.y;
    const SpeciesDev &sp = p.sp[s];
    const long long step = *(volatile long long *)&p.st->step;
    const int P = (int)(step & 1);
    const long long n = (long long)*(volatile unsigned long long *)&p.st->count[s][P];
    const int32_t *__restrict__ cin = sp.cell[P];
    const float4 *__restrict__ vin = sp.pv[P];
    int32_t *__restrict__ cout = sp.cell[P ^ 1];
    float4 *__restrict__ vout = sp.pv[P ^ 1];
    unsigned long long *cnt_out = &p.st->count[s][P ^ 1];
    unsigned long long *acc = p.acc + ((size_t)(P ^ 1) * p.ns + s) * p.nn;

    for (int j = threadIdx.x; j < p.nn; j += kPB) {
        s_hist[j] = 0ULL;
        s_E[j] = p.E[j];
    }
    if (threadIdx.x < 2)
        s_abs[threadIdx.x] = 0u;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long ntiles = (n + kPT - 1) / kPT;
    const long long t0 = ntiles * blockIdx.x / gridDim.x;
    const long long t1 = ntiles * (blockIdx.x + 1) / gridDim.x;

    for (long long t = t0; t < t1; ++t) {
        const long long base = t * kPT;
        int c[kPI];
        float4 q[kPI];
        bool live[kPI];
#pragma unroll
        for (int k = 0; k < kPI; ++k) {
            long long i = base + k * kPB + threadIdx.x;
            live[k] = i < n;
            if (live[k]) {
                c[k] = __ldcs(cin + i);
                q[k] = __ldcs(vin + i);
            }
        }
#pragma unroll
        for (int k = 0; k < kPI; ++k) {
            if (live[k]) {
                int wall = 0;
                live[k] = advance(p, sp, s_E, s_hist, c[k], q[k], wall);
                if (!live[k])
                    atomicAdd(&s_abs[wall], 1u);
            }
        }
        unsigned mask[kPI];
#pragma unroll
        for (int k = 0; k < kPI; ++k) {
            mask[k] = __ballot_sync(0xffffffffu, live[k]);
            if (lane == 0)
                s_off[k * kNW + warp] = __popc(mask[k]);
        }
        __syncthreads();
        if (warp == 0) {
            int v = s_off[lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += y;
            }
            s_off[lane] = incl - v;
            if (lane == 31)
                s_base = incl ? atomicAdd(cnt_out, (unsigned long long)incl) : 0ULL;
        }
        __syncthreads();
        const unsigned long long ob = s_base;
        const unsigned lt = (1u << lane) - 1u;
#pragma unroll
        for (int k = 0; k < kPI; ++k) {
            if (live[k]) {
                unsigned long long o = ob + (unsigned long long)s_off[k * kNW + warp] +
                                       (unsigned long long)__popc(mask[k] & lt);
                __stcs(cout + o, c[k]);
                __stcs(vout + o, q[k]);
            }
        }
        __syncthreads();
    }
    __syncthreads();
    for (int j = threadIdx.x; j < p.nn; j += kPB) {
        unsigned long long v = s_hist[j];
        if (v)
            atomicAdd(acc + j, v);
    }
    if (threadIdx.x < 2 && s_abs[threadIdx.x])
        atomicAdd(&p.st->absorbed_step[s][threadIdx.x], (unsigned long long)s_abs[threadIdx.x]);
}

// ---------------------------------------------------------------------------------
// Deposit of the current particles into acc[step & 1] (used after loading, where
// the deposit of rho^0 uses beta of the loaded v^{-1/2}).
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_deposit(StepParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_hist = reinterpret_cast<unsigned long long *>(smem);
    const int s = blockIdx.y;
    const SpeciesDev &sp = p.sp[s];
    const int P = (int)(p.st->step & 1);
    const long long n = (long long)p.st->count[s][P];
    const int N = p.n_cells;
    for (int j = threadIdx.x; j < p.nn; j += blockDim.x)
        s_hist[j] = 0ULL;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int c = sp.cell[P][i];
        float4 q = sp.pv[P][i];
        int c1 = c + 1;
        if (p.periodic && c1 == N)
            c1 = 0;
        deposit_node(s_hist, c, c1, beta_q(sp.kind, q.y, q.z, q.w, sp.v0), q.x);
    }
    __syncthreads();
    unsigned long long *acc = p.acc + ((size_t)P * p.ns + s) * p.nn;
    for (int j = threadIdx.x; j < p.nn; j += blockDim.x) {
        unsigned long long v = s_hist[j];
        if (v)
            atomicAdd(acc + j, v);
    }
}

// ---------------------------------------------------------------------------------
// Field kernel (one CTA of kFieldThreads).  mode 0: solve from acc[step&1] only.
// mode 1 (end of a step, after k_particles): inject the source particles of this
// step into the output buffer and deposit them, solve from acc[(step+1)&1], clear
// the consumed deposit and counters, advance the step.
//
// Poisson (Appendix A, Eq. LimPtclDynAppendixDotE), nodal 3-point stencil, solved
// exactly by two prefix sums instead of a sequential Thomas sweep: with
// D_j = phi_{j+1} - phi_j the stencil reads D_j - D_{j-1} = -(dx^2/eps0) rho_j, so
//   D_j = D_0 - P_j,  P_j = (dx^2/eps0) sum_{i=1..j} rho_i,
//   phi_j = phi_0 + j D_0 - sum_{i<j} P_i,
// and D_0 follows from phi_N (Dirichlet) or from periodicity (sum_j D_j = 0, after
// removing the mean of rho).  E_j = -(D_{j-1} + D_j)/(2 dx), one-sided at walls.
// ---------------------------------------------------------------------------------
constexpr int kFT = kFieldThreads;
constexpr int kFW = kFT / 32;

// exclusive block scan of one double per thread; *total = sum over the block
__device__ double block_exscan(double v, double *s_w, double *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        double x = (lane < kFW) ? s_w[lane] : 0.0;
        double xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            double y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o)
                xi += y;
        }
        s_w[lane] = xi;  // inclusive over warps
    }
    __syncthreads();
    double before = (warp > 0) ? s_w[warp - 1] : 0.0;
    *total = s_w[kFW - 1];
    __syncthreads();
    return before + incl - v;
}

__device__ double block_sum(double v, double *s_w)
{
    double t;
    block_exscan(v, s_w, &t);
    return t;
}

__device__ void inject_species(const StepParams &p, int s, long long step, long long base,
                               long long k, int Q)
{
    const SpeciesDev &sp = p.sp[s];
    const int N = p.n_cells;
    const unsigned long long key = sm64_stream(p.seed, (unsigned long long)step, (unsigned)s);
    unsigned long long *acc = p.acc + ((size_t)Q * p.ns + s) * p.nn;
    for (long long i = threadIdx.x; i < k; i += blockDim.x) {
        unsigned long long b8 = 8ULL * (unsigned long long)i;
        float u0 = u24(sm64_at(key, b8 + 0));
        float u1 = u24(sm64_at(key, b8 + 1));
        float u2 = u24(sm64_at(key, b8 + 2));
        float u3 = u24(sm64_at(key, b8 + 3));
        float u4 = u24(sm64_at(key, b8 + 4));
        float xc = __fadd_rn(p.src_lo_cells, __fmul_rn(u0, p.src_len_cells));
        float fc = floorf(xc);
        int c = (int)fc;
        float off = xc - fc;
        // physical Maxwellian (Box-Muller); the g-source equals the f-source
        float r1 = sqrtf(-2.0f * logf(u1)), r2 = sqrtf(-2.0f * logf(u3));
        float s2, c2;
        sincospif(2.0f * u2, &s2, &c2);
        float4 q = make_float4(off, sp.vth_src * r1 * c2, sp.vth_src * r1 * s2,
                               sp.vth_src * r2 * cospif(2.0f * u4));
        sp.cell[Q][base + i] = c;
        sp.pv[Q][base + i] = q;
        int c1 = c + 1;
        if (p.periodic && c1 == N)
            c1 = 0;
        unsigned long long qL, qR;
        quantise(beta_q(sp.kind, q.y, q.z, q.w, sp.v0), off, qL, qR);
        atomicAdd(acc + c, qL);
        atomicAdd(acc + c1, qR);
    }
}

__global__ void __launch_bounds__(kFT) k_field(StepParams p, int mode)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_P = reinterpret_cast<double *>(smem);  // [nn]
    __shared__ double s_w[32];
    __shared__ long long s_ninj[kMaxSpecies], s_base[kMaxSpecies];
    __shared__ double s_D0, s_shift;

    DevState *st = p.st;
    const long long step = st->step;
    const int P = (int)(step & 1);
    const int Q = mode ? (P ^ 1) : P;  // deposit to solve from
    const int N = p.n_cells, nn = p.nn;

    if (mode == 1) {
        // ---- source injection (Sec. IV; counts as in the LOSS_MATCHED / RATE readings)
        if (threadIdx.x == 0) {
            double S = 0.0;
            if (p.src_mode == SLPIC_SRC_LOSS_MATCHED) {
                int r = p.src_ref;
                S = (double)(st->absorbed_step[r][0] + st->absorbed_step[r][1]) * p.sp[r].w;
            } else if (p.src_mode == SLPIC_SRC_RATE) {
                S = p.src_rate * p.dt64;
            }
            for (int s = 0; s < p.ns; ++s) {
                long long k = 0;
                if (p.src_mode != SLPIC_SRC_NONE && p.sp[s].vth_src > 0.0f) {
                    double f = st->src_frac[s] + S / p.sp[s].w;
                    k = (long long)floor(f);
                    st->src_frac[s] = f - (double)k;
                }
                long long have = (long long)st->count[s][P ^ 1];
                long long room = p.sp[s].capacity - have;
                if (k > room) {
                    k = room;
                    atomicCAS(&st->error, 0, SLPIC_ERR_CAPACITY);
                }
                s_ninj[s] = k;
                s_base[s] = have;
                st->count[s][P ^ 1] = (unsigned long long)(have + k);
                st->injected_total[s] += k;
                st->absorbed_total[s][0] += (long long)st->absorbed_step[s][0];
                st->absorbed_total[s][1] += (long long)st->absorbed_step[s][1];
                st->absorbed_step[s][0] = 0ULL;
                st->absorbed_step[s][1] = 0ULL;
            }
        }
        __syncthreads();
        for (int s = 0; s < p.ns; ++s)
            if (s_ninj[s] > 0)
                inject_species(p, s, step, s_base[s], s_ninj[s], Q);
        __threadfence();
        __syncthreads();
    }

    // ---- rho_j from the fixed-point deposits (FP64)
    const double scale = 1.0 / 1099511627776.0;  // 2^-40
    const int chunk = (nn + kFT - 1) / kFT;
    const int j0 = min(nn, threadIdx.x * chunk), j1 = min(nn, j0 + chunk);
    double rsum = 0.0;
    for (int j = j0; j < j1; ++j) {
        double r = 0.0;
        for (int s = 0; s < p.ns; ++s) {
            long long a = (long long)__ldcg(p.acc + ((size_t)Q * p.ns + s) * nn + j);
            r += p.sp[s].qw_dx * ((double)a * scale);
        }
        p.rho[j] = r;
        s_P[j] = r;
        rsum += r;
    }
    const double k2 = p.dx * p.dx / p.eps0;
    double mean = 0.0;
    if (p.periodic)
        mean = block_sum(rsum, s_w) / (double)N;
    __syncthreads();
    // P_j = k2 * sum_{i=1..j} (rho_i - mean), j = 0..N-1 (row j=0 contributes nothing)
    const int nD = N;  // D_0..D_{N-1}
    double loc = 0.0;
    for (int j = j0; j < j1; ++j) {
        double r = (j >= 1 && j < nD) ? k2 * (s_P[j] - mean) : 0.0;
        loc += r;
        s_P[j] = loc;  // chunk-local inclusive
    }
    double tot;
    double off = block_exscan(loc, s_w, &tot);
    double psum = 0.0;
    for (int j = j0; j < j1; ++j) {
        s_P[j] += off;
        if (j < nD)
            psum += s_P[j];
    }
    double sumP = block_sum(psum, s_w);
    if (threadIdx.x == 0) {
        if (p.periodic)
            s_D0 = sumP / (double)N;
        else
            s_D0 = (p.phi_hi - p.phi_lo + sumP) / (double)N;
    }
    __syncthreads();
    const double D0 = s_D0;
    // phi_j = phi_0 + j D0 - sum_{i<j} P_i
    double ploc = 0.0;
    for (int j = j0; j < j1; ++j)
        ploc += (j < nD) ? s_P[j] : 0.0;
    double qoff = block_exscan(ploc, s_w, &tot);
    const double phi0 = p.periodic ? 0.0 : p.phi_lo;
    double q = qoff, phsum = 0.0;
    for (int j = j0; j < j1; ++j) {
        double ph = phi0 + (double)j * D0 - q;
        if (!p.periodic && j == N)
            ph = p.phi_hi;
        p.phi[j] = ph;
        phsum += ph;
        if (j < nD)
            q += s_P[j];
    }
    if (p.periodic) {
        double m = block_sum(phsum, s_w) / (double)N;
        if (threadIdx.x == 0)
            s_shift = m;
        __syncthreads();
        for (int j = j0; j < j1; ++j)
            p.phi[j] -= s_shift;
    }
    // E from D_j = D0 - P_j
    const double inv2dx = 0.5 / p.dx;
    for (int j = j0; j < j1; ++j) {
        double e;
        if (p.periodic) {
            int jm = (j == 0) ? N - 1 : j - 1;
            e = -((D0 - s_P[jm]) + (D0 - s_P[j])) * inv2dx;
        } else if (j == 0) {
            e = -(D0 - s_P[0]) / p.dx;
        } else if (j == N) {
            e = -(D0 - s_P[N - 1]) / p.dx;
        } else {
            e = -((D0 - s_P[j - 1]) + (D0 - s_P[j])) * inv2dx;
        }
        p.E64[j] = e;
        p.E[j] = (float)e;
    }

    if (mode == 1) {
        // the deposit of rho^n and the input count are consumed: clear them for
        // the next step's particle kernel, then advance the time level
        for (int idx = threadIdx.x; idx < p.ns * nn; idx += kFT)
            p.acc[(size_t)P * p.ns * nn + idx] = 0ULL;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int s = 0; s < p.ns; ++s)
                st->count[s][P] = 0ULL;
            st->step = step + 1;
        }
    }
}

// ---------------------------------------------------------------------------------
// Diagnostics: per species sum(beta), sum(beta |v|^2) over the live particles.
// out[2*s + 0/1], FP64, zeroed by the caller.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_diag(StepParams p, double *out)
{
    __shared__ double s_a[8], s_b[8];
    const int s = blockIdx.y;
    const SpeciesDev &sp = p.sp[s];
    const int P = (int)(p.st->step & 1);
    const long long n = (long long)p.st->count[s][P];
    double a = 0.0, b = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float4 q = sp.pv[P][i];
        double bt = (double)beta_q(sp.kind, q.y, q.z, q.w, sp.v0);
        double v2 = (double)q.y * q.y + (double)q.z * q.z + (double)q.w * q.w;
        a += bt;
        b += bt * v2;
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_a[warp] = a;
        s_b[warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            ta += s_a[w];
            tb += s_b[w];
        }
        atomicAdd(out + 2 * s, ta);
        atomicAdd(out + 2 * s + 1, tb);
    }
}

// ---------------------------------------------------------------------------------
// Validation of a device-side load: 0 <= cell < N, 0 <= offset < 1, finite v.
// ---------------------------------------------------------------------------------
__global__ void k_validate(const int32_t *cell, const float *off, const float *v, long long n,
                           int n_cells, int *bad)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int c = cell[i];
        float o = off[i];
        bool ok = c >= 0 && c < n_cells && o >= 0.0f && o < 1.0f && isfinite(v[3 * i]) &&
                  isfinite(v[3 * i + 1]) && isfinite(v[3 * i + 2]);
        if (!ok)
            atomicExch(bad, 1);
    }
}

// Pack SoA-of-host-layout (cell[], offset[], v[3n]) into the particle store.
__global__ void k_pack(const int32_t *cell, const float *off, const float *v, long long n,
                       int32_t *cdst, float4 *pdst)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        cdst[i] = cell[i];
        pdst[i] = make_float4(off[i], v[3 * i], v[3 * i + 1], v[3 * i + 2]);
    }
}

__global__ void k_unpack(const int32_t *csrc, const float4 *psrc, long long n, int32_t *cell,
                         float *off, float *v)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        cell[i] = csrc[i];
        float4 q = psrc[i];
        off[i] = q.x;
        v[3 * i] = q.y;
        v[3 * i + 1] = q.z;
        v[3 * i + 2] = q.w;
    }
}

// ---------------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------------
size_t particle_smem_bytes(int nn) { return (size_t)nn * (sizeof(unsigned long long) + sizeof(float)); }
size_t field_smem_bytes(int nn) { return (size_t)nn * sizeof(double); }

cudaError_t configure_kernels(int nn)
{
    cudaError_t e = cudaFuncSetAttribute(k_particles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)particle_smem_bytes(nn));
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(k_deposit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(nn * sizeof(unsigned long long)));
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)field_smem_bytes(nn));
}

cudaError_t particle_ctas_per_sm(int nn, int *out)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_particles, kPB,
                                                         particle_smem_bytes(nn));
}

void launch_particles(const StepParams &p, int ctas_per_species, cudaStream_t st)
{
    dim3 grid(ctas_per_species, p.ns);
    k_particles<<<grid, kPB, particle_smem_bytes(p.nn), st>>>(p);
}

void launch_field(const StepParams &p, int mode, cudaStream_t st)
{
    k_field<<<1, kFT, field_smem_bytes(p.nn), st>>>(p, mode);
}

void launch_deposit(const StepParams &p, int ctas_per_species, cudaStream_t st)
{
    dim3 grid(ctas_per_species, p.ns);
    k_deposit<<<grid, 256, p.nn * sizeof(unsigned long long), st>>>(p);
}

void launch_diag(const StepParams &p, double *out, int ctas_per_species, cudaStream_t st)
{
    dim3 grid(ctas_per_species, p.ns);
    k_diag<<<grid, 256, 0, st>>>(p, out);
}

void launch_validate(const int32_t *cell, const float *off, const float *v, long long n,
                     int n_cells, int *bad, cudaStream_t st)
{
    k_validate<<<1024, 256, 0, st>>>(cell, off, v, n, n_cells, bad);
}

void launch_pack(const int32_t *cell, const float *off, const float *v, long long n,
                 int32_t *cdst, float4 *pdst, cudaStream_t st)
{
    k_pack<<<1024, 256, 0, st>>>(cell, off, v, n, cdst, pdst);
}

void launch_unpack(const int32_t *csrc, const float4 *psrc, long long n, int32_t *cell,
                   float *off, float *v, cudaStream_t st)
{
    k_unpack<<<1024, 256, 0, st>>>(csrc, psrc, n, cell, off, v);
}

}  // namespace slpic
