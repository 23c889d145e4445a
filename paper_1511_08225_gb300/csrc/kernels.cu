// kernels.cu -- the GPU kernels of one SLPIC timestep (1D3V, electrostatic).
//
//   k_particles  gather + push + move + walls + deposit + compaction   (HBM-bound)
//   k_field      source injection, Poisson solve for E, bookkeeping (one 8-CTA cluster)
//   k_potential  rho and phi on demand for read-back                  (one CTA)
//   k_deposit    deposit of the current particles (after a load)
//   k_diag       reductions for slpic_diagnostics
//   k_validate   range checks of device-side particle loads
//
// Citations: Werner et al., arXiv 1511.08225, Appendix A, Eq. (slpicIntegration).
#include <algorithm>
#include <cooperative_groups.h>
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "kernels.h"
#include "particle_step.cuh"
#include "push_math.cuh"
#include "slpic_internal.cuh"

namespace slpic {

// ---------------------------------------------------------------------------------
// Particle kernels: one launch advances every particle of every species by one step.
// Grid (ctas_per_species, n_species); CTA b of species s owns a contiguous range of
// the input buffer.  The whole 1D grid (E as float, the deposit as two 32-bit words
// per node) is staged in shared memory: the gather and the deposit never touch
// global memory, so a step streams 20 B in and 20 B out per particle.
//
// Divergence: most particles take the iteration-free push (push_vx_easy).  The few
// that need the piece walk and Newton (strong field against a slow particle, band
// crossings) would stall their whole warp, so their slots are listed and k_hard
// pushes them afterwards, spread over the whole GPU.
//
// k_particles (most steps) writes each particle back to its own slot of the other
// buffer and a hole (cell = -1) where one is absorbed; its warps never wait for one
// another.  k_particles_compact (every kCompactEvery-th step) packs the survivors:
// per batch, a ballot per warp, one warp scanning the (item, warp) counts, and one
// atomicAdd to reserve the batch's output range (order inside a batch is kept;
// batch order is not).
// ---------------------------------------------------------------------------------
// ---------------------------------------------------------------------------------
// Device time of each kernel of the step (slpic_kernel_spans): thread 0 of every CTA
// takes the earliest start with an atomic, and the last CTA to finish adds the span
// from that start to its own end.  A few atomics per CTA; the next launch of the
// same kernel follows on the stream, so the reset cannot race it.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void span_enter(DevState *st, int k)
{
    if (threadIdx.x == 0)
        atomicMax(&st->span_t0n[k], ~gtimer());
}

// every thread of the CTA calls it, after the CTA's last work
__device__ __forceinline__ void span_exit(DevState *st, int k)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned n = gridDim.x * gridDim.y * gridDim.z;
        if (atomicAdd(&st->span_done[k], 1u) == n - 1u) {
            const unsigned long long t1 = gtimer();
            const unsigned long long t0 = ~atomicExch(&st->span_t0n[k], 0ULL);
            st->span_ns[k] += t1 > t0 ? t1 - t0 : 0ULL;
            st->span_launches[k] += 1ULL;
            st->span_done[k] = 0u;
            __threadfence();
        }
    }
}

constexpr int kPB = kParticleThreads;  // threads per CTA
constexpr int kPI = 4;                 // particles per thread per tile
constexpr int kPT = kPB * kPI;         // particles per tile
constexpr int kNW = kPB / 32;
static_assert(kPI * kNW == 32, "one warp scans the per-(item, warp) counts");

// Compact the live items of NI per thread into out[] (block-wide; all threads call).
template <int NI>
__device__ __forceinline__ void compact_store(const bool (&live)[NI], const int (&c)[NI],
                                              const float4 (&q)[NI], int *s_off,
                                              unsigned long long *s_base,
                                              unsigned long long *cnt_out, int32_t *cout,
                                              float4 *vout)
{
    static_assert(NI * kNW <= 32, "scan fits one warp");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned mask[NI];
#pragma unroll
    for (int k = 0; k < NI; ++k) {
        mask[k] = __ballot_sync(0xffffffffu, live[k]);
        if (lane == 0)
            s_off[k * kNW + warp] = __popc(mask[k]);
    }
    __syncthreads();
    if (warp == 0) {
        int v = lane < NI * kNW ? s_off[lane] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane < NI * kNW)
            s_off[lane] = incl - v;
        if (lane == 31)
            *s_base = incl ? atomicAdd(cnt_out, (unsigned long long)incl) : 0ULL;
    }
    __syncthreads();
    const unsigned long long ob = *s_base;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < NI; ++k) {
        if (live[k]) {
            unsigned long long o = ob + (unsigned long long)s_off[k * kNW + warp] +
                                   (unsigned long long)__popc(mask[k] & lt);
            __stcs(cout + o, c[k]);
            __stcs(vout + o, q[k]);
        }
    }
    __syncthreads();
}

size_t particle_kernel_smem_bytes(int nn) { return (size_t)nn * 3 * sizeof(unsigned); }

// Append this warp's hard particles (slot i, cell c, state q, the gathered ax) to
// the species' list for k_hard (one atomicAdd per warp).
__device__ __forceinline__ void list_hard(bool hard, long long i, int c, const float4 &q,
                                          float ax, const SpeciesDev &sp,
                                          unsigned long long *hard_n)
{
    const unsigned hm = __ballot_sync(0xffffffffu, hard);
    if (!hm)
        return;
    const int lane = threadIdx.x & 31;
    unsigned long long b = 0;
    if (lane == 0)
        b = atomicAdd(hard_n, (unsigned long long)__popc(hm));
    b = __shfl_sync(0xffffffffu, b, 0);
    if (hard) {
        const long long k = (long long)b + __popc(hm & ((1u << lane) - 1u));
        if (k < sp.hard_recs) {
            int4 *r = reinterpret_cast<int4 *>(sp.hard + k);
            r[0] = make_int4((int)i, c, __float_as_int(ax), 0);
            r[1] = make_int4(__float_as_int(q.x), __float_as_int(q.y), __float_as_int(q.z),
                             __float_as_int(q.w));
        } else {
            sp.hard_slot[k] = (int32_t)i;
        }
    }
}

// Bodies of the kernels take the parameters by reference (kernel parameter space
// for one simulation, shared memory for a batch) and the CTA's share of the work.
template <bool kProf, int kKind = kAny, int kPer = kAny>
__device__ __forceinline__ void particles_compact(const StepParams &p, int s, int cta, int nctas)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned *s_lo = reinterpret_cast<unsigned *>(smem);  // [nn] deposit, low words
    unsigned *s_hi = s_lo + p.nn;                         // [nn] deposit, high words
    float *s_E = reinterpret_cast<float *>(s_hi + p.nn);  // [nn]
    __shared__ int s_off[32];
    __shared__ unsigned long long s_base;
    __shared__ unsigned int s_abs[2];

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
        s_lo[j] = 0u;
        s_hi[j] = 0u;
        s_E[j] = p.E[j];
    }
    if (threadIdx.x < 2)
        s_abs[threadIdx.x] = 0u;
    __syncthreads();

    DepositSplit32 dep{s_lo, s_hi};
    const long long ntiles = (n + kPT - 1) / kPT;
    const long long t0 = ntiles * cta / nctas;
    const long long t1 = ntiles * (cta + 1) / nctas;

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
                q[k] = __ldcs(vin + i);  // not behind the cell: no dependent round trip
                live[k] = c[k] >= 0;     // holes are dropped here
            }
        }
#pragma unroll
        for (int k = 0; k < kPI; ++k) {
            bool hard = false;
            float axh = 0.0f;
            if (live[k]) {
                float ax = gather_ax<kPer>(p, sp, s_E, c[k], q[k].x);
                const float v0n = v0_at<kProf>(p, sp, c[k]);
                float vx;
                const int kind = kKind == kAny ? sp.kind : kKind;
                if (push_vx_easy(kind, q[k].y, q[k].z, q[k].w, ax, p.dt, v0n, vx)) {
                    int wall = 0;
                    live[k] = move_and_deposit<kProf, kKind, kPer>(p, sp, dep, c[k], q[k], vx,
                                                                   wall, v0n);
                    if (!live[k])
                        atomicAdd(&s_abs[wall], 1u);
                } else {
                    hard = true;
                    axh = ax;
                    live[k] = false;  // pushed, deposited and stored by k_hard
                }
            }
            list_hard(hard, base + k * kPB + threadIdx.x, c[k], q[k], axh, sp,
                      &p.st->hard_n[s]);
        }
        compact_store<kPI>(live, c, q, s_off, &s_base, cnt_out, cout, vout);
    }

    for (int j = threadIdx.x; j < p.nn; j += kPB) {
        unsigned long long v = ((unsigned long long)s_hi[j] << 32) + s_lo[j];
        if (v)
            atomicAdd(acc + j, v);
    }
    if (threadIdx.x < 2 && s_abs[threadIdx.x])
        atomicAdd(&p.st->absorbed_step[s][threadIdx.x], (unsigned long long)s_abs[threadIdx.x]);
}

constexpr int kWI = 4;           // particles per lane per warp-tile
constexpr int kWT = 32 * kWI;    // particles per warp-tile

size_t particle_inplace_smem_bytes(int nn) { return (size_t)nn * 3 * sizeof(unsigned); }

template <bool kProf, int kKind = kAny, int kPer = kAny>
__device__ __forceinline__ void particles_inplace(const StepParams &p, int s, int cta, int nctas)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned *s_lo = reinterpret_cast<unsigned *>(smem);  // [nn] deposit, low words
    unsigned *s_hi = s_lo + p.nn;                         // [nn] deposit, high words
    float *s_E = reinterpret_cast<float *>(s_hi + p.nn);  // [nn]
    __shared__ unsigned int s_abs[2];

    const SpeciesDev &sp = p.sp[s];
    const long long step = *(volatile long long *)&p.st->step;
    const int P = (int)(step & 1);
    const long long n = (long long)*(volatile unsigned long long *)&p.st->count[s][P];
    const int32_t *__restrict__ cin = sp.cell[P];
    const float4 *__restrict__ vin = sp.pv[P];
    int32_t *__restrict__ cout = sp.cell[P ^ 1];
    float4 *__restrict__ vout = sp.pv[P ^ 1];
    unsigned long long *acc = p.acc + ((size_t)(P ^ 1) * p.ns + s) * p.nn;

    for (int j = threadIdx.x; j < p.nn; j += kPB) {
        s_lo[j] = 0u;
        s_hi[j] = 0u;
        s_E[j] = p.E[j];
    }
    if (threadIdx.x < 2)
        s_abs[threadIdx.x] = 0u;
    __syncthreads();

    DepositSplit32 dep{s_lo, s_hi};
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned nabs0 = 0u, nabs1 = 0u;

    // warp-tiles of kWT consecutive particles: the CTA owns a contiguous range of
    // them and its warps take every kNW-th
    const long long nwt = (n + kWT - 1) / kWT;
    const long long w0 = nwt * cta / nctas;
    const long long w1 = nwt * (cta + 1) / nctas;
    for (long long t = w0 + warp; t < w1; t += kNW) {
        const long long base = t * kWT;
        int c[kWI];
        float4 q[kWI];
        bool act[kWI];
#pragma unroll
        for (int k = 0; k < kWI; ++k) {
            long long i = base + k * 32 + lane;
            act[k] = i < n;
            c[k] = -1;
            if (act[k]) {
                // both loads issued together: a hole's stale float4 is read and
                // ignored rather than waiting for its cell before the load
                c[k] = __ldcs(cin + i);
                q[k] = __ldcs(vin + i);
            }
        }
#pragma unroll
        for (int k = 0; k < kWI; ++k) {
            const long long i = base + k * 32 + lane;
            bool hard = false;
            float axh = 0.0f;
            if (act[k]) {
                if (c[k] < 0) {
                    __stcs(cout + i, -1);  // a hole stays a hole
                } else {
                    float ax = gather_ax<kPer>(p, sp, s_E, c[k], q[k].x);
                    const float v0n = v0_at<kProf>(p, sp, c[k]);
                    float vx;
                    const int kind = kKind == kAny ? sp.kind : kKind;
                    if (push_vx_easy(kind, q[k].y, q[k].z, q[k].w, ax, p.dt, v0n, vx)) {
                        int wall = 0;
                        if (move_and_deposit<kProf, kKind, kPer>(p, sp, dep, c[k], q[k], vx, wall,
                                                                 v0n)) {
                            __stcs(cout + i, c[k]);
                            __stcs(vout + i, q[k]);
                        } else {
                            __stcs(cout + i, -1);
                            if (wall)
                                ++nabs1;
                            else
                                ++nabs0;
                        }
                    } else {
                        hard = true;  // k_hard pushes it and writes its slot
                        axh = ax;
                    }
                }
            }
            list_hard(hard, i, c[k], q[k], axh, sp, &p.st->hard_n[s]);
        }
    }

    unsigned a0 = __reduce_add_sync(0xffffffffu, nabs0);
    unsigned a1 = __reduce_add_sync(0xffffffffu, nabs1);
    if (lane == 0) {
        if (a0)
            atomicAdd(&s_abs[0], a0);
        if (a1)
            atomicAdd(&s_abs[1], a1);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < p.nn; j += kPB) {
        unsigned long long v = ((unsigned long long)s_hi[j] << 32) + s_lo[j];
        if (v)
            atomicAdd(acc + j, v);
    }
    if (threadIdx.x < 2 && s_abs[threadIdx.x])
        atomicAdd(&p.st->absorbed_step[s][threadIdx.x], (unsigned long long)s_abs[threadIdx.x]);
}

// ---------------------------------------------------------------------------------
// The in-place step with the particle stream staged by TMA bulk copies: one CTA of
// kTmaThreads per SM; warp kTmaConsumers/32 is the producer, whose lane 0 keeps a
// ring of kTmaTile-particle tiles (float4 and cell) in flight with
// cp.async.bulk, each stage guarded by a "full" mbarrier (transaction bytes) and an
// "empty" one (one arrival per consumer warp).  Consumer warps read a tile from
// shared memory into registers, free the stage, and then do exactly what
// particles_inplace does per particle.  Loads thus stay in flight while the warps
// compute, independent of how many warps the registers and the deposit histogram
// leave resident.  Each CTA walks every species in turn (the histogram is flushed
// and cleared between species), taking an equal share of each species' tiles.
// Every wait is bounded (about a second of clock64) and stops early once any wait
// in the CTA has failed; the failure is recorded as SLPIC_ERR_TIMEOUT and the warps
// still pass every barrier, so the kernel always returns.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *ptr)
{
    return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// non-blocking test: try_wait may suspend the thread for a while before it returns
// false, long enough for a copy to land, so a limit shorter than that suspension
// needs this form to be able to run out
__device__ __forceinline__ bool mbar_poll(uint64_t *bar, unsigned parity)
{
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; "
        "selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// true once the phase of `parity` has completed; false after `limit` cycles (about
// a second by default) or once another wait of the CTA has failed (*fail set),
// recording SLPIC_ERR_TIMEOUT
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, volatile int *fail,
                                          int *error, long long limit)
{
    const long long t0 = clock64();
    const bool poll = limit < kWaitCycles;  // uniform: a kernel parameter
    while (!(poll ? mbar_poll(bar, parity) : mbar_test(bar, parity))) {
        if (*fail)
            return false;
        if (clock64() - t0 > limit) {
            *fail = 1;
            atomicCAS(error, 0, SLPIC_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// The wait for a copy this CTA issued, before the CTA exits: copies of valid
// memory always land, so it ignores *fail and the wait limit of the pipeline and
// gives up only after kDrainCycles (recording SLPIC_ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_drain(uint64_t *bar, unsigned parity, int *error)
{
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (clock64() - t0 > kDrainCycles) {
            atomicCAS(error, 0, SLPIC_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// named barrier of the consumer warps only
__device__ __forceinline__ void consumers_sync()
{
    asm volatile("bar.sync 1, %0;" ::"n"(kTmaConsumers) : "memory");
}

size_t particle_tma_smem_bytes(int nn, int stages)
{
    // the ring, the histogram's two words, E and the speed-limit profile per node
    return (size_t)16 * stages + (size_t)stages * kTmaTile * 20 + (size_t)nn * 4 * sizeof(unsigned);
}

// slots [r0, r1) of a species of n particles for CTA `cta` of `nctas`: equal shares to
// within 4 slots (a multiple of 4 at every boundary, so that each tile's cells start on
// a 16-byte boundary), walked in tiles of kTmaTile from r0 (the last one partial).  A
// share of whole tiles would leave some CTAs a tile more than others.
__device__ __forceinline__ void tma_share(long long n, int cta, int nctas, long long &r0, long long &r1)
{
    r0 = (n * cta / nctas) & ~3LL;
    r1 = cta + 1 == nctas ? n : (n * (cta + 1) / nctas) & ~3LL;
}

// One species' share of the in-place TMA step, for a consumer thread: its tiles from
// the ring (stage counter k carried across species), each particle gathered, pushed,
// moved, deposited into the shared histogram and written back to its slot (or listed
// for k_hard).  kKind/kPer fix the species' beta kind and the grid's periodicity.
template <bool kProf, int kKind, int kPer>
__device__ __forceinline__ void tma_species(const StepParams &p, int s, int P, int &st,
                                            unsigned &ph, int stages, uint64_t *full,
                                            uint64_t *empty,
                                            const float4 *s_v, const int32_t *s_c,
                                            const float *s_E, const float *s_lam,
                                            DepositSplit32 &dep, volatile int *fail,
                                            unsigned &nabs0, unsigned &nabs1)
{
    const SpeciesDev &sp = p.sp[s];
    const int lane = threadIdx.x & 31;
    const long long n = (long long)*(volatile unsigned long long *)&p.st->count[s][P];
    const int32_t *__restrict__ cin = sp.cell[P];
    int32_t *__restrict__ cout = sp.cell[P ^ 1];
    float4 *__restrict__ vout = sp.pv[P ^ 1];
    long long r0, r1;
    tma_share(n, blockIdx.x, gridDim.x, r0, r1);
    for (long long i0 = r0; i0 < r1; i0 += kTmaTile) {
        const bool ok = !*fail && mbar_wait(&full[st], ph, fail, &p.st->error, p.wait_cycles);
        const int cnt = (int)min((long long)kTmaTile, r1 - i0);
        const int cb = cnt & ~3;
        int c[kTmaPer];
        float4 q[kTmaPer];
        bool act[kTmaPer];
#pragma unroll
        for (int m = 0; m < kTmaPer; ++m) {
            const int j = m * kTmaConsumers + threadIdx.x;
            act[m] = ok && j < cnt;
            c[m] = -1;
            if (act[m]) {
                q[m] = s_v[(size_t)st * kTmaTile + j];
                c[m] = j < cb ? s_c[(size_t)st * kTmaTile + j] : __ldcs(cin + i0 + j);
            }
        }
        __syncwarp();
        if (lane == 0 && ok)
            mbar_arrive(&empty[st]);  // the stage is in registers: free it
#pragma unroll
        for (int m = 0; m < kTmaPer; ++m) {
            const long long i = i0 + m * kTmaConsumers + threadIdx.x;
            bool hard = false;
            float axh = 0.0f;
            if (act[m]) {
                if (c[m] < 0) {
                    __stcs(cout + i, -1);  // a hole stays a hole
                } else {
                    float ax = gather_ax<kPer>(p, sp, s_E, c[m], q[m].x);
                    const float v0n = v0_at<kProf>(p, sp, c[m], s_lam);
                    float vx;
                    const int kind = kKind == kAny ? sp.kind : kKind;
                    if (push_vx_easy(kind, q[m].y, q[m].z, q[m].w, ax, p.dt, v0n, vx)) {
                        int wall = 0;
                        if (move_and_deposit<kProf, kKind, kPer>(p, sp, dep, c[m], q[m], vx, wall,
                                                                v0n, s_lam)) {
                            __stcs(cout + i, c[m]);
                            __stcs(vout + i, q[m]);
                        } else {
                            __stcs(cout + i, -1);
                            if (wall)
                                ++nabs1;
                            else
                                ++nabs0;
                        }
                    } else {
                        hard = true;  // k_hard pushes it and writes its slot
                        axh = ax;
                    }
                }
            }
            list_hard(hard, i, c[m], q[m], axh, sp, &p.st->hard_n[s]);
        }
        // the next tile's stage and phase (the ring's k-th tile sits in stage k mod
        // stages, phase (k / stages) mod 2), counted rather than divided
        if (++st == stages) {
            st = 0;
            ph ^= 1u;
        }
    }
}

template <bool kProf>
__global__ void __launch_bounds__(kTmaThreads, 1) k_particles_tma(const __grid_constant__ StepParams p,
                                                                 int stages)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *full = reinterpret_cast<uint64_t *>(smem);
    uint64_t *empty = full + stages;
    float4 *s_v = reinterpret_cast<float4 *>(smem + 16 * stages);
    int32_t *s_c = reinterpret_cast<int32_t *>(s_v + (size_t)stages * kTmaTile);
    unsigned *s_lo = reinterpret_cast<unsigned *>(s_c + (size_t)stages * kTmaTile);
    unsigned *s_hi = s_lo + p.nn;
    float *s_E = reinterpret_cast<float *>(s_hi + p.nn);
    float *s_lam = s_E + p.nn;  // the speed-limit profile (kProf)
    __shared__ unsigned s_abs[2];
    __shared__ int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = threadIdx.x; j < p.nn; j += kTmaThreads) {
        s_lo[j] = 0u;
        s_hi[j] = 0u;
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < stages; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&empty[k], kTmaConsumers / 32);
        }
        s_abs[0] = s_abs[1] = 0u;
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    span_enter(p.st, 0);
    const long long step = *(volatile long long *)&p.st->step;
    const int P = (int)(step & 1);
    for (int j = threadIdx.x; j < p.nn; j += kTmaThreads) {
        s_E[j] = p.E[j];
        if (kProf)
            s_lam[j] = __ldg(p.lam + j);
    }
    __syncthreads();
    volatile int *fail = &s_fail;

    if (warp == kTmaConsumers / 32) {
        // ---- producer: lane 0 issues every tile of this CTA, species by species
        if (lane == 0) {
            long long k = 0;
            for (int s = 0; s < p.ns && !*fail; ++s) {
                const SpeciesDev &sp = p.sp[s];
                const long long n = (long long)*(volatile unsigned long long *)&p.st->count[s][P];
                long long r0, r1;
                tma_share(n, blockIdx.x, gridDim.x, r0, r1);
                for (long long i0 = r0; i0 < r1; i0 += kTmaTile, ++k) {
                    const int st = (int)(k % stages);
                    const unsigned ph = (unsigned)((k / stages) & 1);
                    if (k >= stages &&
                        !mbar_wait(&empty[st], ph ^ 1u, fail, &p.st->error, p.wait_cycles))
                        break;
                    const int cnt = (int)min((long long)kTmaTile, r1 - i0);
                    const int cb = cnt & ~3;  // cells by bulk copy (16-byte multiple)
                    mbar_expect_tx(&full[st], (unsigned)(cnt * 16 + cb * 4));
                    bulk_load(s_v + (size_t)st * kTmaTile, sp.pv[P] + i0, (unsigned)cnt * 16, &full[st]);
                    if (cb)
                        bulk_load(s_c + (size_t)st * kTmaTile, sp.cell[P] + i0, (unsigned)cb * 4,
                                  &full[st]);
                }
            }
            // every copy issued has landed before the CTA may exit (also after a wait
            // of the pipeline gave up)
            for (long long j = (k > stages ? k - stages : 0); j < k; ++j)
                if (!mbar_drain(&full[j % stages], (unsigned)((j / stages) & 1), &p.st->error))
                    break;
        }
    } else {
        // ---- consumers
        int st = 0;        // stage of the next tile
        unsigned ph = 0u;  // its phase
        for (int s = 0; s < p.ns; ++s) {
            const SpeciesDev &sp = p.sp[s];
            DepositSplit32 dep{s_lo, s_hi};
            unsigned nabs0 = 0u, nabs1 = 0u;
            // the species' tiles: the sheath's common shape (Heaviside beta between
            // plates) with both fixed at compile time, every other shape read at run
            // time (the same arithmetic either way)
            if (sp.kind == SLPIC_BETA_HEAVISIDE && !p.periodic)
                tma_species<kProf, SLPIC_BETA_HEAVISIDE, 0>(p, s, P, st, ph, stages, full, empty,
                                                           s_v, s_c, s_E, s_lam, dep, fail, nabs0,
                                                           nabs1);
            else
                tma_species<kProf, kAny, kAny>(p, s, P, st, ph, stages, full, empty, s_v, s_c,
                                               s_E, s_lam, dep, fail, nabs0, nabs1);
            // species done: absorbed counts, histogram flush and clear
            const unsigned a0 = __reduce_add_sync(0xffffffffu, nabs0);
            const unsigned a1 = __reduce_add_sync(0xffffffffu, nabs1);
            if (lane == 0) {
                if (a0)
                    atomicAdd(&s_abs[0], a0);
                if (a1)
                    atomicAdd(&s_abs[1], a1);
            }
            consumers_sync();
            unsigned long long *acc = p.acc + ((size_t)(P ^ 1) * p.ns + s) * p.nn;
            for (int j = threadIdx.x; j < p.nn; j += kTmaConsumers) {
                const unsigned long long v = ((unsigned long long)s_hi[j] << 32) + s_lo[j];
                if (v)
                    atomicAdd(acc + j, v);
                s_lo[j] = 0u;
                s_hi[j] = 0u;
            }
            if (threadIdx.x < 2) {
                if (s_abs[threadIdx.x])
                    atomicAdd(&p.st->absorbed_step[s][threadIdx.x],
                              (unsigned long long)s_abs[threadIdx.x]);
                s_abs[threadIdx.x] = 0u;
            }
            consumers_sync();
        }
    }
    span_exit(p.st, 0);
}

// Copy one instance's parameters into shared memory (batched kernels).
__device__ __forceinline__ void load_params(StepParams &dst, const StepParams *src)
{
    static_assert(sizeof(StepParams) % 8 == 0, "copied as 8-byte words");
    const unsigned long long *a = reinterpret_cast<const unsigned long long *>(src);
    unsigned long long *b = reinterpret_cast<unsigned long long *>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(StepParams) / 8); k += blockDim.x)
        b[k] = a[k];
    __syncthreads();
}

// kProf: the speed-limit profile p.lam is set
// The body for species blockIdx.y: the sheath's common shape (Heaviside beta between
// plates) with both fixed at compile time, every other shape read at run time (the
// same arithmetic either way).
template <bool kProf>
__global__ void __launch_bounds__(kPB, 3) k_particles_compact(const __grid_constant__ StepParams p)
{
    span_enter(p.st, 0);
    if (p.sp[blockIdx.y].kind == SLPIC_BETA_HEAVISIDE && !p.periodic)
        particles_compact<kProf, SLPIC_BETA_HEAVISIDE, 0>(p, blockIdx.y, blockIdx.x, gridDim.x);
    else
        particles_compact<kProf>(p, blockIdx.y, blockIdx.x, gridDim.x);
    span_exit(p.st, 0);
}

template <bool kProf>
__global__ void __launch_bounds__(kPB, 4) k_particles(const __grid_constant__ StepParams p)
{
    span_enter(p.st, 0);
    if (p.sp[blockIdx.y].kind == SLPIC_BETA_HEAVISIDE && !p.periodic)
        particles_inplace<kProf, SLPIC_BETA_HEAVISIDE, 0>(p, blockIdx.y, blockIdx.x, gridDim.x);
    else
        particles_inplace<kProf>(p, blockIdx.y, blockIdx.x, gridDim.x);
    span_exit(p.st, 0);
}

// Batched forms: CTA b works on (instance, species, share, shares) = work[b].
__global__ void __launch_bounds__(kPB, 3)
    k_particles_compact_batch(const StepParams *__restrict__ ps, const int4 *__restrict__ work)
{
    __shared__ StepParams s_p;
    const int4 w = work[blockIdx.x];
    load_params(s_p, ps + w.x);
    particles_compact<false>(s_p, w.y, w.z, w.w);
}

__global__ void __launch_bounds__(kPB, 4)
    k_particles_batch(const StepParams *__restrict__ ps, const int4 *__restrict__ work)
{
    __shared__ StepParams s_p;
    const int4 w = work[blockIdx.x];
    load_params(s_p, ps + w.x);
    particles_inplace<false>(s_p, w.y, w.z, w.w);
}

// ---------------------------------------------------------------------------------
// k_hard: the particles the particle kernel listed (those needing the piece walk and
// Newton).  They cluster (strong fields, the source band), and each needs a long
// serial computation, so one warp holding many of them would become the critical
// path; spread over a grid-stride loop of the whole GPU their latency hides.  The
// field is gathered from global memory and the deposit goes straight to the global
// int64 accumulator.  After an in-place step a particle returns to its slot (a hole
// if absorbed); after a compacting step survivors are appended to the output.
// ---------------------------------------------------------------------------------
template <bool kProf>
__device__ __forceinline__ void hard_body(const StepParams &p, int compact, long long gwarp,
                                          long long nwarps)
{
    __shared__ unsigned int s_abs[kMaxSpecies][2];
    if (threadIdx.x < 2 * kMaxSpecies)
        s_abs[threadIdx.x >> 1][threadIdx.x & 1] = 0u;
    __syncthreads();
    const long long step = *(volatile long long *)&p.st->step;
    const int P = (int)(step & 1);
    const int lane = threadIdx.x & 31;
    // the species' lists as one index space, so that the serial pushes of different
    // species run side by side rather than one after the other
    long long pre[kMaxSpecies + 1];  // kept in registers: constant indices only
    pre[0] = 0;
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s)
        pre[s + 1] = pre[s] + (s < p.ns ? (long long)*(volatile unsigned long long *)&p.st->hard_n[s] : 0);
    const long long total = pre[kMaxSpecies];
    for (long long b = gwarp * 32; b < total; b += nwarps * 32) {
        const long long t = b + lane;
        bool live = false;
        int s = -1, c = 0, slot = 0;
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (t < total) {
            long long base = 0;
            s = 0;
#pragma unroll
            for (int k = 1; k < kMaxSpecies; ++k)
                if (t >= pre[k]) {
                    s = k;
                    base = pre[k];
                }
            const SpeciesDev &sp = p.sp[s];
            DepositU64 dep{p.acc + ((size_t)(P ^ 1) * p.ns + s) * p.nn};
            const long long k = t - base;
            float ax;
            if (k < sp.hard_recs) {
                const int4 *rec = reinterpret_cast<const int4 *>(sp.hard + k);
                const int4 r0 = __ldcs(rec), r1 = __ldcs(rec + 1);  // one record, no chain
                slot = r0.x;
                c = r0.y;
                ax = __int_as_float(r0.z);
                q = make_float4(__int_as_float(r1.x), __int_as_float(r1.y),
                                __int_as_float(r1.z), __int_as_float(r1.w));
            } else {  // past the records: the slot, then the particle and its field
                slot = sp.hard_slot[k];
                c = sp.cell[P][slot];
                q = sp.pv[P][slot];
                ax = gather_ax(p, sp, p.E, c, q.x);
            }
            const float v0n = v0_at<kProf>(p, sp, c);
            float vx = push_vx_walk(sp.kind, q.y, q.z, q.w, ax, p.dt, v0n);
            int wall = 0;
            live = move_and_deposit<kProf>(p, sp, dep, c, q, vx, wall, v0n);
            if (!live)
                atomicAdd(&s_abs[s][wall], 1u);
        }
        if (compact) {
            // survivors appended to their species' output, one atomic per species present
            for (int s2 = 0; s2 < p.ns; ++s2) {
                const bool mine = live && s == s2;
                const unsigned m = __ballot_sync(0xffffffffu, mine);
                if (!m)
                    continue;
                unsigned long long o = 0;
                if (lane == __ffs(m) - 1)
                    o = atomicAdd(&p.st->count[s2][P ^ 1], (unsigned long long)__popc(m));
                o = __shfl_sync(0xffffffffu, o, __ffs(m) - 1);
                if (mine) {
                    o += __popc(m & ((1u << lane) - 1u));
                    p.sp[s2].cell[P ^ 1][o] = c;
                    p.sp[s2].pv[P ^ 1][o] = q;
                }
            }
        } else if (t < total) {
            const SpeciesDev &sp = p.sp[s];
            sp.cell[P ^ 1][slot] = live ? c : -1;
            if (live)
                sp.pv[P ^ 1][slot] = q;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * kMaxSpecies) {
        const int s = threadIdx.x >> 1, w = threadIdx.x & 1;
        if (s < p.ns && s_abs[s][w])
            atomicAdd(&p.st->absorbed_step[s][w], (unsigned long long)s_abs[s][w]);
    }
}

template <bool kProf>
__global__ void __launch_bounds__(256) k_hard(const __grid_constant__ StepParams p, int compact)
{
    span_enter(p.st, 1);
    hard_body<kProf>(p, compact, (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
              (long long)gridDim.x * (blockDim.x >> 5));
    span_exit(p.st, 1);
}

// batched: grid (CTAs per instance, instances)
__global__ void __launch_bounds__(256) k_hard_batch(const StepParams *__restrict__ ps, int compact)
{
    __shared__ StepParams s_p;
    load_params(s_p, ps + blockIdx.y);
    hard_body<false>(s_p, compact, (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
              (long long)gridDim.x * (blockDim.x >> 5));
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
        if (c < 0)
            continue;  // hole
        float4 q = sp.pv[P][i];
        int c1 = c + 1;
        if (p.periodic && c1 == N)
            c1 = 0;
        deposit_node(s_hist, c, c1, beta_q(sp.kind, q.y, q.z, q.w, v0_cell(p, sp, c)), q.x);
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

// Source particle i of species s for this step (Sec. IV source, the readings of
// LOSS_MATCHED / RATE): it takes uniforms u_j = u24(SplitMix64(key, 8i+j)), key the
// species' stream of the step, for its position in the band (FP32, pinned
// operations) and a physical Maxwellian velocity (Box-Muller): the g-source equals
// the f-source.  It goes to slot base + i of buffer Q, its deposit to acc[Q].
__device__ __forceinline__ void inject_one(const StepParams &p, int s, unsigned long long key,
                                           long long base, long long i, int Q)
{
    const SpeciesDev &sp = p.sp[s];
    const int N = p.n_cells;
    unsigned long long *acc = p.acc + ((size_t)Q * p.ns + s) * p.nn;
    {
        unsigned long long b8 = 8ULL * (unsigned long long)i;
        float u0 = u24(sm64_at(key, b8 + 0));
        float u1 = u24(sm64_at(key, b8 + 1));
        float u2 = u24(sm64_at(key, b8 + 2));
        float u3 = u24(sm64_at(key, b8 + 3));
        float u4 = u24(sm64_at(key, b8 + 4));
        int c;
        float off;
        float4 q;
        if (p.src_mode == SLPIC_SRC_WALL) {
            // through the plate at x = L: the flux-weighted half-Maxwellian (|vx|
            // Rayleigh, towards -x), placed where it has moved since a uniformly
            // random entry time in the step; a position that rounds to the plate is
            // put at the largest cell coordinate below it
            const float vxm = sp.vth_src * sqrtf(-2.0f * logf(u1));
            const float rw = sp.vth_src * sqrtf(-2.0f * logf(u2));
            float sw, cw;
            sincospif(2.0f * u3, &sw, &cw);
            const float vy = rw * cw, vz = rw * sw;
            const float b = beta_q(sp.kind, -vxm, vy, vz, v0_cell(p, sp, N - 1));
            float xc = __fsub_rn((float)N, __fmul_rn(u0, __fmul_rn(__fmul_rn(b, vxm), p.dt_dx)));
            if (!(xc < (float)N))
                xc = __int_as_float(__float_as_int((float)N) - 1);
            xc = fmaxf(xc, 0.0f);
            const float fc = floorf(xc);
            c = (int)fc;
            off = xc - fc;
            q = make_float4(off, -vxm, vy, vz);
        } else {
            float xc = __fadd_rn(p.src_lo_cells, __fmul_rn(u0, p.src_len_cells));
            float fc = floorf(xc);
            c = (int)fc;
            off = xc - fc;
            // physical Maxwellian (Box-Muller); the g-source equals the f-source
            float r1 = sqrtf(-2.0f * logf(u1)), r2 = sqrtf(-2.0f * logf(u3));
            float s2, c2;
            sincospif(2.0f * u2, &s2, &c2);
            q = make_float4(off, sp.vth_src * r1 * c2, sp.vth_src * r1 * s2,
                            sp.vth_src * r2 * cospif(2.0f * u4));
        }
        sp.cell[Q][base + i] = c;
        sp.pv[Q][base + i] = q;
        int c1 = c + 1;
        if (p.periodic && c1 == N)
            c1 = 0;
        unsigned long long qL, qR;
        quantise(beta_q(sp.kind, q.y, q.z, q.w, v0_cell(p, sp, c)), off, qL, qR);
        atomicAdd(acc + c, qL);
        atomicAdd(acc + c1, qR);
    }
}

// The step's source particles of every species (k[s] of species s, to slots base[s]
// on): taken as one index space, so that the species' particles are made side by
// side; this CTA makes the indices first, first + stride, ...
__device__ void inject_all(const StepParams &p, long long step, const long long *base,
                           const long long *k, int Q, int first, int stride)
{
    long long pre[kMaxSpecies + 1];  // registers: constant indices only
    pre[0] = 0;
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s)
        pre[s + 1] = pre[s] + (s < p.ns ? k[s] : 0);
    const long long total = pre[kMaxSpecies];
    for (long long t = first + (long long)threadIdx.x * stride; t < total;
         t += (long long)blockDim.x * stride) {
        int s = 0;
        long long i0 = 0, b = base[0];
#pragma unroll
        for (int r = 1; r < kMaxSpecies; ++r)
            if (t >= pre[r]) {
                s = r;
                i0 = pre[r];
                b = base[r];
            }
        const unsigned long long key = sm64_stream(p.seed, (unsigned long long)step, (unsigned)s);
        inject_one(p, s, key, b, t - i0, Q);
    }
}

// On demand (slpic_fields): rho and phi of the latest deposit acc[step & 1], one CTA.
// The particle step needs only E, which k_field computes; phi is read back rarely.
// The prescribed wave of the test-particle mode at node j and time t: the potential
// phi0(t) sin(k (x_j - vphi t)) and the field -dphi/dx = -phi0(t) k cos(k (x_j - vphi t)).
__device__ __forceinline__ double wave_amplitude(const StepParams &p, double t)
{
    return p.wave_ramp > 0.0 ? p.wave_phi0 * fmin(1.0, t / p.wave_ramp) : p.wave_phi0;
}
__device__ __forceinline__ double wave_phi(const StepParams &p, int j, double t)
{
    return wave_amplitude(p, t) * sin(p.wave_k * ((double)j * p.dx - p.wave_vphi * t));
}
__device__ __forceinline__ double wave_E(const StepParams &p, int j, double t)
{
    return -wave_amplitude(p, t) * p.wave_k * cos(p.wave_k * ((double)j * p.dx - p.wave_vphi * t));
}

// dep: the deposit to solve from, [species][nn] (the latest level's, or a copy of it);
// step: its time level (for a prescribed wave)
__global__ void __launch_bounds__(kFT) k_potential(StepParams p, const unsigned long long *dep,
                                                   long long step)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_P = reinterpret_cast<double *>(smem);  // [nn]
    __shared__ double s_w[32];
    __shared__ double s_D0, s_shift;

    const int N = p.n_cells, nn = p.nn;

    // ---- rho_j from the fixed-point deposits (FP64)
    const double scale = 1.0 / 1099511627776.0;  // 2^-40
    const int chunk = (nn + kFT - 1) / kFT;
    const int j0 = min(nn, threadIdx.x * chunk), j1 = min(nn, j0 + chunk);
    double rsum = 0.0;
    for (int j = j0; j < j1; ++j) {
        double r = 0.0;
        for (int s = 0; s < p.ns; ++s) {
            long long a = (long long)__ldcg(dep + (size_t)s * nn + j);
            r += p.sp[s].qw_dx * ((double)a * scale);
        }
        p.rho[j] = r;
        s_P[j] = r;
        if (j < N)
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
    if (p.wave_on) {
        // test-particle mode: the potential is the prescribed one
        __syncthreads();
        const double t = (double)step * p.dt64;
        for (int j = j0; j < j1; ++j)
            p.phi[j] = wave_phi(p, j, t);
    }
}

// ---------------------------------------------------------------------------------
// Field kernel: one thread-block cluster of kFC CTAs (one per SM).  mode 0: E from
// acc[step&1] (after a load).  mode 1 / 2 (end of a step, after k_particles /
// k_particles_compact and k_hard): the CTAs make this step's source particles (every
// kFC-th each), write them after the output buffer's slots and deposit them; then E
// from acc[(step+1)&1]; the consumed deposit and counters are cleared and the step
// advances.
//
// Poisson (Appendix A, Eq. LimPtclDynAppendixDotE), nodal 3-point stencil, solved
// exactly by prefix sums instead of a sequential Thomas sweep.  With
// D_j = phi_{j+1} - phi_j the stencil reads D_j - D_{j-1} = -(dx^2/eps0) rho_j, so
//   D_j = D_0 - P_j,   P_j = k2 (sum_{i=1..j} rho_i - mean j),   k2 = dx^2/eps0,
//   sum_{j=0}^{N-1} P_j = k2 (sum_{i=1}^{N-1} (N - i) rho_i - mean N(N-1)/2),
// D_0 from phi_N - phi_0 = sum_j D_j (Dirichlet) or sum_j D_j = 0 with the mean of
// rho removed (periodic), and E_j = -(D_{j-1} + D_j)/(2 dx), one-sided at walls.
// Because rho_j = sum_s c_s acc_s[j] with integer deposits, every sum above is a sum
// of integers: the prefix sums A_s[j] = sum_{i=1..j} acc_s[i], the weighted sum
// W_s = sum (N-i) acc_s[i] and the total T_s are formed exactly in 128-bit integers
// (one exchange of per-CTA totals through distributed shared memory), and FP64 -
// narrow on this GPU - is used only to combine them into E.
// ---------------------------------------------------------------------------------
constexpr int kFC = kFieldClusterCtas;
constexpr int kFCT = kFieldClusterThreads;
constexpr int kFCW = kFCT / 32;

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 shfl_up_u128(u128 v, int o)
{
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    lo = __shfl_up_sync(0xffffffffu, lo, o);
    hi = __shfl_up_sync(0xffffffffu, hi, o);
    return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int o)
{
    unsigned long long lo = (unsigned long long)v, hi = (unsigned long long)(v >> 64);
    lo = __shfl_down_sync(0xffffffffu, lo, o);
    hi = __shfl_down_sync(0xffffffffu, hi, o);
    return ((u128)hi << 64) | lo;
}

// x < 2^64 to the nearest double, built on the FP64 add pipe: a 32-bit half h is
// exact as (2^52 + h) - 2^52, the double whose high word is that of 2^52 and whose low
// word is h, minus 2^52; one fused multiply-add then forms hi 2^32 + lo with a single
// rounding: the value of the conversion instruction, on the add pipe.
__device__ __forceinline__ double u64_to_double_rn(unsigned long long x)
{
    const double two52 = 4503599627370496.0;
    const double h = __hiloint2double(0x43300000, (int)(unsigned)(x >> 32)) - two52;
    const double l = __hiloint2double(0x43300000, (int)(unsigned)x) - two52;
    return fma(h, 4294967296.0, l);
}

__device__ __forceinline__ double u128_to_double(u128 v)
{
    unsigned long long hi = (unsigned long long)(v >> 64), lo = (unsigned long long)v;
    double d = u64_to_double_rn(lo);
    if (hi)
        d = fma(u64_to_double_rn(hi), 18446744073709551616.0, d);  // 2^64
    return d;
}

// kC: the CTAs of the cluster
template <int kC>
__device__ __forceinline__ void field_body(const StepParams &p, int mode)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    // per species: this CTA's sum over its rows 1..N-1 (R), weighted sum (W), total
    // over nodes j < N (T)
    __shared__ u128 s_tot[kMaxSpecies][3];
    __shared__ u128 s_warp[kMaxSpecies][kFCW];
    __shared__ u128 s_wpart[kMaxSpecies][kFCW][2];
    __shared__ double s_dbl[kMaxSpecies][3];  // the cluster's R, W, T per species, as doubles
    __shared__ double s_c[4];                 // D0, P_{N-1}, mean, (unused)
    __shared__ u128 s_off[kMaxSpecies];
    __shared__ long long s_ninj[kMaxSpecies], s_base[kMaxSpecies];
    __shared__ double s_frac[kMaxSpecies];

    DevState *st = p.st;
    const int N = p.n_cells, nn = p.nn, ns = p.ns;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // this CTA's nodes [c0, c1); the thread's chunk of them
    const int per_cta = (nn + kC - 1) / kC;
    const int c0 = min(nn, rank * per_cta), c1 = min(nn, c0 + per_cta);
    const int chunk = (per_cta + kFCT - 1) / kFCT;
    const int j0 = min(c1, c0 + (int)threadIdx.x * chunk), j1 = min(c1, j0 + chunk);

    // ---- the step's counters, thread s for species s: every load issued at once
    // (none depends on another, nor on the step index), used below
    const long long step = st->step;
    unsigned long long pf_cnt0 = 0ULL, pf_cnt1 = 0ULL, pf_holes0 = 0ULL, pf_holes1 = 0ULL;
    unsigned long long pf_ab0 = 0ULL, pf_ab1 = 0ULL, pf_ref0 = 0ULL, pf_ref1 = 0ULL, pf_hard = 0ULL;
    long long pf_inj = 0, pf_at0 = 0, pf_at1 = 0, pf_it = 0;
    double pf_frac = 0.0;
    if (mode >= 1 && (int)threadIdx.x < ns) {
        const int s = threadIdx.x, r = p.src_ref;
        pf_cnt0 = st->count[s][0];
        pf_cnt1 = st->count[s][1];
        pf_ref0 = st->absorbed_step[r][0];
        pf_ref1 = st->absorbed_step[r][1];
        pf_frac = st->src_frac[s];
        if (rank == 0) {
            pf_holes0 = st->holes[s][0];
            pf_holes1 = st->holes[s][1];
            pf_ab0 = st->absorbed_step[s][0];
            pf_ab1 = st->absorbed_step[s][1];
            pf_hard = st->hard_n[s];
            pf_inj = st->injected_total[s];
            pf_at0 = st->absorbed_total[s][0];
            pf_at1 = st->absorbed_total[s][1];
            pf_it = st->iterative_total[s];
        }
    }
    const int P = (int)(step & 1);
    const int Q = mode ? (P ^ 1) : P;  // deposit to solve from

    if (mode >= 1) {
        // ---- source injection (Sec. IV; LOSS_MATCHED / RATE readings).  Every CTA
        // derives the same counts from the same state (thread s for species s) and
        // makes every kC-th particle; CTA 0 writes the bookkeeping after the
        // exchange below, when every CTA has read the state.
        const int s = threadIdx.x;
        if (s < ns) {
            double S = 0.0;
            if (p.src_mode == SLPIC_SRC_LOSS_MATCHED) {
                S = (double)(pf_ref0 + pf_ref1) * p.sp[p.src_ref].w;
            } else if (p.src_mode == SLPIC_SRC_RATE) {
                S = p.src_rate * p.dt64;
            }
            long long k = 0;
            double f = pf_frac;
            if (p.src_mode == SLPIC_SRC_WALL) {
                if (p.sp[s].wall_rate > 0.0) {
                    f += p.sp[s].wall_rate;
                    k = (long long)floor(f);
                    f -= (double)k;
                }
            } else if (p.src_mode != SLPIC_SRC_NONE && p.sp[s].vth_src > 0.0f) {
                f = fma(S, p.sp[s].inv_w, f);
                k = (long long)floor(f);
                f -= (double)k;
            }
            // after an in-place step the output uses the input's slots (holes
            // included); after a compacting step its count was reserved by atomics
            long long have = (long long)(mode == 1 ? (P ? pf_cnt1 : pf_cnt0) : (P ? pf_cnt0 : pf_cnt1));
            long long room = p.sp[s].capacity - have;
            s_ninj[s] = k > room ? -room - 1 : k;  // negative: truncated
            s_base[s] = have;
            s_frac[s] = f;
        }
        __syncthreads();
        {
            long long kk[kMaxSpecies], bb[kMaxSpecies];
#pragma unroll
            for (int sp_ = 0; sp_ < kMaxSpecies; ++sp_) {
                const long long k = sp_ < ns ? s_ninj[sp_] : 0;
                kk[sp_] = k < 0 ? -k - 1 : k;
                bb[sp_] = sp_ < ns ? s_base[sp_] : 0;
            }
            inject_all(p, step, bb, kk, Q, rank, kC);
        }
        // every CTA's source deposits are in acc before any CTA reads acc
        __threadfence();
        cl.sync();
    }

    // ---- this CTA's deposits into shared memory, every load in flight at once
    extern __shared__ __align__(16) unsigned char fsmem[];
    unsigned long long *s_acc = reinterpret_cast<unsigned long long *>(fsmem);  // [ns][per_cta]
    for (int k = threadIdx.x; k < ns * per_cta; k += kFCT) {
        const int s = k / per_cta, j = c0 + (k - s * per_cta);
        s_acc[k] = j < c1 ? __ldcg(p.acc + ((size_t)Q * ns + s) * nn + j) : 0ULL;
    }
    __syncthreads();

    // ---- integer sums over this thread's nodes, one species at a time: the rows'
    // inclusive sum R (rows 1..N-1), the weighted sum W = sum (N-j) acc[j] and the
    // total T (nodes j < N); then R's exclusive prefix over the CTA's threads
    u128 before[kMaxSpecies];
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
        before[s] = 0;
        if (s >= ns)
            continue;
        u128 run = 0, wsum = 0, tsum = 0;
        for (int j = j0; j < j1; ++j) {
            const unsigned long long v = s_acc[s * per_cta + (j - c0)];
            if (j < N)
                tsum += v;
            if (j >= 1 && j < N) {
                run += v;
                wsum += (u128)v * (unsigned)(N - j);
            }
        }
        u128 incl = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            u128 y = shfl_up_u128(incl, o);
            if (lane >= o)
                incl += y;
        }
        if (lane == 31)
            s_warp[s][warp] = incl;
        before[s] = incl - run;
        // W and T: warp sums (integers, so order-free), one partial per warp
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            wsum += shfl_down_u128(wsum, o);
            tsum += shfl_down_u128(tsum, o);
        }
        if (lane == 0) {
            s_wpart[s][warp][0] = wsum;
            s_wpart[s][warp][1] = tsum;
        }
    }
    __syncthreads();
    if (threadIdx.x < ns) {
        u128 r = 0, w2 = 0, t2 = 0;
        for (int w = 0; w < kFCW; ++w) {
            r += s_warp[threadIdx.x][w];
            w2 += s_wpart[threadIdx.x][w][0];
            t2 += s_wpart[threadIdx.x][w][1];
        }
        s_tot[threadIdx.x][0] = r;
        s_tot[threadIdx.x][1] = w2;
        s_tot[threadIdx.x][2] = t2;
    }
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
        if (s >= ns)
            break;
        u128 wp = 0;
        for (int w = 0; w < warp; ++w)
            wp += s_warp[s][w];
        before[s] += wp;
    }
    cl.sync();
    // gather the CTAs' totals (distributed shared memory), one remote load per
    // thread; then thread (s, q) sums quantity q of species s over the cluster and
    // converts it (and, for R, the CTAs before this one), and one thread forms the
    // step's scalars
    __shared__ u128 s_all[kMaxSpecies][kC][3];
    if (threadIdx.x < ns * kC * 3) {
        const int s = threadIdx.x / (kC * 3), r = (threadIdx.x / 3) % kC, q = threadIdx.x % 3;
        s_all[s][r][q] = *cl.map_shared_rank(&s_tot[s][q], r);
    }
    // this CTA's reads of the others' shared memory are done; the matching wait
    // before exit keeps every CTA alive until all of them have read
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < ns * 3) {
        const int s = threadIdx.x / 3, q = threadIdx.x % 3;
        u128 tot = 0, off = 0;
        for (int r = 0; r < kC; ++r) {
            tot += s_all[s][r][q];
            if (r < rank)
                off += s_all[s][r][q];
        }
        if (q == 0)
            s_off[s] = off;
        s_dbl[s][q] = u128_to_double(tot);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sumW = 0.0, sumR = 0.0, sumT = 0.0;
        for (int s = 0; s < ns; ++s) {
            const double cs = p.sp[s].rho_unit;
            sumR = fma(cs, s_dbl[s][0], sumR);
            sumW = fma(cs, s_dbl[s][1], sumW);
            sumT = fma(cs, s_dbl[s][2], sumT);
        }
        const double mean = p.periodic ? sumT * p.inv_n : 0.0;
        const double sumP = p.k2 * (sumW - mean * 0.5 * (double)N * (double)(N - 1));
        s_c[0] = p.periodic ? sumP * p.inv_n : (p.phi_hi - p.phi_lo + sumP) * p.inv_n;  // D0
        s_c[1] = p.k2 * (sumR - mean * (double)(N - 1));                                // P_{N-1}
        s_c[2] = mean;
    }
    __syncthreads();
    const double D0 = s_c[0], P_last = s_c[1], mean = s_c[2];
    const double k2 = p.k2, inv2dx = 0.5 * p.inv_dx;

    // ---- E on this thread's nodes.  With P_{j-1} + P_j = k2 (sum_s c_s X_s[j] -
    // mean (2j - 1)), X_s[j] = A_s[j-1] + A_s[j] (the integer pair sum, converted once
    // per species), E_j = (P_{j-1} + P_j - 2 D0) / (2 dx) is
    //   sum_s K_s X_s[j] + (B - a j),  K_s = k2 c_s / (2 dx),
    //   a = 2 k2 mean / (2 dx),  B = (k2 mean - 2 D0) / (2 dx)
    // (a = 0 between plates): one multiply-add per species and node.
    double K[kMaxSpecies];
    u128 A[kMaxSpecies];  // A_s[j0 - 1] (prefix before the chunk's first row)
#pragma unroll
    for (int s = 0; s < kMaxSpecies; ++s) {
        K[s] = (s < ns) ? k2 * p.sp[s].rho_unit * inv2dx : 0.0;
        A[s] = (s < ns) ? s_off[s] + before[s] : (u128)0;
    }
    const double a_j = 2.0 * k2 * mean * inv2dx, B = (k2 * mean - 2.0 * D0) * inv2dx;
    for (int j = j0; j < j1; ++j) {
        double e;
        if (j == 0) {
            e = p.periodic ? ((P_last + 0.0) - 2.0 * D0) * inv2dx : -D0 * p.inv_dx;
        } else if (!p.periodic && j == N) {
            e = (P_last - D0) * p.inv_dx;
        } else {
            e = p.periodic ? fma(-a_j, (double)j, B) : B;
#pragma unroll
            for (int s = 0; s < kMaxSpecies; ++s) {
                if (s >= ns)
                    break;
                const u128 prev = A[s];
                A[s] += s_acc[s * per_cta + (j - c0)];  // row j (1 <= j <= N-1)
                e = fma(K[s], u128_to_double(prev + A[s]), e);
            }
        }
        p.E64[j] = e;
        p.E[j] = (float)e;
    }
    if (p.wave_on) {  // test-particle mode: the prescribed field at this time level instead
        const double tw = (double)(mode >= 1 ? step + 1 : step) * p.dt64;
        for (int j = j0; j < j1; ++j) {
            const double e = wave_E(p, j, tw);
            p.E64[j] = e;
            p.E[j] = (float)e;
        }
    }

    if (mode >= 1) {
        // the deposit of rho^n is consumed: clear this CTA's nodes of it for the next
        // step's particle kernel
        for (int k = threadIdx.x; k < ns * (c1 - c0); k += kFCT) {
            const int s = k / (c1 - c0), j = c0 + (k - s * (c1 - c0));
            p.acc[((size_t)P * ns + s) * nn + j] = 0ULL;
        }
        // every CTA has read the step's state (before the exchange): CTA 0 updates it,
        // thread s for species s, from the counters read at the start
        if (rank == 0 && (int)threadIdx.x < ns) {
            const int s = threadIdx.x;
            const bool cut = s_ninj[s] < 0;
            const long long k = cut ? -s_ninj[s] - 1 : s_ninj[s];
            if (cut)
                atomicCAS(&st->error, 0, SLPIC_ERR_CAPACITY);
            st->src_frac[s] = s_frac[s];
            st->holes[s][P ^ 1] = mode == 1 ? (P ? pf_holes1 : pf_holes0) + pf_ab0 + pf_ab1 : 0ULL;
            st->count[s][P ^ 1] = (unsigned long long)(s_base[s] + k);
            st->injected_total[s] = pf_inj + k;
            st->absorbed_total[s][0] = pf_at0 + (long long)pf_ab0;
            st->absorbed_total[s][1] = pf_at1 + (long long)pf_ab1;
            st->absorbed_step[s][0] = 0ULL;
            st->absorbed_step[s][1] = 0ULL;
            st->count[s][P] = 0ULL;
            st->holes[s][P] = 0ULL;
            st->iterative_total[s] = pf_it + (long long)pf_hard;
            st->hard_n[s] = 0ULL;
        }
        // the step index is read at the start of every CTA: advance it last
        __syncthreads();
        if (rank == 0 && threadIdx.x == 0)
            st->step = step + 1;
    }
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// one CTA per SM: the registers are there for the taking (64 would spill)
__global__ void __cluster_dims__(kFieldClusterCtas, 1, 1) __launch_bounds__(kFieldClusterThreads, 1)
    k_field(const __grid_constant__ StepParams p, int mode)
{
    span_enter(p.st, 2);
    field_body<kFieldClusterCtas>(p, mode);
    span_exit(p.st, 2);
}

// the same on a cluster of kFieldClusterCtasWide CTAs (a non-portable cluster size, used
// where the GPU can schedule it): half the nodes, and half the FP64 work, per SM
__global__ void __cluster_dims__(kFieldClusterCtasWide, 1, 1)
    __launch_bounds__(kFieldClusterThreads, 1) k_field_wide(const __grid_constant__ StepParams p,
                                                            int mode)
{
    span_enter(p.st, 2);
    field_body<kFieldClusterCtasWide>(p, mode);
    span_exit(p.st, 2);
}

// batched: one cluster per instance
__global__ void __cluster_dims__(kFieldClusterCtas, 1, 1) __launch_bounds__(kFieldClusterThreads, 3)
    k_field_batch(const StepParams *__restrict__ ps, int mode)
{
    __shared__ StepParams s_p;
    load_params(s_p, ps + blockIdx.x / kFC);
    field_body<kFieldClusterCtas>(s_p, mode);
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
        const int c = sp.cell[P][i];
        if (c < 0)
            continue;  // hole
        float4 q = sp.pv[P][i];
        double bt = (double)beta_q(sp.kind, q.y, q.z, q.w, v0_cell(p, sp, c));
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
int field_max_nodes() { return 1 << 16; }

// k_field_wide where a cluster of its size fits on this GPU (set by configure_kernels),
// else k_field
static bool g_field_wide = false;

cudaError_t configure_kernels(int nn)
{
    // the attributes only ever grow: simulations of several sizes share the kernels
    static std::mutex mu;
    static int configured = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (nn <= configured)
        return cudaSuccess;
    configured = nn;
    cudaError_t e = cudaSuccess;
    for (auto f : {k_particles_compact<false>, k_particles_compact<true>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)particle_kernel_smem_bytes(nn));
        if (e != cudaSuccess)
            return e;
    }
    for (auto f : {k_particles<false>, k_particles<true>}) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)particle_inplace_smem_bytes(nn));
        if (e != cudaSuccess)
            return e;
    }
    e = cudaFuncSetAttribute(k_deposit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(nn * sizeof(unsigned long long)));
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(k_field, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)field_cluster_smem_bytes(nn, kMaxSpecies, kFC));
    if (e != cudaSuccess)
        return e;
    // the wide field kernel if a cluster of its size can be resident here (else the
    // portable 8-CTA kernel; a refusal is not an error)
    {
        const size_t wsmem = field_cluster_smem_bytes(nn, kMaxSpecies, kFieldClusterCtasWide);
        int nclusters = 0;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kFieldClusterCtasWide, 1, 1);
        cfg.blockDim = dim3(kFCT, 1, 1);
        cfg.dynamicSmemBytes = wsmem;
        g_field_wide =
            cudaFuncSetAttribute(k_field_wide, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_field_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)wsmem) == cudaSuccess &&
            cudaOccupancyMaxActiveClusters(&nclusters, k_field_wide, &cfg) == cudaSuccess &&
            nclusters >= 1;
        cudaGetLastError();
    }
    return cudaFuncSetAttribute(k_potential, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)field_smem_bytes(nn));
}

cudaError_t particle_ctas_per_sm(int nn, int *inplace, int *compacting)
{
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(inplace, k_particles<false>, kPB,
                                                                  particle_inplace_smem_bytes(nn));
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(compacting, k_particles_compact<false>, kPB,
                                                         particle_kernel_smem_bytes(nn));
}

void launch_particles(const StepParams &p, int ctas_per_species, bool compact, cudaStream_t st)
{
    dim3 grid(ctas_per_species, p.ns);
    const size_t smem = compact ? particle_kernel_smem_bytes(p.nn) : particle_inplace_smem_bytes(p.nn);
    if (compact)
        (p.lam ? k_particles_compact<true> : k_particles_compact<false>)<<<grid, kPB, smem, st>>>(p);
    else
        (p.lam ? k_particles<true> : k_particles<false>)<<<grid, kPB, smem, st>>>(p);
}

cudaError_t configure_particles_tma(int nn, int *stages)
{
    *stages = 0;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess)
        return e;
    const long long room = (long long)optin - 1024;  // static shared memory and margin
    int k = 4;
    while (k >= 2 && (long long)particle_tma_smem_bytes(nn, k) > room)
        --k;
    if (k < 2)
        return cudaSuccess;
    e = cudaFuncSetAttribute(k_particles_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_particles_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)room);
    if (e == cudaSuccess)
        *stages = k;
    return e;
}

void launch_particles_tma(const StepParams &p, int ctas, int stages, cudaStream_t st)
{
    (p.lam ? k_particles_tma<true> : k_particles_tma<false>)<<<ctas, kTmaThreads,
                                                               particle_tma_smem_bytes(p.nn, stages),
                                                               st>>>(p, stages);
}

void launch_hard(const StepParams &p, int ctas, bool compact, cudaStream_t st)
{
    (p.lam ? k_hard<true> : k_hard<false>)<<<ctas, 256, 0, st>>>(p, compact ? 1 : 0);
}

void launch_particles_batch(const StepParams *d_params, const int4 *d_work, int n_work,
                            int max_nn, bool compact, cudaStream_t st)
{
    if (compact)
        k_particles_compact_batch<<<n_work, kPB, particle_kernel_smem_bytes(max_nn), st>>>(d_params,
                                                                                          d_work);
    else
        k_particles_batch<<<n_work, kPB, particle_inplace_smem_bytes(max_nn), st>>>(d_params, d_work);
}

void launch_hard_batch(const StepParams *d_params, int m, int ctas_per_instance, bool compact,
                       cudaStream_t st)
{
    k_hard_batch<<<dim3(ctas_per_instance, m), 256, 0, st>>>(d_params, compact ? 1 : 0);
}

void launch_field_batch(const StepParams *d_params, int m, int max_nn, int max_ns, int mode,
                        cudaStream_t st)
{
    k_field_batch<<<m * kFC, kFCT, field_cluster_smem_bytes(max_nn, max_ns, kFC), st>>>(d_params, mode);
}

cudaError_t configure_batch_kernels(int max_nn, int *inplace_per_sm, int *compact_per_sm)
{
    cudaError_t e = cudaFuncSetAttribute(k_particles_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)particle_inplace_smem_bytes(max_nn));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_particles_compact_batch,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)particle_kernel_smem_bytes(max_nn));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_field_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)field_cluster_smem_bytes(max_nn, kMaxSpecies, kFC));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(inplace_per_sm, k_particles_batch, kPB,
                                                          particle_inplace_smem_bytes(max_nn));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(compact_per_sm, k_particles_compact_batch,
                                                          kPB, particle_kernel_smem_bytes(max_nn));
    return e;
}

size_t field_cluster_smem_bytes(int nn, int ns, int ctas)
{
    return (size_t)ns * ((nn + ctas - 1) / ctas) * sizeof(unsigned long long);
}

void launch_field(const StepParams &p, int mode, cudaStream_t st)
{
    if (g_field_wide)
        k_field_wide<<<kFieldClusterCtasWide, kFCT,
                       field_cluster_smem_bytes(p.nn, p.ns, kFieldClusterCtasWide), st>>>(p, mode);
    else
        k_field<<<kFC, kFCT, field_cluster_smem_bytes(p.nn, p.ns, kFC), st>>>(p, mode);
}

// the latest deposit ([species][nn]) and E copied for a read-back that runs beside
// the following steps
__global__ void k_snapshot(const unsigned long long *__restrict__ dep, unsigned long long *__restrict__ dep_out,
                           size_t ndep, const float *__restrict__ E, float *__restrict__ E_out, int nn)
{
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < ndep + nn;
         t += (size_t)gridDim.x * blockDim.x) {
        if (t < ndep)
            dep_out[t] = dep[t];
        else
            E_out[t - ndep] = E[t - ndep];
    }
}

void launch_snapshot(const unsigned long long *dep, unsigned long long *dep_out, size_t ndep,
                     const float *E, float *E_out, int nn, cudaStream_t st)
{
    const size_t n = ndep + (size_t)nn;
    k_snapshot<<<(unsigned)std::min<size_t>((n + 255) / 256, 1024), 256, 0, st>>>(dep, dep_out, ndep,
                                                                                  E, E_out, nn);
}

void launch_potential(const StepParams &p, const unsigned long long *dep, long long step,
                      cudaStream_t st)
{
    k_potential<<<1, kFT, field_smem_bytes(p.nn), st>>>(p, dep, step);
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
