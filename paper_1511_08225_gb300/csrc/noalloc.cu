// noalloc.cu -- one particle step on caller-owned device arrays, allocating nothing.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's step loop whose memory pool owns the whole device, services that
// reserve every byte at start-up and forbid later allocations, and latency-
// critical loops that cannot afford the implicit device synchronisation a
// cudaMalloc/cudaFree may cause.  slpic_particle_step_noalloc serves them: it runs
// the same per-particle step as the simulation handle's particle kernel, but the
// only global scratch it needs (an output counter, two wall counters and the int64
// deposit accumulator) lives in one file-scope __device__ array below, sized for
// at most kNoallocMaxNodes grid nodes.  Every GPU that loads the library holds this
// array (about 128 KiB) until the process exits.
//
// The array's name in host code is only a host-side stand-in, not a device
// address; the host code below asks the runtime for the real address once per
// device (cudaGetSymbolAddress, with that device current) and passes it to the
// kernel.  All calls share the array: each call clears the part it uses before the
// kernel runs, so the array keeps whatever the last call left, and calls that
// overlap on the GPU (different streams, or different host threads at once) race
// on it.
#include <algorithm>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "kernels.h"
#include "particle_step.cuh"
#include "push_math.cuh"
#include "slpic.h"
#include "slpic_internal.cuh"

namespace slpic {

constexpr int kNoallocMaxNodes = 16384;
constexpr int kNoallocCounters = 4;  // [0] survivors, [1] absorbed at x=0, [2] at x=L,
                                     // [3] particles skipped as invalid

static __device__ __align__(256) unsigned long long
    g_noalloc_scratch[kNoallocCounters + kNoallocMaxNodes];

constexpr int kNB = 256;  // threads per CTA
constexpr int kNWarps = kNB / 32;

// One particle per thread per iteration; survivors compacted per block with one
// atomicAdd on the scratch counter.  Deposit into a shared-memory histogram of
// the whole grid, flushed once per CTA into the scratch accumulator.
__global__ void __launch_bounds__(kNB) k_particles_noalloc(StepParams p, SpeciesDev sp,
                                                           long long n, const int32_t *cin,
                                                           const float4 *vin, int32_t *cout,
                                                           float4 *vout,
                                                           unsigned long long *scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *s_hist = reinterpret_cast<unsigned long long *>(smem);
    float *s_E = reinterpret_cast<float *>(s_hist + p.nn);
    __shared__ int s_off[kNWarps];
    __shared__ unsigned long long s_base;
    __shared__ unsigned int s_abs[3];  // absorbed at x=0, at x=L; invalid
    unsigned long long *counters = scratch;
    unsigned long long *acc = scratch + kNoallocCounters;

    for (int j = threadIdx.x; j < p.nn; j += kNB) {
        s_hist[j] = 0ULL;
        s_E[j] = p.E[j];
    }
    if (threadIdx.x < 3)
        s_abs[threadIdx.x] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long stride = (long long)gridDim.x * kNB;
    for (long long b0 = (long long)blockIdx.x * kNB; b0 < n; b0 += stride) {
        long long i = b0 + threadIdx.x;
        bool live = i < n;
        int c = 0;
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (live) {
            c = cin[i];
            q = vin[i];
            // the caller's data index the shared-memory grid: a cell outside the grid
            // or an offset outside [0, 1) is skipped and counted, never used
            if ((unsigned)c >= (unsigned)p.n_cells || !(q.x >= 0.0f && q.x < 1.0f)) {
                live = false;
                atomicAdd(&s_abs[2], 1u);
            } else {
                int wall = 0;
                live = advance(p, sp, s_E, s_hist, c, q, wall);
                if (!live)
                    atomicAdd(&s_abs[wall], 1u);
            }
        }
        unsigned mask = __ballot_sync(0xffffffffu, live);
        if (lane == 0)
            s_off[warp] = __popc(mask);
        __syncthreads();
        if (warp == 0) {
            int v = lane < kNWarps ? s_off[lane] : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o)
                    incl += y;
            }
            if (lane < kNWarps)
                s_off[lane] = incl - v;
            if (lane == 31)
                s_base = incl ? atomicAdd(counters, (unsigned long long)incl) : 0ULL;
        }
        __syncthreads();
        if (live) {
            unsigned long long o =
                s_base + (unsigned long long)s_off[warp] + __popc(mask & ((1u << lane) - 1u));
            cout[o] = c;
            vout[o] = q;
        }
        __syncthreads();
    }
    for (int j = threadIdx.x; j < p.nn; j += kNB) {
        unsigned long long v = s_hist[j];
        if (v)
            atomicAdd(acc + j, v);
    }
    if (threadIdx.x < 3 && s_abs[threadIdx.x])
        atomicAdd(counters + 1 + threadIdx.x, (unsigned long long)s_abs[threadIdx.x]);
}

}  // namespace slpic

using namespace slpic;

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the scratch.
int scratch_address(int dev, unsigned long long **out)
{
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return SLPIC_ERR_CUDA;
        e = cudaFuncSetAttribute(k_particles_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)particle_smem_bytes(kNoallocMaxNodes));
        if (e != cudaSuccess)
            return SLPIC_ERR_CUDA;
        g_scratch_addr[dev] = ptr;
    }
    *out = (unsigned long long *)g_scratch_addr[dev];
    return SLPIC_OK;
}
}  // namespace

extern "C" int slpic_particle_step_noalloc(const slpic_config *cfg, int species, int64_t n,
                                           const int32_t *cell_in, const float *state_in,
                                           const float *E, int32_t *cell_out,
                                           float *state_out, int64_t *charge_out,
                                           int64_t *n_out, int64_t *absorbed, void *stream)
{
    if (!cfg || !n_out || !absorbed || !E || !charge_out || n < 0)
        return SLPIC_ERR_INVALID;
    if (n > 0 && (!cell_in || !state_in || !cell_out || !state_out))
        return SLPIC_ERR_INVALID;
    if (cfg->ndim != 1 || cfg->n_cells < 2 || !(cfg->dx > 0) || !(cfg->dt > 0) ||
        (cfg->bc != SLPIC_BC_PERIODIC && cfg->bc != SLPIC_BC_DIRICHLET_ABSORB))
        return SLPIC_ERR_INVALID;
    if (species < 0 || species >= cfg->n_species || cfg->n_species > SLPIC_MAX_SPECIES)
        return SLPIC_ERR_INVALID;
    const int nn = cfg->bc == SLPIC_BC_PERIODIC ? cfg->n_cells : cfg->n_cells + 1;
    if (nn > kNoallocMaxNodes)  // beyond the fixed scratch
        return SLPIC_ERR_CAPACITY;
    const slpic_species &s = cfg->species[species];
    if (!(s.m > 0) || s.beta_kind < SLPIC_BETA_ONE || s.beta_kind > SLPIC_BETA_RELATIVISTIC ||
        (s.beta_kind != SLPIC_BETA_ONE && !(s.v0 > 0)))
        return SLPIC_ERR_INVALID;
    if (s.beta_kind != SLPIC_BETA_ONE && cfg->dt * s.v0 > cfg->dx * (1.0 + 1e-12))
        return SLPIC_ERR_CFL;
    if (((uintptr_t)state_in | (uintptr_t)state_out) & 15)
        return SLPIC_ERR_INVALID;
    // survivors are packed across CTAs, so an output range that overlaps an input
    // range could overwrite particles another CTA has not read yet
    if (n > 0) {
        auto overlap = [n](const void *a, size_t ea, const void *b, size_t eb) {
            const uintptr_t a0 = (uintptr_t)a, a1 = a0 + (uintptr_t)n * ea;
            const uintptr_t b0 = (uintptr_t)b, b1 = b0 + (uintptr_t)n * eb;
            return a0 < b1 && b0 < a1;
        };
        if (overlap(cell_in, 4, cell_out, 4) || overlap(state_in, 16, state_out, 16) ||
            overlap(cell_in, 4, state_out, 16) || overlap(state_in, 16, cell_out, 4))
            return SLPIC_ERR_INVALID;
    }

    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return SLPIC_ERR_CUDA;
    unsigned long long *scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc)
        return rc;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t st = (cudaStream_t)stream;

    StepParams p{};
    p.n_cells = cfg->n_cells;
    p.nn = nn;
    p.periodic = cfg->bc == SLPIC_BC_PERIODIC;
    p.ns = 1;
    p.dt = (float)cfg->dt;
    p.dt_dx = (float)(cfg->dt / cfg->dx);
    p.E = const_cast<float *>(E);
    SpeciesDev sp{};
    sp.qm = (float)(s.q / s.m);
    sp.v0 = s.beta_kind == SLPIC_BETA_ONE ? INFINITY : (float)s.v0;
    sp.kind = s.beta_kind;

    // the counters and the accumulator must start at zero on every call
    e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (kNoallocCounters + nn), st);
    if (e != cudaSuccess)
        return SLPIC_ERR_CUDA;
    if (n > 0) {
        int blocks =
            (int)std::max<long long>(1, std::min<long long>((n + kNB - 1) / kNB, (long long)sms * 4));
        k_particles_noalloc<<<blocks, kNB, particle_smem_bytes(nn), st>>>(
            p, sp, n, cell_in, reinterpret_cast<const float4 *>(state_in), cell_out,
            reinterpret_cast<float4 *>(state_out), scratch);
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return SLPIC_ERR_CUDA;
    }
    e = cudaMemcpyAsync(charge_out, scratch + kNoallocCounters, sizeof(int64_t) * nn,
                        cudaMemcpyDeviceToDevice, st);
    unsigned long long cnt[4] = {0, 0, 0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cnt, scratch, sizeof(cnt), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return SLPIC_ERR_CUDA;
    *n_out = (int64_t)cnt[0];
    absorbed[0] = (int64_t)cnt[1];
    absorbed[1] = (int64_t)cnt[2];
    return cnt[3] ? SLPIC_ERR_INVALID : SLPIC_OK;
}
