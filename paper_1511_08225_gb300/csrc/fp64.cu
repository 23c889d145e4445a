// fp64.cu -- the plain FP64 form of the 1D SLPIC step (include/slpic_fp64.h).
//
// Per step (Appendix A, Eq. slpicIntegration):
//   k_step64    gather E^n (FP64, grid in shared memory) -> velocity push in FP64
//               -> x^{n+1} = x^n + beta v dt -> walls -> FP64 CIC deposit of
//               rho^{n+1} (global double atomics) -> survivors packed into the
//               other buffer
//   k_inject64  one CTA: source particles (FP64) appended and deposited; bookkeeping
//   k_field64   one CTA: rho = sum_s q_s n_s, Poisson by FP64 prefix sums, E
//
// The velocity push solves the same equation as the mixed-precision library: with
// w the velocity component along a, D = |v_perp|^2 and A = |a|, the time needed to
// go from w_a to w is [H(w) - H(w_a)] / A with H(w) = int_0^w dw'/beta(sqrt(w'^2+D))
// in closed form (int sqrt(w^2+D) dw = (w sqrt(w^2+D) + D asinh(w/sqrt D))/2), and
// the new w solves H(w) = H(w_a) + A dt by Newton kept inside the bracket
// [w_a, w_a + A dt] (H' = 1/beta >= 1).
#include <cmath>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "slpic_fp64.h"

namespace slpic {
int check_config(const slpic_config *c, std::string &why);  // api.cu
void set_create_error(const std::string &msg);              // api.cu
}

namespace slpic64 {

constexpr int kMaxS = SLPIC_MAX_SPECIES;
constexpr int kThreads = 256;
constexpr int kItems = 4;
constexpr int kTile = kThreads * kItems;
constexpr int kWarps = kThreads / 32;
constexpr int kFieldThreads = 1024;

struct Sp64 {
    double *x[2], *vx[2], *vy[2], *vz[2];
    long long capacity;
    double qm, v0, vth, w, inv_w, w_dx;  // w_dx = w / dx
    int kind;
};

struct St64 {
    long long step;
    unsigned long long count[kMaxS][2];
    unsigned long long absorbed_step[kMaxS][2];
    long long absorbed_total[kMaxS][2];
    long long injected_total[kMaxS];
    double src_frac[kMaxS];
    int error;
};

struct P64 {
    int N, nn, periodic, ns;
    double dx, dt, L, k2, phi_lo, phi_hi, q[kMaxS];
    int src_mode, src_ref;
    double src_lo, src_len, src_rate;
    unsigned long long seed;
    Sp64 sp[kMaxS];
    double *dens;  // [ns][nn] number density of the deposit being built
    double *rho, *phi, *E;
    St64 *st;
};

// ---- beta and the time along the velocity line (FP64) ---------------------------
__device__ __forceinline__ double beta64(int kind, double r, double v0)
{
    if (kind == SLPIC_BETA_ONE)
        return 1.0;
    if (kind == SLPIC_BETA_HEAVISIDE)
        return r <= v0 ? 1.0 : v0 / r;
    return v0 / sqrt(r * r + v0 * v0);
}

__device__ __forceinline__ double F64(double w, double D)
{
    if (D <= 0.0)
        return 0.5 * w * fabs(w);
    return 0.5 * (w * sqrt(w * w + D) + D * asinh(w / sqrt(D)));
}

__device__ double H64(int kind, double w, double D, double v0)
{
    if (kind == SLPIC_BETA_ONE)
        return w;
    if (kind == SLPIC_BETA_RELATIVISTIC)
        return F64(w, D + v0 * v0) / v0;
    if (D < v0 * v0) {
        const double W0 = sqrt(v0 * v0 - D);
        if (fabs(w) <= W0)
            return w;
        const double s = w < 0.0 ? -1.0 : 1.0;
        return s * (W0 + (F64(fabs(w), D) - F64(W0, D)) / v0);
    }
    return F64(w, D) / v0;
}

__device__ __forceinline__ double inv_beta64(int kind, double w, double D, double v0)
{
    return 1.0 / beta64(kind, sqrt(w * w + D), v0);
}

// new velocity component along x after one step of the push with a = (ax, 0, 0)
__device__ double push64(int kind, double ux, double uy, double uz, double ax, double dt, double v0)
{
    if (kind == SLPIC_BETA_ONE || ax == 0.0)
        return ux + ax * dt;  // beta == 1 (or no force): plain leapfrog
    const double A = fabs(ax), sg = ax > 0.0 ? 1.0 : -1.0;
    const double wa = sg * ux, D = uy * uy + uz * uz, budget = A * dt;
    const double Ha = H64(kind, wa, D, v0), T = Ha + budget;
    // H is evaluated to a few ulp of its size: below that the residual is noise
    const double gtol = 8.0 * 2.220446049250313e-16 * (fabs(Ha) + budget);
    double lo = wa, hi = wa + budget, w = hi;
    for (int it = 0; it < 60; ++it) {
        const double g = H64(kind, w, D, v0) - T;
        if (fabs(g) <= gtol)
            break;
        if (g > 0.0)
            hi = w;
        else
            lo = w;
        double wn = w - g / inv_beta64(kind, w, D, v0);
        if (!(wn > lo && wn < hi))
            wn = 0.5 * (lo + hi);
        const bool small = fabs(wn - w) <= 1e-14 * fmax(fabs(w), budget);
        w = wn;
        if (small)
            break;
    }
    return sg * w;
}

// ---- counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) ------------------
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double u53(unsigned long long key, unsigned long long i)
{
    // uniform on (0, 1] from the i-th output (top 24 bits, as the mixed form uses)
    const unsigned long long z = mix64(key + (i + 1ULL) * 0x9E3779B97F4A7C15ULL);
    return (double)((z >> 40) + 1ULL) * (1.0 / 16777216.0);
}

// ---- particle step ----------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_step64(P64 p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    double *s_E = reinterpret_cast<double *>(smem);  // [nn]
    __shared__ int s_cnt[kItems * kWarps];
    __shared__ unsigned long long s_base;
    __shared__ unsigned s_abs[2];
    const int s = blockIdx.y;
    const Sp64 &sp = p.sp[s];
    const int P = (int)(p.st->step & 1);
    const long long n = (long long)p.st->count[s][P];
    const int N = p.N, nn = p.nn;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = threadIdx.x; j < nn; j += blockDim.x)
        s_E[j] = p.E[j];
    if (threadIdx.x < 2)
        s_abs[threadIdx.x] = 0u;
    __syncthreads();
    const long long ntiles = (n + kTile - 1) / kTile;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long base = t * kTile;
        bool live[kItems];
        double x[kItems], vx[kItems], vy[kItems], vz[kItems];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const long long i = base + k * kThreads + threadIdx.x;
            live[k] = i < n;
            if (live[k]) {
                x[k] = sp.x[P][i];
                vx[k] = sp.vx[P][i];
                vy[k] = sp.vy[P][i];
                vz[k] = sp.vz[P][i];
            }
        }
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (!live[k])
                continue;
            const double xi = x[k] / p.dx;
            const double cf = floor(xi);
            const int c = min(max((int)cf, 0), N - 1);
            const double d = xi - cf;
            int c1 = c + 1;
            if (p.periodic && c1 == N)
                c1 = 0;
            const double ax = sp.qm * ((1.0 - d) * s_E[c] + d * s_E[c1]);
            vx[k] = push64(sp.kind, vx[k], vy[k], vz[k], ax, p.dt, sp.v0);
            const double b = beta64(sp.kind, sqrt(vx[k] * vx[k] + vy[k] * vy[k] + vz[k] * vz[k]),
                                    sp.v0);
            double xn = x[k] + b * vx[k] * p.dt;
            if (p.periodic) {
                xn -= p.L * floor(xn / p.L);
                if (xn >= p.L)
                    xn -= p.L;
            } else if (xn < 0.0 || xn >= p.L) {
                atomicAdd(&s_abs[xn < 0.0 ? 0 : 1], 1u);
                live[k] = false;
                continue;
            }
            x[k] = xn;
            const double xj = xn / p.dx;
            const double cj = floor(xj);
            const int cn = min(max((int)cj, 0), N - 1);
            const double dn = xj - cj;
            int cn1 = cn + 1;
            if (p.periodic && cn1 == N)
                cn1 = 0;
            atomicAdd(p.dens + (size_t)s * nn + cn, sp.w_dx * b * (1.0 - dn));
            atomicAdd(p.dens + (size_t)s * nn + cn1, sp.w_dx * b * dn);
        }
        // pack the survivors (one global atomic per tile)
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
                sp.x[P ^ 1][o] = x[k];
                sp.vx[P ^ 1][o] = vx[k];
                sp.vy[P ^ 1][o] = vy[k];
                sp.vz[P ^ 1][o] = vz[k];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 2 && s_abs[threadIdx.x])
        atomicAdd(&p.st->absorbed_step[s][threadIdx.x], (unsigned long long)s_abs[threadIdx.x]);
}

// deposit of the current particles (after loading)
__global__ void __launch_bounds__(kThreads) k_deposit64(P64 p)
{
    const int s = blockIdx.y;
    const Sp64 &sp = p.sp[s];
    const int P = (int)(p.st->step & 1);
    const long long n = (long long)p.st->count[s][P];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double xj = sp.x[P][i] / p.dx;
        const double cj = floor(xj);
        const int c = min(max((int)cj, 0), p.N - 1);
        const double d = xj - cj;
        int c1 = c + 1;
        if (p.periodic && c1 == p.N)
            c1 = 0;
        const double vx = sp.vx[P][i], vy = sp.vy[P][i], vz = sp.vz[P][i];
        const double b = beta64(sp.kind, sqrt(vx * vx + vy * vy + vz * vz), sp.v0);
        atomicAdd(p.dens + (size_t)s * p.nn + c, sp.w_dx * b * (1.0 - d));
        atomicAdd(p.dens + (size_t)s * p.nn + c1, sp.w_dx * b * d);
    }
}

// source (the volume source of the library, in FP64) and bookkeeping; one CTA
__global__ void __launch_bounds__(1024) k_inject64(P64 p)
{
    __shared__ long long s_k[kMaxS], s_base[kMaxS];
    __shared__ double s_frac[kMaxS];
    __shared__ int s_cut[kMaxS];
    St64 *st = p.st;
    const long long step = st->step;
    const int P = (int)(step & 1);
    if (threadIdx.x < p.ns) {
        const int s = threadIdx.x;
        double S = 0.0;
        if (p.src_mode == SLPIC_SRC_LOSS_MATCHED) {
            const int r = p.src_ref;
            S = (double)(st->absorbed_step[r][0] + st->absorbed_step[r][1]) * p.sp[r].w;
        } else if (p.src_mode == SLPIC_SRC_RATE) {
            S = p.src_rate * p.dt;
        } else if (p.src_mode == SLPIC_SRC_WALL) {
            // one-sided flux of a stationary Maxwellian of density src_rate
            S = p.src_rate * p.sp[s].vth / sqrt(2.0 * 3.14159265358979323846) * p.dt;
        }
        long long k = 0;
        double f = st->src_frac[s];
        if (p.src_mode != SLPIC_SRC_NONE && p.sp[s].vth > 0.0) {
            f += S / p.sp[s].w;
            k = (long long)floor(f);
            f -= (double)k;
        }
        const long long have = (long long)st->count[s][P ^ 1];
        const long long room = p.sp[s].capacity - have;
        s_cut[s] = k > room;
        s_k[s] = k > room ? room : k;
        s_base[s] = have;
        s_frac[s] = f;
    }
    __syncthreads();
    const double two_pi = 6.283185307179586476925286766559;
    for (int s = 0; s < p.ns; ++s) {
        const Sp64 &sp = p.sp[s];
        const unsigned long long key =
            mix64(p.seed ^ mix64((unsigned long long)step * 16ULL + (unsigned)s + 1ULL));
        for (long long i = threadIdx.x; i < s_k[s]; i += blockDim.x) {
            const unsigned long long b8 = 8ULL * (unsigned long long)i;
            double xc, vx, vy, vz;
            if (p.src_mode == SLPIC_SRC_WALL) {
                // through the plate at x = L (the library's wall source, in FP64)
                const double vxm = sp.vth * sqrt(-2.0 * log(u53(key, b8 + 1)));
                const double rw = sp.vth * sqrt(-2.0 * log(u53(key, b8 + 2)));
                const double ph = two_pi * u53(key, b8 + 3);
                vx = -vxm;
                vy = rw * cos(ph);
                vz = rw * sin(ph);
                const double b = beta64(sp.kind, sqrt(vxm * vxm + vy * vy + vz * vz), sp.v0);
                xc = p.N - u53(key, b8) * b * vxm * p.dt / p.dx;
                if (!(xc < p.N))
                    xc = p.N - 1.0 / 1048576.0;
            } else {
                xc = p.src_lo + u53(key, b8) * p.src_len;
                const double r1 = sqrt(-2.0 * log(u53(key, b8 + 1)));
                const double r2 = sqrt(-2.0 * log(u53(key, b8 + 3)));
                const double ph = two_pi * u53(key, b8 + 2), ph2 = two_pi * u53(key, b8 + 4);
                vx = sp.vth * r1 * cos(ph);
                vy = sp.vth * r1 * sin(ph);
                vz = sp.vth * r2 * cos(ph2);
            }
            const long long o = s_base[s] + i;
            const double x = xc * p.dx;
            sp.x[P ^ 1][o] = x;
            sp.vx[P ^ 1][o] = vx;
            sp.vy[P ^ 1][o] = vy;
            sp.vz[P ^ 1][o] = vz;
            const double cf = floor(xc);
            const int c = min(max((int)cf, 0), p.N - 1);
            const double d = xc - cf;
            int c1 = c + 1;
            if (p.periodic && c1 == p.N)
                c1 = 0;
            const double b = beta64(sp.kind, sqrt(vx * vx + vy * vy + vz * vz), sp.v0);
            atomicAdd(p.dens + (size_t)s * p.nn + c, sp.w_dx * b * (1.0 - d));
            atomicAdd(p.dens + (size_t)s * p.nn + c1, sp.w_dx * b * d);
        }
    }
    __syncthreads();
    if (threadIdx.x < p.ns) {
        const int s = threadIdx.x;
        if (s_cut[s])
            atomicCAS(&st->error, 0, SLPIC_ERR_CAPACITY);
        st->src_frac[s] = s_frac[s];
        st->count[s][P ^ 1] = (unsigned long long)(s_base[s] + s_k[s]);
        st->count[s][P] = 0ULL;
        st->injected_total[s] += s_k[s];
        st->absorbed_total[s][0] += (long long)st->absorbed_step[s][0];
        st->absorbed_total[s][1] += (long long)st->absorbed_step[s][1];
        st->absorbed_step[s][0] = 0ULL;
        st->absorbed_step[s][1] = 0ULL;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        st->step = step + 1;
}

// exclusive block scan (FP64); every thread gets the block total
__device__ double scan64(double v, double *s_w, double *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        double x = lane < nw ? s_w[lane] : 0.0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o)
                x += y;
        }
        s_w[lane] = x;
    }
    __syncthreads();
    const double before = warp ? s_w[warp - 1] : 0.0;
    *total = s_w[nw - 1];
    __syncthreads();
    return before + incl - v;
}

// Poisson (Appendix A, Eq. LimPtclDynAppendixDotE), 3-point stencil, by prefix sums:
// with D_j = phi_{j+1} - phi_j, D_j = D_0 - P_j, P_j = k2 sum_{i=1..j} rho_i (k2 =
// dx^2/eps0); D_0 from sum_j D_j = phi_N - phi_0 (plates) or 0 (periodic, after
// removing the mean of rho); phi_j = phi_0 + j D_0 - sum_{i<j} P_i;
// E_j = -(D_{j-1} + D_j)/(2 dx), one-sided at the plates.  One CTA, each thread a
// contiguous chunk of at most kMaxChunk nodes; the consumed deposit is cleared.
constexpr int kMaxChunk = 64;

__global__ void __launch_bounds__(kFieldThreads) k_field64(P64 p)
{
    __shared__ double s_w[32];
    const int N = p.N, nn = p.nn;
    const int chunk = (nn + blockDim.x - 1) / blockDim.x;
    const int j0 = min(nn, (int)threadIdx.x * chunk), j1 = min(nn, j0 + chunk);
    double rv[kMaxChunk];
    double loc = 0.0;
    for (int k = 0; k < j1 - j0; ++k) {
        const int j = j0 + k;
        double r = 0.0;
        for (int s = 0; s < p.ns; ++s) {
            r += p.q[s] * p.dens[(size_t)s * nn + j];
            p.dens[(size_t)s * nn + j] = 0.0;
        }
        p.rho[j] = r;
        rv[k] = r;
        if (j < N)
            loc += r;
    }
    double tot;
    scan64(loc, s_w, &tot);
    const double mean = p.periodic ? tot / N : 0.0;
    // rows 1..N-1 of (rho - mean)
    double rs = 0.0;
    for (int k = 0; k < j1 - j0; ++k) {
        const int j = j0 + k;
        rv[k] = (j >= 1 && j < N) ? rv[k] - mean : 0.0;
        rs += rv[k];
    }
    double tR;
    const double pre = scan64(rs, s_w, &tR);
    const double Pprev0 = p.k2 * pre;  // P_{j0 - 1}
    double acc = pre, sP = 0.0;
    for (int k = 0; k < j1 - j0; ++k) {
        acc += rv[k];
        rv[k] = (j0 + k < N) ? p.k2 * acc : 0.0;  // now P_j
        sP += rv[k];
    }
    double sumP;
    const double exP = scan64(sP, s_w, &sumP);
    const double Plast = p.k2 * tR;  // P_{N-1}
    const double D0 = p.periodic ? sumP / N : (p.phi_hi - p.phi_lo + sumP) / N;
    const double phi0 = p.periodic ? 0.0 : p.phi_lo;
    double run = exP, phisum = 0.0;
    for (int k = 0; k < j1 - j0; ++k) {
        const int j = j0 + k;
        const double ph = (!p.periodic && j == N) ? p.phi_hi : phi0 + j * D0 - run;
        p.phi[j] = ph;
        if (j < N)
            phisum += ph;
        run += rv[k];
        const double Pm = (k > 0) ? rv[k - 1] : Pprev0;
        double e;
        if (p.periodic)
            e = -(((j == 0) ? D0 - Plast : D0 - Pm) + (D0 - rv[k])) / (2.0 * p.dx);
        else if (j == 0)
            e = -D0 / p.dx;
        else if (j == N)
            e = -(D0 - Plast) / p.dx;
        else
            e = -((D0 - Pm) + (D0 - rv[k])) / (2.0 * p.dx);
        p.E[j] = e;
    }
    if (p.periodic) {
        // gauge: mean(phi) = 0
        double pt;
        scan64(phisum, s_w, &pt);
        for (int j = j0; j < j1; ++j)
            p.phi[j] -= pt / N;
    }
}

}  // namespace slpic64

// =================================================================================
using namespace slpic64;

struct slpic_fp64_sim {
    slpic_config cfg{};
    cudaStream_t stream = nullptr, own_stream = nullptr;
    P64 p{};
    int ctas = 1;
    std::vector<void *> allocs;
    std::string err;
};

#define CK64(h, call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return SLPIC_ERR_CUDA;                                                         \
        }                                                                                  \
    } while (0)

static int fail64(slpic_fp64_t *h, int code, const std::string &m)
{
    h->err = m;
    return code;
}

extern "C" int slpic_fp64_create(const slpic_config *c, slpic_fp64_t **out)
{
    if (!out) {
        slpic::set_create_error("out is NULL");
        return SLPIC_ERR_INVALID;
    }
    std::string why;
    int rc = slpic::check_config(c, why);
    if (rc) {
        slpic::set_create_error(why);
        return rc;
    }
    int dev = 0, sms = 1, max_smem = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        slpic::set_create_error("no CUDA device");
        return SLPIC_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int nn = c->bc == SLPIC_BC_PERIODIC ? c->n_cells : c->n_cells + 1;
    const size_t smem = sizeof(double) * (size_t)nn;
    if (smem + 1024 > (size_t)max_smem || (nn + kFieldThreads - 1) / kFieldThreads > kMaxChunk) {
        slpic::set_create_error("grid too large for the FP64 kernels");
        return SLPIC_ERR_INVALID;
    }
    slpic_fp64_t *h = new slpic_fp64_t();
    h->cfg = *c;
    auto bail = [&](int code, const std::string &m) {
        slpic::set_create_error(m);
        slpic_fp64_destroy(h);
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
    P64 &p = h->p;
    p.N = c->n_cells;
    p.nn = nn;
    p.periodic = c->bc == SLPIC_BC_PERIODIC;
    p.ns = c->n_species;
    p.dx = c->dx;
    p.dt = c->dt;
    p.L = c->dx * c->n_cells;
    p.k2 = c->dx * c->dx / c->eps0;
    p.phi_lo = c->phi_lo;
    p.phi_hi = c->phi_hi;
    p.src_mode = c->src_mode;
    p.src_ref = c->src_ref_species;
    p.src_lo = c->src_lo_cells;
    p.src_len = c->src_len_cells;
    p.src_rate = c->src_rate;
    p.seed = c->seed;
    bool ok = alloc((void **)&p.st, sizeof(St64)) &&
              alloc((void **)&p.dens, sizeof(double) * nn * p.ns) &&
              alloc((void **)&p.rho, sizeof(double) * nn) && alloc((void **)&p.phi, sizeof(double) * nn) &&
              alloc((void **)&p.E, sizeof(double) * nn);
    for (int s = 0; ok && s < p.ns; ++s) {
        const slpic_species &sp = c->species[s];
        Sp64 &d = p.sp[s];
        for (int b = 0; ok && b < 2; ++b)
            ok = alloc((void **)&d.x[b], sizeof(double) * sp.capacity) &&
                 alloc((void **)&d.vx[b], sizeof(double) * sp.capacity) &&
                 alloc((void **)&d.vy[b], sizeof(double) * sp.capacity) &&
                 alloc((void **)&d.vz[b], sizeof(double) * sp.capacity);
        d.capacity = sp.capacity;
        d.qm = sp.q / sp.m;
        d.v0 = sp.v0;
        d.vth = sp.T_src > 0 ? std::sqrt(sp.T_src / sp.m) : 0.0;
        d.w = sp.w;
        d.inv_w = 1.0 / sp.w;
        d.w_dx = sp.w / c->dx;
        d.kind = sp.beta_kind;
        p.q[s] = sp.q;
    }
    if (!ok)
        return bail(SLPIC_ERR_OOM, "device allocation failed");
    cudaError_t e = cudaMemset(p.st, 0, sizeof(St64));
    if (e == cudaSuccess)
        e = cudaMemset(p.dens, 0, sizeof(double) * nn * p.ns);
    if (e == cudaSuccess)
        e = cudaMemset(p.E, 0, sizeof(double) * nn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_step64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step64, kThreads, smem);
    if (e != cudaSuccess || occ < 1)
        return bail(SLPIC_ERR_CUDA, "FP64 particle kernel cannot be resident");
    h->ctas = std::max(1, sms * occ / p.ns);
    *out = h;
    return SLPIC_OK;
}

extern "C" int slpic_fp64_destroy(slpic_fp64_t *h)
{
    if (!h)
        return SLPIC_OK;
    if (h->own_stream)
        cudaStreamSynchronize(h->own_stream);
    for (void *a : h->allocs)
        cudaFree(a);
    if (h->own_stream)
        cudaStreamDestroy(h->own_stream);
    delete h;
    return SLPIC_OK;
}

extern "C" const char *slpic_fp64_last_error(const slpic_fp64_t *h) { return h ? h->err.c_str() : ""; }

extern "C" int slpic_fp64_set_stream(slpic_fp64_t *h, void *stream)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    CK64(h, cudaStreamSynchronize(h->stream));
    h->stream = (cudaStream_t)stream;
    return SLPIC_OK;
}

static int read_state64(slpic_fp64_t *h, St64 &st)
{
    CK64(h, cudaStreamSynchronize(h->stream));
    CK64(h, cudaMemcpy(&st, h->p.st, sizeof(St64), cudaMemcpyDeviceToHost));
    return SLPIC_OK;
}

extern "C" int slpic_fp64_load_particles(slpic_fp64_t *h, int s, int64_t n, const double *x,
                                         const double *v)
{
    if (!h || s < 0 || s >= h->p.ns || n < 0 || (n > 0 && (!x || !v)))
        return h ? fail64(h, SLPIC_ERR_INVALID, "bad arguments") : SLPIC_ERR_INVALID;
    for (int64_t i = 0; i < n; ++i)
        if (!(x[i] >= 0.0 && x[i] < h->p.L) || !std::isfinite(v[3 * i]) ||
            !std::isfinite(v[3 * i + 1]) || !std::isfinite(v[3 * i + 2]))
            return fail64(h, SLPIC_ERR_INVALID, "particle " + std::to_string(i) + " out of range");
    St64 st;
    int rc = read_state64(h, st);
    if (rc)
        return rc;
    const int P = (int)(st.step & 1);
    const long long have = (long long)st.count[s][P];
    if (have + n > h->p.sp[s].capacity)
        return fail64(h, SLPIC_ERR_CAPACITY, "load exceeds the species capacity");
    std::vector<double> vx(n), vy(n), vz(n);
    for (int64_t i = 0; i < n; ++i) {
        vx[i] = v[3 * i];
        vy[i] = v[3 * i + 1];
        vz[i] = v[3 * i + 2];
    }
    const Sp64 &d = h->p.sp[s];
    CK64(h, cudaMemcpy(d.x[P] + have, x, sizeof(double) * n, cudaMemcpyHostToDevice));
    CK64(h, cudaMemcpy(d.vx[P] + have, vx.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CK64(h, cudaMemcpy(d.vy[P] + have, vy.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CK64(h, cudaMemcpy(d.vz[P] + have, vz.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    const unsigned long long cnt = (unsigned long long)(have + n);
    CK64(h, cudaMemcpy(&h->p.st->count[s][P], &cnt, sizeof(cnt), cudaMemcpyHostToDevice));
    return SLPIC_OK;
}

extern "C" int slpic_fp64_prepare(slpic_fp64_t *h)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    P64 &p = h->p;
    CK64(h, cudaMemsetAsync(p.dens, 0, sizeof(double) * p.nn * p.ns, h->stream));
    k_deposit64<<<dim3(h->ctas, p.ns), kThreads, 0, h->stream>>>(p);
    k_field64<<<1, kFieldThreads, 0, h->stream>>>(p);
    CK64(h, cudaGetLastError());
    return slpic_fp64_synchronize(h);
}

extern "C" int slpic_fp64_step(slpic_fp64_t *h, int64_t nsteps)
{
    if (!h || nsteps < 0)
        return h ? fail64(h, SLPIC_ERR_INVALID, "nsteps < 0") : SLPIC_ERR_INVALID;
    P64 &p = h->p;
    const size_t smem = sizeof(double) * (size_t)p.nn;
    for (int64_t k = 0; k < nsteps; ++k) {
        k_step64<<<dim3(h->ctas, p.ns), kThreads, smem, h->stream>>>(p);
        k_inject64<<<1, 1024, 0, h->stream>>>(p);
        k_field64<<<1, kFieldThreads, 0, h->stream>>>(p);
    }
    CK64(h, cudaGetLastError());
    return SLPIC_OK;
}

extern "C" int slpic_fp64_synchronize(slpic_fp64_t *h)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    St64 st;
    int rc = read_state64(h, st);
    if (rc)
        return rc;
    if (st.error)
        return fail64(h, st.error, "particle store full: injection truncated");
    return SLPIC_OK;
}

extern "C" int slpic_fp64_fields(slpic_fp64_t *h, double *rho, double *phi, double *E)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    int rc = slpic_fp64_synchronize(h);
    if (rc)
        return rc;
    const size_t b = sizeof(double) * h->p.nn;
    if (rho)
        CK64(h, cudaMemcpy(rho, h->p.rho, b, cudaMemcpyDeviceToHost));
    if (phi)
        CK64(h, cudaMemcpy(phi, h->p.phi, b, cudaMemcpyDeviceToHost));
    if (E)
        CK64(h, cudaMemcpy(E, h->p.E, b, cudaMemcpyDeviceToHost));
    return SLPIC_OK;
}

extern "C" int slpic_fp64_particle_count(slpic_fp64_t *h, int s, int64_t *n)
{
    if (!h || s < 0 || s >= h->p.ns || !n)
        return h ? fail64(h, SLPIC_ERR_INVALID, "bad arguments") : SLPIC_ERR_INVALID;
    St64 st;
    int rc = read_state64(h, st);
    if (rc)
        return rc;
    *n = (int64_t)st.count[s][st.step & 1];
    return SLPIC_OK;
}

extern "C" int slpic_fp64_get_particles(slpic_fp64_t *h, int s, int64_t cap, double *x, double *v,
                                        int64_t *n)
{
    int64_t cnt = 0;
    int rc = slpic_fp64_particle_count(h, s, &cnt);
    if (rc)
        return rc;
    if (!n || (cnt > 0 && (!x || !v)))
        return fail64(h, SLPIC_ERR_INVALID, "bad arguments");
    if (cap < cnt)
        return fail64(h, SLPIC_ERR_CAPACITY, "output arrays too small");
    St64 st;
    read_state64(h, st);
    const int P = (int)(st.step & 1);
    const Sp64 &d = h->p.sp[s];
    std::vector<double> vx(cnt), vy(cnt), vz(cnt);
    if (cnt) {
        CK64(h, cudaMemcpy(x, d.x[P], sizeof(double) * cnt, cudaMemcpyDeviceToHost));
        CK64(h, cudaMemcpy(vx.data(), d.vx[P], sizeof(double) * cnt, cudaMemcpyDeviceToHost));
        CK64(h, cudaMemcpy(vy.data(), d.vy[P], sizeof(double) * cnt, cudaMemcpyDeviceToHost));
        CK64(h, cudaMemcpy(vz.data(), d.vz[P], sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    }
    for (int64_t i = 0; i < cnt; ++i) {
        v[3 * i] = vx[i];
        v[3 * i + 1] = vy[i];
        v[3 * i + 2] = vz[i];
    }
    *n = cnt;
    return SLPIC_OK;
}
