// unet.cu -- the small convolutional U-Net that warm-starts the 2D CG
// (include/slpic_unet.h): forward, backward and Adam, hand-written.
//
// The paper has no learned part; the network is the plain U-Net pattern at the
// size the 2D solve needs.  Level l = 0..L-1 has C_l = C 2^l channels:
//   encoder  e_0 = relu(conv(x)),  e_l = relu(conv(pool(e_{l-1})))
//   decoder  d_{L-1} = e_{L-1},    d_l = relu(conv(concat(up(d_{l+1}), e_l)))
//   output   y = conv(d_0)
// conv: 3x3, zero padding, bias; pool: 2x2 mean; up: nearest x2; concat: the
// upsampled channels first.  Activations and gradients are FP32 (N, C, H, W);
// the convolutions use BF16 copies of the FP32 master weights (biases stay FP32)
// and accumulate in FP32; weight-gradient sums are FP64 across threads.  The loss
// is the mean squared error; training is Adam.
//
// Tensors are addressed through views (base, channels of the underlying buffer,
// channel offset), so e_l is written straight into the second half of level l's
// concat buffer and its gradient is read from the second half of the concat
// gradient: the concatenation costs no copy.  The ReLU mask is taken from the
// stored activation (a > 0 exactly when z > 0).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "slpic_unet.h"
#include "unet_internal.h"

namespace {

constexpr int kT = 256;   // threads per CTA
constexpr int kOCB = 8;   // output channels per thread in the convolutions

struct TV {               // (n, c, pix) at p[(n*ctot + coff + c)*HW + pix]
    float *p;
    int ctot, coff;
};

__device__ __forceinline__ float *at(TV v, int n, int c, size_t HW)
{
    return v.p + ((size_t)n * v.ctot + v.coff + c) * HW;
}

// ---- convolution forward: a = conv(x) (relu'd when relu != 0) -------------------
// One thread per output pixel and kOCB output channels; blockIdx = (pixel tile,
// channel group, sample).
__global__ void __launch_bounds__(kT) k_conv_fwd(TV x, int cin, const __nv_bfloat16 *__restrict__ w,
                                               const float *__restrict__ b, int cout, TV a,
                                               int relu, int H, int W)
{
    const int pix = blockIdx.x * kT + threadIdx.x;
    if (pix >= H * W)
        return;
    const int i = pix / W, j = pix - i * W;
    const int n = blockIdx.z, o0 = blockIdx.y * kOCB;
    const size_t HW = (size_t)H * W;
    float acc[kOCB];
#pragma unroll
    for (int k = 0; k < kOCB; ++k)
        acc[k] = (o0 + k < cout) ? b[o0 + k] : 0.0f;
    for (int c = 0; c < cin; ++c) {
        const float *xc = at(x, n, c, HW);
        float v[9];
#pragma unroll
        for (int di = 0; di < 3; ++di) {
            const int ii = i + di - 1;
#pragma unroll
            for (int dj = 0; dj < 3; ++dj) {
                const int jj = j + dj - 1;
                v[di * 3 + dj] = (ii >= 0 && ii < H && jj >= 0 && jj < W) ? xc[ii * W + jj] : 0.0f;
            }
        }
#pragma unroll
        for (int k = 0; k < kOCB; ++k) {
            if (o0 + k < cout) {
                const __nv_bfloat16 *wk = w + ((size_t)(o0 + k) * cin + c) * 9;
#pragma unroll
                for (int t = 0; t < 9; ++t)
                    acc[k] = __fmaf_rn(__bfloat162float(wk[t]), v[t], acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kOCB; ++k) {
        if (o0 + k >= cout)
            break;
        at(a, n, o0 + k, HW)[pix] = relu ? fmaxf(acc[k], 0.0f) : acc[k];
    }
}

// ---- convolution forward on the tensor cores (tcgen05) -----------------------------
// Implicit GEMM: D[m][o] = sum_k A[m][k] B[o][k] with m the tile's 128 pixels, o
// the output channels (N = cout padded to a multiple of 16), k = c*9 + di*3 + dj
// (K = cin*9 padded to a multiple of 64).  A is the im2col gather of the FP32
// activations, rounded to BF16 by the threads that build it; B is the BF16 weight
// copy, packed once per parameter change (k_pack_tc) into the exact shared-memory
// image of each 64-wide K chunk.  Both operands are K-major without swizzle: core
// matrices of 8 rows x 16 B, 128 B each, core (row group g, K group j) at g*1024 +
// j*128 within a chunk.  The accumulator lives in TMEM (128 lanes = pixels, N
// columns, FP32); one thread issues the MMAs (4 per chunk, K = 16 each) and
// commits them to the chunk buffer's mbarrier, so the threads build chunk k+1
// while the tensor cores work on chunk k.  The epilogue reads TMEM (tcgen05.ld,
// warp w owns lanes 32w..32w+31), adds the bias, applies the ReLU and stores.
constexpr int kTcM = 128;                 // pixels per CTA tile
constexpr int kTcThreads = 256;           // two threads per pixel build the A chunk
constexpr int kTcKC = 64;                 // K per chunk
constexpr int kTcChunkA = kTcM * kTcKC * 2;  // bytes of one A chunk (16 KB)

__device__ __forceinline__ uint32_t tc_smem(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, leading (K) and stride (row group) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major
__device__ __forceinline__ uint32_t tc_idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ bool tc_wait(uint64_t *bar, unsigned parity, int *flag)
{
    const long long t0 = clock64();
    for (;;) {
        unsigned ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
            "selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(tc_smem(bar)), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if (clock64() - t0 > 2000000000LL) {  // ~1 s: record and give up
            atomicExch(flag, 1);
            return false;
        }
    }
}

// The GEMM's K runs over (tap t, channel c) with the channel fastest and each
// tap's channels padded to cp = cin rounded up to 16: k = t cp + c.  Every 8-k core
// row then lies within one tap.
// packed[conv chunk kc][o/8][j][o%8][kk] = w[o][c][t] for k = 64 kc + 8 j + kk
// (0 for padding)
__global__ void k_pack_tc(const __nv_bfloat16 *__restrict__ w, int cout, int cin, int Np, int nkc,
                          __nv_bfloat16 *__restrict__ packed)
{
    const int cp = (cin + 15) / 16 * 16;
    const size_t total = (size_t)nkc * Np * kTcKC;
    for (size_t e = blockIdx.x * (size_t)kT + threadIdx.x; e < total; e += (size_t)gridDim.x * kT) {
        const int kc = (int)(e / ((size_t)Np * kTcKC));
        const int r = (int)(e - (size_t)kc * Np * kTcKC);
        const int g = r / (8 * kTcKC);  // row group (8 rows x 64 k)
        const int rem = r - g * 8 * kTcKC;
        const int j = rem / 64, rr = (rem / 8) % 8, kk = rem % 8;
        const int o = g * 8 + rr, k = kc * kTcKC + j * 8 + kk;
        const int t = k / cp, c = k - t * cp;
        packed[e] = (o < cout && t < 9 && c < cin) ? w[((size_t)o * cin + c) * 9 + t]
                                                   : __float2bfloat16_rn(0.0f);
    }
}

// The transposed conv of the input gradient, dx = conv^T(dz), is the same conv of dz
// with the weights' channels swapped and taps mirrored: W'[c][o][t] = W[o][c][8 - t].
// packed[kc][c/8][j][c%8][kk] = W[o][c][8 - t] for k = t cpo + o (cpo = cout padded to 16)
__global__ void k_pack_tc_t(const __nv_bfloat16 *__restrict__ w, int cout, int cin, int Np, int nkc,
                            __nv_bfloat16 *__restrict__ packed)
{
    const int cp = (cout + 15) / 16 * 16;
    const size_t total = (size_t)nkc * Np * kTcKC;
    for (size_t e = blockIdx.x * (size_t)kT + threadIdx.x; e < total; e += (size_t)gridDim.x * kT) {
        const int kc = (int)(e / ((size_t)Np * kTcKC));
        const int r = (int)(e - (size_t)kc * Np * kTcKC);
        const int g = r / (8 * kTcKC);
        const int rem = r - g * 8 * kTcKC;
        const int j = rem / 64, rr = (rem / 8) % 8, kk = rem % 8;
        const int c = g * 8 + rr, k = kc * kTcKC + j * 8 + kk;
        const int t = k / cp, o = k - t * cp;
        packed[e] = (c < cin && t < 9 && o < cout) ? w[((size_t)o * cin + c) * 9 + (8 - t)]
                                                   : __float2bfloat16_rn(0.0f);
    }
}

// wp: the packed B of this launch's output channels (a slice of at most 256 rows of a
// packed image whose chunks lie bstride elements apart); b: their biases
__global__ void __launch_bounds__(kTcThreads) k_conv_fwd_tc(TV x, int cin, const __nv_bfloat16 *__restrict__ wp,
                                                    size_t bstride, const float *__restrict__ b, int cout,
                                                    int Np, TV a, int relu, int H, int W, int *flag)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int chunkB = Np * kTcKC * 2;

    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m = tid & (kTcM - 1), half = tid >> 7;  // pixel row; which 4 K groups
    const int n = blockIdx.y;
    const size_t HW = (size_t)H * W;
    const int pix = blockIdx.x * kTcM + m;
    const bool in = pix < (int)HW;
    const int i = in ? pix / W : 0, j = in ? pix - (pix / W) * W : 0;
    const int cp = (cin + 15) / 16 * 16, nkc = (9 * cp + kTcKC - 1) / kTcKC;
    const uint32_t ncols = Np <= 32 ? 32u : Np <= 64 ? 64u : Np <= 128 ? 128u : 256u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem(&s_tmem)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&s_bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&s_bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    // this thread's A row: (row group, row in group) of pixel m
    const int arow = (m >> 3) * 1024 + (m & 7) * 16;
    const float *xn = at(x, n, 0, HW) + (in ? pix : 0);
    // the pixel's 9 taps: offset from the pixel, and whether it lies in the image
    unsigned tapok = 0u;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
        const int ii = i + t / 3 - 1, jj = j + t % 3 - 1;
        if (in && ii >= 0 && ii < H && jj >= 0 && jj < W)
            tapok |= 1u << t;
    }
    for (int kc = 0; kc < nkc; ++kc) {
        const int buf = kc & 1;
        unsigned char *bufA = tsm + buf * kTcChunkA;
        unsigned char *bufB = tsm + 2 * kTcChunkA + buf * chunkB;
        if (kc >= 2 && !s_fail) {
            // the MMAs of chunk kc-2 have read this buffer
            if (!tc_wait(&s_bar[buf], (unsigned)(((kc - 2) >> 1) & 1), flag))
                s_fail = 1;
        }
        __syncthreads();
        if (s_fail)
            break;
        // A: this thread's 4 groups of 8 consecutive k for its pixel (32 loads in
        // flight), one 16-byte store per group
        {
            float v[kTcKC / 2];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                const int k0 = kc * kTcKC + (half * 4 + g) * 8;  // 8 k, one tap
                const int t = k0 / cp, c0 = k0 - t * cp;
                const bool ok = t < 9 && ((tapok >> t) & 1u);
                const float *src = xn + ((t / 3 - 1) * W + (t % 3 - 1)) + (size_t)c0 * HW;
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    v[8 * g + e] = (ok && c0 + e < cin) ? __ldg(src + (size_t)e * HW) : 0.0f;
            }
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                uint32_t w4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * g + 2 * q], v[8 * g + 2 * q + 1]);
                    w4[q] = *reinterpret_cast<const uint32_t *>(&h2);
                }
                *reinterpret_cast<uint4 *>(bufA + arow + (half * 4 + g) * 128) =
                    make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
        }
        // B: the packed chunk image, 16 bytes per thread and step
        const uint4 *src = reinterpret_cast<const uint4 *>(wp + (size_t)kc * bstride);
        uint4 *dst = reinterpret_cast<uint4 *>(bufB);
        for (int e = tid; e < chunkB / 16; e += kTcThreads)
            dst[e] = __ldg(src + e);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = tc_idesc(Np);
#pragma unroll
            for (int kk = 0; kk < kTcKC / 16; ++kk) {
                const uint64_t da = tc_desc(tc_smem(bufA) + kk * 256);
                const uint64_t db = tc_desc(tc_smem(bufB) + kk * 256);
                const uint32_t accum = (kc > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    tc_smem(&s_bar[buf]))
                : "memory");
        }
    }
    // all MMAs done (a commit tracks every earlier MMA of its thread)
    bool ok = !s_fail;
    if (ok)
        ok = tc_wait(&s_bar[(nkc - 1) & 1], (unsigned)(((nkc - 1) >> 1) & 1), flag);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();
    if (__all_sync(0xffffffffu, ok)) {
        // warp w reads TMEM lanes 32 (w mod 4) .. +31; the two warpgroups split the columns
        const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        for (int o0 = half * (Np / 2); o0 < (half + 1) * (Np / 2); o0 += 8) {
            uint32_t v[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7])
                : "r"(lane_base + (uint32_t)o0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (in) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int o = o0 + q;
                    if (o < cout) {
                        const float z = __uint_as_float(v[q]) + b[o];
                        at(a, n, o, HW)[pix] = relu ? fmaxf(z, 0.0f) : z;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---- weight gradient on the tensor cores ---------------------------------------------
// dW[o][c][t] = sum over samples and pixels of dz[o][p] x[c][p + off_t]: a GEMM with
// M = (tap t, channel c) rows r = t cp + c (cp = cin padded to 16), N = output
// channels (padded to 16), K = the nb * HW pixels, split over CTAs (blockIdx.y) and
// added afterwards in a fixed order (k_wgrad_reduce).  A[r][k] = x of the pixel k
// shifted by tap t (zero off the image), B[o][k] = dz[o] at pixel k, both rounded to
// BF16, built by the threads in the K-major core-matrix layout of the forward conv
// (thread: a pair of adjacent pixels, a stripe of rows).  Partial sums FP32 in TMEM.
__global__ void __launch_bounds__(kTcThreads) k_conv_wgrad_tc(TV x, int cin, TV dz, int cout, int Np,
                                                            int H, int W, int nb, int chunks_per,
                                                            float *__restrict__ part, int *flag)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    const int chunkB = Np * kTcKC * 2;
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int HW = H * W;
    const long long npix = (long long)nb * HW;
    const int cp = (cin + 15) / 16 * 16, nrows = 9 * cp;
    const int r0 = blockIdx.x * kTcM;  // this CTA's first row
    const long long c0 = (long long)blockIdx.y * chunks_per;
    const long long nchunk = (npix + kTcKC - 1) / kTcKC;
    const int nkc = (int)max(0LL, min((long long)chunks_per, nchunk - c0));
    const uint32_t ncols = Np <= 32 ? 32u : Np <= 64 ? 64u : Np <= 128 ? 128u : 256u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem(&s_tmem)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&s_bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&s_bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int kp = tid & 31;         // pixel pair of the chunk: k = 2 kp, 2 kp + 1
    const int stripe = tid >> 5;     // rows stripe, 8 and 8 rows apart
    for (int kc = 0; kc < nkc; ++kc) {
        const int buf = kc & 1;
        unsigned char *bufA = tsm + buf * kTcChunkA;
        unsigned char *bufB = tsm + 2 * kTcChunkA + buf * chunkB;
        if (kc >= 2 && !s_fail) {
            if (!tc_wait(&s_bar[buf], (unsigned)(((kc - 2) >> 1) & 1), flag))
                s_fail = 1;
        }
        __syncthreads();
        if (s_fail)
            break;
        // this thread's two pixels
        const long long P0 = (c0 + kc) * kTcKC + 2 * kp;
        int pn[2], pp[2], pi[2], pj[2];
        unsigned tap_ok[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long long P = P0 + u;
            tap_ok[u] = 0u;
            pn[u] = 0;
            pp[u] = 0;
            pi[u] = 0;
            pj[u] = 0;
            if (P < npix) {
                pn[u] = (int)(P / HW);
                pp[u] = (int)(P - (long long)pn[u] * HW);
                pi[u] = pp[u] / W;
                pj[u] = pp[u] - pi[u] * W;
#pragma unroll
                for (int t = 0; t < 9; ++t) {
                    const int ii = pi[u] + t / 3 - 1, jj = pj[u] + t % 3 - 1;
                    if (ii >= 0 && ii < H && jj >= 0 && jj < W)
                        tap_ok[u] |= 1u << t;
                }
            }
        }
        // A: rows r0 + stripe + 8 q, q = 0..15
        const int koff = (kp >> 2) * 128 + (kp & 3) * 4;  // byte offset of k = 2 kp in a row
#pragma unroll 4
        for (int q = 0; q < 16; ++q) {
            const int rl = stripe + 8 * q;  // row within the tile
            const int r = r0 + rl;
            float v2[2] = {0.0f, 0.0f};
            if (r < nrows) {
                const int t = r / cp, c = r - t * cp;
                if (c < cin) {
                    const int off = (t / 3 - 1) * W + (t % 3 - 1);
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        if ((tap_ok[u] >> t) & 1u)
                            v2[u] = __ldg(at(x, pn[u], c, HW) + pp[u] + off);
                }
            }
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v2[0], v2[1]);
            *reinterpret_cast<__nv_bfloat162 *>(bufA + (rl >> 3) * 1024 + (rl & 7) * 16 + koff) = h2;
        }
        // B: rows o = stripe + 8 q
        for (int o = stripe; o < Np; o += 8) {
            float v2[2] = {0.0f, 0.0f};
            if (o < cout) {
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (P0 + u < npix)
                        v2[u] = __ldg(at(dz, pn[u], o, HW) + pp[u]);
            }
            const __nv_bfloat162 h2 = __floats2bfloat162_rn(v2[0], v2[1]);
            *reinterpret_cast<__nv_bfloat162 *>(bufB + (o >> 3) * 1024 + (o & 7) * 16 + koff) = h2;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t idesc = tc_idesc(Np);
#pragma unroll
            for (int kk = 0; kk < kTcKC / 16; ++kk) {
                const uint64_t da = tc_desc(tc_smem(bufA) + kk * 256);
                const uint64_t db = tc_desc(tc_smem(bufB) + kk * 256);
                const uint32_t accum = (kc > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{ .reg .pred p; setp.ne.b32 p, %4, 0; "
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(accum));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    tc_smem(&s_bar[buf]))
                : "memory");
        }
    }
    bool ok = !s_fail && nkc > 0;
    if (ok)
        ok = tc_wait(&s_bar[(nkc - 1) & 1], (unsigned)(((nkc - 1) >> 1) & 1), flag);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncwarp();
    // partial sums of this K range: part[blockIdx.y][r][o] (zero when nothing was summed)
    const int half = tid >> 7, rl = (warp & 3) * 32 + (tid & 31);
    const int r = r0 + rl;
    float *dst = part + ((size_t)blockIdx.y * gridDim.x * kTcM + r) * Np;
    const bool all_ok = __all_sync(0xffffffffu, ok);
    const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    for (int o0 = half * (Np / 2); o0 < (half + 1) * (Np / 2); o0 += 8) {
        uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (all_ok) {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7])
                : "r"(lane_base + (uint32_t)o0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            dst[o0 + q] = __uint_as_float(v[q]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// dW[o][c][t] = sum over the K splits, in split order, of part[s][t cp + c][o]
__global__ void k_wgrad_reduce(const float *__restrict__ part, int splits, int mrows, int Np, int cin,
                               int cout, float *__restrict__ dw)
{
    const int cp = (cin + 15) / 16 * 16;
    const size_t total = (size_t)cout * cin * 9;
    for (size_t e = blockIdx.x * (size_t)kT + threadIdx.x; e < total; e += (size_t)gridDim.x * kT) {
        const int o = (int)(e / ((size_t)cin * 9));
        const int rem = (int)(e - (size_t)o * cin * 9);
        const int c = rem / 9, t = rem - c * 9;
        const int r = t * cp + c;
        double acc = 0.0;
        for (int sp = 0; sp < splits; ++sp)
            acc += (double)part[((size_t)sp * mrows + r) * Np + o];
        dw[e] = (float)acc;
    }
}

// db[o] = sum of dz[o] over samples and pixels (FP64, one CTA per output channel)
__global__ void __launch_bounds__(kT) k_bias_grad(TV dz, int cout, int HW, int nb, float *__restrict__ db)
{
    __shared__ double s_red[kT / 32];
    const int o = blockIdx.x;
    double acc = 0.0;
    for (int n = 0; n < nb; ++n) {
        const float *g = at(dz, n, o, HW);
        for (int p = threadIdx.x; p < HW; p += kT)
            acc += g[p];
    }
    for (int off = 16; off; off >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < kT / 32; ++k)
            v += s_red[k];
        db[o] = (float)v;
    }
}

// ---- gradient of the convolution's input: dx = conv^T(dz) ------------------------
// dx[c,i,j] = sum_{o,di,dj} w[o,c,di,dj] dz[o, i-di+1, j-dj+1]
__global__ void __launch_bounds__(kT) k_conv_bwd_x(TV dz, int cout, const __nv_bfloat16 *__restrict__ w,
                                                 int cin, TV dx, int H, int W)
{
    const int pix = blockIdx.x * kT + threadIdx.x;
    if (pix >= H * W)
        return;
    const int i = pix / W, j = pix - i * W;
    const int n = blockIdx.z, c0 = blockIdx.y * kOCB;
    const size_t HW = (size_t)H * W;
    float acc[kOCB];
#pragma unroll
    for (int k = 0; k < kOCB; ++k)
        acc[k] = 0.0f;
    for (int o = 0; o < cout; ++o) {
        const float *dc = at(dz, n, o, HW);
        float g[9];
#pragma unroll
        for (int di = 0; di < 3; ++di) {
            const int ii = i - di + 1;
#pragma unroll
            for (int dj = 0; dj < 3; ++dj) {
                const int jj = j - dj + 1;
                g[di * 3 + dj] = (ii >= 0 && ii < H && jj >= 0 && jj < W) ? dc[ii * W + jj] : 0.0f;
            }
        }
#pragma unroll
        for (int k = 0; k < kOCB; ++k) {
            if (c0 + k < cin) {
                const __nv_bfloat16 *wk = w + ((size_t)o * cin + c0 + k) * 9;
#pragma unroll
                for (int t = 0; t < 9; ++t)
                    acc[k] = __fmaf_rn(__bfloat162float(wk[t]), g[t], acc[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kOCB; ++k) {
        if (c0 + k >= cin)
            break;
        at(dx, n, c0 + k, HW)[pix] = acc[k];
    }
}

// ---- gradient of the weights and bias: one CTA per (c, o) ----------------------
// dw[o,c,di,dj] = sum_{n,i,j} dz[n,o,i,j] x[n,c,i+di-1,j+dj-1];  db[o] = sum dz[n,o]
// (written by the c = 0 CTA).  FP32 per thread, FP64 across threads.
__global__ void __launch_bounds__(kT) k_conv_bwd_w(TV x, int cin, TV dz, int cout,
                                                 float *__restrict__ dw, float *__restrict__ db,
                                                 int H, int W, int nb, int xbf16)
{
    __shared__ double s_red[kT / 32][10];
    const int c = blockIdx.x, o = blockIdx.y;
    const size_t HW = (size_t)H * W;
    float acc[10];
#pragma unroll
    for (int t = 0; t < 10; ++t)
        acc[t] = 0.0f;
    for (int n = 0; n < nb; ++n) {
        const float *xc = at(x, n, c, HW);
        const float *gc = at(dz, n, o, HW);
        for (int pix = threadIdx.x; pix < H * W; pix += kT) {
            const int i = pix / W, j = pix - i * W;
            const float g = gc[pix];
#pragma unroll
            for (int di = 0; di < 3; ++di) {
                const int ii = i + di - 1;
#pragma unroll
                for (int dj = 0; dj < 3; ++dj) {
                    const int jj = j + dj - 1;
                    float v = (ii >= 0 && ii < H && jj >= 0 && jj < W) ? xc[ii * W + jj] : 0.0f;
                    if (xbf16)  // the forward pass multiplied the BF16-rounded input
                        v = __bfloat162float(__float2bfloat16_rn(v));
                    acc[di * 3 + dj] = __fmaf_rn(g, v, acc[di * 3 + dj]);
                }
            }
            acc[9] += g;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < 10; ++t) {
        double v = acc[t];
        for (int off = 16; off; off >>= 1)
            v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0)
            s_red[warp][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double v = 0.0;
        for (int k = 0; k < kT / 32; ++k)
            v += s_red[k][threadIdx.x];
        if (threadIdx.x < 9)
            dw[((size_t)o * cin + c) * 9 + threadIdx.x] = (float)v;
        else if (c == 0)
            db[o] = (float)v;
    }
}

// ---- elementwise layers: blockIdx.y walks the planes (n, c), x the pixels ----------
// plane q = n*C + c of a view
__device__ __forceinline__ float *plane(TV v, int q, int C, size_t HW)
{
    const int n = q / C, c = q - n * C;
    return at(v, n, c, HW);
}

// g = a > 0 ? g : 0, in place (the ReLU's backward pass, mask from its output)
__global__ void k_relu_bwd(TV a, TV g, int C, int HW, int nplanes)
{
    for (int q = blockIdx.y; q < nplanes; q += gridDim.y) {
        const float *ap = plane(a, q, C, HW);
        float *gp = plane(g, q, C, HW);
        for (int p = blockIdx.x * kT + threadIdx.x; p < HW; p += gridDim.x * kT)
            if (!(ap[p] > 0.0f))
                gp[p] = 0.0f;
    }
}

// out (H/2, W/2) = 2x2 mean of in (H, W)
__global__ void k_pool_fwd(TV in, TV out, int C, int H, int W, int nplanes)
{
    const int h = H / 2, w = W / 2;
    for (int q = blockIdx.y; q < nplanes; q += gridDim.y) {
        const float *ip = plane(in, q, C, (size_t)H * W);
        float *op = plane(out, q, C, (size_t)h * w);
        for (int p = blockIdx.x * kT + threadIdx.x; p < h * w; p += gridDim.x * kT) {
            const int i = p / w, j = p - i * w;
            const float *s = ip + (size_t)(2 * i) * W + 2 * j;
            op[p] = 0.25f * ((s[0] + s[1]) + (s[W] + s[W + 1]));
        }
    }
}

// din (H, W) += pool^T(dout): a quarter of the coarse gradient to each of the four
__global__ void k_pool_bwd_add(TV dout, TV din, int C, int H, int W, int nplanes)
{
    const int w = W / 2;
    for (int q = blockIdx.y; q < nplanes; q += gridDim.y) {
        const float *op = plane(dout, q, C, (size_t)(H / 2) * w);
        float *ip = plane(din, q, C, (size_t)H * W);
        for (int p = blockIdx.x * kT + threadIdx.x; p < H * W; p += gridDim.x * kT) {
            const int i = p / W, j = p - i * W;
            ip[p] += 0.25f * op[(size_t)(i / 2) * w + j / 2];
        }
    }
}

// out (2H, 2W) = nearest-neighbour upsampling of in (H, W)
__global__ void k_up_fwd(TV in, TV out, int C, int H, int W, int nplanes)
{
    const int W2 = 2 * W;
    for (int q = blockIdx.y; q < nplanes; q += gridDim.y) {
        const float *ip = plane(in, q, C, (size_t)H * W);
        float *op = plane(out, q, C, (size_t)4 * H * W);
        for (int p = blockIdx.x * kT + threadIdx.x; p < 4 * H * W; p += gridDim.x * kT) {
            const int i = p / W2, j = p - i * W2;
            op[p] = ip[(size_t)(i / 2) * W + j / 2];
        }
    }
}

// din (H, W) = up^T(dout): the sum of the four fine gradients
__global__ void k_up_bwd(TV dout, TV din, int C, int H, int W, int nplanes)
{
    const int W2 = 2 * W;
    for (int q = blockIdx.y; q < nplanes; q += gridDim.y) {
        const float *op = plane(dout, q, C, (size_t)4 * H * W);
        float *ip = plane(din, q, C, (size_t)H * W);
        for (int p = blockIdx.x * kT + threadIdx.x; p < H * W; p += gridDim.x * kT) {
            const int i = p / W, j = p - i * W;
            const float *s = op + (size_t)(2 * i) * W2 + 2 * j;
            ip[p] = (s[0] + s[1]) + (s[W2] + s[W2 + 1]);
        }
    }
}

// ---- input normalisation: s_n = rms(x_n) (1 for an all-zero sample), xs = x / s_n
// One CTA per sample; FP64 sum.  With normalise == 0, s_n = 1.
__global__ void __launch_bounds__(kT) k_norm_in(const float *__restrict__ x, float *__restrict__ xs,
                                              float *__restrict__ s, size_t HW, int normalise)
{
    __shared__ double s_red[kT / 32];
    __shared__ float s_scale;
    const int n = blockIdx.x;
    const float *xn = x + (size_t)n * HW;
    double acc = 0.0;
    if (normalise)
        for (size_t q = threadIdx.x; q < HW; q += kT)
            acc += (double)xn[q] * xn[q];
    for (int off = 16; off; off >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < kT / 32; ++k)
            v += s_red[k];
        float sc = normalise ? (float)sqrt(v / (double)HW) : 1.0f;
        if (!(sc > 0.0f))
            sc = 1.0f;
        s_scale = sc;
        s[n] = sc;
    }
    __syncthreads();
    const float inv = 1.0f / s_scale;
    for (size_t q = threadIdx.x; q < HW; q += kT)
        xs[(size_t)n * HW + q] = xn[q] * inv;
}

// y = y_net * s_n * out_scale
__global__ void k_scale_out(const float *__restrict__ ynet, float *__restrict__ y,
                            const float *__restrict__ s, float out_scale, size_t HW, int nb)
{
    for (size_t t = blockIdx.x * (size_t)kT + threadIdx.x; t < (size_t)nb * HW;
         t += (size_t)gridDim.x * kT)
        y[t] = ynet[t] * (s[t / HW] * out_scale);
}

// mean squared error against the target in network units, t / (s_n out_scale):
// dy = 2 r / count; per-CTA FP64 partial sums of r^2
__global__ void __launch_bounds__(kT) k_mse(const float *__restrict__ ynet,
                                          const float *__restrict__ t, const float *__restrict__ s,
                                          float out_scale, float *__restrict__ dy, size_t HW,
                                          int nb, double *__restrict__ part)
{
    __shared__ double s_red[kT / 32];
    const size_t count = (size_t)nb * HW;
    double acc = 0.0;
    for (size_t q = blockIdx.x * (size_t)kT + threadIdx.x; q < count; q += (size_t)gridDim.x * kT) {
        const float r = ynet[q] - t[q] / (s[q / HW] * out_scale);
        dy[q] = 2.0f * r / (float)count;
        acc += (double)r * r;
    }
    for (int off = 16; off; off >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < kT / 32; ++k)
            v += s_red[k];
        part[blockIdx.x] = v;
    }
}

// energy-norm loss, pass 1: e = y_net - t / (s_n out_scale), zero on row 0
__global__ void k_energy_err(const float *__restrict__ ynet, const float *__restrict__ t,
                             const float *__restrict__ s, float out_scale, float *__restrict__ e,
                             int H, int W, int nb)
{
    const size_t HW = (size_t)H * W;
    for (size_t q = blockIdx.x * (size_t)kT + threadIdx.x; q < (size_t)nb * HW;
         q += (size_t)gridDim.x * kT) {
        const size_t pix = q % HW;
        e[q] = pix < (size_t)W ? 0.0f : ynet[q] - t[q] / (s[q / HW] * out_scale);
    }
}

// pass 2: dy = 2 A e / count (zero on row 0), per-CTA FP64 partial sums of e . A e;
// A e = 4 e - e(x+-1) (periodic) - e(y+-1) (zero outside rows 0..H-1)
__global__ void __launch_bounds__(kT) k_energy_grad(const float *__restrict__ e,
                                                  float *__restrict__ dy, int H, int W, int nb,
                                                  double *__restrict__ part)
{
    __shared__ double s_red[kT / 32];
    const size_t HW = (size_t)H * W, count = (size_t)nb * HW;
    double acc = 0.0;
    for (size_t q = blockIdx.x * (size_t)kT + threadIdx.x; q < count; q += (size_t)gridDim.x * kT) {
        const size_t pix = q % HW;
        const int i = (int)(pix / W), j = (int)(pix - (size_t)i * W);
        float g = 0.0f;
        if (i > 0) {
            const float *en = e + (q - pix);
            const float c = en[pix];
            const float xl = en[(size_t)i * W + (j == 0 ? W - 1 : j - 1)];
            const float xr = en[(size_t)i * W + (j == W - 1 ? 0 : j + 1)];
            const float yd = en[pix - W];
            const float yu = i + 1 < H ? en[pix + W] : 0.0f;
            const float ae = 4.0f * c - ((xl + xr) + (yd + yu));
            g = 2.0f * ae / (float)count;
            acc += (double)c * ae;
        }
        dy[q] = g;
    }
    for (int off = 16; off; off >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < kT / 32; ++k)
            v += s_red[k];
        part[blockIdx.x] = v;
    }
}

// loss = sum(part[0..np)) / count, in CTA order (one CTA)
__global__ void k_loss(const double *__restrict__ part, int np, double count, double *loss)
{
    __shared__ double s_red[kT / 32];
    double acc = 0.0;
    for (int q = threadIdx.x; q < np; q += kT)
        acc += part[q];
    for (int off = 16; off; off >>= 1)
        acc += __shfl_down_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0)
        s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int k = 0; k < kT / 32; ++k)
            v += s_red[k];
        *loss = v / count;
    }
}

// Adam (Kingma & Ba, 2015) on the FP32 master parameters; the BF16 copy follows.
// c1 = 1 - b1^t and c2 = 1 - b2^t are the bias corrections of step t.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __nv_bfloat16 *__restrict__ pb, size_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2)
{
    for (size_t t = blockIdx.x * (size_t)kT + threadIdx.x; t < n; t += (size_t)gridDim.x * kT) {
        const float gt = g[t];
        const float mt = b1 * m[t] + (1.0f - b1) * gt;
        const float vt = b2 * v[t] + (1.0f - b2) * gt * gt;
        m[t] = mt;
        v[t] = vt;
        const float w = p[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
        p[t] = w;
        pb[t] = __float2bfloat16_rn(w);
    }
}

__global__ void k_to_bf16(const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb, size_t n)
{
    for (size_t t = blockIdx.x * (size_t)kT + threadIdx.x; t < n; t += (size_t)gridDim.x * kT)
        pb[t] = __float2bfloat16_rn(p[t]);
}

}  // namespace

// =====================================================================================
// Host side: buffers, the layer schedule, the C ABI.
// =====================================================================================
struct ConvSpec {
    int cin, cout, level;   // level: the grid the conv runs on
    size_t w_off, b_off;    // into the flat parameter array
    int Np = 0, nkc = 0;    // tensor-core form: padded N, K chunks
    size_t tc_off = 0;      // its packed weights in wtc
    int Npt = 0, nkct = 0;  // the transposed conv (input gradient): padded N, K chunks
    size_t tct_off = 0;     // its packed weights in wtct
};

struct slpic_unet {
    slpic_unet_config cfg{};
    int L = 0, C = 0, H = 0, W = 0, nbmax = 0;
    std::vector<ConvSpec> conv;   // 2L convs in parameter order
    size_t nparam = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *pb = nullptr;
    // forward activations (per level; see the schedule below)
    float *xin = nullptr, *s = nullptr, *ynet = nullptr;
    std::vector<float *> cat, d, pin;  // cat, d: levels 0..L-2; pin: levels 1..L-1
    float *etop = nullptr;             // e_{L-1}
    // gradients (allocated on first use)
    bool have_grads = false;
    float *dy = nullptr, *eb = nullptr;  // eb: the error image of the energy loss
    std::vector<float *> dcat, gd, dpool;  // dcat: 0..L-2; gd: 0..L-1; dpool: 1..L-1
    double *part = nullptr, *loss = nullptr;
    long long adam_t = 0;
    // tensor-core forward (cfg.tensor_cores): packed BF16 weights, stale after a
    // parameter change until the next forward repacks them
    __nv_bfloat16 *wtc = nullptr, *wtct = nullptr;
    float *zeros = nullptr;  // zero biases of the transposed convs
    float *wpart = nullptr;  // K-split partial weight gradients
    size_t wpart_n = 0;
    bool tc_dirty = true;
    int *d_flag = nullptr;  // a bounded wait of a tensor-core kernel ran out
    cudaStream_t stream = nullptr;
    std::vector<void *> allocs;
    std::string err;
};

namespace {

constexpr int kMseCtas = 608;  // 4 per SM

#define CKU(h, call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return e_ == cudaErrorMemoryAllocation ? SLPIC_ERR_OOM : SLPIC_ERR_CUDA;       \
        }                                                                                  \
    } while (0)

int failu(slpic_unet_t *h, int code, const std::string &msg)
{
    h->err = msg;
    return code;
}

// after a synchronisation: a bounded wait of a tensor-core kernel that ran out
int check_flag(slpic_unet_t *h)
{
    if (!h->d_flag)
        return SLPIC_OK;
    int f = 0;
    CKU(h, cudaMemcpy(&f, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost));
    return f ? failu(h, SLPIC_ERR_TIMEOUT, "a tensor-core convolution timed out") : SLPIC_OK;
}

int ch(const slpic_unet_t *h, int l) { return h->C << l; }
int hl(const slpic_unet_t *h, int l) { return h->H >> l; }
int wl(const slpic_unet_t *h, int l) { return h->W >> l; }
size_t hwl(const slpic_unet_t *h, int l) { return (size_t)hl(h, l) * wl(h, l); }

int alloc(slpic_unet_t *h, void **ptr, size_t bytes)
{
    CKU(h, cudaMalloc(ptr, bytes));
    h->allocs.push_back(*ptr);
    return SLPIC_OK;
}

int alloc_f(slpic_unet_t *h, float **ptr, size_t count)
{
    return alloc(h, (void **)ptr, sizeof(float) * count);
}

// views: e_l (inside cat[l] for l <= L-2), d_l, the conv input of level l
TV view_e(slpic_unet_t *h, int l)
{
    if (l == h->L - 1)
        return TV{h->etop, ch(h, l), 0};
    return TV{h->cat[l], ch(h, l + 1) + ch(h, l), ch(h, l + 1)};
}
TV view_d(slpic_unet_t *h, int l) { return l == h->L - 1 ? view_e(h, l) : TV{h->d[l], ch(h, l), 0}; }
TV view_enc_in(slpic_unet_t *h, int l)
{
    return l == 0 ? TV{h->xin, 1, 0} : TV{h->pin[l], ch(h, l - 1), 0};
}
// gradient at e_l: inside dcat[l] for l <= L-2, else gd[L-1]
TV view_de(slpic_unet_t *h, int l)
{
    if (l == h->L - 1)
        return TV{h->gd[l], ch(h, l), 0};
    return TV{h->dcat[l], ch(h, l + 1) + ch(h, l), ch(h, l + 1)};
}

unsigned grid_for(size_t n)
{
    size_t b = (n + kT - 1) / kT;
    if (b > 152 * 16)
        b = 152 * 16;
    return (unsigned)(b ? b : 1);
}

constexpr int kTcMaxN = 256;

size_t tc_smem_bytes(int Np) { return 2 * (size_t)kTcChunkA + 2 * (size_t)Np * kTcKC * 2; }

// a tensor-core conv at `level` over all Np packed output channels, in slices of at
// most kTcMaxN (one launch each)
void conv_tc(slpic_unet_t *h, TV x, int cin, const __nv_bfloat16 *wp, int Np, const float *bias,
             int cout, TV a, int relu, int level, int nb, cudaStream_t st)
{
    const int H = hl(h, level), W = wl(h, level);
    dim3 g((unsigned)((H * W + kTcM - 1) / kTcM), (unsigned)nb);
    for (int o0 = 0; o0 < Np; o0 += kTcMaxN) {
        const int n = std::min(kTcMaxN, Np - o0);
        TV as = a;
        as.coff += o0;
        k_conv_fwd_tc<<<g, kTcThreads, tc_smem_bytes(n), st>>>(
            x, cin, wp + (size_t)o0 * kTcKC, (size_t)Np * kTcKC, bias + o0, std::min(cout - o0, n), n,
            as, relu, H, W, h->d_flag);
    }
}

void conv_fwd(slpic_unet_t *h, int k, TV x, TV a, int relu, int nb, cudaStream_t st)
{
    const ConvSpec &c = h->conv[k];
    const int H = hl(h, c.level), W = wl(h, c.level);
    if (h->cfg.tensor_cores) {
        conv_tc(h, x, c.cin, h->wtc + c.tc_off, c.Np, h->p + c.b_off, c.cout, a, relu, c.level, nb, st);
        return;
    }
    dim3 grid((unsigned)((H * W + kT - 1) / kT), (unsigned)((c.cout + kOCB - 1) / kOCB), (unsigned)nb);
    k_conv_fwd<<<grid, kT, 0, st>>>(x, c.cin, h->pb + c.w_off, h->p + c.b_off, c.cout, a, relu, H, W);
}

// K split of the tensor-core weight gradient: (M tiles, splits, 64-pixel chunks per split)
void wgrad_split(const slpic_unet_t *h, const ConvSpec &c, int nb, int *mt, int *splits, int *per)
{
    const long long npix = (long long)nb * hwl(h, c.level);
    const long long nchunk = (npix + kTcKC - 1) / kTcKC;
    *mt = (9 * ((c.cin + 15) / 16 * 16) + kTcM - 1) / kTcM;
    long long sp = std::max(1LL, std::min(nchunk, (long long)(2 * 152 + *mt - 1) / *mt));
    *per = (int)((nchunk + sp - 1) / sp);
    *splits = (int)((nchunk + *per - 1) / *per);
}

void conv_bwd(slpic_unet_t *h, int k, TV x, TV dz, TV *dx, int nb, cudaStream_t st)
{
    const ConvSpec &c = h->conv[k];
    const int H = hl(h, c.level), W = wl(h, c.level);
    if (h->cfg.tensor_cores && c.Np <= kTcMaxN) {
        int mt, splits, per;
        wgrad_split(h, c, nb, &mt, &splits, &per);
        k_conv_wgrad_tc<<<dim3((unsigned)mt, (unsigned)splits), kTcThreads, tc_smem_bytes(c.Np), st>>>(
            x, c.cin, dz, c.cout, c.Np, H, W, nb, per, h->wpart, h->d_flag);
        k_wgrad_reduce<<<grid_for((size_t)c.cout * c.cin * 9), kT, 0, st>>>(
            h->wpart, splits, mt * kTcM, c.Np, c.cin, c.cout, h->g + c.w_off);
        k_bias_grad<<<c.cout, kT, 0, st>>>(dz, c.cout, H * W, nb, h->g + c.b_off);
    } else {
        k_conv_bwd_w<<<dim3((unsigned)c.cin, (unsigned)c.cout), kT, 0, st>>>(
            x, c.cin, dz, c.cout, h->g + c.w_off, h->g + c.b_off, H, W, nb, h->cfg.tensor_cores ? 1 : 0);
    }
    if (dx && h->cfg.tensor_cores) {
        conv_tc(h, dz, c.cout, h->wtct + c.tct_off, c.Npt, h->zeros, c.cin, *dx, 0, c.level, nb, st);
    } else if (dx) {
        dim3 grid((unsigned)((H * W + kT - 1) / kT), (unsigned)((c.cin + kOCB - 1) / kOCB),
                  (unsigned)nb);
        k_conv_bwd_x<<<grid, kT, 0, st>>>(dz, c.cout, h->pb + c.w_off, c.cin, *dx, H, W);
    }
}

// (pixel blocks, planes) for an elementwise kernel over `pixels` per plane
dim3 plane_grid(size_t pixels, int nplanes)
{
    const size_t bx = std::min<size_t>((pixels + kT - 1) / kT, 1024);
    return dim3((unsigned)std::max<size_t>(bx, 1), (unsigned)std::min(nplanes, 65535));
}

void relu_bwd(slpic_unet_t *h, TV a, TV gv, int C, int level, int nb, cudaStream_t st)
{
    const size_t HW = hwl(h, level);
    k_relu_bwd<<<plane_grid(HW, nb * C), kT, 0, st>>>(a, gv, C, (int)HW, nb * C);
}

// The forward pass on the normalised input h->xin: fills every activation and
// h->ynet (network units).
void forward_net(slpic_unet_t *h, int nb, cudaStream_t st)
{
    const int L = h->L;
    if (h->cfg.tensor_cores && h->tc_dirty) {
        for (const ConvSpec &c : h->conv) {
            k_pack_tc<<<grid_for((size_t)c.nkc * c.Np * kTcKC), kT, 0, st>>>(
                h->pb + c.w_off, c.cout, c.cin, c.Np, c.nkc, h->wtc + c.tc_off);
            k_pack_tc_t<<<grid_for((size_t)c.nkct * c.Npt * kTcKC), kT, 0, st>>>(
                h->pb + c.w_off, c.cout, c.cin, c.Npt, c.nkct, h->wtct + c.tct_off);
        }
        h->tc_dirty = false;
    }
    for (int l = 0; l < L; ++l) {
        if (l > 0)
            k_pool_fwd<<<plane_grid(hwl(h, l), nb * ch(h, l - 1)), kT, 0, st>>>(
                view_e(h, l - 1), view_enc_in(h, l), ch(h, l - 1), hl(h, l - 1), wl(h, l - 1),
                nb * ch(h, l - 1));
        conv_fwd(h, l, view_enc_in(h, l), view_e(h, l), 1, nb, st);
    }
    for (int l = L - 2; l >= 0; --l) {
        TV up_dst{h->cat[l], ch(h, l + 1) + ch(h, l), 0};
        k_up_fwd<<<plane_grid(hwl(h, l), nb * ch(h, l + 1)), kT, 0, st>>>(
            view_d(h, l + 1), up_dst, ch(h, l + 1), hl(h, l + 1), wl(h, l + 1), nb * ch(h, l + 1));
        conv_fwd(h, L + (L - 2 - l), TV{h->cat[l], ch(h, l + 1) + ch(h, l), 0}, view_d(h, l), 1, nb,
                 st);
    }
    conv_fwd(h, 2 * L - 1, view_d(h, 0), TV{h->ynet, 1, 0}, 0, nb, st);
}

// The backward pass from h->dy (network units); parameter gradients into h->g.
void backward_net(slpic_unet_t *h, int nb, cudaStream_t st)
{
    const int L = h->L;
    TV gd0{h->gd[0], ch(h, 0), 0};
    conv_bwd(h, 2 * L - 1, view_d(h, 0), TV{h->dy, 1, 0}, &gd0, nb, st);
    for (int l = 0; l <= L - 2; ++l) {
        const int k = L + (L - 2 - l);
        TV gdl{h->gd[l], ch(h, l), 0};
        relu_bwd(h, view_d(h, l), gdl, ch(h, l), l, nb, st);
        TV catv{h->cat[l], ch(h, l + 1) + ch(h, l), 0};
        TV dcatv{h->dcat[l], ch(h, l + 1) + ch(h, l), 0};
        conv_bwd(h, k, catv, gdl, &dcatv, nb, st);
        k_up_bwd<<<plane_grid(hwl(h, l + 1), nb * ch(h, l + 1)), kT, 0, st>>>(
            dcatv, TV{h->gd[l + 1], ch(h, l + 1), 0}, ch(h, l + 1), hl(h, l + 1), wl(h, l + 1),
            nb * ch(h, l + 1));
    }
    for (int l = L - 1; l >= 0; --l) {
        TV de = view_de(h, l);
        relu_bwd(h, view_e(h, l), de, ch(h, l), l, nb, st);
        if (l > 0) {
            TV dp{h->dpool[l], ch(h, l - 1), 0};
            conv_bwd(h, l, view_enc_in(h, l), de, &dp, nb, st);
            k_pool_bwd_add<<<plane_grid(hwl(h, l - 1), nb * ch(h, l - 1)), kT, 0, st>>>(
                dp, view_de(h, l - 1), ch(h, l - 1), hl(h, l - 1), wl(h, l - 1), nb * ch(h, l - 1));
        } else {
            conv_bwd(h, l, view_enc_in(h, l), de, nullptr, nb, st);
        }
    }
}

int ensure_grads(slpic_unet_t *h)
{
    if (h->have_grads)
        return SLPIC_OK;
    const int L = h->L, nb = h->nbmax;
    int rc;
    if ((rc = alloc_f(h, &h->g, h->nparam)) || (rc = alloc_f(h, &h->m, h->nparam)) ||
        (rc = alloc_f(h, &h->v, h->nparam)) || (rc = alloc_f(h, &h->dy, (size_t)nb * hwl(h, 0))))
        return rc;
    if (h->cfg.loss == SLPIC_UNET_LOSS_ENERGY && (rc = alloc_f(h, &h->eb, (size_t)nb * hwl(h, 0))))
        return rc;
    if ((rc = alloc(h, (void **)&h->part, sizeof(double) * kMseCtas)) ||
        (rc = alloc(h, (void **)&h->loss, sizeof(double))))
        return rc;
    h->dcat.assign(L, nullptr);
    h->gd.assign(L, nullptr);
    h->dpool.assign(L, nullptr);
    for (int l = 0; l < L; ++l) {
        if ((rc = alloc_f(h, &h->gd[l], (size_t)nb * ch(h, l) * hwl(h, l))))
            return rc;
        if (l <= L - 2 &&
            (rc = alloc_f(h, &h->dcat[l], (size_t)nb * (ch(h, l + 1) + ch(h, l)) * hwl(h, l))))
            return rc;
        if (l >= 1 && (rc = alloc_f(h, &h->dpool[l], (size_t)nb * ch(h, l - 1) * hwl(h, l))))
            return rc;
    }
    if (h->cfg.tensor_cores) {
        size_t need = 1;
        for (const ConvSpec &c : h->conv) {
            if (c.Np > kTcMaxN)
                continue;
            for (int b = 1; b <= nb; ++b) {  // the split depends on the batch of the call
                int mt, splits, per;
                wgrad_split(h, c, b, &mt, &splits, &per);
                need = std::max(need, (size_t)splits * mt * kTcM * c.Np);
            }
        }
        if ((rc = alloc_f(h, &h->wpart, need)))
            return rc;
        h->wpart_n = need;
    }
    CKU(h, cudaMemsetAsync(h->m, 0, sizeof(float) * h->nparam, h->stream));
    CKU(h, cudaMemsetAsync(h->v, 0, sizeof(float) * h->nparam, h->stream));
    h->adam_t = 0;
    h->have_grads = true;
    return SLPIC_OK;
}

// SplitMix64 (Steele, Lea & Flood, 2014) and Box-Muller for the initial weights
uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

double uniform01(uint64_t &x) { return ((splitmix64(x) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

int check_batch(slpic_unet_t *h, int nb, const void *a, const void *b)
{
    if (nb < 1 || nb > h->nbmax)
        return failu(h, SLPIC_ERR_INVALID, "nb outside 1..max_batch");
    if (!a || !b)
        return failu(h, SLPIC_ERR_INVALID, "null array");
    return SLPIC_OK;
}

int run_gradients(slpic_unet_t *h, int nb, const float *x, const float *t, cudaStream_t st)
{
    int rc = ensure_grads(h);
    if (rc)
        return rc;
    const size_t HW = hwl(h, 0);
    k_norm_in<<<nb, kT, 0, st>>>(x, h->xin, h->s, HW, h->cfg.normalise);
    forward_net(h, nb, st);
    if (h->cfg.loss == SLPIC_UNET_LOSS_ENERGY) {
        k_energy_err<<<grid_for((size_t)nb * HW), kT, 0, st>>>(h->ynet, t, h->s, (float)h->cfg.out_scale,
                                                               h->eb, h->H, h->W, nb);
        k_energy_grad<<<kMseCtas, kT, 0, st>>>(h->eb, h->dy, h->H, h->W, nb, h->part);
    } else {
        k_mse<<<kMseCtas, kT, 0, st>>>(h->ynet, t, h->s, (float)h->cfg.out_scale, h->dy, HW, nb,
                                       h->part);
    }
    k_loss<<<1, kT, 0, st>>>(h->part, kMseCtas, (double)nb * HW, h->loss);
    backward_net(h, nb, st);
    CKU(h, cudaGetLastError());
    return SLPIC_OK;
}

}  // namespace

extern "C" int slpic_unet_create(const slpic_unet_config *cfg, slpic_unet_t **out)
{
    if (!cfg || !out)
        return SLPIC_ERR_INVALID;
    *out = nullptr;
    const slpic_unet_config &c = *cfg;
    if (c.levels < 1 || c.levels > 12 || c.base < 1 || c.max_batch < 1 || c.height < 1 ||
        c.width < 1 || !(c.out_scale > 0) ||
        (c.loss != SLPIC_UNET_LOSS_MSE && c.loss != SLPIC_UNET_LOSS_ENERGY) ||
        (c.tensor_cores != 0 && c.tensor_cores != 1))
        return SLPIC_ERR_INVALID;
    const int f = 1 << (c.levels - 1);
    if (c.height % f || c.width % f || (long long)c.height * c.width > (1LL << 28) ||
        ((long long)c.base << (c.levels - 1)) > 4096)
        return SLPIC_ERR_INVALID;
    slpic_unet_t *h = new slpic_unet_t;
    h->cfg = c;
    if (!(h->cfg.adam_beta1 > 0))
        h->cfg.adam_beta1 = 0.9;
    if (!(h->cfg.adam_beta2 > 0))
        h->cfg.adam_beta2 = 0.999;
    if (!(h->cfg.adam_eps > 0))
        h->cfg.adam_eps = 1e-8;
    h->L = c.levels;
    h->C = c.base;
    h->H = c.height;
    h->W = c.width;
    h->nbmax = c.max_batch;
    const int L = h->L;
    // parameter layout: encoder 0..L-1, decoder L-2..0, output
    auto add = [&](int cin, int cout, int level) {
        ConvSpec s{cin, cout, level, h->nparam, h->nparam + (size_t)cout * cin * 9};
        h->nparam = s.b_off + cout;
        h->conv.push_back(s);
    };
    add(1, ch(h, 0), 0);
    for (int l = 1; l < L; ++l)
        add(ch(h, l - 1), ch(h, l), l);
    for (int l = L - 2; l >= 0; --l)
        add(ch(h, l + 1) + ch(h, l), ch(h, l), l);
    add(ch(h, 0), 1, 0);
    size_t ntc = 0, ntct = 0;  // packed tensor-core weights: forward, transposed
    int maxc = 1;
    for (ConvSpec &s : h->conv) {
        s.Np = (s.cout + 15) / 16 * 16;
        s.nkc = (9 * ((s.cin + 15) / 16 * 16) + kTcKC - 1) / kTcKC;
        s.tc_off = ntc;
        ntc += (size_t)s.nkc * s.Np * kTcKC;
        s.Npt = (s.cin + 15) / 16 * 16;
        s.nkct = (9 * ((s.cout + 15) / 16 * 16) + kTcKC - 1) / kTcKC;
        s.tct_off = ntct;
        ntct += (size_t)s.nkct * s.Npt * kTcKC;
        maxc = std::max(maxc, std::max(s.Np, s.Npt));
    }

    const int nb = h->nbmax;
    int rc = SLPIC_OK;
    h->cat.assign(L, nullptr);
    h->d.assign(L, nullptr);
    h->pin.assign(L, nullptr);
    if (!rc) rc = alloc_f(h, &h->p, h->nparam);
    if (!rc) rc = alloc(h, (void **)&h->pb, sizeof(__nv_bfloat16) * h->nparam);
    if (!rc && c.tensor_cores) {
        rc = alloc(h, (void **)&h->wtc, sizeof(__nv_bfloat16) * ntc);
        if (!rc)
            rc = alloc(h, (void **)&h->wtct, sizeof(__nv_bfloat16) * ntct);
        if (!rc)
            rc = alloc_f(h, &h->zeros, (size_t)maxc);
        if (!rc)
            rc = alloc(h, (void **)&h->d_flag, sizeof(int));
        if (!rc) {
            cudaError_t e = cudaMemset(h->d_flag, 0, sizeof(int));
            if (e == cudaSuccess)
                e = cudaMemset(h->zeros, 0, sizeof(float) * maxc);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_conv_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes(kTcMaxN));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_conv_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes(kTcMaxN));
            if (e != cudaSuccess)
                rc = failu(h, SLPIC_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    if (!rc) rc = alloc_f(h, &h->xin, (size_t)nb * hwl(h, 0));
    if (!rc) rc = alloc_f(h, &h->s, (size_t)nb);
    if (!rc) rc = alloc_f(h, &h->ynet, (size_t)nb * hwl(h, 0));
    if (!rc) rc = alloc_f(h, &h->etop, (size_t)nb * ch(h, L - 1) * hwl(h, L - 1));
    for (int l = 0; l < L && !rc; ++l) {
        if (l <= L - 2) {
            rc = alloc_f(h, &h->cat[l], (size_t)nb * (ch(h, l + 1) + ch(h, l)) * hwl(h, l));
            if (!rc)
                rc = alloc_f(h, &h->d[l], (size_t)nb * ch(h, l) * hwl(h, l));
        }
        if (!rc && l >= 1)
            rc = alloc_f(h, &h->pin[l], (size_t)nb * ch(h, l - 1) * hwl(h, l));
    }
    if (!rc) {
        // He-normal weights, zero biases
        std::vector<float> init(h->nparam, 0.0f);
        uint64_t st = c.seed;
        for (const ConvSpec &s : h->conv) {
            const double sd = std::sqrt(2.0 / (9.0 * s.cin));
            for (size_t q = 0; q < (size_t)s.cout * s.cin * 9; q += 2) {
                const double u1 = uniform01(st), u2 = uniform01(st);
                const double r = std::sqrt(-2.0 * std::log(u1));
                init[s.w_off + q] = (float)(sd * r * std::cos(6.283185307179586 * u2));
                if (q + 1 < (size_t)s.cout * s.cin * 9)
                    init[s.w_off + q + 1] = (float)(sd * r * std::sin(6.283185307179586 * u2));
            }
        }
        rc = slpic_unet_set_params(h, init.data());
    }
    if (rc) {
        slpic_unet_destroy(h);
        return rc;
    }
    *out = h;
    return SLPIC_OK;
}

extern "C" int slpic_unet_destroy(slpic_unet_t *h)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    cudaStreamSynchronize(h->stream);
    for (void *a : h->allocs)
        cudaFree(a);
    delete h;
    return SLPIC_OK;
}

extern "C" const char *slpic_unet_last_error(slpic_unet_t *h) { return h ? h->err.c_str() : "null handle"; }

extern "C" int slpic_unet_set_stream(slpic_unet_t *h, void *stream)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    h->stream = (cudaStream_t)stream;
    return SLPIC_OK;
}

extern "C" int slpic_unet_param_count(slpic_unet_t *h, int64_t *n)
{
    if (!h || !n)
        return SLPIC_ERR_INVALID;
    *n = (int64_t)h->nparam;
    return SLPIC_OK;
}

extern "C" int slpic_unet_set_params(slpic_unet_t *h, const float *params)
{
    if (!h || !params)
        return h ? failu(h, SLPIC_ERR_INVALID, "null array") : SLPIC_ERR_INVALID;
    CKU(h, cudaMemcpyAsync(h->p, params, sizeof(float) * h->nparam, cudaMemcpyHostToDevice, h->stream));
    k_to_bf16<<<grid_for(h->nparam), kT, 0, h->stream>>>(h->p, h->pb, h->nparam);
    h->tc_dirty = true;
    CKU(h, cudaGetLastError());
    CKU(h, cudaStreamSynchronize(h->stream));
    return SLPIC_OK;
}

extern "C" int slpic_unet_get_params(slpic_unet_t *h, float *params)
{
    if (!h || !params)
        return h ? failu(h, SLPIC_ERR_INVALID, "null array") : SLPIC_ERR_INVALID;
    CKU(h, cudaMemcpyAsync(params, h->p, sizeof(float) * h->nparam, cudaMemcpyDeviceToHost, h->stream));
    CKU(h, cudaStreamSynchronize(h->stream));
    return check_flag(h);
}

int slpic_unet_forward_on(slpic_unet_t *h, int nb, const float *x, float *y, cudaStream_t st)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    int rc = check_batch(h, nb, x, y);
    if (rc)
        return rc;
    const size_t HW = hwl(h, 0);
    k_norm_in<<<nb, kT, 0, st>>>(x, h->xin, h->s, HW, h->cfg.normalise);
    forward_net(h, nb, st);
    k_scale_out<<<grid_for((size_t)nb * HW), kT, 0, st>>>(h->ynet, y, h->s, (float)h->cfg.out_scale,
                                                          HW, nb);
    CKU(h, cudaGetLastError());
    return SLPIC_OK;
}

void slpic_unet_shape(const slpic_unet_t *h, int *height, int *width, int *max_batch)
{
    *height = h->H;
    *width = h->W;
    *max_batch = h->nbmax;
}

extern "C" int slpic_unet_forward(slpic_unet_t *h, int32_t nb, const float *x, float *y)
{
    return h ? slpic_unet_forward_on(h, nb, x, y, h->stream) : SLPIC_ERR_INVALID;
}

extern "C" int slpic_unet_gradients(slpic_unet_t *h, int32_t nb, const float *x, const float *t,
                                    double *loss, float *grads)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    int rc = check_batch(h, nb, x, t);
    if (rc || (rc = run_gradients(h, nb, x, t, h->stream)))
        return rc;
    if (grads)
        CKU(h, cudaMemcpyAsync(grads, h->g, sizeof(float) * h->nparam, cudaMemcpyDeviceToHost,
                               h->stream));
    if (loss)
        CKU(h, cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (grads || loss) {
        CKU(h, cudaStreamSynchronize(h->stream));
        return check_flag(h);
    }
    return SLPIC_OK;
}

extern "C" int slpic_unet_train_step(slpic_unet_t *h, int32_t nb, const float *x, const float *t,
                                     double lr, double *loss)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    if (!(lr > 0))
        return failu(h, SLPIC_ERR_INVALID, "lr must be > 0");
    int rc = check_batch(h, nb, x, t);
    if (rc || (rc = run_gradients(h, nb, x, t, h->stream)))
        return rc;
    ++h->adam_t;
    const double b1 = h->cfg.adam_beta1, b2 = h->cfg.adam_beta2;
    const double c1 = 1.0 - std::pow(b1, (double)h->adam_t);
    const double c2 = 1.0 - std::pow(b2, (double)h->adam_t);
    h->tc_dirty = true;
    k_adam<<<grid_for(h->nparam), kT, 0, h->stream>>>(h->p, h->g, h->m, h->v, h->pb, h->nparam,
                                                     (float)lr, (float)b1, (float)b2,
                                                     (float)h->cfg.adam_eps, (float)c1, (float)c2);
    CKU(h, cudaGetLastError());
    if (loss) {
        CKU(h, cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CKU(h, cudaStreamSynchronize(h->stream));
        return check_flag(h);
    }
    return SLPIC_OK;
}

extern "C" int slpic_unet_reset_optimizer(slpic_unet_t *h)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    if (h->have_grads) {
        CKU(h, cudaMemsetAsync(h->m, 0, sizeof(float) * h->nparam, h->stream));
        CKU(h, cudaMemsetAsync(h->v, 0, sizeof(float) * h->nparam, h->stream));
    }
    h->adam_t = 0;
    return SLPIC_OK;
}
