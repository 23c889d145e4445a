// api.cu -- the C ABI declared in include/slpic.h.
//
// The handle owns all device memory of one simulation; the timestep runs as a
// captured CUDA graph (particle kernel, then field kernel) whose kernels read
// the time level from device memory, so one graph serves every step.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.h"
#include "slpic.h"
#include "slpic_internal.cuh"

using namespace slpic;

struct slpic_sim {
    slpic_config cfg{};
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;     // work stream (caller may replace)
    cudaStream_t own_stream = nullptr; // created here
    cudaStream_t cap_stream = nullptr; // private stream used only for graph capture
    StepParams p{};
    int nn = 0, ns = 0;
    int ctas = 1;        // in-place particle-kernel CTAs per species
    int ctas_c = 1;      // compacting particle-kernel CTAs per species
    int hard_ctas = 1;   // k_hard CTAs
    int tma_stages = 0;  // k_particles_tma ring stages for in-place steps (0: k_particles)
    // performance settings (slpic_set_tuning / slpic_autotune); results do not depend
    // on them
    int compact_every = kCompactEvery;  // a compacting particle step every this many
    int particle_kernel = 0;            // in-place steps: 0 TMA-staged if it fits, 1 per-warp
    int batch_waves = 2;                // batches: work items ~ waves x resident CTAs
    int batch_min_share = 4096;         // batches: fewest particles per work item
    int small_ctas = 1;  // CTAs per species for deposit / diag
    long long step = 0;  // host mirror of DevState::step
    bool dirty = true;   // particles loaded since the last deposit/solve

    DevState *d_state = nullptr;
    unsigned long long *d_acc = nullptr;
    float *d_E = nullptr;
    double *d_E64 = nullptr, *d_phi = nullptr, *d_rho = nullptr;
    int32_t *d_cell[kMaxSpecies][2] = {};
    float4 *d_pv[kMaxSpecies][2] = {};
    HardRec *d_hard[kMaxSpecies] = {};
    int32_t *d_hard_slot[kMaxSpecies] = {};
    double *d_diag = nullptr;
    int *d_bad = nullptr;
    float *d_lam = nullptr;  // speed-limit profile (slpic_set_speed_limit_profile)
    double lam_max = 1.0;    // its largest factor (1 without a profile)
    void *d_stage = nullptr;  // load/read-back staging
    size_t stage_bytes = 0;

    cudaGraphExec_t g1 = nullptr;   // one in-place step
    cudaGraphExec_t gc = nullptr;   // one compacting step
    cudaGraphExec_t gK = nullptr;   // one cycle: compact_every - 1 in-place steps, 1 compacting
    cudaGraphExec_t gt = nullptr;   // timed graph: t_len steps from phase t_phase, with events
    std::vector<cudaEvent_t> events; // 3 per step of the timed graph
    long long t_len = 0;             // steps per timed graph (0 = timing off)
    long long t_phase = -1;          // step % compact_every at which gt starts
    long long t_launched = 0;        // timed-graph launches since timing was enabled

    // a batch of independent simulations (slpic_create_batch): each member does its
    // own per-instance work (loads, read-back, diagnostics); the batch advances all
    // of them together with the batched kernels, captured in g1 / gc / gK
    // slpic_fields_async: the latest deposit and E copied on the step stream, the
    // potential and the host copies on a private read-back stream
    cudaStream_t rb_stream = nullptr;
    cudaEvent_t ev_snap = nullptr, ev_rb = nullptr;
    unsigned long long *d_snap_acc = nullptr;
    float *d_snap_E = nullptr;
    bool rb_used = false;

    std::vector<slpic_sim *> members;
    StepParams *d_params = nullptr;  // [members] on the device
    int4 *d_work = nullptr;          // particle-kernel work items
    int n_work = 0, max_nn = 0, max_ns = 0, batch_hard_ctas = 4;

    std::string err;
};

static thread_local std::string g_create_err;

#define CK(h, call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (h)->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
            return SLPIC_ERR_CUDA;                                                         \
        }                                                                                  \
    } while (0)

static int fail(slpic_t *h, int code, const std::string &msg)
{
    h->err = msg;
    return code;
}

// Records for the particles needing the iterative push: an eighth of the capacity
// (a step lists well under 1 % on the headline sheath), at least 64k; beyond that
// the list continues as bare slots.
static long long hard_records(long long capacity)
{
    return std::min(capacity, std::max(capacity / 8, 65536LL));
}

// A batch handle forwards a per-instance call to its member (as instance 0).
#define BATCH_FORWARD(h, instance, expr)                                                   \
    do {                                                                                   \
        if ((h) && !(h)->members.empty()) {                                                \
            if ((instance) < 0 || (instance) >= (int)(h)->members.size())                  \
                return fail((h), SLPIC_ERR_INVALID, "instance out of range");              \
            slpic_t *m_ = (h)->members[(instance)];                                        \
            const int rc_ = (expr);                                                        \
            if (rc_)                                                                       \
                (h)->err = m_->err;                                                        \
            return rc_;                                                                    \
        }                                                                                  \
    } while (0)

static bool is_batch(const slpic_t *h) { return h && !h->members.empty(); }

static int check_handle(slpic_t *h, int instance)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    if (instance != 0)
        return fail(h, SLPIC_ERR_INVALID, "instance must be 0");
    h->err.clear();
    CK(h, cudaSetDevice(h->device));
    return SLPIC_OK;
}

// Checks that need no device (the shared-memory fit is checked in slpic_create).
static int validate_config(const slpic_config *c, std::string &why)
{
    if (!c) {
        why = "cfg is NULL";
        return SLPIC_ERR_INVALID;
    }
    if (c->ndim != 1) {
        why = "ndim must be 1";
        return SLPIC_ERR_INVALID;
    }
    if (c->n_cells < 2 || !(c->dx > 0) || !(c->dt > 0) || !(c->eps0 > 0)) {
        why = "need n_cells >= 2 and dx, dt, eps0 > 0";
        return SLPIC_ERR_INVALID;
    }
    if (c->bc != SLPIC_BC_PERIODIC && c->bc != SLPIC_BC_DIRICHLET_ABSORB) {
        why = "unknown bc";
        return SLPIC_ERR_INVALID;
    }
    if (c->n_species < 1 || c->n_species > SLPIC_MAX_SPECIES) {
        why = "n_species must be 1..4";
        return SLPIC_ERR_INVALID;
    }
    for (int s = 0; s < c->n_species; ++s) {
        const slpic_species &sp = c->species[s];
        if (!(sp.m > 0) || !(sp.w > 0) || sp.capacity <= 0 || !std::isfinite(sp.q)) {
            why = "species " + std::to_string(s) + ": need m > 0, w > 0, capacity > 0";
            return SLPIC_ERR_INVALID;
        }
        if (sp.beta_kind < SLPIC_BETA_ONE || sp.beta_kind > SLPIC_BETA_RELATIVISTIC) {
            why = "species " + std::to_string(s) + ": unknown beta_kind";
            return SLPIC_ERR_INVALID;
        }
        if (sp.capacity > (1LL << 31) - 1) {
            why = "species " + std::to_string(s) + ": capacity above 2^31-1";
            return SLPIC_ERR_INVALID;
        }
        if (sp.beta_kind != SLPIC_BETA_ONE) {
            if (!(sp.v0 > 0)) {
                why = "species " + std::to_string(s) + ": v0 must be > 0";
                return SLPIC_ERR_INVALID;
            }
            // |beta v| <= v0, so dt v0 <= dx keeps every move within one cell
            if (c->dt * sp.v0 > c->dx * (1.0 + 1e-12)) {
                why = "species " + std::to_string(s) + ": dt * v0 > dx";
                return SLPIC_ERR_CFL;
            }
        } else if (c->max_speed > 0 && c->dt * c->max_speed > c->dx * (1.0 + 1e-12)) {
            why = "species " + std::to_string(s) + ": dt * max_speed > dx";
            return SLPIC_ERR_CFL;
        }
        if (sp.T_src < 0) {
            why = "species " + std::to_string(s) + ": T_src < 0";
            return SLPIC_ERR_INVALID;
        }
    }
    if (c->src_mode == SLPIC_SRC_WALL) {
        if (c->bc != SLPIC_BC_DIRICHLET_ABSORB) {
            why = "the wall source needs the absorbing plates";
            return SLPIC_ERR_INVALID;
        }
        if (!(c->src_rate >= 0)) {
            why = "src_rate (source density) < 0";
            return SLPIC_ERR_INVALID;
        }
    } else if (c->src_mode != SLPIC_SRC_NONE) {
        if (c->src_mode != SLPIC_SRC_LOSS_MATCHED && c->src_mode != SLPIC_SRC_RATE) {
            why = "unknown src_mode";
            return SLPIC_ERR_INVALID;
        }
        if (!(c->src_lo_cells >= 0) || !(c->src_len_cells > 0) ||
            !(c->src_lo_cells + c->src_len_cells < c->n_cells)) {
            why = "source band must satisfy 0 <= lo, len > 0, lo + len < n_cells";
            return SLPIC_ERR_INVALID;
        }
        if (c->src_mode == SLPIC_SRC_LOSS_MATCHED &&
            (c->src_ref_species < 0 || c->src_ref_species >= c->n_species)) {
            why = "src_ref_species out of range";
            return SLPIC_ERR_INVALID;
        }
        if (c->src_mode == SLPIC_SRC_RATE && !(c->src_rate >= 0)) {
            why = "src_rate < 0";
            return SLPIC_ERR_INVALID;
        }
    }
    return SLPIC_OK;
}

static void free_all(slpic_t *h)
{
    cudaSetDevice(h->device);
    if (h->g1)
        cudaGraphExecDestroy(h->g1);
    if (h->gc)
        cudaGraphExecDestroy(h->gc);
    if (h->gK)
        cudaGraphExecDestroy(h->gK);
    if (h->gt)
        cudaGraphExecDestroy(h->gt);
    for (cudaEvent_t e : h->events)
        cudaEventDestroy(e);
    if (h->rb_stream) {
        cudaStreamSynchronize(h->rb_stream);
        cudaStreamDestroy(h->rb_stream);
    }
    if (h->ev_snap)
        cudaEventDestroy(h->ev_snap);
    if (h->ev_rb)
        cudaEventDestroy(h->ev_rb);
    cudaFree(h->d_snap_acc);
    cudaFree(h->d_snap_E);
    cudaFree(h->d_state);
    cudaFree(h->d_acc);
    cudaFree(h->d_E);
    cudaFree(h->d_E64);
    cudaFree(h->d_phi);
    cudaFree(h->d_rho);
    cudaFree(h->d_diag);
    cudaFree(h->d_bad);
    cudaFree(h->d_lam);
    cudaFree(h->d_stage);
    for (int s = 0; s < kMaxSpecies; ++s) {
        for (int b = 0; b < 2; ++b) {
            cudaFree(h->d_cell[s][b]);
            cudaFree(h->d_pv[s][b]);
        }
        cudaFree(h->d_hard[s]);
        cudaFree(h->d_hard_slot[s]);
    }
    if (h->own_stream)
        cudaStreamDestroy(h->own_stream);
    if (h->cap_stream)
        cudaStreamDestroy(h->cap_stream);
}

extern "C" const char *slpic_create_error(void) { return g_create_err.c_str(); }

namespace slpic {
// slpic2d_create and slpic_fp64_create report their failures through
// slpic_create_error too, and the FP64 form validates its config as slpic_create does
void set_create_error(const std::string &msg) { g_create_err = msg; }
int check_config(const slpic_config *c, std::string &why) { return validate_config(c, why); }
}  // namespace slpic

extern "C" int slpic_create(const slpic_config *cfg, slpic_t **out)
{
    g_create_err.clear();
    if (!out) {
        g_create_err = "out is NULL";
        return SLPIC_ERR_INVALID;
    }
    std::string why;
    int rc = validate_config(cfg, why);
    if (rc != SLPIC_OK) {
        g_create_err = why;
        return rc;
    }
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) {
        g_create_err = std::string("no CUDA device: ") + cudaGetErrorString(ce);
        return SLPIC_ERR_CUDA;
    }
    int max_smem = 0, sms = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    {
        int nn_ = cfg->bc == SLPIC_BC_PERIODIC ? cfg->n_cells : cfg->n_cells + 1;
        // the particle kernel's E and deposit, plus its static shared memory; the field
        // kernel's deposits and prefixes per cluster CTA, plus its static shared memory
        if (particle_kernel_smem_bytes(nn_) + 1024 > (size_t)max_smem ||
            field_cluster_smem_bytes(nn_, kMaxSpecies, kFieldClusterCtas) + 4096 > (size_t)max_smem ||
            nn_ > field_max_nodes()) {
            g_create_err = "grid does not fit in shared memory (n_cells too large for the 1D kernel)";
            return SLPIC_ERR_INVALID;
        }
    }
    slpic_t *h = new slpic_sim();
    h->cfg = *cfg;
    h->device = dev;
    h->num_sms = sms;
    h->ns = cfg->n_species;
    h->nn = cfg->bc == SLPIC_BC_PERIODIC ? cfg->n_cells : cfg->n_cells + 1;

    auto bail = [&](int code, const std::string &msg) {
        g_create_err = msg;
        free_all(h);
        delete h;
        return code;
    };
#define CKC(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return bail(e_ == cudaErrorMemoryAllocation ? SLPIC_ERR_OOM : SLPIC_ERR_CUDA,  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

    CKC(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    CKC(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    h->stream = h->own_stream;
    const int nn = h->nn, ns = h->ns;
    CKC(cudaMalloc(&h->d_state, sizeof(DevState)));
    CKC(cudaMalloc(&h->d_acc, sizeof(unsigned long long) * 2 * ns * nn));
    CKC(cudaMalloc(&h->d_E, sizeof(float) * nn));
    CKC(cudaMalloc(&h->d_E64, sizeof(double) * nn));
    CKC(cudaMalloc(&h->d_phi, sizeof(double) * nn));
    CKC(cudaMalloc(&h->d_rho, sizeof(double) * nn));
    CKC(cudaMalloc(&h->d_diag, sizeof(double) * 2 * kMaxSpecies));
    CKC(cudaMalloc(&h->d_bad, sizeof(int)));
    for (int s = 0; s < ns; ++s) {
        for (int b = 0; b < 2; ++b) {
            CKC(cudaMalloc(&h->d_cell[s][b], sizeof(int32_t) * cfg->species[s].capacity));
            CKC(cudaMalloc(&h->d_pv[s][b], sizeof(float4) * cfg->species[s].capacity));
            // every slot starts as a hole (cell -1): a step cut short by a wait that
            // gave up leaves slots unwritten, and a later step must find them valid
            CKC(cudaMemset(h->d_cell[s][b], 0xFF, sizeof(int32_t) * cfg->species[s].capacity));
        }
        CKC(cudaMalloc(&h->d_hard[s], sizeof(HardRec) * hard_records(cfg->species[s].capacity)));
        CKC(cudaMalloc(&h->d_hard_slot[s], sizeof(int32_t) * cfg->species[s].capacity));
    }
    CKC(cudaMemset(h->d_state, 0, sizeof(DevState)));
    CKC(cudaMemset(h->d_acc, 0, sizeof(unsigned long long) * 2 * ns * nn));
    CKC(cudaMemset(h->d_E, 0, sizeof(float) * nn));
    CKC(cudaMemset(h->d_E64, 0, sizeof(double) * nn));
    CKC(cudaMemset(h->d_phi, 0, sizeof(double) * nn));
    CKC(cudaMemset(h->d_rho, 0, sizeof(double) * nn));
    CKC(configure_kernels(nn));
    int occ = 0, occ_c = 0;
    CKC(particle_ctas_per_sm(nn, &occ, &occ_c));
    if (occ < 1 || occ_c < 1)
        return bail(SLPIC_ERR_INVALID, "particle kernel cannot be resident (shared memory)");
    // persistent grids: every SM holds `occ` particle CTAs, shared among species
    h->ctas = std::max(1, sms * occ / ns);
    h->ctas_c = std::max(1, sms * occ_c / ns);
    h->small_ctas = std::max(1, sms * 2 / ns);
    // k_hard: 2 CTAs of 256 threads per SM, one lane per listed particle for the
    // ~20k-80k a step lists here (a grid-stride loop beyond); measured against 4 and 8
    // per SM, whose idle CTAs cost about a microsecond
    h->hard_ctas = sms * 2;
    CKC(configure_particles_tma(nn, &h->tma_stages));

    StepParams &p = h->p;
    p.n_cells = cfg->n_cells;
    p.nn = nn;
    p.periodic = cfg->bc == SLPIC_BC_PERIODIC;
    p.ns = ns;
    p.dt = (float)cfg->dt;
    p.dt_dx = (float)(cfg->dt / cfg->dx);
    p.dx = cfg->dx;
    p.dt64 = cfg->dt;
    p.eps0 = cfg->eps0;
    p.phi_lo = cfg->phi_lo;
    p.phi_hi = cfg->phi_hi;
    p.inv_n = 1.0 / cfg->n_cells;
    p.inv_dx = 1.0 / cfg->dx;
    p.k2 = cfg->dx * cfg->dx / cfg->eps0;
    p.src_mode = cfg->src_mode;
    p.src_ref = cfg->src_ref_species;
    p.src_lo_cells = (float)cfg->src_lo_cells;
    p.src_len_cells = (float)cfg->src_len_cells;
    p.src_rate = cfg->src_rate;
    p.seed = cfg->seed;
    for (int s = 0; s < ns; ++s) {
        const slpic_species &sp = cfg->species[s];
        SpeciesDev &d = p.sp[s];
        for (int b = 0; b < 2; ++b) {
            d.cell[b] = h->d_cell[s][b];
            d.pv[b] = h->d_pv[s][b];
        }
        d.hard = h->d_hard[s];
        d.hard_slot = h->d_hard_slot[s];
        d.hard_recs = hard_records(cfg->species[s].capacity);
        d.capacity = sp.capacity;
        d.qm = (float)(sp.q / sp.m);
        d.v0 = sp.beta_kind == SLPIC_BETA_ONE ? INFINITY : (float)sp.v0;
        d.vth_src = sp.T_src > 0 ? (float)std::sqrt(sp.T_src / sp.m) : 0.0f;
        d.kind = sp.beta_kind;
        d.qw_dx = sp.q * sp.w / cfg->dx;
        d.rho_unit = d.qw_dx / 1099511627776.0;
        d.w = sp.w;
        d.inv_w = 1.0 / sp.w;
        // wall source: macroparticles per step of the one-sided Maxwellian flux
        d.wall_rate = cfg->src_mode == SLPIC_SRC_WALL && sp.T_src > 0
                          ? cfg->src_rate * std::sqrt(sp.T_src / sp.m) /
                                std::sqrt(2.0 * 3.14159265358979323846) * cfg->dt / sp.w
                          : 0.0;
    }
    p.acc = h->d_acc;
    p.E = h->d_E;
    p.E64 = h->d_E64;
    p.phi = h->d_phi;
    p.rho = h->d_rho;
    p.st = h->d_state;
    p.wait_cycles = kWaitCycles;
#undef CKC
    *out = h;
    return SLPIC_OK;
}

extern "C" int slpic_destroy(slpic_t *h)
{
    if (!h)
        return SLPIC_OK;
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    for (slpic_t *m : h->members)
        slpic_destroy(m);
    cudaFree(h->d_params);
    cudaFree(h->d_work);
    free_all(h);
    delete h;
    return SLPIC_OK;
}

extern "C" const char *slpic_last_error(const slpic_t *h) { return h ? h->err.c_str() : ""; }

extern "C" int slpic_set_stream(slpic_t *h, void *stream)
{
    if (!h)
        return SLPIC_ERR_INVALID;
    CK(h, cudaSetDevice(h->device));
    CK(h, cudaStreamSynchronize(h->stream));
    h->stream = (cudaStream_t)stream;
    for (slpic_t *m : h->members)
        m->stream = h->stream;
    return SLPIC_OK;
}

static int ensure_stage(slpic_t *h, size_t bytes)
{
    if (bytes <= h->stage_bytes)
        return SLPIC_OK;
    CK(h, cudaStreamSynchronize(h->stream));
    cudaFree(h->d_stage);
    h->d_stage = nullptr;
    h->stage_bytes = 0;
    CK(h, cudaMalloc(&h->d_stage, bytes));
    h->stage_bytes = bytes;
    return SLPIC_OK;
}

static int read_state(slpic_t *h, DevState *st)
{
    CK(h, cudaMemcpyAsync(st, h->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return SLPIC_OK;
}

// Append n particles already on the device (cell, off, v in host layout).
static int append_dev(slpic_t *h, int s, long long n, const int32_t *cell, const float *off,
                      const float *v)
{
    DevState st;
    int rc = read_state(h, &st);
    if (rc)
        return rc;
    const int P = (int)(h->step & 1);
    long long have = (long long)st.count[s][P];
    if (have + n > h->cfg.species[s].capacity)
        return fail(h, SLPIC_ERR_CAPACITY, "load exceeds the species capacity");
    CK(h, cudaMemsetAsync(h->d_bad, 0, sizeof(int), h->stream));
    launch_validate(cell, off, v, n, h->cfg.n_cells, h->d_bad, h->stream);
    CK(h, cudaGetLastError());
    int bad = 0;
    CK(h, cudaMemcpyAsync(&bad, h->d_bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (bad)
        return fail(h, SLPIC_ERR_INVALID,
                    "particle data out of range (cell not in [0,N), offset not in [0,1), or non-finite v)");
    launch_pack(cell, off, v, n, h->d_cell[s][P] + have, h->d_pv[s][P] + have, h->stream);
    CK(h, cudaGetLastError());
    unsigned long long nc = (unsigned long long)(have + n);
    CK(h, cudaMemcpyAsync(&h->d_state->count[s][P], &nc, sizeof(nc), cudaMemcpyHostToDevice,
                          h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->dirty = true;
    return SLPIC_OK;
}

extern "C" int slpic_load_particles(slpic_t *h, int instance, int species, int64_t n,
                                    const int32_t *cell, const float *offset, const float *v)
{
    if (is_batch(h))
        h->dirty = true;
    BATCH_FORWARD(h, instance, slpic_load_particles(m_, 0, species, n, cell, offset, v));
    int rc = check_handle(h, instance);
    if (rc)
        return rc;
    if (species < 0 || species >= h->ns || n < 0 || (n > 0 && (!cell || !offset || !v)))
        return fail(h, SLPIC_ERR_INVALID, "bad species, count or pointer");
    if (n == 0)
        return SLPIC_OK;
    size_t bc = sizeof(int32_t) * n, bo = sizeof(float) * n, bv = sizeof(float) * 3 * n;
    rc = ensure_stage(h, bc + bo + bv + 64);
    if (rc)
        return rc;
    char *base = (char *)h->d_stage;
    int32_t *dc = (int32_t *)base;
    float *doff = (float *)(base + ((bc + 15) & ~size_t(15)));
    float *dv = (float *)((char *)doff + ((bo + 15) & ~size_t(15)));
    CK(h, cudaMemcpyAsync(dc, cell, bc, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(doff, offset, bo, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(dv, v, bv, cudaMemcpyHostToDevice, h->stream));
    return append_dev(h, species, n, dc, doff, dv);
}

extern "C" int slpic_load_particles_dev(slpic_t *h, int instance, int species, int64_t n,
                                        const int32_t *cell, const float *offset,
                                        const float *v)
{
    if (is_batch(h))
        h->dirty = true;
    BATCH_FORWARD(h, instance, slpic_load_particles_dev(m_, 0, species, n, cell, offset, v));
    int rc = check_handle(h, instance);
    if (rc)
        return rc;
    if (species < 0 || species >= h->ns || n < 0 || (n > 0 && (!cell || !offset || !v)))
        return fail(h, SLPIC_ERR_INVALID, "bad species, count or pointer");
    if (n == 0)
        return SLPIC_OK;
    return append_dev(h, species, n, cell, offset, v);
}

extern "C" int slpic_load_particles_f64(slpic_t *h, int instance, int species, int64_t n,
                                        const double *x, const double *v)
{
    if (is_batch(h))
        h->dirty = true;
    BATCH_FORWARD(h, instance, slpic_load_particles_f64(m_, 0, species, n, x, v));
    int rc = check_handle(h, instance);
    if (rc)
        return rc;
    if (species < 0 || species >= h->ns || n < 0 || (n > 0 && (!x || !v)))
        return fail(h, SLPIC_ERR_INVALID, "bad species, count or pointer");
    std::vector<int32_t> c(n);
    std::vector<float> o(n), vf(3 * n);
    const double L = h->cfg.dx * h->cfg.n_cells;
    for (int64_t i = 0; i < n; ++i) {
        if (!(x[i] >= 0.0 && x[i] < L))
            return fail(h, SLPIC_ERR_INVALID, "x outside [0, L)");
        double xi = x[i] / h->cfg.dx;
        double cf = std::floor(xi);
        int ci = (int)cf;
        float of = (float)(xi - cf);
        if (of >= 1.0f) {
            of = 0.0f;
            ci += 1;
        }
        if (ci >= h->cfg.n_cells) {
            ci = h->cfg.n_cells - 1;
            of = std::nextafter(1.0f, 0.0f);
        }
        c[i] = ci;
        o[i] = of;
        for (int k = 0; k < 3; ++k)
            vf[3 * i + k] = (float)v[3 * i + k];
    }
    return slpic_load_particles(h, instance, species, n, c.data(), o.data(), vf.data());
}

static int batch_prepare(slpic_t *h);
static int batch_step(slpic_t *h, int64_t nsteps);

extern "C" int slpic_prepare(slpic_t *h)
{
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (is_batch(h))
        return batch_prepare(h);
    const int P = (int)(h->step & 1);
    CK(h, cudaMemsetAsync(h->d_acc, 0, sizeof(unsigned long long) * 2 * h->ns * h->nn, h->stream));
    for (int s = 0; s < h->ns; ++s) {
        CK(h, cudaMemsetAsync(&h->d_state->count[s][P ^ 1], 0, sizeof(unsigned long long),
                              h->stream));
        CK(h, cudaMemsetAsync(&h->d_state->holes[s][P ^ 1], 0, sizeof(unsigned long long),
                              h->stream));
    }
    launch_deposit(h->p, h->small_ctas, h->stream);
    CK(h, cudaGetLastError());
    launch_field(h->p, 0, h->stream);
    CK(h, cudaGetLastError());
    h->dirty = false;
    return SLPIC_OK;
}

// Capture the timesteps first_step .. first_step + nsteps - 1 into a graph: an
// in-place particle step, or a compacting one on every compact_every-th step, each
// followed by k_hard and the field kernel.  With `timed`, event-record nodes (4 per
// step, from h->events) bracket the three kernels; every replay re-records them, so
// the events describe the most recent replay.
static int capture(slpic_t *h, long long first_step, int nsteps, bool timed,
                   cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < nsteps; ++k) {
        const bool compact = (first_step + k) % h->compact_every == h->compact_every - 1;
        // "external" records become event-record nodes of the graph (a plain
        // record inside a capture only orders streams)
        if (timed)
            cudaEventRecordWithFlags(h->events[4 * k], h->cap_stream, cudaEventRecordExternal);
        // one SM left free: the TMA kernel holds a whole SM per CTA, so other work
        // on the GPU (the overlapped read-back's potential kernel) would otherwise
        // delay one of its CTAs, and with it the kernel, by that work's length
        if (!compact && h->tma_stages && h->particle_kernel == 0)
            launch_particles_tma(h->p, std::max(1, h->num_sms - 1), h->tma_stages, h->cap_stream);
        else
            launch_particles(h->p, compact ? h->ctas_c : h->ctas, compact, h->cap_stream);
        if (timed)
            cudaEventRecordWithFlags(h->events[4 * k + 1], h->cap_stream, cudaEventRecordExternal);
        launch_hard(h->p, h->hard_ctas, compact, h->cap_stream);
        if (timed)
            cudaEventRecordWithFlags(h->events[4 * k + 2], h->cap_stream, cudaEventRecordExternal);
        launch_field(h->p, compact ? 2 : 1, h->cap_stream);
        if (timed)
            cudaEventRecordWithFlags(h->events[4 * k + 3], h->cap_stream, cudaEventRecordExternal);
    }
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess) {
        h->err = std::string("graph capture: ") + cudaGetErrorString(e);
        return SLPIC_ERR_CUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(h, e);
    return SLPIC_OK;
}

extern "C" int slpic_step(slpic_t *h, int64_t nsteps)
{
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (is_batch(h))
        return batch_step(h, nsteps);
    if (nsteps < 0)
        return fail(h, SLPIC_ERR_INVALID, "nsteps < 0");
    if (h->dirty && (rc = slpic_prepare(h)))
        return rc;
    if (nsteps == 0)
        return SLPIC_OK;
    // graphs: steps whose index is 0 mod compact_every start a cycle
    if (!h->g1 && (rc = capture(h, 0, 1, false, &h->g1)))
        return rc;
    if (!h->gc && (rc = capture(h, h->compact_every - 1, 1, false, &h->gc)))
        return rc;
    int64_t left = nsteps;
    while (left > 0) {
        const long long phase = h->step % h->compact_every;
        if (h->t_len > 0 && left >= h->t_len) {
            if (h->gt && h->t_phase != phase) {
                cudaGraphExecDestroy(h->gt);
                h->gt = nullptr;
            }
            if (!h->gt && (rc = capture(h, phase, (int)h->t_len, true, &h->gt)))
                return rc;
            h->t_phase = phase;
            CK(h, cudaGraphLaunch(h->gt, h->stream));
            h->t_launched++;
            h->step += h->t_len;
            left -= h->t_len;
        } else if (phase == 0 && left >= h->compact_every) {
            if (!h->gK && (rc = capture(h, 0, h->compact_every, false, &h->gK)))
                return rc;
            CK(h, cudaGraphLaunch(h->gK, h->stream));
            h->step += h->compact_every;
            left -= h->compact_every;
        } else {
            CK(h, cudaGraphLaunch(phase == h->compact_every - 1 ? h->gc : h->g1, h->stream));
            h->step += 1;
            left -= 1;
        }
    }
    return SLPIC_OK;
}

extern "C" int slpic_synchronize(slpic_t *h)
{
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (is_batch(h)) {
        CK(h, cudaStreamSynchronize(h->stream));
        for (slpic_t *m : h->members)
            if ((rc = slpic_synchronize(m))) {
                h->err = m->err;
                return rc;
            }
        return SLPIC_OK;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->rb_stream)
        CK(h, cudaStreamSynchronize(h->rb_stream));
    int e = 0;
    CK(h, cudaMemcpy(&e, &h->d_state->error, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        int zero = 0;
        CK(h, cudaMemcpy(&h->d_state->error, &zero, sizeof(int), cudaMemcpyHostToDevice));
        return fail(h, e, e == SLPIC_ERR_CAPACITY  ? "particle store full: injection truncated"
                          : e == SLPIC_ERR_TIMEOUT ? "a bounded wait of the particle kernel ran out"
                                                   : "device error");
    }
    return SLPIC_OK;
}

static int sync_prepared(slpic_t *h, int instance)
{
    int rc = check_handle(h, instance);
    if (rc)
        return rc;
    if (h->dirty && (rc = slpic_prepare(h)))
        return rc;
    return slpic_synchronize(h);
}

extern "C" int slpic_fields(slpic_t *h, int instance, double *rho, double *phi, float *E)
{
    BATCH_FORWARD(h, instance, slpic_fields(m_, 0, rho, phi, E));
    int rc = sync_prepared(h, instance);
    if (rc)
        return rc;
    if (rho || phi) {
        // the step computes E only; rho and phi of the latest deposit on demand
        launch_potential(h->p, h->d_acc + (size_t)(h->step & 1) * h->ns * h->nn, h->step,
                         h->stream);
        CK(h, cudaGetLastError());
        CK(h, cudaStreamSynchronize(h->stream));
    }
    if (rho)
        CK(h, cudaMemcpy(rho, h->d_rho, sizeof(double) * h->nn, cudaMemcpyDeviceToHost));
    if (phi)
        CK(h, cudaMemcpy(phi, h->d_phi, sizeof(double) * h->nn, cudaMemcpyDeviceToHost));
    if (E)
        CK(h, cudaMemcpy(E, h->d_E, sizeof(float) * h->nn, cudaMemcpyDeviceToHost));
    return SLPIC_OK;
}

extern "C" int slpic_fields_async(slpic_t *h, int instance, double *rho, double *phi, float *E)
{
    BATCH_FORWARD(h, instance, slpic_fields_async(m_, 0, rho, phi, E));
    int rc = check_handle(h, instance);
    if (rc)
        return rc;
    if (h->dirty && (rc = slpic_prepare(h)))
        return rc;
    if (!h->rb_stream) {
        CK(h, cudaStreamCreateWithFlags(&h->rb_stream, cudaStreamNonBlocking));
        CK(h, cudaEventCreateWithFlags(&h->ev_snap, cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ev_rb, cudaEventDisableTiming));
        CK(h, cudaMalloc(&h->d_snap_acc, sizeof(unsigned long long) * h->ns * h->nn));
        CK(h, cudaMalloc(&h->d_snap_E, sizeof(float) * h->nn));
    }
    // the previous read-back has finished with the snapshot before it is replaced
    if (h->rb_used)
        CK(h, cudaStreamWaitEvent(h->stream, h->ev_rb, 0));
    launch_snapshot(h->d_acc + (size_t)(h->step & 1) * h->ns * h->nn, h->d_snap_acc,
                    (size_t)h->ns * h->nn, h->d_E, h->d_snap_E, h->nn, h->stream);
    CK(h, cudaGetLastError());
    CK(h, cudaEventRecord(h->ev_snap, h->stream));
    CK(h, cudaStreamWaitEvent(h->rb_stream, h->ev_snap, 0));
    if (rho || phi) {
        launch_potential(h->p, h->d_snap_acc, h->step, h->rb_stream);
        CK(h, cudaGetLastError());
    }
    if (rho)
        CK(h, cudaMemcpyAsync(rho, h->d_rho, sizeof(double) * h->nn, cudaMemcpyDeviceToHost,
                              h->rb_stream));
    if (phi)
        CK(h, cudaMemcpyAsync(phi, h->d_phi, sizeof(double) * h->nn, cudaMemcpyDeviceToHost,
                              h->rb_stream));
    if (E)
        CK(h, cudaMemcpyAsync(E, h->d_snap_E, sizeof(float) * h->nn, cudaMemcpyDeviceToHost,
                              h->rb_stream));
    CK(h, cudaEventRecord(h->ev_rb, h->rb_stream));
    h->rb_used = true;
    return SLPIC_OK;
}

extern "C" int slpic_charge_raw(slpic_t *h, int instance, int species, int64_t *acc)
{
    BATCH_FORWARD(h, instance, slpic_charge_raw(m_, 0, species, acc));
    int rc = sync_prepared(h, instance);
    if (rc)
        return rc;
    if (species < 0 || species >= h->ns || !acc)
        return fail(h, SLPIC_ERR_INVALID, "bad species or pointer");
    const int P = (int)(h->step & 1);
    CK(h, cudaMemcpy(acc, h->d_acc + ((size_t)P * h->ns + species) * h->nn,
                     sizeof(int64_t) * h->nn, cudaMemcpyDeviceToHost));
    return SLPIC_OK;
}

extern "C" int slpic_density(slpic_t *h, int instance, int species, double *n)
{
    BATCH_FORWARD(h, instance, slpic_density(m_, 0, species, n));
    if (!n)
        return h ? fail(h, SLPIC_ERR_INVALID, "n is NULL") : SLPIC_ERR_INVALID;
    std::vector<int64_t> acc(h ? h->nn : 0);
    int rc = slpic_charge_raw(h, instance, species, acc.data());
    if (rc)
        return rc;
    const double f = h->cfg.species[species].w / h->cfg.dx / 1099511627776.0;
    for (int j = 0; j < h->nn; ++j)
        n[j] = (double)acc[j] * f;
    return SLPIC_OK;
}

extern "C" int slpic_particle_count(slpic_t *h, int instance, int species, int64_t *n)
{
    BATCH_FORWARD(h, instance, slpic_particle_count(m_, 0, species, n));
    int rc = sync_prepared(h, instance);
    if (rc)
        return rc;
    if (species < 0 || species >= h->ns || !n)
        return fail(h, SLPIC_ERR_INVALID, "bad species or pointer");
    DevState st;
    if ((rc = read_state(h, &st)))
        return rc;
    const int P = (int)(h->step & 1);
    *n = (int64_t)(st.count[species][P] - st.holes[species][P]);
    return SLPIC_OK;
}

extern "C" int slpic_get_particles(slpic_t *h, int instance, int species, int64_t cap,
                                   int32_t *cell, float *offset, float *v, int64_t *n_out)
{
    BATCH_FORWARD(h, instance, slpic_get_particles(m_, 0, species, cap, cell, offset, v, n_out));
    int64_t n_live = 0;
    int rc = slpic_particle_count(h, instance, species, &n_live);
    if (rc)
        return rc;
    if (cap < 0 || (cap > 0 && (!cell || !offset || !v)))
        return fail(h, SLPIC_ERR_INVALID, "bad cap or pointer");
    if (n_out)
        *n_out = 0;
    DevState st;
    if ((rc = read_state(h, &st)))
        return rc;
    const int P = (int)(h->step & 1);
    const int64_t slots = (int64_t)st.count[species][P];
    if (slots == 0 || cap == 0)
        return SLPIC_OK;
    size_t bc = sizeof(int32_t) * slots, bo = sizeof(float) * slots, bv = sizeof(float) * 3 * slots;
    if ((rc = ensure_stage(h, bc + bo + bv + 64)))
        return rc;
    char *base = (char *)h->d_stage;
    int32_t *dc = (int32_t *)base;
    float *doff = (float *)(base + ((bc + 15) & ~size_t(15)));
    float *dv = (float *)((char *)doff + ((bo + 15) & ~size_t(15)));
    launch_unpack(h->d_cell[species][P], h->d_pv[species][P], slots, dc, doff, dv, h->stream);
    CK(h, cudaGetLastError());
    std::vector<int32_t> hc(slots);
    std::vector<float> ho(slots), hv(3 * slots);
    CK(h, cudaMemcpyAsync(hc.data(), dc, bc, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(ho.data(), doff, bo, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaMemcpyAsync(hv.data(), dv, bv, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    int64_t k = 0;
    for (int64_t i = 0; i < slots && k < cap; ++i) {
        if (hc[i] < 0)
            continue;  // hole left by an absorbed particle
        cell[k] = hc[i];
        offset[k] = ho[i];
        v[3 * k] = hv[3 * i];
        v[3 * k + 1] = hv[3 * i + 1];
        v[3 * k + 2] = hv[3 * i + 2];
        ++k;
    }
    if (n_out)
        *n_out = k;
    return SLPIC_OK;
}

extern "C" int slpic_diagnostics(slpic_t *h, int instance, slpic_diag *out)
{
    BATCH_FORWARD(h, instance, slpic_diagnostics(m_, 0, out));
    int rc = sync_prepared(h, instance);
    if (rc)
        return rc;
    if (!out)
        return fail(h, SLPIC_ERR_INVALID, "out is NULL");
    std::memset(out, 0, sizeof(*out));
    CK(h, cudaMemsetAsync(h->d_diag, 0, sizeof(double) * 2 * kMaxSpecies, h->stream));
    launch_diag(h->p, h->d_diag, h->small_ctas, h->stream);
    CK(h, cudaGetLastError());
    double red[2 * kMaxSpecies];
    CK(h, cudaMemcpyAsync(red, h->d_diag, sizeof(red), cudaMemcpyDeviceToHost, h->stream));
    DevState st;
    if ((rc = read_state(h, &st)))
        return rc;
    std::vector<double> E(h->nn);
    CK(h, cudaMemcpy(E.data(), h->d_E64, sizeof(double) * h->nn, cudaMemcpyDeviceToHost));
    const int P = (int)(h->step & 1);
    out->step = st.step;
    out->time = (double)st.step * h->cfg.dt;
    for (int s = 0; s < h->ns; ++s) {
        const slpic_species &sp = h->cfg.species[s];
        const int64_t live = (int64_t)(st.count[s][P] - st.holes[s][P]);
        out->count[s] = live;
        out->sum_w[s] = sp.w * (double)live;
        out->sum_wbeta[s] = sp.w * red[2 * s];
        out->kinetic[s] = 0.5 * sp.m * sp.w * red[2 * s + 1];
        out->absorbed[s][0] = st.absorbed_total[s][0];
        out->absorbed[s][1] = st.absorbed_total[s][1];
        out->injected[s] = st.injected_total[s];
        out->iterative[s] = st.iterative_total[s];
    }
    double fe = 0.0;
    for (int j = 0; j < h->nn; ++j) {
        double wgt = (!h->p.periodic && (j == 0 || j == h->nn - 1)) ? 0.5 : 1.0;
        fe += wgt * E[j] * E[j];
    }
    out->field_energy = 0.5 * h->cfg.eps0 * h->cfg.dx * fe;
    return SLPIC_OK;
}

// ---- checkpoint -------------------------------------------------------------------
namespace {
struct SaveHeader {
    char magic[8];
    int32_t version, ns, nn, pad;
    int64_t step;
    int64_t count[kMaxSpecies];
};
}  // namespace

extern "C" int slpic_save(slpic_t *h, void *buf, size_t *size)
{
    if (is_batch(h))
        return fail(h, SLPIC_ERR_INVALID, "not available for a batch handle");
    int rc = sync_prepared(h, 0);
    if (rc)
        return rc;
    if (!size)
        return fail(h, SLPIC_ERR_INVALID, "size is NULL");
    DevState st;
    if ((rc = read_state(h, &st)))
        return rc;
    const int P = (int)(h->step & 1);
    size_t need = sizeof(SaveHeader) + sizeof(DevState) +
                  sizeof(unsigned long long) * 2 * h->ns * h->nn + sizeof(float) * h->nn +
                  3 * sizeof(double) * h->nn;
    for (int s = 0; s < h->ns; ++s)
        need += st.count[s][P] * (sizeof(int32_t) + sizeof(float4));
    if (!buf) {
        *size = need;
        return SLPIC_OK;
    }
    if (*size < need)
        return fail(h, SLPIC_ERR_INVALID, "buffer too small");
    char *o = (char *)buf;
    SaveHeader hd{};
    std::memcpy(hd.magic, "SLPIC1D", 8);
    hd.version = 2;
    hd.ns = h->ns;
    hd.nn = h->nn;
    hd.step = h->step;
    for (int s = 0; s < h->ns; ++s)
        hd.count[s] = (int64_t)st.count[s][P];
    std::memcpy(o, &hd, sizeof(hd));
    o += sizeof(hd);
    std::memcpy(o, &st, sizeof(st));
    o += sizeof(st);
    auto d2h = [&](const void *src, size_t b) -> int {
        CK(h, cudaMemcpy(o, src, b, cudaMemcpyDeviceToHost));
        o += b;
        return SLPIC_OK;
    };
    if ((rc = d2h(h->d_acc, sizeof(unsigned long long) * 2 * h->ns * h->nn)) ||
        (rc = d2h(h->d_E, sizeof(float) * h->nn)) || (rc = d2h(h->d_E64, sizeof(double) * h->nn)) ||
        (rc = d2h(h->d_phi, sizeof(double) * h->nn)) || (rc = d2h(h->d_rho, sizeof(double) * h->nn)))
        return rc;
    for (int s = 0; s < h->ns; ++s) {
        size_t n = st.count[s][P];
        if ((rc = d2h(h->d_cell[s][P], sizeof(int32_t) * n)) ||
            (rc = d2h(h->d_pv[s][P], sizeof(float4) * n)))
            return rc;
    }
    *size = need;
    return SLPIC_OK;
}

extern "C" int slpic_restore(slpic_t *h, const void *buf, size_t size)
{
    if (is_batch(h))
        return fail(h, SLPIC_ERR_INVALID, "not available for a batch handle");
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (!buf || size < sizeof(SaveHeader) + sizeof(DevState))
        return fail(h, SLPIC_ERR_INVALID, "buffer too small");
    const char *i = (const char *)buf;
    SaveHeader hd;
    std::memcpy(&hd, i, sizeof(hd));
    i += sizeof(hd);
    if (std::memcmp(hd.magic, "SLPIC1D", 8) != 0 || hd.version != 2 || hd.ns != h->ns ||
        hd.nn != h->nn)
        return fail(h, SLPIC_ERR_INVALID, "checkpoint does not match this configuration");
    for (int s = 0; s < h->ns; ++s)
        if (hd.count[s] > h->cfg.species[s].capacity)
            return fail(h, SLPIC_ERR_CAPACITY, "checkpoint exceeds the species capacity");
    CK(h, cudaStreamSynchronize(h->stream));
    DevState st;
    std::memcpy(&st, i, sizeof(st));
    i += sizeof(st);
    const int P = (int)(hd.step & 1);
    auto h2d = [&](void *dst, size_t b) -> int {
        CK(h, cudaMemcpy(dst, i, b, cudaMemcpyHostToDevice));
        i += b;
        return SLPIC_OK;
    };
    CK(h, cudaMemcpy(h->d_state, &st, sizeof(st), cudaMemcpyHostToDevice));
    if ((rc = h2d(h->d_acc, sizeof(unsigned long long) * 2 * h->ns * h->nn)) ||
        (rc = h2d(h->d_E, sizeof(float) * h->nn)) || (rc = h2d(h->d_E64, sizeof(double) * h->nn)) ||
        (rc = h2d(h->d_phi, sizeof(double) * h->nn)) || (rc = h2d(h->d_rho, sizeof(double) * h->nn)))
        return rc;
    for (int s = 0; s < h->ns; ++s) {
        size_t n = (size_t)hd.count[s];
        if ((rc = h2d(h->d_cell[s][P], sizeof(int32_t) * n)) ||
            (rc = h2d(h->d_pv[s][P], sizeof(float4) * n)))
            return rc;
    }
    h->step = hd.step;
    h->dirty = false;
    return SLPIC_OK;
}

// ---- timing ----------------------------------------------------------------------
extern "C" int slpic_enable_kernel_timing(slpic_t *h, int64_t steps_per_graph)
{
    if (is_batch(h))
        return fail(h, SLPIC_ERR_INVALID, "not available for a batch handle");
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (steps_per_graph < 0 || steps_per_graph > 4096)
        return fail(h, SLPIC_ERR_INVALID, "steps_per_graph must be in 0..4096");
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->gt) {
        cudaGraphExecDestroy(h->gt);
        h->gt = nullptr;
    }
    for (cudaEvent_t e : h->events)
        cudaEventDestroy(e);
    h->events.clear();
    h->t_launched = 0;
    h->t_phase = -1;
    h->t_len = steps_per_graph;
    h->events.resize(4 * steps_per_graph);
    for (auto &e : h->events)
        CK(h, cudaEventCreate(&e));
    return SLPIC_OK;
}

extern "C" int slpic_kernel_times(slpic_t *h, double *particle_ms, double *hard_ms,
                                  double *field_ms, int64_t *steps)
{
    if (is_batch(h))
        return fail(h, SLPIC_ERR_INVALID, "not available for a batch handle");
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    double a = 0.0, b = 0.0, c = 0.0;
    long long n = h->t_launched > 0 ? h->t_len : 0;
    for (long long k = 0; k < n; ++k) {
        float x = 0.f, y = 0.f, z = 0.f;
        CK(h, cudaEventElapsedTime(&x, h->events[4 * k], h->events[4 * k + 1]));
        CK(h, cudaEventElapsedTime(&y, h->events[4 * k + 1], h->events[4 * k + 2]));
        CK(h, cudaEventElapsedTime(&z, h->events[4 * k + 2], h->events[4 * k + 3]));
        a += x;
        b += y;
        c += z;
    }
    if (particle_ms)
        *particle_ms = n ? a / n : 0.0;
    if (hard_ms)
        *hard_ms = n ? b / n : 0.0;
    if (field_ms)
        *field_ms = n ? c / n : 0.0;
    if (steps)
        *steps = n;
    return SLPIC_OK;
}

static void drop_graphs(slpic_t *h);

extern "C" int slpic_set_wait_limit(slpic_t *h, int64_t cycles)
{
    if (is_batch(h))
        return fail(h, SLPIC_ERR_INVALID, "not available for a batch handle");
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (cycles < 0)
        return fail(h, SLPIC_ERR_INVALID, "cycles < 0");
    CK(h, cudaStreamSynchronize(h->stream));
    h->p.wait_cycles = cycles ? (long long)cycles : kWaitCycles;
    drop_graphs(h);
    return SLPIC_OK;
}

extern "C" int slpic_kernel_spans(slpic_t *h, double *ms, int64_t *launches)
{
    if (is_batch(h))
        return fail(h, SLPIC_ERR_INVALID, "not available for a batch handle");
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    DevState st;
    if ((rc = read_state(h, &st)))
        return rc;
    for (int k = 0; k < 3; ++k) {
        if (ms)
            ms[k] = 1e-6 * (double)st.span_ns[k];
        if (launches)
            launches[k] = (int64_t)st.span_launches[k];
    }
    return SLPIC_OK;
}

extern "C" int slpic_kernels_per_step(slpic_t *h, int *n)
{
    if (!h || !n)
        return SLPIC_ERR_INVALID;
    *n = 3;
    return SLPIC_OK;
}

// The step graphs hold the parameters by value: drop them so that the next step
// captures them again.
static void drop_graphs(slpic_t *h)
{
    for (cudaGraphExec_t *g : {&h->g1, &h->gc, &h->gK, &h->gt})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
}

// A batch keeps its members' parameters on the device as well.
static int batch_refresh_params(slpic_t *h)
{
    std::vector<StepParams> ps;
    for (slpic_t *m : h->members)
        ps.push_back(m->p);
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(h->d_params, ps.data(), sizeof(StepParams) * ps.size(),
                     cudaMemcpyHostToDevice));
    drop_graphs(h);
    return SLPIC_OK;
}

extern "C" int slpic_set_speed_limit(slpic_t *h, int instance, int species, double v0)
{
    if (is_batch(h)) {
        if (instance < 0 || instance >= (int)h->members.size())
            return fail(h, SLPIC_ERR_INVALID, "instance out of range");
        slpic_t *m = h->members[instance];
        int rc = slpic_set_speed_limit(m, 0, species, v0);
        if (rc) {
            h->err = m->err;
            return rc;
        }
        return batch_refresh_params(h);
    }
    int rc = check_handle(h, instance);
    if (rc)
        return rc;
    if (species < 0 || species >= h->ns)
        return fail(h, SLPIC_ERR_INVALID, "species out of range");
    const slpic_species &sp = h->cfg.species[species];
    if (sp.beta_kind == SLPIC_BETA_ONE)
        return fail(h, SLPIC_ERR_INVALID, "species has no speed limit (beta == 1)");
    if (!(v0 > 0) || !std::isfinite(v0))
        return fail(h, SLPIC_ERR_INVALID, "v0 must be > 0");
    if (h->cfg.dt * v0 * h->lam_max > h->cfg.dx)
        return fail(h, SLPIC_ERR_CFL, "dt * v0 * (largest profile factor) > dx: lower the timestep first");
    CK(h, cudaStreamSynchronize(h->stream));
    h->cfg.species[species].v0 = v0;
    h->p.sp[species].v0 = (float)v0;
    drop_graphs(h);
    return SLPIC_OK;
}

extern "C" int slpic_set_speed_limit_profile(slpic_t *h, const double *lambda, int n_cells)
{
    if (is_batch(h))
        return fail(h, SLPIC_ERR_INVALID, "not available for a batch handle");
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (!lambda) {
        CK(h, cudaStreamSynchronize(h->stream));
        h->p.lam = nullptr;
        h->lam_max = 1.0;
        drop_graphs(h);
        return SLPIC_OK;
    }
    if (n_cells != h->cfg.n_cells)
        return fail(h, SLPIC_ERR_INVALID, "the profile needs one factor per cell");
    std::vector<float> lam32(n_cells);
    double mx = 0.0;
    for (int c = 0; c < n_cells; ++c) {
        lam32[c] = (float)lambda[c];
        if (!(lambda[c] > 0) || !std::isfinite(lambda[c]) || !(lam32[c] > 0.0f) ||
            !std::isfinite(lam32[c]))
            return fail(h, SLPIC_ERR_INVALID, "profile factors must be finite and > 0 in FP32");
        mx = std::max(mx, (double)lam32[c]);
    }
    for (int s = 0; s < h->ns; ++s) {
        const slpic_species &sp = h->cfg.species[s];
        if (sp.beta_kind != SLPIC_BETA_ONE && h->cfg.dt * sp.v0 * mx > h->cfg.dx)
            return fail(h, SLPIC_ERR_CFL, "dt * v0 * (largest factor) > dx for species " +
                                              std::to_string(s));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (!h->d_lam)
        CK(h, cudaMalloc(&h->d_lam, sizeof(float) * n_cells));
    CK(h, cudaMemcpy(h->d_lam, lam32.data(), sizeof(float) * n_cells, cudaMemcpyHostToDevice));
    h->p.lam = h->d_lam;
    h->lam_max = mx;
    drop_graphs(h);
    return SLPIC_OK;
}

extern "C" int slpic_set_wave(slpic_t *h, double phi0, double k, double vphi, double t_ramp)
{
    if (is_batch(h))
        return fail(h, SLPIC_ERR_INVALID, "not available for a batch handle");
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (h->cfg.bc != SLPIC_BC_PERIODIC)
        return fail(h, SLPIC_ERR_INVALID, "the prescribed wave needs a periodic grid");
    if (!std::isfinite(phi0) || !std::isfinite(k) || !std::isfinite(vphi) || !(t_ramp >= 0) ||
        !std::isfinite(t_ramp) || k < 0)
        return fail(h, SLPIC_ERR_INVALID, "bad wave parameters");
    if (h->dirty && (rc = slpic_prepare(h)))
        return rc;
    CK(h, cudaStreamSynchronize(h->stream));
    StepParams &p = h->p;
    p.wave_on = k > 0.0;
    p.wave_phi0 = phi0;
    p.wave_k = k;
    p.wave_vphi = vphi;
    p.wave_ramp = t_ramp;
    drop_graphs(h);
    // E of the current time level from the new setting (no deposit is consumed)
    launch_field(h->p, 0, h->stream);
    CK(h, cudaGetLastError());
    return SLPIC_OK;
}

extern "C" int slpic_set_timestep(slpic_t *h, double dt)
{
    if (is_batch(h))
        return fail(h, SLPIC_ERR_INVALID, "set the timestep of each instance before batching");
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (!(dt > 0) || !std::isfinite(dt))
        return fail(h, SLPIC_ERR_INVALID, "dt must be > 0");
    for (int s = 0; s < h->ns; ++s) {
        const slpic_species &sp = h->cfg.species[s];
        if (sp.beta_kind != SLPIC_BETA_ONE && dt * sp.v0 * h->lam_max > h->cfg.dx)
            return fail(h, SLPIC_ERR_CFL, "dt * v0 > dx for species " + std::to_string(s) +
                                              " (v0 times the largest profile factor)");
        if (sp.beta_kind == SLPIC_BETA_ONE && h->cfg.max_speed > 0 &&
            dt * h->cfg.max_speed > h->cfg.dx)
            return fail(h, SLPIC_ERR_CFL, "dt * max_speed > dx");
    }
    CK(h, cudaStreamSynchronize(h->stream));
    const double old = h->cfg.dt;
    h->cfg.dt = dt;
    StepParams &p = h->p;
    p.dt = (float)dt;
    p.dt_dx = (float)(dt / h->cfg.dx);
    p.dt64 = dt;
    for (int s = 0; s < h->ns; ++s)
        p.sp[s].wall_rate *= dt / old;  // the wall source's macroparticles per step
    drop_graphs(h);
    return SLPIC_OK;
}

// =================================================================================
// Batches of independent simulations (many sheaths of uneven size advanced together)
// =================================================================================

extern "C" int slpic_create_batch(const slpic_config *cfgs, int m, slpic_t **out)
{
    g_create_err.clear();
    if (!cfgs || !out || m < 1) {
        g_create_err = "need cfgs, out and m >= 1";
        return SLPIC_ERR_INVALID;
    }
    std::vector<slpic_t *> members;
    for (int i = 0; i < m; ++i) {
        slpic_t *mh = nullptr;
        const int rc = slpic_create(&cfgs[i], &mh);
        if (rc) {
            const std::string why = "instance " + std::to_string(i) + ": " + g_create_err;
            for (slpic_t *x : members)
                slpic_destroy(x);
            g_create_err = why;
            return rc;
        }
        members.push_back(mh);
    }
    slpic_t *h = new slpic_sim();
    h->cfg = cfgs[0];
    h->device = members[0]->device;
    h->num_sms = members[0]->num_sms;
    h->members = members;
    for (slpic_t *x : members) {
        h->max_nn = std::max(h->max_nn, x->nn);
        h->max_ns = std::max(h->max_ns, x->ns);
    }
    auto bail = [&](int code, const std::string &msg) {
        g_create_err = msg;
        slpic_destroy(h);
        return code;
    };
    if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return bail(SLPIC_ERR_CUDA, "stream creation failed");
    h->stream = h->own_stream;
    for (slpic_t *x : members)
        x->stream = h->stream;
    if (cudaMalloc(&h->d_params, sizeof(StepParams) * m) != cudaSuccess)
        return bail(SLPIC_ERR_OOM, "device allocation failed");
    int occ = 0, occ_c = 0;
    if (configure_batch_kernels(h->max_nn, &occ, &occ_c) != cudaSuccess || occ < 1 || occ_c < 1)
        return bail(SLPIC_ERR_INVALID, "batched particle kernel cannot be resident");
    h->ctas = occ;     // resident batched CTAs per SM (work-table sizing)
    h->ctas_c = occ_c;
    // the iterative-push kernel: the single simulation's whole-GPU grid, shared out
    h->batch_hard_ctas = std::max(4, h->num_sms * 8 / m);
    *out = h;
    return SLPIC_OK;
}

// Work items of the batched particle kernels: every (instance, species) gets CTAs
// in proportion to its particles (at least one), about `waves` full waves of the GPU.
static int batch_tables(slpic_t *h)
{
    std::vector<long long> n;
    long long total = 0;
    for (slpic_t *m : h->members) {
        DevState st;
        int rc = read_state(m, &st);
        if (rc) {
            h->err = m->err;
            return rc;
        }
        const int P = (int)(m->step & 1);
        for (int s = 0; s < m->ns; ++s) {
            n.push_back((long long)st.count[s][P]);
            total += (long long)st.count[s][P];
        }
    }
    const int waves = h->batch_waves;
    const long long budget = (long long)h->num_sms * std::min(h->ctas, h->ctas_c) * waves;
    std::vector<int4> work;
    size_t k = 0;
    for (int i = 0; i < (int)h->members.size(); ++i) {
        for (int s = 0; s < h->members[i]->ns; ++s, ++k) {
            long long c = total > 0 ? (n[k] * budget + total - 1) / total : 1;
            // a share large enough to amortise the per-CTA grid staging
            const long long per = std::max(1LL, n[k] / h->batch_min_share);
            c = std::max(1LL, std::min(c, per));
            for (int j = 0; j < (int)c; ++j)
                work.push_back(make_int4(i, s, j, (int)c));
        }
    }
    cudaFree(h->d_work);
    h->d_work = nullptr;
    CK(h, cudaMalloc(&h->d_work, sizeof(int4) * work.size()));
    CK(h, cudaMemcpy(h->d_work, work.data(), sizeof(int4) * work.size(), cudaMemcpyHostToDevice));
    h->n_work = (int)work.size();
    return SLPIC_OK;
}

static int batch_prepare(slpic_t *h)
{
    int rc;
    for (slpic_t *m : h->members) {
        if ((rc = slpic_prepare(m))) {
            h->err = m->err;
            return rc;
        }
    }
    std::vector<StepParams> ps;
    for (slpic_t *m : h->members)
        ps.push_back(m->p);
    CK(h, cudaMemcpyAsync(h->d_params, ps.data(), sizeof(StepParams) * ps.size(),
                          cudaMemcpyHostToDevice, h->stream));
    if ((rc = batch_tables(h)))
        return rc;
    // work items changed: the graphs are captured again on the next step
    for (cudaGraphExec_t *g : {&h->g1, &h->gc, &h->gK})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
    h->dirty = false;
    return SLPIC_OK;
}

static int batch_capture(slpic_t *h, long long first_step, int nsteps, cudaGraphExec_t *out)
{
    const int m = (int)h->members.size();
    cudaGraph_t g = nullptr;
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < nsteps; ++k) {
        const bool compact = (first_step + k) % h->compact_every == h->compact_every - 1;
        launch_particles_batch(h->d_params, h->d_work, h->n_work, h->max_nn, compact,
                               h->cap_stream);
        launch_hard_batch(h->d_params, m, h->batch_hard_ctas, compact, h->cap_stream);
        launch_field_batch(h->d_params, m, h->max_nn, h->max_ns, compact ? 2 : 1, h->cap_stream);
    }
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    if (e != cudaSuccess) {
        h->err = std::string("graph capture: ") + cudaGetErrorString(e);
        return SLPIC_ERR_CUDA;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    CK(h, e);
    return SLPIC_OK;
}

static int batch_step(slpic_t *h, int64_t nsteps)
{
    int rc;
    if (nsteps < 0)
        return fail(h, SLPIC_ERR_INVALID, "nsteps < 0");
    if (h->dirty && (rc = batch_prepare(h)))
        return rc;
    if (nsteps == 0)
        return SLPIC_OK;
    if (!h->g1 && (rc = batch_capture(h, 0, 1, &h->g1)))
        return rc;
    if (!h->gc && (rc = batch_capture(h, h->compact_every - 1, 1, &h->gc)))
        return rc;
    int64_t left = nsteps;
    while (left > 0) {
        const long long phase = h->step % h->compact_every;
        int64_t adv = 1;
        if (phase == 0 && left >= h->compact_every) {
            if (!h->gK && (rc = batch_capture(h, 0, h->compact_every, &h->gK)))
                return rc;
            CK(h, cudaGraphLaunch(h->gK, h->stream));
            adv = h->compact_every;
        } else {
            CK(h, cudaGraphLaunch(phase == h->compact_every - 1 ? h->gc : h->g1, h->stream));
        }
        h->step += adv;
        for (slpic_t *m : h->members)
            m->step += adv;
        left -= adv;
    }
    return SLPIC_OK;
}

// ---- performance settings and the autotuner -----------------------------------------
// Neither the compaction interval, the particle kernel nor a batch's work split
// changes a result: the source draws its random numbers by (seed, step, species,
// particle index), the deposit is an integer sum, and the field solve follows from
// the deposit, so only the slots the particles occupy differ.
static int tuning_valid(const slpic_tuning *t)
{
    return t && t->compact_every >= 2 && t->compact_every <= 1024 &&
           (t->particle_kernel == 0 || t->particle_kernel == 1) && t->batch_waves >= 1 &&
           t->batch_waves <= 16 && t->batch_min_share >= 256 && t->batch_min_share <= (1 << 20);
}

extern "C" int slpic_get_tuning(slpic_t *h, slpic_tuning *out)
{
    if (!h || !out)
        return SLPIC_ERR_INVALID;
    out->compact_every = h->compact_every;
    out->particle_kernel = h->particle_kernel;
    out->batch_waves = h->batch_waves;
    out->batch_min_share = h->batch_min_share;
    return SLPIC_OK;
}

extern "C" int slpic_set_tuning(slpic_t *h, const slpic_tuning *t)
{
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (!tuning_valid(t))
        return fail(h, SLPIC_ERR_INVALID, "tuning out of range");
    CK(h, cudaStreamSynchronize(h->stream));
    const bool split = is_batch(h) && (t->batch_waves != h->batch_waves ||
                                       t->batch_min_share != h->batch_min_share);
    h->compact_every = t->compact_every;
    h->particle_kernel = t->particle_kernel;
    h->batch_waves = t->batch_waves;
    h->batch_min_share = t->batch_min_share;
    drop_graphs(h);
    if (split && !h->dirty && (rc = batch_tables(h)))
        return rc;
    return SLPIC_OK;
}

// The smallest (free slots) / (slots one step may add) over instances and species:
// a step adds the source's particles (twice the mean rate so far, plus a margin),
// and holes stay until the next compacting step, so an interval of `every` steps
// is safe while this is well above `every`.
// Per member and species, the injected total and step index at a point of the run, so
// that the rate of the steps since then can be taken (slots_headroom).
struct InjectionMark {
    std::vector<std::vector<long long>> injected;  // [member][species]
    std::vector<long long> step;                   // [member]
};

static int mark_injection(slpic_t *h, InjectionMark *mk)
{
    std::vector<slpic_t *> sims = is_batch(h) ? h->members : std::vector<slpic_t *>{h};
    mk->injected.assign(sims.size(), {});
    mk->step.assign(sims.size(), 0);
    for (size_t i = 0; i < sims.size(); ++i) {
        DevState a;
        int rc = read_state(sims[i], &a);
        if (rc)
            return rc;
        mk->step[i] = sims[i]->step;
        for (int s = 0; s < sims[i]->ns; ++s)
            mk->injected[i].push_back(a.injected_total[s]);
    }
    return SLPIC_OK;
}

// How many steps of source injection the slots left free can take, at the worst of each
// species' mean rate since the start and its rate since `mk` (a sheath's losses, and so
// a loss-matched source, can still be growing), over every member: an interval of v
// in-place steps between compactions leaves holes of up to v steps' worth of particles.
static int slots_headroom(slpic_t *h, const InjectionMark &mk, long long *ratio)
{
    std::vector<slpic_t *> sims = is_batch(h) ? h->members : std::vector<slpic_t *>{h};
    long long best = 1LL << 40;
    for (size_t i = 0; i < sims.size(); ++i) {
        slpic_t *m = sims[i];
        DevState a;
        int rc = read_state(m, &a);
        if (rc)
            return rc;
        const int P = (int)(m->step & 1);
        for (int s = 0; s < m->ns; ++s) {
            const long long used = (long long)a.count[s][P];
            const long long cap = m->cfg.species[s].capacity;
            long long inj = m->step > 0 ? a.injected_total[s] / std::max(1LL, m->step) : 0;
            const long long dn = m->step - mk.step[i];
            if (dn > 0 && s < (int)mk.injected[i].size())
                inj = std::max(inj, (a.injected_total[s] - mk.injected[i][s] + dn - 1) / dn);
            best = std::min(best, (cap - used) / (2 * inj + 64));
        }
    }
    *ratio = best;
    return SLPIC_OK;
}

static int time_steps(slpic_t *h, long long n, double *ms_per_step)
{
    cudaEvent_t a, b;
    CK(h, cudaEventCreate(&a));
    CK(h, cudaEventCreate(&b));
    cudaEventRecord(a, h->stream);
    int rc = slpic_step(h, n);
    cudaEventRecord(b, h->stream);
    if (rc == SLPIC_OK) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(b);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess)
            rc = fail(h, SLPIC_ERR_CUDA, cudaGetErrorString(e));
        *ms_per_step = ms / (double)n;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return rc == SLPIC_OK ? slpic_synchronize(h) : rc;
}

extern "C" int slpic_autotune(slpic_t *h, int32_t steps_per_trial, slpic_tuning *chosen,
                              double *ms_per_step)
{
    int rc = check_handle(h, 0);
    if (rc)
        return rc;
    if (steps_per_trial < 1 || steps_per_trial > 100000)
        return fail(h, SLPIC_ERR_INVALID, "steps_per_trial must be in 1..100000");
    if ((rc = slpic_step(h, 0)) || (rc = slpic_synchronize(h)))
        return rc;
    // one trial: the settings, steps up to a cycle boundary plus one cycle (the
    // graphs are captured there), then whole cycles timed with events
    auto trial = [&](const slpic_tuning &t, double *ms) -> int {
        int r = slpic_set_tuning(h, &t);
        if (r)
            return r;
        const long long cyc = t.compact_every;
        if ((r = slpic_step(h, cyc + (cyc - h->step % cyc) % cyc)))
            return r;
        return time_steps(h, (steps_per_trial + cyc - 1) / cyc * cyc, ms);
    };
    slpic_tuning best{};
    slpic_get_tuning(h, &best);
    double best_ms = 0.0;
    InjectionMark mark;
    if ((rc = mark_injection(h, &mark)) || (rc = trial(best, &best_ms)))
        return rc;
    // coordinate search: each setting in turn over its candidates, the others held
    // at their best so far
    enum { kEvery, kKernel, kWaves, kShare };
    std::vector<int> order = {kEvery};
    if (is_batch(h)) {
        order.push_back(kWaves);
        order.push_back(kShare);
    } else if (h->tma_stages) {
        order.push_back(kKernel);
    }
    for (int which : order) {
        const slpic_tuning base = best;
        std::vector<slpic_tuning> cands;
        const std::vector<int> vals =
            which == kEvery ? std::vector<int>{8, 16, 32, 64}
            : which == kKernel ? std::vector<int>{0, 1}
            : which == kWaves  ? std::vector<int>{1, 2, 4, 8}
                               : std::vector<int>{1024, 4096, 16384, 65536};
        for (int v : vals) {
            slpic_tuning t = base;
            (which == kEvery ? t.compact_every : which == kKernel ? t.particle_kernel
                             : which == kWaves ? t.batch_waves : t.batch_min_share) = v;
            if (memcmp(&t, &base, sizeof t) == 0)
                continue;  // measured already
            if (which == kEvery) {
                long long ratio = 0;
                if ((rc = slots_headroom(h, mark, &ratio)))
                    return rc;
                if (ratio < 4LL * v)
                    continue;  // its holes might not fit: never risk a truncated source
            }
            double ms = 0.0;
            if ((rc = trial(t, &ms)))
                return rc;
            if (ms < best_ms) {
                best_ms = ms;
                best = t;
            }
        }
    }
    if ((rc = slpic_set_tuning(h, &best)))
        return rc;
    if (chosen)
        *chosen = best;
    if (ms_per_step)
        *ms_per_step = best_ms;
    return SLPIC_OK;
}
