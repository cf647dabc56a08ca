// usp_api.cu -- host side of the C ABI declared in include/usp.h: parameter
// derivation (Eqs. 35-37), device memory, the step sequence captured into a
// CUDA graph, debug access and batching.
#include "usp.h"
#include "usp_internal.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace usp;

namespace {

struct Graphs {
    cudaGraphExec_t one = nullptr;    // one step
    cudaGraphExec_t many = nullptr;   // kGraphSteps steps
};
constexpr int kGraphSteps = 8;

void destroy_graphs(Graphs& g) {
    if (g.one) cudaGraphExecDestroy(g.one);
    if (g.many) cudaGraphExecDestroy(g.many);
    g.one = g.many = nullptr;
}

int persistent_grid(int ntiles, int per_sm) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int g = sms * per_sm;
    if (ntiles < g) g = ntiles > 0 ? ntiles : 1;
    return g;
}

}  // namespace

// a second stream and two events for the forked part of a fused step
struct Fork {
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool make() {
        if (side) return true;
        if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            release();
            return false;
        }
        return true;
    }
    void release() {
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
        side = nullptr;
        ev_fork = ev_join = nullptr;
    }
    void attach(Launch& L) const {
        L.side = side;
        L.ev_fork = ev_fork;
        L.ev_join = ev_join;
    }
};

struct usp_handle {
    SimDev host{};            // host copy of the simulation description
    SimDev* d_sim = nullptr;  // device copy
    SimDyn* d_dyn = nullptr;
    int precision = USP_FP64;
    int pipeline = USP_PIPE_PLAIN;
    double capacity_factor = 0;
    double n_ref = 0;                 // reference number density and particles per cell,
    int ppc_ref = 1;                  // for the initial particle counts
    int slab_group = 0;               // spatial decomposition group (0: none)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    usp_allocator alloc{};
    bool has_alloc = false;
    bool misaligned_alloc = false;    // the last allocator call was rejected for its alignment
    std::vector<void*> cell_allocs;   // per-cell arrays (lifetime of the handle)
    std::vector<void*> part_allocs;   // particle storage (replaced on re-init)
    size_t cell_bytes = 0, part_bytes = 0;
    int2* d_ptiles = nullptr;
    int2* d_ctiles = nullptr;
    int* d_ntiles = nullptr;          // [0] particle tiles, [1] cell tiles, [2..3] k_g2 work queue
    int nptiles = 0, nctiles = 0;
    Graphs graphs;
    bool initialised = false;
    bool mid_step = false;            // data in buffer cur^1 (after the sort stage)
    bool sorted = false;              // storage order is by cell with valid start[]
    std::string err;
    std::vector<uint32_t> inj_count_host;
    int batch_refs = 0;
    int fused_R = 8;                  // k_g2 consumer warps per CTA: 3, 7, 15 for R = 4, 8, 12
    int grid_per_sm = 8;              // persistent blocks per SM of the tiled kernels
    cudaStream_t batch_stream = nullptr;   // stream of the batch the handle is admitted to
    void* b1_block = nullptr;         // buffer 1 and the cell plane (one allocation)
    size_t b1_bytes = 0;
    cudaEvent_t upload_ev = nullptr;  // usp_set_particles: the caller's arrays have been read
    Fork fork;                        // fused steps: layout beside the moments and parameters
};

struct usp_batch {
    size_t budget = 0;
    int max_sims = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<usp_handle*> members;
    SimDev* d_sims = nullptr;
    int2* d_ptiles = nullptr;
    int2* d_ctiles = nullptr;
    int* d_ntiles = nullptr;
    size_t ptile_cap = 0, ctile_cap = 0;
    int nptiles = 0, nctiles = 0;
    Graphs graphs;
    int graph_nsims = -1;             // nsims the graphs were captured with
    int lay_tiles = 1;                // layout tiles of the largest member seen (grid of the layout kernels)
    bool dirty = true;
    int precision = -1, pipeline = -1;
    std::string err;
    Fork fork;
};

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
static int fail(usp_handle* h, int code, const std::string& msg) {
    if (h) {
        h->err = msg;
        if (h->misaligned_alloc) h->err += " (the allocator returned memory not aligned to 256 bytes)";
        h->misaligned_alloc = false;
    }
    return code;
}

#define CK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return fail(h, USP_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

static void* dalloc(usp_handle* h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (h->has_alloc) {
        p = h->alloc.alloc(bytes, h->alloc.ctx);
        if (p && ((uintptr_t)p & 255u) != 0) {   // the bulk copies need 16-byte aligned planes
            h->alloc.free(p, h->alloc.ctx);
            h->misaligned_alloc = true;
            p = nullptr;
        }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}

static void dfree(usp_handle* h, void* p) {
    if (!p) return;
    if (h->has_alloc) h->alloc.free(p, h->alloc.ctx);
    else cudaFree(p);
}

static int cell_alloc(usp_handle* h, size_t bytes, void** out) {
    void* p = dalloc(h, bytes);
    if (!p) return fail(h, USP_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    h->cell_allocs.push_back(p);
    h->cell_bytes += bytes;
    *out = p;
    return USP_OK;
}

static void free_particles(usp_handle* h) {
    for (void* p : h->part_allocs) dfree(h, p);
    h->part_allocs.clear();
    h->part_bytes = 0;
    h->b1_block = nullptr;
    h->b1_bytes = 0;
}

static int upload_sim(usp_handle* h) {
    CK(cudaMemcpyAsync(h->d_sim, &h->host, sizeof(SimDev), cudaMemcpyHostToDevice, h->stream));
    return USP_OK;
}

static Launch make_launch(usp_handle* h) {
    Launch L;
    L.sims = h->d_sim;
    L.ptiles = h->d_ptiles;
    L.nptiles = h->d_ntiles;
    L.ctiles = h->d_ctiles;
    L.nctiles = h->d_ntiles + 1;
    L.wq = (uint32_t*)(h->d_ntiles + 2);
    L.nsims = 1;
    L.dims = h->host.dim == 1 ? 1 : 2;
    L.flux = h->host.flux_axis != 0;
    L.grid_p = persistent_grid(h->nptiles, h->grid_per_sm);
    L.grid_c = persistent_grid(h->nctiles, h->grid_per_sm);
    L.lay_tiles = (h->host.K + kLayTile - 1) / kLayTile;
    L.stream = h->stream;
    return L;
}

// one full step of the plain pipeline (every stage in order)
static void enqueue_step(const Launch& L, bool fp64, bool reservoir) {
    launch_stream(L, fp64);
    launch_scan(L);
    launch_scatter(L, fp64);
    if (reservoir) launch_inject(L, fp64);
    launch_moments(L, fp64);
    launch_params(L);
    launch_relax(L, fp64);
    launch_finish(L);
}

// one full step of the fused FP32 pipeline.  The next step's bucket layout
// depends only on this step's arrivals, so it runs on a second stream beside
// the moments and parameters; the end of the step waits for both.
static void enqueue_fused_step(const Launch& L, int R, bool reservoir) {
    launch_fused_relax_stream(L, R, false);
    if (reservoir) launch_fused_inject(L);
    if (L.side) {
        cudaEventRecord(L.ev_fork, L.stream);
        cudaStreamWaitEvent(L.side, L.ev_fork, 0);
        Launch Ls = L;
        Ls.stream = L.side;
        launch_fused_layout_parts(Ls);
        cudaEventRecord(L.ev_join, L.side);
        launch_fused_moments(L, R);
        launch_fused_params(L);
        cudaStreamWaitEvent(L.stream, L.ev_join, 0);
        launch_fused_step_end(L);
        return;
    }
    launch_fused_moments(L, R);
    launch_fused_params(L);
    launch_fused_layout(L);   // ends the step too
}

static void enqueue_any(usp_handle* h, const Launch& L) {
    if (h->host.weighted) enqueue_weighted_step(L);
    else if (h->pipeline == USP_PIPE_FUSED) enqueue_fused_step(L, h->fused_R, h->host.has_reservoir != 0);
    else enqueue_step(L, h->precision == USP_FP64, h->host.has_reservoir != 0);
}

// default k_g2 configuration (7 consumer warps per CTA, two CTAs per SM):
// the fastest of the three on every workload measured; the autotuner may
// pick another (the staged cell size no longer depends on it)
static int choose_R(uint32_t max_count) {
    (void)max_count;
    return 8;
}

static int count_for_density(const SimDev& s, double n, double n_ref, int ppc_ref) {
    (void)s;
    return (int)std::floor(n / n_ref * ppc_ref + 0.5);
}

static int buffer_face_host(const SimDev& s, int cell) {
    int ix = cell % s.nx, iy = cell / s.nx;
    for (int f = 0; f < 4; ++f) {
        if (s.face[f].kind != kBcReservoir) continue;
        int axis = f >> 1;
        if (s.dim == 1 && axis == 0) continue;
        int i = axis == 0 ? ix : iy;
        int n = axis == 0 ? s.nx : s.ny;
        if (((f & 1) == 0 && i < s.reservoir_cols) || ((f & 1) == 1 && i >= n - s.reservoir_cols)) return f;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// creation
// ---------------------------------------------------------------------------
extern "C" int usp_create(const usp_gas* gas, const usp_grid* grid, const usp_bc faces[4],
                          const usp_wall_segment* segs, int nseg, const usp_params* prm,
                          const usp_allocator* allocator, void* stream, usp_handle** out) {
    if (!out) return USP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!gas || !grid || !faces || !prm || nseg < 0 || nseg > USP_MAXSEG || (nseg > 0 && !segs))
        return USP_ERR_INVALID_ARG;
    if (grid->dim != 1 && grid->dim != 2) return USP_ERR_INVALID_ARG;
    const int nx = grid->dim == 1 ? 1 : grid->nx;
    if (grid->ny < 1 || nx < 1 || (int64_t)nx * grid->ny > (int64_t)1 << 28) return USP_ERR_INVALID_ARG;
    if (!(grid->hi[1] > grid->lo[1]) || (grid->dim == 2 && !(grid->hi[0] > grid->lo[0]))) return USP_ERR_INVALID_ARG;
    if (!(gas->mass > 0) || !(gas->T_ref > 0) || !(gas->Pr > 0) || gas->mu_ref < 0) return USP_ERR_INVALID_ARG;
    if (!(prm->n_ref > 0) || prm->ppc_ref < 1 || prm->n_avg < 1) return USP_ERR_INVALID_ARG;
    if (gas->mu_ref == 0 && !(prm->Kn > 0 && prm->L_ref > 0)) return USP_ERR_INVALID_ARG;
    if (!(prm->dt > 0) && !(prm->dt_over_tauc > 0)) return USP_ERR_INVALID_ARG;
    if (prm->mode < 0 || prm->mode > 3) return USP_ERR_INVALID_ARG;
    if (prm->selection < 0 || prm->selection > 1 || prm->es_sampler < 0 || prm->es_sampler > 1)
        return USP_ERR_INVALID_ARG;
    if (prm->precision != USP_FP64 && prm->precision != USP_FP32_MIXED) return USP_ERR_INVALID_ARG;
    if (prm->weighted < 0 || prm->weighted > 1 || prm->weight_average < 0 || prm->weight_average > 1)
        return USP_ERR_INVALID_ARG;
    if (prm->weighted) {
        // the weighted particles run on the plain FP64 pipeline, one domain,
        // without reservoirs, with the default selection and sampler
        if (prm->pipeline != USP_PIPE_PLAIN || prm->precision != USP_FP64 || !(prm->r_p > 0)) return USP_ERR_INVALID_ARG;
        if (prm->selection || prm->es_sampler || prm->slab_count > 1) return USP_ERR_INVALID_ARG;
        for (int f = 0; f < 4; ++f)
            if (faces[f].kind == USP_BC_RESERVOIR) return USP_ERR_INVALID_ARG;
    }
    if (prm->pipeline != USP_PIPE_PLAIN && prm->pipeline != USP_PIPE_FUSED) return USP_ERR_INVALID_ARG;
    if (prm->pipeline == USP_PIPE_FUSED && prm->precision != USP_FP32_MIXED) return USP_ERR_INVALID_ARG;
    if (prm->body_accel[1] != 0 || (grid->dim == 2 && prm->body_accel[0] != 0)) return USP_ERR_INVALID_ARG;
    if (prm->capacity_factor != 0 && prm->capacity_factor < 1) return USP_ERR_INVALID_ARG;
    bool any_res = false;
    for (int f = 0; f < 4; ++f) {
        if (faces[f].kind < 0 || faces[f].kind > 3) return USP_ERR_INVALID_ARG;
        if (grid->dim == 1 && f < 2) continue;
        if ((faces[f].kind == USP_BC_PERIODIC) != (faces[f ^ 1].kind == USP_BC_PERIODIC)) return USP_ERR_INVALID_ARG;
        if (faces[f].kind == USP_BC_DIFFUSE && !(faces[f].T > 0)) return USP_ERR_INVALID_ARG;
        if (faces[f].kind == USP_BC_RESERVOIR) {
            if (!(faces[f].T > 0) || faces[f].n < 0) return USP_ERR_INVALID_ARG;
            any_res = true;
        }
    }
    if (any_res && prm->reservoir_cols < 1) return USP_ERR_INVALID_ARG;
    if (prm->flux_axis < 0 || prm->flux_axis > 2) return USP_ERR_INVALID_ARG;
    if (prm->gll_average < 0 || prm->gll_average > 1) return USP_ERR_INVALID_ARG;
    if (prm->flux_axis) {
        const int a = prm->flux_axis - 1;
        if (a == 0 && grid->dim != 2) return USP_ERR_INVALID_ARG;
        if (faces[2 * a].kind == USP_BC_PERIODIC) return USP_ERR_INVALID_ARG;
        if (!(prm->flux_pos > grid->lo[a] && prm->flux_pos < grid->hi[a])) return USP_ERR_INVALID_ARG;
    }
    const bool slab = prm->slab_count > 1;
    if (prm->slab_count < 0) return USP_ERR_INVALID_ARG;
    if (slab && (prm->pipeline != USP_PIPE_FUSED || any_res || grid->ny % prm->slab_count != 0 ||
                 prm->slab_index < 0 || prm->slab_index >= prm->slab_count))
        return USP_ERR_INVALID_ARG;
    for (int g = 0; g < nseg; ++g) {
        if (grid->dim != 2) return USP_ERR_INVALID_ARG;
        if (segs[g].kind != USP_BC_DIFFUSE && segs[g].kind != USP_BC_SPECULAR) return USP_ERR_INVALID_ARG;
        if (segs[g].kind == USP_BC_DIFFUSE && !(segs[g].T > 0)) return USP_ERR_INVALID_ARG;
    }

    if (prm->pipeline == USP_PIPE_FUSED) fused_prepare_attributes();
    usp_handle* h = new usp_handle();
    h->precision = prm->precision;
    h->pipeline = prm->pipeline;
    h->capacity_factor = prm->capacity_factor;
    h->n_ref = prm->n_ref;
    h->ppc_ref = prm->ppc_ref;
    if (allocator && allocator->alloc && allocator->free) {
        h->alloc = *allocator;
        h->has_alloc = true;
    }
    if (stream) {
        h->stream = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return USP_ERR_CUDA;
        }
        h->own_stream = true;
    }

    SimDev& s = h->host;
    s.dim = grid->dim;
    s.nx = nx;
    s.ny = grid->ny;
    s.slab_count = slab ? prm->slab_count : 1;
    s.slab_index = slab ? prm->slab_index : 0;
    s.slab_first = -1;
    s.rows = grid->ny / s.slab_count;
    s.row0 = s.slab_index * s.rows;
    s.K = nx * s.rows;
    h->slab_group = slab ? prm->slab_group : 0;
    for (int i = 0; i < 2; ++i) {
        s.lo[i] = grid->lo[i];
        s.hi[i] = grid->hi[i];
    }
    s.dy = (grid->hi[1] - grid->lo[1]) / grid->ny;
    s.dx = grid->dim == 2 ? (grid->hi[0] - grid->lo[0]) / nx : 1.0;
    s.mass = gas->mass;
    s.R = kBoltzmann / gas->mass;
    s.T_ref = gas->T_ref;
    s.omega = gas->omega;
    s.Pr = gas->Pr;
    // reference viscosity from Kn through Eq. 36 at (n_ref, T_ref)
    const double rho_ref = prm->n_ref * gas->mass;
    const double p_ref = prm->n_ref * kBoltzmann * gas->T_ref;
    double mu_ref = gas->mu_ref;
    if (mu_ref <= 0) mu_ref = prm->Kn * prm->L_ref * 5.0 * std::sqrt(2.0 * kPi) / 16.0 * std::sqrt(rho_ref * p_ref);
    s.mu_ref = mu_ref;
    // dt from the mean collision time (Eq. 37)
    const double lam_ref = 16.0 / (5.0 * std::sqrt(2.0 * kPi)) * mu_ref / std::sqrt(rho_ref * p_ref);
    const double tau_c = lam_ref / std::sqrt(8.0 * kBoltzmann * gas->T_ref / (kPi * gas->mass));
    s.dt = prm->dt > 0 ? prm->dt : prm->dt_over_tauc * tau_c;
    s.w = prm->n_ref / (double)prm->ppc_ref;
    s.avg_keep = (prm->n_avg - 1.0) / prm->n_avg;
    s.avg_new = 1.0 / prm->n_avg;
    s.mode = prm->mode;
    s.fixed_pne = prm->fixed_pne;
    s.flux_axis = prm->flux_axis;
    s.flux_pos = prm->flux_pos;
    s.f_flux_pos = (float)prm->flux_pos;
    s.gll_average = prm->gll_average != 0;
    s.selection = prm->selection;
    s.es_sampler = prm->es_sampler;
    s.weighted = prm->weighted;
    s.weight_average = prm->weight_average;
    s.r_p = prm->weighted ? prm->r_p : 0.0;
    for (int d = 0; d < 3; ++d) s.body[d] = prm->body_accel[d];
    for (int f = 0; f < 4; ++f) {
        s.face[f].kind = faces[f].kind;
        s.face[f].T = faces[f].T;
        s.face[f].theta = s.R * faces[f].T;
        s.face[f].sqrt_theta = std::sqrt(s.face[f].theta);
        for (int d = 0; d < 3; ++d) s.face[f].u[d] = faces[f].u[d];
    }
    if (s.dim == 1) s.face[0].kind = s.face[1].kind = kBcPeriodic;
    s.periodic_x = s.face[0].kind == kBcPeriodic;
    s.periodic_y = s.face[2].kind == kBcPeriodic;
    s.nseg = nseg;
    for (int g = 0; g < nseg; ++g) {
        s.seg[g].pos = segs[g].pos;
        s.seg[g].lo = segs[g].lo;
        s.seg[g].hi = segs[g].hi;
        s.seg[g].kind = segs[g].kind;
        s.seg[g].theta = s.R * segs[g].T;
        s.seg[g].sqrt_theta = std::sqrt(s.seg[g].theta);
        for (int d = 0; d < 3; ++d) s.seg[g].u[d] = segs[g].u[d];
    }
    s.has_reservoir = any_res;
    s.reservoir_cols = any_res ? prm->reservoir_cols : 0;
    s.f_dt = (float)s.dt;
    for (int i = 0; i < 2; ++i) {
        s.f_lo[i] = (float)s.lo[i];
        s.f_hi[i] = (float)s.hi[i];
    }
    s.f_inv_dx = (float)(1.0 / s.dx);
    s.f_inv_dy = (float)(1.0 / s.dy);
    for (int d = 0; d < 3; ++d) s.f_bdt[d] = (float)(s.body[d] * s.dt);
    s.f_w = (float)s.w;
    s.f_inv_R = (float)(1.0 / s.R);
    s.inv_R = 1.0 / s.R;
    s.es_b = 1.0 - 1.0 / s.Pr;

    const int K = s.K;
    int rc = USP_OK;
    void* p;
#define CALLOC(field, type, count)                                        \
    if ((rc = cell_alloc(h, sizeof(type) * (size_t)(count), &p)) != 0) { \
        usp_destroy(h);                                                   \
        return rc;                                                        \
    }                                                                     \
    s.field = (type*)p;
    CALLOC(count, uint32_t, K + 1);
    CALLOC(start, uint32_t, K + 2);
    CALLOC(fill, uint32_t, K + 1);
    CALLOC(mom, double, (size_t)kNMom * K);
    CALLOC(prm, double, (size_t)kNPrm * K);
    CALLOC(inst, double, (size_t)kNFields * K);
    CALLOC(avg, double, (size_t)kNFields * K);
    CALLOC(ushift, double, 3 * (size_t)K);
    CALLOC(inj_count, uint32_t, K);
    CALLOC(inj_pidoff, uint32_t, K);
    CALLOC(fprm, float, (size_t)kNFPrm * K);
    if (prm->gll_average && prm->pipeline == USP_PIPE_PLAIN) { CALLOC(gavg, double, 3 * (size_t)K); }
    if (prm->pipeline == USP_PIPE_PLAIN) { CALLOC(gloc, double, 6 * (size_t)K); }
    if (prm->weighted) {
        CALLOC(wneff, double, K);
        CALLOC(wst, double, 9 * (size_t)K);
        CALLOC(wfs, double, (size_t)kNWF * K);
        CALLOC(wan, double, (size_t)kNWF * K);
        CALLOC(was, double, (size_t)kNWF * K);
        CALLOC(wna, uint32_t, K);
        CALLOC(woff, uint32_t, K + 1);
    }
    if (prm->pipeline == USP_PIPE_FUSED) {
        CALLOC(momf, float, 16 * (size_t)K);
        CALLOC(floc, float, 4 * (size_t)K);
        for (int b = 0; b < 2; ++b) {
            CALLOC(lay[b], uint32_t, K + 1);
            if (b == 0) { CALLOC(lay_part, unsigned long long, 3 * (size_t)((K + kLayTile - 1) / kLayTile) + 2); }
            CALLOC(cnt[b], uint32_t, K);
            CALLOC(sp_pos[b][0], float, kSpillCap);
            CALLOC(sp_pos[b][1], float, kSpillCap);
            for (int d = 0; d < 3; ++d) { CALLOC(sp_vel[b][d], float, kSpillCap); }
            CALLOC(sp_pid[b], uint32_t, kSpillCap);
            CALLOC(sp_cell[b], uint32_t, kSpillCap);
        }
    }
#undef CALLOC
    if ((rc = cell_alloc(h, sizeof(SimDev), &p)) != 0) { usp_destroy(h); return rc; }
    h->d_sim = (SimDev*)p;
    if ((rc = cell_alloc(h, sizeof(SimDyn), &p)) != 0) { usp_destroy(h); return rc; }
    h->d_dyn = (SimDyn*)p;
    s.dyn = h->d_dyn;
    if ((rc = cell_alloc(h, 4 * sizeof(int), &p)) != 0) { usp_destroy(h); return rc; }
    h->d_ntiles = (int*)p;
    h->nctiles = (K + kCTile - 1) / kCTile;
    if ((rc = cell_alloc(h, sizeof(int2) * (size_t)h->nctiles, &p)) != 0) { usp_destroy(h); return rc; }
    h->d_ctiles = (int2*)p;

    // reservoir refill table: count per buffer cell, pid offsets in (face, cell) order
    h->inj_count_host.assign(K, 0);
    std::vector<uint32_t> off(K, 0);
    uint32_t total = 0;
    if (any_res) {
        for (int f = 0; f < 4; ++f) {
            if (s.face[f].kind != kBcReservoir) continue;
            for (int c = 0; c < K; ++c) {
                if (buffer_face_host(s, c) != f) continue;
                uint32_t cnt = (uint32_t)count_for_density(s, faces[f].n, prm->n_ref, prm->ppc_ref);
                h->inj_count_host[c] = cnt;
                off[c] = total;
                total += cnt;
            }
        }
    }
    s.inj_total = total;
    std::vector<int2> ct(h->nctiles);
    for (int t = 0; t < h->nctiles; ++t) ct[t] = make_int2(0, t * kCTile);
    int nt[4] = {0, h->nctiles, 0, 0};
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.inj_count, h->inj_count_host.data(), sizeof(uint32_t) * K, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.inj_pidoff, off.data(), sizeof(uint32_t) * K, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_ctiles, ct.data(), sizeof(int2) * ct.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_ntiles, nt, sizeof(nt), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.count, 0, sizeof(uint32_t) * (K + 1), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.fill, 0, sizeof(uint32_t) * (K + 1), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s.ushift, 0, sizeof(double) * 3 * K, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_dyn, 0, sizeof(SimDyn), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // host vectors above go out of scope
    if (e != cudaSuccess) {
        cudaGetLastError();
        usp_destroy(h);
        return USP_ERR_CUDA;
    }
    if (upload_sim(h) != USP_OK) {
        usp_destroy(h);
        return USP_ERR_CUDA;
    }
    *out = h;
    return USP_OK;
}

// ---------------------------------------------------------------------------
// particle storage
// ---------------------------------------------------------------------------
static int alloc_particles(usp_handle* h, int64_t n) {
    SimDev& s = h->host;
    double f = h->capacity_factor > 0 ? h->capacity_factor : (s.has_reservoir ? 2.0 : 1.25);
    // weighted particles: the three stages of a step add up to 3 N / r_p
    // before the deletions of Eq. 28, and the population settles up to
    // ~20 % above its start
    if (s.weighted) f = std::max(f, 1.5 * (1.0 + 3.0 / s.r_p));
    int64_t cap = (int64_t)std::ceil(n * f) + 2 * (int64_t)s.inj_total + 1024;
    if (h->pipeline == USP_PIPE_FUSED) {
        // slack buckets: about 1.25 x the largest neighbouring count + 16 per cell
        const double ff = h->capacity_factor > 0 ? std::max(h->capacity_factor, 1.6) : (s.has_reservoir ? 2.5 : 1.6);
        cap = (int64_t)std::ceil(n * ff) + 24 * (int64_t)s.K + 4 * (int64_t)s.inj_total + 4096;
    }
    cap = (cap + 3) & ~(int64_t)3;   // whole 16-byte groups of FP32 slots (bulk copies of the fused pipeline)
    if (cap > (int64_t)0x7FFFFFFFll) return fail(h, USP_ERR_CAPACITY, "particle capacity exceeds 2^31 - 1");
    destroy_graphs(h->graphs);
    // storage of a similar size is kept (a re-load of the same problem
    // allocates nothing); the tile tables depend only on the capacity
    if (!h->part_allocs.empty() && cap <= s.cap && 2 * cap > s.cap) return USP_OK;
    free_particles(h);
    const size_t es = h->precision == USP_FP64 ? 8 : 4;
    auto grab = [&](size_t bytes) -> void* {
        void* p = dalloc(h, bytes);
        if (p) {
            h->part_allocs.push_back(p);
            h->part_bytes += bytes;
        }
        return p;
    };
    // buffer 0 plane by plane; buffer 1 and the cell plane as one block
    // (usp_set_particles stages the caller's FP64 arrays there before the
    // sort fills it); every plane starts on a 16-byte boundary (cap is a
    // multiple of 4)
    const size_t plane = es * (size_t)cap, slots = 4 * (size_t)cap;
    const size_t b1_bytes = (s.dim == 2 ? 5 : 4) * plane + 2 * slots;
    char* blk = (char*)grab(b1_bytes);
    h->b1_block = blk;
    h->b1_bytes = blk ? b1_bytes : 0;
    for (int b = 0; b < 2; ++b) {
        auto take = [&](size_t bytes) -> void* {
            if (b == 0) return grab(bytes);
            if (!blk) return nullptr;
            void* r = blk;
            blk += bytes;
            return r;
        };
        s.pos[b][0] = s.dim == 2 ? take(plane) : nullptr;
        s.pos[b][1] = take(plane);
        for (int d = 0; d < 3; ++d) s.vel[b][d] = take(plane);
        s.pid[b] = (uint32_t*)take(slots);
        if ((s.dim == 2 && !s.pos[b][0]) || !s.pos[b][1] || !s.vel[b][0] || !s.vel[b][1] || !s.vel[b][2] || !s.pid[b]) {
            free_particles(h);
            return fail(h, USP_ERR_OOM, "particle storage allocation failed");
        }
    }
    s.cell = blk ? (uint32_t*)blk : nullptr;
    if (s.weighted) {
        s.wgt[0] = (double*)grab(8 * cap);
        s.wgt[1] = (double*)grab(8 * cap);
        if (!s.wgt[0] || !s.wgt[1]) {
            free_particles(h);
            return fail(h, USP_ERR_OOM, "particle weight allocation failed");
        }
    }
    if (!s.cell) {
        free_particles(h);
        return fail(h, USP_ERR_OOM, "particle storage allocation failed");
    }
    s.cap = cap;
    h->nptiles = (int)((cap + kPTile - 1) / kPTile);
    if (h->d_ptiles) {
        // replace the previous table
        for (size_t i = 0; i < h->cell_allocs.size(); ++i)
            if (h->cell_allocs[i] == h->d_ptiles) {
                dfree(h, h->d_ptiles);
                h->cell_allocs.erase(h->cell_allocs.begin() + i);
                break;
            }
        h->d_ptiles = nullptr;
    }
    void* p;
    int rc = cell_alloc(h, sizeof(int2) * (size_t)h->nptiles, &p);
    if (rc) return rc;
    h->d_ptiles = (int2*)p;
    std::vector<int2> pt(h->nptiles);
    for (int t = 0; t < h->nptiles; ++t) pt[t] = make_int2(0, t * kPTile);
    int nt[2] = {h->nptiles, h->nctiles};
    cudaError_t e = cudaMemcpyAsync(h->d_ptiles, pt.data(), sizeof(int2) * pt.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_ntiles, nt, sizeof(nt), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, USP_ERR_CUDA, cudaGetErrorString(e));
    return USP_OK;
}

static int reset_dynamic(usp_handle* h, uint32_t n, uint32_t next_pid) {
    SimDyn d{};
    d.n = n;
    d.next_pid = next_pid;
    const int K = h->host.K;
    CK(cudaMemcpyAsync(h->d_dyn, &d, sizeof(d), cudaMemcpyHostToDevice, h->stream));   // pageable: copied out now
    // counts, shifts, fields, averages and parameters cleared in one launch
    const size_t k = (size_t)K;
    ZeroList z{{h->host.count, h->host.fill, h->host.ushift, h->host.inst, h->host.avg, h->host.prm},
               {k + 1, k + 1, 2 * 3 * k, 2 * (size_t)kNFields * k, 2 * (size_t)kNFields * k, 2 * (size_t)kNPrm * k},
               6};
    launch_zero(z, h->stream);
    CK(cudaGetLastError());
    return USP_OK;
}

// weighted particles: every loaded particle has weight 1, the parameters
// (P_ne of the first step 2) and the weight-field averages start at zero
static int weighted_setup(usp_handle* h) {
    SimDev& s = h->host;
    if (!s.weighted) return USP_OK;
    const size_t K = (size_t)s.K;
    CK(cudaMemsetAsync(s.prm, 0, sizeof(double) * kNPrm * K, h->stream));
    CK(cudaMemsetAsync(s.wan, 0, sizeof(double) * kNWF * K, h->stream));
    CK(cudaMemsetAsync(s.was, 0, sizeof(double) * kNWF * K, h->stream));
    Launch L = make_launch(h);
    launch_weighted_init(L);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    return USP_OK;
}

extern "C" int usp_init_particles(usp_handle* h, const usp_region* regions, int nregions, uint64_t seed) {
    if (!h) return USP_ERR_INVALID_ARG;
    if (nregions < 0 || (nregions > 0 && !regions)) return fail(h, USP_ERR_INVALID_ARG, "bad regions");
    if (h->batch_refs) return fail(h, USP_ERR_STATE, "handle is admitted to a batch");
    if (h->host.slab_count > 1) return fail(h, USP_ERR_STATE, "a slab is loaded with usp_set_particles");
    SimDev& s = h->host;
    const int K = s.K;
    std::vector<int> reg(K, -1);
    std::vector<uint32_t> start(K + 2, 0);
    uint64_t total = 0;
    for (int c = 0; c < K; ++c) {
        const int ix = c % s.nx, iy = c / s.nx;
        const double xl = s.dim == 2 ? s.lo[0] + ix * s.dx : 0.0;
        const double yl = s.lo[1] + iy * s.dy;
        const double xc = xl + 0.5 * s.dx, yc = yl + 0.5 * s.dy;
        int r = -1;
        for (int i = 0; i < nregions; ++i) {
            const bool in_y = yc >= regions[i].lo[1] && yc < regions[i].hi[1];
            const bool in_x = s.dim == 1 || (xc >= regions[i].lo[0] && xc < regions[i].hi[0]);
            if (in_x && in_y) r = i;
        }
        start[c] = (uint32_t)total;
        if (r < 0) continue;
        if (!(regions[r].T > 0) || regions[r].n < 0) return fail(h, USP_ERR_INVALID_ARG, "bad region state");
        reg[c] = r;
        total += (uint64_t)count_for_density(s, regions[r].n, h->n_ref, h->ppc_ref);
        if (total > 0xFFFFFFF0ull / 2) return fail(h, USP_ERR_CAPACITY, "too many particles");
    }
    start[K] = start[K + 1] = (uint32_t)total;
    int rc = alloc_particles(h, (int64_t)total);
    if (rc) return rc;
    s.key0 = (uint32_t)seed;
    s.key1 = (uint32_t)(seed >> 32);
    if ((rc = upload_sim(h)) != 0) return rc;
    std::vector<double> th(std::max(1, nregions)), uu(3 * std::max(1, nregions));
    for (int i = 0; i < nregions; ++i) {
        th[i] = s.R * regions[i].T;
        for (int d = 0; d < 3; ++d) uu[3 * i + d] = regions[i].u[d];
    }
    double *d_th = nullptr, *d_u = nullptr;
    int* d_reg = nullptr;
    d_th = (double*)dalloc(h, sizeof(double) * th.size());
    d_u = (double*)dalloc(h, sizeof(double) * uu.size());
    d_reg = (int*)dalloc(h, sizeof(int) * K);
    if (!d_th || !d_u || !d_reg) {
        dfree(h, d_th); dfree(h, d_u); dfree(h, d_reg);
        return fail(h, USP_ERR_OOM, "init scratch allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(d_th, th.data(), sizeof(double) * th.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_u, uu.data(), sizeof(double) * uu.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_reg, reg.data(), sizeof(int) * K, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.start, start.data(), sizeof(uint32_t) * (K + 2), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) {
        rc = reset_dynamic(h, (uint32_t)total, (uint32_t)total);
        if (rc == USP_OK) {
            Launch L = make_launch(h);
            launch_init(L, h->precision == USP_FP64, d_th, d_u, d_reg);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dfree(h, d_th); dfree(h, d_u); dfree(h, d_reg);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(h, USP_ERR_CUDA, std::string("init: ") + cudaGetErrorString(e));
    if (h->pipeline == USP_PIPE_FUSED) {
        uint32_t mx = 0;
        for (int c = 0; c < K; ++c) mx = std::max(mx, start[c + 1] - start[c]);
        h->fused_R = choose_R(mx + mx / 4);
        Launch L = make_launch(h);
        // no parameters yet: zero shift for the first moments, no relaxation
        CK(cudaMemsetAsync(h->host.fprm, 0, sizeof(float) * kNFPrm * (size_t)K, h->stream));
        launch_fused_setup(L);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(h->stream));
    }
    if ((rc = weighted_setup(h)) != 0) return rc;
    h->initialised = true;
    h->mid_step = false;
    h->sorted = true;
    return USP_OK;
}

// order a freshly loaded state by cell (assign + scan + scatter into buffer 1)
// and build the bucket layout of the fused pipeline
static int fused_from_unsorted(usp_handle* h) {
    SimDev& s = h->host;
    const int K = s.K;
    Launch L = make_launch(h);
    launch_assign(L, false);
    launch_scan(L, false);   // the loaded particles only: no room for a refill
    launch_scatter(L, false);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(s.fill, 0, sizeof(uint32_t) * (K + 1), h->stream));
    // no parameters yet: zero shift for the first moments, no relaxation
    CK(cudaMemsetAsync(s.fprm, 0, sizeof(float) * kNFPrm * (size_t)K, h->stream));
    int one = 1;   // pageable: copied out before the call returns
    CK(cudaMemcpyAsync(&h->d_dyn->cur, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    h->fused_R = choose_R(0);
    launch_fused_setup(L);
    CK(cudaGetLastError());
    return USP_OK;
}

// the device address of a page-locked host array (mapped into the device's
// address space), or null for pageable memory
static const void* mapped_host(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

extern "C" int usp_set_particles(usp_handle* h, int64_t n, const double* pos, const double* vel, const uint32_t* pid,
                                 uint32_t next_pid, uint64_t seed) {
    if (!h) return USP_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!pos || !vel || !pid))) return fail(h, USP_ERR_INVALID_ARG, "bad particle arrays");
    if (h->batch_refs) return fail(h, USP_ERR_STATE, "handle is admitted to a batch");
    if (n > (int64_t)0x7FFFFFF0) return fail(h, USP_ERR_CAPACITY, "too many particles");
    int rc = alloc_particles(h, n);
    if (rc) return rc;
    SimDev& s = h->host;
    s.key0 = (uint32_t)seed;
    s.key1 = (uint32_t)(seed >> 32);
    if ((rc = upload_sim(h)) != 0) return rc;
    const bool fp64 = h->precision == USP_FP64;
    const bool auto_pid = next_pid == USP_NEXT_PID_AUTO;
    // the dynamic state first: with auto_pid its next_pid starts at 0 and
    // the unpack pass raises it to one past the largest loaded id
    if ((rc = reset_dynamic(h, (uint32_t)n, auto_pid ? 0u : next_pid)) != 0) return rc;
    uint32_t* d_next = auto_pid ? &h->d_dyn->next_pid : nullptr;
    cudaError_t e = cudaSuccess;
    const double* mpos = n > 0 ? (const double*)mapped_host(pos) : nullptr;
    const double* mvel = n > 0 ? (const double*)mapped_host(vel) : nullptr;
    const uint32_t* mpid = n > 0 ? (const uint32_t*)mapped_host(pid) : nullptr;
    const bool direct = mpos && mvel && mpid;
    if (direct) {
        // page-locked arrays: one pass reads them in place over the host
        // link (measured faster than copy-engine transfers plus a transpose)
        launch_unpack(s, fp64, mpos, mvel, mpid, true, d_next, n, h->stream);
        e = cudaGetLastError();
    } else if (n > 0) {
        // pageable arrays go to the device as they are: the ids into their
        // plane, the FP64 positions and then the velocities into buffer 1
        // and the cell plane (at least 24 bytes per slot, filled by the sort
        // only afterwards), each transposed into buffer 0's planes
        if (h->b1_bytes < 24 * (size_t)n) return fail(h, USP_ERR_CAPACITY, "staging area smaller than the load");
        double* stg = (double*)h->b1_block;
        e = cudaMemcpyAsync(s.pid[0], pid, 4 * n, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(stg, pos, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) {
            launch_unpack(s, fp64, stg, nullptr, nullptr, false, nullptr, n, h->stream);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(stg, vel, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream);
    }
    // the point on the stream after which the caller's arrays are no longer read
    if (e == cudaSuccess && !h->upload_ev) e = cudaEventCreateWithFlags(&h->upload_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(h->upload_ev, h->stream);
    if (e == cudaSuccess && !direct && n > 0) {
        launch_unpack(s, fp64, nullptr, (const double*)h->b1_block, s.pid[0], false, d_next, n, h->stream);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaStreamSynchronize(h->stream);
        return fail(h, USP_ERR_CUDA, cudaGetErrorString(e));
    }
    if (h->pipeline == USP_PIPE_FUSED) rc = fused_from_unsorted(h);
    // return once the arrays have been read; the set-up kernels behind the
    // event run on the handle's stream like a step
    e = cudaEventSynchronize(h->upload_ev);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(h, USP_ERR_CUDA, cudaGetErrorString(e));
    if ((rc = weighted_setup(h)) != 0) return rc;
    h->initialised = true;
    h->mid_step = false;
    h->sorted = h->pipeline == USP_PIPE_FUSED;
    return USP_OK;
}

// ---------------------------------------------------------------------------
// stepping
// ---------------------------------------------------------------------------
static int capture(usp_handle* h, int nsteps, cudaGraphExec_t* exec) {
    Launch L = make_launch(h);
    if (h->pipeline == USP_PIPE_FUSED && !h->host.weighted && h->fork.make()) h->fork.attach(L);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < nsteps; ++i) enqueue_any(h, L);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (e != cudaSuccess) return fail(h, USP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, USP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return USP_OK;
}

extern "C" int usp_step(usp_handle* h, int nsteps) {
    if (!h) return USP_ERR_INVALID_ARG;
    if (nsteps < 0) return fail(h, USP_ERR_INVALID_ARG, "nsteps < 0");
    if (!h->initialised) return fail(h, USP_ERR_STATE, "particles not initialised");
    if (h->mid_step) return fail(h, USP_ERR_STATE, "a staged step is in progress");
    if (h->batch_refs) return fail(h, USP_ERR_STATE, "handle is admitted to a batch");
    if (h->host.slab_count > 1) return fail(h, USP_ERR_STATE, "a slab steps only in a batch with its neighbours");
    if (nsteps == 0) return USP_OK;
    int rc;
    if (!h->graphs.one && (rc = capture(h, 1, &h->graphs.one)) != 0) return rc;
    if (nsteps >= kGraphSteps && !h->graphs.many && (rc = capture(h, kGraphSteps, &h->graphs.many)) != 0) return rc;
    int left = nsteps;
    while (left >= kGraphSteps) {
        CK(cudaGraphLaunch(h->graphs.many, h->stream));
        left -= kGraphSteps;
    }
    while (left-- > 0) CK(cudaGraphLaunch(h->graphs.one, h->stream));
    h->sorted = true;
    return USP_OK;
}

// one stage of a step: plain pipeline 0..6, fused pipeline 10..14
static int stage_launch(const Launch& L, int pipeline, bool fp64, int R, bool reservoir, int stage) {
    if (pipeline == USP_PIPE_FUSED) {
        switch (stage) {
        case 10: launch_fused_relax_stream(L, R, false); return 0;
        case 11: if (reservoir) launch_fused_inject(L); return 0;
        case 12: launch_fused_moments(L, R); return 0;
        case 13: launch_fused_params(L); return 0;
        case 14: launch_fused_layout(L); return 0;   // layout + end of step
        default: return -1;
        }
    }
    switch (stage) {
    case 0: launch_stream(L, fp64); return 0;
    case 1: return 0;   // reservoir removal happens in stage 0, refill in stage 2
    case 2:
        launch_scan(L);
        launch_scatter(L, fp64);
        if (reservoir) launch_inject(L, fp64);
        return 0;
    case 3: launch_moments(L, fp64); return 0;
    case 4: launch_params(L); return 0;
    case 5: launch_relax(L, fp64); return 0;
    case 6: launch_finish(L); return 0;
    default: return -1;
    }
}

extern "C" int usp_run_stage(usp_handle* h, int stage) {
    if (!h) return USP_ERR_INVALID_ARG;
    if (!h->initialised) return fail(h, USP_ERR_STATE, "particles not initialised");
    if (h->host.weighted) return fail(h, USP_ERR_STATE, "weighted particles step whole steps only");
    if (h->batch_refs) return fail(h, USP_ERR_STATE, "handle is admitted to a batch");
    if (h->host.slab_count > 1) return fail(h, USP_ERR_STATE, "a slab steps only in a batch with its neighbours");
    Launch L = make_launch(h);
    if (stage_launch(L, h->pipeline, h->precision == USP_FP64, h->fused_R, h->host.has_reservoir != 0, stage))
        return fail(h, USP_ERR_INVALID_ARG, "stage must be 0..6 (plain) or 10..14 (fused)");
    if (h->pipeline == USP_PIPE_PLAIN) {
        if (stage == 0) h->sorted = false;
        if (stage == 2) h->mid_step = h->sorted = true;
        if (stage == 6) h->mid_step = false;
    } else {
        h->mid_step = stage >= 10 && stage < 14;
    }
    CK(cudaGetLastError());
    return USP_OK;
}

// ---------------------------------------------------------------------------
// read-back
// ---------------------------------------------------------------------------
// wait for everything queued for this handle (its own stream and, while it is
// admitted, the stream of its batch)
static int sync_handle(usp_handle* h) {
    CK(cudaStreamSynchronize(h->stream));
    if (h->batch_stream) CK(cudaStreamSynchronize(h->batch_stream));
    return USP_OK;
}

static int read_dyn(usp_handle* h, SimDyn* d) {
    if (int rc = sync_handle(h)) return rc;
    CK(cudaMemcpy(d, h->d_dyn, sizeof(SimDyn), cudaMemcpyDeviceToHost));
    if (d->counters[kCntOverflow]) return fail(h, USP_ERR_CAPACITY, "particle slots overflowed during a step");
    return USP_OK;
}

extern "C" int usp_synchronize(usp_handle* h) {
    if (!h) return USP_ERR_INVALID_ARG;
    SimDyn d;
    return read_dyn(h, &d);
}

extern "C" int usp_sample_macro(usp_handle* h, int which, double* out, size_t out_len, int out_on_device) {
    if (!h || !out) return USP_ERR_INVALID_ARG;
    const size_t need = (size_t)kNFields * h->host.K;
    if (out_len < need) return fail(h, USP_ERR_INVALID_ARG, "output too small");
    if (which != USP_SAMPLE_INSTANT && which != USP_SAMPLE_AVERAGED) return fail(h, USP_ERR_INVALID_ARG, "bad field set");
    if (int rc = sync_handle(h)) return rc;
    const double* src = which == USP_SAMPLE_INSTANT ? h->host.inst : h->host.avg;
    CK(cudaMemcpy(out, src, need * sizeof(double), out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return USP_OK;
}

// fused pipeline: apply the pending relaxation, then gather the buckets and the
// spill list of the current buffer in cell order
static int get_particles_fused(usp_handle* h, double* pos, double* vel, uint32_t* pid, int32_t* cell, int64_t cap,
                               int64_t* n_out) {
    if (h->mid_step) return fail(h, USP_ERR_STATE, "a staged step is in progress");
    SimDyn d;
    int rc = read_dyn(h, &d);
    if (rc && rc != USP_ERR_CAPACITY) return rc;
    if (d.relax_pending) {
        Launch L = make_launch(h);
        launch_fused_relax_stream(L, h->fused_R, true);
        CK(cudaGetLastError());
        int rc2 = read_dyn(h, &d);
        if (rc2 && rc2 != USP_ERR_CAPACITY) return rc2;
    }
    const SimDev& s = h->host;
    const int K = s.K;
    const int b = d.cur;
    std::vector<uint32_t> lay(K + 1), cnt(K);
    CK(cudaMemcpy(lay.data(), s.lay[b], sizeof(uint32_t) * (K + 1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cnt.data(), s.cnt[b], sizeof(uint32_t) * K, cudaMemcpyDeviceToHost));
    const uint32_t nsp = std::min<uint32_t>(d.sp_n[b], (uint32_t)kSpillCap);
    int64_t n = 0;
    for (int c = 0; c < K; ++c) n += cnt[c];
    if (n_out) *n_out = n;
    if (n > cap) return fail(h, USP_ERR_CAPACITY, "output arrays too small");
    const int64_t slots = std::min<int64_t>(lay[K], s.cap);
    for (int c = 0; c <= K; ++c) lay[c] = (uint32_t)std::min<int64_t>(lay[c], s.cap);
    std::vector<float> P[5];
    const int planes[5][2] = {{0, 0}, {0, 1}, {1, 0}, {1, 1}, {1, 2}};
    for (int k = 0; k < 5; ++k) {
        if (k == 0 && s.dim == 1) continue;
        P[k].resize(std::max<int64_t>(slots, 1));
        const void* src = planes[k][0] == 0 ? s.pos[b][planes[k][1]] : s.vel[b][planes[k][1]];
        CK(cudaMemcpy(P[k].data(), src, 4 * slots, cudaMemcpyDeviceToHost));
    }
    std::vector<uint32_t> ids(std::max<int64_t>(slots, 1));
    CK(cudaMemcpy(ids.data(), s.pid[b], 4 * slots, cudaMemcpyDeviceToHost));
    std::vector<float> SP[5];
    std::vector<uint32_t> spid(nsp + 1), scell(nsp + 1);
    for (int k = 0; k < 5; ++k) {
        if (k == 0 && s.dim == 1) continue;
        SP[k].resize(nsp + 1);
        const float* src = planes[k][0] == 0 ? s.sp_pos[b][planes[k][1]] : s.sp_vel[b][planes[k][1]];
        if (nsp) CK(cudaMemcpy(SP[k].data(), src, 4 * nsp, cudaMemcpyDeviceToHost));
    }
    if (nsp) {
        CK(cudaMemcpy(spid.data(), s.sp_pid[b], 4 * nsp, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(scell.data(), s.sp_cell[b], 4 * nsp, cudaMemcpyDeviceToHost));
    }
    int64_t o = 0;
    auto put = [&](const std::vector<float>* A, size_t i, uint32_t id, int c) {
        if (pos) {
            pos[2 * o] = s.dim == 2 ? A[0][i] : 0.0;
            pos[2 * o + 1] = A[1][i];
        }
        if (vel)
            for (int k = 0; k < 3; ++k) vel[3 * o + k] = A[2 + k][i];
        if (pid) pid[o] = id;
        if (cell) cell[o] = c + s.row0 * s.nx;   // global cell id (slabs own a row range)
        ++o;
    };
    for (int c = 0; c < K; ++c) {
        const uint32_t capc = lay[c + 1] - lay[c];
        const uint32_t nb = std::min(cnt[c], capc);
        for (uint32_t j = 0; j < nb; ++j) put(P, lay[c] + j, ids[lay[c] + j], c);
        if (cnt[c] > nb)
            for (uint32_t k = 0; k < nsp; ++k)
                if ((int)scell[k] == c) put(SP, k, spid[k], c);
    }
    if (n_out) *n_out = o;
    return rc;
}

extern "C" int usp_get_particles(usp_handle* h, double* pos, double* vel, uint32_t* pid, int32_t* cell, int64_t cap,
                                 int64_t* n_out) {
    if (!h) return USP_ERR_INVALID_ARG;
    if (h->pipeline == USP_PIPE_FUSED && h->initialised) return get_particles_fused(h, pos, vel, pid, cell, cap, n_out);
    SimDyn d;
    int rc = read_dyn(h, &d);
    if (rc && rc != USP_ERR_CAPACITY) return rc;
    const SimDev& s = h->host;
    const int K = s.K;
    std::vector<uint32_t> start(K + 2);
    CK(cudaMemcpy(start.data(), s.start, sizeof(uint32_t) * (K + 2), cudaMemcpyDeviceToHost));
    int buf = d.cur;
    int64_t n = d.n;
    if (h->mid_step) {
        buf ^= 1;
        n = start[K];
    }
    if (n_out) *n_out = n;
    if (n > cap) return fail(h, USP_ERR_CAPACITY, "output arrays too small");
    if (!h->initialised || n == 0) return USP_OK;
    const bool fp64 = h->precision == USP_FP64;
    const size_t es = fp64 ? 8 : 4;
    std::vector<unsigned char> tmp(es * n);
    auto get = [&](const void* src, double* dst, int stride, int comp) -> cudaError_t {
        cudaError_t e = cudaMemcpy(tmp.data(), src, es * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        for (int64_t i = 0; i < n; ++i)
            dst[stride * i + comp] = fp64 ? ((double*)tmp.data())[i] : (double)((float*)tmp.data())[i];
        return cudaSuccess;
    };
    cudaError_t e = cudaSuccess;
    if (pos) {
        if (s.dim == 2) e = get(s.pos[buf][0], pos, 2, 0);
        else for (int64_t i = 0; i < n; ++i) pos[2 * i] = 0.0;
        if (e == cudaSuccess) e = get(s.pos[buf][1], pos, 2, 1);
    }
    for (int dd = 0; dd < 3 && vel && e == cudaSuccess; ++dd) e = get(s.vel[buf][dd], vel, 3, dd);
    if (pid && e == cudaSuccess) e = cudaMemcpy(pid, s.pid[buf], 4 * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(h, USP_ERR_CUDA, cudaGetErrorString(e));
    if (cell) {
        if (h->sorted) {
            int c = 0;
            for (int64_t i = 0; i < n; ++i) {
                while (c < K && (uint32_t)i >= start[c + 1]) ++c;
                cell[i] = c;
            }
        } else {
            for (int64_t i = 0; i < n; ++i) cell[i] = -1;
        }
    }
    return rc;
}

extern "C" int usp_get_params(usp_handle* h, double* out, size_t out_len) {
    if (!h || !out) return USP_ERR_INVALID_ARG;
    const int K = h->host.K;
    if (out_len < (size_t)kNPrm * K) return fail(h, USP_ERR_INVALID_ARG, "output too small");
    if (int rc = sync_handle(h)) return rc;
    std::vector<double> t((size_t)kNPrm * K);
    CK(cudaMemcpy(t.data(), h->host.prm, sizeof(double) * t.size(), cudaMemcpyDeviceToHost));
    for (int c = 0; c < K; ++c)
        for (int k = 0; k < kNPrm; ++k) out[(size_t)c * kNPrm + k] = t[(size_t)k * K + c];
    return USP_OK;
}

extern "C" int usp_get_weights(usp_handle* h, double* w, int64_t cap, int64_t* n_out) {
    if (!h || !w || !n_out) return USP_ERR_INVALID_ARG;
    if (!h->host.weighted) return fail(h, USP_ERR_STATE, "the handle has no particle weights");
    SimDyn d;
    int rc = read_dyn(h, &d);
    if (rc && rc != USP_ERR_CAPACITY) return rc;
    if ((int64_t)d.n > cap) return fail(h, USP_ERR_INVALID_ARG, "output too small");
    *n_out = d.n;
    if (d.n) CK(cudaMemcpy(w, h->host.wgt[d.cur], sizeof(double) * d.n, cudaMemcpyDeviceToHost));
    return USP_OK;
}

extern "C" int usp_get_info(usp_handle* h, usp_info* info) {
    if (!h || !info) return USP_ERR_INVALID_ARG;
    SimDyn d{};
    int rc = read_dyn(h, &d);
    if (rc && rc != USP_ERR_CAPACITY) return rc;
    memset(info, 0, sizeof(*info));
    info->n_particles = d.n;
    info->capacity = h->host.cap;
    info->n_cells = h->host.K;
    info->precision = h->precision;
    info->pipeline = h->pipeline;
    info->step = d.step;
    info->dt = h->host.dt;
    info->mu_ref = h->host.mu_ref;
    for (int i = 0; i < 8; ++i) info->counters[i] = (int64_t)d.counters[i];
    info->device_bytes = h->cell_bytes + h->part_bytes;
    info->next_pid = d.next_pid;
    return rc;
}

extern "C" int usp_debug_philox(int64_t n, const uint32_t* ctr, uint32_t key0, uint32_t key1, uint32_t* out) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return USP_ERR_INVALID_ARG;
    if (n == 0) return USP_OK;
    uint32_t *dc = nullptr, *dout = nullptr;
    if (cudaMalloc(&dc, 16 * n) != cudaSuccess || cudaMalloc(&dout, 16 * n) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dc);
        return USP_ERR_OOM;
    }
    cudaError_t e = cudaMemcpy(dc, ctr, 16 * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = debug_philox(n, dc, key0, key1, dout, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, 16 * n, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    return e == cudaSuccess ? USP_OK : USP_ERR_CUDA;
}

extern "C" int usp_destroy(usp_handle* h) {
    if (!h) return USP_ERR_INVALID_ARG;
    if (h->batch_refs) return fail(h, USP_ERR_STATE, "handle is admitted to a batch");
    if (h->stream) cudaStreamSynchronize(h->stream);
    destroy_graphs(h->graphs);
    free_particles(h);
    for (void* p : h->cell_allocs) dfree(h, p);
    h->cell_allocs.clear();
    if (h->upload_ev) cudaEventDestroy(h->upload_ev);
    h->fork.release();
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return USP_OK;
}

extern "C" const char* usp_last_error(const usp_handle* h) { return h ? h->err.c_str() : "null handle"; }

extern "C" const char* usp_status_string(int status) {
    switch (status) {
    case USP_OK: return "ok";
    case USP_ERR_INVALID_ARG: return "invalid argument";
    case USP_ERR_OOM: return "out of device memory";
    case USP_ERR_CUDA: return "CUDA error";
    case USP_ERR_CAPACITY: return "capacity exceeded";
    case USP_ERR_TIMEOUT: return "timeout";
    case USP_ERR_STATE: return "invalid state";
    default: return "unknown status";
    }
}

// ---------------------------------------------------------------------------
// batching
// ---------------------------------------------------------------------------
static int bfail(usp_batch* b, int code, const std::string& m) {
    if (b) b->err = m;
    return code;
}

extern "C" int usp_batch_create(size_t hbm_budget, int max_sims, void* stream, usp_batch** out) {
    if (!out || max_sims < 1) return USP_ERR_INVALID_ARG;
    *out = nullptr;
    usp_batch* b = new usp_batch();
    b->budget = hbm_budget;
    b->max_sims = max_sims;
    if (stream) b->stream = (cudaStream_t)stream;
    else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return USP_ERR_CUDA;
        }
        b->own_stream = true;
    }
    if (cudaMalloc(&b->d_sims, sizeof(SimDev) * max_sims) != cudaSuccess ||
        cudaMalloc(&b->d_ntiles, 4 * sizeof(int)) != cudaSuccess ||
        cudaMemsetAsync(b->d_ntiles, 0, 4 * sizeof(int), b->stream) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->d_sims);
        cudaFree(b->d_ntiles);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return USP_ERR_OOM;
    }
    *out = b;
    return USP_OK;
}

static size_t handle_bytes(const usp_handle* h) { return h->cell_bytes + h->part_bytes; }

extern "C" int usp_batch_info(usp_batch* b, int* n_sims, size_t* bytes) {
    if (!b) return USP_ERR_INVALID_ARG;
    size_t used = 0;
    for (auto* h : b->members) used += handle_bytes(h);
    if (n_sims) *n_sims = (int)b->members.size();
    if (bytes) *bytes = used;
    return USP_OK;
}

extern "C" int usp_batch_admit(usp_batch* b, usp_handle* h) {
    if (!b || !h) return USP_ERR_INVALID_ARG;
    if (!h->initialised || h->mid_step) return bfail(b, USP_ERR_STATE, "handle not ready");
    if (h->host.weighted) return bfail(b, USP_ERR_INVALID_ARG, "weighted particles step alone");
    for (auto* m : b->members)
        if (m == h) return bfail(b, USP_ERR_STATE, "already admitted");
    if ((int)b->members.size() >= b->max_sims) return bfail(b, USP_ERR_CAPACITY, "no free slot");
    size_t used = 0;
    for (auto* m : b->members) used += handle_bytes(m);
    if (used + handle_bytes(h) > b->budget) return bfail(b, USP_ERR_CAPACITY, "HBM budget exceeded");
    if (!b->members.empty() && (h->precision != b->precision || h->pipeline != b->pipeline))
        return bfail(b, USP_ERR_INVALID_ARG, "precision / pipeline differ from the batch");
    if (b->members.empty()) {
        b->precision = h->precision;
        b->pipeline = h->pipeline;
    }
    // the handle's own stream must be idle before the batch stream takes over
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bfail(b, USP_ERR_CUDA, "handle stream error");
    b->members.push_back(h);
    h->batch_refs++;
    h->batch_stream = b->stream;
    b->dirty = true;
    return USP_OK;
}

extern "C" int usp_batch_retire(usp_batch* b, usp_handle* h) {
    if (!b || !h) return USP_ERR_INVALID_ARG;
    for (size_t i = 0; i < b->members.size(); ++i) {
        if (b->members[i] != h) continue;
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, USP_ERR_CUDA, "batch stream error");
        b->members.erase(b->members.begin() + i);
        h->batch_refs--;
        h->batch_stream = nullptr;
        h->sorted = true;
        b->dirty = true;
        return USP_OK;
    }
    return bfail(b, USP_ERR_INVALID_ARG, "handle not in batch");
}

// rebuild the device tables of the batch (simulation list and tiles)
static int batch_rebuild(usp_batch* b) {
    std::vector<SimDev> sims;
    std::vector<int2> pt, ct;
    for (size_t i = 0; i < b->members.size(); ++i) {
        usp_handle* h = b->members[i];
        sims.push_back(h->host);
        for (int t = 0; t < h->nptiles; ++t) pt.push_back(make_int2((int)i, t * kPTile));
        for (int t = 0; t < h->nctiles; ++t) ct.push_back(make_int2((int)i, t * kCTile));
    }
    // the slabs of a decomposed domain must sit consecutively, in slab order,
    // each one pointing at slab 0 of its group
    for (size_t i = 0; i < sims.size(); ++i) {
        SimDev& d = sims[i];
        if (d.slab_count <= 1) continue;
        const int first = (int)i - d.slab_index;
        bool ok = first >= 0 && first + d.slab_count <= (int)sims.size();
        for (int k = 0; ok && k < d.slab_count; ++k) {
            const usp_handle* o = b->members[first + k];
            ok = o->slab_group == b->members[i]->slab_group && o->host.slab_count == d.slab_count &&
                 o->host.slab_index == k && o->host.nx == d.nx && o->host.ny == d.ny;
        }
        if (!ok) return bfail(b, USP_ERR_STATE, "the slabs of a group must be admitted together and in slab order");
        d.slab_first = first;
    }
    bool regraph = false;
    if (pt.size() > b->ptile_cap) {
        cudaFree(b->d_ptiles);
        b->ptile_cap = std::max(pt.size(), 2 * b->ptile_cap);
        if (cudaMalloc(&b->d_ptiles, sizeof(int2) * b->ptile_cap) != cudaSuccess) {
            cudaGetLastError();
            b->d_ptiles = nullptr;
            b->ptile_cap = 0;
            return bfail(b, USP_ERR_OOM, "tile table");
        }
        regraph = true;
    }
    if (ct.size() > b->ctile_cap) {
        cudaFree(b->d_ctiles);
        b->ctile_cap = std::max(ct.size(), 2 * b->ctile_cap);
        if (cudaMalloc(&b->d_ctiles, sizeof(int2) * b->ctile_cap) != cudaSuccess) {
            cudaGetLastError();
            b->d_ctiles = nullptr;
            b->ctile_cap = 0;
            return bfail(b, USP_ERR_OOM, "tile table");
        }
        regraph = true;
    }
    if ((int)sims.size() != b->graph_nsims) regraph = true;
    for (auto* h : b->members) {
        const int t = (h->host.K + kLayTile - 1) / kLayTile;
        if (t > b->lay_tiles) {   // the layout grid only grows: extra blocks find no tile
            b->lay_tiles = t;
            regraph = true;
        }
    }
    b->nptiles = (int)pt.size();
    b->nctiles = (int)ct.size();
    int nt[2] = {b->nptiles, b->nctiles};
    cudaError_t e = cudaSuccess;
    if (!sims.empty()) e = cudaMemcpyAsync(b->d_sims, sims.data(), sizeof(SimDev) * sims.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !pt.empty()) e = cudaMemcpyAsync(b->d_ptiles, pt.data(), sizeof(int2) * pt.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && !ct.empty()) e = cudaMemcpyAsync(b->d_ctiles, ct.data(), sizeof(int2) * ct.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ntiles, nt, sizeof(nt), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(b, USP_ERR_CUDA, cudaGetErrorString(e));
    if (regraph) destroy_graphs(b->graphs);
    b->dirty = false;
    return USP_OK;
}

static Launch batch_launch(usp_batch* b) {
    Launch L;
    L.sims = b->d_sims;
    L.ptiles = b->d_ptiles;
    L.nptiles = b->d_ntiles;
    L.ctiles = b->d_ctiles;
    L.nctiles = b->d_ntiles + 1;
    L.wq = (uint32_t*)(b->d_ntiles + 2);
    L.nsims = (int)b->members.size();
    L.dims = 0;
    for (auto* h : b->members) L.dims |= h->host.dim == 1 ? 1 : 2;
    for (auto* h : b->members) {
        L.slabs |= h->host.slab_count > 1;
        L.flux |= h->host.flux_axis != 0;
    }
    // fixed persistent grids: the tile counts are read on the device, so the
    // captured graph stays valid while simulations come and go
    int per_sm = 1;
    for (auto* h : b->members) per_sm = std::max(per_sm, h->grid_per_sm);
    L.grid_p = persistent_grid(1 << 30, per_sm);
    L.grid_c = persistent_grid(1 << 30, per_sm);
    L.lay_tiles = b->lay_tiles;
    L.stream = b->stream;
    return L;
}

static int batch_capture(usp_batch* b, int nsteps, cudaGraphExec_t* exec) {
    Launch L = batch_launch(b);
    const bool fp64 = b->precision == USP_FP64;
    bool res = false;
    int R = 4;
    for (auto* h : b->members) {
        res |= h->host.has_reservoir != 0;
        R = std::max(R, h->fused_R);
    }
    if (b->pipeline == USP_PIPE_FUSED && b->fork.make()) b->fork.attach(L);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, USP_ERR_CUDA, cudaGetErrorString(e));
    for (int i = 0; i < nsteps; ++i) {
        if (b->pipeline == USP_PIPE_FUSED) enqueue_fused_step(L, R, res);
        else enqueue_step(L, fp64, res);
    }
    e = cudaStreamEndCapture(b->stream, &g);
    if (e != cudaSuccess) return bfail(b, USP_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, USP_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    b->graph_nsims = (int)b->members.size();
    return USP_OK;
}

extern "C" int usp_batch_step(usp_batch* b, int nsteps) {
    if (!b || nsteps < 0) return USP_ERR_INVALID_ARG;
    if (b->members.empty() || nsteps == 0) return USP_OK;
    int rc;
    if (b->dirty && (rc = batch_rebuild(b)) != 0) return rc;
    if (!b->graphs.one && (rc = batch_capture(b, 1, &b->graphs.one)) != 0) return rc;
    if (nsteps >= kGraphSteps && !b->graphs.many && (rc = batch_capture(b, kGraphSteps, &b->graphs.many)) != 0)
        return rc;
    int left = nsteps;
    cudaError_t e = cudaSuccess;
    while (left >= kGraphSteps && e == cudaSuccess) {
        e = cudaGraphLaunch(b->graphs.many, b->stream);
        left -= kGraphSteps;
    }
    while (left-- > 0 && e == cudaSuccess) e = cudaGraphLaunch(b->graphs.one, b->stream);
    if (e != cudaSuccess) return bfail(b, USP_ERR_CUDA, cudaGetErrorString(e));
    return USP_OK;
}

extern "C" int usp_batch_destroy(usp_batch* b) {
    if (!b) return USP_ERR_INVALID_ARG;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto* h : b->members) {
        h->batch_refs--;
        h->batch_stream = nullptr;
    }
    b->members.clear();
    destroy_graphs(b->graphs);
    cudaFree(b->d_sims);
    cudaFree(b->d_ptiles);
    cudaFree(b->d_ctiles);
    cudaFree(b->d_ntiles);
    b->fork.release();
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return USP_OK;
}

// Debug / profiling: run one stage of the plain pipeline over every admitted
// simulation (same stage numbers as usp_run_stage).
extern "C" int usp_batch_run_stage(usp_batch* b, int stage) {
    if (!b) return USP_ERR_INVALID_ARG;
    if (b->members.empty()) return USP_OK;
    int rc;
    if (b->dirty && (rc = batch_rebuild(b)) != 0) return rc;
    Launch L = batch_launch(b);
    const bool fp64 = b->precision == USP_FP64;
    bool res = false;
    int R = 4;
    for (auto* h : b->members) {
        res |= h->host.has_reservoir != 0;
        R = std::max(R, h->fused_R);
    }
    if (stage_launch(L, b->pipeline, fp64, R, res, stage))
        return bfail(b, USP_ERR_INVALID_ARG, "stage must be 0..6 (plain) or 10..14 (fused)");
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? USP_OK : bfail(b, USP_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" int usp_fused_supported(void) { return 1; }

// Tuning knobs chosen by the autotuner: fused staging capacity (R = 4, 8 or
// 12, i.e. 128, 256 or 416 particles per cell pass; 0 keeps the current) and
// persistent blocks per SM (1..32; 0 keeps).  Captured graphs are rebuilt.
extern "C" int usp_set_tuning(usp_handle* h, int fused_R, int grid_per_sm) {
    if (!h) return USP_ERR_INVALID_ARG;
    if (h->batch_refs) return fail(h, USP_ERR_STATE, "handle is admitted to a batch");
    if (fused_R != 0 && fused_R != 4 && fused_R != 8 && fused_R != 12) return fail(h, USP_ERR_INVALID_ARG, "R");
    if (grid_per_sm < 0 || grid_per_sm > 32) return fail(h, USP_ERR_INVALID_ARG, "grid_per_sm");
    if (fused_R) h->fused_R = fused_R;
    if (grid_per_sm) h->grid_per_sm = grid_per_sm;
    destroy_graphs(h->graphs);
    return USP_OK;
}

extern "C" int usp_get_tuning(usp_handle* h, int* fused_R, int* grid_per_sm) {
    if (!h) return USP_ERR_INVALID_ARG;
    if (fused_R) *fused_R = h->fused_R;
    if (grid_per_sm) *grid_per_sm = h->grid_per_sm;
    return USP_OK;
}
