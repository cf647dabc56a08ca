// usp_fused.cu -- the fused FP32 pipeline of the USP-ESBGK step (sm_103a).
//
// One step n reads buffer p = cur and writes buffer q = cur ^ 1:
//   k_g2      per cell (one consumer warp, the cell's planes copied into a
//             shared-memory ring by a producer warp of the same CTA): the
//             relaxation of step n-1 still pending on the cell's particles
//             (Eqs. 8b, 9, 27, 29-32 with the per-cell momentum / energy
//             conservation), then advection of step n with the boundaries,
//             the new cell, and the write into that cell's bucket of buffer
//             q (the scatter of the counting sort; the bucket sizes come from
//             the previous histogram plus slack).
//   k_inject  reservoir buffer cells refilled into buffer q.
//   k_g1      per cell (one warp): moments of Eq. 1 in one pass, as sums
//             about the cell's mean velocity of the previous step, and the
//             cell's n, T, |u| for its neighbours' Kn_GLL.
//   k_params  per cell: Kn_GLL and P_ne (Eqs. 16-18), sigma* and q* (Eq. 33),
//             the Cholesky factor of the ES covariance (Eq. 6c), the fields
//             and the average of Eq. 34.
//   k_layout  per simulation: histogram -> bucket sizes -> exclusive scan,
//             the layout that the next step writes with; then the end of
//             the step (swap buffers, advance the step).
// All arithmetic of a step is FP32 except the number density and the Eq. 34
// running averages (FP64, in k_params_f).  FP64 issue rate is scarce on
// GB300 (about two FP64 FMA per clock per SM).  The moments are sums about
// the previous step's cell mean and the conservation factors use sums about
// the cell mean, so no subtraction cancels: the per-cell state, Eq. 33 and
// the Cholesky factor lose nothing in FP32 that the FP32 sums still carry.
// Each particle is read once and written once by k_g2 and its velocity is
// read once more by k_g1.
#include <algorithm>

#include "usp_device.cuh"

namespace usp {

namespace {

constexpr uint32_t kNoCell = 0xFFFFFFFFu;

struct FCell {
    float u[3], th, M[6], pr, nu, nues, pne;   // M = L L^T - theta I (lower triangle, row-major)
    int valid;
};

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// collect up to 32 spill-list indices of `cell` into spl (per warp); returns the count
__device__ uint32_t collect_spill(const SimDev& s, int b, int cell, uint32_t* spl, int lane) {
    const uint32_t n = min(s.dyn->sp_n[b], (uint32_t)kSpillCap);
    uint32_t found = 0;
    for (uint32_t base = 0; base < n && found < 32; base += 32) {
        const uint32_t i = base + lane;
        const bool hit = i < n && s.sp_cell[b][i] == (uint32_t)cell;
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        const uint32_t pos = found + __popc(m & lanemask_lt());
        if (hit && pos < 32) spl[pos] = i;
        found += __popc(m);
    }
    __syncwarp();
    if (found > 32) {
        if (lane == 0) atomicAdd(&s.dyn->counters[kCntOverflow], (unsigned long long)(found - 32));
        found = 32;
    }
    return found;
}

template <int DIM>
__device__ __forceinline__ void load_particle(const SimDev& s, int b, uint32_t base, uint32_t nb, const uint32_t* spl,
                                              uint32_t j, float& x, float& y, float& v0, float& v1, float& v2,
                                              uint32_t& id) {
    if (j < nb) {
        const uint32_t i = base + j;
        if (DIM == 2) x = ((const float*)s.pos[b][0])[i];
        y = ((const float*)s.pos[b][1])[i];
        v0 = ((const float*)s.vel[b][0])[i];
        v1 = ((const float*)s.vel[b][1])[i];
        v2 = ((const float*)s.vel[b][2])[i];
        id = s.pid[b][i];
    } else {
        const uint32_t i = spl[j - nb];
        if (DIM == 2) x = s.sp_pos[b][0][i];
        y = s.sp_pos[b][1][i];
        v0 = s.sp_vel[b][0][i];
        v1 = s.sp_vel[b][1][i];
        v2 = s.sp_vel[b][2][i];
        id = s.sp_pid[b][i];
    }
}

template <int DIM>
__device__ __forceinline__ void store_velocity(const SimDev& s, int b, uint32_t base, uint32_t nb, const uint32_t* spl,
                                               uint32_t j, float v0, float v1, float v2) {
    if (j < nb) {
        const uint32_t i = base + j;
        ((float*)s.vel[b][0])[i] = v0;
        ((float*)s.vel[b][1])[i] = v1;
        ((float*)s.vel[b][2])[i] = v2;
    } else {
        const uint32_t i = spl[j - nb];
        s.sp_vel[b][0][i] = v0;
        s.sp_vel[b][1][i] = v1;
        s.sp_vel[b][2][i] = v2;
    }
}

// register copy of the source buffer's planes for the particles of one cell
struct Src {
    const float* x;
    const float* y;
    const float* v0;
    const float* v1;
    const float* v2;
    const uint32_t* id;
};

__device__ __forceinline__ Src src_of(const SimDev& s, int b) {
    Src P;
    P.x = (const float*)s.pos[b][0];
    P.y = (const float*)s.pos[b][1];
    P.v0 = (const float*)s.vel[b][0];
    P.v1 = (const float*)s.vel[b][1];
    P.v2 = (const float*)s.vel[b][2];
    P.id = s.pid[b];
    return P;
}

// per-cell constants of the time-instant draw (Eq. 30)
struct TimeDraw {
    float dt, a, em1, ema, inv_nues, inv_pr;
};

// Relaxation draw from the four words of one Philox call (counter
// (pid, step, relax, 0)).  It samples the law of the FP64 path's two-call
// scheme with fewer variates:
//  * u = u01(w.x) selects the particle (u < P_relax); given the selection,
//    u / P_relax is uniform on (0, 1], so it also gives the time instant
//    of Eq. 30;
//  * the sum sqrt(s) L xi1 + sqrt((1 - s) theta) xi2 of two independent
//    Gaussians (Eqs. 31-32) is one Gaussian of covariance
//    s L L^T + (1 - s) theta I = theta I + s M, sampled through its own
//    Cholesky factor from three normals: a Box-Muller pair (w.y, w.z) and
//    one Box-Muller normal from w.w and the bits the other uniforms leave
//    unused.
__device__ __forceinline__ void es_draw1(const FCell& f, const TimeDraw& td, float u, const uint4& w, float* C) {
    const float U1 = fminf(u * td.inv_pr, 1.0f);
    const float t = td.a < 1.0f ? __logf(1.0f + U1 * td.em1) * td.inv_nues
                                : td.dt + __logf(U1 + (1.0f - U1) * td.ema) * td.inv_nues;
    const float sf = f.pne + (1.0f - f.pne) * __expf(-f.nu * t);          // Eq. 32
    float z0, z1;
    box_muller<float>(w.y, w.z, z0, z1);
    // third normal: Box-Muller on w.w and the 23 low bits that the uniforms
    // of w.x, w.y and w.z leave unused (each takes the top 23 bits)
    const uint32_t lo = (w.x & 511u) | ((w.y & 511u) << 9) | ((w.z & 31u) << 18);
    const float r2 = sqrtf(-1.3862943611198906f * __log2f(u01<float>(w.w)));
    const float z2 = r2 * __cosf(6.283185307179586f * (((float)lo + 0.5f) * 1.1920928955078125e-7f) - 3.14159265358979f);
    const float S00 = f.th + sf * f.M[0], S10 = sf * f.M[1], S11 = f.th + sf * f.M[2];
    const float S20 = sf * f.M[3], S21 = sf * f.M[4], S22 = f.th + sf * f.M[5];
    const float r0 = rsqrtf(S00);
    const float l00 = S00 * r0, l10 = S10 * r0, l20 = S20 * r0;
    const float d1 = fmaxf(S11 - l10 * l10, 1e-12f * f.th);
    const float r1 = rsqrtf(d1);
    const float l11 = d1 * r1, l21 = (S21 - l20 * l10) * r1;
    const float l22 = sqrtf(fmaxf(S22 - l20 * l20 - l21 * l21, 0.0f));
    C[0] = l00 * z0;
    C[1] = l10 * z0 + l11 * z1;
    C[2] = l20 * z0 + l21 * z1 + l22 * z2;
}

// The Gallis-Torczynski draw (Eqs. 10-11) of the SP-ESBGK ablations: a
// thermal velocity sqrt(theta) z, with z three independent normals drawn as
// in es_draw1, transformed by S = I - s B, B = ((1 - Pr)/(2 Pr)) sigma* /
// (rho theta) (symmetric; f.M holds its lower triangle) and s of Eq. 32 at
// the time instant.
__device__ __forceinline__ void es_draw_gt(const FCell& f, const TimeDraw& td, float u, const uint4& w, float* C) {
    const float U1 = fminf(u * td.inv_pr, 1.0f);
    const float t = td.a < 1.0f ? __logf(1.0f + U1 * td.em1) * td.inv_nues
                                : td.dt + __logf(U1 + (1.0f - U1) * td.ema) * td.inv_nues;
    const float sf = f.pne + (1.0f - f.pne) * __expf(-f.nu * t);          // Eq. 32
    float z0, z1;
    box_muller<float>(w.y, w.z, z0, z1);
    const uint32_t lo = (w.x & 511u) | ((w.y & 511u) << 9) | ((w.z & 31u) << 18);
    const float r2 = sqrtf(-1.3862943611198906f * __log2f(u01<float>(w.w)));
    const float z2 = r2 * __cosf(6.283185307179586f * (((float)lo + 0.5f) * 1.1920928955078125e-7f) - 3.14159265358979f);
    const float st = sqrtf(f.th);
    const float c0 = st * z0, c1 = st * z1, c2 = st * z2;
    const float b00 = f.M[0], b10 = f.M[1], b11 = f.M[2], b20 = f.M[3], b21 = f.M[4], b22 = f.M[5];
    C[0] = c0 - sf * (b00 * c0 + b10 * c1 + b20 * c2);
    C[1] = c1 - sf * (b10 * c0 + b11 * c1 + b21 * c2);
    C[2] = c2 - sf * (b20 * c0 + b21 * c1 + b22 * c2);
}

// ---------------------------------------------------------------------------
// k_g2: pending relaxation + advection + bucket scatter, as a producer /
// consumer pipeline inside each CTA.
//
// Warp 0 of a CTA is the producer.  It takes runs of kG2Run cells from the
// per-simulation queues (SimDyn::qnext), reads their bucket bounds with one
// load per lane, allocates room for each cell in a ring buffer in shared
// memory and starts bulk asynchronous copies (cp.async.bulk) of the cell's
// particle planes and of its 64-byte FP32 parameter record; the copies
// complete on the descriptor's mbarrier ("full").
//
// The other NC warps are consumers.  Each takes the next descriptor in
// order, waits for its copies and processes the cell with rolled loops over
// the staged particles (so the per-particle code appears once):
//   relax    relaxation draws of the pending step (one Philox call per
//            particle), conservation sums;
//   pass A   conservation, advection, destination cell and its slot in the
//            cell's 64-cell destination window; each particle's rank among
//            the arrivals of its slot;
//   pass B   one atomic reservation per occupied slot in the destination
//            buckets (one round trip for the whole cell);
//   writes   each particle at its slot's reserved start plus its rank, so
//            the lanes of one slot write consecutive words of one bucket.
// Then it releases the descriptor ("empty" mbarrier) and the producer may
// reuse its ring space.  While a consumer works on a cell, the copies of the
// cells behind it are in flight, so HBM latency is paid once per run of
// cells rather than several times per cell.
//
// Cells whose bucket is not 16-byte aligned (the compact layout right after
// a set-up sort) are loaded by the consumer itself; cells above the largest
// ring allocation (max_stage particles) are processed in chunks with the
// conservation sums in a first sweep and the update in a second one that
// redraws the same counter-based random numbers.
//
// Every wait on an mbarrier is bounded (kG2WaitNs of global time); a wait
// that runs out adds kG2TimeoutMark to the overflow counter of simulation 0
// and ends the warp's work, so a fault in the pipeline shows up as lost
// particles instead of a hung GPU.
// ---------------------------------------------------------------------------
// the general advection (wall and plate hits), out of line; the particle
// goes in and out by value so that the common path keeps it in registers
// (reference arguments to a call would pass through local memory)
struct AdvOut {
    float x, y, c0, c1, c2;
    int alive;
};

__device__ __noinline__ AdvOut advect_slow(const SimDev& s, uint32_t step, uint32_t pid, float x, float y, float c0,
                                           float c1, float c2) {
    float c[3] = {c0, c1, c2};
    AdvOut o;
    o.alive = advect<float>(s, step, pid, x, y, c) ? 1 : 0;
    o.x = x;
    o.y = y;
    o.c0 = c[0];
    o.c1 = c[1];
    o.c2 = c[2];
    return o;
}

// per-cell register copy of what the advection and the scatter need
struct Ctx {
    float tau, lo0, hi0, lo1, hi1, inv_dx, inv_dy, b0, b1, b2;
    int nx, nxm1, nym1, nseg, reservoir, K, cell0;   // cell0: first global cell of a slab
    float* dx_;   // destination planes
    float* dy_;
    float* dv0;
    float* dv1;
    float* dv2;
    uint32_t* did;
    const uint32_t* dlay;
    uint32_t* dcnt;
    uint32_t cap;
};

__device__ __forceinline__ void make_ctx(const SimDev& s, int q, Ctx& C) {
    C.tau = s.f_dt;
    C.lo0 = s.f_lo[0];
    C.hi0 = s.f_hi[0];
    C.lo1 = s.f_lo[1];
    C.hi1 = s.f_hi[1];
    C.inv_dx = s.f_inv_dx;
    C.inv_dy = s.f_inv_dy;
    C.b0 = s.f_bdt[0];
    C.b1 = s.f_bdt[1];
    C.b2 = s.f_bdt[2];
    C.nx = s.nx;
    C.nxm1 = s.nx - 1;
    C.nym1 = s.ny - 1;
    C.nseg = s.nseg;
    C.reservoir = s.has_reservoir;
    C.K = s.K;
    C.dx_ = (float*)s.pos[q][0];
    C.dy_ = (float*)s.pos[q][1];
    C.dv0 = (float*)s.vel[q][0];
    C.dv1 = (float*)s.vel[q][1];
    C.dv2 = (float*)s.vel[q][2];
    C.did = s.pid[q];
    C.dlay = s.lay[q];
    C.dcnt = s.cnt[q];
    C.cap = (uint32_t)s.cap;
    C.cell0 = s.row0 * s.nx;
}

// column and row of an FP32 position: floor of the scaled offset, clamped
// to the grid (1-D: ix = 0)
template <int DIM>
__device__ __forceinline__ void cell_xy(const Ctx& C, float x, float y, int& ix, int& iy) {
    iy = (int)fminf(fmaxf(floorf((y - C.lo1) * C.inv_dy), 0.0f), (float)C.nym1);
    ix = DIM == 1 ? 0 : (int)fminf(fmaxf(floorf((x - C.lo0) * C.inv_dx), 0.0f), (float)C.nxm1);
}

template <int DIM>
__device__ __forceinline__ int cell_f(const Ctx& C, float x, float y) {
    int ix, iy;
    cell_xy<DIM>(C, x, y, ix, iy);
    return DIM == 1 ? iy : iy * C.nx + ix;
}

template <int DIM>
__device__ __forceinline__ bool advect_fast(const SimDev& s, const Ctx& C, uint32_t step, uint32_t pid, float& x,
                                            float& y, float* c) {
    const float yn = y + c[1] * C.tau;
    bool inside = yn > C.lo1 && yn < C.hi1;
    float xn = x;
    if (DIM == 2) {
        xn = x + c[0] * C.tau;
        inside = inside && xn > C.lo0 && xn < C.hi0;
        for (int g = 0; g < C.nseg; ++g) {
            const float ps = (float)s.seg[g].pos;
            if ((x - ps) * (xn - ps) <= 0.0f) inside = false;
        }
    }
    if (inside) {
        y = yn;
        if (DIM == 2) x = xn;
        c[0] += C.b0;
        c[1] += C.b1;
        c[2] += C.b2;
        return true;
    }
    const AdvOut o = advect_slow(s, step, pid, x, y, c[0], c[1], c[2]);
    x = o.x;
    y = o.y;
    c[0] = o.c0;
    c[1] = o.c1;
    c[2] = o.c2;
    return o.alive != 0;
}

// append one particle to the bucket of its cell (all 32 lanes call this
// together; key == kNoCell for lanes with nothing to write)
template <int DIM>
__device__ __forceinline__ void emit_c(const SimDev& s, const Ctx& C, int b, uint32_t key, float x, float y, float v0,
                                       float v1, float v2, uint32_t id, int lane) {
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    if (key == kNoCell) return;
    const int leader = __ffs(grp) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&C.dcnt[key], (uint32_t)__popc(grp));
    base = __shfl_sync(grp, base, leader);
    const uint32_t rank = base + (uint32_t)__popc(grp & lanemask_lt());
    const uint32_t lo = C.dlay[key];
    const uint32_t hi = min(C.dlay[key + 1], C.cap);
    if (lo + rank < hi) {
        const uint32_t i = lo + rank;
        if (DIM == 2) C.dx_[i] = x;
        C.dy_[i] = y;
        C.dv0[i] = v0;
        C.dv1[i] = v1;
        C.dv2[i] = v2;
        C.did[i] = id;
    } else {
        const uint32_t k = atomicAdd(&s.dyn->sp_n[b], 1u);
        atomicAdd(&s.dyn->counters[kCntSpilled], 1ull);
        if (k < (uint32_t)kSpillCap) {
            if (DIM == 2) s.sp_pos[b][0][k] = x;
            s.sp_pos[b][1][k] = y;
            s.sp_vel[b][0][k] = v0;
            s.sp_vel[b][1][k] = v1;
            s.sp_vel[b][2][k] = v2;
            s.sp_pid[b][k] = id;
            s.sp_cell[b][k] = key;
        } else {
            atomicAdd(&s.dyn->counters[kCntOverflow], 1ull);
        }
    }
}

// Destination window of a cell: the 64 cells that its particles can reach in
// one step without leaving it (1-D: offsets -32..31; 2-D: an 8 x 8 block
// around the cell).  The warp counts its arrivals per window slot in shared
// memory, reserves each slot's range in the destination bucket with one
// global atomic, then writes; particles that land outside the window reserve
// their place one at a time.
constexpr int kWin = 64;
constexpr unsigned char kSlotNone = 0xFF;   // removed, nothing to write
constexpr unsigned char kSlotFar = 0xFE;    // outside the window
constexpr unsigned char kSlotOther = 0xFD;  // in another slab of a decomposed domain

template <int DIM>
__device__ __forceinline__ int win_slot_xy(int ix, int iy, int cell, int cx, int cy) {
    if (DIM == 1) {
        const int o = iy - cell + 32;
        return (o >= 0 && o < kWin) ? o : -1;
    }
    const int oy = iy - cy + 4, ox = ix - cx + 4;
    return ((unsigned)oy < 8u && (unsigned)ox < 8u) ? oy * 8 + ox : -1;
}

template <int DIM>
__device__ __forceinline__ int win_cell(int k, int cell, int cx, int cy, int nx) {
    if (DIM == 1) return cell + k - 32;
    return (cy + (k >> 3) - 4) * nx + (cx + (k & 7) - 4);
}

// a particle that crossed into another slab of a decomposed domain: its
// place is reserved in that slab's bucket (or spill list) of buffer q, all
// slabs of a domain stepping together
template <int DIM>
__device__ __noinline__ void emit_other(const SimDev* __restrict__ sims, const SimDev& s, int q, float x, float y,
                                        float v0, float v1, float v2, uint32_t id) {
    const float fy = fminf(fmaxf(floorf((y - s.f_lo[1]) * s.f_inv_dy), 0.0f), (float)(s.ny - 1));
    const int row = (int)fy;
    int gc = row;
    if (DIM == 2) gc = row * s.nx + (int)fminf(fmaxf(floorf((x - s.f_lo[0]) * s.f_inv_dx), 0.0f), (float)(s.nx - 1));
    const SimDev& o = sims[s.slab_first + row / s.rows];
    const int dc = gc - o.row0 * o.nx;
    const uint32_t i = o.lay[q][dc] + atomicAdd(&o.cnt[q][dc], 1u);
    const uint32_t hi = min(o.lay[q][dc + 1], (uint32_t)o.cap);
    if (i < hi) {
        if (DIM == 2) ((float*)o.pos[q][0])[i] = x;
        ((float*)o.pos[q][1])[i] = y;
        ((float*)o.vel[q][0])[i] = v0;
        ((float*)o.vel[q][1])[i] = v1;
        ((float*)o.vel[q][2])[i] = v2;
        o.pid[q][i] = id;
        return;
    }
    const uint32_t k = atomicAdd(&o.dyn->sp_n[q], 1u);
    atomicAdd(&o.dyn->counters[kCntSpilled], 1ull);
    if (k < (uint32_t)kSpillCap) {
        if (DIM == 2) o.sp_pos[q][0][k] = x;
        o.sp_pos[q][1][k] = y;
        o.sp_vel[q][0][k] = v0;
        o.sp_vel[q][1][k] = v1;
        o.sp_vel[q][2][k] = v2;
        o.sp_pid[q][k] = id;
        o.sp_cell[q][k] = (uint32_t)dc;
    } else {
        atomicAdd(&o.dyn->counters[kCntOverflow], 1ull);
    }
}

// write a particle into slot i of its own simulation's destination bucket
// (buffer q), or into the spill list when the bucket is full (dc: its cell)
template <int DIM>
__device__ __forceinline__ void put_own(const SimDev& s, const Ctx& C, int q, uint32_t i, uint32_t hi, int dc, float x,
                                        float y, float v0, float v1, float v2, uint32_t id) {
    if (i < hi) {
        if (DIM == 2) C.dx_[i] = x;
        C.dy_[i] = y;
        C.dv0[i] = v0;
        C.dv1[i] = v1;
        C.dv2[i] = v2;
        C.did[i] = id;
        return;
    }
    const uint32_t k = atomicAdd(&s.dyn->sp_n[q], 1u);
    atomicAdd(&s.dyn->counters[kCntSpilled], 1ull);
    if (k < (uint32_t)kSpillCap) {
        if (DIM == 2) s.sp_pos[q][0][k] = x;
        s.sp_pos[q][1][k] = y;
        s.sp_vel[q][0][k] = v0;
        s.sp_vel[q][1][k] = v1;
        s.sp_vel[q][2][k] = v2;
        s.sp_pid[q][k] = id;
        s.sp_cell[q][k] = (uint32_t)dc;
    } else {
        atomicAdd(&s.dyn->counters[kCntOverflow], 1ull);
    }
}

// kFullSlab: kFull for batches holding slabs of a decomposed domain (routes
// particles that leave the slab; the plain kFull code carries no such check).
// kFullFlux: kFull for batches where some simulation counts particles
// through a plane (kFullSlab counts too).  kRelaxOnly applies the pending
// relaxation in place (before the particles are read back).
enum { kFull = 0, kRelaxOnly = 1, kFullSlab = 2, kFullFlux = 3 };

// ---- pipeline constants ----------------------------------------------------
constexpr int kG2Desc = 32;            // descriptors (cells in flight) per CTA
constexpr int kG2Run = 16;             // cells taken from a queue at once by the producer
constexpr int kG2Spill = 32;           // spill-list entries a cell may add to its bucket
constexpr unsigned long long kG2WaitNs = 2000000000ull;   // bound of one mbarrier wait
constexpr unsigned long long kG2TimeoutMark = 1ull << 40;

enum : uint32_t { kDescBulk = 1u, kDescPending = 2u, kDescParity = 4u };

// One cell handed from the producer to a consumer.  prm is filled by a bulk
// copy of the cell's parameter record; the rest by the producer.
struct alignas(16) G2Desc {
    float prm[kNFPrm];   // u[3], theta, L[6], P_relax, nu, nu_ES, P_ne, valid, spare
    uint32_t base;       // first slot of the cell's bucket in buffer p
    uint32_t nb;         // particles in the bucket (arrivals beyond it are in the spill list)
    uint32_t arrived;    // arrivals into the cell (bucket + spill list)
    uint32_t off;        // byte offset of the cell's area in the ring
    uint32_t m;          // particle slots of that area
    int cell;            // -1: no more cells for this consumer
    int ent;             // simulation descriptor entry in shared memory
    uint32_t step;       // step counter of the simulation (Philox word 1)
    uint32_t flags;      // kDesc*
    uint32_t end;        // ring counter after this allocation (producer bookkeeping)
};

// bytes of ring per staged particle: (x,) y, v0, v1, v2, id; slot; rank
template <int DIM>
__host__ __device__ constexpr uint32_t g2_bytes_per_particle() {
    return (DIM == 2 ? 24u : 20u) + 1u + 2u;
}

struct G2Stage {
    float* x;
    float* y;
    float* v0;
    float* v1;
    float* v2;
    uint32_t* id;
    unsigned char* sel;
    uint16_t* rank;
};

template <int DIM>
__device__ __forceinline__ G2Stage g2_stage(unsigned char* ring, uint32_t off, uint32_t m) {
    float* f = (float*)(ring + off);
    G2Stage S;
    S.x = nullptr;
    if (DIM == 2) {
        S.x = f;
        f += m;
    }
    S.y = f;
    S.v0 = f + m;
    S.v1 = f + 2 * m;
    S.v2 = f + 3 * m;
    S.id = (uint32_t*)(f + 4 * m);
    S.sel = (unsigned char*)(f + 5 * m);
    S.rank = (uint16_t*)(S.sel + m);
    return S;
}

// ---- mbarrier and bulk-copy primitives (PTX, sm_90+) ----------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t tx) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
                 "r"(tx)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase of `bar` with the given parity to complete, at most
// kG2WaitNs; false when the bound ran out
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 64; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kG2WaitNs) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// order this thread's generic-proxy accesses to shared memory before later
// bulk copies (async proxy) into the same bytes
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ void g2_timeout(const SimDev* __restrict__ sims) {
    atomicAdd(&sims[0].dyn->counters[kCntOverflow], kG2TimeoutMark);
}

// counters a consumer accumulates in registers and adds once per simulation
struct G2Acc {
    unsigned long long relaxed, removed;
};

__device__ __forceinline__ void g2_flush(G2Acc& a, SimDyn* dyn, int lane) {
    if (dyn && lane == 0) {
        if (a.relaxed) atomicAdd(&dyn->counters[kCntRelaxed], a.relaxed);
        if (a.removed) atomicAdd(&dyn->counters[kCntRemoved], a.removed);
    }
    a.relaxed = a.removed = 0;
}

// ---- consumer: one cell ------------------------------------------------------
// conservation sums over the relaxed subset of a cell: old peculiar
// velocities about the cell mean (a) and new peculiar velocities (b)
struct G2Sums {
    float a0, a1, a2, ae, b0, b1, b2, be, nr;
};

// per-cell factors of the momentum / energy correction
struct G2Cons {
    float uo0, uo1, uo2, mn0, mn1, mn2, alpha;
    bool apply;
};

// staged particles [0, cnt) of a cell area from their bucket (at bucket
// index off) and spill-list entries; with `have_bucket` the bucket part is
// already there (bulk copy)
template <int DIM>
__device__ __forceinline__ void g2_load(const SimDev& s, const G2Stage& S, int p, uint32_t base, uint32_t nb,
                                        const uint32_t* spl, uint32_t off, uint32_t cnt, bool have_bucket, int lane) {
    const uint32_t mb = off < nb ? min(cnt, nb - off) : 0u;
    __syncwarp();
    if (!have_bucket) {
        const Src P = src_of(s, p);
#pragma unroll 2
        for (uint32_t j = lane; j < mb; j += 32) {
            const uint32_t i = base + off + j;
            if (DIM == 2) S.x[j] = P.x[i];
            S.y[j] = P.y[i];
            S.v0[j] = P.v0[i];
            S.v1[j] = P.v1[i];
            S.v2[j] = P.v2[i];
            S.id[j] = P.id[i];
        }
    }
#pragma unroll 1
    for (uint32_t j = mb + lane; j < cnt; j += 32) {
        float x = 0.0f, y, v0, v1, v2;
        uint32_t id;
        load_particle<DIM>(s, p, base, nb, spl, off + j, x, y, v0, v1, v2, id);
        if (DIM == 2) S.x[j] = x;
        S.y[j] = y; S.v0[j] = v0; S.v1[j] = v1; S.v2[j] = v2; S.id[j] = id;
    }
    __syncwarp();
}

// Relaxation draws of the staged particles [0, cnt): a relaxed particle
// gets its new peculiar velocity in v0..v2 and sel = 1 (else sel = 0);
// with SUMS the conservation sums of the relaxed subset are accumulated.
// The cell's FP32 parameters live only in this scope.
template <bool SUMS>
__device__ __forceinline__ void g2_relax(const float* prm, const SimDev& s, const G2Stage& S, uint32_t cnt,
                                         uint32_t step, bool relax, int lane, G2Sums& R) {
    FCell f;
#pragma unroll
    for (int d = 0; d < 3; ++d) f.u[d] = prm[d];
    f.th = prm[3];
    {   // M = L L^T - theta I from the FP64-built factor L
        const float L0 = prm[4], L1 = prm[5], L2 = prm[6], L3 = prm[7], L4 = prm[8], L5 = prm[9];
        f.M[0] = L0 * L0 - f.th;
        f.M[1] = L1 * L0;
        f.M[2] = L1 * L1 + L2 * L2 - f.th;
        f.M[3] = L3 * L0;
        f.M[4] = L3 * L1 + L4 * L2;
        f.M[5] = L3 * L3 + L4 * L4 + L5 * L5 - f.th;
    }
    f.pr = prm[10];
    f.nu = prm[11];
    f.nues = prm[12];
    f.pne = prm[13];
    TimeDraw td;
    td.dt = s.f_dt;
    td.a = f.nues * td.dt;
    td.em1 = expm1f(td.a);
    td.ema = __expf(-td.a);
    td.inv_nues = 1.0f / f.nues;
    td.inv_pr = f.pr > 0.0f ? 1.0f / f.pr : 0.0f;
    const uint2 key = make_uint2(s.key0, s.key1);
#pragma unroll 1
    for (uint32_t j0 = lane; j0 < cnt; j0 += 64) {
        const uint32_t j1 = j0 + 32;
        const bool has1 = j1 < cnt;
        unsigned char s0 = 0, s1 = 0;
        if (relax) {
            const uint32_t id0 = S.id[j0];
            const uint32_t id1 = has1 ? S.id[j1] : 0u;
            const uint4 w0 = philox(make_uint4(id0, step, kRelax, 0), key);
            const uint4 w1 = philox(make_uint4(id1, step, kRelax, 0), key);
            const float x0 = u01<float>(w0.x), x1 = u01<float>(w1.x);
            s0 = x0 < f.pr;
            s1 = has1 && x1 < f.pr;
            if (s0 | s1) {
                float C0[3], C1[3];
                es_draw1(f, td, x0, w0, C0);
                es_draw1(f, td, x1, w1, C1);
                if (s0) {
                    if (SUMS) {
                        const float o0 = S.v0[j0] - f.u[0], o1 = S.v1[j0] - f.u[1], o2 = S.v2[j0] - f.u[2];
                        R.a0 += o0; R.a1 += o1; R.a2 += o2;
                        R.ae += o0 * o0 + o1 * o1 + o2 * o2;
                        R.b0 += C0[0]; R.b1 += C0[1]; R.b2 += C0[2];
                        R.be += C0[0] * C0[0] + C0[1] * C0[1] + C0[2] * C0[2];
                        R.nr += 1.0f;
                    }
                    S.v0[j0] = C0[0]; S.v1[j0] = C0[1]; S.v2[j0] = C0[2];
                }
                if (s1) {
                    if (SUMS) {
                        const float o0 = S.v0[j1] - f.u[0], o1 = S.v1[j1] - f.u[1], o2 = S.v2[j1] - f.u[2];
                        R.a0 += o0; R.a1 += o1; R.a2 += o2;
                        R.ae += o0 * o0 + o1 * o1 + o2 * o2;
                        R.b0 += C1[0]; R.b1 += C1[1]; R.b2 += C1[2];
                        R.be += C1[0] * C1[0] + C1[1] * C1[1] + C1[2] * C1[2];
                        R.nr += 1.0f;
                    }
                    S.v0[j1] = C1[0]; S.v1[j1] = C1[1]; S.v2[j1] = C1[2];
                }
            }
        }
        S.sel[j0] = s0;
        if (has1) S.sel[j1] = s1;
    }
    __syncwarp();
}

// Eq. 9 fixed count for one cell: the ns = nearest-int(n P_relax) particles
// with the smallest selection words w.x (ties: lower staged position).  T is
// the ns-th smallest word and `quota` the number of particles with word T
// that are taken; the (ns+1)-th smallest word T2 scales the time instants
// (given T2, the ns smallest words are independent and uniform below it).
struct G2Fixed {
    uint32_t T, quota, ties, ns;
    float inv_thr;
};

// the words of the staged particles [0, cnt) one chunk at a time: the
// radix select of the ns-th smallest (four passes of 8-bit digits counted
// in the warp's window array), then the ties and T2.  Cells above the
// ring allocation reload each chunk in every pass.
template <int DIM>
__device__ __noinline__ G2Fixed g2_fixed(const SimDev& s, const G2Desc& D, const G2Stage& S, uint32_t n,
                                          const uint32_t* spl, uint32_t* hist, int lane) {
    const int p = (D.flags & kDescParity) ? 1 : 0;
    const uint32_t m = D.m, nch = (n + m - 1) / m;
    const uint2 key = make_uint2(s.key0, s.key1);
    G2Fixed F;
    F.ns = (uint32_t)floorf((float)n * D.prm[10] + 0.5f);
    F.ns = min(F.ns, n);
    F.ties = 0;
    F.T = 0xFFFFFFFFu;
    F.quota = 0;
    F.inv_thr = 1.0f;
    if (F.ns == 0) return F;
    uint32_t prefix = 0, mask = 0, rem = F.ns;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int b = lane; b < 256; b += 32) hist[b] = 0u;
        __syncwarp();
        for (uint32_t ch = 0; ch < nch; ++ch) {
            const uint32_t cnt = min(m, n - ch * m);
            if (nch > 1) g2_load<DIM>(s, S, p, D.base, D.nb, spl, ch * m, cnt, false, lane);
            for (uint32_t j = lane; j < cnt; j += 32) {
                const uint32_t k = philox(make_uint4(S.id[j], D.step, kRelax, 0), key).x;
                if ((k & mask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
            }
            __syncwarp();
        }
        // lane l holds digits [8l, 8l + 8): the digit where the running count reaches rem
        uint32_t h[8], tot = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            h[i] = hist[8 * lane + i];
            tot += h[i];
        }
        uint32_t inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t exc = inc - tot;
        const unsigned own = __ballot_sync(0xffffffffu, exc < rem && rem <= inc);
        const int L = __ffs(own) - 1;
        uint32_t d = 0, below = exc;
        if (lane == L) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if (below + h[i] >= rem) {
                    d = 8u * lane + i;
                    break;
                }
                below += h[i];
            }
        }
        d = __shfl_sync(0xffffffffu, d, L);
        below = __shfl_sync(0xffffffffu, below, L);
        rem -= below;
        prefix |= d << shift;
        mask |= 0xFFu << shift;
        __syncwarp();
    }
    F.T = prefix;
    F.quota = rem;
    // words equal to T, and the smallest word above it
    uint32_t eq = 0, above = 0xFFFFFFFFu;
    bool any_above = false;
    for (uint32_t ch = 0; ch < nch; ++ch) {
        const uint32_t cnt = min(m, n - ch * m);
        if (nch > 1) g2_load<DIM>(s, S, p, D.base, D.nb, spl, ch * m, cnt, false, lane);
        for (uint32_t j = lane; j < cnt; j += 32) {
            const uint32_t k = philox(make_uint4(S.id[j], D.step, kRelax, 0), key).x;
            eq += k == F.T;
            if (k > F.T) {
                any_above = true;
                above = min(above, k);
            }
        }
    }
    eq = __reduce_add_sync(0xffffffffu, eq);
    above = __reduce_min_sync(0xffffffffu, above);
    any_above = __any_sync(0xffffffffu, any_above);
    uint32_t T2 = 0;
    bool has2 = true;
    if (eq > F.quota) T2 = F.T;
    else if (any_above) T2 = above;
    else has2 = false;
    F.inv_thr = has2 ? 1.0f / u01<float>(T2) : 1.0f;
    return F;
}

// Relaxation draws of the SP-ESBGK ablations (same contract as g2_relax):
// the Bernoulli or fixed-count selection (Eq. 9), the ES Cholesky or
// Gallis-Torczynski sampler (Eqs. 10-11).  The loop is warp-uniform so
// that the ties of the fixed count are ranked by position with ballots.
template <bool SUMS>
__device__ __forceinline__ void g2_relax_abl(const float* prm, const SimDev& s, const G2Stage& S, uint32_t cnt,
                                             uint32_t step, bool relax, int lane, G2Sums& R, G2Fixed& X) {
    FCell f;
#pragma unroll
    for (int d = 0; d < 3; ++d) f.u[d] = prm[d];
    f.th = prm[3];
    const bool gt = s.es_sampler != 0, fixed = s.selection != 0;
    if (gt) {   // B of Eq. 11 (lower triangle)
#pragma unroll
        for (int k = 0; k < 6; ++k) f.M[k] = prm[4 + k];
    } else {
        const float L0 = prm[4], L1 = prm[5], L2 = prm[6], L3 = prm[7], L4 = prm[8], L5 = prm[9];
        f.M[0] = L0 * L0 - f.th;
        f.M[1] = L1 * L0;
        f.M[2] = L1 * L1 + L2 * L2 - f.th;
        f.M[3] = L3 * L0;
        f.M[4] = L3 * L1 + L4 * L2;
        f.M[5] = L3 * L3 + L4 * L4 + L5 * L5 - f.th;
    }
    f.pr = prm[10];
    f.nu = prm[11];
    f.nues = prm[12];
    f.pne = prm[13];
    TimeDraw td;
    td.dt = s.f_dt;
    td.a = f.nues * td.dt;
    td.em1 = expm1f(td.a);
    td.ema = __expf(-td.a);
    td.inv_nues = 1.0f / f.nues;
    td.inv_pr = fixed ? X.inv_thr : (f.pr > 0.0f ? 1.0f / f.pr : 0.0f);
    const uint2 key = make_uint2(s.key0, s.key1);
    const unsigned lt = lanemask_lt();
#pragma unroll 1
    for (uint32_t b = 0; b < cnt; b += 32) {
        const uint32_t j = b + lane;
        const bool has = j < cnt;
        bool sel = false;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (relax) {
            w = philox(make_uint4(has ? S.id[j] : 0u, step, kRelax, 0), key);
            if (fixed) {
                const bool tie = has && w.x == X.T;
                const unsigned tb = __ballot_sync(0xffffffffu, tie);
                const uint32_t rank = X.ties + (uint32_t)__popc(tb & lt);
                X.ties += (uint32_t)__popc(tb);
                sel = has && X.ns > 0 && (w.x < X.T || (tie && rank < X.quota));
            } else {
                sel = has && u01<float>(w.x) < f.pr;
            }
            if (sel) {
                float C[3];
                const float u = u01<float>(w.x);
                if (gt) es_draw_gt(f, td, u, w, C);
                else es_draw1(f, td, u, w, C);
                if (SUMS) {
                    const float o0 = S.v0[j] - f.u[0], o1 = S.v1[j] - f.u[1], o2 = S.v2[j] - f.u[2];
                    R.a0 += o0; R.a1 += o1; R.a2 += o2;
                    R.ae += o0 * o0 + o1 * o1 + o2 * o2;
                    R.b0 += C[0]; R.b1 += C[1]; R.b2 += C[2];
                    R.be += C[0] * C[0] + C[1] * C[1] + C[2] * C[2];
                    R.nr += 1.0f;
                }
                S.v0[j] = C[0]; S.v1[j] = C[1]; S.v2[j] = C[2];
            }
        }
        if (has) S.sel[j] = sel ? 1 : 0;
    }
    __syncwarp();
}

// conservation factors of the cell from the warp's partial sums
__device__ __forceinline__ G2Cons g2_factors(const float* prm, G2Sums R, bool relax, G2Acc& acc) {
    G2Cons K;
    K.apply = false;
    K.uo0 = K.uo1 = K.uo2 = K.mn0 = K.mn1 = K.mn2 = 0.0f;
    K.alpha = 1.0f;
    if (!relax) return K;
    const float nr = warp_sumf(R.nr);
    if (nr < 2.0f) return K;
    const float a0 = warp_sumf(R.a0), a1 = warp_sumf(R.a1), a2 = warp_sumf(R.a2), ae = warp_sumf(R.ae);
    const float b0 = warp_sumf(R.b0), b1 = warp_sumf(R.b1), b2 = warp_sumf(R.b2), be = warp_sumf(R.be);
    // FP32: the sums are taken about the cell mean, so the differences
    // below do not cancel.  The butterfly sums are bitwise the same on
    // every lane (each stage adds the same two values), so every lane
    // computes the same factors without a broadcast.
    const float inv = 1.0f / nr;
    const float Eo = ae - (a0 * a0 + a1 * a1 + a2 * a2) * inv;
    const float En = be - (b0 * b0 + b1 * b1 + b2 * b2) * inv;
    if (En > 0.0f && Eo >= 0.0f) {
        K.apply = true;
        K.alpha = sqrtf(Eo / En);
        K.uo0 = prm[0] + a0 * inv;
        K.uo1 = prm[1] + a1 * inv;
        K.uo2 = prm[2] + a2 * inv;
        K.mn0 = b0 * inv;
        K.mn1 = b1 * inv;
        K.mn2 = b2 * inv;
        acc.relaxed += (unsigned long long)(unsigned)nr;
    }
    return K;
}

// the relaxed velocity of staged particle j (conservation applied), or its
// old velocity when the cell had a single relaxed particle (reverted)
template <int DIM>
__device__ __forceinline__ void g2_velocity(const SimDev& s, const G2Stage& S, const G2Cons& K, int p, uint32_t base,
                                            uint32_t nb, const uint32_t* spl, uint32_t off, uint32_t j, float* c) {
    c[0] = S.v0[j];
    c[1] = S.v1[j];
    c[2] = S.v2[j];
    if (S.sel[j]) {
        if (K.apply) {
            c[0] = K.uo0 + K.alpha * (c[0] - K.mn0);
            c[1] = K.uo1 + K.alpha * (c[1] - K.mn1);
            c[2] = K.uo2 + K.alpha * (c[2] - K.mn2);
        } else {
            float ox, oy;
            uint32_t oid;
            load_particle<DIM>(s, p, base, nb, spl, off + j, ox, oy, c[0], c[1], c[2], oid);
        }
    }
}

// relaxed velocities written back in place (MODE kRelaxOnly)
template <int DIM>
__device__ __forceinline__ void g2_store_relaxed(const SimDev& s, const G2Stage& S, const G2Cons& K, int p,
                                                 uint32_t base, uint32_t nb, const uint32_t* spl, uint32_t off,
                                                 uint32_t cnt, int lane) {
    if (!K.apply) return;
#pragma unroll 1
    for (uint32_t j = lane; j < cnt; j += 32) {
        if (!S.sel[j]) continue;
        float c[3];
        g2_velocity<DIM>(s, S, K, p, base, nb, spl, off, j, c);
        store_velocity<DIM>(s, p, base, nb, spl, off + j, c[0], c[1], c[2]);
    }
    __syncwarp();
}

// passes A, B and the write pass over the staged particles [0, cnt)
template <int DIM, int MODE>
__device__ __forceinline__ void g2_move(const SimDev* __restrict__ sims, const SimDev& s, const G2Stage& S,
                                        const G2Cons& K, int cell, int p, uint32_t base, uint32_t nb,
                                        const uint32_t* spl, uint32_t off, uint32_t cnt, uint32_t step,
                                        uint32_t* win, int lane, uint32_t& removed) {
    const int q = p ^ 1;
    Ctx C;
    make_ctx(s, q, C);
    const int cy = DIM == 2 ? cell / C.nx : 0;
    const int cx = DIM == 2 ? cell - cy * C.nx : 0;
    const int gcell = cell + (MODE == kFullSlab && DIM == 1 ? C.cell0 : 0);   // 1-D: global cell of the slab's cell
    const int row0 = MODE == kFullSlab && DIM == 2 ? s.row0 : 0;
    uint32_t* wcnt = win;              // arrivals per window slot
    uint32_t* wstart = win + kWin;     // first reserved index of each slot in its bucket
    uint32_t* wend = win + 2 * kWin;   // end of that bucket
    wcnt[lane] = 0;
    wcnt[lane + 32] = 0;
    __syncwarp();
    // pass A: conservation, advection, destination slot, rank in the slot
#pragma unroll 1
    for (uint32_t b = 0; b < cnt; b += 32) {
        const uint32_t j = b + lane;
        int slot = -2;   // -2: nothing to count
        if (j < cnt) {
            float x = DIM == 2 ? S.x[j] : 0.0f, y = S.y[j], c[3];
            g2_velocity<DIM>(s, S, K, p, base, nb, spl, off, j, c);
            unsigned char ws = kSlotNone;
            if (advect_fast<DIM>(s, C, step, S.id[j], x, y, c)) {
                int ix, iy;
                cell_xy<DIM>(C, x, y, ix, iy);
                const int dc = (DIM == 2 ? iy * C.nx + ix : iy) - (MODE == kFullSlab ? C.cell0 : 0);   // local
                if (MODE == kFullSlab && (unsigned)dc >= (unsigned)C.K) {
                    ws = kSlotOther;
                } else if (!C.reservoir || !in_buffer(s, dc)) {
                    slot = win_slot_xy<DIM>(ix, iy - row0, gcell, cx, cy);
                    ws = slot >= 0 ? (unsigned char)slot : kSlotFar;
                } else {
                    ++removed;
                }
            }
            if ((MODE == kFullFlux || MODE == kFullSlab) && s.flux_axis)
                count_flux<float>(s, DIM == 2 ? S.x[j] : 0.0f, S.y[j], x, y);
            if (DIM == 2) S.x[j] = x;
            S.y[j] = y; S.v0[j] = c[0]; S.v1[j] = c[1]; S.v2[j] = c[2];
            S.sel[j] = ws;
        }
        // the particle's rank among the arrivals of its slot: one shared
        // atomic (lanes of one slot are served one after another)
        if (slot >= 0) S.rank[j] = (uint16_t)atomicAdd(&wcnt[slot], 1u);
    }
    __syncwarp();
    // pass B: one reservation per occupied slot, all in flight together
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = lane + 32 * h;
        const uint32_t cntk = wcnt[k];
        if (cntk) {
            const int dest = win_cell<DIM>(k, cell, cx, cy, C.nx);
            const uint32_t r = atomicAdd(&C.dcnt[dest], cntk);
            wstart[k] = C.dlay[dest] + r;
            wend[k] = min(C.dlay[dest + 1], C.cap);
        }
    }
    __syncwarp();
    // write pass: consecutive lanes write particles of the same few
    // destination buckets (a window slot's particles go to consecutive
    // slots of its bucket, in rank order); particles leaving the window or
    // the slab take their own reservation
#pragma unroll 1
    for (uint32_t j = lane; j < cnt; j += 32) {
        const unsigned char ws = S.sel[j];
        if (ws == kSlotNone) continue;
        const float x = DIM == 2 ? S.x[j] : 0.0f, y = S.y[j];
        if (ws < kWin) {
            const uint32_t i = wstart[ws] + S.rank[j];
            const uint32_t hi = wend[ws];
            const int dc = i < hi ? 0 : cell_f<DIM>(C, x, y) - (MODE == kFullSlab ? C.cell0 : 0);
            put_own<DIM>(s, C, q, i, hi, dc, x, y, S.v0[j], S.v1[j], S.v2[j], S.id[j]);
        } else if (MODE == kFullSlab && ws == kSlotOther) {   // into the buckets of another slab
            emit_other<DIM>(sims, s, q, x, y, S.v0[j], S.v1[j], S.v2[j], S.id[j]);
        } else {   // outside the window: a reservation of its own
            const int dc = cell_f<DIM>(C, x, y) - (MODE == kFullSlab ? C.cell0 : 0);
            const uint32_t i = C.dlay[dc] + atomicAdd(&C.dcnt[dc], 1u);
            const uint32_t hi = min(C.dlay[dc + 1], C.cap);
            put_own<DIM>(s, C, q, i, hi, dc, x, y, S.v0[j], S.v1[j], S.v2[j], S.id[j]);
        }
    }
    __syncwarp();
}

// a cell above the largest ring area: conservation sums in a first sweep
// over its chunks, the update in a second sweep that reloads each chunk and
// redraws the same counter-based random numbers
template <int DIM, int MODE>
__device__ __noinline__ void g2_cell_chunked(const SimDev* __restrict__ sims, const SimDev& s, const G2Desc& D,
                                             const G2Stage& S, uint32_t n, bool relax, const uint32_t* spl,
                                             uint32_t* win, int lane, G2Acc& acc) {
    const int p = (D.flags & kDescParity) ? 1 : 0;
    const uint32_t m = D.m, nch = (n + m - 1) / m;
    const bool abl = s.selection | s.es_sampler;
    G2Fixed X = {0u, 0u, 0u, 0u, 1.0f};
    if (relax && s.selection) X = g2_fixed<DIM>(s, D, S, n, spl, win, lane);
    G2Sums R = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t ch = 0; ch < nch; ++ch) {
        const uint32_t cnt = min(m, n - ch * m);
        g2_load<DIM>(s, S, p, D.base, D.nb, spl, ch * m, cnt, false, lane);
        if (abl) g2_relax_abl<true>(D.prm, s, S, cnt, D.step, relax, lane, R, X);
        else g2_relax<true>(D.prm, s, S, cnt, D.step, relax, lane, R);
    }
    const G2Cons K = g2_factors(D.prm, R, relax, acc);
    uint32_t removed = 0;
    X.ties = 0;
    for (uint32_t ch = 0; ch < nch; ++ch) {
        const uint32_t cnt = min(m, n - ch * m);
        g2_load<DIM>(s, S, p, D.base, D.nb, spl, ch * m, cnt, false, lane);
        if (abl) g2_relax_abl<false>(D.prm, s, S, cnt, D.step, relax, lane, R, X);
        else g2_relax<false>(D.prm, s, S, cnt, D.step, relax, lane, R);
        if (MODE == kRelaxOnly) g2_store_relaxed<DIM>(s, S, K, p, D.base, D.nb, spl, ch * m, cnt, lane);
        else g2_move<DIM, MODE>(sims, s, S, K, D.cell, p, D.base, D.nb, spl, ch * m, cnt, D.step, win, lane, removed);
    }
    if (s.has_reservoir) acc.removed += __reduce_add_sync(0xffffffffu, removed);
}

template <int DIM, int MODE>
__device__ __forceinline__ void g2_cell(const SimDev* __restrict__ sims, const SimDev& s, const G2Desc& D,
                                        unsigned char* ring, uint32_t* win, uint32_t* spl, int lane, G2Acc& acc) {
    const int p = (D.flags & kDescParity) ? 1 : 0;
    uint32_t nsp = 0;
    if (D.arrived > D.nb) nsp = collect_spill(s, p, D.cell, spl, lane);
    const uint32_t n = D.nb + nsp;
    if (n == 0) return;
    const bool relax = (D.flags & kDescPending) && D.prm[14] != 0.0f;
    if (MODE == kRelaxOnly && !relax) return;
    const G2Stage S = g2_stage<DIM>(ring, D.off, D.m);
    if (n > D.m) {
        g2_cell_chunked<DIM, MODE>(sims, s, D, S, n, relax, spl, win, lane, acc);
        return;
    }
    g2_load<DIM>(s, S, p, D.base, D.nb, spl, 0u, n, (D.flags & kDescBulk) != 0, lane);
    G2Sums R = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (s.selection | s.es_sampler) {   // the SP-ESBGK ablations
        G2Fixed X = {0u, 0u, 0u, 0u, 1.0f};
        if (relax && s.selection) X = g2_fixed<DIM>(s, D, S, n, spl, win, lane);
        g2_relax_abl<true>(D.prm, s, S, n, D.step, relax, lane, R, X);
    } else {
        g2_relax<true>(D.prm, s, S, n, D.step, relax, lane, R);
    }
    const G2Cons K = g2_factors(D.prm, R, relax, acc);
    if (MODE == kRelaxOnly) {
        g2_store_relaxed<DIM>(s, S, K, p, D.base, D.nb, spl, 0u, n, lane);
        return;
    }
    uint32_t removed = 0;
    g2_move<DIM, MODE>(sims, s, S, K, D.cell, p, D.base, D.nb, spl, 0u, n, D.step, win, lane, removed);
    if (s.has_reservoir) acc.removed += __reduce_add_sync(0xffffffffu, removed);
}

// copy one simulation descriptor into shared memory (one warp)
__device__ __forceinline__ void load_sim_warp(SimDev& dst, const SimDev& src, int lane) {
    const int4* a = reinterpret_cast<const int4*>(&src);
    int4* b = reinterpret_cast<int4*>(&dst);
    for (int i = lane; i < (int)(sizeof(SimDev) / 16); i += 32) b[i] = a[i];
}

// next simulation with cells left in its queue, after `from` (32 candidates
// per round); -1 when every queue of this dimension is empty
template <int DIM>
__device__ __forceinline__ int find_sim(const SimDev* __restrict__ sims, int nsims, int from, int lane) {
    for (int base = 0; base < nsims; base += 32) {
        const int k = base + lane;
        bool ok = false;
        int idx = 0;
        if (k < nsims) {
            idx = from + 1 + k;
            if (idx >= nsims) idx -= nsims;
            const SimDev& c = sims[idx];
            ok = c.dim == DIM && __ldcg(&c.dyn->qnext) < (uint32_t)c.K;
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (m) return __shfl_sync(0xffffffffu, idx, __ffs(m) - 1);
    }
    return -1;
}

// shared state of one CTA of k_g2
template <int NC>
struct G2Shared {
    SimDev sim[2];                 // simulation descriptors in use (the producer alternates)
    G2Desc desc[kG2Desc];
    uint64_t full[kG2Desc];        // copies of a descriptor landed (producer arrive + bytes)
    uint64_t empty[kG2Desc];       // consumer done with a descriptor
    uint32_t win[NC][4 * kWin];
    uint32_t spl[NC][32];
    uint32_t take;                 // next descriptor for a consumer
};

// ---- producer --------------------------------------------------------------
template <int DIM, int MODE, int NC>
__device__ void g2_producer(const SimDev* __restrict__ sims, int nsims, G2Shared<NC>& sh, unsigned char* ring,
                            uint32_t ring_bytes, uint32_t max_stage, int lane) {
    constexpr uint32_t bpp = g2_bytes_per_particle<DIM>();
    constexpr int NP = DIM == 2 ? 6 : 5;   // planes
    uint32_t seq = 0, oldest = 0;          // descriptors issued / reclaimed
    uint32_t head = 0, tail = 0;           // ring bytes allocated / freed (monotonic)
    uint32_t last_use[2] = {0u, 0u};
    bool used[2] = {false, false};
    int ent = 1;
    bool ok = true;

    // reclaim the oldest descriptor once its consumer released it
    auto reclaim = [&]() -> bool {
        const uint32_t slot = oldest % kG2Desc;
        if (!mbar_wait(&sh.empty[slot], (oldest / kG2Desc) & 1u)) return false;
        tail = sh.desc[slot].end;
        ++oldest;
        return true;
    };
    // a free descriptor and `bytes` of contiguous ring; returns the ring offset
    auto reserve = [&](uint32_t bytes, uint32_t& off) -> bool {
        while (seq - oldest >= (uint32_t)kG2Desc)
            if (!reclaim()) return false;
        for (;;) {
            const uint32_t pos = head % ring_bytes;
            // an allocation never wraps: with no room before the end it starts at offset 0
            const uint32_t start = pos + bytes > ring_bytes ? head + (ring_bytes - pos) : head;
            if (start + bytes - tail <= ring_bytes) {
                head = start;
                off = start % ring_bytes;
                return true;
            }
            if (oldest == seq) {   // empty ring: restart it at the chosen offset
                head = tail = start;
            } else if (!reclaim()) {
                return false;
            }
        }
    };

    int h = (int)(blockIdx.x % (unsigned)nsims);
    if (sims[h].dim != DIM) h = find_sim<DIM>(sims, nsims, h, lane);
    while (h >= 0 && ok) {
        const int e = ent ^ 1;
        if (used[e])
            while (ok && oldest <= last_use[e]) ok = reclaim();
        if (!ok) break;
        __syncwarp();
        load_sim_warp(sh.sim[e], sims[h], lane);
        __syncwarp();
        const SimDev& s = sh.sim[e];
        const int p = s.dyn->cur;
        const uint32_t step = s.dyn->step;
        const bool pending = s.dyn->relax_pending != 0;
        const uint32_t K = (uint32_t)s.K;
        if (MODE == kRelaxOnly && !pending) {   // nothing to apply: close its queue
            if (lane == 0) atomicMax(&s.dyn->qnext, K);
            h = find_sim<DIM>(sims, nsims, h, lane);
            continue;
        }
        ent = e;
        // bulk copies need 16-byte aligned planes (and buckets)
        uintptr_t al = (uintptr_t)s.pos[p][1] | (uintptr_t)s.vel[p][0] | (uintptr_t)s.vel[p][1] |
                       (uintptr_t)s.vel[p][2] | (uintptr_t)s.pid[p] | (uintptr_t)s.fprm;
        if (DIM == 2) al |= (uintptr_t)s.pos[p][0];
        const bool planes_aligned = (al & 15u) == 0;
        const uint32_t flags0 = (pending ? kDescPending : 0u) | (p ? kDescParity : 0u);
        const uint32_t cap = (uint32_t)s.cap;
        for (;;) {
            uint32_t c0 = 0;
            if (lane == 0) c0 = atomicAdd(&s.dyn->qnext, (uint32_t)kG2Run);
            c0 = __shfl_sync(0xffffffffu, c0, 0);
            if (c0 >= K) break;
            uint32_t lo = 0, hi = 0, ar = 0;
            if (lane < kG2Run && c0 + lane < K) {
                lo = s.lay[p][c0 + lane];
                hi = min(s.lay[p][c0 + lane + 1], cap);
                ar = s.cnt[p][c0 + lane];
            }
            const uint32_t nrun = min((uint32_t)kG2Run, K - c0);
            for (uint32_t i = 0; i < nrun && ok; ++i) {
                const uint32_t bs = __shfl_sync(0xffffffffu, lo, i);
                const uint32_t tp = __shfl_sync(0xffffffffu, hi, i);
                const uint32_t arv = __shfl_sync(0xffffffffu, ar, i);
                const uint32_t capc = tp > bs ? tp - bs : 0u;
                const uint32_t nb = min(arv, capc);
                const bool spill = arv > nb;
                if (nb == 0 && !spill) continue;
                const uint32_t need = nb + (spill ? (uint32_t)kG2Spill : 0u);
                const bool chunked = need > max_stage;
                const uint32_t m = chunked ? max_stage : ((need + 3u) & ~3u);
                const uint32_t bytes = (bpp * m + 15u) & ~15u;
                const bool bulk = !chunked && planes_aligned && (bs & 3u) == 0 && nb > 0 &&
                                  bs + ((nb + 3u) & ~3u) <= cap;
                uint32_t off = 0;
                if (!reserve(bytes, off)) {
                    ok = false;
                    break;
                }
                const uint32_t slot = seq % kG2Desc;
                G2Desc& d = sh.desc[slot];
                if (lane == 0) {
                    d.base = bs;
                    d.nb = nb;
                    d.arrived = arv;
                    d.off = off;
                    d.m = m;
                    d.cell = (int)(c0 + i);
                    d.ent = e;
                    d.step = step;
                    d.flags = flags0 | (bulk ? kDescBulk : 0u);
                    d.end = head + bytes;
                    const uint32_t nb4 = (nb + 3u) & ~3u;
                    mbar_arrive_tx(&sh.full[slot], 64u + (bulk ? (uint32_t)NP * 4u * nb4 : 0u));
                    bulk_g2s(d.prm, s.fprm + (size_t)(c0 + i) * kNFPrm, 64u, &sh.full[slot]);
                    if (bulk) {
                        unsigned char* dst = ring + off;
                        const uint32_t pb = 4u * m;   // bytes of one staged plane
                        int k = 0;
                        if (DIM == 2) bulk_g2s(dst + pb * k++, (const float*)s.pos[p][0] + bs, 4u * nb4, &sh.full[slot]);
                        bulk_g2s(dst + pb * k++, (const float*)s.pos[p][1] + bs, 4u * nb4, &sh.full[slot]);
                        bulk_g2s(dst + pb * k++, (const float*)s.vel[p][0] + bs, 4u * nb4, &sh.full[slot]);
                        bulk_g2s(dst + pb * k++, (const float*)s.vel[p][1] + bs, 4u * nb4, &sh.full[slot]);
                        bulk_g2s(dst + pb * k++, (const float*)s.vel[p][2] + bs, 4u * nb4, &sh.full[slot]);
                        bulk_g2s(dst + pb * k, s.pid[p] + bs, 4u * nb4, &sh.full[slot]);
                    }
                }
                __syncwarp();
                head += bytes;
                last_use[e] = seq;
                used[e] = true;
                ++seq;
            }
        }
        if (!ok) break;
        h = find_sim<DIM>(sims, nsims, h, lane);
    }
    // one end marker per consumer (they take descriptors in order)
    for (int k = 0; k < NC && ok; ++k) {
        uint32_t off;
        if (!reserve(0u, off)) {
            ok = false;
            break;
        }
        const uint32_t slot = seq % kG2Desc;
        if (lane == 0) {
            sh.desc[slot].cell = -1;
            sh.desc[slot].end = head;
            mbar_arrive(&sh.full[slot]);
        }
        __syncwarp();
        ++seq;
    }
    if (!ok) {
        if (lane == 0) g2_timeout(sims);
        // copies still in flight land before the CTA may exit
        for (uint32_t t = oldest; t < seq; ++t) mbar_wait(&sh.full[t % kG2Desc], (t / kG2Desc) & 1u);
    }
}

template <int DIM, int MODE, int NC>
__global__ void __launch_bounds__(32 * (NC + 1), 16 / (NC + 1)) k_g2(const SimDev* __restrict__ sims, int nsims,
                                                     uint32_t* __restrict__ wq, uint32_t ring_bytes,
                                                     uint32_t max_stage) {
    extern __shared__ __align__(128) unsigned char g2_ring[];
    __shared__ G2Shared<NC> sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kG2Desc; ++i) {
            mbar_init(&sh.full[i], 1);
            mbar_init(&sh.empty[i], 1);
        }
        sh.take = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        g2_producer<DIM, MODE, NC>(sims, nsims, sh, g2_ring, ring_bytes, max_stage, lane);
    } else {
        uint32_t* win = sh.win[warp - 1];
        uint32_t* spl = sh.spl[warp - 1];
        G2Acc acc = {0ull, 0ull};
        SimDyn* acc_dyn = nullptr;
        for (;;) {
            uint32_t my = 0;
            if (lane == 0) my = atomicAdd(&sh.take, 1u);
            my = __shfl_sync(0xffffffffu, my, 0);
            const uint32_t slot = my % kG2Desc;
            if (!mbar_wait(&sh.full[slot], (my / kG2Desc) & 1u)) {
                if (lane == 0) g2_timeout(sims);
                break;
            }
            const G2Desc& D = sh.desc[slot];
            if (D.cell < 0) break;
            const SimDev& s = sh.sim[D.ent];
            if (s.dyn != acc_dyn) {
                g2_flush(acc, acc_dyn, lane);
                acc_dyn = s.dyn;
            }
            g2_cell<DIM, MODE>(sims, s, D, g2_ring, win, spl, lane, acc);
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh.empty[slot]);
        }
        g2_flush(acc, acc_dyn, lane);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&wq[0], 1u);
        if (done == gridDim.x - 1) {   // the last CTA resets the queues for the next launch
            wq[0] = 0;
            for (int i = 0; i < nsims; ++i) sims[i].dyn->qnext = 0;
        }
    }
}


// ---------------------------------------------------------------------------
// k_g1: per-cell moments (Eq. 1) in one pass, as sums of C = c - u_s about a
// shift u_s: the cell's mean velocity of the previous step (the parameters
// of that step, still in fprm).  The mean moves little in one step, so the
// FP32 sums of the centred velocities do not cancel; k_params_f promotes
// them to FP64 with the shift taken into account.
// ---------------------------------------------------------------------------
constexpr int kG1Warps = 4;     // warps per block; a block takes one 32-cell tile at a time
constexpr int kG1Stage = 384;   // slots of one pipeline stage (a multiple of 4)

// per-lane asynchronous global -> shared copies (completion waited with
// cp.async.wait_group by the issuing lane, then made visible to the warp
// with __syncwarp)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__global__ void __launch_bounds__(32 * kG1Warps) k_g1(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                     const int* __restrict__ ntiles) {
    __shared__ uint32_t spl_all[kG1Warps][32];
    // the tile's per-cell headers, fetched in one round for all 32 cells:
    // bucket start, particles in the bucket, arrivals, and the shift u_s
    __shared__ uint32_t h_base[kCTile], h_nb[kCTile], h_arr[kCTile];
    __shared__ float4 h_us[kCTile];
    // each warp's two pipeline stages of the three velocity planes
    __shared__ __align__(16) float stage[kG1Warps][2][3][kG1Stage];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ SimDev sim_sh;
    const int nt = *ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        __syncthreads();
        load_sim(sim_sh, sims[tile.x]);
        __syncthreads();
        const SimDev& s = sim_sh;
        const int K = s.K;
        const int q = s.dyn->cur ^ 1;
        if (threadIdx.x < kCTile && tile.y + (int)threadIdx.x < K) {
            const int cell = tile.y + (int)threadIdx.x;
            const uint32_t base = s.lay[q][cell];
            const uint32_t top = min(s.lay[q][cell + 1], (uint32_t)s.cap);
            const uint32_t capc = top > base ? top - base : 0u;
            const uint32_t arrived = s.cnt[q][cell];
            h_base[threadIdx.x] = base;
            h_nb[threadIdx.x] = min(arrived, capc);
            h_arr[threadIdx.x] = arrived;
            h_us[threadIdx.x] = reinterpret_cast<const float4*>(s.fprm)[(size_t)cell * (kNFPrm / 4)];
        }
        __syncthreads();
        const float* V0 = (const float*)s.vel[q][0];
        const float* V1 = (const float*)s.vel[q][1];
        const float* V2 = (const float*)s.vel[q][2];
        // The warp's cells (cc = warp, warp + kG1Warps, ...) are read as a
        // sequence of chunks of at most kG1Stage slots, each copied into one
        // of two stages while the chunk before it is summed: a cell's whole
        // bucket is in flight at once, and its round trip overlaps the
        // previous chunk's work.  (c, o) is the next chunk to copy.
        auto live = [&](int c) { return c < kCTile && tile.y + c < K; };
        auto copy_chunk = [&](int c, uint32_t o, int b) {
            const uint32_t g = h_base[c] + o;
            const uint32_t len = min(h_nb[c] - o, (uint32_t)kG1Stage);
            float* d0 = stage[warp][b][0];
            float* d1 = stage[warp][b][1];
            float* d2 = stage[warp][b][2];
            if ((g & 3u) == 0u) {
                // 16-byte groups up to the next multiple of four slots: the
                // bucket start and the capacity are multiples of four, so the
                // copy stays inside the plane
                const uint32_t n4 = (len + 3u) >> 2;
                for (uint32_t k = lane; k < n4; k += 32) {
                    cp_async16(d0 + 4 * k, V0 + g + 4 * k);
                    cp_async16(d1 + 4 * k, V1 + g + 4 * k);
                    cp_async16(d2 + 4 * k, V2 + g + 4 * k);
                }
            } else {   // the compact layout right after a set-up sort
                for (uint32_t k = lane; k < len; k += 32) {
                    cp_async4(d0 + k, V0 + g + k);
                    cp_async4(d1 + k, V1 + g + k);
                    cp_async4(d2 + k, V2 + g + k);
                }
            }
            cp_async_commit();
        };
        // the chunk after (c, o), skipping cells with an empty bucket
        auto advance = [&](int& c, uint32_t& o) {
            o += kG1Stage;
            if (o < h_nb[c]) return;
            o = 0;
            c += kG1Warps;
            while (live(c) && h_nb[c] == 0) c += kG1Warps;
        };
        int ic = warp;
        uint32_t io = 0;
        while (live(ic) && h_nb[ic] == 0) ic += kG1Warps;
        if (live(ic)) copy_chunk(ic, io, 0);
        int done = 0;   // chunks summed so far (stage done & 1 holds the next)
        for (int cc = warp; live(cc); cc += kG1Warps) {
            const int cell = tile.y + cc;
            const uint32_t nb = h_nb[cc];
            const uint32_t arrived = h_arr[cc];
            const float4 us = h_us[cc];
            const float u0 = us.x, u1 = us.y, u2 = us.z;
            uint32_t nsp = 0;
            if (arrived > nb) nsp = collect_spill(s, q, cell, spl_all[warp], lane);
            const uint32_t n = nb + nsp;
            float S[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) S[k] = 0.0f;
            auto add = [&](float a, float b, float c) {
                const float C0 = a - u0, C1 = b - u1, C2 = c - u2;
                const float c2 = C0 * C0 + C1 * C1 + C2 * C2;
                S[0] += C0; S[1] += C1; S[2] += C2;
                S[3] += C0 * C0; S[4] += C1 * C1; S[5] += C2 * C2;
                S[6] += C0 * C1; S[7] += C0 * C2; S[8] += C1 * C2;
                S[9] += c2 * C0; S[10] += c2 * C1; S[11] += c2 * C2;
            };
            for (uint32_t o = 0; o < nb; o += kG1Stage) {
                // (ic, io) is this chunk: copy the next one, then wait for this one
                advance(ic, io);
                if (live(ic)) {
                    copy_chunk(ic, io, (done + 1) & 1);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncwarp();
                const float* b0 = stage[warp][done & 1][0];
                const float* b1 = stage[warp][done & 1][1];
                const float* b2 = stage[warp][done & 1][2];
                const uint32_t len = min(nb - o, (uint32_t)kG1Stage);
#pragma unroll 4
                for (uint32_t j = lane; j < len; j += 32) add(b0[j], b1[j], b2[j]);
                __syncwarp();   // the stage is refilled by the copy issued two chunks on
                ++done;
            }
            for (uint32_t j = nb + lane; j < n; j += 32) {   // spill-list entries of the cell
                const uint32_t i = spl_all[warp][j - nb];
                add(s.sp_vel[q][0][i], s.sp_vel[q][1][i], s.sp_vel[q][2][i]);
            }
            // The cell's 64-byte record [N, 12 sums, shift u_s] as a warp
            // reduce-scatter: at each of four halving stages a lane keeps half
            // of its values and adds the partner's copy of that half (16
            // shuffles instead of 60 for twelve butterfly sums); lane 2v then
            // holds entry v of the record and writes it.  N and u_s come from
            // lane 0 alone.  FP32 sums only: their promotion to FP64 happens in
            // k_params_f, one cell per thread (an FP64 instruction costs the
            // same for one lane).
            float v[16];
            v[0] = lane == 0 ? (float)n : 0.0f;
#pragma unroll
            for (int k = 0; k < 12; ++k) v[1 + k] = S[k];
            v[13] = lane == 0 ? u0 : 0.0f;
            v[14] = lane == 0 ? u1 : 0.0f;
            v[15] = lane == 0 ? u2 : 0.0f;
#pragma unroll
            for (int half = 8; half >= 1; half >>= 1) {
                const bool up = (lane & (2 * half)) != 0;
#pragma unroll
                for (int i = 0; i < half; ++i) {
                    const float send = up ? v[i] : v[i + half];
                    const float recv = __shfl_xor_sync(0xffffffffu, send, 2 * half);
                    v[i] = (up ? v[i + half] : v[i]) + recv;
                }
            }
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
            if ((lane & 1) == 0) s.momf[(size_t)cell * 16 + (lane >> 1)] = v[0];   // one 64-byte record per cell
            // the totals of the first six sums (entries 1..6, on lanes 2..12) for the local state
#pragma unroll
            for (int k = 0; k < 6; ++k) S[k] = __shfl_sync(0xffffffffu, v[0], 2 * (k + 1));
            if (lane == 31) {
                // local state of the cell for its neighbours' Kn_GLL (FP32):
                // the instantaneous one, or the Eq. 34 average as it stood at
                // the start of the step (k_params_f updates it later)
                float nn = (float)n * s.f_w, T = 0.0f, um = 0.0f, valid = 0.0f;
                if (s.gll_average && s.dyn->nsamples > 0) {
                    const int K = s.K;
                    const double a1 = s.avg[(size_t)1 * K + cell], a2 = s.avg[(size_t)2 * K + cell],
                                 a3 = s.avg[(size_t)3 * K + cell];
                    nn = (float)s.avg[cell];
                    T = (float)s.avg[(size_t)4 * K + cell];
                    um = (float)sqrt(a1 * a1 + a2 * a2 + a3 * a3);
                    valid = nn > 0.0f && T > 0.0f ? 1.0f : 0.0f;
                } else if (n >= 2) {
                    const float inv2 = 1.0f / (float)n;
                    const float d0 = S[0] * inv2, d1 = S[1] * inv2, d2 = S[2] * inv2;
                    const float th = ((S[3] + S[4] + S[5]) * inv2 - (d0 * d0 + d1 * d1 + d2 * d2)) * (1.0f / 3.0f);
                    if (th > 0.0f) {
                        valid = 1.0f;
                        T = th * s.f_inv_R;
                        const float w0 = u0 + d0, w1 = u1 + d1, w2 = u2 + d2;
                        um = sqrtf(w0 * w0 + w1 * w1 + w2 * w2);
                    }
                }
                reinterpret_cast<float4*>(s.floc)[cell] = make_float4(nn, T, um, valid);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_params_f: per-cell parameters; FP64 for the stress tensor, Eq. 33 and the
// Cholesky factor, FP32 for viscosity, mean free path, Kn_GLL and P_ne
// ---------------------------------------------------------------------------
struct LocalF {
    int valid, N;
    float n, T, umag;
};

// the cell's state from its FP32 shifted sums: mean velocity, pressure
// tensor per unit density (P / rho) and theta = R T; inv = 1 / N.  The sums
// are about the previous mean, so the subtractions below do not cancel and
// FP32 keeps the accuracy the FP32 sums carry.
__device__ __forceinline__ void local_f(const SimDev& s, const float* M, LocalF& L, float* u, float* P, float* theta,
                                        float& inv) {
    const int N = (int)M[0];
    L.N = N;
    L.valid = 0;
    L.n = (float)N * s.f_w;
    L.T = 0;
    L.umag = 0;
    inv = 0.0f;
    if (N < 1) return;
    inv = 1.0f / (float)N;
    const float d0 = M[1] * inv, d1 = M[2] * inv, d2 = M[3] * inv;
    u[0] = M[13] + d0; u[1] = M[14] + d1; u[2] = M[15] + d2;
    P[0] = M[4] * inv - d0 * d0;
    P[1] = M[5] * inv - d1 * d1;
    P[2] = M[6] * inv - d2 * d2;
    P[3] = M[7] * inv - d0 * d1;
    P[4] = M[8] * inv - d0 * d2;
    P[5] = M[9] * inv - d1 * d2;
    const float th = (P[0] + P[1] + P[2]) * (1.0f / 3.0f);
    *theta = th;
    L.valid = N >= 2 && th > 0.0f;
    if (!L.valid) return;
    L.T = th * s.f_inv_R;
    L.umag = sqrtf(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

// neighbour state for the Kn_GLL stencil, written in FP32 by k_g1
__device__ __forceinline__ void local_nb(const SimDev& s, int cell, LocalF& L) {
    const float4 f = reinterpret_cast<const float4*>(s.floc)[cell];
    L.n = f.x;
    L.T = f.y;
    L.umag = f.z;
    L.valid = f.w != 0.0f;
    L.N = 0;
}

// state of the neighbour of `cell` along `axis` (dir = -1 / +1) for the
// Kn_GLL stencil; across a slab boundary it is the adjacent slab's row.
// Returns whether the neighbour exists and is valid.
__device__ __forceinline__ bool nb_state(const SimDev* __restrict__ sims, const SimDev& s, int cell, int axis, int dir,
                                         LocalF& L) {
    const int ix = cell % s.nx, iy = cell / s.nx;
    const SimDev* t = &s;
    int c;
    if (axis == 0) {
        int j = ix + dir;
        if (j < 0 || j >= s.nx) {
            if (!s.periodic_x) return false;
            j = (j + s.nx) % s.nx;
        }
        c = iy * s.nx + j;
    } else {
        int gj = s.row0 + iy + dir;   // global row
        if (gj < 0 || gj >= s.ny) {
            if (!s.periodic_y) return false;
            gj = (gj + s.ny) % s.ny;
        }
        const int r = gj - s.row0;
        if (r >= 0 && r < s.rows) {
            c = r * s.nx + ix;
        } else {
            t = &sims[s.slab_first + gj / s.rows];
            c = (gj - t->row0) * s.nx + ix;
        }
    }
    local_nb(*t, c, L);
    return L.valid != 0;
}

__global__ void __launch_bounds__(128) k_params_f(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                  const int* __restrict__ ntiles) {
    __shared__ SimDev sim_sh;
    const int nt = *ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        __syncthreads();
        load_sim(sim_sh, sims[tile.x]);
        __syncthreads();
        const SimDev& s = sim_sh;
        const int K = s.K;
        for (int cc = threadIdx.x; cc < kCTile; cc += blockDim.x) {
            const int cell = tile.y + cc;
            if (cell >= K) break;
            // every load of the cell first (one round of latency): the
            // running averages, the neighbours' states for the stencil, then
            // the cell's own sums
            const bool first = s.dyn->nsamples == 0;
            double av[kNFields];
#pragma unroll
            for (int k = 0; k < kNFields; ++k) av[k] = first ? 0.0 : s.avg[(size_t)k * K + cell];
            LocalF Nm[2] = {}, Np[2] = {};
            bool hm[2] = {false, false}, hp[2] = {false, false};
            if (s.mode == kModeUSP) {
                for (int axis = s.dim == 1 ? 1 : 0; axis < 2; ++axis) {
                    hm[axis] = nb_state(sims, s, cell, axis, -1, Nm[axis]);
                    hp[axis] = nb_state(sims, s, cell, axis, +1, Np[axis]);
                }
            }
            LocalF L;
            const float* M = s.momf + (size_t)cell * 16;   // N, 12 sums, shift[3]
            float u[3] = {0, 0, 0}, P[6], th = 0, inv;
            local_f(s, M, L, u, P, &th, inv);
            float f[kNFields];
            for (int k = 0; k < kNFields; ++k) f[k] = 0.0f;
            f[0] = L.n;
            f[15] = (float)L.N;
            if (L.N >= 1) {
                f[1] = u[0]; f[2] = u[1]; f[3] = u[2];
            }
            float pr[kNFPrm];
            for (int k = 0; k < kNFPrm; ++k) pr[k] = 0.0f;
            pr[0] = u[0]; pr[1] = u[1]; pr[2] = u[2];
            pr[3] = th;
            if (L.valid) {
                const float thf = th;
                const float rho = L.n * (float)s.mass;
                const float pf = rho * thf;
                const float mu = (float)s.mu_ref * __powf(L.T / (float)s.T_ref, (float)s.omega);   // Eq. 35
                const float nu = pf / mu;
                const float lam = 1.2766152f * mu / sqrtf(rho * pf);     // Eq. 36: 16 / (5 sqrt(2 pi))
                float pne;
                if (s.mode == kModeSP || s.mode == kModeSPESBGK) pne = 0.0f;
                else if (s.mode == kModeFixed) pne = (float)s.fixed_pne;
                else {
                    // the cell's own stencil state: instantaneous, or the
                    // Eq. 34 average (loaded above, before this step's update)
                    float gn = L.n, gT = L.T, gu = L.umag, glam = lam, ga = sqrtf((float)kGammaMono * thf);
                    bool gvalid = true;
                    if (s.gll_average && !first) {
                        gn = (float)av[0];
                        gT = (float)av[4];
                        gu = (float)sqrt(av[1] * av[1] + av[2] * av[2] + av[3] * av[3]);
                        gvalid = gn > 0.0f && gT > 0.0f;
                        if (gvalid) {
                            const float gth = gT * (float)s.R;
                            const float grho = gn * (float)s.mass;
                            const float gmu = (float)s.mu_ref * __powf(gT / (float)s.T_ref, (float)s.omega);
                            glam = 1.2766152f * gmu / sqrtf(grho * grho * gth);   // Eq. 36 at the averaged state
                            ga = sqrtf((float)kGammaMono * gth);
                        }
                    }
                    // the gradients are taken relative to the cell's own value
                    // (|grad Q| / Q): absolute density gradients (~1e25 m^-3 over
                    // sub-micron cells) would overflow FP32 when squared
                    const float a_s = ga;
                    const float Qc[3] = {gn, gT, gu};
                    const float rq[3] = {1.0f / gn, 1.0f / gT, 1.0f / fmaxf(gu, a_s)};
                    float g2[3] = {0, 0, 0};
                    for (int axis = s.dim == 1 ? 1 : 0; axis < 2; ++axis) {
                        const float h = (float)(axis == 0 ? s.dx : s.dy);
                        const LocalF& Lm = Nm[axis];
                        const LocalF& Lp = Np[axis];
                        const int m = hm[axis] ? 1 : -1;
                        const int p = hp[axis] ? 1 : -1;
                        const float Qm[3] = {Lm.n, Lm.T, Lm.umag}, Qp[3] = {Lp.n, Lp.T, Lp.umag};
                        for (int k = 0; k < 3; ++k) {
                            float d = 0.0f;
                            if (m >= 0 && p >= 0) d = (Qp[k] - Qm[k]) * rq[k] / (2.0f * h);
                            else if (p >= 0) d = (Qp[k] - Qc[k]) * rq[k] / h;
                            else if (m >= 0) d = (Qc[k] - Qm[k]) * rq[k] / h;
                            g2[k] += d * d;
                        }
                    }
                    const float kn = gvalid ? glam * sqrtf(fmaxf(g2[0], fmaxf(g2[1], g2[2]))) : 0.0f;
                    pne = __expf(-kn / (float)kKnC);                                              // Eqs. 16-18
                }
                // Eq. 33
                const float ifs = 1.0f / (1.0f + 0.5f * s.f_dt * nu * pne);
                const float ifq = 1.0f / (1.0f + 0.5f * s.f_dt * nu * (float)s.Pr * pne);
                const float sig[6] = {(P[0] - th) * ifs, (P[1] - th) * ifs, (P[2] - th) * ifs, P[3] * ifs, P[4] * ifs,
                                      P[5] * ifs};
                const float b = (float)s.es_b;                                                  // Eq. 6c
                const float A00 = th + b * sig[0], A11 = th + b * sig[1], A22 = th + b * sig[2];
                const float A10 = b * sig[3], A20 = b * sig[4], A21 = b * sig[5];
                float l00 = 0, l10 = 0, l11 = 0, l20 = 0, l21 = 0, l22 = 0;
                bool ok = A00 > 0.0f;
                if (s.es_sampler) {
                    // Gallis-Torczynski (Eq. 11): B = ((1 - Pr)/(2 Pr)) sigma* / (rho theta)
                    // in the factor's slots, lower triangle row-major
                    const float beta = (1.0f - (float)s.Pr) / (2.0f * (float)s.Pr * th);
                    l00 = beta * sig[0]; l10 = beta * sig[3]; l11 = beta * sig[1];
                    l20 = beta * sig[4]; l21 = beta * sig[5]; l22 = beta * sig[2];
                    ok = true;
                } else if (ok) {
                    const float r0 = rsqrtf(A00);
                    l00 = A00 * r0;
                    l10 = A10 * r0;
                    l20 = A20 * r0;
                    const float d1 = A11 - l10 * l10;
                    ok = d1 > 0.0f;
                    if (ok) {
                        const float r1 = rsqrtf(d1);
                        l11 = d1 * r1;
                        l21 = (A21 - l20 * l10) * r1;
                        const float d2 = A22 - l20 * l20 - l21 * l21;
                        ok = d2 > 0.0f;
                        if (ok) l22 = d2 * rsqrtf(d2);
                    }
                }
                if (!ok) {
                    const float r = sqrtf(th);
                    l00 = l11 = l22 = r;
                    l10 = l20 = l21 = 0.0f;
                    atomicAdd(&s.dyn->counters[kCntChol], 1ull);
                }
                const float nues = (float)s.Pr * nu;
                pr[4] = l00; pr[5] = l10; pr[6] = l11;
                pr[7] = l20; pr[8] = l21; pr[9] = l22;
                pr[10] = -expm1f(-nues * s.f_dt);                                             // Eqs. 8b, 9
                // the decay rate of Eq. 32; the SP-ESBGK step holds its target
                // for the whole step (Eq. 8b): with P_ne = 0 a rate of 0 gives s = 1
                pr[11] = s.mode == kModeSPESBGK ? 0.0f : nu;
                pr[12] = nues;
                pr[13] = pne;
                pr[14] = 1.0f;
                // heat flux from the third central moment of the shifted sums
                const float d0 = M[1] * inv, d1 = M[2] * inv, d2 = M[3] * inv;
                const float m00 = M[4] * inv, m11 = M[5] * inv, m22 = M[6] * inv;
                const float m01 = M[7] * inv, m02 = M[8] * inv, m12 = M[9] * inv;
                const float t0 = M[10] * inv, t1 = M[11] * inv, t2 = M[12] * inv;
                const float tr = m00 + m11 + m22, dd = d0 * d0 + d1 * d1 + d2 * d2;
                const float Q0 = 0.5f * (t0 - d0 * tr - 2.0f * (m00 * d0 + m01 * d1 + m02 * d2) + 2.0f * d0 * dd);
                const float Q1 = 0.5f * (t1 - d1 * tr - 2.0f * (m01 * d0 + m11 * d1 + m12 * d2) + 2.0f * d1 * dd);
                const float Q2 = 0.5f * (t2 - d2 * tr - 2.0f * (m02 * d0 + m12 * d1 + m22 * d2) + 2.0f * d2 * dd);
                const float rhod = rho, pd = pf;
                f[4] = L.T;
                f[5] = pd + rhod * sig[0];
                f[6] = pd + rhod * sig[1];
                f[7] = pd + rhod * sig[2];
                f[8] = rhod * sig[3];
                f[9] = rhod * sig[4];
                f[10] = rhod * sig[5];
                f[11] = rhod * Q0 * ifq;
                f[12] = rhod * Q1 * ifq;
                f[13] = rhod * Q2 * ifq;
                f[14] = pne;
            }
            {   // one 64-byte parameter record per cell
                float4* dst = reinterpret_cast<float4*>(s.fprm) + (size_t)cell * (kNFPrm / 4);
#pragma unroll
                for (int k = 0; k < kNFPrm / 4; ++k) dst[k] = make_float4(pr[4 * k], pr[4 * k + 1], pr[4 * k + 2], pr[4 * k + 3]);
            }
            // the number density in FP64 (N w exactly as the FP64 paths form
            // it: a closed box keeps its domain total to the last bit)
            const double n_d = (double)L.N * s.w;
#pragma unroll
            for (int k = 0; k < kNFields; ++k) {
                const double fk = k == 0 ? n_d : (double)f[k];
                s.inst[(size_t)k * K + cell] = fk;
                s.avg[(size_t)k * K + cell] = first ? fk : s.avg_keep * av[k] + fk * s.avg_new;   // Eq. 34, FP64
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_inject_f: reservoir buffer cells, written into buffer q
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(256) k_inject_f(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                  const int* __restrict__ ntiles) {
    __shared__ SimDev sim_sh;
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        __syncthreads();
        load_sim(sim_sh, sims[tile.x]);
        __syncthreads();
        const SimDev& s = sim_sh;
        if (!s.has_reservoir || s.dim != DIM) continue;
        const uint32_t step = s.dyn->step, next_pid = s.dyn->next_pid;
        const int q = s.dyn->cur ^ 1;
        Ctx C;
        make_ctx(s, q, C);
        for (int cc = warp; cc < kCTile; cc += 8) {
            const int cell = tile.y + cc;
            if (cell >= s.K) break;
            const uint32_t cnt = s.inj_count[cell];
            if (cnt == 0) continue;
            const FaceDev& F = s.face[buffer_face(s, cell)];
            for (uint32_t k0 = 0; k0 < cnt; k0 += 32) {
                const uint32_t k = k0 + lane;
                uint32_t key = kNoCell;
                float x = 0, y = 0, c[3] = {0, 0, 0};
                uint32_t pid = 0;
                if (k < cnt) {
                    pid = next_pid + s.inj_pidoff[cell] + k;
                    make_particle<float>(s, cell, pid, step, kInject, F.theta, F.u, x, y, c);
                    key = (uint32_t)cell;
                }
                emit_c<DIM>(s, C, q, key, x, y, c[0], c[1], c[2], pid, lane);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// k_layout: histogram -> bucket sizes (slack for arrivals) -> exclusive scan
// setup == true builds the write layout of buffer cur ^ 1 right after the
// initial fill (counts of buffer cur from the exact start offsets).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bucket_size(const SimDev& s, const uint32_t* cnt, int c) {
    const int ix = c % s.nx, iy = c / s.nx;
    uint32_t m = 0;
    for (int dy = -1; dy <= 1; ++dy) {
        const int jy = iy + dy;
        if (jy < 0 || jy >= s.ny) continue;
        for (int dx = (s.dim == 2 ? -1 : 0); dx <= (s.dim == 2 ? 1 : 0); ++dx) {
            const int jx = ix + dx;
            if (jx < 0 || jx >= s.nx) continue;
            m = max(m, cnt[jy * s.nx + jx]);
        }
    }
    // a multiple of four slots, so that every bucket starts on a 16-byte
    // boundary (the bulk copies of k_g2 need it)
    return (m + (m >> 2) + 16u + (s.has_reservoir ? s.inj_count[c] : 0u) + 3u) & ~3u;
}

template <bool SETUP>
__global__ void __launch_bounds__(1024) k_layout(const SimDev* __restrict__ sims, int nsims) {
    __shared__ uint32_t warp_sums[32];
    __shared__ unsigned long long tot_full, tot_exact;
    __shared__ uint32_t carry;
    for (int si = blockIdx.x; si < nsims; si += gridDim.x) {
        const SimDev& s = sims[si];
        SimDyn* dyn = s.dyn;
        const int K = s.K;
        const int cur = dyn->cur;
        const int src = SETUP ? cur : cur ^ 1;   // counts of the freshly written buffer
        const int dst = SETUP ? cur ^ 1 : cur;   // layout for the next write
        if (SETUP) {
            for (int c = threadIdx.x; c <= K; c += blockDim.x) {
                s.lay[cur][c] = s.start[c];
                if (c < K) s.cnt[cur][c] = s.start[c + 1] - s.start[c];
            }
            __syncthreads();
        }
        const uint32_t* C = s.cnt[src];
        if (threadIdx.x == 0) {
            tot_full = 0;
            tot_exact = 0;
            carry = 0;
        }
        __syncthreads();
        unsigned long long lf = 0, le = 0;
        for (int c = threadIdx.x; c < K; c += blockDim.x) {
            lf += bucket_size(s, C, c);
            le += C[c];
        }
        // warp sums first: one shared atomic per warp instead of per thread
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lf += __shfl_xor_sync(0xffffffffu, lf, o);
            le += __shfl_xor_sync(0xffffffffu, le, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&tot_full, lf);
            atomicAdd(&tot_exact, le);
        }
        __syncthreads();
        // bucket sizes with slack when they fit, else the exact demand plus an even share of what is left
        const unsigned long long demand = tot_exact + (s.has_reservoir ? s.inj_total : 0u);
        const bool full = tot_full <= (unsigned long long)s.cap;
        // (each bucket rounded up to a multiple of four: up to 3 K more slots)
        const unsigned long long room = demand + 3ull * (unsigned long long)K;
        const uint32_t extra = (!full && room < (unsigned long long)s.cap)
                                   ? (uint32_t)(((unsigned long long)s.cap - room) / (unsigned long long)K)
                                   : 0u;
        if (!full && demand > (unsigned long long)s.cap && threadIdx.x == 0)
            atomicAdd(&dyn->counters[kCntOverflow], 1ull);
        for (int base = 0; base < K; base += blockDim.x) {
            const int c = base + threadIdx.x;
            uint32_t v = 0;
            if (c < K) v = full ? bucket_size(s, C, c) : (C[c] + (s.has_reservoir ? s.inj_count[c] : 0u) + extra + 3u) & ~3u;
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if ((threadIdx.x & 31) >= o) x += y;
            }
            if ((threadIdx.x & 31) == 31) warp_sums[threadIdx.x >> 5] = x;
            __syncthreads();
            if (threadIdx.x < 32) {
                uint32_t ws = threadIdx.x < (blockDim.x >> 5) ? warp_sums[threadIdx.x] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
                    if (threadIdx.x >= o) ws += y;
                }
                warp_sums[threadIdx.x] = ws;
            }
            __syncthreads();
            const uint32_t before = (threadIdx.x >= 32 ? warp_sums[(threadIdx.x >> 5) - 1] : 0u) + carry;
            if (c < K) s.lay[dst][c] = before + x - v;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) carry = before + x;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s.lay[dst][K] = carry;
            if (!SETUP) dyn->n = (uint32_t)min(tot_exact, (unsigned long long)0xFFFFFFFFu);
            dyn->sp_n[dst] = 0;
            if (SETUP) {
                dyn->sp_n[cur] = 0;
                dyn->relax_pending = 0;
            }
        }
        for (int c = threadIdx.x; c < K; c += blockDim.x) s.cnt[dst][c] = 0;
        __syncthreads();
        if (!SETUP && threadIdx.x == 0) {   // end of the step (every thread has read cur)
            if (s.has_reservoir) {
                dyn->next_pid += s.inj_total;
                dyn->counters[kCntInjected] += s.inj_total;
            }
            dyn->cur ^= 1;
            dyn->step += 1;
            dyn->nsamples += 1;
            dyn->relax_pending = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Per-step layout of the next write, over tiles of kLayTile cells so that a
// large domain is laid out by many blocks at once:
//   k_lay_sum   per tile: sums of the bucket sizes with slack (bucket_size),
//               of the counts rounded up to four slots (tight) and of the
//               exact counts;
//   k_lay_scan  per simulation: the choice between slack and tight buckets
//               (tight ones get an even share of the spare slots, a multiple
//               of four), the exclusive scan of the tile sums into tile
//               offsets, the totals, and the end of the step;
//   k_lay_put   per tile: the bucket offsets of its cells and cleared counts.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tight_size(const SimDev& s, const uint32_t* C, int c) {
    return (C[c] + (s.has_reservoir ? s.inj_count[c] : 0u) + 3u) & ~3u;
}

// sum over a block of 1024 threads (every thread gets the total)
__device__ __forceinline__ unsigned long long block_sum_1024(unsigned long long v, unsigned long long* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    v = threadIdx.x < 32 ? sh[threadIdx.x] : 0ull;
    if (threadIdx.x < 32) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) sh[32] = v;
    }
    __syncthreads();
    return sh[32];
}

// exclusive scan over a block of 1024 threads; *total receives the sum
__device__ __forceinline__ unsigned long long block_scan_1024(unsigned long long v, unsigned long long* sh,
                                                              unsigned long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned long long t = sh[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sh[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    *total = sh[31];
    return (w ? sh[w - 1] : 0ull) + x - v;
}

__global__ void __launch_bounds__(kLayTile) k_lay_sum(const SimDev* __restrict__ sims) {
    __shared__ unsigned long long sh[33];
    const SimDev& s = sims[blockIdx.y];
    const int K = s.K;
    const int T = (K + kLayTile - 1) / kLayTile;
    const int src = s.dyn->cur ^ 1;   // counts of the buffer this step wrote
    const uint32_t* C = s.cnt[src];
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
        const int c = t * kLayTile + threadIdx.x;
        unsigned long long f = 0, g = 0, e = 0;
        if (c < K) {
            f = bucket_size(s, C, c);
            g = tight_size(s, C, c);
            e = C[c];
        }
        f = block_sum_1024(f, sh);
        g = block_sum_1024(g, sh);
        e = block_sum_1024(e, sh);
        if (threadIdx.x == 0) {
            s.lay_part[3 * t] = f;
            s.lay_part[3 * t + 1] = g;
            s.lay_part[3 * t + 2] = e;
        }
    }
}

__global__ void __launch_bounds__(kLayTile) k_lay_scan(const SimDev* __restrict__ sims, int nsims) {
    __shared__ unsigned long long sh[33];
    __shared__ unsigned long long carry;
    for (int si = blockIdx.x; si < nsims; si += gridDim.x) {
        const SimDev& s = sims[si];
        SimDyn* dyn = s.dyn;
        const int K = s.K;
        const int T = (K + kLayTile - 1) / kLayTile;
        const int cur = dyn->cur;
        unsigned long long P = 0, G = 0, E = 0;
        for (int t = threadIdx.x; t < T; t += blockDim.x) {
            P += s.lay_part[3 * t];
            G += s.lay_part[3 * t + 1];
            E += s.lay_part[3 * t + 2];
        }
        const unsigned long long tot_full = block_sum_1024(P, sh);
        const unsigned long long tot_tight = block_sum_1024(G, sh);
        const unsigned long long tot_exact = block_sum_1024(E, sh);
        const unsigned long long cap = (unsigned long long)s.cap;
        const bool full = tot_full <= cap;
        const unsigned long long extra =
            (!full && tot_tight < cap) ? ((cap - tot_tight) / (unsigned long long)K) & ~3ull : 0ull;
        const unsigned long long demand = tot_exact + (s.has_reservoir ? s.inj_total : 0u);
        if (threadIdx.x == 0) {
            carry = 0;
            if (!full && demand > cap) atomicAdd(&dyn->counters[kCntOverflow], 1ull);
        }
        __syncthreads();
        for (int base = 0; base < T; base += blockDim.x) {
            const int t = base + threadIdx.x;
            unsigned long long v = 0;
            if (t < T) {
                const int cells = min(kLayTile, K - t * kLayTile);
                v = full ? s.lay_part[3 * t] : s.lay_part[3 * t + 1] + extra * (unsigned long long)cells;
            }
            unsigned long long tot;
            const unsigned long long x = block_scan_1024(v, sh, &tot);
            if (t < T) s.lay_part[3 * t] = carry + x;   // tile offset
            __syncthreads();
            if (threadIdx.x == 0) carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s.lay_part[3 * T] = full ? 1ull : 0ull;
            s.lay_part[3 * T + 1] = extra;
            s.lay[cur][K] = (uint32_t)min(carry, 0xFFFFFFFFull);
            dyn->n = (uint32_t)min(tot_exact, 0xFFFFFFFFull);
            dyn->sp_n[cur] = 0;
            dyn->lay_dst = (uint32_t)cur;
        }
        __syncthreads();
    }
}

// end of the step (after the layout and the parameters): buffers swap, the
// step counter and the sample count advance, the relaxation becomes pending
__global__ void k_step_end(const SimDev* __restrict__ sims, int nsims) {
    for (int si = blockIdx.x * blockDim.x + threadIdx.x; si < nsims; si += gridDim.x * blockDim.x) {
        const SimDev& s = sims[si];
        SimDyn* dyn = s.dyn;
        if (s.has_reservoir) {
            dyn->next_pid += s.inj_total;
            dyn->counters[kCntInjected] += s.inj_total;
        }
        dyn->cur ^= 1;
        dyn->step += 1;
        dyn->nsamples += 1;
        dyn->relax_pending = 1;
    }
}

__global__ void __launch_bounds__(kLayTile) k_lay_put(const SimDev* __restrict__ sims) {
    __shared__ unsigned long long sh[33];
    const SimDev& s = sims[blockIdx.y];
    const int K = s.K;
    const int T = (K + kLayTile - 1) / kLayTile;
    const int dst = (int)s.dyn->lay_dst;
    const uint32_t* C = s.cnt[dst ^ 1];
    const bool full = s.lay_part[3 * T] != 0;
    const uint32_t extra = (uint32_t)s.lay_part[3 * T + 1];
    for (int t = blockIdx.x; t < T; t += gridDim.x) {
        const int c = t * kLayTile + threadIdx.x;
        unsigned long long v = 0;
        if (c < K) v = full ? bucket_size(s, C, c) : tight_size(s, C, c) + extra;
        unsigned long long tot;
        const unsigned long long x = block_scan_1024(v, sh, &tot);
        if (c < K) {
            s.lay[dst][c] = (uint32_t)min(s.lay_part[3 * t] + x, 0xFFFFFFFFull);
            s.cnt[dst][c] = 0;
        }
        __syncthreads();
    }
}

// end of a fused step (mode 0) or after a flush of the pending relaxation (mode 1)
// clears the pending relaxation once it has been applied in place before a
// read-back (the end of a step is part of k_layout)
__global__ void k_clear_pending(const SimDev* __restrict__ sims, int nsims) {
    for (int si = blockIdx.x * blockDim.x + threadIdx.x; si < nsims; si += gridDim.x * blockDim.x)
        sims[si].dyn->relax_pending = 0;
}

// ---------------------------------------------------------------------------
// k_g2 launch configuration: NC consumer warps per CTA, 16 / (NC + 1) CTAs
// per SM sharing its shared memory, the rest of which is each CTA's ring
// ---------------------------------------------------------------------------
struct G2Config {
    int grid;
    uint32_t ring, max_stage;
};

template <int DIM, int MODE, int NC>
const G2Config& g2_config() {
    static G2Config cfg = {0, 0u, 0u};
    if (!cfg.grid) {
        int dev = 0, sms = 152, optin = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaFuncAttributes fa;
        cudaFuncGetAttributes(&fa, k_g2<DIM, MODE, NC>);
        const int ctas = 16 / (NC + 1);
        int ring = std::min(per_sm / ctas - 1024, optin) - (int)fa.sharedSizeBytes;
        ring &= ~1023;
        int per = 0;
        for (; ring >= 16384; ring -= 4096) {
            cudaFuncSetAttribute(k_g2<DIM, MODE, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, ring);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_g2<DIM, MODE, NC>, 32 * (NC + 1), ring);
            if (per >= ctas) break;
        }
        constexpr uint32_t bpp = g2_bytes_per_particle<DIM>();
        cfg.ring = (uint32_t)ring;
        cfg.max_stage = std::min(1024u, ((uint32_t)ring / (2u * bpp)) & ~3u);
        cfg.grid = sms * std::max(per, 1);
    }
    return cfg;
}

template <int DIM, int MODE, int NC>
void launch_g2_one(const Launch& L) {
    const G2Config& c = g2_config<DIM, MODE, NC>();
    k_g2<DIM, MODE, NC><<<c.grid, 32 * (NC + 1), c.ring, L.stream>>>(L.sims, L.nsims, L.wq, c.ring, c.max_stage);
}

template <int MODE, int NC>
void launch_g2(const Launch& L) {
    if (L.dims & 1) launch_g2_one<1, MODE, NC>(L);
    if (L.dims & 2) launch_g2_one<2, MODE, NC>(L);
}

// R (tuning): 4, 8, 12 select 3, 7 or 15 consumer warps per CTA
template <int MODE>
void launch_g2_R(const Launch& L, int R) {
    if (R <= 4) launch_g2<MODE, 3>(L);
    else if (R <= 8) launch_g2<MODE, 7>(L);
    else launch_g2<MODE, 15>(L);
}

template <int MODE, int NC>
void prepare_g2() {
    g2_config<1, MODE, NC>();
    g2_config<2, MODE, NC>();
}

template <int MODE>
void prepare_g2_all() {
    prepare_g2<MODE, 3>();
    prepare_g2<MODE, 7>();
    prepare_g2<MODE, 15>();
}

}  // namespace

void launch_fused_setup(const Launch& L) { k_layout<true><<<L.nsims, 1024, 0, L.stream>>>(L.sims, L.nsims); }

void launch_fused_relax_stream(const Launch& L, int R, bool flush_only) {
    if (flush_only) {
        launch_g2_R<kRelaxOnly>(L, R);
        k_clear_pending<<<(L.nsims + 127) / 128, 128, 0, L.stream>>>(L.sims, L.nsims);
        return;
    }
    if (L.slabs) launch_g2_R<kFullSlab>(L, R);
    else if (L.flux) launch_g2_R<kFullFlux>(L, R);
    else launch_g2_R<kFull>(L, R);
}

// shared-memory limits and grids of the pipelined kernel, set once outside
// any stream capture
void fused_prepare_attributes() {
    static bool done = false;
    if (done) return;
    done = true;
    prepare_g2_all<kFull>();
    prepare_g2_all<kRelaxOnly>();
    prepare_g2_all<kFullSlab>();
    prepare_g2_all<kFullFlux>();
    cudaGetLastError();
}

void launch_fused_inject(const Launch& L) {
    if (L.dims & 1) k_inject_f<1><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    if (L.dims & 2) k_inject_f<2><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
}

void launch_fused_moments(const Launch& L, int R) {
    (void)R;
    k_g1<<<L.grid_c, 32 * kG1Warps, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
}

void launch_fused_params(const Launch& L) { k_params_f<<<L.grid_c, 32, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles); }

// the bucket layout of the next step's destination buffer (reads only the
// arrivals of this step, so it may run beside k_g1 and k_params_f)
void launch_fused_layout_parts(const Launch& L) {
    const dim3 grid((unsigned)std::min(L.lay_tiles, 1024), (unsigned)L.nsims);
    k_lay_sum<<<grid, kLayTile, 0, L.stream>>>(L.sims);
    k_lay_scan<<<L.nsims, kLayTile, 0, L.stream>>>(L.sims, L.nsims);
    k_lay_put<<<grid, kLayTile, 0, L.stream>>>(L.sims);
}

void launch_fused_step_end(const Launch& L) { k_step_end<<<(L.nsims + 127) / 128, 128, 0, L.stream>>>(L.sims, L.nsims); }

void launch_fused_layout(const Launch& L) {
    launch_fused_layout_parts(L);
    launch_fused_step_end(L);
}


}  // namespace usp
