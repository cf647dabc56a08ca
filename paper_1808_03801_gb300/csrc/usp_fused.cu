// usp_fused.cu -- the fused FP32 pipeline of the USP-ESBGK step (sm_103a).
//
// One step n reads buffer p = cur and writes buffer q = cur ^ 1:
//   k_g2      per cell (one warp): the relaxation of step n-1 still pending
//             on the cell's particles (Eqs. 8b, 9, 27, 29-32 with the per-cell
//             momentum / energy conservation), then advection of step n with
//             the boundaries, the new cell, and the write into that cell's
//             bucket of buffer q (the scatter of the counting sort; the
//             bucket sizes come from the previous histogram plus slack).
//   k_inject  reservoir buffer cells refilled into buffer q.
//   k_g1      per cell (one warp): moments of Eq. 1 in one pass, as sums
//             about the cell's mean velocity of the previous step, and the
//             cell's n, T, |u| for its neighbours' Kn_GLL.
//   k_params  per cell: Kn_GLL and P_ne (Eqs. 16-18), sigma* and q* (Eq. 33),
//             the Cholesky factor of the ES covariance (Eq. 6c) in FP64, the
//             fields and the average of Eq. 34.
//   k_layout  per simulation: histogram -> bucket sizes -> exclusive scan,
//             the layout that the next step writes with; then the end of
//             the step (swap buffers, advance the step).
// Per particle all arithmetic is FP32.  FP64 is used per cell in k_params_f
// (one cell per thread): the promotion of the moment sums, the stress
// tensor, Eq. 33 and the Cholesky factor.  FP64 issue rate is scarce on
// GB300 and an FP64 instruction costs about as much for one lane as for a
// whole warp, so the warp-per-cell kernels keep their per-cell arithmetic
// in FP32: moments are sums about the previous step's cell mean and the
// conservation factors use sums about the cell mean, so neither cancels.
// Each particle is read once and written once by k_g2 and its velocity is
// read once more by k_g1.
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

// ---------------------------------------------------------------------------
// k_g2: pending relaxation + advection + bucket scatter.  MODE kFull does
// both; kRelaxOnly applies the pending relaxation in place (before the
// particles are read back).
//
// One warp per cell.  The cell's particles are copied (cp.async, the whole
// cell at once) into a per-warp shared memory area of CAP entries and every
// pass walks them with a rolled loop, so that the per-particle code (the
// Philox draw, the ES sample, advection) appears once in the binary:
//   stage    relaxation draws, conservation sums;
//   pass A   conservation, advection, destination cell, arrivals counted per
//            slot of the cell's destination window;
//   pass B   one atomic reservation per occupied slot in the destination
//            buckets (a single round trip for the whole cell) and each
//            slot's offset in a slot-ordered list of the cell's particles;
//   pass C   rank within the slot -> the particle's place in that list;
//   pass D   the list written out: consecutive lanes write consecutive
//            places of a destination bucket (whole lines, not scattered
//            words).
// Cells above CAP particles are processed in chunks: the conservation sums in
// a first sweep, the update in a second sweep that redraws the same
// counter-based random numbers.
// ---------------------------------------------------------------------------
__device__ __noinline__ bool advect_slow(const SimDev& s, uint32_t step, uint32_t pid, float& x, float& y, float* c) {
    return advect<float>(s, step, pid, x, y, c);
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

// cell of an FP32 position: floor of the scaled offset, clamped to the grid
template <int DIM>
__device__ __forceinline__ int cell_f(const Ctx& C, float x, float y) {
    const float fy = fminf(fmaxf(floorf((y - C.lo1) * C.inv_dy), 0.0f), (float)C.nym1);
    if (DIM == 1) return (int)fy;
    const float fx = fminf(fmaxf(floorf((x - C.lo0) * C.inv_dx), 0.0f), (float)C.nxm1);
    return (int)fy * C.nx + (int)fx;
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
    return advect_slow(s, step, pid, x, y, c);
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

// per-warp staging area
struct Stage {
    float* x;
    float* y;
    float* v0;
    float* v1;
    float* v2;
    uint32_t* id;
    unsigned char* sel;
};

// largest staging area per warp: holds a 360-particle cell with its
// fluctuations (+3 standard deviations) while leaving part of the SM's
// shared memory / L1 carve-out to the cache
constexpr int kCapMax = 416;

// bytes per staged particle: (x,) y, v0, v1, v2, id, relaxation flag
template <int CAP, int DIM>
__host__ __device__ constexpr int stage_bytes() {
    return CAP * (DIM == 2 ? 25 : 21);
}

template <int CAP, int DIM>
__device__ __forceinline__ Stage stage_of(unsigned char* base, int warp) {
    float* f = (float*)(base + (size_t)warp * stage_bytes<CAP, DIM>());
    Stage S;
    S.x = nullptr;
    if (DIM == 2) {
        S.x = f;
        f += CAP;
    }
    S.y = f;
    S.v0 = S.y + CAP;
    S.v1 = S.v0 + CAP;
    S.v2 = S.v1 + CAP;
    S.id = (uint32_t*)(S.v2 + CAP);
    S.sel = (unsigned char*)(S.id + CAP);
    return S;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Destination window of a cell: the 64 cells that its particles can reach in
// one step without leaving it (1-D: offsets -32..31; 2-D: an 8 x 8 block
// around the cell).  The warp counts its arrivals per window slot in shared
// memory, reserves each slot's range in the destination bucket with one
// global atomic, then writes; particles that land outside the window reserve
// their place one group at a time.
constexpr int kWin = 64;
constexpr unsigned char kSlotNone = 0xFF;   // removed, nothing to write
constexpr unsigned char kSlotFar = 0xFE;    // outside the window
constexpr unsigned char kSlotOther = 0xFD;  // in another slab of a decomposed domain

template <int DIM>
__device__ __forceinline__ int win_slot(int dc, int cell, int cx, int cy, int nx) {
    if (DIM == 1) {
        const int o = dc - cell + 32;
        return (o >= 0 && o < kWin) ? o : -1;
    }
    const int iy = dc / nx, ix = dc - iy * nx;
    const int oy = iy - cy + 4, ox = ix - cx + 4;
    return (oy >= 0 && oy < 8 && ox >= 0 && ox < 8) ? oy * 8 + ox : -1;
}

template <int DIM>
__device__ __forceinline__ int win_cell(int k, int cell, int cx, int cy, int nx) {
    if (DIM == 1) return cell + k - 32;
    return (cy + (k >> 3) - 4) * nx + (cx + (k & 7) - 4);
}

// Per-warp copy of the header of one cell: bucket bounds, arrivals and the
// FP32 relaxation parameters, fetched with one round of cp.async (one word
// per lane) instead of two dependent rounds of loads.
struct alignas(16) Hdr {
    float prm[kNFPrm];   // the cell's parameter record: u[3], theta, L[6], P_relax, nu, nu_ES, P_ne, valid
    uint32_t lay[2];
    uint32_t cnt;
};

__device__ __forceinline__ void cp_async16_ca(void* dst, const void* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void fetch_hdr(const SimDev& s, int p, int cell, Hdr& H, int lane) {
    if (lane < 2) cp_async4(&H.lay[lane], s.lay[p] + cell + lane);
    else if (lane == 2) cp_async4(&H.cnt, s.cnt[p] + cell);
    else if (lane < 7) cp_async16_ca(&H.prm[4 * (lane - 3)], s.fprm + (size_t)cell * kNFPrm + 4 * (lane - 3));
    cp_async_wait_all();
    __syncwarp();
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
// through a plane (kFullSlab counts too)
enum { kFull = 0, kRelaxOnly = 1, kFullSlab = 2, kFullFlux = 3 };

template <int CAP, int DIM, int MODE>
__device__ void g2_cell(const SimDev* __restrict__ sims, const SimDev& s, int cell, const Hdr& H, int p, uint32_t step,
                        bool pending, uint32_t* spl,
                        const Stage& S, uint32_t* win, uint16_t* perm, int lane) {
    const uint32_t base = H.lay[0];
    const uint32_t top = min(H.lay[1], (uint32_t)s.cap);
    const uint32_t capc = top > base ? top - base : 0u;
    const uint32_t arrived = H.cnt;
    const uint32_t nb = min(arrived, capc);
    uint32_t nsp = 0;
    if (arrived > nb) nsp = collect_spill(s, p, cell, spl, lane);
    const uint32_t n = nb + nsp;
    if (n == 0) return;
    FCell f;
#pragma unroll
    for (int d = 0; d < 3; ++d) f.u[d] = H.prm[d];
    f.th = H.prm[3];
    {   // M = L L^T - theta I from the FP64-built factor L
        const float L0 = H.prm[4], L1 = H.prm[5], L2 = H.prm[6], L3 = H.prm[7], L4 = H.prm[8], L5 = H.prm[9];
        f.M[0] = L0 * L0 - f.th;
        f.M[1] = L1 * L0;
        f.M[2] = L1 * L1 + L2 * L2 - f.th;
        f.M[3] = L3 * L0;
        f.M[4] = L3 * L1 + L4 * L2;
        f.M[5] = L3 * L3 + L4 * L4 + L5 * L5 - f.th;
    }
    f.pr = H.prm[10];
    f.nu = H.prm[11];
    f.nues = H.prm[12];
    f.pne = H.prm[13];
    f.valid = H.prm[14] != 0.0f;
    const bool relax = pending && f.valid;
    if (MODE == kRelaxOnly && !relax) return;
    TimeDraw td;
    td.dt = s.f_dt;
    td.a = f.nues * td.dt;
    td.em1 = expm1f(td.a);
    td.ema = __expf(-td.a);
    td.inv_nues = 1.0f / f.nues;
    td.inv_pr = f.pr > 0.0f ? 1.0f / f.pr : 0.0f;
    const int q = p ^ 1;
    const uint32_t nch = (n + CAP - 1) / CAP;
    const Src P = src_of(s, p);
    const uint2 key = make_uint2(s.key0, s.key1);

    // stage chunk ch: the particles are copied into the staging planes
    // (asynchronously from the bucket, directly from the spill list), then
    // relaxed particles get their new peculiar velocity in v0..v2 and their
    // flag in sel; if `sums`, the conservation sums are accumulated
    float a0 = 0, a1 = 0, a2 = 0, ae = 0, b0 = 0, b1 = 0, b2 = 0, be = 0, nr = 0;
    auto stage_chunk = [&](uint32_t ch, bool sums) -> uint32_t {
        const uint32_t off = ch * CAP;
        const uint32_t m = min((uint32_t)CAP, n - off);
        const uint32_t mb = off < nb ? min(m, nb - off) : 0u;
        __syncwarp();
#pragma unroll 1
        for (uint32_t j = lane; j < mb; j += 32) {
            const uint32_t i = base + off + j;
            if (DIM == 2) cp_async4(S.x + j, P.x + i);
            cp_async4(S.y + j, P.y + i);
            cp_async4(S.v0 + j, P.v0 + i);
            cp_async4(S.v1 + j, P.v1 + i);
            cp_async4(S.v2 + j, P.v2 + i);
            cp_async4(S.id + j, P.id + i);
        }
#pragma unroll 1
        for (uint32_t j = mb + lane; j < m; j += 32) {
            float x = 0.0f, y, v0, v1, v2;
            uint32_t id;
            load_particle<DIM>(s, p, base, nb, spl, off + j, x, y, v0, v1, v2, id);
            if (DIM == 2) S.x[j] = x;
            S.y[j] = y; S.v0[j] = v0; S.v1[j] = v1; S.v2[j] = v2; S.id[j] = id;
        }
        cp_async_wait_all();
        __syncwarp();
#pragma unroll 1
        for (uint32_t j0 = lane; j0 < m; j0 += 64) {
            const uint32_t j1 = j0 + 32;
            const bool has1 = j1 < m;
            unsigned char s0 = 0, s1 = 0;
            if (relax) {
                const float p0 = S.v0[j0], q0 = S.v1[j0], r0 = S.v2[j0];
                const uint32_t id0 = S.id[j0];
                float p1 = 0.0f, q1 = 0.0f, r1 = 0.0f;
                uint32_t id1 = 0;
                if (has1) {
                    p1 = S.v0[j1]; q1 = S.v1[j1]; r1 = S.v2[j1];
                    id1 = S.id[j1];
                }
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
                        if (sums) {
                            const float o0 = p0 - f.u[0], o1 = q0 - f.u[1], o2 = r0 - f.u[2];
                            a0 += o0; a1 += o1; a2 += o2;
                            ae += o0 * o0 + o1 * o1 + o2 * o2;
                            b0 += C0[0]; b1 += C0[1]; b2 += C0[2];
                            be += C0[0] * C0[0] + C0[1] * C0[1] + C0[2] * C0[2];
                            nr += 1.0f;
                        }
                        S.v0[j0] = C0[0]; S.v1[j0] = C0[1]; S.v2[j0] = C0[2];
                    }
                    if (s1) {
                        if (sums) {
                            const float o0 = p1 - f.u[0], o1 = q1 - f.u[1], o2 = r1 - f.u[2];
                            a0 += o0; a1 += o1; a2 += o2;
                            ae += o0 * o0 + o1 * o1 + o2 * o2;
                            b0 += C1[0]; b1 += C1[1]; b2 += C1[2];
                            be += C1[0] * C1[0] + C1[1] * C1[1] + C1[2] * C1[2];
                            nr += 1.0f;
                        }
                        S.v0[j1] = C1[0]; S.v1[j1] = C1[1]; S.v2[j1] = C1[2];
                    }
                }
            }
            S.sel[j0] = s0;
            if (has1) S.sel[j1] = s1;
        }
        __syncwarp();
        return m;
    };

    uint32_t m_last = 0;
    for (uint32_t ch = 0; ch < nch; ++ch) m_last = stage_chunk(ch, true);

    // conservation factors of the cell
    bool apply = false;
    float uo0 = 0, uo1 = 0, uo2 = 0, mn0 = 0, mn1 = 0, mn2 = 0, alpha = 1;
    if (relax) {
        nr = warp_sumf(nr);
        if (nr >= 2.0f) {
            a0 = warp_sumf(a0); a1 = warp_sumf(a1); a2 = warp_sumf(a2); ae = warp_sumf(ae);
            b0 = warp_sumf(b0); b1 = warp_sumf(b1); b2 = warp_sumf(b2); be = warp_sumf(be);
            // FP32: the sums are taken about the cell mean, so the differences
            // below do not cancel.  The butterfly sums are bitwise the same on
            // every lane (each stage adds the same two values), so every lane
            // computes the same factors without a broadcast.
            const float inv = 1.0f / nr;
            const float Eo = ae - (a0 * a0 + a1 * a1 + a2 * a2) * inv;
            const float En = be - (b0 * b0 + b1 * b1 + b2 * b2) * inv;
            if (En > 0.0f && Eo >= 0.0f) {
                apply = true;
                alpha = sqrtf(Eo / En);
                uo0 = f.u[0] + a0 * inv;
                uo1 = f.u[1] + a1 * inv;
                uo2 = f.u[2] + a2 * inv;
                mn0 = b0 * inv;
                mn1 = b1 * inv;
                mn2 = b2 * inv;
                if (lane == 0) atomicAdd(&s.dyn->counters[kCntRelaxed], (unsigned long long)(unsigned)nr);
            }
        }
    }

    // the relaxed velocity of staged particle j (conservation applied), or
    // its old velocity when the cell had a single relaxed particle
    auto final_velocity = [&](uint32_t off, uint32_t j, float* c) {
        c[0] = S.v0[j];
        c[1] = S.v1[j];
        c[2] = S.v2[j];
        if (S.sel[j]) {
            if (apply) {
                c[0] = uo0 + alpha * (c[0] - mn0);
                c[1] = uo1 + alpha * (c[1] - mn1);
                c[2] = uo2 + alpha * (c[2] - mn2);
            } else {
                float ox, oy;
                uint32_t oid;
                load_particle<DIM>(s, p, base, nb, spl, off + j, ox, oy, c[0], c[1], c[2], oid);
            }
        }
    };

    if (MODE == kRelaxOnly) {
        for (uint32_t ch = 0; ch < nch; ++ch) {
            const uint32_t m = nch > 1 ? stage_chunk(ch, false) : m_last;
            const uint32_t off = ch * CAP;
#pragma unroll 1
            for (uint32_t j = lane; j < m; j += 32) {
                if (!(S.sel[j] && apply)) continue;
                float c[3];
                final_velocity(off, j, c);
                store_velocity<DIM>(s, p, base, nb, spl, off + j, c[0], c[1], c[2]);
            }
        }
        __syncwarp();
        return;
    }

    Ctx C;
    make_ctx(s, q, C);
    const int cy = DIM == 2 ? cell / C.nx : 0;
    const int cx = DIM == 2 ? cell - cy * C.nx : 0;
    uint32_t* wcnt = win;              // arrivals per window slot, then the running rank
    uint32_t* wstart = win + kWin;     // first reserved index of each slot in its bucket
    uint32_t* wend = win + 2 * kWin;   // end of that bucket
    uint32_t* woff = win + 3 * kWin;   // offset of the slot in the slot-ordered list
    for (uint32_t ch = 0; ch < nch; ++ch) {
        const uint32_t m = nch > 1 ? stage_chunk(ch, false) : m_last;
        const uint32_t off = ch * CAP;
        for (int k = lane; k < kWin; k += 32) wcnt[k] = 0;
        __syncwarp();
        // pass A: conservation, advection, destination slot; count per slot
#pragma unroll 1
        for (uint32_t b = 0; b < m; b += 32) {
            const uint32_t j = b + lane;
            int slot = -2;   // -2: nothing to count
            if (j < m) {
                float x = DIM == 2 ? S.x[j] : 0.0f, y = S.y[j], c[3];
                final_velocity(off, j, c);
                unsigned char ws = kSlotNone;
                if (advect_fast<DIM>(s, C, step, S.id[j], x, y, c)) {
                    const int dc = cell_f<DIM>(C, x, y) - (MODE == kFullSlab ? C.cell0 : 0);   // local cell
                    if (MODE == kFullSlab && (unsigned)dc >= (unsigned)C.K) {
                        ws = kSlotOther;
                    } else if (!C.reservoir || !in_buffer(s, dc)) {
                        slot = win_slot<DIM>(dc, cell, cx, cy, C.nx);
                        ws = slot >= 0 ? (unsigned char)slot : kSlotFar;
                    } else {
                        atomicAdd(&s.dyn->counters[kCntRemoved], 1ull);
                    }
                }
                if ((MODE == kFullFlux || MODE == kFullSlab) && s.flux_axis)
                    count_flux<float>(s, DIM == 2 ? S.x[j] : 0.0f, S.y[j], x, y);
                if (DIM == 2) S.x[j] = x;
                S.y[j] = y; S.v0[j] = c[0]; S.v1[j] = c[1]; S.v2[j] = c[2];
                S.sel[j] = ws;
            }
            const unsigned grp = __match_any_sync(0xffffffffu, slot);
            if (slot >= 0 && lane == __ffs(grp) - 1) wcnt[slot] += (uint32_t)__popc(grp);
            __syncwarp();
        }
        // pass B: one reservation per occupied slot, all in flight together;
        // the slot's first index, the end of its bucket and its offset in the
        // slot-ordered list of the cell's particles go to shared memory
        uint32_t tot_win = 0;
        {
            const uint32_t c0 = wcnt[lane], c1 = wcnt[lane + 32];
            uint32_t x0 = c0, x1 = c1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y0 = __shfl_up_sync(0xffffffffu, x0, o);
                const uint32_t y1 = __shfl_up_sync(0xffffffffu, x1, o);
                if (lane >= o) {
                    x0 += y0;
                    x1 += y1;
                }
            }
            const uint32_t t0 = __shfl_sync(0xffffffffu, x0, 31);
            woff[lane] = x0 - c0;
            woff[lane + 32] = t0 + x1 - c1;
            tot_win = t0 + __shfl_sync(0xffffffffu, x1, 31);
        }
        for (int k = lane; k < kWin; k += 32) {
            const uint32_t cnt = wcnt[k];
            if (cnt) {
                const int dest = win_cell<DIM>(k, cell, cx, cy, C.nx);
                const uint32_t r = atomicAdd(&C.dcnt[dest], cnt);
                wstart[k] = C.dlay[dest] + r;
                wend[k] = min(C.dlay[dest + 1], C.cap);
            }
            wcnt[k] = 0;
        }
        __syncwarp();
        // pass C: rank within the slot -> position in the slot-ordered list
        // (particles leaving the window are written here, one by one)
#pragma unroll 1
        for (uint32_t b = 0; b < m; b += 32) {
            const uint32_t j = b + lane;
            const unsigned char ws = j < m ? S.sel[j] : kSlotNone;
            const unsigned grp = __match_any_sync(0xffffffffu, (unsigned)ws);
            if (MODE == kFullSlab && ws == kSlotOther) {   // into the buckets of another slab
                emit_other<DIM>(sims, s, q, DIM == 2 ? S.x[j] : 0.0f, S.y[j], S.v0[j], S.v1[j], S.v2[j], S.id[j]);
            } else if (ws < kWin) {
                const int leader = __ffs(grp) - 1;
                uint32_t r0 = 0;
                if (lane == leader) {
                    r0 = wcnt[ws];
                    wcnt[ws] = r0 + (uint32_t)__popc(grp);
                }
                const uint32_t rank = __shfl_sync(grp, r0, leader) + (uint32_t)__popc(grp & lanemask_lt());
                perm[woff[ws] + rank] = (uint16_t)j;
            } else if (ws == kSlotFar) {   // outside the window: a reservation of its own
                const float x = DIM == 2 ? S.x[j] : 0.0f, y = S.y[j];
                const int dc = cell_f<DIM>(C, x, y) - (MODE == kFullSlab ? C.cell0 : 0);
                const uint32_t i = C.dlay[dc] + atomicAdd(&C.dcnt[dc], 1u);
                const uint32_t hi = min(C.dlay[dc + 1], C.cap);
                put_own<DIM>(s, C, q, i, hi, dc, x, y, S.v0[j], S.v1[j], S.v2[j], S.id[j]);
            }
            __syncwarp();
        }
        // pass D: the slot-ordered list written out, consecutive lanes to
        // consecutive slots of the destination buckets
#pragma unroll 1
        for (uint32_t k = lane; k < tot_win; k += 32) {
            const uint32_t j = perm[k];
            const unsigned char ws = S.sel[j];
            const uint32_t i = wstart[ws] + (k - woff[ws]);
            const float x = DIM == 2 ? S.x[j] : 0.0f, y = S.y[j];
            const int dc = i < wend[ws] ? 0 : cell_f<DIM>(C, x, y) - (MODE == kFullSlab ? C.cell0 : 0);
            put_own<DIM>(s, C, q, i, wend[ws], dc, x, y, S.v0[j], S.v1[j], S.v2[j], S.id[j]);
        }
        __syncwarp();
    }
    __syncwarp();
}

// copy one simulation descriptor into shared memory (one warp)
__device__ __forceinline__ void load_sim_warp(SimDev& dst, const SimDev& src, int lane) {
    const int4* a = reinterpret_cast<const int4*>(&src);
    int4* b = reinterpret_cast<int4*>(&dst);
    for (int i = lane; i < (int)(sizeof(SimDev) / 16); i += 32) b[i] = a[i];
}

// Cells are handed out one at a time from per-simulation queues
// (SimDyn::qnext): each warp starts on a home simulation and takes its next
// cell from it, so its descriptor stays in shared memory and neighbouring
// cells are processed together; when the home simulation runs out, the warp
// looks for one with cells left (32 candidates per round).  The next cell is
// requested while the current one is processed.  wq[0] counts the warps that
// left; the last one resets every queue for the next launch.
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

template <int CAP, int DIM, int MODE>
__global__ void __launch_bounds__(128, 4) k_g2(const SimDev* __restrict__ sims, int nsims, uint32_t* __restrict__ wq) {
    extern __shared__ __align__(16) unsigned char g2_smem[];
    __shared__ SimDev sim_w[4];
    __shared__ uint32_t spl_all[4][32];
    __shared__ uint32_t win_all[4][4 * kWin];
    __shared__ uint16_t perm_all[4][kCapMax];
    __shared__ Hdr hdr_all[4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Stage S = stage_of<CAP, DIM>(g2_smem, warp);
    const uint32_t nwarps = gridDim.x * (blockDim.x / 32);
    SimDev& s = sim_w[warp];
    int h = (int)((blockIdx.x * (blockDim.x / 32) + warp) % (unsigned)nsims);
    if (sims[h].dim != DIM) h = find_sim<DIM>(sims, nsims, h, lane);
    while (h >= 0) {
        __syncwarp();
        load_sim_warp(s, sims[h], lane);
        __syncwarp();
        const int p = s.dyn->cur;
        const uint32_t step = s.dyn->step;
        const bool pending = s.dyn->relax_pending != 0;
        const uint32_t K = (uint32_t)s.K;
        if (MODE == kRelaxOnly && !pending) {   // nothing to apply: close its queue
            if (lane == 0) atomicMax(&s.dyn->qnext, K);
            h = find_sim<DIM>(sims, nsims, h, lane);
            continue;
        }
        uint32_t c = 0;
        if (lane == 0) c = atomicAdd(&s.dyn->qnext, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        while (c < K) {
            uint32_t cn = 0;   // the next cell, requested now
            if (lane == 0) cn = atomicAdd(&s.dyn->qnext, 1u);
            fetch_hdr(s, p, (int)c, hdr_all[warp], lane);
            g2_cell<CAP, DIM, MODE>(sims, s, (int)c, hdr_all[warp], p, step, pending, spl_all[warp], S, win_all[warp],
                                    perm_all[warp], lane);
            c = __shfl_sync(0xffffffffu, cn, 0);
        }
        h = find_sim<DIM>(sims, nsims, h, lane);
    }
    if (lane == 0) {
        __threadfence();
        const uint32_t done = atomicAdd(&wq[0], 1u);
        if (done == nwarps - 1) {
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
__global__ void __launch_bounds__(256) k_g1(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                            const int* __restrict__ ntiles) {
    __shared__ uint32_t spl_all[8][32];
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
        const float* V0 = (const float*)s.vel[q][0];
        const float* V1 = (const float*)s.vel[q][1];
        const float* V2 = (const float*)s.vel[q][2];
        for (int cc = warp; cc < kCTile; cc += 8) {
            const int cell = tile.y + cc;
            if (cell >= K) break;
            const uint32_t base = s.lay[q][cell];
            const uint32_t top = min(s.lay[q][cell + 1], (uint32_t)s.cap);
            const uint32_t capc = top > base ? top - base : 0u;
            const uint32_t arrived = s.cnt[q][cell];
            const uint32_t nb = min(arrived, capc);
            const float4 us = reinterpret_cast<const float4*>(s.fprm)[(size_t)cell * (kNFPrm / 4)];
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
#pragma unroll 4
            for (uint32_t j = lane; j < nb; j += 32) add(V0[base + j], V1[base + j], V2[base + j]);
            for (uint32_t j = nb + lane; j < n; j += 32) {   // spill-list entries of the cell
                const uint32_t i = spl_all[warp][j - nb];
                add(s.sp_vel[q][0][i], s.sp_vel[q][1][i], s.sp_vel[q][2][i]);
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) S[k] = warp_sumf(S[k]);
            // FP32 sums only: their promotion to FP64 happens in k_params_f, one
            // cell per thread (an FP64 instruction costs the same for one lane)
            if (lane < 16) {
                float v;
                if (lane == 0) v = (float)n;
                else if (lane <= 12) v = S[0];
                else v = lane == 13 ? u0 : (lane == 14 ? u1 : u2);
                // lanes 1..12 need S[lane - 1]: select without dynamic indexing
#pragma unroll
                for (int k = 1; k < 12; ++k)
                    if (lane == k + 1) v = S[k];
                s.momf[(size_t)cell * 16 + lane] = v;   // one 64-byte record per cell
            }
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

// promotion of the cell's FP32 shifted sums: mean velocity, pressure tensor
// per unit density (P / rho) and theta = R T; inv = 1 / N
__device__ __forceinline__ void local_f(const SimDev& s, int cell, LocalF& L, double* u, double* P, double* theta,
                                        double& inv) {
    const float* M = s.momf + (size_t)cell * 16;   // N, 12 sums, shift[3]
    const int N = (int)M[0];
    L.N = N;
    L.valid = 0;
    L.n = (float)(N * s.w);
    L.T = 0;
    L.umag = 0;
    inv = 0.0;
    if (N < 1) return;
    inv = 1.0 / N;
    const double d0 = M[1] * inv, d1 = M[2] * inv, d2 = M[3] * inv;
    const double uu[3] = {M[13] + d0, M[14] + d1, M[15] + d2};
    const double p0 = M[4] * inv - d0 * d0, p1 = M[5] * inv - d1 * d1,
                 p2 = M[6] * inv - d2 * d2;
    const double th = (p0 + p1 + p2) * (1.0 / 3.0);
    u[0] = uu[0]; u[1] = uu[1]; u[2] = uu[2];
    P[0] = p0; P[1] = p1; P[2] = p2;
    P[3] = M[7] * inv - d0 * d1;
    P[4] = M[8] * inv - d0 * d2;
    P[5] = M[9] * inv - d1 * d2;
    *theta = th;
    L.valid = N >= 2 && th > 0.0;
    if (!L.valid) return;
    L.T = (float)(th * s.inv_R);
    L.umag = sqrtf((float)(uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2]));
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
            double u[3] = {0, 0, 0}, P[6], th = 0, inv;
            local_f(s, cell, L, u, P, &th, inv);
            double f[kNFields];
            for (int k = 0; k < kNFields; ++k) f[k] = 0.0;
            f[0] = L.N * s.w;
            f[15] = L.N;
            if (L.N >= 1) {
                f[1] = u[0]; f[2] = u[1]; f[3] = u[2];
            }
            float pr[kNFPrm];
            for (int k = 0; k < kNFPrm; ++k) pr[k] = 0.0f;
            pr[0] = (float)u[0]; pr[1] = (float)u[1]; pr[2] = (float)u[2];
            pr[3] = (float)th;
            if (L.valid) {
                const float thf = (float)th;
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
                // Eq. 33; FP64 divisions are costly here, so each factor is
                // inverted once
                const double ifs = 1.0 / (1.0 + 0.5 * s.dt * (double)nu * pne);
                const double ifq = 1.0 / (1.0 + 0.5 * s.dt * (double)nu * s.Pr * pne);
                const double sig[6] = {(P[0] - th) * ifs, (P[1] - th) * ifs, (P[2] - th) * ifs, P[3] * ifs, P[4] * ifs,
                                       P[5] * ifs};
                const double b = s.es_b;                                                        // Eq. 6c
                const double A00 = th + b * sig[0], A11 = th + b * sig[1], A22 = th + b * sig[2];
                const double A10 = b * sig[3], A20 = b * sig[4], A21 = b * sig[5];
                // Cholesky factor with reciprocal square roots (no FP64 divisions)
                double l00 = 0, l10 = 0, l11 = 0, l20 = 0, l21 = 0, l22 = 0;
                bool ok = A00 > 0.0;
                if (ok) {
                    const double r0 = rsqrt(A00);
                    l00 = A00 * r0;
                    l10 = A10 * r0;
                    l20 = A20 * r0;
                    const double d1 = A11 - l10 * l10;
                    ok = d1 > 0.0;
                    if (ok) {
                        const double r1 = rsqrt(d1);
                        l11 = d1 * r1;
                        l21 = (A21 - l20 * l10) * r1;
                        const double d2 = A22 - l20 * l20 - l21 * l21;
                        ok = d2 > 0.0;
                        if (ok) l22 = d2 * rsqrt(d2);
                    }
                }
                if (!ok) {
                    const double r = sqrt(th);
                    l00 = l11 = l22 = r;
                    l10 = l20 = l21 = 0.0;
                    atomicAdd(&s.dyn->counters[kCntChol], 1ull);
                }
                const float nues = (float)s.Pr * nu;
                pr[4] = (float)l00; pr[5] = (float)l10; pr[6] = (float)l11;
                pr[7] = (float)l20; pr[8] = (float)l21; pr[9] = (float)l22;
                pr[10] = -expm1f(-nues * (float)s.dt);                                        // Eqs. 8b, 9
                // the decay rate of Eq. 32; the SP-ESBGK step holds its target
                // for the whole step (Eq. 8b): with P_ne = 0 a rate of 0 gives s = 1
                pr[11] = s.mode == kModeSPESBGK ? 0.0f : nu;
                pr[12] = nues;
                pr[13] = pne;
                pr[14] = 1.0f;
                // heat flux from the third central moment of the shifted sums
                const float* M = s.momf + (size_t)cell * 16;
                const double d0 = M[1] * inv, d1 = M[2] * inv, d2 = M[3] * inv;
                const double m00 = M[4] * inv, m11 = M[5] * inv, m22 = M[6] * inv;
                const double m01 = M[7] * inv, m02 = M[8] * inv, m12 = M[9] * inv;
                const double t0 = M[10] * inv, t1 = M[11] * inv, t2 = M[12] * inv;
                const double tr = m00 + m11 + m22, dd = d0 * d0 + d1 * d1 + d2 * d2;
                const double Q0 = 0.5 * (t0 - d0 * tr - 2.0 * (m00 * d0 + m01 * d1 + m02 * d2) + 2.0 * d0 * dd);
                const double Q1 = 0.5 * (t1 - d1 * tr - 2.0 * (m01 * d0 + m11 * d1 + m12 * d2) + 2.0 * d1 * dd);
                const double Q2 = 0.5 * (t2 - d2 * tr - 2.0 * (m02 * d0 + m12 * d1 + m22 * d2) + 2.0 * d2 * dd);
                const double rhod = L.N * s.w * s.mass, pd = rhod * th;
                f[4] = th * s.inv_R;
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
#pragma unroll
            for (int k = 0; k < kNFields; ++k) {
                s.inst[(size_t)k * K + cell] = f[k];
                s.avg[(size_t)k * K + cell] = first ? f[k] : s.avg_keep * av[k] + f[k] * s.avg_new;   // Eq. 34
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
    return m + (m >> 2) + 16u + (s.has_reservoir ? s.inj_count[c] : 0u);
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
        const uint32_t extra = (!full && demand < (unsigned long long)s.cap)
                                   ? (uint32_t)(((unsigned long long)s.cap - demand) / (unsigned long long)K)
                                   : 0u;
        if (!full && demand > (unsigned long long)s.cap && threadIdx.x == 0)
            atomicAdd(&dyn->counters[kCntOverflow], 1ull);
        for (int base = 0; base < K; base += blockDim.x) {
            const int c = base + threadIdx.x;
            uint32_t v = 0;
            if (c < K) v = full ? bucket_size(s, C, c) : C[c] + (s.has_reservoir ? s.inj_count[c] : 0u) + extra;
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

// end of a fused step (mode 0) or after a flush of the pending relaxation (mode 1)
// clears the pending relaxation once it has been applied in place before a
// read-back (the end of a step is part of k_layout)
__global__ void k_clear_pending(const SimDev* __restrict__ sims, int nsims) {
    for (int si = blockIdx.x * blockDim.x + threadIdx.x; si < nsims; si += gridDim.x * blockDim.x)
        sims[si].dyn->relax_pending = 0;
}

// one wave of resident blocks: late blocks would only find empty queues
template <int CAP, int DIM, int MODE>
int g2_grid(int smem) {
    static int grid = 0;
    if (!grid) {
        int dev = 0, sms = 152, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_g2<CAP, DIM, MODE>, 128, smem);
        grid = sms * (per > 0 ? per : 1);
    }
    return grid;
}

template <int CAP, int DIM, int MODE>
void launch_g2_one(const Launch& L) {
    const int smem = 4 * stage_bytes<CAP, DIM>();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_g2<CAP, DIM, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        attr = true;
    }
    k_g2<CAP, DIM, MODE><<<g2_grid<CAP, DIM, MODE>(smem), 128, smem, L.stream>>>(L.sims, L.nsims, L.wq);
}

template <int CAP, int MODE>
void launch_g2(const Launch& L) {
    if (L.dims & 1) launch_g2_one<CAP, 1, MODE>(L);
    if (L.dims & 2) launch_g2_one<CAP, 2, MODE>(L);
}

}  // namespace

void launch_fused_setup(const Launch& L) { k_layout<true><<<L.nsims, 1024, 0, L.stream>>>(L.sims, L.nsims); }

template <int MODE>
void launch_g2_R(const Launch& L, int R) {
    if (R <= 4) launch_g2<128, MODE>(L);
    else if (R <= 8) launch_g2<256, MODE>(L);
    else launch_g2<kCapMax, MODE>(L);
}

// R: particles per lane of the largest expected cell (staging area of 32 R)
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

// set the shared-memory limits of the staged kernels once, outside any capture
template <int CAP, int MODE>
void set_g2_smem() {
    cudaFuncSetAttribute(k_g2<CAP, 1, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * stage_bytes<CAP, 1>());
    cudaFuncSetAttribute(k_g2<CAP, 2, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4 * stage_bytes<CAP, 2>());
    g2_grid<CAP, 1, MODE>(4 * stage_bytes<CAP, 1>());
    g2_grid<CAP, 2, MODE>(4 * stage_bytes<CAP, 2>());
}

void fused_prepare_attributes() {
    static bool done = false;
    if (done) return;
    done = true;
    set_g2_smem<128, kFull>();
    set_g2_smem<256, kFull>();
    set_g2_smem<kCapMax, kFull>();
    set_g2_smem<128, kRelaxOnly>();
    set_g2_smem<256, kRelaxOnly>();
    set_g2_smem<kCapMax, kRelaxOnly>();
    set_g2_smem<128, kFullSlab>();
    set_g2_smem<256, kFullSlab>();
    set_g2_smem<kCapMax, kFullSlab>();
    set_g2_smem<128, kFullFlux>();
    set_g2_smem<256, kFullFlux>();
    set_g2_smem<kCapMax, kFullFlux>();
    cudaGetLastError();
}

void launch_fused_inject(const Launch& L) {
    if (L.dims & 1) k_inject_f<1><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    if (L.dims & 2) k_inject_f<2><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
}

void launch_fused_moments(const Launch& L, int R) {
    (void)R;
    k_g1<<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
}

void launch_fused_params(const Launch& L) { k_params_f<<<L.grid_c, 32, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles); }

void launch_fused_layout(const Launch& L) { k_layout<false><<<L.nsims, 1024, 0, L.stream>>>(L.sims, L.nsims); }


}  // namespace usp
