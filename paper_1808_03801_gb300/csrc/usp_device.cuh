// usp_device.cuh -- device functions shared by the plain and the fused
// kernels: particle views, cell index, advection with boundaries, warp
// aggregation, particle creation, per-cell local state, ES sampling.
#pragma once
#include "usp_internal.cuh"

namespace usp {

// ---------------------------------------------------------------------------
// particle views
// ---------------------------------------------------------------------------
template <class T>
struct PView {
    T* x;
    T* y;
    T* c0;
    T* c1;
    T* c2;
    uint32_t* pid;
};

template <class T>
__device__ __forceinline__ PView<T> view(const SimDev& s, int buf) {
    PView<T> v;
    v.x = (T*)s.pos[buf][0];
    v.y = (T*)s.pos[buf][1];
    v.c0 = (T*)s.vel[buf][0];
    v.c1 = (T*)s.vel[buf][1];
    v.c2 = (T*)s.vel[buf][2];
    v.pid = s.pid[buf];
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// cells
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ int cell_index(const SimDev& s, T x, T y) {
    T fy = dev_floor<T>((y - (T)s.lo[1]) / (T)s.dy);
    fy = fy < (T)0 ? (T)0 : (fy > (T)(s.ny - 1) ? (T)(s.ny - 1) : fy);
    int iy = (int)fy;
    if (s.dim == 1) return iy;
    T fx = dev_floor<T>((x - (T)s.lo[0]) / (T)s.dx);
    fx = fx < (T)0 ? (T)0 : (fx > (T)(s.nx - 1) ? (T)(s.nx - 1) : fx);
    return iy * s.nx + (int)fx;
}

// reservoir buffer cell?  (the cell layers next to a reservoir face)
__device__ __forceinline__ bool in_buffer(const SimDev& s, int cell) {
    if (!s.has_reservoir) return false;
    int ix = cell % s.nx, iy = cell / s.nx;
    int nb = s.reservoir_cols;
    for (int f = 0; f < 4; ++f) {
        if (s.face[f].kind != kBcReservoir) continue;
        int axis = f >> 1;
        if (s.dim == 1 && axis == 0) continue;
        int i = axis == 0 ? ix : iy;
        int n = axis == 0 ? s.nx : s.ny;
        if (((f & 1) == 0 && i < nb) || ((f & 1) == 1 && i >= n - nb)) return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// advection with boundaries ("similar to DSMC", Table 1 steps 1-2)
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void fly(const SimDev& s, T& x, T& y, T* c, T t) {
    if (s.dim == 2) x += c[0] * t;
    y += c[1] * t;
    c[0] += (T)s.body[0] * t;
    c[1] += (T)s.body[1] * t;
    c[2] += (T)s.body[2] * t;
}

// Earliest surface reached within tau, skipping the one left last; faces
// 0..3 first, then plates; ties keep the lower index.  -1: none.
template <class T>
__device__ __forceinline__ int next_hit(const SimDev& s, T x, T y, const T* c, T tau, int last, T& t_hit) {
    int best = -1;
    T tb = 0;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        if (f == last) continue;
        int axis = f >> 1;
        if (s.dim == 1 && axis == 0) continue;
        if (s.face[f].kind == kBcPeriodic) continue;
        T pos = axis == 0 ? x : y;
        T vel = c[axis];
        T t;
        if ((f & 1) == 0) {
            if (!(vel < (T)0)) continue;
            t = ((T)s.lo[axis] - pos) / vel;
        } else {
            if (!(vel > (T)0)) continue;
            t = ((T)s.hi[axis] - pos) / vel;
        }
        if (t < (T)0) t = 0;
        if (t <= tau && (best < 0 || t < tb)) {
            best = f;
            tb = t;
        }
    }
    if (s.dim == 2) {
        for (int g = 0; g < s.nseg; ++g) {
            if (4 + g == last) continue;
            T vel = c[0];
            if (vel == (T)0) continue;
            T t = ((T)s.seg[g].pos - x) / vel;
            if (!(t > (T)0) || t > tau) continue;
            T yh = y + c[1] * t;
            if (yh < (T)s.seg[g].lo || yh > (T)s.seg[g].hi) continue;
            if (best < 0 || t < tb) {
                best = 4 + g;
                tb = t;
            }
        }
    }
    t_hit = tb;
    return best;
}

// full accommodation: Rayleigh normal speed, Gaussian tangential components
template <class T>
__device__ __forceinline__ void diffuse(const SimDev& s, uint32_t pid, uint32_t step, uint32_t k, int axis, T dir,
                                        double theta, double sqrt_theta, const double* u, T* c) {
    uint4 w = draw(s, pid, step, kWall, k);
    T cn = dev_sqrt<T>((T)(-2.0) * (T)theta * dev_log<T>(u01<T>(w.x)));
    T z0, z1;
    box_muller<T>(w.y, w.z, z0, z1);
    T st = (T)sqrt_theta;
    if (axis == 1) {
        c[1] = dir * cn;
        c[0] = (T)u[0] + st * z0;
        c[2] = (T)u[2] + st * z1;
    } else {
        c[0] = dir * cn;
        c[1] = (T)u[1] + st * z0;
        c[2] = (T)u[2] + st * z1;
    }
}

template <class T>
__device__ __forceinline__ T wrap(T v, double lo, double hi) {
    T L = (T)(hi - lo);
    T r = fmod(v - (T)lo, L);
    if (r < (T)0) r += L;
    return (T)lo + r;
}

// returns false when the particle left through a reservoir face
template <class T>
__device__ bool advect(const SimDev& s, uint32_t step, uint32_t pid, T& x, T& y, T* c) {
    T tau = (T)s.dt;
    int last = -1;
    for (int k = 0;; ++k) {
        T th;
        int hit = next_hit<T>(s, x, y, c, tau, last, th);
        if (hit < 0) {
            fly<T>(s, x, y, c, tau);
            break;
        }
        if (k == kMaxBounce) {
            fly<T>(s, x, y, c, tau);
            if (s.dim == 2 && !s.periodic_x) x = fmin(fmax(x, (T)s.lo[0]), (T)s.hi[0]);
            if (!s.periodic_y) y = fmin(fmax(y, (T)s.lo[1]), (T)s.hi[1]);
            atomicAdd(&s.dyn->counters[kCntClamp], 1ull);
            break;
        }
        fly<T>(s, x, y, c, th);
        tau -= th;
        last = hit;
        if (hit < 4) {
            int axis = hit >> 1;
            T wall = (hit & 1) ? (T)s.hi[axis] : (T)s.lo[axis];
            if (axis == 0) x = wall;
            else y = wall;
            T dir = (hit & 1) ? (T)-1 : (T)1;
            const FaceDev& F = s.face[hit];
            if (F.kind == kBcSpecular) {
                c[axis] = -c[axis];
            } else if (F.kind == kBcDiffuse) {
                diffuse<T>(s, pid, step, (uint32_t)k, axis, dir, F.theta, F.sqrt_theta, F.u, c);
            } else {
                atomicAdd(&s.dyn->counters[kCntRemoved], 1ull);
                return false;
            }
        } else {
            const SegDev& G = s.seg[hit - 4];
            T dir = c[0] > (T)0 ? (T)-1 : (T)1;
            x = (T)G.pos;
            if (G.kind == kBcSpecular) c[0] = -c[0];
            else diffuse<T>(s, pid, step, (uint32_t)k, 0, dir, G.theta, G.sqrt_theta, G.u, c);
        }
    }
    if (s.dim == 2 && s.periodic_x) x = wrap<T>(x, s.lo[0], s.hi[0]);
    if (s.periodic_y) y = wrap<T>(y, s.lo[1], s.hi[1]);
    return true;
}

// net flow through the counting plane: +1 for a particle that moved from
// below the plane to at or above it, -1 for the reverse (the FP32 path
// compares with the plane position rounded to FP32)
template <class T>
__device__ __forceinline__ void count_flux(const SimDev& s, T x0, T y0, T x1, T y1) {
    const T p = sizeof(T) == 4 ? (T)s.f_flux_pos : (T)s.flux_pos;
    const bool a = (s.flux_axis == 1 ? x0 : y0) >= p;
    const bool b = (s.flux_axis == 1 ? x1 : y1) >= p;
    if (a != b) atomicAdd(&s.dyn->counters[kCntFlux], b ? 1ull : ~0ull);   // ~0 is -1 modulo 2^64
}

// warp-aggregated increment of counter[key]; returns this lane's offset
__device__ __forceinline__ uint32_t aggregated_add(uint32_t* counter, uint32_t key) {
    unsigned active = __activemask();
    unsigned group = __match_any_sync(active, key);
    int leader = __ffs(group) - 1;
    uint32_t base = 0;
    if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(&counter[key], (uint32_t)__popc(group));
    base = __shfl_sync(group, base, leader);
    return base + (uint32_t)__popc(group & lanemask_lt());
}


template <class T>
__device__ __forceinline__ void make_particle(const SimDev& s, int cell, uint32_t pid, uint32_t step,
                                              uint32_t purpose, double theta, const double* u, T& x, T& y,
                                              T* c) {
    const int ix = cell % s.nx, iy = cell / s.nx;
    const uint4 w = draw(s, pid, step, purpose, 0);
    const uint4 v = draw(s, pid, step, purpose, 1);
    const double xl = s.dim == 2 ? s.lo[0] + ix * s.dx : 0.0;
    const double yl = s.lo[1] + iy * s.dy;
    x = s.dim == 2 ? (T)xl + u01<T>(w.x) * (T)s.dx : (T)0;
    y = (T)yl + u01<T>(w.y) * (T)s.dy;
    T z0, z1, z2, z3;
    box_muller<T>(v.x, v.y, z0, z1);
    box_muller<T>(v.z, v.w, z2, z3);
    const T sq = dev_sqrt<T>((T)theta);
    c[0] = (T)u[0] + sq * z0;
    c[1] = (T)u[1] + sq * z1;
    c[2] = (T)u[2] + sq * z2;
}

__device__ __forceinline__ int buffer_face(const SimDev& s, int cell) {
    int ix = cell % s.nx, iy = cell / s.nx;
    int nb = s.reservoir_cols;
    for (int f = 0; f < 4; ++f) {
        if (s.face[f].kind != kBcReservoir) continue;
        int axis = f >> 1;
        if (s.dim == 1 && axis == 0) continue;
        int i = axis == 0 ? ix : iy;
        int n = axis == 0 ? s.nx : s.ny;
        if (((f & 1) == 0 && i < nb) || ((f & 1) == 1 && i >= n - nb)) return f;
    }
    return -1;
}


__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}


struct Local {
    int valid;
    int N;
    double n, T, umag, a_sound, lambda, mu, nu, p, rho, theta;
    double u[3];
};

// local state of one cell from its shifted sums (means, Eq. 1; Eqs. 35-36)
__device__ __forceinline__ void local_state(const SimDev& s, int cell, Local& L, double* P6, double* Q3) {
    const int K = s.K;
    const double* M = s.mom;
    const int N = (int)M[cell];
    // with weighted particles the sums are W-weighted and N_eff = sum W
    // stands for N in the means and the density
    const double we = s.weighted ? s.wneff[cell] : (double)N;
    L.N = N;
    L.valid = 0;
    L.n = we * s.w;
    L.u[0] = L.u[1] = L.u[2] = 0.0;
    L.theta = 0.0;
    if (N < 1 || !(we > 0.0)) return;
    const double inv = 1.0 / we;
    const double d0 = M[K + cell] * inv, d1 = M[2 * K + cell] * inv, d2 = M[3 * K + cell] * inv;
    L.u[0] = s.ushift[cell] + d0;
    L.u[1] = s.ushift[K + cell] + d1;
    L.u[2] = s.ushift[2 * K + cell] + d2;
    const double m00 = M[4 * K + cell] * inv, m11 = M[5 * K + cell] * inv, m22 = M[6 * K + cell] * inv;
    const double m01 = M[7 * K + cell] * inv, m02 = M[8 * K + cell] * inv, m12 = M[9 * K + cell] * inv;
    double P[6] = {m00 - d0 * d0, m11 - d1 * d1, m22 - d2 * d2, m01 - d0 * d1, m02 - d0 * d2, m12 - d1 * d2};
    L.theta = (P[0] + P[1] + P[2]) / 3.0;
    if (P6)
        for (int k = 0; k < 6; ++k) P6[k] = P[k];
    if (Q3) {
        // central third moment from shifted raw moments: with d the mean of the
        // shifted velocities, E[|C|^2 C_i] = T3_i - d_i tr M2 - 2 (M2 d)_i + 2 d_i |d|^2
        const double t0 = M[10 * K + cell] * inv, t1 = M[11 * K + cell] * inv, t2 = M[12 * K + cell] * inv;
        const double tr = m00 + m11 + m22, dd = d0 * d0 + d1 * d1 + d2 * d2;
        const double md0 = m00 * d0 + m01 * d1 + m02 * d2;
        const double md1 = m01 * d0 + m11 * d1 + m12 * d2;
        const double md2 = m02 * d0 + m12 * d1 + m22 * d2;
        Q3[0] = 0.5 * (t0 - d0 * tr - 2.0 * md0 + 2.0 * d0 * dd);
        Q3[1] = 0.5 * (t1 - d1 * tr - 2.0 * md1 + 2.0 * d1 * dd);
        Q3[2] = 0.5 * (t2 - d2 * tr - 2.0 * md2 + 2.0 * d2 * dd);
    }
    L.valid = N >= 2 && (!s.weighted || we > 1.0) && L.theta > 0.0;
    if (!L.valid) return;
    L.T = L.theta / s.R;
    L.umag = sqrt(L.u[0] * L.u[0] + L.u[1] * L.u[1] + L.u[2] * L.u[2]);
    L.a_sound = sqrt(kGammaMono * L.theta);
    L.rho = L.n * s.mass;
    L.p = L.rho * L.theta;
    L.mu = s.mu_ref * pow(L.T / s.T_ref, s.omega);                              // Eq. 35
    L.nu = L.p / L.mu;                                                          // nu = p / mu
    L.lambda = 16.0 / (5.0 * sqrt(2.0 * kPi)) * L.mu / sqrt(L.rho * L.p);       // Eq. 36
}

// state a cell contributes to the Kn_GLL stencil (Eqs. 17-18): its
// instantaneous state, or (gll_average, after the first sample) the Eq. 34
// averages of n, u, T with lambda of Eq. 36 at that state
struct GradState {
    int valid;
    double n, T, umag, a_sound, lambda;
};

// plain pipeline only: the snapshot exists for handles created with gll_average
__device__ __forceinline__ bool gll_averaged(const SimDev& s) {
    return s.gll_average && s.gavg != nullptr && s.dyn->nsamples > 0;
}

// plain pipeline: k_moments copies the averaged n, T, |u| of its cell into
// gavg ([3][K]) before k_params updates the averages, so that the stencil
// reads every neighbour's average as it stood at the start of the step
__device__ __forceinline__ void snap_avg(const SimDev& s, int cell) {
    const int K = s.K;
    const double* A = s.avg;
    const double u0 = A[(size_t)1 * K + cell], u1 = A[(size_t)2 * K + cell], u2 = A[(size_t)3 * K + cell];
    s.gavg[cell] = A[cell];
    s.gavg[(size_t)K + cell] = A[(size_t)4 * K + cell];
    s.gavg[(size_t)2 * K + cell] = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
}

__device__ __forceinline__ void grad_from_avg(const SimDev& s, int cell, GradState& G) {
    const int K = s.K;
    G.n = s.gavg[cell];
    G.T = s.gavg[(size_t)K + cell];
    G.umag = s.gavg[(size_t)2 * K + cell];
    G.valid = G.n > 0.0 && G.T > 0.0;
    G.a_sound = G.lambda = 0.0;
    if (!G.valid) return;
    const double theta = s.R * G.T;
    G.a_sound = sqrt(kGammaMono * theta);
    const double rho = G.n * s.mass, p = rho * theta;
    const double mu = s.mu_ref * pow(G.T / s.T_ref, s.omega);                 // Eq. 35
    G.lambda = 16.0 / (5.0 * sqrt(2.0 * kPi)) * mu / sqrt(rho * p);           // Eq. 36
}

__device__ __forceinline__ void grad_from_local(const Local& L, GradState& G) {
    G.valid = L.valid;
    G.n = L.n;
    G.T = L.T;
    G.umag = L.umag;
    G.a_sound = L.a_sound;
    G.lambda = L.lambda;
}

// the stencil state of a cell as k_moments stored it (plain pipeline), or
// computed from its sums when no store exists
__device__ __forceinline__ void store_grad_state(const SimDev& s, int cell, const GradState& G) {
    const size_t K = (size_t)s.K;
    s.gloc[cell] = G.valid ? 1.0 : 0.0;
    s.gloc[K + cell] = G.n;
    s.gloc[2 * K + cell] = G.T;
    s.gloc[3 * K + cell] = G.umag;
    s.gloc[4 * K + cell] = G.a_sound;
    s.gloc[5 * K + cell] = G.lambda;
}

__device__ __forceinline__ void load_grad_state(const SimDev& s, int cell, GradState& G) {
    const size_t K = (size_t)s.K;
    G.valid = s.gloc[cell] != 0.0;
    G.n = s.gloc[K + cell];
    G.T = s.gloc[2 * K + cell];
    G.umag = s.gloc[3 * K + cell];
    G.a_sound = s.gloc[4 * K + cell];
    G.lambda = s.gloc[5 * K + cell];
}

__device__ __forceinline__ int neighbor(const SimDev& s, int cell, int axis, int dir) {
    const int ix = cell % s.nx, iy = cell / s.nx;
    if (axis == 0) {
        int j = ix + dir;
        if (j < 0 || j >= s.nx) {
            if (!s.periodic_x) return -1;
            j = (j + s.nx) % s.nx;
        }
        return iy * s.nx + j;
    }
    int j = iy + dir;
    if (j < 0 || j >= s.ny) {
        if (!s.periodic_y) return -1;
        j = (j + s.ny) % s.ny;
    }
    return j * s.nx + ix;
}


// time instant since t_n drawn from g_time (Eqs. 29-30), overflow-free form
template <class T>
__device__ __forceinline__ T sample_time(T U, T nu_es, T dt) {
    const T a = nu_es * dt;
    if (a < (T)1) return log1p(U * expm1(a)) / nu_es;
    return dt + log(U + ((T)1 - U) * exp(-a)) / nu_es;
}

struct CellRelax {
    double u[3], theta, L[6], p_relax, nu, nu_es, pne;
};

// new peculiar velocity of a relaxed particle: ES Gaussian with covariance
// theta I + s (1 - 1/Pr) sigma*/rho = s L L^T + (1 - s) theta I, s from Eq. 32
template <class T>
__device__ __forceinline__ void es_draw(const SimDev& s, const CellRelax& R, uint32_t pid, uint32_t step,
                                        const uint4& w, T* C) {
    const T t = sample_time<T>(u01<T>(w.y), (T)R.nu_es, (T)s.dt);
    // Eq. 32; the SP-ESBGK step holds the target for the whole step (Eq. 8b)
    const T sf = s.mode == kModeSPESBGK ? (T)1 : (T)R.pne + (T)(1.0 - R.pne) * exp(-(T)R.nu * t);
    const uint4 v = draw(s, pid, step, kRelax, 1);
    T z[6];
    box_muller<T>(w.z, w.w, z[0], z[1]);
    box_muller<T>(v.x, v.y, z[2], z[3]);
    box_muller<T>(v.z, v.w, z[4], z[5]);
    if (s.es_sampler) {
        // Eq. 10: one thermal component per (cosine) Box-Muller pair; Eq. 11:
        // C = S C*, S = I - s B, B = ((1 - Pr)/(2 Pr)) sigma*/(rho theta) in
        // the L slots (xx, yy, zz, xy, xz, yz)
        const T st = dev_sqrt<T>((T)R.theta);
        const T c0 = st * z[0], c1 = st * z[2], c2 = st * z[4];
        const T b00 = sf * (T)R.L[0], b11 = sf * (T)R.L[1], b22 = sf * (T)R.L[2];
        const T b01 = sf * (T)R.L[3], b02 = sf * (T)R.L[4], b12 = sf * (T)R.L[5];
        C[0] = ((T)1 - b00) * c0 - b01 * c1 - b02 * c2;
        C[1] = -b01 * c0 + ((T)1 - b11) * c1 - b12 * c2;
        C[2] = -b02 * c0 - b12 * c1 + ((T)1 - b22) * c2;
        return;
    }
    const T a = dev_sqrt<T>(sf), b = dev_sqrt<T>(((T)1 - sf) * (T)R.theta);
    C[0] = a * ((T)R.L[0] * z[0]) + b * z[3];
    C[1] = a * ((T)R.L[1] * z[0] + (T)R.L[2] * z[1]) + b * z[4];
    C[2] = a * ((T)R.L[3] * z[0] + (T)R.L[4] * z[1] + (T)R.L[5] * z[2]) + b * z[5];
}


}  // namespace usp
