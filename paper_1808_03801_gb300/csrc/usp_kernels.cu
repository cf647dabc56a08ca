// usp_kernels.cu -- sm_103a kernels of the plain (one kernel per stage)
// USP-ESBGK step.  Each kernel walks a device-resident tile table, so the
// same launches serve one simulation or a batch of them and stay valid when
// captured in a CUDA graph.
//
// Stage order of one step n (Table 2 of the paper, unit particle weights):
//   k_stream   advection + boundaries, new cell, cell histogram     (Table 2 step 3)
//   k_scan     exclusive scan of the histogram                      (counting sort)
//   k_scatter  particles to their sorted slots                      (counting sort)
//   k_inject   refill of reservoir buffer cells
//   k_moments  per-cell sums of shifted velocities                  (Eq. 1)
//   k_params   per-cell P_ne, sigma*, q*, Cholesky, fields, Eq. 34  (Eqs. 16-18, 33, 35-36, 6c)
//   k_relax    Bernoulli relaxation, ES sampling, conservation      (Eqs. 8b, 9, 27, 29-32)
//   k_finish   advance the step counter and swap buffers
#include "usp_internal.cuh"

#include <cstdio>

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

// ---------------------------------------------------------------------------
// K1: advection, new cell, histogram
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_stream(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                const int* __restrict__ ntiles) {
    const int nt = *ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        const SimDev& s = sims[tile.x];
        const uint32_t n = s.dyn->n;
        const uint32_t step = s.dyn->step;
        const int cur = s.dyn->cur;
        PView<T> P = view<T>(s, cur);
        for (int j = threadIdx.x; j < kPTile; j += blockDim.x) {
            const int64_t i = (int64_t)tile.y + j;
            if (i >= (int64_t)n) break;
            T x = s.dim == 2 ? P.x[i] : (T)0;
            T y = P.y[i];
            T c[3] = {P.c0[i], P.c1[i], P.c2[i]};
            const uint32_t pid = P.pid[i];
            bool alive = advect<T>(s, step, pid, x, y, c);
            int cell = s.K;
            if (alive) {
                cell = cell_index<T>(s, x, y);
                if (in_buffer(s, cell)) {
                    cell = s.K;
                    atomicAdd(&s.dyn->counters[kCntRemoved], 1ull);
                }
            }
            if (s.dim == 2) P.x[i] = x;
            P.y[i] = y;
            P.c0[i] = c[0];
            P.c1[i] = c[1];
            P.c2[i] = c[2];
            s.cell[i] = (uint32_t)cell;
            if (cell < s.K) aggregated_add(s.count, (uint32_t)cell);
        }
    }
}

// ---------------------------------------------------------------------------
// K2: per-simulation exclusive scan of counts (+ injected) -> start
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan(const SimDev* __restrict__ sims, int nsims) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    for (int si = blockIdx.x; si < nsims; si += gridDim.x) {
        const SimDev& s = sims[si];
        const int K = s.K;
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (int base = 0; base <= K; base += blockDim.x) {
            const int c = base + threadIdx.x;
            uint32_t v = 0;
            if (c < K) {
                v = s.count[c] + (s.has_reservoir ? s.inj_count[c] : 0u);
                s.count[c] = 0;
            } else if (c == K) {
                s.count[c] = 0;   // removed particles are not kept
            }
            // inclusive warp scan
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if ((threadIdx.x & 31) >= o) x += y;
            }
            if ((threadIdx.x & 31) == 31) warp_sums[threadIdx.x >> 5] = x;
            __syncthreads();
            if (threadIdx.x < 32) {
                uint32_t ws = threadIdx.x < (blockDim.x >> 5) ? warp_sums[threadIdx.x] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
                    if (threadIdx.x >= o) ws += y;
                }
                warp_sums[threadIdx.x] = ws;
            }
            __syncthreads();
            const uint32_t before = (threadIdx.x >= 32 ? warp_sums[(threadIdx.x >> 5) - 1] : 0u) + carry;
            if (c <= K) s.start[c] = before + x - v;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) carry = before + x;
            __syncthreads();
        }
        if (threadIdx.x == 0) s.start[K + 1] = carry;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// K3: scatter to sorted slots
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_scatter(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                 const int* __restrict__ ntiles) {
    const int nt = *ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        const SimDev& s = sims[tile.x];
        const uint32_t n = s.dyn->n;
        const int cur = s.dyn->cur;
        PView<T> A = view<T>(s, cur), B = view<T>(s, cur ^ 1);
        for (int j = threadIdx.x; j < kPTile; j += blockDim.x) {
            const int64_t i = (int64_t)tile.y + j;
            if (i >= (int64_t)n) break;
            const uint32_t cell = s.cell[i];
            if (cell >= (uint32_t)s.K) continue;
            const uint32_t slot = s.start[cell] + aggregated_add(s.fill, cell);
            if ((int64_t)slot >= s.cap) {
                atomicAdd(&s.dyn->counters[kCntOverflow], 1ull);
                continue;
            }
            if (s.dim == 2) B.x[slot] = A.x[i];
            B.y[slot] = A.y[i];
            B.c0[slot] = A.c0[i];
            B.c1[slot] = A.c1[i];
            B.c2[slot] = A.c2[i];
            B.pid[slot] = A.pid[i];
        }
    }
}

// ---------------------------------------------------------------------------
// K4: reservoir buffer cells: fresh particles from the reservoir Maxwellian
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void make_particle(const SimDev& s, int cell, uint32_t pid, uint32_t step,
                                              uint32_t purpose, double theta, const double* u, T& x, T& y,
                                              T* c) {
    const int ix = cell % s.nx, iy = cell / s.nx;
    const uint4 w = draw(s, pid, step, purpose, 0);
    const uint4 v = draw(s, pid, step, purpose, 1);
    const double xl = s.dim == 2 ? s.lo[0] + ix * s.dx : 0.0;
    const double yl = s.lo[1] + iy * s.dy;
    x = (T)(s.dim == 2 ? xl + u01<double>(w.x) * s.dx : 0.0);
    y = (T)(yl + u01<double>(w.y) * s.dy);
    double z0, z1, z2, z3;
    box_muller<double>(v.x, v.y, z0, z1);
    box_muller<double>(v.z, v.w, z2, z3);
    const double sq = sqrt(theta);
    c[0] = (T)(u[0] + sq * z0);
    c[1] = (T)(u[1] + sq * z1);
    c[2] = (T)(u[2] + sq * z2);
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

template <class T>
__global__ void __launch_bounds__(256) k_inject(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                const int* __restrict__ ntiles) {
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        const SimDev& s = sims[tile.x];
        if (!s.has_reservoir) continue;
        const uint32_t step = s.dyn->step, next_pid = s.dyn->next_pid;
        PView<T> B = view<T>(s, s.dyn->cur ^ 1);
        for (int cc = warp; cc < kCTile; cc += nwarps) {
            const int cell = tile.y + cc;
            if (cell >= s.K) break;
            const uint32_t cnt = s.inj_count[cell];
            if (cnt == 0) continue;
            const int f = buffer_face(s, cell);
            const FaceDev& F = s.face[f];
            const uint32_t base = s.start[cell] + s.fill[cell];
            for (uint32_t k = lane; k < cnt; k += 32) {
                const uint32_t slot = base + k;
                if ((int64_t)slot >= s.cap) {
                    atomicAdd(&s.dyn->counters[kCntOverflow], 1ull);
                    continue;
                }
                const uint32_t pid = next_pid + s.inj_pidoff[cell] + k;
                T x, y, c[3];
                make_particle<T>(s, cell, pid, step, kInject, F.theta, F.u, x, y, c);
                if (s.dim == 2) B.x[slot] = x;
                B.y[slot] = y;
                B.c0[slot] = c[0];
                B.c1[slot] = c[1];
                B.c2[slot] = c[2];
                B.pid[slot] = pid;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K5: per-cell sums of velocities shifted by the previous cell mean (Eq. 1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__global__ void __launch_bounds__(256) k_moments(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                 const int* __restrict__ ntiles) {
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        const SimDev& s = sims[tile.x];
        const int K = s.K;
        PView<T> B = view<T>(s, s.dyn->cur ^ 1);
        if (tile.y == 0 && threadIdx.x == 0) s.fill[K] = 0;
        for (int cc = warp; cc < kCTile; cc += nwarps) {
            const int cell = tile.y + cc;
            if (cell >= K) break;
            const uint32_t cap = (uint32_t)s.cap;
            const uint32_t b = min(s.start[cell], cap), e = min(s.start[cell + 1], cap);
            const double sh0 = s.ushift[cell], sh1 = s.ushift[K + cell], sh2 = s.ushift[2 * K + cell];
            double a[12];
#pragma unroll
            for (int m = 0; m < 12; ++m) a[m] = 0.0;
            for (uint32_t i = b + lane; i < e; i += 32) {
                const double C0 = (double)B.c0[i] - sh0, C1 = (double)B.c1[i] - sh1, C2 = (double)B.c2[i] - sh2;
                const double c2 = C0 * C0 + C1 * C1 + C2 * C2;
                a[0] += C0; a[1] += C1; a[2] += C2;
                a[3] += C0 * C0; a[4] += C1 * C1; a[5] += C2 * C2;
                a[6] += C0 * C1; a[7] += C0 * C2; a[8] += C1 * C2;
                a[9] += c2 * C0; a[10] += c2 * C1; a[11] += c2 * C2;
            }
#pragma unroll
            for (int m = 0; m < 12; ++m) a[m] = warp_sum(a[m]);
            if (lane == 0) {
                s.mom[cell] = (double)(e - b);
#pragma unroll
                for (int m = 0; m < 12; ++m) s.mom[(size_t)(m + 1) * K + cell] = a[m];
                s.fill[cell] = 0;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K6: per-cell USP parameters, fields and the Eq. 34 average
// ---------------------------------------------------------------------------
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
    L.N = N;
    L.valid = 0;
    L.n = N * s.w;
    L.u[0] = L.u[1] = L.u[2] = 0.0;
    L.theta = 0.0;
    if (N < 1) return;
    const double inv = 1.0 / N;
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
    L.valid = N >= 2 && L.theta > 0.0;
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

__global__ void __launch_bounds__(128) k_params(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                const int* __restrict__ ntiles) {
    const int nt = *ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        const SimDev& s = sims[tile.x];
        const int K = s.K;
        for (int cc = threadIdx.x; cc < kCTile; cc += blockDim.x) {
            const int cell = tile.y + cc;
            if (cell >= K) break;
            Local L;
            double P[6], Q[3];
            local_state(s, cell, L, P, Q);
            double f[kNFields];
            for (int k = 0; k < kNFields; ++k) f[k] = 0.0;
            f[0] = L.n;
            f[15] = L.N;
            if (L.N >= 1) {
                f[1] = L.u[0];
                f[2] = L.u[1];
                f[3] = L.u[2];
            }
            double* prm = s.prm;
            double pr[kNPrm];
            for (int k = 0; k < kNPrm; ++k) pr[k] = 0.0;
            pr[0] = L.u[0];
            pr[1] = L.u[1];
            pr[2] = L.u[2];
            pr[3] = L.theta;
            if (L.valid) {
                double pne;
                if (s.mode == kModeSP) pne = 0.0;
                else if (s.mode == kModeFixed) pne = s.fixed_pne;
                else {
                    // gradient-length local Knudsen number (Eqs. 17-18): central
                    // differences, one-sided next to a missing or invalid neighbour
                    double Qc[3] = {L.n, L.T, L.umag};
                    double g2[3] = {0.0, 0.0, 0.0};
                    for (int axis = s.dim == 1 ? 1 : 0; axis < 2; ++axis) {
                        const double h = axis == 0 ? s.dx : s.dy;
                        int m = neighbor(s, cell, axis, -1), p = neighbor(s, cell, axis, +1);
                        Local Lm, Lp;
                        if (m >= 0) {
                            local_state(s, m, Lm, nullptr, nullptr);
                            if (!Lm.valid) m = -1;
                        }
                        if (p >= 0) {
                            local_state(s, p, Lp, nullptr, nullptr);
                            if (!Lp.valid) p = -1;
                        }
                        double Qm[3], Qp[3];
                        if (m >= 0) { Qm[0] = Lm.n; Qm[1] = Lm.T; Qm[2] = Lm.umag; }
                        if (p >= 0) { Qp[0] = Lp.n; Qp[1] = Lp.T; Qp[2] = Lp.umag; }
                        for (int q = 0; q < 3; ++q) {
                            double d = 0.0;
                            if (m >= 0 && p >= 0) d = (Qp[q] - Qm[q]) / (2.0 * h);
                            else if (p >= 0) d = (Qp[q] - Qc[q]) / h;
                            else if (m >= 0) d = (Qc[q] - Qm[q]) / h;
                            g2[q] += d * d;
                        }
                    }
                    const double kn_rho = L.lambda * sqrt(g2[0]) / L.n;
                    const double kn_T = L.lambda * sqrt(g2[1]) / L.T;
                    const double kn_u = L.lambda * sqrt(g2[2]) / fmax(L.umag, L.a_sound);
                    const double kn = fmax(kn_rho, fmax(kn_T, kn_u));       // Eq. 17
                    pne = exp(-kn / kKnC);                                   // Eq. 16
                }
                const double fs = 1.0 + 0.5 * s.dt * L.nu * pne;            // Eq. 33
                const double fq = 1.0 + 0.5 * s.dt * L.nu * s.Pr * pne;
                const double sig[6] = {(P[0] - L.theta) / fs, (P[1] - L.theta) / fs, (P[2] - L.theta) / fs,
                                       P[3] / fs, P[4] / fs, P[5] / fs};
                const double b = 1.0 - 1.0 / s.Pr;                          // Eq. 6c
                const double A00 = L.theta + b * sig[0], A11 = L.theta + b * sig[1], A22 = L.theta + b * sig[2];
                const double A10 = b * sig[3], A20 = b * sig[4], A21 = b * sig[5];
                double l00 = 0, l10 = 0, l11 = 0, l20 = 0, l21 = 0, l22 = 0;
                bool ok = A00 > 0.0;
                if (ok) {
                    l00 = sqrt(A00);
                    l10 = A10 / l00;
                    l20 = A20 / l00;
                    const double d1 = A11 - l10 * l10;
                    ok = d1 > 0.0;
                    if (ok) {
                        l11 = sqrt(d1);
                        l21 = (A21 - l20 * l10) / l11;
                        const double d2 = A22 - l20 * l20 - l21 * l21;
                        ok = d2 > 0.0;
                        if (ok) l22 = sqrt(d2);
                    }
                }
                if (!ok) {
                    const double r = sqrt(L.theta);
                    l00 = l11 = l22 = r;
                    l10 = l20 = l21 = 0.0;
                    atomicAdd(&s.dyn->counters[kCntChol], 1ull);
                }
                pr[4] = l00; pr[5] = l10; pr[6] = l11; pr[7] = l20; pr[8] = l21; pr[9] = l22;
                pr[10] = -expm1(-s.Pr * L.nu * s.dt);                       // Eqs. 8b, 9
                pr[11] = L.nu;
                pr[12] = s.Pr * L.nu;
                pr[13] = pne;
                pr[14] = 1.0;
                f[4] = L.T;
                f[5] = L.p + L.rho * sig[0];
                f[6] = L.p + L.rho * sig[1];
                f[7] = L.p + L.rho * sig[2];
                f[8] = L.rho * sig[3];
                f[9] = L.rho * sig[4];
                f[10] = L.rho * sig[5];
                f[11] = L.rho * Q[0] / fq;
                f[12] = L.rho * Q[1] / fq;
                f[13] = L.rho * Q[2] / fq;
                f[14] = pne;
            }
            for (int k = 0; k < kNPrm; ++k) prm[(size_t)k * K + cell] = pr[k];
            const bool first = s.dyn->nsamples == 0;
            for (int k = 0; k < kNFields; ++k) {
                s.inst[(size_t)k * K + cell] = f[k];
                double* a = &s.avg[(size_t)k * K + cell];
                *a = first ? f[k] : s.avg_keep * *a + f[k] * s.avg_new;   // Eq. 34
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K7: relaxation of each cell with conservation of momentum and energy
// ---------------------------------------------------------------------------
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
    const T sf = (T)R.pne + (T)(1.0 - R.pne) * exp(-(T)R.nu * t);
    const uint4 v = draw(s, pid, step, kRelax, 1);
    T z[6];
    box_muller<T>(w.z, w.w, z[0], z[1]);
    box_muller<T>(v.x, v.y, z[2], z[3]);
    box_muller<T>(v.z, v.w, z[4], z[5]);
    const T a = dev_sqrt<T>(sf), b = dev_sqrt<T>(((T)1 - sf) * (T)R.theta);
    C[0] = a * ((T)R.L[0] * z[0]) + b * z[3];
    C[1] = a * ((T)R.L[1] * z[0] + (T)R.L[2] * z[1]) + b * z[4];
    C[2] = a * ((T)R.L[3] * z[0] + (T)R.L[4] * z[1] + (T)R.L[5] * z[2]) + b * z[5];
}

template <class T>
__global__ void __launch_bounds__(256) k_relax(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                               const int* __restrict__ ntiles) {
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        const SimDev& s = sims[tile.x];
        const int K = s.K;
        const uint32_t step = s.dyn->step;
        PView<T> B = view<T>(s, s.dyn->cur ^ 1);
        for (int cc = warp; cc < kCTile; cc += nwarps) {
            const int cell = tile.y + cc;
            if (cell >= K) break;
            const double* pr = s.prm;
            const bool valid = pr[(size_t)14 * K + cell] != 0.0;
            CellRelax R;
            for (int d = 0; d < 3; ++d) R.u[d] = pr[(size_t)d * K + cell];
            if (lane == 0 && s.mom[cell] >= 1.0)
                for (int d = 0; d < 3; ++d) s.ushift[(size_t)d * K + cell] = R.u[d];
            if (!valid) continue;
            R.theta = pr[(size_t)3 * K + cell];
            for (int d = 0; d < 6; ++d) R.L[d] = pr[(size_t)(4 + d) * K + cell];
            R.p_relax = pr[(size_t)10 * K + cell];
            R.nu = pr[(size_t)11 * K + cell];
            R.nu_es = pr[(size_t)12 * K + cell];
            R.pne = pr[(size_t)13 * K + cell];
            const uint32_t cap = (uint32_t)s.cap;
            const uint32_t b = min(s.start[cell], cap), e = min(s.start[cell + 1], cap);
            const T pth = (T)R.p_relax;
            // pass 1: sums over the relaxed subset (velocities relative to the cell mean)
            double nr = 0, so[3] = {0, 0, 0}, eo = 0, sn[3] = {0, 0, 0}, en = 0;
            for (uint32_t i = b + lane; i < e; i += 32) {
                const uint32_t pid = B.pid[i];
                const uint4 w = draw(s, pid, step, kRelax, 0);
                if (!(u01<T>(w.x) < pth)) continue;
                T C[3];
                es_draw<T>(s, R, pid, step, w, C);
                const double o0 = (double)B.c0[i] - R.u[0], o1 = (double)B.c1[i] - R.u[1],
                             o2 = (double)B.c2[i] - R.u[2];
                nr += 1.0;
                so[0] += o0; so[1] += o1; so[2] += o2;
                eo += o0 * o0 + o1 * o1 + o2 * o2;
                sn[0] += (double)C[0]; sn[1] += (double)C[1]; sn[2] += (double)C[2];
                en += (double)C[0] * C[0] + (double)C[1] * C[1] + (double)C[2] * C[2];
            }
            nr = warp_sum(nr);
            for (int d = 0; d < 3; ++d) {
                so[d] = warp_sum(so[d]);
                sn[d] = warp_sum(sn[d]);
            }
            eo = warp_sum(eo);
            en = warp_sum(en);
            int applied = 0;
            if (nr >= 2.0) {
                const double inv = 1.0 / nr;
                const double Eo = eo - (so[0] * so[0] + so[1] * so[1] + so[2] * so[2]) * inv;
                const double En = en - (sn[0] * sn[0] + sn[1] * sn[1] + sn[2] * sn[2]) * inv;
                if (En > 0.0) {
                    applied = (int)nr;
                    const double alpha = sqrt(Eo / En);
                    const double uo[3] = {R.u[0] + so[0] * inv, R.u[1] + so[1] * inv, R.u[2] + so[2] * inv};
                    const double mn[3] = {sn[0] * inv, sn[1] * inv, sn[2] * inv};
                    // pass 2: redraw and apply c = ubar_old + alpha (c' - ubar_new)
                    for (uint32_t i = b + lane; i < e; i += 32) {
                        const uint32_t pid = B.pid[i];
                        const uint4 w = draw(s, pid, step, kRelax, 0);
                        if (!(u01<T>(w.x) < pth)) continue;
                        T C[3];
                        es_draw<T>(s, R, pid, step, w, C);
                        B.c0[i] = (T)(uo[0] + alpha * ((double)C[0] - mn[0]));
                        B.c1[i] = (T)(uo[1] + alpha * ((double)C[1] - mn[1]));
                        B.c2[i] = (T)(uo[2] + alpha * ((double)C[2] - mn[2]));
                    }
                }
            }
            if (lane == 0) {
                s.prm[(size_t)15 * K + cell] = applied;
                if (applied) atomicAdd(&s.dyn->counters[kCntRelaxed], (unsigned long long)applied);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K8: end of step
// ---------------------------------------------------------------------------
__global__ void k_finish(const SimDev* __restrict__ sims, int nsims) {
    for (int si = blockIdx.x * blockDim.x + threadIdx.x; si < nsims; si += gridDim.x * blockDim.x) {
        const SimDev& s = sims[si];
        SimDyn* d = s.dyn;
        uint32_t n = s.start[s.K];
        if ((int64_t)n > s.cap) n = (uint32_t)s.cap;
        d->n = n;
        if (s.has_reservoir) {
            d->next_pid += s.inj_total;
            d->counters[kCntInjected] += s.inj_total;
        }
        d->cur ^= 1;
        d->step += 1;
        d->nsamples += 1;
    }
}

// ---------------------------------------------------------------------------
// initial fill (Table 2 step 1): warp per cell; counts and offsets from the host
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_init_fill(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                   const int* __restrict__ ntiles, const double* __restrict__ reg_theta,
                                                   const double* __restrict__ reg_u, const int* __restrict__ cell_reg) {
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        const SimDev& s = sims[tile.x];
        PView<T> A = view<T>(s, 0);
        for (int cc = warp; cc < kCTile; cc += nwarps) {
            const int cell = tile.y + cc;
            if (cell >= s.K) break;
            const int r = cell_reg[cell];
            if (r < 0) continue;
            const uint32_t b = s.start[cell], e = s.start[cell + 1];
            for (uint32_t i = b + lane; i < e; i += 32) {
                T x, y, c[3];
                make_particle<T>(s, cell, i, 0u, kInit, reg_theta[r], reg_u + 3 * r, x, y, c);
                if (s.dim == 2) A.x[i] = x;
                A.y[i] = y;
                A.c0[i] = c[0];
                A.c1[i] = c[1];
                A.c2[i] = c[2];
                A.pid[i] = i;
            }
        }
    }
}

__global__ void k_debug_philox(int64_t n, const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1,
                               uint32_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint4 r = philox(make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]), make_uint2(k0, k1));
        out[4 * i] = r.x;
        out[4 * i + 1] = r.y;
        out[4 * i + 2] = r.z;
        out[4 * i + 3] = r.w;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void launch_stream(const Launch& L, bool fp64) {
    if (fp64) k_stream<double><<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
    else k_stream<float><<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
}
void launch_scan(const Launch& L) { k_scan<<<L.nsims, 1024, 0, L.stream>>>(L.sims, L.nsims); }
void launch_scatter(const Launch& L, bool fp64) {
    if (fp64) k_scatter<double><<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
    else k_scatter<float><<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
}
void launch_inject(const Launch& L, bool fp64) {
    if (fp64) k_inject<double><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    else k_inject<float><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
}
void launch_moments(const Launch& L, bool fp64) {
    if (fp64) k_moments<double><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    else k_moments<float><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
}
void launch_params(const Launch& L) { k_params<<<L.grid_c, 64, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles); }
void launch_relax(const Launch& L, bool fp64) {
    if (fp64) k_relax<double><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    else k_relax<float><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
}
void launch_finish(const Launch& L) { k_finish<<<(L.nsims + 127) / 128, 128, 0, L.stream>>>(L.sims, L.nsims); }

void launch_init(const Launch& L, bool fp64, const double* reg_theta, const double* reg_u, const int* cell_reg) {
    if (fp64)
        k_init_fill<double><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles, reg_theta, reg_u, cell_reg);
    else
        k_init_fill<float><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles, reg_theta, reg_u, cell_reg);
}

cudaError_t debug_philox(int64_t n, const uint32_t* d_ctr, uint32_t k0, uint32_t k1, uint32_t* d_out,
                         cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_debug_philox<<<grid, 256, 0, st>>>(n, d_ctr, k0, k1, d_out);
    return cudaGetLastError();
}

}  // namespace usp
