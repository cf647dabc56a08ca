// usp_kernels.cu -- sm_103a kernels of the plain (one kernel per stage)
// USP-ESBGK step.  Each kernel walks a device-resident tile table, so the
// same launches serve one simulation or a batch of them and stay valid when
// captured in a CUDA graph.
//
// Stage order of one step n (Table 2 of the paper, unit particle weights):
//   k_stream   advection + boundaries, new cell, cell histogram,    (Table 2 step 3)
//              net count through the counting plane                 (Eq. 41)
//   k_scan     exclusive scan of the histogram                      (counting sort)
//   k_scatter  particles to their sorted slots                      (counting sort)
//   k_inject   refill of reservoir buffer cells
//   k_moments  per-cell sums of shifted velocities                  (Eq. 1)
//   k_params   per-cell P_ne, sigma*, q*, Cholesky, fields, Eq. 34  (Eqs. 16-18, 33, 35-36, 6c)
//   k_relax    Bernoulli or fixed-count selection, ES Gaussian or   (Eqs. 8b, 9, 27, 29-32,
//              Gallis-Torczynski sampling, conservation              10-11)
//   k_finish   advance the step counter and swap buffers
#include <algorithm>

#include "usp_device.cuh"

#include <cstdio>

namespace usp {

// ---------------------------------------------------------------------------
// K1: advection, new cell, histogram
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_stream(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                const int* __restrict__ ntiles) {
    __shared__ SimDev sim_sh;
    const int nt = *ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        __syncthreads();
        load_sim(sim_sh, sims[tile.x]);
        __syncthreads();
        const SimDev& s = sim_sh;
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
            const T x0 = x, y0 = y;
            bool alive = advect<T>(s, step, pid, x, y, c);
            if (s.flux_axis) count_flux<T>(s, x0, y0, x, y);
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

// cell of every particle without moving it (ordering an arbitrary loaded state)
template <class T>
__global__ void __launch_bounds__(256) k_assign(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                const int* __restrict__ ntiles) {
    __shared__ SimDev sim_sh;
    const int nt = *ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        __syncthreads();
        load_sim(sim_sh, sims[tile.x]);
        __syncthreads();
        const SimDev& s = sim_sh;
        const uint32_t n = s.dyn->n;
        PView<T> P = view<T>(s, s.dyn->cur);
        for (int j = threadIdx.x; j < kPTile; j += blockDim.x) {
            const int64_t i = (int64_t)tile.y + j;
            if (i >= (int64_t)n) break;
            // local cell of a slab (row0 = 0 without a decomposition),
            // clamped into the slab's cell range
            const int cell = min(max(cell_index<T>(s, s.dim == 2 ? P.x[i] : (T)0, P.y[i]) - s.row0 * s.nx, 0),
                                 s.K - 1);
            s.cell[i] = (uint32_t)cell;
            aggregated_add(s.count, (uint32_t)cell);
        }
    }
}

// ---------------------------------------------------------------------------
// K2: per-simulation exclusive scan of counts (+ injected) -> start
// ---------------------------------------------------------------------------
// with_inj: leave room for the reservoir refill of the step (the plain step);
// 0 when a loaded state is only being sorted (fused set-up)
__global__ void __launch_bounds__(1024) k_scan(const SimDev* __restrict__ sims, int nsims, int with_inj) {
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
                v = s.count[c] + (with_inj && s.has_reservoir ? s.inj_count[c] : 0u);
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
    __shared__ SimDev sim_sh;
    const int nt = *ntiles;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        __syncthreads();
        load_sim(sim_sh, sims[tile.x]);
        __syncthreads();
        const SimDev& s = sim_sh;
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
__global__ void __launch_bounds__(256) k_inject(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                const int* __restrict__ ntiles) {
    __shared__ SimDev sim_sh;
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        __syncthreads();
        load_sim(sim_sh, sims[tile.x]);
        __syncthreads();
        const SimDev& s = sim_sh;
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
// src_cur: the sums of the current buffer (the weighted step's moments of
// f^n) instead of the sorted one; with weighted particles every sum is
// W-weighted and the cell's weight sum goes to wneff
// One warp per block, the blocks striding over single cells: the FP64 sums
// are latency-bound, so even a domain of a hundred cells should spread
// over a hundred SMs.
template <class T>
__global__ void __launch_bounds__(32) k_moments(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                const int* __restrict__ ntiles, int src_cur) {
    __shared__ SimDev sim_sh;
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31;
    int loaded = -1;
    for (int g = blockIdx.x; g < nt * kCTile; g += gridDim.x) {
        const int2 tile = tiles[g / kCTile];
        if (tile.x != loaded) {
            __syncwarp();
            load_sim(sim_sh, sims[tile.x]);
            __syncwarp();
            loaded = tile.x;
        }
        const SimDev& s = sim_sh;
        const int K = s.K;
        const int buf = src_cur ? s.dyn->cur : s.dyn->cur ^ 1;
        PView<T> B = view<T>(s, buf);
        const double* Wt = s.weighted ? s.wgt[buf] : nullptr;
        const int cell = tile.y + g % kCTile;
        if (cell == 0 && lane == 0) s.fill[K] = 0;
        if (cell >= K) continue;
        {
            const uint32_t cap = (uint32_t)s.cap;
            const uint32_t b = min(s.start[cell], cap), e = min(s.start[cell + 1], cap);
            const double sh0 = s.ushift[cell], sh1 = s.ushift[K + cell], sh2 = s.ushift[2 * K + cell];
            double a[12], we = 0.0;
#pragma unroll
            for (int m = 0; m < 12; ++m) a[m] = 0.0;
            for (uint32_t i = b + lane; i < e; i += 32) {
                const double C0 = (double)B.c0[i] - sh0, C1 = (double)B.c1[i] - sh1, C2 = (double)B.c2[i] - sh2;
                const double c2 = C0 * C0 + C1 * C1 + C2 * C2;
                if (Wt) {
                    const double w = Wt[i];
                    we += w;
                    a[0] += w * C0; a[1] += w * C1; a[2] += w * C2;
                    a[3] += w * C0 * C0; a[4] += w * C1 * C1; a[5] += w * C2 * C2;
                    a[6] += w * C0 * C1; a[7] += w * C0 * C2; a[8] += w * C1 * C2;
                    a[9] += w * c2 * C0; a[10] += w * c2 * C1; a[11] += w * c2 * C2;
                    continue;
                }
                a[0] += C0; a[1] += C1; a[2] += C2;
                a[3] += C0 * C0; a[4] += C1 * C1; a[5] += C2 * C2;
                a[6] += C0 * C1; a[7] += C0 * C2; a[8] += C1 * C2;
                a[9] += c2 * C0; a[10] += c2 * C1; a[11] += c2 * C2;
            }
#pragma unroll
            for (int m = 0; m < 12; ++m) a[m] = warp_sum(a[m]);
            if (Wt) we = warp_sum(we);
            if (lane == 0) {
                s.mom[cell] = (double)(e - b);
                if (Wt) s.wneff[cell] = we;
#pragma unroll
                for (int m = 0; m < 12; ++m) s.mom[(size_t)(m + 1) * K + cell] = a[m];
                if (s.gloc) {
                    // the cell's stencil state once (from the sums just
                    // stored), for its neighbours' Kn_GLL
                    Local L;
                    local_state(s, cell, L, nullptr, nullptr);
                    GradState G;
                    grad_from_local(L, G);
                    store_grad_state(s, cell, G);
                }
                s.fill[cell] = 0;
                if (gll_averaged(s)) snap_avg(s, cell);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// K6: per-cell USP parameters, fields and the Eq. 34 average
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_params(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
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
                if (s.mode == kModeSP || s.mode == kModeSPESBGK) pne = 0.0;
                else if (s.mode == kModeFixed) pne = s.fixed_pne;
                else {
                    // gradient-length local Knudsen number (Eqs. 17-18): central
                    // differences, one-sided next to a missing or invalid neighbour
                    const bool avg = gll_averaged(s);
                    GradState G;
                    if (avg) grad_from_avg(s, cell, G);
                    else grad_from_local(L, G);
                    double kn = 0.0;   // no stencil state of its own: no gradient
                    if (G.valid) {
                        double Qc[3] = {G.n, G.T, G.umag};
                        double g2[3] = {0.0, 0.0, 0.0};
                        for (int axis = s.dim == 1 ? 1 : 0; axis < 2; ++axis) {
                            const double h = axis == 0 ? s.dx : s.dy;
                            int m = neighbor(s, cell, axis, -1), p = neighbor(s, cell, axis, +1);
                            GradState Gm, Gp;
                            if (m >= 0) {
                                if (avg) grad_from_avg(s, m, Gm);
                                else if (s.gloc) load_grad_state(s, m, Gm);
                                else {
                                    Local Lm;
                                    local_state(s, m, Lm, nullptr, nullptr);
                                    grad_from_local(Lm, Gm);
                                }
                                if (!Gm.valid) m = -1;
                            }
                            if (p >= 0) {
                                if (avg) grad_from_avg(s, p, Gp);
                                else if (s.gloc) load_grad_state(s, p, Gp);
                                else {
                                    Local Lp;
                                    local_state(s, p, Lp, nullptr, nullptr);
                                    grad_from_local(Lp, Gp);
                                }
                                if (!Gp.valid) p = -1;
                            }
                            double Qm[3], Qp[3];
                            if (m >= 0) { Qm[0] = Gm.n; Qm[1] = Gm.T; Qm[2] = Gm.umag; }
                            if (p >= 0) { Qp[0] = Gp.n; Qp[1] = Gp.T; Qp[2] = Gp.umag; }
                            for (int q = 0; q < 3; ++q) {
                                double d = 0.0;
                                if (m >= 0 && p >= 0) d = (Qp[q] - Qm[q]) / (2.0 * h);
                                else if (p >= 0) d = (Qp[q] - Qc[q]) / h;
                                else if (m >= 0) d = (Qc[q] - Qm[q]) / h;
                                g2[q] += d * d;
                            }
                        }
                        const double kn_rho = G.lambda * sqrt(g2[0]) / G.n;
                        const double kn_T = G.lambda * sqrt(g2[1]) / G.T;
                        const double kn_u = G.lambda * sqrt(g2[2]) / fmax(G.umag, G.a_sound);
                        kn = fmax(kn_rho, fmax(kn_T, kn_u));                 // Eq. 17
                    }
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
                if (s.es_sampler) {
                    // Eq. 11: B = ((1 - Pr)/(2 Pr)) sigma*/(rho theta); S = I - s B
                    const double beta = (1.0 - s.Pr) / (2.0 * s.Pr) / L.theta;
                    for (int k = 0; k < 6; ++k) pr[4 + k] = beta * sig[k];
                }
                if (s.weighted) {
                    // sigma* and q* per unit density for the weights of steps 4 and 7
                    for (int k = 0; k < 6; ++k) s.wst[(size_t)k * K + cell] = sig[k];
                    for (int k = 0; k < 3; ++k) s.wst[(size_t)(6 + k) * K + cell] = Q[k] / fq;
                }
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
// is the particle at slot i of the cell [b, e) relaxed?  Bernoulli: its
// selection word against the probability; fixed count (Eq. 9): its rank
// among the cell's selection words below ns.  `words` holds the cell's
// selection words (staged once per cell) when the cell fits, else null and
// the words are drawn again.
constexpr uint32_t kRelaxWords = 1024;
// new peculiar velocities of a cell's relaxed particles kept from the sums
// pass for the apply pass (larger cells draw them again)
constexpr uint32_t kRelaxKeep = 512;

template <class T>
__device__ __forceinline__ bool selected(const SimDev& s, const PView<T>& B, uint32_t b, uint32_t e, uint32_t i,
                                         uint32_t wx, T pth, uint32_t ns, uint32_t step, const uint32_t* words) {
    if (!s.selection) return u01<T>(wx) < pth;
    if (ns == 0) return false;
    uint32_t rank = 0;
    for (uint32_t j = b; j < e && rank < ns; ++j) {
        const uint32_t xj = words ? words[j - b] : draw(s, B.pid[j], step, kRelax, 0).x;
        rank += (xj < wx || (xj == wx && j < i)) ? 1u : 0u;
    }
    return rank < ns;
}

// One warp per block, the blocks striding over single cells (not tiles of
// cells): the relaxation is bound by FP64 issue (about two FP64 FMA per clock
// per SM on GB300), so even a domain of a hundred cells should spread over a
// hundred SMs.
template <class T>
__global__ void __launch_bounds__(32) k_relax(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                              const int* __restrict__ ntiles) {
    __shared__ SimDev sim_sh;
    __shared__ uint32_t sel_words[kRelaxWords];
    __shared__ double keep_c[3][kRelaxKeep];
    __shared__ unsigned char keep_sel[kRelaxKeep];
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31;
    int loaded = -1;
    for (int g = blockIdx.x; g < nt * kCTile; g += gridDim.x) {
        const int2 tile = tiles[g / kCTile];
        if (tile.x != loaded) {
            __syncwarp();
            load_sim(sim_sh, sims[tile.x]);
            __syncwarp();
            loaded = tile.x;
        }
        const SimDev& s = sim_sh;
        const int K = s.K;
        const uint32_t step = s.dyn->step;
        PView<T> B = view<T>(s, s.dyn->cur ^ 1);
        {
            const int cell = tile.y + g % kCTile;
            if (cell >= K) continue;
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
            // Eq. 9 fixed count: the ns particles with the smallest selection
            // words (ties: lower position first)
            const uint32_t ns = s.selection ? (uint32_t)floor((double)(e - b) * R.p_relax + 0.5) : 0u;
            const uint32_t* words = nullptr;
            if (s.selection && e - b <= kRelaxWords) {
                __syncwarp();
                for (uint32_t i = b + lane; i < e; i += 32) sel_words[i - b] = draw(s, B.pid[i], step, kRelax, 0).x;
                __syncwarp();
                words = sel_words;
            }
            const bool keep = e - b <= kRelaxKeep;
            __syncwarp();
            for (uint32_t i = b + lane; i < e; i += 32) {
                const uint32_t pid = B.pid[i];
                const uint4 w = draw(s, pid, step, kRelax, 0);
                const bool sel = selected<T>(s, B, b, e, i, w.x, pth, ns, step, words);
                if (keep) keep_sel[i - b] = sel ? 1 : 0;
                if (!sel) continue;
                T C[3];
                es_draw<T>(s, R, pid, step, w, C);
                if (keep)
                    for (int d = 0; d < 3; ++d) keep_c[d][i - b] = (double)C[d];
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
                    // pass 2: apply c = ubar_old + alpha (c' - ubar_new), with c'
                    // kept from pass 1 or drawn again
                    __syncwarp();
                    for (uint32_t i = b + lane; i < e; i += 32) {
                        T C[3];
                        if (keep) {
                            if (!keep_sel[i - b]) continue;
                            for (int d = 0; d < 3; ++d) C[d] = (T)keep_c[d][i - b];
                        } else {
                            const uint32_t pid = B.pid[i];
                            const uint4 w = draw(s, pid, step, kRelax, 0);
                            if (!selected<T>(s, B, b, e, i, w.x, pth, ns, step, words)) continue;
                            es_draw<T>(s, R, pid, step, w, C);
                        }
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
    __shared__ SimDev sim_sh;
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int t = blockIdx.x; t < nt; t += gridDim.x) {
        const int2 tile = tiles[t];
        __syncthreads();
        load_sim(sim_sh, sims[tile.x]);
        __syncthreads();
        const SimDev& s = sim_sh;
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
void launch_assign(const Launch& L, bool fp64) {
    if (fp64) k_assign<double><<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
    else k_assign<float><<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
}
void launch_scan(const Launch& L, bool with_inj) { k_scan<<<L.nsims, 1024, 0, L.stream>>>(L.sims, L.nsims, with_inj ? 1 : 0); }
void launch_scatter(const Launch& L, bool fp64) {
    if (fp64) k_scatter<double><<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
    else k_scatter<float><<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
}
void launch_inject(const Launch& L, bool fp64) {
    if (fp64) k_inject<double><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    else k_inject<float><<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
}
void launch_moments(const Launch& L, bool fp64) { launch_moments_src(L, fp64, false); }
void launch_moments_src(const Launch& L, bool fp64, bool src_cur) {
    const int sc = src_cur ? 1 : 0;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(L.grid_c * kCTile, 32 * sms));
    if (fp64) k_moments<double><<<grid, 32, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles, sc);
    else k_moments<float><<<grid, 32, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles, sc);
}
void launch_params(const Launch& L) { k_params<<<L.grid_c, 32, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles); }
void launch_relax(const Launch& L, bool fp64) {
    // one warp per cell slot of the tiles, at most 32 one-warp blocks per SM
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(L.grid_c * kCTile, 32 * sms));
    if (fp64) k_relax<double><<<grid, 32, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    else k_relax<float><<<grid, 32, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
}
void launch_finish(const Launch& L) { k_finish<<<(L.nsims + 127) / 128, 128, 0, L.stream>>>(L.sims, L.nsims); }

// user-supplied particles (host layout: pos[n][2], vel[n][3] in FP64) into
// the storage planes of buffer 0.  pos, vel and ids are device copies of the
// caller's arrays or, for page-locked host memory, the arrays themselves
// read through their mapped device addresses; any of pos, vel, ids may be
// null (that part is not read).  ids go to pid (when non-null); with
// next_pid non-null, one past the largest id is folded into *next_pid (one
// atomic per warp).
template <class T>
__global__ void k_unpack(const double* __restrict__ pos, const double* __restrict__ vel,
                         const uint32_t* __restrict__ ids, int64_t n, int dim, T* x, T* y, T* v0, T* v1, T* v2,
                         uint32_t* pid, uint32_t* next_pid) {
    uint32_t top = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (pos) {
            if (dim == 2) x[i] = (T)pos[2 * i];
            y[i] = (T)pos[2 * i + 1];
        }
        if (vel) {
            v0[i] = (T)vel[3 * i];
            v1[i] = (T)vel[3 * i + 1];
            v2[i] = (T)vel[3 * i + 2];
        }
        if (ids) {
            const uint32_t id = ids[i];
            if (pid) pid[i] = id;
            top = max(top, id + 1u);
        }
    }
    if (next_pid) {
        top = __reduce_max_sync(0xffffffffu, top);
        if ((threadIdx.x & 31) == 0 && top) atomicMax(next_pid, top);
    }
}

void launch_unpack(const SimDev& s, bool fp64, const double* pos, const double* vel, const uint32_t* ids,
                   bool ids_to_plane, uint32_t* next_pid, int64_t n, cudaStream_t st) {
    if (n <= 0) return;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    uint32_t* pid = ids_to_plane ? s.pid[0] : nullptr;
    if (fp64)
        k_unpack<double><<<grid, 256, 0, st>>>(pos, vel, ids, n, s.dim, (double*)s.pos[0][0], (double*)s.pos[0][1],
                                               (double*)s.vel[0][0], (double*)s.vel[0][1], (double*)s.vel[0][2],
                                               pid, next_pid);
    else
        k_unpack<float><<<grid, 256, 0, st>>>(pos, vel, ids, n, s.dim, (float*)s.pos[0][0], (float*)s.pos[0][1],
                                              (float*)s.vel[0][0], (float*)s.vel[0][1], (float*)s.vel[0][2],
                                              pid, next_pid);
}

// clear up to kZeroRanges device ranges of 32-bit words in one launch
__global__ void k_zero(ZeroList z) {
    for (int r = 0; r < z.n; ++r) {
        uint32_t* p = (uint32_t*)z.p[r];
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < z.words[r];
             i += (size_t)gridDim.x * blockDim.x)
            p[i] = 0u;
    }
}

void launch_zero(const ZeroList& z, cudaStream_t st) {
    size_t most = 0;
    for (int r = 0; r < z.n; ++r) most = std::max(most, z.words[r]);
    if (most == 0) return;
    const int grid = (int)std::min<size_t>((most + 255) / 256, 152 * 8);
    k_zero<<<grid, 256, 0, st>>>(z);
}

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
