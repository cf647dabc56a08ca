// usp_weighted.cu -- the weighted added particles of the USP-ESBGK scheme
// (Table 2 steps 2, 4 and 7; Eqs. 22-28 and the third term of Eq. 27) on the
// plain FP64 pipeline, one simulation per handle.
//
// One step, in the order of Table 2:
//   sort       the state in cell order (cell, histogram, scan, scatter)
//   step 2     W-weighted moments of f^n per cell; N_a particles per cell,
//              Maxwellian at u^n, theta^n, weights W^n of Eq. 26
//   step 3     the flight of every particle (k_stream), the counting sort
//   moments    W-weighted moments and parameters of f~* (k_moments, k_params)
//   step 4     N_a particles per cell with weights W* from sigma*, q* of
//              Eq. 33; sorted into their cells
//   steps 5-6  Bernoulli selection (Eq. 9); int(sum of the selected weights)
//              of them, smallest selection words first, take weight 1 and a
//              velocity from f_G(t) (Eqs. 28-32); the other selected ones are
//              deleted; the reassigned set carries the selected set's mean
//              velocity and thermal energy per unit weight
//   step 7     N_a particles per cell with W' = -W* 2 (1 - e^-a) / a, the
//              third term of Eq. 27
//   sort       compaction (deleted particles go) and the step-7 particles
//              into their cells; end of the step
// The readings behind the choices (the N_a rounding and weight prefactor,
// the averaged weight fields, the Eq. 28 rounding and order) are those of
// the reference implementation in the oracle; the random numbers come from
// the same counters: purpose kAdd keyed by the new particle's id, purpose
// kCellDraw keyed by the cell with the stage in the last word.
#include <algorithm>

#include "usp_device.cuh"

namespace usp {

namespace {

// Eq. 26 for one velocity C about the stage's mean: the weight that makes a
// Maxwellian particle represent (dt J / 2) / f_e, with sigma and q per unit
// density (sigma/p = (sigma/rho)/theta, q/(p theta) = (q/rho)/theta^2)
__device__ __forceinline__ double eq26_weight(const double* C, const double* F, double pne, double dt, double Pr) {
    const double theta = F[kWFTh];
    const double* sig = F + kWFSig;
    const double* q = F + kWFQ;
    const double quad = sig[0] * C[0] * C[0] + sig[1] * C[1] * C[1] + sig[2] * C[2] * C[2] +
                        2.0 * (sig[3] * C[0] * C[1] + sig[4] * C[0] * C[2] + sig[5] * C[1] * C[2]);
    const double c2 = C[0] * C[0] + C[1] * C[1] + C[2] * C[2];
    const double qc = q[0] * C[0] + q[1] * C[1] + q[2] * C[2];
    const double bracket = quad / (2.0 * theta * theta) + 0.4 * Pr * qc / (theta * theta) * (c2 / (2.0 * theta) - 2.5);
    return -0.5 * F[kWFNu] * pne * dt * bracket;
}

// P_ne of a cell as the weights see it: 0 (SP modes), the fixed value, or the
// Eq. 16 value of the last parameter evaluation
__device__ __forceinline__ double pne_of(const SimDev& s, int cell) {
    if (s.mode == kModeSP || s.mode == kModeSPESBGK) return 0.0;
    if (s.mode == kModeFixed) return s.fixed_pne;
    return s.prm[(size_t)13 * s.K + cell];
}

// BGK collision frequency nu = p / mu (Eq. 35) of a cell state
__device__ __forceinline__ double nu_of_state(const SimDev& s, double neff, double theta) {
    const double n = neff * s.w, T = theta / s.R;
    const double rho = n * s.mass, p = rho * theta;
    const double mu = s.mu_ref * pow(T / s.T_ref, s.omega);
    return p / mu;
}

// Eq. 34 average of a weight-field record, started at zero stress and heat
// flux and at the first u, theta, nu
__device__ __forceinline__ void average_record(const SimDev& s, double* a, const double* f, bool first) {
    for (int k = 0; k < kWFPref; ++k) {
        if (first) a[k] = (k >= kWFSig && k < kWFNu) ? 0.0 : f[k];
        else a[k] = s.avg_keep * a[k] + s.avg_new * f[k];
    }
}

// ---------------------------------------------------------------------------
// one stage of added particles: the record each cell's particles are drawn
// from and their count N_a (Eq. 25, rounded at random with the cell-keyed
// draw of the stage).  STAGE 1: step 2, from the moments of f^n (k_moments
// on the current buffer); 2: step 4, from u, theta, nu of the parameters and
// sigma*, q* of Eq. 33; 3: step 7, the step-4 record with the Eq. 27 factor.
// ---------------------------------------------------------------------------
template <int STAGE>
__global__ void __launch_bounds__(128) k_w_stage(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
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
        const uint32_t step = s.dyn->step;
        for (int cc = threadIdx.x; cc < kCTile; cc += blockDim.x) {
            const int cell = tile.y + cc;
            if (cell >= K) break;
            const double neff = s.wneff[cell];
            double rec[kNWF];
            for (int k = 0; k < kNWF; ++k) rec[k] = 0.0;
            bool live = false;   // the cell may receive particles at this stage
            double pne = 0.0, factor = 1.0;
            if (STAGE == 1) {
                Local L;
                double P[6], Q[3];
                local_state(s, cell, L, P, Q);
                if (neff > 1.0 && L.theta > 0.0 && L.N >= 1) {
                    for (int d = 0; d < 3; ++d) rec[kWFU + d] = L.u[d];
                    rec[kWFTh] = L.theta;
                    for (int d = 0; d < 3; ++d) rec[kWFSig + d] = P[d] - L.theta;
                    for (int d = 0; d < 3; ++d) rec[kWFSig + 3 + d] = P[3 + d];
                    for (int d = 0; d < 3; ++d) rec[kWFQ + d] = Q[d];
                    rec[kWFNu] = nu_of_state(s, neff, L.theta);
                }
                if (s.weight_average) {
                    double* a = s.wan + (size_t)kNWF * cell;
                    average_record(s, a, rec, !(s.dyn->w_started & 1u));
                    for (int k = 0; k < kWFPref; ++k) rec[k] = a[k];
                }
                pne = pne_of(s, cell);
                live = pne != 0.0 && neff > 1.0;
            } else if (STAGE == 2) {
                const bool valid = s.prm[(size_t)14 * K + cell] != 0.0;
                if (valid) {
                    for (int d = 0; d < 3; ++d) rec[kWFU + d] = s.prm[(size_t)d * K + cell];
                    rec[kWFTh] = s.prm[(size_t)3 * K + cell];
                    for (int d = 0; d < 6; ++d) rec[kWFSig + d] = s.wst[(size_t)d * K + cell];
                    for (int d = 0; d < 3; ++d) rec[kWFQ + d] = s.wst[(size_t)(6 + d) * K + cell];
                    rec[kWFNu] = s.prm[(size_t)11 * K + cell];
                }
                if (s.weight_average) {
                    double* a = s.was + (size_t)kNWF * cell;
                    average_record(s, a, rec, !(s.dyn->w_started & 2u));
                    for (int k = 0; k < kWFPref; ++k) rec[k] = a[k];
                }
                pne = pne_of(s, cell);
                live = valid && pne != 0.0;
            } else {
                const bool valid = s.prm[(size_t)14 * K + cell] != 0.0;
                for (int k = 0; k < kNWF; ++k) rec[k] = s.wfs[(size_t)kNWF * cell + k];
                pne = rec[kWFPne];
                live = valid && pne != 0.0;
                if (live) {
                    const double a = s.prm[(size_t)12 * K + cell] * s.dt;
                    factor = -2.0 * (-expm1(-a)) / a;
                }
            }
            // N_a of Eq. 25: N_eff min(1, nu_ES dt) / r_p, rounded at random;
            // each weight carries r_p / min(1, nu_ES dt)
            const double kap = fmin(1.0, s.Pr * rec[kWFNu] * s.dt);
            const double pref = kap > 0.0 ? s.r_p / kap : 0.0;
            uint32_t na = 0;
            if (live && neff > 0.0 && kap > 0.0) {
                const uint4 w = draw(s, (uint32_t)cell, step, kCellDraw, (uint32_t)STAGE);
                const double x = floor(neff * kap / s.r_p + u01<double>(w.x));
                na = x > 0.0 && rec[kWFTh] > 0.0 ? (uint32_t)x : 0u;
            }
            rec[kWFPref] = factor * pref;
            rec[kWFPne] = pne;
            if (STAGE == 2 || na) {
                for (int k = 0; k < kNWF; ++k) s.wfs[(size_t)kNWF * cell + k] = rec[k];
            }
            s.wna[cell] = na;
        }
    }
}

// exclusive scan of the per-cell counts of one stage (one block per
// simulation); the total goes to dyn->w_added
__global__ void __launch_bounds__(1024) k_w_scan(const SimDev* __restrict__ sims, int nsims) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    for (int si = blockIdx.x; si < nsims; si += gridDim.x) {
        const SimDev& s = sims[si];
        if (!s.weighted) continue;
        const int K = s.K;
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (int base = 0; base < K; base += blockDim.x) {
            const int c = base + threadIdx.x;
            const uint32_t v = c < K ? s.wna[c] : 0u;
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
            if (c < K) s.woff[c] = before + x - v;
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) carry = before + x;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            s.woff[K] = carry;
            s.dyn->w_added = carry;
        }
        __syncthreads();
    }
}

// the particles of one stage, appended to buffer `cur` after its n live
// entries in (cell, k) order; ids continue from next_pid in the same order.
// Positions uniform in the cell, velocities Maxwellian at the record's u and
// theta, weights pref * factor * Eq. 26.
__global__ void __launch_bounds__(256) k_w_add(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
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
        const int cur = s.dyn->cur;
        const uint32_t n0 = s.dyn->n, pid0 = s.dyn->next_pid, step = s.dyn->step;
        PView<double> P = view<double>(s, cur);
        double* W = s.wgt[cur];
        for (int cc = warp; cc < kCTile; cc += nwarps) {
            const int cell = tile.y + cc;
            if (cell >= s.K) break;
            const uint32_t na = s.wna[cell];
            if (!na) continue;
            const double* F = s.wfs + (size_t)kNWF * cell;
            const int ix = cell % s.nx, iy = cell / s.nx;
            const double xl = s.dim == 2 ? s.lo[0] + ix * s.dx : 0.0;
            const double yl = s.lo[1] + iy * s.dy;
            const double sq = sqrt(F[kWFTh]);
            for (uint32_t k = lane; k < na; k += 32) {
                const uint32_t off = s.woff[cell] + k;
                const int64_t i = (int64_t)n0 + off;
                if (i >= s.cap) {
                    atomicAdd(&s.dyn->counters[kCntOverflow], 1ull);
                    continue;
                }
                const uint32_t pid = pid0 + off;
                const uint4 w = draw(s, pid, step, kAdd, 0);
                const uint4 v = draw(s, pid, step, kAdd, 1);
                double z0, z1, z2, z3;
                box_muller<double>(v.x, v.y, z0, z1);
                box_muller<double>(v.z, v.w, z2, z3);
                const double C[3] = {sq * z0, sq * z1, sq * z2};
                if (s.dim == 2) P.x[i] = xl + u01<double>(w.x) * s.dx;
                P.y[i] = yl + u01<double>(w.y) * s.dy;
                P.c0[i] = F[kWFU] + C[0];
                P.c1[i] = F[kWFU + 1] + C[1];
                P.c2[i] = F[kWFU + 2] + C[2];
                P.pid[i] = pid;
                W[i] = F[kWFPref] * eq26_weight(C, F, F[kWFPne], s.dt, s.Pr);
            }
        }
    }
}

// after an add: the live count and the next id move on; `bits` marks the
// weight-field averages that now exist
__global__ void k_w_commit(const SimDev* __restrict__ sims, int nsims, uint32_t bits) {
    for (int si = blockIdx.x * blockDim.x + threadIdx.x; si < nsims; si += gridDim.x * blockDim.x) {
        const SimDev& s = sims[si];
        if (!s.weighted) continue;
        SimDyn* d = s.dyn;
        const int64_t n = (int64_t)d->n + d->w_added;
        d->n = (uint32_t)(n < s.cap ? n : s.cap);
        d->next_pid += d->w_added;
        d->w_added = 0;
        d->w_started |= bits;
    }
}

// cell and histogram of the n entries of buffer `cur` (a deleted particle,
// weight NaN, goes to the sentinel K and is dropped by the scatter)
__global__ void __launch_bounds__(256) k_w_assign(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
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
        PView<double> P = view<double>(s, cur);
        const double* W = s.wgt[cur];
        for (int j = threadIdx.x; j < kPTile; j += blockDim.x) {
            const int64_t i = (int64_t)tile.y + j;
            if (i >= (int64_t)n) break;
            uint32_t cell = (uint32_t)s.K;
            if (!isnan(W[i])) {
                cell = (uint32_t)min(max(cell_index<double>(s, s.dim == 2 ? P.x[i] : 0.0, P.y[i]), 0), s.K - 1);
                aggregated_add(s.count, cell);
            }
            s.cell[i] = cell;
        }
    }
}

// particles and weights of buffer cur to their sorted slots in cur ^ 1
__global__ void __launch_bounds__(256) k_w_scatter(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
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
        PView<double> A = view<double>(s, cur), B = view<double>(s, cur ^ 1);
        const double* WA = s.wgt[cur];
        double* WB = s.wgt[cur ^ 1];
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
            WB[slot] = WA[i];
        }
    }
}

// after a sort: the sorted buffer becomes current (swap = 1), or stays the
// other one (swap = 0); the live count is the sorted total; fill is cleared
__global__ void k_w_sorted(const SimDev* __restrict__ sims, int nsims, int swap) {
    for (int si = blockIdx.x; si < nsims; si += gridDim.x) {
        const SimDev& s = sims[si];
        if (!s.weighted) continue;
        for (int c = threadIdx.x; c <= s.K; c += blockDim.x) s.fill[c] = 0;
        if (threadIdx.x == 0) {
            SimDyn* d = s.dyn;
            const int64_t n = (int64_t)s.start[s.K];
            d->n = (uint32_t)(n < s.cap ? n : s.cap);
            if (swap) d->cur ^= 1;
        }
    }
}

// buffer cur ^ 1 holds the sorted state: make it current for an add (the
// add appends to `cur`), keeping its live count
__global__ void k_w_take_sorted(const SimDev* __restrict__ sims, int nsims) {
    for (int si = blockIdx.x * blockDim.x + threadIdx.x; si < nsims; si += gridDim.x * blockDim.x) {
        const SimDev& s = sims[si];
        if (!s.weighted) continue;
        SimDyn* d = s.dyn;
        d->cur ^= 1;
        const int64_t n = (int64_t)s.start[s.K];
        d->n = (uint32_t)(n < s.cap ? n : s.cap);
    }
}

// ---------------------------------------------------------------------------
// steps 5-6 on the sorted buffer cur ^ 1, one warp per cell
// ---------------------------------------------------------------------------
constexpr int kWKeys = 2048;   // selection words cached per cell (larger cells redraw them)

// the m-th smallest (1-based) selection word of the cell's slots [b, e): a
// radix select over 8-bit digits counted in `hist` (256 entries)
template <class KeyOf>
__device__ uint32_t w_kth_word(uint32_t b, uint32_t e, uint32_t m, const KeyOf& key_of, uint32_t* hist, int lane,
                               uint32_t& below_out) {
    uint32_t prefix = 0, mask = 0, rem = m;
    for (int shift = 24; shift >= 0; shift -= 8) {
        for (int k = lane; k < 256; k += 32) hist[k] = 0u;
        __syncwarp();
        for (uint32_t i = b + lane; i < e; i += 32) {
            const uint32_t x = key_of(i);
            if ((x & mask) == prefix) atomicAdd(&hist[(x >> shift) & 255u], 1u);
        }
        __syncwarp();
        uint32_t h[8], tot = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            h[k] = hist[8 * lane + k];
            tot += h[k];
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
            for (int k = 0; k < 8; ++k) {
                if (below + h[k] >= rem) {
                    d = 8u * lane + k;
                    break;
                }
                below += h[k];
            }
        }
        d = __shfl_sync(0xffffffffu, d, L);
        below = __shfl_sync(0xffffffffu, below, L);
        rem -= below;
        prefix |= d << shift;
        mask |= 0xFFu << shift;
        __syncwarp();
    }
    below_out = m - rem;   // words strictly below the result
    return prefix;
}

__global__ void __launch_bounds__(32) k_w_relax(const SimDev* __restrict__ sims, const int2* __restrict__ tiles,
                                                const int* __restrict__ ntiles) {
    __shared__ SimDev sim_sh;
    __shared__ uint32_t keys[kWKeys];
    __shared__ uint32_t hist[256];
    const int nt = *ntiles;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
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
        const int cell = tile.y + g % kCTile;
        if (cell >= K) continue;
        const uint32_t step = s.dyn->step;
        const int buf = s.dyn->cur ^ 1;
        PView<double> B = view<double>(s, buf);
        double* W = s.wgt[buf];
        const double* pr = s.prm;
        CellRelax R;
        for (int d = 0; d < 3; ++d) R.u[d] = pr[(size_t)d * K + cell];
        if (lane == 0 && s.mom[cell] >= 1.0)
            for (int d = 0; d < 3; ++d) s.ushift[(size_t)d * K + cell] = R.u[d];
        __syncwarp();
        const bool valid = pr[(size_t)14 * K + cell] != 0.0;
        if (!valid) {
            if (lane == 0) s.prm[(size_t)15 * K + cell] = 0.0;
            continue;
        }
        R.theta = pr[(size_t)3 * K + cell];
        for (int d = 0; d < 6; ++d) R.L[d] = pr[(size_t)(4 + d) * K + cell];
        R.p_relax = pr[(size_t)10 * K + cell];
        R.nu = pr[(size_t)11 * K + cell];
        R.nu_es = pr[(size_t)12 * K + cell];
        R.pne = pr[(size_t)13 * K + cell];
        const uint32_t cap = (uint32_t)s.cap;
        const uint32_t b = min(s.start[cell], cap), e = min(s.start[cell + 1], cap);
        const bool cached = e - b <= (uint32_t)kWKeys;
        auto key_of = [&](uint32_t i) -> uint32_t {
            return cached ? keys[i - b] : draw(s, B.pid[i], step, kRelax, 0).x;
        };
        // step 5: Bernoulli selection (Eq. 9); the selected set's weight and momentum
        double ns = 0, sw = 0, su[3] = {0, 0, 0};
        for (uint32_t i = b + lane; i < e; i += 32) {
            const uint32_t x = draw(s, B.pid[i], step, kRelax, 0).x;
            if (cached) keys[i - b] = x;
            if (!(u01<double>(x) < R.p_relax)) continue;
            const double w = W[i];
            ns += 1.0;
            sw += w;
            su[0] += w * B.c0[i];
            su[1] += w * B.c1[i];
            su[2] += w * B.c2[i];
        }
        __syncwarp();
        ns = warp_sum(ns);
        if (ns == 0.0) {
            if (lane == 0) s.prm[(size_t)15 * K + cell] = 0.0;
            continue;
        }
        sw = warp_sum(sw);
        for (int d = 0; d < 3; ++d) su[d] = warp_sum(su[d]);
        // Eq. 28: int(sum of the selected weights), rounded at random
        const uint4 wc = draw(s, (uint32_t)cell, step, kCellDraw, 0);
        double md = sw > 0.0 ? floor(sw + u01<double>(wc.x)) : 0.0;
        if (md > ns) md = ns;
        const uint32_t m = (uint32_t)md;
        double uo[3] = {0, 0, 0}, eo = 0;
        if (sw > 0.0) {
            for (int d = 0; d < 3; ++d) uo[d] = su[d] / sw;
            for (uint32_t i = b + lane; i < e; i += 32) {
                if (!(u01<double>(key_of(i)) < R.p_relax)) continue;
                const double a0 = B.c0[i] - uo[0], a1 = B.c1[i] - uo[1], a2 = B.c2[i] - uo[2];
                eo += W[i] * (a0 * a0 + a1 * a1 + a2 * a2);
            }
            eo = warp_sum(eo) / sw;
        }
        // step 6: the m selected particles with the smallest words (the
        // selected words lie below all the others) are reassigned at weight 1
        // from f_G(t); ties at the m-th word go to the lower slot.  The other
        // selected particles are deleted (weight NaN).
        uint32_t T = 0, quota = 0;
        if (m > 0) {
            uint32_t below = 0;
            T = w_kth_word(b, e, m, key_of, hist, lane, below);
            quota = m - below;
        }
        double un[3] = {0, 0, 0};
        uint32_t ties = 0;
        for (uint32_t i0 = b; i0 < e; i0 += 32) {
            const uint32_t i = i0 + lane;
            const bool has = i < e;
            const uint32_t x = has ? key_of(i) : 0xFFFFFFFFu;
            const bool sel = has && u01<double>(x) < R.p_relax;
            const bool tie = sel && m > 0 && x == T;
            const unsigned tb = __ballot_sync(0xffffffffu, tie);
            const uint32_t trank = ties + (uint32_t)__popc(tb & lt);
            ties += (uint32_t)__popc(tb);
            if (!sel) continue;
            const bool keep = m > 0 && (x < T || (tie && trank < quota));
            if (!keep) {
                W[i] = __longlong_as_double(0x7FF8000000000000ll);   // deleted
                continue;
            }
            const uint32_t pid = B.pid[i];
            const uint4 w = draw(s, pid, step, kRelax, 0);
            double C[3];
            es_draw<double>(s, R, pid, step, w, C);
            B.c0[i] = R.u[0] + C[0];
            B.c1[i] = R.u[1] + C[1];
            B.c2[i] = R.u[2] + C[2];
            W[i] = 1.0;
            un[0] += B.c0[i];
            un[1] += B.c1[i];
            un[2] += B.c2[i];
        }
        __syncwarp();
        for (int d = 0; d < 3; ++d) un[d] = warp_sum(un[d]);
        // the reassigned set carries the selected set's mean velocity and
        // thermal energy per unit weight
        auto reassigned = [&](uint32_t i) { return W[i] == 1.0 && u01<double>(key_of(i)) < R.p_relax; };
        if (m >= 2 && sw > 0.0) {
            for (int d = 0; d < 3; ++d) un[d] /= md;
            double en = 0;
            for (uint32_t i = b + lane; i < e; i += 32) {
                if (!reassigned(i)) continue;
                const double a0 = B.c0[i] - un[0], a1 = B.c1[i] - un[1], a2 = B.c2[i] - un[2];
                en += a0 * a0 + a1 * a1 + a2 * a2;
            }
            en = warp_sum(en) / md;
            const double alpha = (en > 0.0 && eo > 0.0) ? sqrt(eo / en) : 1.0;
            for (uint32_t i = b + lane; i < e; i += 32) {
                if (!reassigned(i)) continue;
                B.c0[i] = uo[0] + alpha * (B.c0[i] - un[0]);
                B.c1[i] = uo[1] + alpha * (B.c1[i] - un[1]);
                B.c2[i] = uo[2] + alpha * (B.c2[i] - un[2]);
            }
        } else if (m == 1 && sw > 0.0) {
            const double f = sqrt(eo > 0.0 ? eo / (3.0 * R.theta) : 1.0);
            for (uint32_t i = b + lane; i < e; i += 32) {
                if (!reassigned(i)) continue;
                B.c0[i] = uo[0] + (B.c0[i] - un[0]) * f;
                B.c1[i] = uo[1] + (B.c1[i] - un[1]) * f;
                B.c2[i] = uo[2] + (B.c2[i] - un[2]) * f;
            }
        }
        __syncwarp();
        if (lane == 0) {
            s.prm[(size_t)15 * K + cell] = md;
            if (m > 0) atomicAdd(&s.dyn->counters[kCntRelaxed], (unsigned long long)m);
        }
    }
}

// initial weights 1 of the n live particles of buffer cur; the averages of
// the weight fields start afresh
__global__ void k_w_init(const SimDev* __restrict__ sims, int nsims) {
    for (int si = blockIdx.y; si < nsims; si += gridDim.y) {
        const SimDev& s = sims[si];
        if (!s.weighted) continue;
        const int cur = s.dyn->cur;
        const uint32_t n = s.dyn->n;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)n;
             i += (int64_t)gridDim.x * blockDim.x)
            s.wgt[cur][i] = 1.0;
        if (blockIdx.x == 0 && threadIdx.x == 0) s.dyn->w_started = 0;
    }
}

}  // namespace

// the counting sort of the weighted path: buffer cur -> cur ^ 1 by cell;
// swap makes the sorted buffer current
static void w_sort(const Launch& L, int swap) {
    k_w_assign<<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
    launch_scan(L, false);
    k_w_scatter<<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
    k_w_sorted<<<L.nsims, 256, 0, L.stream>>>(L.sims, L.nsims, swap);
}

// one stage of added particles appended to buffer cur
template <int STAGE>
static void w_add(const Launch& L, uint32_t bits) {
    k_w_stage<STAGE><<<L.grid_c, 32, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    k_w_scan<<<L.nsims, 1024, 0, L.stream>>>(L.sims, L.nsims);
    k_w_add<<<L.grid_c, 256, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    k_w_commit<<<1, 32, 0, L.stream>>>(L.sims, L.nsims, bits);
}

void enqueue_weighted_step(const Launch& L) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the state in cell order, then the W-weighted moments of f^n
    w_sort(L, 1);
    launch_moments_src(L, true, true);
    // Table 2 step 2
    w_add<1>(L, 1u);
    // step 3: flight and counting sort into cur ^ 1 (the weights follow)
    launch_stream(L, true);
    launch_scan(L, false);
    k_w_scatter<<<L.grid_p, 256, 0, L.stream>>>(L.sims, L.ptiles, L.nptiles);
    k_w_sorted<<<L.nsims, 256, 0, L.stream>>>(L.sims, L.nsims, 0);
    // moments and parameters of f~* (Eqs. 1, 16-18, 33)
    launch_moments(L, true);
    launch_params(L);
    // step 4, then the new particles into their cells (sorted into cur ^ 1)
    k_w_take_sorted<<<1, 32, 0, L.stream>>>(L.sims, L.nsims);
    w_add<2>(L, 2u);
    w_sort(L, 0);
    // steps 5-6
    const int grid = std::max(1, std::min(L.grid_c * kCTile, 32 * sms));
    k_w_relax<<<grid, 32, 0, L.stream>>>(L.sims, L.ctiles, L.nctiles);
    // step 7 appended to the relaxed buffer; compaction and sort end the step
    k_w_take_sorted<<<1, 32, 0, L.stream>>>(L.sims, L.nsims);
    w_add<3>(L, 0u);
    w_sort(L, 0);
    launch_finish(L);
}

void launch_weighted_init(const Launch& L) {
    k_w_init<<<dim3(256, L.nsims), 256, 0, L.stream>>>(L.sims, L.nsims);
}

}  // namespace usp
