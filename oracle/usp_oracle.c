/*
 * usp_oracle.c -- plain, slow, FP64 CPU oracle of the USP-ESBGK time step.
 *
 * TEST INFRASTRUCTURE: loaded only by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py.  It shares nothing with the CUDA library.
 *
 * One time step n -> n+1 (Table 2 of the paper, weighted-particle steps 2, 4
 * and 7 left out; all weights equal 1):
 *   1. advect every particle for dt and apply the wall / reservoir boundary
 *      conditions "similar to DSMC" (Table 1 steps 1-2, Table 2 step 3);
 *   2. refill reservoir buffer cells (slit inflow / outflow);
 *   3. cell index of every particle and a sort by (cell, pid);
 *   4. per-cell moments, Eq. 1, in two passes (mean, then central sums);
 *   5. per-cell USP parameters: viscosity Eq. 35, relaxation frequencies
 *      (nu = p/mu, nu_ES = Pr nu, Sec. 2), mean free path Eq. 36, gradient-
 *      length local Knudsen number Eqs. 17-18, P_ne Eq. 16, corrected stress
 *      and heat flux Eq. 33, ES covariance Eq. 6c;
 *   6. relaxation: each particle relaxes with probability 1 - exp(-nu_ES dt)
 *      (Eqs. 8b, 9); a relaxed particle draws a time instant from g_time
 *      (Eqs. 29-30), takes sigma(t) from Eq. 32 and a velocity from the ES
 *      Gaussian f_G(t) (Eq. 6b); then the relaxed subset of each cell is
 *      shifted and scaled so that its momentum and energy are unchanged;
 *   7. instantaneous fields and the exponential average of Eq. 34.
 *
 * Random numbers: Philox4x32-10 with key = seed and counter =
 * (pid, step, purpose, k); purpose 0 = initialisation, 1 = relaxation,
 * 2 = wall re-emission (k = bounce index), 3 = reservoir injection.
 */
#include "usp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define KB 1.380649e-23           /* Boltzmann constant, J/K (exact SI value) */
#define GAMMA_MONO (5.0 / 3.0)    /* ratio of specific heats, monatomic gas */
#define KN_C 0.1                  /* reference Knudsen number of Eq. 16 */
#define MAX_BOUNCE 8              /* wall interactions per particle per step */
#define PI 3.14159265358979323846

enum { P_INIT = 0, P_RELAX = 1, P_WALL = 2, P_INJECT = 3, P_ADD = 4, P_CELL = 5 };

/* fields that define the weights of added particles (Eq. 26), per cell:
 * u[3], theta, sigma/rho (xx yy zz xy xz yz), q/rho, nu */
enum { WF_U = 0, WF_TH = 3, WF_SIG = 4, WF_Q = 10, WF_NU = 13, WF_N = 14 };

typedef struct {
    double x, y, c[3];
    double w;              /* particle weight (1 unless created by Table 2 steps 2, 4, 7) */
    uint32_t pid;
    int cell;
    int alive;
} particle;

typedef struct {
    int n;                 /* particles in the cell */
    double neff;           /* sum of their weights (= n when every weight is 1) */
    double u[3];           /* mean velocity */
    double theta;          /* R T = sum |C|^2 / (3 N) */
    double P[6];           /* sum C_i C_j / N: xx, yy, zz, xy, xz, yz */
    double Q[3];           /* sum C^2 C_i / (2 N) */
} cell_moments;

typedef struct {
    int valid;
    double n, T, umag, a_sound, lambda;
    double mu, nu, nu_es, p;
    double pne;
    double sig_star[6];    /* sigma* / rho (Eq. 33) */
    double q_star[3];      /* q* / rho (Eq. 33) */
    double L[6];           /* Cholesky factor of theta I + (1 - 1/Pr) sigma* / rho: 00,10,11,20,21,22 */
    double p_relax;
    int n_relaxed;
} cell_params;

/* the state a cell contributes to the Kn_GLL stencil (Eqs. 17-18) */
typedef struct {
    int valid;
    double n, T, umag, a_sound, lambda;
} grad_state;

struct orc_sim {
    orc_config cfg;
    double R, dt, mu_ref, w;     /* gas constant, time step, reference viscosity, density per particle */
    double dx, dy;
    int K;
    particle* p;
    int64_t np, cap;
    uint32_t key[2];
    uint32_t next_pid;
    uint32_t step;
    int nsamples;
    cell_moments* mom;
    cell_params* par;
    grad_state* gs;
    double* inst;                /* ORC_NFIELDS x K */
    double* avg;
    int64_t counters[5];
    /* weighted particles: fields of f^n (step 2) and f* (steps 4, 7), and
     * their Eq. 34 averages, WF_N per cell */
    double* wf_n;
    double* wf_s;
    double* wa_n;
    double* wa_s;
    int wa_started;
};

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, as defined by Salmon, Moraes, Dror and Shaw, "Parallel      */
/* random numbers: as easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64    */
/* multiplications with the round keys bumped by the Weyl constants.          */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0; k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform on the open interval (0, 1) */
double orc_u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

static void draw(const orc_sim* s, uint32_t pid, uint32_t step, uint32_t purpose, uint32_t k, uint32_t out[4]) {
    uint32_t ctr[4] = {pid, step, purpose, k};
    orc_philox4x32_10(ctr, s->key, out);
}

/* Box-Muller: two standard normals from two uniform words (Eq. 10 in standard form) */
static void box_muller(uint32_t wa, uint32_t wb, double* z0, double* z1) {
    double ua = orc_u01(wa), ub = orc_u01(wb);
    double r = sqrt(-2.0 * log(ua));
    *z0 = r * cos(2.0 * PI * ub);
    *z1 = r * sin(2.0 * PI * ub);
}

/* ------------------------------------------------------------------------ */
/* set-up: reference viscosity from Kn (Eq. 36), dt from tau_c (Eq. 37)       */
/* ------------------------------------------------------------------------ */
orc_sim* orc_create(const orc_config* cfg) {
    if (!cfg) return NULL;
    if (cfg->dim != 1 && cfg->dim != 2) return NULL;
    if (cfg->ny < 1 || (cfg->dim == 2 && cfg->nx < 1)) return NULL;
    if (cfg->mass <= 0 || cfg->T_ref <= 0 || cfg->Pr <= 0 || cfg->n_ref <= 0 || cfg->ppc_ref < 1) return NULL;
    /* a body force may act only along directions that are not resolved */
    if (cfg->body_accel[1] != 0 || (cfg->dim == 2 && cfg->body_accel[0] != 0)) return NULL;
    /* the counting plane lies strictly inside the domain, across an axis
     * whose faces are not periodic */
    if (cfg->mode < ORC_MODE_USP || cfg->mode > ORC_MODE_SPESBGK) return NULL;
    if (cfg->selection < 0 || cfg->selection > 1 || cfg->es_sampler < 0 || cfg->es_sampler > 1) return NULL;
    if (cfg->flux_axis < 0 || cfg->flux_axis > 2) return NULL;
    if (cfg->flux_axis) {
        int a = cfg->flux_axis - 1;
        if (a == 0 && cfg->dim != 2) return NULL;
        if (cfg->face_kind[2 * a] == ORC_BC_PERIODIC) return NULL;
        if (!(cfg->flux_pos > cfg->lo[a] && cfg->flux_pos < cfg->hi[a])) return NULL;
    }
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->cfg = *cfg;
    if (cfg->dim == 1) s->cfg.nx = 1;
    s->R = KB / cfg->mass;
    double rho_ref = cfg->n_ref * cfg->mass;
    double p_ref = cfg->n_ref * KB * cfg->T_ref;
    double mu_ref = cfg->mu_ref;
    if (mu_ref <= 0) {
        /* Eq. 36 solved for mu at the reference state, with lambda = Kn L_ref */
        double lam = cfg->Kn * cfg->L_ref;
        mu_ref = lam * 5.0 * sqrt(2.0 * PI) / 16.0 * sqrt(rho_ref * p_ref);
    }
    s->mu_ref = mu_ref;
    double lam_ref = 16.0 / (5.0 * sqrt(2.0 * PI)) * mu_ref / sqrt(rho_ref * p_ref);
    double tau_c = lam_ref / sqrt(8.0 * KB * cfg->T_ref / (PI * cfg->mass));
    s->dt = cfg->dt > 0 ? cfg->dt : cfg->dt_over_tauc * tau_c;
    s->w = cfg->n_ref / (double)cfg->ppc_ref;
    s->dy = (cfg->hi[1] - cfg->lo[1]) / cfg->ny;
    s->dx = cfg->dim == 2 ? (cfg->hi[0] - cfg->lo[0]) / cfg->nx : 1.0;
    s->K = s->cfg.nx * cfg->ny;
    s->mom = (cell_moments*)calloc(s->K, sizeof(cell_moments));
    s->par = (cell_params*)calloc(s->K, sizeof(cell_params));
    s->gs = (grad_state*)calloc((size_t)s->K, sizeof(grad_state));
    s->inst = (double*)calloc((size_t)ORC_NFIELDS * s->K, sizeof(double));
    s->avg = (double*)calloc((size_t)ORC_NFIELDS * s->K, sizeof(double));
    if (s->cfg.r_p <= 0) s->cfg.r_p = 10.0;
    if (s->cfg.weighted) {
        s->wf_n = (double*)calloc((size_t)WF_N * s->K, sizeof(double));
        s->wf_s = (double*)calloc((size_t)WF_N * s->K, sizeof(double));
        s->wa_n = (double*)calloc((size_t)WF_N * s->K, sizeof(double));
        s->wa_s = (double*)calloc((size_t)WF_N * s->K, sizeof(double));
    }
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    free(s->p); free(s->mom); free(s->par); free(s->gs); free(s->inst); free(s->avg);
    free(s->wf_n); free(s->wf_s); free(s->wa_n); free(s->wa_s);
    free(s);
}

static void reserve(orc_sim* s, int64_t n) {
    if (n <= s->cap) return;
    int64_t c = s->cap ? s->cap : 1024;
    while (c < n) c *= 2;
    s->p = (particle*)realloc(s->p, (size_t)c * sizeof(particle));
    s->cap = c;
}

static void set_key(orc_sim* s, uint64_t seed) {
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
}

static int cell_of(const orc_sim* s, double x, double y) {
    const orc_config* c = &s->cfg;
    int iy = (int)floor((y - c->lo[1]) / s->dy);
    if (iy < 0) iy = 0;
    if (iy > c->ny - 1) iy = c->ny - 1;
    if (c->dim == 1) return iy;
    int ix = (int)floor((x - c->lo[0]) / s->dx);
    if (ix < 0) ix = 0;
    if (ix > c->nx - 1) ix = c->nx - 1;
    return iy * c->nx + ix;
}

static void cell_lo(const orc_sim* s, int cell, double* xl, double* yl) {
    const orc_config* c = &s->cfg;
    int ix = cell % c->nx, iy = cell / c->nx;
    *xl = c->dim == 2 ? c->lo[0] + ix * s->dx : 0.0;
    *yl = c->lo[1] + iy * s->dy;
}

/* Particles created inside one cell: uniform position, Maxwellian velocity. */
static void fill_cell(orc_sim* s, int cell, int count, double T, const double* u, uint32_t purpose) {
    double xl, yl;
    cell_lo(s, cell, &xl, &yl);
    double sq = sqrt(s->R * T);
    reserve(s, s->np + count);
    for (int k = 0; k < count; ++k) {
        particle* q = &s->p[s->np++];
        uint32_t pid = s->next_pid++;
        uint32_t w[4], v[4];
        draw(s, pid, s->step, purpose, 0, w);
        draw(s, pid, s->step, purpose, 1, v);
        q->x = s->cfg.dim == 2 ? xl + orc_u01(w[0]) * s->dx : 0.0;
        q->y = yl + orc_u01(w[1]) * s->dy;
        double z0, z1, z2, z3;
        box_muller(v[0], v[1], &z0, &z1);
        box_muller(v[2], v[3], &z2, &z3);
        q->c[0] = u[0] + sq * z0;
        q->c[1] = u[1] + sq * z1;
        q->c[2] = u[2] + sq * z2;
        q->pid = pid;
        q->cell = cell;
        q->alive = 1;
        q->w = 1.0;
    }
}

static int count_for_density(const orc_sim* s, double n) {
    return (int)floor(n / s->cfg.n_ref * s->cfg.ppc_ref + 0.5);
}

/* Table 2 step 1: particles per cell from the region containing the cell centre
 * (the last listed region wins), pids assigned in cell order. */
int orc_init_particles(orc_sim* s, const orc_region* regs, int nreg, uint64_t seed) {
    if (!s || (nreg > 0 && !regs)) return -1;
    set_key(s, seed);
    s->np = 0; s->next_pid = 0; s->step = 0; s->nsamples = 0;
    memset(s->counters, 0, sizeof(s->counters));
    for (int cell = 0; cell < s->K; ++cell) {
        double xl, yl;
        cell_lo(s, cell, &xl, &yl);
        double xc = xl + 0.5 * s->dx, yc = yl + 0.5 * s->dy;
        int r = -1;
        for (int i = 0; i < nreg; ++i) {
            int in_y = yc >= regs[i].lo[1] && yc < regs[i].hi[1];
            int in_x = s->cfg.dim == 1 || (xc >= regs[i].lo[0] && xc < regs[i].hi[0]);
            if (in_x && in_y) r = i;
        }
        if (r < 0) continue;
        fill_cell(s, cell, count_for_density(s, regs[r].n), regs[r].T, regs[r].u, P_INIT);
    }
    return 0;
}

int orc_set_particles(orc_sim* s, int64_t n, const double* pos, const double* vel,
                      const uint32_t* pid, uint32_t next_pid, uint64_t seed) {
    if (!s || n < 0) return -1;
    set_key(s, seed);
    reserve(s, n);
    s->np = n; s->next_pid = next_pid; s->step = 0; s->nsamples = 0;
    memset(s->counters, 0, sizeof(s->counters));
    for (int64_t i = 0; i < n; ++i) {
        particle* q = &s->p[i];
        q->x = s->cfg.dim == 2 ? pos[2 * i] : 0.0;
        q->y = pos[2 * i + 1];
        for (int d = 0; d < 3; ++d) q->c[d] = vel[3 * i + d];
        q->pid = pid[i];
        q->cell = cell_of(s, q->x, q->y);
        q->alive = 1;
        q->w = 1.0;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 1. advection with boundary conditions                                     */
/* ------------------------------------------------------------------------ */
/* Earliest surface the particle reaches within time tau, skipping the surface
 * it left last.  Surfaces 0..3 are the faces, 4.. the plates.  Ties go to the
 * lower index.  Returns -1 when nothing is hit. */
static int next_hit(const orc_sim* s, const particle* q, double tau, int last, double* t_hit) {
    const orc_config* c = &s->cfg;
    int best = -1;
    double tb = 0;
    for (int f = 0; f < 4; ++f) {
        if (f == last) continue;
        int axis = f / 2;
        if (c->dim == 1 && axis == 0) continue;
        if (c->face_kind[f] == ORC_BC_PERIODIC) continue;
        double pos = axis == 0 ? q->x : q->y;
        double vel = q->c[axis];
        double t;
        if (f % 2 == 0) {
            if (!(vel < 0)) continue;
            t = (c->lo[axis] - pos) / vel;
        } else {
            if (!(vel > 0)) continue;
            t = (c->hi[axis] - pos) / vel;
        }
        if (t < 0) t = 0;
        if (t <= tau && (best < 0 || t < tb)) { best = f; tb = t; }
    }
    if (c->dim == 2) {
        for (int g = 0; g < c->nseg; ++g) {
            if (4 + g == last) continue;
            double vel = q->c[0];
            if (vel == 0) continue;
            double t = (c->seg_pos[g] - q->x) / vel;
            if (!(t > 0) || t > tau) continue;
            double yh = q->y + q->c[1] * t;
            if (yh < c->seg_lo[g] || yh > c->seg_hi[g]) continue;
            if (best < 0 || t < tb) { best = 4 + g; tb = t; }
        }
    }
    *t_hit = tb;
    return best;
}

/* Full accommodation at temperature T with wall velocity u; normal axis `axis`,
 * re-emitted towards sign `dir`: flux-weighted Rayleigh normal speed,
 * Gaussian tangential components. */
static void diffuse(const orc_sim* s, particle* q, int axis, double dir, double T, const double* u, uint32_t k) {
    uint32_t w[4];
    draw(s, q->pid, s->step, P_WALL, k, w);
    double th = s->R * T;
    double cn = sqrt(-2.0 * th * log(orc_u01(w[0])));
    double z0, z1;
    box_muller(w[1], w[2], &z0, &z1);
    double st = sqrt(th);
    if (axis == 1) {
        q->c[1] = dir * cn;
        q->c[0] = u[0] + st * z0;
        q->c[2] = u[2] + st * z1;
    } else {
        q->c[0] = dir * cn;
        q->c[1] = u[1] + st * z0;
        q->c[2] = u[2] + st * z1;
    }
}

static void fly(const orc_sim* s, particle* q, double t) {
    if (s->cfg.dim == 2) q->x += q->c[0] * t;
    q->y += q->c[1] * t;
    for (int d = 0; d < 3; ++d) q->c[d] += s->cfg.body_accel[d] * t;
}

static double wrap(double v, double lo, double hi) {
    double L = hi - lo;
    double r = fmod(v - lo, L);
    if (r < 0) r += L;
    return lo + r;
}

static void stream_one(orc_sim* s, particle* q) {
    const orc_config* c = &s->cfg;
    double tau = s->dt;
    int last = -1;
    int k = 0;
    for (;;) {
        double th;
        int hit = next_hit(s, q, tau, last, &th);
        if (hit < 0) { fly(s, q, tau); break; }
        if (k == MAX_BOUNCE) {
            /* bounce cap: fly the rest and clamp inside the domain */
            fly(s, q, tau);
            if (c->dim == 2 && c->face_kind[0] != ORC_BC_PERIODIC) q->x = fmin(fmax(q->x, c->lo[0]), c->hi[0]);
            if (c->face_kind[2] != ORC_BC_PERIODIC) q->y = fmin(fmax(q->y, c->lo[1]), c->hi[1]);
            s->counters[1]++;
            break;
        }
        fly(s, q, th);
        tau -= th;
        last = hit;
        if (hit < 4) {
            int axis = hit / 2;
            double wall = hit % 2 == 0 ? c->lo[axis] : c->hi[axis];
            if (axis == 0) q->x = wall; else q->y = wall;
            double dir = hit % 2 == 0 ? 1.0 : -1.0;
            int kind = c->face_kind[hit];
            if (kind == ORC_BC_SPECULAR) {
                q->c[axis] = -q->c[axis];
            } else if (kind == ORC_BC_DIFFUSE) {
                diffuse(s, q, axis, dir, c->face_T[hit], c->face_u[hit], (uint32_t)k);
            } else { /* reservoir: the particle leaves the domain */
                q->alive = 0;
                s->counters[2]++;
                return;
            }
        } else {
            int g = hit - 4;
            double dir = q->c[0] > 0 ? -1.0 : 1.0;
            q->x = c->seg_pos[g];
            if (c->seg_kind[g] == ORC_BC_SPECULAR) q->c[0] = -q->c[0];
            else diffuse(s, q, 0, dir, c->seg_T[g], c->seg_u[g], (uint32_t)k);
        }
        ++k;
    }
    if (c->dim == 2 && c->face_kind[0] == ORC_BC_PERIODIC) q->x = wrap(q->x, c->lo[0], c->hi[0]);
    if (c->face_kind[2] == ORC_BC_PERIODIC) q->y = wrap(q->y, c->lo[1], c->hi[1]);
}

/* 1 when the particle is at or above the counting plane, 0 below it */
static int flux_side(const orc_config* c, const particle* q) {
    double v = c->flux_axis == 1 ? q->x : q->y;
    return v >= c->flux_pos;
}

/* advection of every particle; the net flow through the counting plane is
 * the change of side summed over the particles (a particle that leaves
 * through a reservoir face ends on that face) */
static void weighted_step2(orc_sim* s);

static void stream_phase(orc_sim* s) {
    if (s->cfg.weighted) weighted_step2(s);   /* Table 2 step 2 precedes the advection */
    for (int64_t i = 0; i < s->np; ++i) {
        particle* q = &s->p[i];
        int before = s->cfg.flux_axis ? flux_side(&s->cfg, q) : 0;
        stream_one(s, q);
        if (s->cfg.flux_axis) s->counters[4] += flux_side(&s->cfg, q) - before;
    }
}

/* ------------------------------------------------------------------------ */
/* 2. reservoir buffer cells: remove what is in them, refill from the         */
/*    reservoir Maxwellian with new pids in (face, cell, k) order             */
/* ------------------------------------------------------------------------ */
static int in_buffer(const orc_sim* s, int cell, int* face_out) {
    const orc_config* c = &s->cfg;
    int ix = cell % c->nx, iy = cell / c->nx;
    int nb = c->reservoir_cols;
    for (int f = 0; f < 4; ++f) {
        if (c->face_kind[f] != ORC_BC_RESERVOIR) continue;
        int axis = f / 2;
        if (c->dim == 1 && axis == 0) continue;
        int i = axis == 0 ? ix : iy;
        int n = axis == 0 ? c->nx : c->ny;
        if ((f % 2 == 0 && i < nb) || (f % 2 == 1 && i >= n - nb)) { *face_out = f; return 1; }
    }
    return 0;
}

static void reservoir_phase(orc_sim* s) {
    const orc_config* c = &s->cfg;
    int any = 0;
    for (int f = 0; f < 4; ++f) any |= c->face_kind[f] == ORC_BC_RESERVOIR;
    /* drop particles that left the domain */
    int64_t m = 0;
    for (int64_t i = 0; i < s->np; ++i) {
        particle* q = &s->p[i];
        if (!q->alive) continue;
        int f;
        if (any && c->reservoir_cols > 0 && in_buffer(s, cell_of(s, q->x, q->y), &f)) { s->counters[2]++; continue; }
        s->p[m++] = *q;
    }
    s->np = m;
    if (!any || c->reservoir_cols <= 0) return;
    for (int f = 0; f < 4; ++f) {
        if (c->face_kind[f] != ORC_BC_RESERVOIR) continue;
        for (int cell = 0; cell < s->K; ++cell) {
            int ff;
            if (!in_buffer(s, cell, &ff) || ff != f) continue;
            int cnt = count_for_density(s, c->face_n[f]);
            fill_cell(s, cell, cnt, c->face_T[f], c->face_u[f], P_INJECT);
            s->counters[3] += cnt;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 3. cell index and sort by (cell, pid)                                     */
/* ------------------------------------------------------------------------ */
static int cmp_cell_pid(const void* a, const void* b) {
    const particle* p = (const particle*)a;
    const particle* q = (const particle*)b;
    if (p->cell != q->cell) return p->cell < q->cell ? -1 : 1;
    if (p->pid != q->pid) return p->pid < q->pid ? -1 : 1;
    return 0;
}

static void sort_phase(orc_sim* s) {
    for (int64_t i = 0; i < s->np; ++i) s->p[i].cell = cell_of(s, s->p[i].x, s->p[i].y);
    qsort(s->p, (size_t)s->np, sizeof(particle), cmp_cell_pid);
}

/* ------------------------------------------------------------------------ */
/* 4. moments (Eq. 1), two passes per cell                                   */
/* ------------------------------------------------------------------------ */
static void moments_phase(orc_sim* s) {
    memset(s->mom, 0, (size_t)s->K * sizeof(cell_moments));
    int64_t i = 0;
    while (i < s->np) {
        int cell = s->p[i].cell;
        int64_t j = i;
        while (j < s->np && s->p[j].cell == cell) ++j;
        cell_moments* M = &s->mom[cell];
        int n = (int)(j - i);
        M->n = n;
        /* weighted sums over the particles of the cell (every weight is 1
         * unless the weighted particles of Table 2 are in use) */
        double we = 0;
        for (int64_t k = i; k < j; ++k) we += s->p[k].w;
        M->neff = we;
        if (!(we > 0)) { i = j; continue; }
        for (int d = 0; d < 3; ++d) {
            double sum = 0;
            for (int64_t k = i; k < j; ++k) sum += s->p[k].w * s->p[k].c[d];
            M->u[d] = sum / we;
        }
        double e = 0, P[6] = {0}, Q[3] = {0};
        for (int64_t k = i; k < j; ++k) {
            double wk = s->p[k].w;
            double C0 = s->p[k].c[0] - M->u[0];
            double C1 = s->p[k].c[1] - M->u[1];
            double C2 = s->p[k].c[2] - M->u[2];
            double c2 = C0 * C0 + C1 * C1 + C2 * C2;
            e += wk * c2;
            P[0] += wk * C0 * C0; P[1] += wk * C1 * C1; P[2] += wk * C2 * C2;
            P[3] += wk * C0 * C1; P[4] += wk * C0 * C2; P[5] += wk * C1 * C2;
            Q[0] += wk * c2 * C0; Q[1] += wk * c2 * C1; Q[2] += wk * c2 * C2;
        }
        M->theta = e / (3.0 * we);
        for (int d = 0; d < 6; ++d) M->P[d] = P[d] / we;
        for (int d = 0; d < 3; ++d) M->Q[d] = Q[d] / (2.0 * we);
        i = j;
    }
}

/* ------------------------------------------------------------------------ */
/* 5. per-cell USP parameters                                                */
/* ------------------------------------------------------------------------ */
static int neighbor(const orc_sim* s, int cell, int axis, int dir) {
    const orc_config* c = &s->cfg;
    int ix = cell % c->nx, iy = cell / c->nx;
    if (axis == 0) {
        int j = ix + dir;
        if (j < 0 || j >= c->nx) {
            if (c->face_kind[j < 0 ? 0 : 1] != ORC_BC_PERIODIC) return -1;
            j = (j + c->nx) % c->nx;
        }
        return iy * c->nx + j;
    }
    int j = iy + dir;
    if (j < 0 || j >= c->ny) {
        if (c->face_kind[j < 0 ? 2 : 3] != ORC_BC_PERIODIC) return -1;
        j = (j + c->ny) % c->ny;
    }
    return j * c->nx + ix;
}

/* derivative of one cell field along one axis: central difference between the
 * two neighbours, one-sided next to a missing (absent or invalid) neighbour */
static double deriv(const orc_sim* s, int cell, int axis, int which) {
    double h = axis == 0 ? s->dx : s->dy;
    int m = neighbor(s, cell, axis, -1), p = neighbor(s, cell, axis, +1);
    if (m >= 0 && !s->gs[m].valid) m = -1;
    if (p >= 0 && !s->gs[p].valid) p = -1;
    const grad_state* P = s->gs;
    double qc, qm = 0, qp = 0;
#define FIELD(i) (which == 0 ? P[i].n : which == 1 ? P[i].T : P[i].umag)
    qc = FIELD(cell);
    if (m >= 0) qm = FIELD(m);
    if (p >= 0) qp = FIELD(p);
#undef FIELD
    if (m >= 0 && p >= 0) return (qp - qm) / (2.0 * h);
    if (p >= 0) return (qp - qc) / h;
    if (m >= 0) return (qc - qm) / h;
    return 0.0;
}

static void params_phase(orc_sim* s) {
    const orc_config* c = &s->cfg;
    /* pass 1: local state of every cell */
    for (int cell = 0; cell < s->K; ++cell) {
        cell_moments* M = &s->mom[cell];
        cell_params* P = &s->par[cell];
        memset(P, 0, sizeof(*P));
        P->valid = M->n >= 2 && M->neff > 1.0 && M->theta > 0;
        if (!P->valid) continue;
        P->n = M->neff * s->w;
        P->T = M->theta / s->R;
        P->umag = sqrt(M->u[0] * M->u[0] + M->u[1] * M->u[1] + M->u[2] * M->u[2]);
        P->a_sound = sqrt(GAMMA_MONO * M->theta);
        double rho = P->n * c->mass;
        P->p = rho * M->theta;
        P->mu = s->mu_ref * pow(P->T / c->T_ref, c->omega);          /* Eq. 35 */
        P->nu = P->p / P->mu;                                        /* BGK frequency, Sec. 2 */
        P->nu_es = c->Pr * P->nu;                                    /* ESBGK frequency, Eq. 6a */
        P->lambda = 16.0 / (5.0 * sqrt(2.0 * PI)) * P->mu / sqrt(rho * P->p);   /* Eq. 36 */
    }
    /* states seen by the Kn_GLL stencil: the instantaneous ones, or the
     * Eq. 34 averages of n, u, T (with lambda of Eq. 36 at the averaged
     * state) */
    const int averaged = c->gll_average && s->nsamples > 0;
    for (int cell = 0; cell < s->K; ++cell) {
        grad_state* G = &s->gs[cell];
        const cell_params* P = &s->par[cell];
        if (!averaged) {
            G->valid = P->valid;
            G->n = P->n; G->T = P->T; G->umag = P->umag; G->a_sound = P->a_sound; G->lambda = P->lambda;
            continue;
        }
        const double* A = s->avg;
        const int K = s->K;
        G->n = A[cell];
        G->T = A[(size_t)4 * K + cell];
        double u0 = A[(size_t)1 * K + cell], u1 = A[(size_t)2 * K + cell], u2 = A[(size_t)3 * K + cell];
        G->umag = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
        G->valid = G->n > 0 && G->T > 0;
        if (!G->valid) continue;
        double theta = s->R * G->T;
        G->a_sound = sqrt(GAMMA_MONO * theta);
        double rho = G->n * c->mass, p = rho * theta;
        double mu = s->mu_ref * pow(G->T / c->T_ref, c->omega);                  /* Eq. 35 */
        G->lambda = 16.0 / (5.0 * sqrt(2.0 * PI)) * mu / sqrt(rho * p);           /* Eq. 36 */
    }
    /* pass 2: GLL Knudsen number, P_ne, corrected moments, ES covariance */
    for (int cell = 0; cell < s->K; ++cell) {
        cell_moments* M = &s->mom[cell];
        cell_params* P = &s->par[cell];
        if (!P->valid) continue;
        double pne;
        if (c->mode == ORC_MODE_SP || c->mode == ORC_MODE_SPESBGK) pne = 0.0;
        else if (c->mode == ORC_MODE_FIXED_PNE) pne = c->fixed_pne;
        else {
            /* a cell whose own stencil state is missing (never sampled as
             * valid) has no gradient: Kn_GLL = 0 */
            const grad_state* G = &s->gs[cell];
            double kn = 0.0;
            if (G->valid) {
                double g[3];
                for (int q = 0; q < 3; ++q) {
                    double sum = 0;
                    for (int axis = c->dim == 1 ? 1 : 0; axis < 2; ++axis) {
                        double d = deriv(s, cell, axis, q);
                        sum += d * d;
                    }
                    g[q] = sqrt(sum);
                }
                double kn_rho = G->lambda * g[0] / G->n;                      /* Eq. 18, Q = rho */
                double kn_T = G->lambda * g[1] / G->T;                        /* Eq. 18, Q = T */
                double kn_u = G->lambda * g[2] / fmax(G->umag, G->a_sound);   /* Eq. 18, Q = |u| */
                kn = fmax(kn_rho, fmax(kn_T, kn_u));                          /* Eq. 17 */
            }
            pne = exp(-kn / KN_C);                                            /* Eq. 16 */
        }
        P->pne = pne;
        double fs = 1.0 + 0.5 * s->dt * P->nu * pne;            /* Eq. 33, stress */
        double fq = 1.0 + 0.5 * s->dt * P->nu * c->Pr * pne;    /* Eq. 33, heat flux */
        double sig[6] = {M->P[0] - M->theta, M->P[1] - M->theta, M->P[2] - M->theta, M->P[3], M->P[4], M->P[5]};
        for (int d = 0; d < 6; ++d) P->sig_star[d] = sig[d] / fs;
        for (int d = 0; d < 3; ++d) P->q_star[d] = M->Q[d] / fq;
        /* lambda_ij = theta delta_ij + (1 - 1/Pr) sigma*_ij / rho (Eq. 6c), lower Cholesky factor */
        double b = 1.0 - 1.0 / c->Pr;
        double A00 = M->theta + b * P->sig_star[0];
        double A11 = M->theta + b * P->sig_star[1];
        double A22 = M->theta + b * P->sig_star[2];
        double A10 = b * P->sig_star[3], A20 = b * P->sig_star[4], A21 = b * P->sig_star[5];
        int ok = A00 > 0;
        double L00 = 0, L10 = 0, L11 = 0, L20 = 0, L21 = 0, L22 = 0;
        if (ok) {
            L00 = sqrt(A00);
            L10 = A10 / L00;
            L20 = A20 / L00;
            double d1 = A11 - L10 * L10;
            ok = d1 > 0;
            if (ok) {
                L11 = sqrt(d1);
                L21 = (A21 - L20 * L10) / L11;
                double d2 = A22 - L20 * L20 - L21 * L21;
                ok = d2 > 0;
                if (ok) L22 = sqrt(d2);
            }
        }
        if (!ok) {
            double r = sqrt(M->theta);
            L00 = L11 = L22 = r;
            L10 = L20 = L21 = 0;
            s->counters[0]++;
        }
        P->L[0] = L00; P->L[1] = L10; P->L[2] = L11; P->L[3] = L20; P->L[4] = L21; P->L[5] = L22;
        P->p_relax = -expm1(-P->nu_es * s->dt);                 /* 1 - exp(-nu_ES dt), Eqs. 8b, 9 */
    }
}

/* ------------------------------------------------------------------------ */
/* 6. relaxation and per-cell conservation                                   */
/* ------------------------------------------------------------------------ */
/* time instant since t_n drawn from g_time (Eqs. 29-30), in a form that does
 * not overflow for large nu_ES dt */
static double sample_time(double U, double nu_es, double dt) {
    double a = nu_es * dt;
    if (a < 1.0) return log1p(U * expm1(a)) / nu_es;
    return dt + log(U + (1.0 - U) * exp(-a)) / nu_es;
}

typedef struct {
    double key;
    int64_t pos;
} key_pos;

static int cmp_key_pos(const void* a, const void* b) {
    const key_pos* x = (const key_pos*)a;
    const key_pos* y = (const key_pos*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->pos < y->pos ? -1 : (x->pos > y->pos);
}

/* ------------------------------------------------------------------------ */
/* Weighted added particles (Table 2 steps 2, 4, 7; Eqs. 22-28)              */
/* ------------------------------------------------------------------------ */
/* Eq. 26 for one velocity C about the cell mean: the weight that makes a    */
/* Maxwellian particle represent r_p (dt J / 2) / f_e, with the stress and   */
/* heat flux per unit density (sigma/rho, q/rho), so that sigma/p =          */
/* (sigma/rho)/theta and q/(p theta) = (q/rho)/theta^2.                       */
static double eq26_weight(const double* C, double theta, const double* sig, const double* q, double nu, double pne,
                          double dt, double Pr) {
    double quad = sig[0] * C[0] * C[0] + sig[1] * C[1] * C[1] + sig[2] * C[2] * C[2] +
                  2.0 * (sig[3] * C[0] * C[1] + sig[4] * C[0] * C[2] + sig[5] * C[1] * C[2]);
    double c2 = C[0] * C[0] + C[1] * C[1] + C[2] * C[2];
    double qc = q[0] * C[0] + q[1] * C[1] + q[2] * C[2];
    double bracket = quad / (2.0 * theta * theta) + 0.4 * Pr * qc / (theta * theta) * (c2 / (2.0 * theta) - 2.5);
    return -0.5 * nu * pne * dt * bracket;
}

/* N_a of Eq. 25 for a cell of N_eff particle weights: N_eff min(1, nu_ES dt)
 * / r_p, rounded up or down at random (its expectation is the printed
 * value); the weight of each added particle carries r_p / min(1, nu_ES dt)
 * so that, whatever the count, the added particles represent the PDF of
 * Eq. 22 (or 24, 27) in expectation. */
static int added_count(const orc_sim* s, int cell, double neff, double nu, uint32_t stage, double* prefactor) {
    double kap = fmin(1.0, s->cfg.Pr * nu * s->dt);
    *prefactor = kap > 0 ? s->cfg.r_p / kap : 0.0;
    if (!(neff > 0) || !(kap > 0)) return 0;
    uint32_t w[4];
    draw(s, (uint32_t)cell, s->step, P_CELL, stage, w);
    return (int)floor(neff * kap / s->cfg.r_p + orc_u01(w[0]));
}

/* Add the particles of one Table 2 stage to one cell: uniform positions,
 * Maxwellian velocities at the field's (u, theta), weights from Eq. 26 with
 * the field's (sigma, q, nu) times `factor` (1 for steps 2 and 4, the
 * Eq. 27 factor -2 (1 - e^-a)/a for step 7). */
static void add_weighted(orc_sim* s, int cell, double neff, const double* F, double pne, double factor, uint32_t stage) {
    double pref;
    int na = added_count(s, cell, neff, F[WF_NU], stage, &pref);
    if (na <= 0 || !(F[WF_TH] > 0)) return;
    double xl, yl;
    cell_lo(s, cell, &xl, &yl);
    double sq = sqrt(F[WF_TH]);
    reserve(s, s->np + na);
    for (int k = 0; k < na; ++k) {
        particle* q = &s->p[s->np++];
        uint32_t pid = s->next_pid++;
        uint32_t w[4], v[4];
        draw(s, pid, s->step, P_ADD, 0, w);
        draw(s, pid, s->step, P_ADD, 1, v);
        q->x = s->cfg.dim == 2 ? xl + orc_u01(w[0]) * s->dx : 0.0;
        q->y = yl + orc_u01(w[1]) * s->dy;
        double z0, z1, z2, z3;
        box_muller(v[0], v[1], &z0, &z1);
        box_muller(v[2], v[3], &z2, &z3);
        double C[3] = {sq * z0, sq * z1, sq * z2};
        for (int d = 0; d < 3; ++d) q->c[d] = F[WF_U + d] + C[d];
        q->w = factor * pref * eq26_weight(C, F[WF_TH], &F[WF_SIG], &F[WF_Q], F[WF_NU], pne, s->dt, s->cfg.Pr);
        q->pid = pid;
        q->cell = cell;
        q->alive = 1;
    }
}

/* Eq. 34 average of a weight field, started at zero stress and heat flux
 * (the Maxwellian initial state) and at the first mean velocity, theta, nu */
static void average_fields(const orc_sim* s, double* avg, const double* inst, int first) {
    const double keep = (s->cfg.n_avg - 1.0) / s->cfg.n_avg, add = 1.0 / s->cfg.n_avg;
    for (int cell = 0; cell < s->K; ++cell) {
        double* a = avg + (size_t)WF_N * cell;
        const double* f = inst + (size_t)WF_N * cell;
        for (int k = 0; k < WF_N; ++k) {
            if (first) a[k] = (k >= WF_SIG && k < WF_NU) ? 0.0 : f[k];
            else a[k] = keep * a[k] + add * f[k];
        }
    }
}

static double nu_of_state(const orc_sim* s, double neff, double theta) {
    double n = neff * s->w, T = theta / s->R;
    double rho = n * s->cfg.mass, p = rho * theta;
    double mu = s->mu_ref * pow(T / s->cfg.T_ref, s->cfg.omega);    /* Eq. 35 */
    return p / mu;
}

static double pne_of(const orc_sim* s, int cell) {
    const orc_config* c = &s->cfg;
    if (c->mode == ORC_MODE_SP || c->mode == ORC_MODE_SPESBGK) return 0.0;
    if (c->mode == ORC_MODE_FIXED_PNE) return c->fixed_pne;
    return s->par[cell].pne;   /* Eq. 16, from the last parameter evaluation */
}

/* Table 2 step 2, at t_n: the weighted moments of f^n in every cell (the
 * particles sit in the cells of the last sort; step-7 particles were
 * created in theirs), then N_a particles per cell with weights W^n. */
static void weighted_step2(orc_sim* s) {
    const int K = s->K;
    double* acc = (double*)calloc((size_t)K * 14, sizeof(double));
    for (int64_t i = 0; i < s->np; ++i) {
        const particle* q = &s->p[i];
        double* a = acc + (size_t)14 * q->cell;
        a[0] += q->w;
        for (int d = 0; d < 3; ++d) a[1 + d] += q->w * q->c[d];
    }
    for (int cell = 0; cell < K; ++cell) {
        double* a = acc + (size_t)14 * cell;
        if (a[0] > 0) for (int d = 0; d < 3; ++d) a[1 + d] /= a[0];
    }
    for (int64_t i = 0; i < s->np; ++i) {
        const particle* q = &s->p[i];
        double* a = acc + (size_t)14 * q->cell;
        double C[3] = {q->c[0] - a[1], q->c[1] - a[2], q->c[2] - a[3]};
        double c2 = C[0] * C[0] + C[1] * C[1] + C[2] * C[2];
        a[4] += q->w * c2;
        a[5] += q->w * C[0] * C[0]; a[6] += q->w * C[1] * C[1]; a[7] += q->w * C[2] * C[2];
        a[8] += q->w * C[0] * C[1]; a[9] += q->w * C[0] * C[2]; a[10] += q->w * C[1] * C[2];
        for (int d = 0; d < 3; ++d) a[11 + d] += q->w * c2 * C[d];
    }
    double* neff = (double*)calloc((size_t)K, sizeof(double));
    for (int cell = 0; cell < K; ++cell) {
        const double* a = acc + (size_t)14 * cell;
        double* F = s->wf_n + (size_t)WF_N * cell;
        memset(F, 0, WF_N * sizeof(double));
        neff[cell] = a[0];
        if (!(a[0] > 1.0) || !(a[4] > 0)) continue;
        double th = a[4] / (3.0 * a[0]);
        for (int d = 0; d < 3; ++d) F[WF_U + d] = a[1 + d];
        F[WF_TH] = th;
        for (int d = 0; d < 3; ++d) F[WF_SIG + d] = a[5 + d] / a[0] - th;
        for (int d = 0; d < 3; ++d) F[WF_SIG + 3 + d] = a[8 + d] / a[0];
        for (int d = 0; d < 3; ++d) F[WF_Q + d] = a[11 + d] / (2.0 * a[0]);
        F[WF_NU] = nu_of_state(s, a[0], th);
    }
    const double* use = s->wf_n;
    if (s->cfg.weight_average) {
        average_fields(s, s->wa_n, s->wf_n, !(s->wa_started & 1));
        s->wa_started |= 1;
        use = s->wa_n;
    }
    for (int cell = 0; cell < K; ++cell) {
        double pne = pne_of(s, cell);
        if (pne == 0.0 || !(neff[cell] > 1.0)) continue;
        add_weighted(s, cell, neff[cell], use + (size_t)WF_N * cell, pne, 1.0, 1);
    }
    free(acc);
    free(neff);
}

/* fields of f* for steps 4 and 7 from this step's moments and parameters
 * (sigma* and q* of Eq. 33, per unit density) */
static const double* star_fields(orc_sim* s) {
    for (int cell = 0; cell < s->K; ++cell) {
        const cell_moments* M = &s->mom[cell];
        const cell_params* P = &s->par[cell];
        double* F = s->wf_s + (size_t)WF_N * cell;
        memset(F, 0, WF_N * sizeof(double));
        if (!P->valid) continue;
        for (int d = 0; d < 3; ++d) F[WF_U + d] = M->u[d];
        F[WF_TH] = M->theta;
        for (int d = 0; d < 6; ++d) F[WF_SIG + d] = P->sig_star[d];
        for (int d = 0; d < 3; ++d) F[WF_Q + d] = P->q_star[d];
        F[WF_NU] = P->nu;
    }
    if (!s->cfg.weight_average) return s->wf_s;
    average_fields(s, s->wa_s, s->wf_s, !(s->wa_started & 2));
    s->wa_started |= 2;
    return s->wa_s;
}

/* Table 2 steps 4-7 in place of the plain relaxation: step 4 adds weighted
 * particles for f*; steps 5-6 select (Bernoulli, as the plain path), give
 * int(sum of the selected weights) of them, in selection-key order, weight 1
 * and a velocity from f_G(t) (Eq. 28, the count rounded at random so that
 * mass is kept in expectation), delete the others and restore the momentum
 * and thermal energy per unit weight of the selected set; step 7 adds
 * weighted particles for the third term of Eq. 27. */
static void relax_weighted(orc_sim* s) {
    const orc_config* c = &s->cfg;
    const double* F = star_fields(s);
    for (int cell = 0; cell < s->K; ++cell) {
        const cell_params* P = &s->par[cell];
        double pne = pne_of(s, cell);
        if (!P->valid || pne == 0.0) continue;
        add_weighted(s, cell, s->mom[cell].neff, F + (size_t)WF_N * cell, pne, 1.0, 2);
    }
    /* the step-4 particles join their cells */
    qsort(s->p, (size_t)s->np, sizeof(particle), cmp_cell_pid);
    int64_t i = 0, cap = 0;
    double* cold = NULL;
    key_pos* order = NULL;
    int* sel = NULL;
    while (i < s->np) {
        int cell = s->p[i].cell;
        int64_t j = i;
        while (j < s->np && s->p[j].cell == cell) ++j;
        cell_params* P = &s->par[cell];
        cell_moments* M = &s->mom[cell];
        int64_t n = j - i;
        if (n > cap) {
            cap = n;
            cold = (double*)realloc(cold, (size_t)cap * 3 * sizeof(double));
            sel = (int*)realloc(sel, (size_t)cap * sizeof(int));
            order = (key_pos*)realloc(order, (size_t)cap * sizeof(key_pos));
        }
        P->n_relaxed = 0;
        if (!P->valid) { i = j; continue; }
        /* step 5: selection, and the selected set's weight, momentum, energy */
        int64_t ns = 0;
        double sw = 0, su[3] = {0, 0, 0};
        for (int64_t k = i; k < j; ++k) {
            uint32_t w[4];
            draw(s, s->p[k].pid, s->step, P_RELAX, 0, w);
            double key = orc_u01(w[0]);
            sel[k - i] = key < P->p_relax;
            if (!sel[k - i]) continue;
            order[ns].key = key;
            order[ns].pos = k - i;
            ++ns;
            sw += s->p[k].w;
            for (int d = 0; d < 3; ++d) su[d] += s->p[k].w * s->p[k].c[d];
        }
        if (ns == 0) { i = j; continue; }
        /* Eq. 28: int(sum W) of the selected keep weight 1, the rest go */
        uint32_t w4[4];
        draw(s, (uint32_t)cell, s->step, P_CELL, 0, w4);
        int64_t m = sw > 0 ? (int64_t)floor(sw + orc_u01(w4[0])) : 0;
        if (m > ns) m = ns;
        qsort(order, (size_t)ns, sizeof(key_pos), cmp_key_pos);
        double uo[3] = {0, 0, 0}, eo = 0;
        if (sw > 0) {
            for (int d = 0; d < 3; ++d) uo[d] = su[d] / sw;
            for (int64_t r = 0; r < ns; ++r) {
                const particle* q = &s->p[i + order[r].pos];
                for (int d = 0; d < 3; ++d) eo += q->w * (q->c[d] - uo[d]) * (q->c[d] - uo[d]);
            }
            eo /= sw;
        }
        for (int64_t r = m; r < ns; ++r) s->p[i + order[r].pos].alive = 0;
        /* step 6: the reassigned particles from f_G(t) (Eqs. 29-32) */
        double un[3] = {0, 0, 0};
        for (int64_t r = 0; r < m; ++r) {
            particle* q = &s->p[i + order[r].pos];
            uint32_t w[4], v[4];
            draw(s, q->pid, s->step, P_RELAX, 0, w);
            double t = sample_time(orc_u01(w[1]), P->nu_es, s->dt);
            double sfac = c->mode == ORC_MODE_SPESBGK ? 1.0 : P->pne + (1.0 - P->pne) * exp(-P->nu * t);
            if (c->mode == ORC_MODE_FIXED_PNE) sfac = c->fixed_pne + (1.0 - c->fixed_pne) * exp(-P->nu * t);
            draw(s, q->pid, s->step, P_RELAX, 1, v);
            double z[6];
            box_muller(w[2], w[3], &z[0], &z[1]);
            box_muller(v[0], v[1], &z[2], &z[3]);
            box_muller(v[2], v[3], &z[4], &z[5]);
            const double* L = P->L;
            double a = sqrt(sfac), bb = sqrt((1.0 - sfac) * M->theta);
            double C0 = a * (L[0] * z[0]) + bb * z[3];
            double C1 = a * (L[1] * z[0] + L[2] * z[1]) + bb * z[4];
            double C2 = a * (L[3] * z[0] + L[4] * z[1] + L[5] * z[2]) + bb * z[5];
            q->c[0] = M->u[0] + C0;
            q->c[1] = M->u[1] + C1;
            q->c[2] = M->u[2] + C2;
            q->w = 1.0;
            for (int d = 0; d < 3; ++d) un[d] += q->c[d];
        }
        /* conservation: the reassigned set carries the selected set's mean
         * velocity and thermal energy per unit weight */
        if (m >= 2 && sw > 0) {
            for (int d = 0; d < 3; ++d) un[d] /= m;
            double en = 0;
            for (int64_t r = 0; r < m; ++r) {
                const particle* q = &s->p[i + order[r].pos];
                for (int d = 0; d < 3; ++d) en += (q->c[d] - un[d]) * (q->c[d] - un[d]);
            }
            en /= m;
            double alpha = (en > 0 && eo > 0) ? sqrt(eo / en) : 1.0;
            for (int64_t r = 0; r < m; ++r) {
                particle* q = &s->p[i + order[r].pos];
                for (int d = 0; d < 3; ++d) q->c[d] = uo[d] + alpha * (q->c[d] - un[d]);
            }
        } else if (m == 1 && sw > 0) {
            particle* q = &s->p[i + order[0].pos];
            for (int d = 0; d < 3; ++d) q->c[d] = uo[d] + (q->c[d] - un[d]) * sqrt(eo > 0 ? eo / (3.0 * M->theta) : 1.0);
        }
        P->n_relaxed = (int)m;
        (void)cold;
        i = j;
    }
    free(cold);
    free(sel);
    free(order);
    /* deleted particles leave */
    int64_t k = 0;
    for (int64_t r = 0; r < s->np; ++r)
        if (s->p[r].alive) s->p[k++] = s->p[r];
    s->np = k;
    /* step 7: the third term of Eq. 27, -(1 - e^-a)/nu_ES J*: weights
     * W' = -W* 2 (1 - e^-a) / a, a = nu_ES dt */
    for (int cell = 0; cell < s->K; ++cell) {
        const cell_params* P = &s->par[cell];
        double pne = pne_of(s, cell);
        if (!P->valid || pne == 0.0) continue;
        double a = P->nu_es * s->dt;
        double fac = -2.0 * (-expm1(-a)) / a;
        add_weighted(s, cell, s->mom[cell].neff, F + (size_t)WF_N * cell, pne, fac, 3);
    }
}

static void relax_phase(orc_sim* s) {
    if (s->cfg.weighted) {
        relax_weighted(s);
        return;
    }
    int64_t i = 0;
    double* cold = NULL;
    double* ukey = NULL;
    key_pos* order = NULL;
    int* sel = NULL;
    int64_t cap = 0;
    while (i < s->np) {
        int cell = s->p[i].cell;
        int64_t j = i;
        while (j < s->np && s->p[j].cell == cell) ++j;
        cell_params* P = &s->par[cell];
        cell_moments* M = &s->mom[cell];
        int64_t n = j - i;
        if (n > cap) {
            cap = n;
            cold = (double*)realloc(cold, (size_t)cap * 3 * sizeof(double));
            sel = (int*)realloc(sel, (size_t)cap * sizeof(int));
            ukey = (double*)realloc(ukey, (size_t)cap * sizeof(double));
            order = (key_pos*)realloc(order, (size_t)cap * sizeof(key_pos));
        }
        P->n_relaxed = 0;
        if (!P->valid) { i = j; continue; }
        const orc_config* c = &s->cfg;
        /* selection: Bernoulli per particle, or the fixed count of Eq. 9 */
        for (int64_t k = i; k < j; ++k) {
            uint32_t w[4];
            draw(s, s->p[k].pid, s->step, P_RELAX, 0, w);
            ukey[k - i] = orc_u01(w[0]);
            sel[k - i] = ukey[k - i] < P->p_relax;
        }
        if (c->selection == ORC_SELECT_FIXED_COUNT) {
            /* Eq. 9: the ns particles with the smallest keys (ties: lower
             * position first), ns the nearest integer to N_c (1 - e^-a) */
            int64_t ns = (int64_t)floor((double)n * P->p_relax + 0.5);
            for (int64_t r = 0; r < n; ++r) { order[r].key = ukey[r]; order[r].pos = r; sel[r] = 0; }
            qsort(order, (size_t)n, sizeof(key_pos), cmp_key_pos);
            for (int64_t r = 0; r < ns; ++r) sel[order[r].pos] = 1;
        }
        int nr = 0;
        for (int64_t k = i; k < j; ++k) {
            particle* q = &s->p[k];
            int64_t r = k - i;
            if (!sel[r]) continue;
            ++nr;
            uint32_t w[4];
            draw(s, q->pid, s->step, P_RELAX, 0, w);
            for (int d = 0; d < 3; ++d) cold[3 * r + d] = q->c[d];
            double t = sample_time(orc_u01(w[1]), P->nu_es, s->dt);
            /* Eq. 32; SP-ESBGK holds the target for the whole step (Eq. 8b) */
            double sfac = c->mode == ORC_MODE_SPESBGK ? 1.0 : P->pne + (1.0 - P->pne) * exp(-P->nu * t);
            uint32_t v[4];
            draw(s, q->pid, s->step, P_RELAX, 1, v);
            double z[6];
            box_muller(w[2], w[3], &z[0], &z[1]);
            box_muller(v[0], v[1], &z[2], &z[3]);
            box_muller(v[2], v[3], &z[4], &z[5]);
            double C0, C1, C2;
            if (c->es_sampler == ORC_SAMPLER_GALLIS_TORCZYNSKI) {
                /* Eq. 10: one thermal component per (cosine) Box-Muller pair;
                 * Eq. 11: C = S C*, S = I - (1 - Pr)/(2 Pr) (P/theta - I), with
                 * P/theta - I = s sigma* / (rho theta) at the time instant */
                double st = sqrt(M->theta);
                double cs[3] = {st * z[0], st * z[2], st * z[4]};
                double beta = (1.0 - c->Pr) / (2.0 * c->Pr) * sfac / M->theta;
                const double* g = P->sig_star;   /* xx, yy, zz, xy, xz, yz (per unit density) */
                double S[3][3] = {{1.0 - beta * g[0], -beta * g[3], -beta * g[4]},
                                  {-beta * g[3], 1.0 - beta * g[1], -beta * g[5]},
                                  {-beta * g[4], -beta * g[5], 1.0 - beta * g[2]}};
                C0 = S[0][0] * cs[0] + S[0][1] * cs[1] + S[0][2] * cs[2];
                C1 = S[1][0] * cs[0] + S[1][1] * cs[1] + S[1][2] * cs[2];
                C2 = S[2][0] * cs[0] + S[2][1] * cs[1] + S[2][2] * cs[2];
            } else {
                /* covariance theta I + s (1 - 1/Pr) sigma* / rho = s L L^T + (1 - s) theta I */
                const double* L = P->L;
                double a = sqrt(sfac), bb = sqrt((1.0 - sfac) * M->theta);
                C0 = a * (L[0] * z[0]) + bb * z[3];
                C1 = a * (L[1] * z[0] + L[2] * z[1]) + bb * z[4];
                C2 = a * (L[3] * z[0] + L[4] * z[1] + L[5] * z[2]) + bb * z[5];
            }
            q->c[0] = M->u[0] + C0;
            q->c[1] = M->u[1] + C1;
            q->c[2] = M->u[2] + C2;
        }
        /* conservation over the relaxed subset R of the cell */
        if (nr == 1) {
            for (int64_t k = i; k < j; ++k)
                if (sel[k - i]) for (int d = 0; d < 3; ++d) s->p[k].c[d] = cold[3 * (k - i) + d];
            nr = 0;
        } else if (nr >= 2) {
            double uo[3] = {0, 0, 0}, un[3] = {0, 0, 0};
            for (int64_t k = i; k < j; ++k) {
                if (!sel[k - i]) continue;
                for (int d = 0; d < 3; ++d) { uo[d] += cold[3 * (k - i) + d]; un[d] += s->p[k].c[d]; }
            }
            for (int d = 0; d < 3; ++d) { uo[d] /= nr; un[d] /= nr; }
            double eo = 0, en = 0;
            for (int64_t k = i; k < j; ++k) {
                if (!sel[k - i]) continue;
                for (int d = 0; d < 3; ++d) {
                    double a = cold[3 * (k - i) + d] - uo[d];
                    double b = s->p[k].c[d] - un[d];
                    eo += a * a;
                    en += b * b;
                }
            }
            if (en > 0) {
                double alpha = sqrt(eo / en);
                for (int64_t k = i; k < j; ++k) {
                    if (!sel[k - i]) continue;
                    for (int d = 0; d < 3; ++d) s->p[k].c[d] = uo[d] + alpha * (s->p[k].c[d] - un[d]);
                }
            } else {
                for (int64_t k = i; k < j; ++k)
                    if (sel[k - i]) for (int d = 0; d < 3; ++d) s->p[k].c[d] = cold[3 * (k - i) + d];
                nr = 0;
            }
        }
        P->n_relaxed = nr;
        i = j;
    }
    free(cold);
    free(sel);
    free(ukey);
    free(order);
}

/* ------------------------------------------------------------------------ */
/* 7. sampling: instantaneous fields and Eq. 34                              */
/* ------------------------------------------------------------------------ */
static void sample_phase(orc_sim* s) {
    const orc_config* c = &s->cfg;
    int K = s->K;
    for (int cell = 0; cell < K; ++cell) {
        cell_moments* M = &s->mom[cell];
        cell_params* P = &s->par[cell];
        double f[ORC_NFIELDS];
        memset(f, 0, sizeof(f));
        f[0] = M->neff * s->w;
        f[15] = M->n;
        if (M->n >= 1) for (int d = 0; d < 3; ++d) f[1 + d] = M->u[d];
        if (P->valid) {
            double rho = P->n * c->mass;
            f[4] = P->T;
            f[5] = P->p + rho * P->sig_star[0];
            f[6] = P->p + rho * P->sig_star[1];
            f[7] = P->p + rho * P->sig_star[2];
            f[8] = rho * P->sig_star[3];
            f[9] = rho * P->sig_star[4];
            f[10] = rho * P->sig_star[5];
            for (int d = 0; d < 3; ++d) f[11 + d] = rho * P->q_star[d];
            f[14] = P->pne;
        }
        for (int q = 0; q < ORC_NFIELDS; ++q) {
            s->inst[(size_t)q * K + cell] = f[q];
            double* a = &s->avg[(size_t)q * K + cell];
            if (s->nsamples == 0) *a = f[q];
            else *a = ((c->n_avg - 1.0) / c->n_avg) * *a + f[q] / c->n_avg;
        }
    }
    s->nsamples++;
}

int orc_phase(orc_sim* s, int phase) {
    if (!s) return -1;
    switch (phase) {
    case ORC_PH_STREAM: stream_phase(s); return 0;
    case ORC_PH_RESERVOIR: reservoir_phase(s); return 0;
    case ORC_PH_SORT: sort_phase(s); return 0;
    case ORC_PH_MOMENTS: moments_phase(s); return 0;
    case ORC_PH_PARAMS: params_phase(s); return 0;
    case ORC_PH_RELAX: relax_phase(s); return 0;
    case ORC_PH_SAMPLE: sample_phase(s); s->step++; return 0;
    default: return -1;
    }
}

int orc_step(orc_sim* s, int nsteps) {
    if (!s || nsteps < 0) return -1;
    for (int n = 0; n < nsteps; ++n)
        for (int ph = ORC_PH_STREAM; ph <= ORC_PH_SAMPLE; ++ph) orc_phase(s, ph);
    return 0;
}

int64_t orc_num_particles(const orc_sim* s) { return s ? s->np : -1; }
int orc_num_cells(const orc_sim* s) { return s ? s->K : -1; }
double orc_dt(const orc_sim* s) { return s ? s->dt : 0; }
double orc_mu_ref(const orc_sim* s) { return s ? s->mu_ref : 0; }
uint32_t orc_step_index(const orc_sim* s) { return s ? s->step : 0; }

int orc_get_particles(const orc_sim* s, double* pos, double* vel, uint32_t* pid, int32_t* cell) {
    if (!s) return -1;
    for (int64_t i = 0; i < s->np; ++i) {
        const particle* q = &s->p[i];
        if (pos) { pos[2 * i] = q->x; pos[2 * i + 1] = q->y; }
        if (vel) for (int d = 0; d < 3; ++d) vel[3 * i + d] = q->c[d];
        if (pid) pid[i] = q->pid;
        if (cell) cell[i] = cell_of(s, q->x, q->y);
    }
    return 0;
}

int orc_get_weights(const orc_sim* s, double* w) {
    if (!s) return -1;
    for (int64_t i = 0; i < s->np; ++i) w[i] = s->p[i].w;
    return 0;
}

int orc_get_counts(const orc_sim* s, int32_t* counts) {
    if (!s) return -1;
    memset(counts, 0, (size_t)s->K * sizeof(int32_t));
    for (int64_t i = 0; i < s->np; ++i) counts[cell_of(s, s->p[i].x, s->p[i].y)]++;
    return 0;
}

int orc_get_fields(const orc_sim* s, int averaged, double* out) {
    if (!s) return -1;
    memcpy(out, averaged ? s->avg : s->inst, (size_t)ORC_NFIELDS * s->K * sizeof(double));
    return 0;
}

int orc_get_params(const orc_sim* s, double* out) {
    if (!s) return -1;
    for (int cell = 0; cell < s->K; ++cell) {
        const cell_params* P = &s->par[cell];
        const cell_moments* M = &s->mom[cell];
        double* o = out + 16 * (size_t)cell;
        for (int d = 0; d < 3; ++d) o[d] = M->u[d];
        o[3] = M->theta;
        for (int d = 0; d < 6; ++d) o[4 + d] = P->L[d];
        o[10] = P->p_relax;
        o[11] = P->nu;
        o[12] = P->nu_es;
        o[13] = P->pne;
        o[14] = P->valid;
        o[15] = P->n_relaxed;
    }
    return 0;
}

int orc_get_counters(const orc_sim* s, int64_t* out) {
    if (!s) return -1;
    memcpy(out, s->counters, sizeof(s->counters));
    return 0;
}
