/*
 * usp_oracle.h -- plain FP64 CPU oracle of the USP-ESBGK particle update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or helper with the CUDA library in paper_1808_03801_gb300/;
 * the only thing both sides agree on is the published definition of the
 * Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the way
 * its words are mapped to variates, each written out independently.
 *
 * The oracle follows the paper (Fei, Zhang, Li, Liu, "A unified stochastic
 * particle BGK method for multiscale gas flows", arXiv:1808.03801):
 *   moments ............ Sec. 2, Eq. 1
 *   ES Gaussian ........ Eqs. 6a-6c
 *   relaxation ......... Eqs. 8b, 9, 27 (first two terms), 29-32
 *   USP parameters ..... Eqs. 16-18 (P_ne), 33 (sigma*, q*), 35-37
 *   sampling ........... Eq. 34
 *   step outline ....... Table 2 with the weighted-particle steps 2, 4, 7
 *                        left out (all particle weights are 1).
 *   options ............ counting plane for the slit mass flow (Eq. 41);
 *                        Kn_GLL from the Eq. 34 averages; SP-ESBGK step
 *                        (Eq. 8b), fixed-count selection (Eq. 9) and the
 *                        Gallis-Torczynski sampler (Eqs. 10-11).
 * Every stage is a plain loop in FP64 over particles in (cell, pid) order.
 */
#ifndef USP_ORACLE_H
#define USP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_DIFFUSE = 0, ORC_BC_SPECULAR = 1, ORC_BC_PERIODIC = 2, ORC_BC_RESERVOIR = 3 };
/* ORC_MODE_SPESBGK: the SP-ESBGK step of Sec. 2 (Eq. 8b, Table 1): the
 * Gaussian target is held at the post-convection state for the whole step
 * (no time instant, no Eq. 33 division) */
enum { ORC_MODE_USP = 0, ORC_MODE_SP = 1, ORC_MODE_FIXED_PNE = 2, ORC_MODE_SPESBGK = 3 };
enum { ORC_SELECT_BERNOULLI = 0, ORC_SELECT_FIXED_COUNT = 1 };
enum { ORC_SAMPLER_CHOLESKY = 0, ORC_SAMPLER_GALLIS_TORCZYNSKI = 1 };
enum { ORC_NFIELDS = 16 };
#define ORC_MAXSEG 4

/* Faces: 0 = x-lo, 1 = x-hi, 2 = y-lo, 3 = y-hi.  A 1-D grid resolves y only. */
typedef struct {
    /* gas: molecular mass [kg], viscosity law mu = mu_ref (T/T_ref)^omega (Eq. 35), Prandtl number */
    double mass, T_ref, mu_ref, omega, Pr;
    /* uniform grid */
    int dim, nx, ny;
    double lo[2], hi[2];
    /* one boundary condition per face */
    int face_kind[4];
    double face_T[4];
    double face_u[4][3];
    double face_n[4];          /* reservoir number density [1/m^3] */
    /* zero-thickness plates normal to x (slit walls) */
    int nseg;
    double seg_pos[ORC_MAXSEG], seg_lo[ORC_MAXSEG], seg_hi[ORC_MAXSEG];
    int seg_kind[ORC_MAXSEG];
    double seg_T[ORC_MAXSEG];
    double seg_u[ORC_MAXSEG][3];
    /* run parameters */
    double Kn, L_ref, n_ref;   /* reference state: number density n_ref at T_ref */
    double dt, dt_over_tauc;   /* dt used when > 0, else dt_over_tauc * tau_c(ref) (Eq. 37) */
    double body_accel[3];
    int ppc_ref;               /* particles per cell at n_ref */
    int n_avg;                 /* n_a of Eq. 34 */
    int mode;                  /* ORC_MODE_* */
    double fixed_pne;
    int reservoir_cols;        /* buffer cell layers next to a reservoir face */
    /* counting plane for the mass flow rate of Eq. 41: normal to x (1) or
     * y (2) at flux_pos; 0 = none */
    int flux_axis;
    double flux_pos;
    /* 1: the Kn_GLL of Eqs. 17-18 is taken from the Eq. 34 averaged fields
     * (n, u, T of every cell) once at least one sample exists -- the time
     * averaging that Sec. 3 applies to steady flows to cut statistical
     * noise; 0: from the instantaneous moments */
    int gll_average;
    /* selection: ORC_SELECT_BERNOULLI (each particle relaxes with 1 - e^-a)
     * or ORC_SELECT_FIXED_COUNT (Eq. 9: the N_s = nearest-int(N_c (1 - e^-a))
     * particles of the cell with the smallest selection uniforms);
     * es_sampler: ORC_SAMPLER_CHOLESKY (Gaussian through the Cholesky factor)
     * or ORC_SAMPLER_GALLIS_TORCZYNSKI (thermal velocities of Eq. 10
     * transformed by S of Eq. 11) */
    int selection, es_sampler;
    /* weighted: 1 adds the weighted particles of Table 2 steps 2, 4 and 7
     * (Eqs. 22-28, the third term of Eq. 27); r_p the scale of Eq. 25 (0:
     * 10, the paper's value); weight_average: the fields that define the
     * weights (u, theta, sigma, q, nu of Eq. 26) are the Eq. 34 averages,
     * stress and heat flux starting from zero */
    int weighted;
    double r_p;
    int weight_average;
} orc_config;

typedef struct {
    double lo[2], hi[2];
    double n, T, u[3];
} orc_region;

typedef struct orc_sim orc_sim;

/* Philox4x32-10 (Salmon et al. 2011): counter ctr[4], key key[2] -> out[4]. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_u01(uint32_t x);

orc_sim* orc_create(const orc_config* cfg);
void orc_destroy(orc_sim* s);
int orc_init_particles(orc_sim* s, const orc_region* regs, int nreg, uint64_t seed);
/* load an arbitrary state (pos is n x 2: x, y; x ignored in 1-D) */
int orc_set_particles(orc_sim* s, int64_t n, const double* pos, const double* vel,
                      const uint32_t* pid, uint32_t next_pid, uint64_t seed);

/* Phases of one step, in order; orc_step runs all of them nsteps times. */
enum { ORC_PH_STREAM = 0, ORC_PH_RESERVOIR = 1, ORC_PH_SORT = 2, ORC_PH_MOMENTS = 3,
       ORC_PH_PARAMS = 4, ORC_PH_RELAX = 5, ORC_PH_SAMPLE = 6 };
int orc_phase(orc_sim* s, int phase);
int orc_step(orc_sim* s, int nsteps);

/* queries */
int64_t orc_num_particles(const orc_sim* s);
int orc_num_cells(const orc_sim* s);
double orc_dt(const orc_sim* s);
double orc_mu_ref(const orc_sim* s);
uint32_t orc_step_index(const orc_sim* s);
/* particles in storage order ((cell, pid) after a sort) */
int orc_get_particles(const orc_sim* s, double* pos, double* vel, uint32_t* pid, int32_t* cell);
/* particle weights in the order of orc_get_particles */
int orc_get_weights(const orc_sim* s, double* w);
/* per-cell: counts, fields (ORC_NFIELDS x K, [field][cell]) */
int orc_get_counts(const orc_sim* s, int32_t* counts);
int orc_get_fields(const orc_sim* s, int averaged, double* out);
/* per-cell relaxation parameters: [K][16] = u0,u1,u2, theta, L00,L10,L11,L20,L21,L22,
 * P_relax, nu, nu_ES, P_ne, valid, n_relaxed */
int orc_get_params(const orc_sim* s, double* out);
/* counters: [0] Cholesky fallbacks, [1] bounce-cap clamps, [2] removed, [3] injected,
 * [4] net particles through the counting plane (+1 for each advection that
 * starts below flux_pos and ends at or above it, -1 for the reverse) */
int orc_get_counters(const orc_sim* s, int64_t* out);

#ifdef __cplusplus
}
#endif
#endif
