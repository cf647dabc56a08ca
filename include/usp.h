/*
 * usp.h -- C ABI of the GB300 (sm_103a) particle update of the unified
 * stochastic particle ESBGK method (USP-ESBGK) of Fei, Zhang, Li and Liu,
 * arXiv:1808.03801.
 *
 * One time step follows the paper's Table 2 with all particle weights equal
 * to one (its weighted-particle steps 2, 4 and 7 are not part of this
 * library):
 *   advection with wall / reservoir boundaries   Table 1 steps 1-2, Table 2 step 3
 *   cell counting-sort                           (cells of Sec. 3.2; N_c of Eq. 9)
 *   per-cell moments n, u, T, p_ij, q_i          Eq. 1
 *   per-cell USP parameters                      Eqs. 16-18 (P_ne), 33 (sigma*, q*),
 *                                                35-36 (mu, lambda), 6c (ES covariance)
 *   relaxation with probability 1 - e^(-nu_ES dt) Eqs. 8b, 9
 *   ES Gaussian at a time instant from g_time     Eqs. 27 (first two terms), 29-32, 6b
 *   per-cell momentum / energy conservation
 *   sampling and exponential time average        Eq. 34
 *
 * Conventions for every call:
 *   - the return value is a status: USP_OK (0) or a negative USP_ERR_* code;
 *     no call aborts, traps or exits the process;
 *   - a handle owns all device memory it allocates; the caller owns every
 *     buffer it passes in (host or device, as stated per argument);
 *   - work is queued on the CUDA stream given at creation; calls that return
 *     data to the host synchronise that stream first;
 *   - a handle is not thread-safe; distinct handles are independent;
 *   - after an error, usp_last_error() describes it.
 * Units are SI throughout (m, s, kg, K).
 */
#ifndef USP_H
#define USP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define USP_OK 0
#define USP_ERR_INVALID_ARG (-1)
#define USP_ERR_OOM (-2)
#define USP_ERR_CUDA (-3)
#define USP_ERR_CAPACITY (-4)
#define USP_ERR_TIMEOUT (-5)
#define USP_ERR_STATE (-6)

/* boundary kinds (one per domain face; plates use DIFFUSE or SPECULAR) */
#define USP_BC_DIFFUSE 0   /* full accommodation at T, wall velocity u */
#define USP_BC_SPECULAR 1  /* mirror reflection */
#define USP_BC_PERIODIC 2  /* both faces of the axis must be periodic */
#define USP_BC_RESERVOIR 3 /* particles leaving are removed; buffer cells refilled at (n, T, u) */

/* relaxation modes */
#define USP_MODE_USP 0       /* P_ne from the gradient-length local Knudsen number, Eq. 16 */
#define USP_MODE_SP 1        /* P_ne = 0: the SP-ESBGK scheme (Appendix B limit) */
#define USP_MODE_FIXED_PNE 2 /* P_ne = params.fixed_pne everywhere */
#define USP_MODE_SPESBGK 3   /* the SP-ESBGK step of Sec. 2 (Eq. 8b): the Gaussian target held at the
                                post-convection state (no time instant, no Eq. 33 division) */

/* relaxation selection and sampler (the SP-ESBGK ablations of Sec. 2; both pipelines) */
#define USP_SELECT_BERNOULLI 0        /* each particle relaxes with probability 1 - exp(-nu_ES dt) */
#define USP_SELECT_FIXED_COUNT 1      /* Eq. 9: the nearest integer to N_c (1 - exp(-nu_ES dt)) particles
                                         of the cell with the smallest selection words */
#define USP_SAMPLER_CHOLESKY 0        /* ES Gaussian through the Cholesky factor of its covariance */
#define USP_SAMPLER_GALLIS_TORCZYNSKI 1 /* Eq. 10 thermal velocities transformed by S of Eq. 11 */

/* particle storage precision */
#define USP_FP64 0       /* positions and velocities stored and streamed in FP64 */
#define USP_FP32_MIXED 1 /* FP32 storage and per-particle math; plain pipeline: FP64 per-cell sums and
                            parameters; fused: FP32 centred sums and parameters, FP64 field averages */

/* step pipeline */
#define USP_PIPE_PLAIN 0 /* one kernel per stage */
#define USP_PIPE_FUSED 1 /* relaxation fused with the next advection; FP32_MIXED only */

/* which field set usp_sample_macro returns */
#define USP_SAMPLE_INSTANT 0
#define USP_SAMPLE_AVERAGED 1

/* per-cell fields returned by usp_sample_macro, layout [field][cell] */
#define USP_NFIELDS 16
/* 0 n [1/m^3], 1-3 u [m/s], 4 T [K], 5-10 p_xx p_yy p_zz p_xy p_xz p_yz [Pa]
 * (p delta_ij + sigma*_ij of Eq. 33), 11-13 q* [W/m^2] (Eq. 33), 14 P_ne,
 * 15 particles in the cell.  Cells with fewer than two particles report
 * n, u (if one particle) and the count, zeros elsewhere. */

#define USP_MAXSEG 4

typedef struct usp_handle usp_handle;
typedef struct usp_batch usp_batch;

/* Gas: molecular mass, viscosity law mu = mu_ref (T/T_ref)^omega (Eq. 35;
 * omega = 0.5 hard sphere, 0.81 argon), Prandtl number (2/3 monatomic).
 * mu_ref = 0 derives it from params.Kn through Eq. 36 at (n_ref, T_ref). */
typedef struct {
    double mass, T_ref, mu_ref, omega, Pr;
} usp_gas;

/* Uniform Cartesian grid.  dim = 1 resolves y only (nx ignored, x and z
 * homogeneous); dim = 2 resolves x and y (z homogeneous).  Cell index
 * iy * nx + ix.  Only hi - lo matters along an unresolved axis. */
typedef struct {
    int dim, nx, ny;
    double lo[2], hi[2];
} usp_grid;

/* Boundary of one face (order x-lo, x-hi, y-lo, y-hi): kind, wall or
 * reservoir temperature T, wall or reservoir velocity u, reservoir number
 * density n.  The normal component of a wall velocity is ignored. */
typedef struct {
    int kind;
    double T;
    double u[3];
    double n;
} usp_bc;

/* Zero-thickness plate normal to x at x = pos, spanning lo <= y <= hi
 * (the slit walls of Sec. 4.5).  dim = 2 only. */
typedef struct {
    double pos, lo, hi;
    int kind;
    double T;
    double u[3];
} usp_wall_segment;

/* Run parameters (Sec. 4, Eqs. 35-37).
 *   Kn, L_ref    : Knudsen number and its reference length (lambda_ref = Kn L_ref)
 *   n_ref        : reference number density (with gas.T_ref)
 *   dt           : time step [s]; 0 selects dt_over_tauc * tau_c(ref) (Eq. 37)
 *   body_accel   : acceleration; allowed only along unresolved axes
 *   ppc_ref      : particles per cell at n_ref (each particle stands for
 *                  n_ref V_cell / ppc_ref molecules)
 *   n_avg        : n_a of Eq. 34
 *   mode         : USP_MODE_*; fixed_pne used by USP_MODE_FIXED_PNE
 *   reservoir_cols: buffer cell layers next to each reservoir face
 *   precision    : USP_FP64 or USP_FP32_MIXED
 *   pipeline     : USP_PIPE_PLAIN or USP_PIPE_FUSED
 *   capacity_factor: particle slots allocated = factor * initial count
 *                  (>= 1; 0 selects 1.25, or 2 with reservoirs)
 *   slab_count, slab_index, slab_group: spatial decomposition (not in the
 *                  paper: how one domain is split over several devices,
 *                  exercised here inside one GPU).  slab_count > 1 makes the
 *                  handle own the rows [slab_index*ny/slab_count,
 *                  (slab_index+1)*ny/slab_count) of the grid (cells along y
 *                  in 1-D) while advection sees the whole grid and its faces.
 *                  The slabs of one domain share slab_group, are admitted to
 *                  one batch consecutively in slab_index order, and are only
 *                  stepped through that batch: particles crossing into
 *                  another slab are written into that slab's buckets, and the
 *                  Kn_GLL stencil (Eq. 18) reads the adjacent slab's row.
 *                  Requires the fused pipeline, no reservoir faces, and ny a
 *                  multiple of slab_count; 0 or 1 means no decomposition.
 *   flux_axis, flux_pos: a counting plane normal to axis x (flux_axis 1) or
 *                  y (2) at coordinate flux_pos, strictly inside the domain
 *                  along a non-periodic axis (1-D grids: y only); 0 = none.
 *                  Every advection adds +1 to counters[7] for a particle
 *                  that starts below the plane (coordinate < flux_pos) and
 *                  ends at or above it, -1 for the reverse; a particle that
 *                  leaves through a reservoir face ends at that face.  The
 *                  sum is the net number of particles through the plane,
 *                  which gives the mass flow rate of Eq. 41 (slit).
 *   gll_average  : 1 takes the Kn_GLL of Eqs. 17-18 (hence P_ne, Eq. 16)
 *                  from the Eq. 34 averaged fields n, u, T of every cell
 *                  (lambda of Eq. 36 at the averaged state) once a sample
 *                  exists -- the time averaging the paper applies to steady
 *                  flows to cut statistical noise; a cell whose averaged
 *                  state is empty has Kn_GLL = 0.  0 (default): from the
 *                  instantaneous moments of the step.
 *   selection, es_sampler: USP_SELECT_* and USP_SAMPLER_* (0, 0 = the
 *                  defaults).  With the Gallis-Torczynski sampler,
 *                  usp_get_params slots 4-9 (plain pipeline) hold
 *                  B = ((1 - Pr)/(2 Pr)) sigma* / (rho theta) (xx, yy, zz, xy,
 *                  xz, yz; S = I - s B at the time instant of Eq. 32)
 *                  instead of the Cholesky factor.  The fused pipeline takes
 *                  the same N_s particles of Eq. 9 (the smallest selection
 *                  words; ties go to the lower position in the cell's
 *                  bucket, which the arrival order sets) and scales their
 *                  time instants by the (N_s + 1)-th smallest word.
 *   weighted     : 1 runs the full USP step of Table 2 with weighted added
 *                  particles (steps 2, 4 and 7; Eqs. 22-28 and the third
 *                  term of Eq. 27): per cell N_a = N_eff min(1, nu_ES dt) /
 *                  r_p particles (rounded at random), Maxwellian, with the
 *                  weights of Eq. 26 times r_p / min(1, nu_ES dt); Eq. 28
 *                  keeps int(sum of the selected weights), rounded at random,
 *                  of the selected particles (smallest selection words) at
 *                  weight 1 and deletes the others.  Needs the plain FP64
 *                  pipeline, one domain (no slabs, no batch), no reservoir
 *                  face, the default selection and sampler (INVALID_ARG
 *                  otherwise).  Every moment is W-weighted.
 *   r_p          : the scale of Eq. 25 (> 0 when weighted; the paper's 10).
 *   weight_average: 1 feeds the weights with Eq. 34 averages (n_avg) of the
 *                  fields they are built from, the stress and heat flux
 *                  started at zero (steady flows); 0: instantaneous. */
typedef struct {
    double Kn, L_ref, n_ref;
    double dt, dt_over_tauc;
    double body_accel[3];
    int ppc_ref, n_avg, mode;
    double fixed_pne;
    int reservoir_cols;
    int precision;
    int pipeline;
    double capacity_factor;
    int slab_count, slab_index, slab_group;
    int flux_axis;
    double flux_pos;
    int gll_average;
    int selection, es_sampler;
    int weighted;
    double r_p;
    int weight_average;
} usp_params;

/* A box of initial gas at number density n, temperature T, velocity u. */
typedef struct {
    double lo[2], hi[2];
    double n, T;
    double u[3];
} usp_region;

/* Optional device allocator (for example a framework's caching allocator).
 * alloc returns a device pointer aligned to 256 bytes (as cudaMalloc's are:
 * the kernels copy particle planes in 16-byte units) or NULL; a pointer
 * with a coarser alignment is handed back to free and the call that needed
 * it fails with OOM.  NULL allocator => cudaMalloc. */
typedef struct {
    void* (*alloc)(size_t bytes, void* ctx);
    void (*free)(void* ptr, void* ctx);
    void* ctx;
} usp_allocator;

/* Read-only state of a handle. */
typedef struct {
    int64_t n_particles;  /* live particles after the last completed step */
    int64_t capacity;     /* particle slots */
    int32_t n_cells;
    int32_t precision, pipeline;
    uint32_t step;        /* completed steps */
    double dt, mu_ref;    /* derived time step and reference viscosity */
    int64_t counters[8];  /* cumulative: 0 Cholesky fallbacks, 1 bounce-cap clamps,
                             2 removed, 3 injected, 4 relaxed, 5 particles lost to
                             slot overflow (must stay 0), 6 particles spilled past
                             a full bucket (fused pipeline), 7 net particles
                             through the counting plane (signed; params.flux_axis) */
    size_t device_bytes;  /* device memory held by the handle */
    uint32_t next_pid;    /* id the next injected particle receives */
} usp_info;

/* Create a simulation.  faces[4] in order x-lo, x-hi, y-lo, y-hi; segs may be
 * NULL when nseg == 0; stream is a cudaStream_t (NULL: the handle creates
 * and owns a non-blocking stream, since steps are captured into CUDA graphs
 * and the legacy default stream cannot be captured).  Derives mu_ref (Eq. 36) and dt (Eq. 37), allocates per-cell
 * arrays; particle storage is allocated by usp_init_particles /
 * usp_set_particles.  Errors: INVALID_ARG for inconsistent input (periodic
 * on one face of an axis, resolved-axis body force, non-positive sizes, a
 * counting plane outside the domain or on a periodic axis),
 * OOM, CUDA. */
int usp_create(const usp_gas* gas, const usp_grid* grid, const usp_bc faces[4],
               const usp_wall_segment* segs, int nseg, const usp_params* params,
               const usp_allocator* allocator, void* stream, usp_handle** out);

/* Table 2 step 1: fill every cell from the region containing its centre
 * (the last listed region wins): round(n / n_ref * ppc_ref) particles with
 * uniform positions in the cell and Maxwellian velocities at (T, u);
 * particle ids 0.. in cell order; random numbers keyed by seed.  Resets the
 * step counter and the averages.  STATE for a slab of a decomposed domain
 * (slabs are loaded with usp_set_particles). */
int usp_init_particles(usp_handle* h, const usp_region* regions, int nregions, uint64_t seed);

/* Load an arbitrary state from HOST arrays: pos[n][2] (x, y; x ignored in
 * 1-D), vel[n][3], pid[n]; next_pid is the first id given to injected
 * particles (USP_NEXT_PID_AUTO: one past the largest id of pid, found on the
 * device).  Page-locked (pinned) arrays are read in place by one device pass
 * through their mapped addresses; pageable ones are copied as they are into
 * the handle's second particle buffer, which the sort fills only afterwards
 * (no staging area of its own).  Either way they are transposed into the
 * storage planes on the device; the particle storage of an earlier load of
 * a similar size is reused.  The reset of the per-cell state and the sort
 * into cells run on the handle's stream.  Returns once the arrays have been
 * read (they may be reused at once); the set-up kernels behind that point
 * are asynchronous like usp_step, and a later failure of theirs is reported
 * by the next synchronising call.  A slab keeps particles outside its rows
 * in its edge cells until they move.  Resets the step counter and the
 * averages. */
/* next_pid value of usp_set_particles: one past the largest loaded id,
 * found on the device while the ids are loaded (0 for an empty load) */
#define USP_NEXT_PID_AUTO 0xFFFFFFFFu

int usp_set_particles(usp_handle* h, int64_t n, const double* pos, const double* vel,
                      const uint32_t* pid, uint32_t next_pid, uint64_t seed);

/* Advance nsteps time steps on the handle's stream (asynchronous).  Steps
 * are replayed from a captured CUDA graph.  Returns CAPACITY if injection
 * would exceed the particle slots (checked before launching), STATE for a
 * slab of a decomposed domain (slabs step only through a batch). */
int usp_step(usp_handle* h, int nsteps);

/* Copy the USP_NFIELDS x n_cells FP64 fields ([field][cell]) into out
 * (out_len doubles; a device pointer when out_on_device != 0, else host).
 * Synchronises the handle's stream. */
int usp_sample_macro(usp_handle* h, int which, double* out, size_t out_len, int out_on_device);

/* Debug / test: copy the particles in storage order to HOST arrays (any may
 * be NULL): pos[cap][2], vel[cap][3], pid[cap], cell[cap].  *n_out receives
 * the live count; CAPACITY if cap is too small. */
int usp_get_particles(usp_handle* h, double* pos, double* vel, uint32_t* pid, int32_t* cell,
                      int64_t cap, int64_t* n_out);

/* Particle weights W (Table 2; 1 for a particle of the initial state) of a
 * handle created with params.weighted, in the storage order of
 * usp_get_particles, into the HOST array w[cap].  *n_out receives the live
 * count.  STATE for a handle without weights, INVALID_ARG if cap is too
 * small. */
int usp_get_weights(usp_handle* h, double* w, int64_t cap, int64_t* n_out);

/* Debug / test: run one stage of the plain pipeline (same stage numbers as
 * the step order above: 0 advect, 1 reservoir refill, 2 sort, 3 moments,
 * 4 parameters, 5 relaxation, 6 sample-and-advance).  A full step is the
 * stages 0..6 in order. */
int usp_run_stage(usp_handle* h, int stage);

/* Debug / test: per-cell relaxation parameters of the last step to HOST,
 * [n_cells][16]: u0 u1 u2, RT, L00 L10 L11 L20 L21 L22, P_relax, nu, nu_ES,
 * P_ne, valid, relaxed count. */
int usp_get_params(usp_handle* h, double* out, size_t out_len);

/* Debug / test: Philox4x32-10 on the device for n HOST counters ctr[n][4]
 * with key (key0, key1); words to HOST out[n][4]. */
int usp_debug_philox(int64_t n, const uint32_t* ctr, uint32_t key0, uint32_t key1, uint32_t* out);

int usp_get_info(usp_handle* h, usp_info* info);
int usp_synchronize(usp_handle* h);
int usp_destroy(usp_handle* h);
const char* usp_last_error(const usp_handle* h);
const char* usp_status_string(int status);

/* ---------------------------------------------------------------------- */
/* Batching: many independent simulations advanced by the same launches.   */
/* A batch does not own its handles.  Handles of one batch share precision */
/* and pipeline.  hbm_budget bounds the device bytes of admitted handles.  */
/* ---------------------------------------------------------------------- */
int usp_batch_create(size_t hbm_budget, int max_sims, void* stream, usp_batch** out);
/* CAPACITY when the handle does not fit the budget or the slot count. */
int usp_batch_admit(usp_batch* b, usp_handle* h);
/* Advance every admitted handle nsteps steps.  STATE when the slabs of a
 * decomposed domain are not all admitted, consecutively and in slab order. */
int usp_batch_step(usp_batch* b, int nsteps);
int usp_batch_retire(usp_batch* b, usp_handle* h);
int usp_batch_info(usp_batch* b, int* n_sims, size_t* bytes_in_use);
/* Debug / profiling: run one stage (as usp_run_stage) over every admitted
 * simulation; a full step is the stages in order. */
int usp_batch_run_stage(usp_batch* b, int stage);

/* ---------------------------------------------------------------------- */
/* Cell sort that allocates nothing.  The paper has no counterpart: this   */
/* is a library service for callers that cannot allocate device memory at  */
/* the point of the call (code inside host callbacks or custom allocators,  */
/* plug-ins whose host owns every device allocation or enforces a memory   */
/* budget, paths that must not trigger the implicit synchronisation of     */
/* cudaMalloc / cudaFree).                                                  */
/* ---------------------------------------------------------------------- */
#define USP_STATIC_MAX_CELLS (1 << 18)

/* Counting sort of n particles by cell of `grid` (same cell rule as the
 * FP64 step: floor((y - lo) / dy), and in 2-D floor((x - lo) / dx), clamped
 * to the grid).  pos: DEVICE array [n][2] of FP64 (x, y; x ignored in 1-D).
 * Outputs, DEVICE arrays owned by the caller: cell_start[K + 1] (exclusive
 * offsets, cell_start[K] = n) and perm[n] (particle indices grouped by cell;
 * the order inside a cell is the order in which atomics landed, so it can
 * differ between calls).  Work is queued on `stream` (a cudaStream_t, NULL
 * for the legacy default stream) and the call does not wait for it.
 *   - Histogram and cursors live in one file-scope device array of
 *     2 * (USP_STATIC_MAX_CELLS + 1) 32-bit words (2 MB) that every GPU
 *     loading the library holds until the process exits; the call clears
 *     it on the GPU before use and calls no cudaMalloc, cudaFree or other
 *     allocating routine.
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress, which allocates nothing), so the entry point
 *     stays valid after cudaDeviceReset; the first call on a device also
 *     loads the module there, so make that first call before any stream
 *     capture.
 *   - Every call shares the array: calls whose work overlaps on the GPU
 *     (different streams without ordering, several host threads) race and
 *     give wrong results; order them on one stream.
 * Errors: INVALID_ARG (null pointers, bad grid), CAPACITY when the grid has
 * more than USP_STATIC_MAX_CELLS cells or n > 2^31 - 1, CUDA. */
int usp_cell_sort_static(const usp_grid* grid, int64_t n, const double* pos, uint32_t* cell_start,
                         uint32_t* perm, void* stream);

/* Launch tuning (set by the autotuner, paper_1808_03801_gb300/autotune.py):
 * fused_R in {4, 8, 12} sets the fused kernels' staging capacity to 32 R
 * particles per cell pass (larger cells take two sweeps); grid_per_sm in
 * 1..32 sets the persistent blocks per SM of the tiled kernels; 0 keeps a
 * value.  A batch uses the largest values of its members.  STATE while the
 * handle is admitted to a batch. */
int usp_set_tuning(usp_handle* h, int fused_R, int grid_per_sm);
int usp_get_tuning(usp_handle* h, int* fused_R, int* grid_per_sm);

/* 1 when the library carries the fused FP32 pipeline (USP_PIPE_FUSED).  Its
 * stages for usp_run_stage / usp_batch_run_stage are 10 relaxation of the
 * previous step + advection + bucket scatter, 11 reservoir refill, 12
 * moments, 13 parameters and fields, 14 bucket layout and end of step. */
int usp_fused_supported(void);
int usp_batch_destroy(usp_batch* b);

#ifdef __cplusplus
}
#endif
#endif
