// usp_internal.cuh -- device-side state and helpers shared by the kernels and
// the host API of the USP-ESBGK library.  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace usp {

constexpr int kMaxSeg = 4;
constexpr int kNFields = 16;
constexpr int kNMom = 13;     // N, S1[3], S2[6], S3[3] (sums of shifted velocities)
constexpr int kNPrm = 16;     // u[3], theta, L[6], P_relax, nu, nu_ES, P_ne, valid, relaxed
constexpr int kMaxBounce = 8; // wall interactions per particle per step
constexpr double kBoltzmann = 1.380649e-23;   // J/K (exact SI value)
constexpr double kPi = 3.14159265358979323846;
constexpr double kKnC = 0.1;                    // Kn_c of Eq. 16
constexpr double kGammaMono = 5.0 / 3.0;

// Philox purposes (third counter word); the first two words are (pid, step).
enum : uint32_t { kInit = 0, kRelax = 1, kWall = 2, kInject = 3, kAdd = 4, kCellDraw = 5 };
enum { kBcDiffuse = 0, kBcSpecular = 1, kBcPeriodic = 2, kBcReservoir = 3 };
enum { kModeUSP = 0, kModeSP = 1, kModeFixed = 2, kModeSPESBGK = 3 };

// counters (u64, device)
enum { kCntChol = 0, kCntClamp = 1, kCntRemoved = 2, kCntInjected = 3, kCntRelaxed = 4, kCntOverflow = 5,
       kCntSpilled = 6, kCntFlux = 7 };

struct FaceDev {
    int kind;
    double T, theta, sqrt_theta;   // wall temperature and R T
    double u[3];
};

struct SegDev {
    double pos, lo, hi;
    int kind;
    double theta, sqrt_theta;
    double u[3];
};

// Mutable per-simulation state, kept on the device so that captured graphs
// stay valid from step to step.
struct SimDyn {
    uint32_t step;      // index n of the step being taken (Philox counter word 1)
    uint32_t n;         // live particles in buffer `cur`
    uint32_t next_pid;  // first id of the next injected particle
    uint32_t nsamples;  // samples folded into the Eq. 34 average
    int cur;            // buffer holding the current state
    int relax_pending;  // fused pipeline: the relaxation of the last step is still to be applied
    uint32_t sp_n[2];   // fused pipeline: entries in the spill lists
    uint32_t qnext;     // fused pipeline: next cell handed out by k_g2 (zero between launches)
    uint32_t lay_dst;   // fused pipeline: buffer whose bucket layout the layout kernels build
    uint32_t w_started; // weighted particles: bit 0 / 1, the step-2 / step-4,7 weight-field averages exist
    uint32_t w_added;   // weighted particles: particles added by the current stage
    unsigned long long counters[8];
};

// Everything a kernel needs to know about one simulation.  Lives in device
// memory (one entry per simulation of a batch); kernels stage it in shared
// memory so that its fields stay cheap to read next to global stores.
struct alignas(16) SimDev {
    int dim, nx, ny, K;
    double lo[2], hi[2], dx, dy;
    FaceDev face[4];
    int nseg;
    SegDev seg[kMaxSeg];
    int periodic_x, periodic_y;
    int has_reservoir, reservoir_cols;
    double R, mass, mu_ref, T_ref, omega, Pr, dt, w;   // w: number density carried by one particle
    double avg_keep, avg_new;                          // (n_a - 1)/n_a, 1/n_a
    double inv_R, es_b;                                // 1/R and 1 - 1/Pr (Eq. 6c), set on the host
    // spatial decomposition: this handle owns rows [row0, row0 + rows) of the
    // grid above (K = nx * rows cells, local index = global - row0 * nx);
    // slab_first is the batch index of slab 0 (-1 outside a batch)
    int slab_count, slab_index, slab_first, row0, rows;
    // single-precision copies for the FP32 kernels (set on the host)
    float f_dt, f_lo[2], f_hi[2], f_inv_dx, f_inv_dy, f_bdt[3], f_w, f_inv_R, f_flux_pos;
    int mode;
    double fixed_pne;
    // counting plane of the mass flow (Eq. 41): normal to x (1) or y (2) at
    // flux_pos; 0 = none
    int flux_axis;
    double flux_pos;
    int gll_average;      // Kn_GLL from the Eq. 34 averages once a sample exists
    int selection;        // 1: fixed count of Eq. 9 (plain pipeline)
    int es_sampler;       // 1: Gallis-Torczynski, Eqs. 10-11 (plain pipeline)
    double body[3];
    uint32_t key0, key1;
    int64_t cap;
    // storage: [buffer][plane]; 1-D uses plane 1 of pos only
    void* pos[2][2];
    void* vel[2][3];
    uint32_t* pid[2];
    uint32_t* cell;       // per-slot cell id (plain pipeline)
    uint32_t* count;      // K + 1 (sentinel K = removed)
    uint32_t* start;      // K + 2
    uint32_t* fill;       // K + 1
    double* mom;          // kNMom x K
    double* prm;          // kNPrm x K
    double* inst;         // kNFields x K
    double* avg;          // kNFields x K
    double* ushift;       // 3 x K, previous mean velocity (shift of the sums)
    double* gavg;         // 3 x K, averaged n, T, |u| at the start of the step (plain pipeline, gll_average)
    double* gloc;         // 6 x K, each cell's stencil state (valid, n, T, |u|, a, lambda) of this step (plain)
    uint32_t* inj_count;  // K (buffer cells only)
    uint32_t* inj_pidoff; // K
    uint32_t inj_total;
    // fused pipeline (FP32 storage): slack-bucket layout per buffer parity
    uint32_t* lay[2];     // K + 1 bucket offsets of buffer b
    uint32_t* cnt[2];     // K arrivals into buffer b (bucket + spilled)
    unsigned long long* lay_part;   // 3 per kLayTile-cell tile + 2: tile sums, then tile offsets (layout kernels)
    float* sp_pos[2][2];  // spill lists (kSpillCap entries) per parity
    float* sp_vel[2][3];
    uint32_t* sp_pid[2];
    uint32_t* sp_cell[2];
    float* fprm;          // [K][kNFPrm] relaxation parameters in FP32 (one 64-byte record per cell)
    float* momf;          // [K][16]: N, 12 sums of C = c - u_s, the shift u_s[3]  (fused moments)
    float* floc;          // [K][4]: n, T, |u|, valid of each cell for the Kn_GLL stencil
    // weighted added particles (Table 2 steps 2, 4, 7; plain FP64 pipeline)
    int weighted, weight_average;
    double r_p;           // scale of Eq. 25
    double* wgt[2];       // particle weights per buffer
    double* wneff;        // K: sum of the weights in each cell (N_eff)
    double* wst;          // 9 x K: sigma* (6) and q* (3) per unit density (Eq. 33)
    double* wfs;          // kNWF x K: the weight fields of steps 4 and 7 as used
    double* wan;          // kNWF x K: Eq. 34 average of the step-2 weight fields
    double* was;          // kNWF x K: Eq. 34 average of the step-4/7 weight fields
    uint32_t* wna;        // K: particles added to each cell by the current stage
    uint32_t* woff;       // K + 1: their exclusive offsets
    SimDyn* dyn;
};

// fields behind the weights of Eq. 26: u[3], theta, sigma[6] and q[3] per
// unit density, nu, and the stage's pref (r_p / min(1, nu_ES dt)) and P_ne
constexpr int kNWF = 16;
enum { kWFU = 0, kWFTh = 3, kWFSig = 4, kWFQ = 10, kWFNu = 13, kWFPref = 14, kWFPne = 15 };

// copy one simulation descriptor into shared memory (whole block)
__device__ __forceinline__ void load_sim(SimDev& dst, const SimDev& src) {
    const int4* a = reinterpret_cast<const int4*>(&src);
    int4* b = reinterpret_cast<int4*>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(SimDev) / 16); i += blockDim.x) b[i] = a[i];
}

// -------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32->64-bit products and a key bump by the Weyl constants.
// -------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32 -> 64-bit product per half (a single wide multiply-add)
        const uint64_t p0 = (uint64_t)M0 * c.x;
        const uint64_t p1 = (uint64_t)M1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y, (uint32_t)p0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

__device__ __forceinline__ uint4 draw(const SimDev& s, uint32_t pid, uint32_t step, uint32_t purpose, uint32_t k) {
    return philox(make_uint4(pid, step, purpose, k), make_uint2(s.key0, s.key1));
}

// Uniform variates on the open interval (0, 1).
// FP64: (x + 1/2) 2^-32, exact.  FP32: (2 (x >> 9) + 1) 2^-24, exact in float.
template <class T> __device__ __forceinline__ T u01(uint32_t x);
template <> __device__ __forceinline__ double u01<double>(uint32_t x) {
    return fma((double)x, 2.3283064365386963e-10, 1.1641532182693481e-10);
}
template <> __device__ __forceinline__ float u01<float>(uint32_t x) {
    // 1 + k 2^-23 built from the bits, minus (1 - 2^-24): exactly k 2^-23 + 2^-24
    return __uint_as_float(0x3F800000u | (x >> 9)) - 0.99999994039535522f;
}

// Box-Muller pair from two words.
template <class T> __device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, T& z0, T& z1);
template <> __device__ __forceinline__ void box_muller<double>(uint32_t a, uint32_t b, double& z0, double& z1) {
    double r = sqrt(-2.0 * log(u01<double>(a)));
    double sn, cs;
    sincospi(2.0 * u01<double>(b), &sn, &cs);
    z0 = r * cs;
    z1 = r * sn;
}
template <> __device__ __forceinline__ void box_muller<float>(uint32_t a, uint32_t b, float& z0, float& z1) {
    // -2 ln u = -2 ln2 * log2(u); the angle is shifted by pi, which flips the
    // sign of both normals and leaves their joint law unchanged.
    float r = sqrtf(-1.3862943611198906f * __log2f(u01<float>(a)));
    float sn, cs;
    __sincosf(6.283185307179586f * u01<float>(b) - 3.14159265358979f, &sn, &cs);
    z0 = r * cs;
    z1 = r * sn;
}

template <class T> __device__ __forceinline__ T dev_sqrt(T x);
template <> __device__ __forceinline__ double dev_sqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float dev_sqrt<float>(float x) { return sqrtf(x); }
template <class T> __device__ __forceinline__ T dev_log(T x);
template <> __device__ __forceinline__ double dev_log<double>(double x) { return log(x); }
template <> __device__ __forceinline__ float dev_log<float>(float x) { return 0.6931471805599453f * __log2f(x); }
template <class T> __device__ __forceinline__ T dev_floor(T x);
template <> __device__ __forceinline__ double dev_floor<double>(double x) { return floor(x); }
template <> __device__ __forceinline__ float dev_floor<float>(float x) { return floorf(x); }

// -------------------------------------------------------------------------
// launch helpers (defined in usp_kernels.cu)
// -------------------------------------------------------------------------
struct Launch {
    const SimDev* sims;   // device array
    const int2* ptiles;   // (sim, first particle slot) tiles
    const int* nptiles;   // device scalar
    const int2* ctiles;   // (sim, first cell) tiles
    const int* nctiles;   // device scalar
    uint32_t* wq;         // k_g2: warps done (2 words, zero between launches)
    int nsims;
    int dims;             // bit 0: some simulation is 1-D, bit 1: some is 2-D
    int slabs = 0;        // some simulation is a slab of a decomposed domain
    int flux = 0;         // some simulation counts particles through a plane
    int grid_p, grid_c;   // persistent grid sizes
    int lay_tiles = 1;    // layout tiles (kLayTile cells) of the largest simulation
    cudaStream_t stream;
    // fused step: a second stream and two events let the layout kernels run
    // beside k_g1 and k_params_f (null: one stream)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

constexpr int kPTile = 512;   // particles per tile (small domains still spread over many SMs)
constexpr int kCTile = 32;    // cells per tile (balances the per-cell kernels across SMs)
constexpr int kSpillCap = 4096;  // spill entries per parity (fused pipeline)
constexpr int kNFPrm = 16;       // u[3], theta, L[6], P_relax, nu, nu_ES, P_ne, valid, spare
constexpr int kLayTile = 1024;   // cells per block of the layout kernels (fused pipeline)

void launch_stream(const Launch& L, bool fp64);
void enqueue_weighted_step(const Launch& L);
void launch_scan(const Launch& L, bool with_inj = true);
void launch_scatter(const Launch& L, bool fp64);
void launch_inject(const Launch& L, bool fp64);
void launch_moments(const Launch& L, bool fp64);
void launch_moments_src(const Launch& L, bool fp64, bool src_cur);
void launch_weighted_init(const Launch& L);
void launch_params(const Launch& L);
void launch_relax(const Launch& L, bool fp64);
void launch_finish(const Launch& L);
void launch_init(const Launch& L, bool fp64, const double* reg_theta, const double* reg_u, const int* cell_reg);
void launch_assign(const Launch& L, bool fp64);
void launch_unpack(const SimDev& s, bool fp64, const double* pos, const double* vel, const uint32_t* ids,
                   bool ids_to_plane, uint32_t* next_pid, int64_t n, cudaStream_t st);
constexpr int kZeroRanges = 8;
struct ZeroList {   // device ranges of 32-bit words to clear
    void* p[kZeroRanges];
    size_t words[kZeroRanges];
    int n;
};
void launch_zero(const ZeroList& z, cudaStream_t st);
// fused FP32 pipeline (usp_fused.cu); R = particles per lane held in registers
void launch_fused_setup(const Launch& L);
void launch_fused_relax_stream(const Launch& L, int R, bool flush_only);
void launch_fused_inject(const Launch& L);
void launch_fused_moments(const Launch& L, int R);
void launch_fused_params(const Launch& L);
void launch_fused_layout(const Launch& L);
void launch_fused_layout_parts(const Launch& L);
void launch_fused_step_end(const Launch& L);
void fused_prepare_attributes();
cudaError_t debug_philox(int64_t n, const uint32_t* d_ctr, uint32_t k0, uint32_t k1, uint32_t* d_out, cudaStream_t st);

}  // namespace usp
