// usp_static.cu -- counting sort of particles by cell that allocates no device
// memory.
//
// Some callers cannot call cudaMalloc at the point where they need the sort:
// code running inside a host callback or a custom allocator, plug-ins whose
// host application owns every device allocation (a fixed memory pool or a
// budget it enforces), and code paths that must not trigger an implicit
// device synchronisation.  For them, the histogram and the insertion cursors
// of the sort live in a file-scope device array of fixed size instead of
// handle-owned memory.  The caller still passes the positions and receives
// the cell offsets and the permutation in its own buffers.
#include "usp.h"
#include "usp_internal.cuh"

#include <algorithm>

namespace {

// counts[0..K] followed by cursors[0..K]; every GPU that loads the library
// holds these 2 MB until the process exits
static __device__ __align__(256) uint32_t g_sort_scratch[2 * (USP_STATIC_MAX_CELLS + 1)];


struct GridF64 {
    int dim, nx, ny, K;
    double lo0, lo1, dx, dy;
};

// same cell rule as the FP64 step: floor of the offset over the cell size,
// clamped to the grid
__device__ __forceinline__ uint32_t cell_of(const GridF64& g, double x, double y) {
    double fy = floor((y - g.lo1) / g.dy);
    fy = fy < 0.0 ? 0.0 : (fy > (double)(g.ny - 1) ? (double)(g.ny - 1) : fy);
    if (g.dim == 1) return (uint32_t)fy;
    double fx = floor((x - g.lo0) / g.dx);
    fx = fx < 0.0 ? 0.0 : (fx > (double)(g.nx - 1) ? (double)(g.nx - 1) : fx);
    return (uint32_t)fy * (uint32_t)g.nx + (uint32_t)fx;
}

__global__ void k_static_zero(uint32_t* scratch, int K) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * (K + 1); i += gridDim.x * blockDim.x) scratch[i] = 0;
}

__global__ void k_static_count(GridF64 g, int64_t n, const double* __restrict__ pos, uint32_t* scratch) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&scratch[cell_of(g, pos[2 * i], pos[2 * i + 1])], 1u);
}

__global__ void __launch_bounds__(1024) k_static_scan(int K, const uint32_t* __restrict__ scratch,
                                                      uint32_t* __restrict__ start) {
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < K; base += blockDim.x) {
        const int c = base + threadIdx.x;
        const uint32_t v = c < K ? scratch[c] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= o) x += y;
        }
        if ((threadIdx.x & 31) == 31) warp_sums[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t ws = threadIdx.x < (blockDim.x >> 5) ? warp_sums[threadIdx.x] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, ws, o);
                if (threadIdx.x >= o) ws += y;
            }
            warp_sums[threadIdx.x] = ws;
        }
        __syncthreads();
        const uint32_t before = (threadIdx.x >= 32 ? warp_sums[(threadIdx.x >> 5) - 1] : 0u) + carry;
        if (c < K) start[c] = before + x - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + x;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[K] = carry;
}

__global__ void k_static_scatter(GridF64 g, int64_t n, const double* __restrict__ pos,
                                 const uint32_t* __restrict__ start, uint32_t* scratch, uint32_t* __restrict__ perm) {
    uint32_t* cursor = scratch + (g.K + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = cell_of(g, pos[2 * i], pos[2 * i + 1]);
        perm[start[c] + atomicAdd(&cursor[c], 1u)] = (uint32_t)i;
    }
}

// device address of the scratch array on the current device.  Looked up on
// every call (the lookup allocates nothing): a cached address would dangle
// after cudaDeviceReset, which unloads the module and places the array anew
// on the next use.
int scratch_address(uint32_t** out) {
    uint32_t* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_sort_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return USP_ERR_CUDA;
    }
    *out = p;
    return USP_OK;
}

}  // namespace

extern "C" int usp_cell_sort_static(const usp_grid* grid, int64_t n, const double* pos, uint32_t* cell_start,
                                    uint32_t* perm, void* stream) {
    if (!grid || n < 0 || !cell_start || (n > 0 && (!pos || !perm))) return USP_ERR_INVALID_ARG;
    if (grid->dim != 1 && grid->dim != 2) return USP_ERR_INVALID_ARG;
    const int nx = grid->dim == 1 ? 1 : grid->nx;
    if (nx < 1 || grid->ny < 1) return USP_ERR_INVALID_ARG;
    if ((int64_t)nx * grid->ny > USP_STATIC_MAX_CELLS) return USP_ERR_CAPACITY;
    if (n > (int64_t)0x7FFFFFFF) return USP_ERR_CAPACITY;
    if (!(grid->hi[1] > grid->lo[1]) || (grid->dim == 2 && !(grid->hi[0] > grid->lo[0]))) return USP_ERR_INVALID_ARG;
    uint32_t* scratch = nullptr;
    if (int rc = scratch_address(&scratch)) return rc;
    GridF64 g;
    g.dim = grid->dim;
    g.nx = nx;
    g.ny = grid->ny;
    g.K = nx * grid->ny;
    g.lo0 = grid->lo[0];
    g.lo1 = grid->lo[1];
    g.dx = grid->dim == 2 ? (grid->hi[0] - grid->lo[0]) / nx : 1.0;
    g.dy = (grid->hi[1] - grid->lo[1]) / grid->ny;
    cudaStream_t st = (cudaStream_t)stream;
    const int blocks = (int)std::min<int64_t>(4096, std::max<int64_t>(1, (n + 255) / 256));
    k_static_zero<<<std::max(1, std::min(1024, (2 * (g.K + 1) + 255) / 256)), 256, 0, st>>>(scratch, g.K);
    if (n > 0) k_static_count<<<blocks, 256, 0, st>>>(g, n, pos, scratch);
    k_static_scan<<<1, 1024, 0, st>>>(g.K, scratch, cell_start);
    if (n > 0) k_static_scatter<<<blocks, 256, 0, st>>>(g, n, pos, cell_start, scratch, perm);
    return cudaGetLastError() == cudaSuccess ? USP_OK : USP_ERR_CUDA;
}
