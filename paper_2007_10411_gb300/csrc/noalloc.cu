// Allocation-free variant of the budgets reduction (jfnk_budgets_static).
//
// Some callers cannot call cudaMalloc at all: code running where device
// allocation is forbidden or unsafe (inside a CUDA stream capture that must
// not allocate, under an allocator that owns all device memory, or in a
// long-running service with a fixed memory budget).  jfnk_budgets needs a
// handle, and jfnk_create allocates the workspace.  This entry point needs
// no handle: the inputs and outputs belong to the caller, and the only scratch
// it uses -- one float64 partial sum per block and value, plus the
// last-block counter -- lives in a file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

namespace jfnk {
namespace {

constexpr int SB_VALUES = 12;                        // E_k, E_p, sum theta, sum div, max[4], -min[4]
constexpr int SB_POINTS_PER_BLOCK = NTHREADS * 8;    // a thread reduces at most 8 points
constexpr int SB_MAX_BLOCKS = JFNK_BUDGETS_STATIC_MAX_POINTS / SB_POINTS_PER_BLOCK;
constexpr size_t SB_PART_DOUBLES = (size_t)SB_VALUES * SB_MAX_BLOCKS;

// Scratch shared by every call on a device: partial sums, then the counter.
struct StaticScratch {
    double part[SB_PART_DOUBLES];
    unsigned int counter;
};
static __device__ __align__(256) StaticScratch g_budget_scratch;

__device__ __forceinline__ int sb_mirror_z(int gz, int nz, int& side) {
    side = 0;
    if (gz < 0) { side = 1; return -1 - gz; }
    if (gz >= nz) { side = 2; return 2 * nz - 1 - gz; }
    return gz;
}

__device__ __forceinline__ int sb_wrap_x(int gx, int nx) {
    int r = gx % nx;
    return r < 0 ? r + nx : r;
}

// Same quantities as the handle-based budgets kernel, one block per
// SB_POINTS_PER_BLOCK points; scratch passed in as a device address.
__global__ void __launch_bounds__(NTHREADS)
budgets_static_k(int nx, int nz, double inv_dx, double inv_dz, double dV,
                 double dz, double lz, const double* __restrict__ u, double* part,
                 unsigned int* counter, double* __restrict__ out) {
    const int npt = nx * nz;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    double mx[8];
    for (int f = 0; f < 8; ++f) mx[f] = -1e300;
    const double* U = u;
    const double* W = u + npt;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npt; p += gridDim.x * blockDim.x) {
        const int z = p / nx, x = p - z * nx;
        const double zc = (z + 0.5) * dz;
        s[0] += 0.5 * (U[p] * U[p] + W[p] * W[p]);
        s[1] += (lz - zc) * u[2 * npt + p];
        s[2] += u[2 * npt + p];
        double ux = 0.0, wz = 0.0;
        for (int l = 1; l <= 2; ++l) {
            const double c = l == 1 ? 2.0 / 3.0 : -1.0 / 12.0;
            ux += c * (U[z * nx + sb_wrap_x(x + l, nx)] - U[z * nx + sb_wrap_x(x - l, nx)]);
            int sp_, sm_;
            const int zp = sb_mirror_z(z + l, nz, sp_), zm = sb_mirror_z(z - l, nz, sm_);
            const double gp = sp_ == 2 ? -1.0 : 1.0, gm = sm_ == 1 ? -1.0 : 1.0;   // w is odd at both walls
            wz += c * (gp * W[zp * nx + x] - gm * W[zm * nx + x]);
        }
        s[3] += ux * inv_dx + wz * inv_dz;
        for (int f = 0; f < 4; ++f) {
            const double v = u[(size_t)f * npt + p];
            mx[f] = max_nan(mx[f], v);
            mx[4 + f] = max_nan(mx[4 + f], -v);
        }
    }
    double* pmax = part + 4 * gridDim.x;
    block_partials<4>(s, 4, part, gridDim.x, blockIdx.x);
    block_partials_max<8>(mx, 8, pmax, gridDim.x, blockIdx.x);
    if (arrive_last(counter, gridDim.x)) {
        __shared__ double tot[12];
        final_sums(part, gridDim.x, 4, tot);
        final_maxes(pmax, gridDim.x, 8, tot + 4);
        if (threadIdx.x == 0) {
            for (int i = 0; i < 4; ++i) out[i] = tot[i] * dV;
            for (int f = 0; f < 4; ++f) { out[4 + f] = tot[4 + f]; out[8 + f] = -tot[8 + f]; }
        }
    }
}

// Device address of the scratch array.  A __device__ symbol's address belongs
// to a CUDA context, not to a device: it changes when the primary context is
// reset (cudaDeviceReset) and differs in any other context a caller makes
// current.  The cache is therefore keyed on the context's process-unique id
// (cuCtxGetId: a reset context comes back with a new id), and it is filled
// under a mutex so that several host threads may make their first call at
// once.  The two driver calls are reached through the runtime's driver entry
// points, so the library does not link libcuda itself.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

constexpr int SB_CACHE = 16;
struct ScratchSlot {
    unsigned long long ctx_id;
    StaticScratch* addr;
};
ScratchSlot g_slots[SB_CACHE];
int g_nslots = 0, g_next_evict = 0;
std::mutex g_slot_mutex;
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;

cudaError_t driver_entry_points() {
    if (g_ctx_get_current && g_ctx_get_id) return cudaSuccess;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess) return e;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return e;
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
        return cudaErrorNotSupported;
    g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
    g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(f2);
    return cudaSuccess;
}

// Id of the context current on this thread; 0 when none is current yet.
cudaError_t current_context_id(unsigned long long* id) {
    *id = 0;
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    if (ctx == nullptr) return cudaSuccess;
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

cudaError_t scratch_for_current_context(StaticScratch** out) {
    std::lock_guard<std::mutex> lock(g_slot_mutex);
    cudaError_t e = driver_entry_points();
    if (e != cudaSuccess) return e;
    unsigned long long id = 0;
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    if (id != 0)
        for (int i = 0; i < g_nslots; ++i)
            if (g_slots[i].ctx_id == id) {
                *out = g_slots[i].addr;
                return cudaSuccess;
            }
    // first call in this context: the lookup makes the runtime's context
    // current when none was (the device's primary context)
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_budget_scratch);
    if (e != cudaSuccess) return e;
    if (id == 0) {
        e = current_context_id(&id);
        if (e != cudaSuccess) return e;
        if (id == 0) return cudaErrorDeviceUninitialized;
    }
    int slot = g_nslots < SB_CACHE ? g_nslots++ : g_next_evict++ % SB_CACHE;
    g_slots[slot].ctx_id = id;
    g_slots[slot].addr = static_cast<StaticScratch*>(ptr);
    *out = g_slots[slot].addr;
    return cudaSuccess;
}

}  // namespace
}  // namespace jfnk

extern "C" jfnk_status jfnk_budgets_static(const jfnk_grid* grid, const double* u, double* out,
                                           void* cuda_stream) {
    using namespace jfnk;
    if (!grid || !u || !out) return JFNK_ERR_INVALID_ARG;
    if (grid->dim != 2) return grid->dim == 3 ? JFNK_ERR_UNSUPPORTED : JFNK_ERR_INVALID_ARG;
    if (grid->nx < 1 || grid->nz < 4 || !(grid->lx > 0.0) || !(grid->lz > 0.0) ||
        (grid->bc_bottom != JFNK_FREESLIP && grid->bc_bottom != JFNK_NOSLIP) ||
        (grid->bc_top != JFNK_FREESLIP && grid->bc_top != JFNK_NOSLIP))
        return JFNK_ERR_INVALID_ARG;
    const long long npt = (long long)grid->nx * grid->nz;
    const long long blocks = (npt + SB_POINTS_PER_BLOCK - 1) / SB_POINTS_PER_BLOCK;
    if (npt > JFNK_BUDGETS_STATIC_MAX_POINTS || blocks > SB_MAX_BLOCKS) return JFNK_ERR_INVALID_ARG;
    StaticScratch* scratch = nullptr;
    if (scratch_for_current_context(&scratch) != cudaSuccess) return JFNK_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the counter must start at zero; the partial sums are fully overwritten
    if (cudaMemsetAsync(&scratch->counter, 0, sizeof(unsigned int), s) != cudaSuccess) return JFNK_ERR_CUDA;
    const double dx = grid->lx / grid->nx, dz = grid->lz / grid->nz;
    budgets_static_k<<<(int)blocks, NTHREADS, 0, s>>>(grid->nx, grid->nz, 1.0 / dx, 1.0 / dz, dx * dz,
                                                      dz, grid->lz, u, scratch->part,
                                                      &scratch->counter, out);
    return cudaGetLastError() == cudaSuccess ? JFNK_OK : JFNK_ERR_CUDA;
}
