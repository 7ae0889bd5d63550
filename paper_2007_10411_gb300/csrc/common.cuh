// Device-side definitions shared by the kernels of libjfnk (sm_103a).
//
// Vectors are field-major planes [field][z][x] (x fastest), n = nf * npt
// entries.  Krylov vectors live in scaled units (every field divided by its
// scale U, U, Theta, P); the state and the Newton residual are float64 and
// unscaled.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/jfnk.h"

namespace jfnk {

constexpr int KMAX = 32;          // largest restart length the kernels are built for
constexpr int NTHREADS = 256;     // threads per block of every streaming kernel
constexpr int MAX_STREAM_BLOCKS = 2 * 152;  // streaming grid: two CTAs per SM
constexpr int MAX_DOT_BLOCKS = 3 * 152;     // Arnoldi passes A and C: three CTAs per SM
constexpr int MAX_REDUCE_BLOCKS = 8192;     // multi-dot grids grow so a thread sums <= 64 vectors' worth
constexpr int MAX_PC_SWEEPS = 64;

// Geometry and physics constants, passed by value to the stencil kernels.
struct Geo {
    int dim, nx, ny, nz, npt, nf;     // 2-D: ny = 1, nf = 4 (u, w, theta, p); 3-D: nf = 5 (u, v, w, theta, p)
    double inv_dy;
    int pb[5], pt[5];                 // mirror parity per field at bottom / top (+1 / -1)
    double inv_dx, inv_dz;
    double theta0, beta, pbar, g, gamma_p, heat_coef;   // heat_coef = 1/(rho0 cp dz)
    int smag;                         // eddy coefficients from the strain (Smagorinsky or Deardorff)
    int sgs;                          // 0 constant K, 1 Smagorinsky, 2 Deardorff (anisotropic)
    double K_M, K_H, cs2;             // cs2 = (Cs Delta)^2
    // Deardorff closure in terms of s = sqrt(2 S:S): K_m = dd_cm s, K_M = dd_cM s,
    // K_h = K_m (1 + dd_ah l), K_H = K_M (1 + dd_az l), l = min(dd_delta, dd_cl s)
    // (dd_cl < 0: l = dd_delta)
    double dd_cm, dd_cM, dd_cl, dd_delta, dd_ah, dd_az;
    // float32 derivative weights with 1/h folded in: D f = w1 (f_{+1} - f_{-1}) + w2 (f_{+2} - f_{-2})
    float fx1, fx2, fz1, fz2;
    double inv_Pr;
    double two_over_dt;
    double scale[5], inv_scale[5];
    const double* heat;               // surface flux H(x) or nullptr
    int tile_jv, tile_pc;             // tile shapes of the float32 Jv / preconditioner kernels
    int pc_schur;                     // preconditioner: 0 field-block, 1 acoustic Schur complement (2-D)
    // acoustic Schur complement constants (host-computed): Helmholtz coefficient
    // a = gamma_p pbar theta0 dt/2, c_div = gamma_p pbar (dt/2) s_u/s_p,
    // c_grad = theta0 s_p/s_u, dt/2
    double helm_a, schur_cdiv, schur_cgrad, half_dt;
    void* s3;                         // 3-D: scratch of the split stencil passes (stencil3d_scratch_bytes)
};

constexpr int NUM_TILE_SHAPES = 4;

// Solver control block in device memory.  Written by the "last block" of the
// reduction kernels, read by later kernels and, after a stream sync, by the host.
struct Ctl {
    int done;            // current GMRES cycle finished: later cycle kernels return at once
    int converged;       // |g_{j+1}| <= target (or lucky breakdown)
    int breakdown;
    int nan;
    int k;               // columns in the finished cycle
    int iters;           // Krylov iterations in this Newton solve
    int m;               // restart length
    int ncap;            // training pairs recorded for the learned preconditioner
    int eps_part;        // > 0: ||z||^2 of the last preconditioner apply is pending as that many
                         // float-float partials at the head of the partial buffer (float32 2-D
                         // field-block path); the Jacobian-product kernel forms eps from them.
                         // 0: eps_jv holds the step.  Every writer of eps_jv clears it.
    int pad_;
    double beta0;        // ||b|| of the Newton system
    double target;       // eta * beta0
    double res2;         // ||W R||^2 of the last residual evaluation
    double unorm2;       // ||W u||^2 of the same state
    double eps_mach;     // unit roundoff of the stencil precision
    double eps_jv;       // finite-difference step of the next Jacobian-vector product
    double kmax;         // max eddy coefficient K_M (preconditioner bounds)
    double gstart;       // ||r|| at the start of the current GMRES cycle
    double gres;         // rotated residual |g_{j+1}| after the latest Arnoldi step
    double scratch[8];   // misc reductions (||x||^2, ||r||^2, ...)
    double h1[KMAX + 1];      // first-projection coefficients (pass B block 0, for the Hessenberg column)
    double Hbar[KMAX + 1][KMAX];     // Hessenberg as built (row, col)
    double Rt[KMAX][KMAX];           // rotated upper-triangular factor
    double cs[KMAX], sn[KMAX];
    double g[KMAX + 1];
    double y[KMAX];
    double zscale[KMAX];      // direction k of the cycle enters the update as zscale[k] y_k z_k
                              // (1 unless the lagged second projection normalised w_k on the fly)
    // Chebyshev coefficients per field block and sweep: 1/theta_c, rho_k rho_{k-1}, 2 rho_k / delta
    double cheb[6][MAX_PC_SWEEPS][3];   // slot 5: pressure Helmholtz of the Schur complement
    unsigned int counter[8];         // last-block counters, one per kernel family
};

// Programmatic dependent launch.  Kernels of the Arnoldi step are launched
// with launch_pdl: the next kernel may be scheduled before this one has
// finished, so every such kernel calls pdl_wait() before its first global read
// (it returns once the preceding grid has completed and its writes are
// visible) and pdl_trigger() once its main loop is done (only the reduction
// tail remains), letting the successor's launch overlap that tail.  Both are
// no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

enum CounterSlot { CNT_STENCIL = 0, CNT_UPDATE, CNT_RESTART, CNT_PC, CNT_EDDY, CNT_MISC };

// ---------------------------------------------------------------- reductions
// Sum NV thread-local values over the block and store them, as float64, at
// part[k * stride + blk] (k < nv).  Deterministic (fixed shuffle tree).  The
// tree runs in the type of the thread values: float32 kernels reduce their
// float32 partials in float32 within a block (GB300's float64 rate is a small
// fraction of its float32 rate) and switch to float64 across blocks.
template <int NV, typename TA>
__device__ __forceinline__ void block_partials(const TA (&v)[NV], int nv, double* part,
                                               int stride, int blk) {
    __shared__ TA red[NV][NTHREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (k < nv) {
            TA s = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) red[k][warp] = s;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += (double)red[k][w];
        part[(size_t)k * stride + blk] = s;
        __threadfence();          // publish before the block's arrival is counted
    }
}

// Maximum that propagates NaN (fmax drops a NaN operand): a NaN in any value
// makes the reduced maximum NaN, so a diagnostic cannot report finite extrema
// for a state that holds NaN.
__device__ __forceinline__ double max_nan(double a, double b) { return (a > b || a != a) ? a : b; }

template <int NV>
__device__ __forceinline__ void block_partials_max(const double (&v)[NV], int nv, double* part,
                                                   int stride, int blk) {
    __shared__ double red[NV][NTHREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (k < nv) {
            double s = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s = max_nan(s, __shfl_down_sync(0xffffffffu, s, o));
            if (lane == 0) red[k][warp] = s;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        double s = red[k][0];
        for (int w = 1; w < nw; ++w) s = max_nan(s, red[k][w]);
        part[(size_t)k * stride + blk] = s;
        __threadfence();          // publish before the block's arrival is counted
    }
}

// Double-float addition of unevaluated float32 pairs (x = hi, y = lo): TwoSum
// of the high parts (Knuth, TAOCP vol. 2), low parts added, renormalised
// (Dekker 1971).  ~2^-44 relative rounding on the float32 pipes.
__device__ __forceinline__ float2 ff_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb);
    const float lo = e + (a.y + b.y);
    const float hi = s + lo;
    return make_float2(hi, lo - (hi - s));
}

// One float-float partial of a block's float32 values: fixed shuffle tree per
// warp, warps added in order by thread 0, stored at p[blk].
__device__ __forceinline__ void block_partial_ff(float v, float2* p, int blk) {
    __shared__ float red[NTHREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = make_float2(red[0], 0.f);
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = ff_add(t, make_float2(red[w], 0.f));
        p[blk] = t;
    }
}

// Finite-difference step of a Jacobian product: eps_jv, or, when ctl->eps_part
// > 0, eps = sqrt(eps_mach (1 + ||u||)) / ||z|| with ||z||^2 summed from the
// pending float-float partials in one fixed order (every block of the launch
// obtains bitwise the same value).  Called by all threads of the block.
__device__ __forceinline__ double pending_eps(const Ctl* ctl, const double* part) {
    __shared__ double wsum[NTHREADS / 32];
    __shared__ double eps_s;
    const int np = ctl->eps_part;
    if (np > 0) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const float2* p = reinterpret_cast<const float2*>(part);
        float2 s = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int b = threadIdx.x; b < np; b += blockDim.x) s = ff_add(s, __ldcg(p + b));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            s = ff_add(s, make_float2(__shfl_down_sync(0xffffffffu, s.x, o), __shfl_down_sync(0xffffffffu, s.y, o)));
        if (lane == 0) wsum[warp] = (double)s.x + (double)s.y;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
            const double zn = sqrt(t);
            eps_s = zn > 0.0 ? sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2))) / zn : 0.0;
        }
    } else if (threadIdx.x == 0) {
        eps_s = ctl->eps_jv;
    }
    __syncthreads();
    return eps_s;
}

// True in exactly one block: the last one to arrive.  The threads that wrote
// the block's partial sums fenced them (block_partials); the barrier orders
// those fences before thread 0's arrival.  Counters wrap to zero by
// themselves (atomicInc limit), so no reset is needed between launches.
__device__ __forceinline__ bool arrive_last(unsigned int* counter, unsigned int total) {
    __shared__ bool am_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();      // cumulative: orders the block's fenced partials before the count
        unsigned int t = atomicInc(counter, total - 1);
        am_last = (t == total - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// In the last block: out[k] = sum over blocks of part[k * nblk + b], in a fixed
// order (deterministic).  Loads are issued four at a time into independent
// accumulators so that a lane never waits on one L2 round trip per partial;
// a single value is reduced by the whole block, several values warp by warp.
template <bool MAXOP>
__device__ __forceinline__ double combine(double a, double b) { return MAXOP ? max_nan(a, b) : a + b; }

template <bool MAXOP>
__device__ __forceinline__ double strided_reduce(const double* p, int n, int start, int stride) {
    const double id = MAXOP ? -1.0e300 : 0.0;
    double s0 = id, s1 = id, s2 = id, s3 = id;
    int b = start;
    for (; b + 3 * stride < n; b += 4 * stride) {
        const double v0 = __ldcg(p + b), v1 = __ldcg(p + b + stride);
        const double v2 = __ldcg(p + b + 2 * stride), v3 = __ldcg(p + b + 3 * stride);
        s0 = combine<MAXOP>(s0, v0);
        s1 = combine<MAXOP>(s1, v1);
        s2 = combine<MAXOP>(s2, v2);
        s3 = combine<MAXOP>(s3, v3);
    }
    for (; b < n; b += stride) s0 = combine<MAXOP>(s0, __ldcg(p + b));
    return combine<MAXOP>(combine<MAXOP>(s0, s1), combine<MAXOP>(s2, s3));
}

template <bool MAXOP>
__device__ __forceinline__ double warp_reduce(double s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = combine<MAXOP>(s, __shfl_down_sync(0xffffffffu, s, o));
    return s;
}

template <bool MAXOP>
__device__ __forceinline__ void final_reduce(const double* part, int nblk, int nv, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    if (nv == 1) {
        __shared__ double red[NTHREADS / 32];
        const double s = warp_reduce<MAXOP>(strided_reduce<MAXOP>(part, nblk, threadIdx.x, blockDim.x));
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = red[0];
            for (int w = 1; w < nw; ++w) t = combine<MAXOP>(t, red[w]);
            out[0] = t;
        }
        __syncthreads();
        return;
    }
    for (int k = warp; k < nv; k += nw) {
        const double s = warp_reduce<MAXOP>(strided_reduce<MAXOP>(part + (size_t)k * nblk, nblk, lane, 32));
        if (lane == 0) out[k] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void final_sums(const double* part, int nblk, int nv, double* out) {
    final_reduce<false>(part, nblk, nv, out);
}

__device__ __forceinline__ void final_maxes(const double* part, int nblk, int nv, double* out) {
    final_reduce<true>(part, nblk, nv, out);
}

}  // namespace jfnk
