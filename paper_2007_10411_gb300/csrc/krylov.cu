// Krylov kernels of libjfnk: restarted GMRES(m) with right preconditioning in
// the flexible (stored z_j) form, classical Gram-Schmidt applied twice.
//
// One Arnoldi step j (w = J z_j already formed) is three streaming passes over
// the basis V = [v_0 .. v_j]:
//   A:  h1 = V^T w                                  (multi-dot)
//   B:  w' = w - V h1 (stored over w),  h2 = V^T w',  ||w'||^2
//   C:  v_{j+1} = (w' - V h2) / h_{j+1,j},  h_{j+1,j} = sqrt(||w'||^2 - ||h2||^2)
//       (multi-axpy + scale); one extra block of the same launch forms the
//       Hessenberg column h = h1 + h2, applies the Givens rotations, updates
//       the residual estimate |g_{j+1}|, takes the stopping test and (when
//       the cycle ends) solves the triangular system for y
// The second projection is subtracted from the stored w', as in classical
// Gram-Schmidt applied twice: the rounding of w - V h1 is then part of what
// h2 removes, and the last rounding is relative to ||w'||, not ||w||.
// Reductions are two-stage and deterministic: every block of a pass writes
// its partial sums, and every block of the NEXT pass adds all of them in one
// fixed order (grid_sums), so that no pass ends in a serial last-block tail
// and all blocks hold bitwise the same coefficients.  A thread accumulates
// its partial dot products in the basis precision over at most 64 vector
// elements (the grid grows with n), then the block and grid sums run in
// float64.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace jfnk {

constexpr int PER_THREAD = 64;   // vector loads (of one basis vector) a multi-dot thread accumulates

template <typename T> struct V4;
template <> struct V4<float> { using type = float4; static constexpr int W = 4; };
template <> struct V4<double> { using type = double2; static constexpr int W = 2; };

__device__ __forceinline__ float dotv(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ double dotv(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ float4 axpyv(float4 y, float a, float4 x) {
    return make_float4(y.x - a * x.x, y.y - a * x.y, y.z - a * x.z, y.w - a * x.w);
}
__device__ __forceinline__ double2 axpyv(double2 y, double a, double2 x) {
    return make_double2(y.x - a * x.x, y.y - a * x.y);
}
__device__ __forceinline__ float4 scalev(float4 x, float a) { return make_float4(a * x.x, a * x.y, a * x.z, a * x.w); }
__device__ __forceinline__ double2 scalev(double2 x, double a) { return make_double2(a * x.x, a * x.y); }

__device__ __forceinline__ float4 reload(const float4* p) {
    float4 r;
    asm volatile("ld.global.ca.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ double2 reload(const double2* p) {
    double2 r;
    asm volatile("ld.global.ca.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
    return r;
}

// Field of vector entry i (planes of npt entries); 32-bit division where it fits.
__device__ __forceinline__ int field_of(size_t i, int npt) {
    return i <= 0xffffffffull ? (int)((unsigned)i / (unsigned)npt) : (int)(i / (size_t)npt);
}

// Order in which a grid-stride loop visits its elements.  The Arnoldi passes
// alternate direction (A and C backwards on odd j + 1, B backwards on even):
// each pass then starts on the basis lines the previous pass touched last,
// which the 129 MB L2 still holds, instead of on the ones it evicted first.
// A thread visits the same elements either way (only their order changes).
struct Walk {
    size_t first, stride, cnt;
    bool rev;
    __device__ __forceinline__ size_t at(size_t c) const { return first + (rev ? cnt - 1 - c : c) * stride; }
};
__device__ __forceinline__ Walk make_walk(size_t first, size_t stride, size_t n, bool rev) {
    Walk w;
    w.first = first;
    w.stride = stride;
    w.cnt = first < n ? (n - 1 - first) / stride + 1 : 0;
    w.rev = rev;
    return w;
}

static int stream_blocks(size_t n) {
    size_t b = (n + NTHREADS - 1) / NTHREADS;
    return (int)(b < (size_t)MAX_STREAM_BLOCKS ? (b > 0 ? b : 1) : MAX_STREAM_BLOCKS);
}

// Grid of the multi-dot kernels: >= two CTAs per SM, and enough CTAs that no
// thread accumulates more than PER_THREAD vector elements in low precision.
// Grid of Arnoldi passes A and C (register use fits three CTAs per SM).
static int dot_blocks(size_t nvec) {
    size_t b = (nvec + NTHREADS - 1) / NTHREADS;
    return (int)(b < (size_t)MAX_DOT_BLOCKS ? (b > 0 ? b : 1) : MAX_DOT_BLOCKS);
}

static int reduce_blocks(size_t nvec) {
    size_t b = (nvec + (size_t)NTHREADS * PER_THREAD - 1) / ((size_t)NTHREADS * PER_THREAD);
    if (b < (size_t)MAX_STREAM_BLOCKS) return stream_blocks(nvec);
    return (int)(b < (size_t)MAX_REDUCE_BLOCKS ? b : MAX_REDUCE_BLOCKS);
}

// Partial sums of the Arnoldi passes.  A float64 basis keeps float64
// partials.  A float32 basis keeps each partial as an unevaluated pair of
// float32 numbers hi + lo (double-float: Dekker 1971; TwoSum: Knuth, TAOCP
// vol. 2), so that the grid-level sums, which every block of the next pass
// repeats, run on the float32 pipes (GB300's float64 rate is a small
// fraction of its float32 rate) with ~2^-44 relative rounding per addition.
template <typename T> struct PartOf;
template <> struct PartOf<float> { using type = float2; };     // x = hi, y = lo
template <> struct PartOf<double> { using type = double; };

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return ff_add(a, b); }
__device__ __forceinline__ double padd(double a, double b) { return a + b; }
__device__ __forceinline__ double pval(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ double pval(double a) { return a; }
__device__ __forceinline__ void pset(float2& p, float v) { p = make_float2(v, 0.f); }
__device__ __forceinline__ void pset(double& p, double v) { p = v; }
__device__ __forceinline__ float2 pzero(float2) { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double pzero(double) { return 0.0; }
__device__ __forceinline__ float2 pshfl_down(float2 a, int o) {
    return make_float2(__shfl_down_sync(0xffffffffu, a.x, o), __shfl_down_sync(0xffffffffu, a.y, o));
}
__device__ __forceinline__ double pshfl_down(double a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
__device__ __forceinline__ float2 pload(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ double pload(const double* p) { return __ldcg(p); }

// Block partial of NV per-warp sums red[k][w] (k < nv) into part[k * stride + blk].
template <typename T, int NV, typename P>
__device__ __forceinline__ void store_partials(const T (*red)[NTHREADS / 32], int nv, P* part, int stride, int blk) {
    const int nw = blockDim.x >> 5;
    for (int k = threadIdx.x; k < nv; k += blockDim.x) {
        P t;
        pset(t, red[k][0]);
        for (int ww = 1; ww < nw; ++ww) {
            P u;
            pset(u, red[k][ww]);
            t = padd(t, u);
        }
        part[(size_t)k * stride + blk] = t;
    }
}

// Every block: out[k] = sum over b < nblk of part[k * nblk + b], k < nv, in one
// fixed order, so all blocks of a launch obtain bitwise the same sums.  Warp w
// takes the values w, w + nw (together), w + 2 nw, ...; a lane adds
// b = lane + 32 r with all its loads of a 512-block chunk in flight, then a
// fixed tree over r and a fixed shuffle tree over the lanes.
template <typename P>
__device__ __forceinline__ P chunk_sum(const P* p, int nblk, int b0, int lane) {
    P v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
        const int b = b0 + lane + 32 * r;
        v[r] = b < nblk ? pload(p + b) : pzero(P());
    }
#pragma unroll
    for (int h = 8; h > 0; h >>= 1)
#pragma unroll
        for (int r = 0; r < h; ++r) v[r] = padd(v[r], v[r + h]);
    return v[0];
}

template <typename P, typename TO>
__device__ void grid_sums(const P* part, int nblk, int nv, double* out, TO* outT) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    for (int k = warp; k < nv; k += 2 * nw) {
        const int k2 = k + nw;
        const P* p = part + (size_t)k * nblk;
        const P* p2 = part + (size_t)(k2 < nv ? k2 : k) * nblk;
        P s = pzero(P()), s2 = pzero(P());
        for (int b0 = 0; b0 < nblk; b0 += 512) {
            const P c = chunk_sum(p, nblk, b0, lane);
            const P c2 = chunk_sum(p2, nblk, b0, lane);
            s = padd(s, c);
            s2 = padd(s2, c2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s = padd(s, pshfl_down(s, o));
            s2 = padd(s2, pshfl_down(s2, o));
        }
        if (lane == 0) {
            out[k] = pval(s);
            outT[k] = TO(out[k]);
            if (k2 < nv) {
                out[k2] = pval(s2);
                outT[k2] = TO(out[k2]);
            }
        }
    }
    __syncthreads();
}

// h_{j+1,j}^2 = ||w'||^2 - ||h2||^2 by one warp (nv <= 32): every lane returns
// the same value.  The Givens block and the streaming blocks of pass C both
// call it, so the Hessenberg entry and the normalisation of v_{j+1} are the
// same number.
__device__ __forceinline__ double subdiag2(const double* h2, int nv, double wn2) {
    const int lane = threadIdx.x & 31;
    double q = lane < nv ? h2[lane] * h2[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    return wn2 - __shfl_sync(0xffffffffu, q, 0);
}

// ---------------------------------------------------------------- pass A
template <typename T, int NV>
__global__ void __launch_bounds__(NTHREADS, 3)
arnoldi_a(const T* __restrict__ V, size_t ldv, const T* __restrict__ w, size_t n, int nv,
          double* part, Ctl* ctl) {
    pdl_wait();
    if (ctl->done) return;
    using VT = typename V4<T>::type;
    constexpr int W = V4<T>::W;
    T acc_t[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc_t[k] = T(0);
    const size_t nvec = n / W;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const Walk wk = make_walk(blockIdx.x * (size_t)blockDim.x + threadIdx.x, stride, nvec, nv & 1);
    for (size_t c = 0; c < wk.cnt; ++c) {
        const size_t i = wk.at(c);
        const VT wv = reinterpret_cast<const VT*>(w)[i];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (k < nv) acc_t[k] += dotv(reinterpret_cast<const VT*>(V + k * ldv)[i], wv);
    }
    for (size_t i = nvec * W + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (k < nv) acc_t[k] += V[k * ldv + i] * w[i];
    }
    pdl_trigger();
    __shared__ T red[NV][NTHREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (k < nv) {
            T x = acc_t[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) red[k][warp] = x;
        }
    }
    __syncthreads();
    store_partials<T, NV>(red, nv, reinterpret_cast<typename PartOf<T>::type*>(part), gridDim.x, blockIdx.x);
}



// ---------------------------------------------------------------- pass B
// Hessenberg column j, its Givens rotation, the residual estimate, the
// stopping test and (when the cycle ends) the triangular solve R y = g, by
// one whole block.  It runs beside the streaming blocks of pass C, whose
// traffic makes every global round trip slow, so all threads first stage the
// operands in shared memory with their loads in flight together; the
// rotation sequence then runs in thread 0 on shared memory, and the stores
// and the solve are spread over the block.
__device__ void givens_update(Ctl* c, int j, int m, const double* h2, double wn2) {
    __shared__ double col[KMAX + 1], csv[KMAX], snv[KMAX], gv[KMAX + 1], ys[KMAX];
    __shared__ double Rs[KMAX][KMAX + 1];
    __shared__ int finish;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) {
        const double hk = c->h1[k] + h2[k];
        col[k] = hk;
        gv[k] = c->g[k];
        if (k < j) {
            csv[k] = c->cs[k];
            snv[k] = c->sn[k];
        }
        c->Hbar[k][j] = hk;
    }
    __syncthreads();
    double hn2 = 0.0;
    if (threadIdx.x < 32) hn2 = subdiag2(h2, j + 1, wn2);
    if (threadIdx.x == 0) {
        const double target = c->target;
        const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
        col[j + 1] = hn;
        for (int i = 0; i < j; ++i) {
            const double t = csv[i] * col[i] + snv[i] * col[i + 1];
            col[i + 1] = -snv[i] * col[i] + csv[i] * col[i + 1];
            col[i] = t;
        }
        double cs = 1.0, sn = 0.0;
        if (col[j + 1] != 0.0) {
            const double rho = hypot(col[j], col[j + 1]);
            cs = col[j] / rho;
            sn = col[j + 1] / rho;
        }
        const double rjj = cs * col[j] + sn * col[j + 1];
        col[j] = rjj;
        const double gj = gv[j];
        const double gn = -sn * gj;
        gv[j] = cs * gj;
        gv[j + 1] = gn;
        c->Hbar[j + 1][j] = hn;
        c->cs[j] = cs;
        c->sn[j] = sn;
        c->Rt[j][j] = rjj;
        c->g[j + 1] = gn;
        c->g[j] = gv[j];
        c->gres = fabs(gn);
        c->iters += 1;
        const bool finite = isfinite(hn2) && isfinite(gn) && isfinite(rjj);
        const bool conv = fabs(gn) <= target;
        const bool brk = hn == 0.0;
        finish = 0;
        if (!finite) {
            c->nan = 1;
            c->k = 0;
            c->done = 1;
        } else if (conv || brk || j == m - 1) {
            c->converged = conv || brk;
            c->breakdown = brk && !conv;
            finish = 1;
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < j; k += blockDim.x) c->Rt[k][j] = col[k];
    if (!finish) return;
    // back substitution R y = g, column by column (R from earlier columns in
    // global memory, column j in col)
    const int K = j + 1;
    for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
        const int i = e / K, l = e - i * K;
        Rs[i][l] = l == j ? col[i] : (i <= l ? c->Rt[i][l] : 0.0);
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x) ys[i] = gv[i];
    __syncthreads();
    for (int i = K - 1; i >= 0; --i) {
        if (threadIdx.x == 0) ys[i] = ys[i] / Rs[i][i];
        __syncthreads();
        for (int l = threadIdx.x; l < i; l += blockDim.x) ys[l] -= Rs[l][i] * ys[i];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < K; i += blockDim.x) c->y[i] = ys[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        c->k = K;
        c->done = 1;
    }
}

__device__ __forceinline__ float4 shfl_xor_v(unsigned mask, float4 v, int m) {
    return make_float4(__shfl_xor_sync(mask, v.x, m), __shfl_xor_sync(mask, v.y, m), __shfl_xor_sync(mask, v.z, m),
                       __shfl_xor_sync(mask, v.w, m));
}
__device__ __forceinline__ double2 shfl_xor_v(unsigned mask, double2 v, int m) {
    return make_double2(__shfl_xor_sync(mask, v.x, m), __shfl_xor_sync(mask, v.y, m));
}
__device__ __forceinline__ float shfl_xor_v(unsigned mask, float v, int m) { return __shfl_xor_sync(mask, v, m); }
__device__ __forceinline__ double shfl_xor_v(unsigned mask, double v, int m) { return __shfl_xor_sync(mask, v, m); }
__device__ __forceinline__ float4 addv(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
__device__ __forceinline__ double2 addv(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float addv(float a, float b) { return a + b; }
__device__ __forceinline__ double addv(double a, double b) { return a + b; }
__device__ __forceinline__ float4 fmav(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ double2 fmav(double a, double2 x, double2 y) { return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y)); }
__device__ __forceinline__ float fmav(float a, float x, float y) { return fmaf(a, x, y); }
__device__ __forceinline__ double fmav(double a, double x, double y) { return fma(a, x, y); }
__device__ __forceinline__ float4 subv(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ double2 subv(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float subv(float a, float b) { return a - b; }
__device__ __forceinline__ double subv(double a, double b) { return a - b; }
__device__ __forceinline__ float dotv(float a, float b) { return a * b; }
__device__ __forceinline__ double dotv(double a, double b) { return a * b; }
template <typename VT> __device__ __forceinline__ VT zerov();
template <> __device__ __forceinline__ float4 zerov<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 zerov<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float zerov<float>() { return 0.f; }
template <> __device__ __forceinline__ double zerov<double>() { return 0.0; }

// Pass B loads of one element (a VT vector of W entries, or a scalar in the
// tail) for lane q of its group, which owns basis vectors q*CH .. q*CH+CH-1.
template <typename T, typename VT, int CH>
__device__ __forceinline__ void load_b(const T* __restrict__ V, size_t ldv, size_t i, int nv, int q, VT (&v)[CH]) {
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        const int k = q * CH + c;
        v[c] = k < nv ? reinterpret_cast<const VT*>(V + (size_t)k * ldv)[i] : zerov<VT>();
    }
}

// Pass B arithmetic of one element: the group's partial sums of V h1 meet by
// shuffles, w' = w - V h1 is stored by lane 0, every lane dots its vectors with w'.
template <typename T, typename VT, int CH, int KS>
__device__ __forceinline__ void work_b(const VT (&v)[CH], VT wv, T* __restrict__ w, size_t i, int q, const T* h1s,
                                       T (&acc)[CH], T& accn) {
    VT sum = zerov<VT>();
#pragma unroll
    for (int c = 0; c < CH; ++c) sum = fmav(h1s[q * CH + c], v[c], sum);
    const unsigned mask = __activemask();     // the KS lanes of a group are active together
#pragma unroll
    for (int o = 1; o < KS; o <<= 1) sum = addv(sum, shfl_xor_v(mask, sum, o));
    const VT wp = subv(wv, sum);
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] += dotv(v[c], wp);
    if (q == 0) {
        accn += dotv(wp, wp);
        reinterpret_cast<VT*>(w)[i] = wp;
    }
}

// Pass B, split over KS lanes per element: h1 from pass A's partials (every
// block, grid_sums), w' = w - V h1 (stored over w), ||w'||^2 and h2 = V^T w'
// into this pass's partials.  Each lane keeps its CH basis entries in
// registers for both uses, so every basis vector is read from memory once;
// with at most eight entries per lane the next element's loads are issued
// before the current one is combined (software pipeline).
template <typename T, int NV>
__global__ void __launch_bounds__(NTHREADS, 2)
arnoldi_b(const T* __restrict__ V, size_t ldv, T* __restrict__ w, size_t n, int nv,
          const double* partA, int nblkA, double* part, Ctl* ctl, int jscale) {
    pdl_wait();
    const int done = ctl->done;     // no writer during this launch; read beside the partials
    // jscale >= 0: w is used as zscale[jscale] w (lagged second projection, see arnoldi_ca)
    const T sig = jscale >= 0 ? T(ctl->zscale[jscale]) : T(1);
    // one lane per element up to NV = 16, two above (four for a float64 basis at
    // NV = 32, where two would not fit the registers): a lane keeps up to sixteen
    // loads in flight, and the instantiation nearest above nv (8, 12, 16, 24, 32)
    // leaves few of its entries empty
    constexpr int KS = NV <= 16 ? 1 : ((sizeof(T) == sizeof(double) && NV > 24) ? 4 : 2), CH = NV / KS;
    // the next element's loads are issued ahead (software pipeline) where the
    // registers allow it; twelve or more entries per lane are deep enough without
    constexpr bool PF = CH <= 8;
    static_assert(CH * KS == NV && CH <= 16, "lane split");
    __shared__ double h1d[NV];
    __shared__ T h1s[NV];
    __shared__ T red[NV + 1][NTHREADS / 32];
    using P = typename PartOf<T>::type;
    for (int k = nv + threadIdx.x; k < NV; k += blockDim.x) h1s[k] = T(0);
    grid_sums(reinterpret_cast<const P*>(partA), nblkA, nv, h1d, h1s);
    if (done) return;
    if (blockIdx.x == 0)       // h1 for the Hessenberg column
        for (int k = threadIdx.x; k < nv; k += blockDim.x) ctl->h1[k] = h1d[k];
    using VT = typename V4<T>::type;
    constexpr int W = V4<T>::W;
    const int q = threadIdx.x & (KS - 1);
    T acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = T(0);
    T accn = T(0);
    const size_t nvec = n / W;
    const size_t g0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) / KS;
    const size_t gstride = (size_t)gridDim.x * blockDim.x / KS;
    const Walk wk = make_walk(g0, gstride, nvec, !(nv & 1));
    if constexpr (!PF) {
        for (size_t cc = 0; cc < wk.cnt; ++cc) {
            const size_t i = wk.at(cc);
            VT v[CH];
            load_b<T, VT, CH>(V, ldv, i, nv, q, v);
            work_b<T, VT, CH, KS>(v, scalev(reinterpret_cast<const VT*>(w)[i], sig), w, i, q, h1s, acc, accn);
        }
    } else {
        VT vn[CH], wn = zerov<VT>();
        if (wk.cnt > 0) {
            load_b<T, VT, CH>(V, ldv, wk.at(0), nv, q, vn);
            wn = scalev(reinterpret_cast<const VT*>(w)[wk.at(0)], sig);
        }
        for (size_t cc = 0; cc < wk.cnt; ++cc) {
            const size_t i = wk.at(cc);
            VT v[CH];
#pragma unroll
            for (int c = 0; c < CH; ++c) v[c] = vn[c];
            const VT wv = wn;
            if (cc + 1 < wk.cnt) {
                const size_t inext = wk.at(cc + 1);
                load_b<T, VT, CH>(V, ldv, inext, nv, q, vn);
                wn = scalev(reinterpret_cast<const VT*>(w)[inext], sig);
            }
            work_b<T, VT, CH, KS>(v, wv, w, i, q, h1s, acc, accn);
        }
    }
    for (size_t i = nvec * W + g0; i < n; i += gstride) {
        T v[CH];
        load_b<T, T, CH>(V, ldv, i, nv, q, v);
        work_b<T, T, CH, KS>(v, sig * w[i], w, i, q, h1s, acc, accn);
    }
    pdl_trigger();
    // block sums: slot 0 = ||w'||^2, slot 1 + k = v_k . w' (fixed shuffle trees, then the partial type across warps)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        T x = acc[c];
#pragma unroll
        for (int o = KS; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane < KS) red[1 + lane * CH + c][warp] = x;
    }
    {
        T x = accn;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[0][warp] = x;
    }
    __syncthreads();
    store_partials<T, NV + 1>(red, nv + 1, reinterpret_cast<P*>(part), gridDim.x, blockIdx.x);
}

// ---------------------------------------------------------------- pass C
// Every block sums pass B's partials (||w'||^2, h2).  Block 0 runs the serial
// Hessenberg / Givens update for column j = nv - 1 while blocks 1.. stream
// v_{j+1}.  A streaming block that starts after block 0 has ended the cycle
// (converged, breakdown or m steps) finds done set and returns: v_{j+1} is
// not used after the cycle's last step.
template <typename T, int NV>
__global__ void __launch_bounds__(NTHREADS, 3)
arnoldi_c(T* __restrict__ V, size_t ldv, const T* __restrict__ w, size_t n, int nv, int m,
          const double* partB, int nblkB, Ctl* ctl) {
    pdl_wait();
    using VT = typename V4<T>::type;
    constexpr int W = V4<T>::W;
    __shared__ double tot[NV + 1];
    __shared__ T tots[NV + 1];      // tots[1 + k] = h2_k rounded to T
    __shared__ T inv_s;
    __shared__ int done;
    // block 0 writes ctl->done during this launch: one thread reads it for the
    // whole block, so that every thread of a block takes the same branch
    if (threadIdx.x == 0) done = *(volatile int*)&ctl->done;
    for (int k = nv + 1 + threadIdx.x; k <= NV; k += blockDim.x) tots[k] = T(0);   // h2 past the basis: zero
    grid_sums(reinterpret_cast<const typename PartOf<T>::type*>(partB), nblkB, nv + 1, tot, tots);
    if (done) return;
    if (blockIdx.x == 0) {
        givens_update(ctl, nv - 1, m, tot + 1, tot[0]);
        return;
    }
    const T* hs = tots + 1;
    if (threadIdx.x < 32) {
        const double hn2 = subdiag2(tot + 1, nv, tot[0]);
        const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
        if (threadIdx.x == 0) inv_s = T(hn > 0.0 ? 1.0 / hn : 0.0);
    }
    __syncthreads();
    const T inv = inv_s;
    // KS = NV / 8 lanes per element (at most eight basis entries per lane, within
    // the registers of three CTAs per SM); a lane loads all its entries before it
    // combines them, the lanes' parts of V h2 meet by shuffles and lane 0 stores
    constexpr int KS = NV <= 8 ? 1 : NV / 8, CH = NV / KS;
    const int q = threadIdx.x & (KS - 1);
    const size_t nvec = n / W;
    const size_t nblk = gridDim.x - 1, blk = blockIdx.x - 1;
    const size_t g0 = (blk * blockDim.x + threadIdx.x) / KS;
    const size_t gstride = nblk * blockDim.x / KS;
    T* vout = V + (size_t)nv * ldv;
    const Walk wk = make_walk(g0, gstride, nvec, nv & 1);
    for (size_t cc = 0; cc < wk.cnt; ++cc) {
        const size_t i = wk.at(cc);
        VT v[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int k = q * CH + c;
            v[c] = k < nv ? reinterpret_cast<const VT*>(V + k * ldv)[i] : zerov<VT>();
        }
        const VT wv = reinterpret_cast<const VT*>(w)[i];
        VT sum = zerov<VT>();
#pragma unroll
        for (int c = 0; c < CH; ++c) sum = fmav(hs[q * CH + c], v[c], sum);
        if (KS > 1) {
            const unsigned mask = __activemask();     // the KS lanes of an element are active together
#pragma unroll
            for (int o = 1; o < KS; o <<= 1) sum = addv(sum, shfl_xor_v(mask, sum, o));
        }
        if (q == 0) reinterpret_cast<VT*>(vout)[i] = scalev(subv(wv, sum), inv);
    }
    for (size_t i = nvec * W + g0; i < n; i += gstride) {
        T sum = T(0);
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int k = q * CH + c;
            if (k < nv) sum = fmav(hs[k], V[k * ldv + i], sum);
        }
        if (KS > 1) {
            const unsigned mask = __activemask();
#pragma unroll
            for (int o = 1; o < KS; o <<= 1) sum += __shfl_xor_sync(mask, sum, o);
        }
        if (q == 0) vout[i] = (w[i] - sum) * inv;
    }
}

// ---------------------------------------------------------------- pass CA
// Right-preconditioned path: pass C of step j-1 fused with pass A of step j
// (the second projection of CGS2 is lagged behind the next Jacobian
// product).  Step j takes as its direction the once-projected vector of the
// previous step instead of v_j:  z_j = M^{-1} w'_{j-1},  w_j = J z_j,  with
// w'_{j-1} = w_{j-1} - V h1 from pass B.  Flexible GMRES accepts any z_j
// (x = x_0 + Z y minimises ||b - J x|| over span Z for every choice), and for
// a fixed linear M the span is that of M^{-1} v_0 .. M^{-1} v_j, because
// w'_{j-1} = h_{j,j-1} v_j + V h2 with V h2 in the span of the earlier basis:
// the iterates are those of right-preconditioned GMRES in exact arithmetic.
// One sweep then forms v_j = (w'_{j-1} - V h2) / h_{j,j-1} and the first
// projection h1 = [v_0 .. v_j]^T w_j of step j, reading every basis vector
// once; block 0 runs the Hessenberg / Givens update of column j-1 (as pass
// C's block 0 does).  Partials (j + 1 values) are indexed by streaming block.
template <typename T, int NV>
__global__ void __launch_bounds__(NTHREADS, 2)
arnoldi_ca(T* __restrict__ V, size_t ldv, const T* __restrict__ wprev, const T* __restrict__ w, size_t n,
           int j, int m, const double* partB, int nblkB, double* partA, Ctl* ctl) {
    pdl_wait();
    using VT = typename V4<T>::type;
    using P = typename PartOf<T>::type;
    constexpr int W = V4<T>::W;
    __shared__ double tot[NV + 1];
    __shared__ T tots[NV + 1];      // tots[1 + k] = h2_k rounded to T
    __shared__ T inv_s;
    __shared__ int done;
    __shared__ T red[NV + 1][NTHREADS / 32];
    // block 0 writes ctl->done during this launch: one thread reads it for the whole block
    if (threadIdx.x == 0) done = *(volatile int*)&ctl->done;
    for (int k = j + 1 + threadIdx.x; k <= NV; k += blockDim.x) tots[k] = T(0);   // h2 past the basis: zero
    grid_sums(reinterpret_cast<const P*>(partB), nblkB, j + 1, tot, tots);   // ||w'||^2, h2_0 .. h2_{j-1}
    if (done) return;
    if (blockIdx.x == 0) {
        givens_update(ctl, j - 1, m, tot + 1, tot[0]);
        return;
    }
    const T* hs = tots + 1;
    __shared__ T sig_s;
    if (threadIdx.x < 32) {
        const double hn2 = subdiag2(tot + 1, j, tot[0]);
        const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
        if (threadIdx.x == 0) {
            inv_s = T(hn > 0.0 ? 1.0 / hn : 0.0);
            // z_j = M^{-1} w'_{j-1} carries the scale ||w'_{j-1}||: w_j = J z_j is used
            // as sigma w_j with sigma = 1 / ||w'_{j-1}||, and z_j enters the update as sigma z_j
            const double sg = tot[0] > 0.0 ? 1.0 / sqrt(tot[0]) : 0.0;
            sig_s = T(sg);
            if (blockIdx.x == 1) ctl->zscale[j] = (double)T(sg);
        }
    }
    __syncthreads();
    const T inv = inv_s;
    const T sig = sig_s;
    // KS lanes per element (one up to NV = 16, two above; four for a float64
    // basis at NV = 32): a lane loads all its basis entries before it combines
    // them, so that they are in flight together; the lanes' parts of V h2 meet
    // by shuffles and lane 0 stores v_j
    constexpr int KS = NV <= 16 ? 1 : ((sizeof(T) == sizeof(double) && NV > 24) ? 4 : 2), CH = NV / KS;
    const int q = threadIdx.x & (KS - 1);
    T acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = T(0);
    T accn = T(0);                  // v_j . w_j (v_j is formed in registers)
    const size_t nvec = n / W;
    const size_t nblk = gridDim.x - 1, blk = blockIdx.x - 1;
    const size_t g0 = (blk * blockDim.x + threadIdx.x) / KS;
    const size_t gstride = nblk * blockDim.x / KS;
    T* vout = V + (size_t)j * ldv;
    const Walk wk = make_walk(g0, gstride, nvec, (j + 1) & 1);
    for (size_t cc = 0; cc < wk.cnt; ++cc) {
        const size_t i = wk.at(cc);
        VT v[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int k = q * CH + c;
            v[c] = k < j ? reinterpret_cast<const VT*>(V + k * ldv)[i] : zerov<VT>();
        }
        const VT wpv = reinterpret_cast<const VT*>(wprev)[i];
        const VT wv = scalev(reinterpret_cast<const VT*>(w)[i], sig);
        VT sum = zerov<VT>();
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            sum = fmav(hs[q * CH + c], v[c], sum);
            acc[c] += dotv(v[c], wv);
        }
        if (KS > 1) {
            const unsigned mask = __activemask();     // the KS lanes of an element are active together
#pragma unroll
            for (int o = 1; o < KS; o <<= 1) sum = addv(sum, shfl_xor_v(mask, sum, o));
        }
        const VT vn = scalev(subv(wpv, sum), inv);
        if (q == 0) {
            reinterpret_cast<VT*>(vout)[i] = vn;
            accn += dotv(vn, wv);
        }
    }
    for (size_t i = nvec * W + g0; i < n; i += gstride) {
        const T wv = sig * w[i];
        T sum = T(0);
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const int k = q * CH + c;
            if (k < j) {
                const T vk = V[k * ldv + i];
                sum = fmav(hs[k], vk, sum);
                acc[c] += vk * wv;
            }
        }
        if (KS > 1) {
            const unsigned mask = __activemask();
#pragma unroll
            for (int o = 1; o < KS; o <<= 1) sum += __shfl_xor_sync(mask, sum, o);
        }
        const T vn = (wprev[i] - sum) * inv;
        if (q == 0) {
            vout[i] = vn;
            accn += vn * wv;
        }
    }
    pdl_trigger();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        T x = acc[c];
#pragma unroll
        for (int o = KS; o < 32; o <<= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane < KS && lane * CH + c < j) red[lane * CH + c][warp] = x;
    }
    {
        T x = accn;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[j][warp] = x;
    }
    __syncthreads();
    store_partials<T, NV + 1>(red, j + 1, reinterpret_cast<P*>(partA), (int)nblk, (int)blk);
}

// ---------------------------------------------------------------- update
// x += sum_{k < K} y_k z_k, xT = x rounded to T, eps_jv for J x.
// The directions z_k enter exactly and their combination carries no extra
// rounding: float64 basis -> float64 FMAs; float32 basis -> a double-float
// (hi + lo float32 pair) sum with error-free products and TwoSum additions
// (Dekker 1971; Knuth TAOCP vol. 2), ~2^-44 relative, then one float64 add.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

template <typename T, int NV>
__global__ void __launch_bounds__(NTHREADS, 2)
update_x(const T* __restrict__ Z, size_t ldz, double* __restrict__ x, T* __restrict__ xT, size_t n,
         double* part, Ctl* ctl) {
    const int K = ctl->k;
    __shared__ double ys[NV];
    __shared__ float yh[NV], yl[NV];
    for (int k = threadIdx.x; k < NV; k += blockDim.x) {
        const double y = k < K ? ctl->y[k] * ctl->zscale[k] : 0.0;
        ys[k] = y;
        yh[k] = (float)y;
        yl[k] = (float)(y - (double)(float)y);
    }
    __syncthreads();
    T acc[1] = {T(0)};
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        // all K loads of the element are issued before the (serial) combination
        T zv[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) zv[k] = k < K ? Z[k * ldz + i] : T(0);
        double s;
        if (sizeof(T) == sizeof(double)) {
            s = x[i];
#pragma unroll
            for (int k = 0; k < NV; ++k)
                if (k < K) s += ys[k] * (double)zv[k];
        } else {
            float hi = 0.0f, lo = 0.0f;
#pragma unroll
            for (int k = 0; k < NV; ++k)
                if (k < K) {
                    const float z = (float)zv[k];
                    const float ph = yh[k] * z;
                    const float pl = fmaf(yh[k], z, -ph);      // exact product error
                    float t, e;
                    two_sum(hi, ph, t, e);
                    hi = t;
                    lo += e + pl + yl[k] * z;
                }
            s = x[i] + ((double)hi + (double)lo);
        }
        x[i] = s;
        if (xT != nullptr) xT[i] = T(s);
        acc[0] += T(s) * T(s);
    }
    block_partials<1, T>(acc, 1, part, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_UPDATE], gridDim.x)) {
        __shared__ double tot[1];
        final_sums(part, gridDim.x, 1, tot);
        if (threadIdx.x == 0) {
            ctl->scratch[0] = tot[0];
            const double xn = sqrt(tot[0]);
            ctl->eps_jv = xn > 0.0 ? sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2))) / xn : 0.0;
            ctl->eps_part = 0;
        }
    }
}

// ---------------------------------------------------------------- cycle start
// First cycle of a Newton solve: b = -W R, v_0 = b / ||b||, x = 0, control reset.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
cycle_init(Geo G, const double* __restrict__ R, T* __restrict__ V0, double* __restrict__ x, size_t n,
           double eta, int m, int pc_none, Ctl* ctl) {
    const double beta = sqrt(ctl->res2);
    const double inv = beta > 0.0 ? 1.0 / beta : 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int f = field_of(i, G.npt);
        V0[i] = T(-R[i] * G.inv_scale[f] * inv);
        x[i] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->beta0 = beta;
        ctl->target = eta * beta;
        ctl->g[0] = beta;
        ctl->gstart = beta;
        ctl->gres = beta;
        ctl->done = 0;
        ctl->converged = beta == 0.0;
        ctl->breakdown = 0;
        ctl->k = 0;
        ctl->iters = 0;
        ctl->m = m;
        for (int k = 0; k < KMAX; ++k) ctl->zscale[k] = 1.0;
        if (pc_none) {
            ctl->eps_jv = sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2)));
            ctl->eps_part = 0;
        }
    }
}

// Restart: r = b - w with w = J x, stored unnormalised in v_0 plus ||r||^2.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
restart_residual(Geo G, const double* __restrict__ R, const T* __restrict__ w, T* __restrict__ V0,
                 size_t n, double* part, Ctl* ctl) {
    double acc[1] = {0.0};
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int f = field_of(i, G.npt);
        const double r = -R[i] * G.inv_scale[f] - (double)w[i];
        V0[i] = T(r);
        acc[0] += r * r;
    }
    block_partials<1>(acc, 1, part, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_RESTART], gridDim.x)) {
        __shared__ double tot[1];
        final_sums(part, gridDim.x, 1, tot);
        if (threadIdx.x == 0) ctl->scratch[1] = tot[0];
    }
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
restart_scale(T* __restrict__ V0, size_t n, int pc_none, Ctl* ctl) {
    const double beta = sqrt(ctl->scratch[1]);
    const T inv = T(beta > 0.0 ? 1.0 / beta : 0.0);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) V0[i] *= inv;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->g[0] = beta;
        ctl->gstart = beta;
        ctl->gres = beta;
        ctl->done = 0;
        ctl->converged = 0;
        ctl->breakdown = 0;
        ctl->k = 0;
        for (int k = 0; k < KMAX; ++k) ctl->zscale[k] = 1.0;
        if (pc_none) {
            ctl->eps_jv = sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2)));
            ctl->eps_part = 0;
        }
    }
}

// Left preconditioning (nonlinear preconditioning): the cycle starts from
// z = M^{-1} r with ||z||^2 in scratch[1].  v_0 = z / ||z||; on the first cycle
// of a Newton solve (r = b / ||b|| from cycle_init) the preconditioned right-
// hand side has norm beta0 ||z||, which rescales beta0 and the target; on a
// restart (r = b - J x unnormalised) g_0 = ||z||.  The Jacobian products of
// the cycle act on unit vectors: eps from ||u|| alone.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
left_scale(const T* __restrict__ z, T* __restrict__ V0, size_t n, int first, Ctl* ctl) {
    const double zn = sqrt(ctl->scratch[1]);
    const T inv = T(zn > 0.0 ? 1.0 / zn : 0.0);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) V0[i] = z[i] * inv;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double g0 = zn;
        if (first) {
            g0 = ctl->beta0 * zn;
            ctl->beta0 = g0;
            ctl->target *= zn;
            ctl->converged = g0 == 0.0;
        } else {
            ctl->converged = 0;
        }
        ctl->g[0] = g0;
        ctl->gstart = g0;
        ctl->gres = g0;
        ctl->done = 0;
        ctl->breakdown = 0;
        ctl->k = 0;
        ctl->eps_jv = sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2)));
        ctl->eps_part = 0;
    }
}

// The finite-difference step of a Jacobian product on a unit vector (left
// preconditioning: restores it after a preconditioner apply left its own).
__global__ void unit_eps_k(Ctl* ctl) {
    ctl->eps_jv = sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2)));
    ctl->eps_part = 0;
}

// u += W^{-1} x (float64), uT = u rounded to T.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
newton_update(Geo G, double* __restrict__ u, const double* __restrict__ x, T* __restrict__ uT, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int f = field_of(i, G.npt);
        const double v = u[i] + G.scale[f] * x[i];
        u[i] = v;
        if (uT != nullptr) uT[i] = T(v);
    }
}

// ---------------------------------------------------------------- utilities
template <typename TI, typename TO>
__global__ void __launch_bounds__(NTHREADS) convert_k(const TI* __restrict__ in, TO* __restrict__ out, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) out[i] = TO(in[i]);
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(NTHREADS)
rescale_k(Geo G, const TI* __restrict__ in, TO* __restrict__ out, size_t n, int multiply) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int f = field_of(i, G.npt);
        out[i] = TO((double)in[i] * (multiply ? G.scale[f] : G.inv_scale[f]));
    }
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
norm2_k(Geo G, const T* __restrict__ a, size_t n, int weighted, int slot, double* part, Ctl* ctl) {
    double acc[1] = {0.0};
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        double v = (double)a[i];
        if (weighted) v *= G.inv_scale[field_of(i, G.npt)];
        acc[0] += v * v;
    }
    block_partials<1>(acc, 1, part, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_MISC], gridDim.x)) {
        __shared__ double tot[1];
        final_sums(part, gridDim.x, 1, tot);
        if (threadIdx.x == 0) ctl->scratch[slot] = tot[0];
    }
}

__global__ void set_eps_k(double eps, int su, int sv, Ctl* ctl) {
    ctl->eps_part = 0;
    if (eps > 0.0) {
        ctl->eps_jv = eps;
    } else {
        const double vn = sqrt(ctl->scratch[sv]);
        ctl->eps_jv = vn > 0.0 ? sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->scratch[su]))) / vn : 0.0;
    }
}

// ------------------------------------------------- learned preconditioner
// Training pairs are staged in fixed buffers and copied into slot ctl->ncap of
// the pair store by the last kernel of the sequence, so that steps enqueued
// after a GMRES cycle finished (ctl->done) record nothing.
constexpr int PAIR_SLOT = 6;   // ctl->scratch slot of ||w||^2

// ||w||^2 of an Arnoldi product.
__global__ void __launch_bounds__(NTHREADS)
pair_norm_k(const float* __restrict__ w, size_t n, double* part, Ctl* ctl) {
    if (ctl->done) return;
    float acc[1] = {0.f};
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) acc[0] = fmaf(w[i], w[i], acc[0]);
    block_partials<1>(acc, 1, part, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_MISC], gridDim.x)) {
        __shared__ double tot[1];
        final_sums(part, gridDim.x, 1, tot);
        if (threadIdx.x == 0) ctl->scratch[PAIR_SLOT] = tot[0];
    }
}

// Arnoldi pair input X = w / ||w||.
__global__ void __launch_bounds__(NTHREADS)
pair_stage_arnoldi_k(const float* __restrict__ w, float* __restrict__ X, size_t n, const Ctl* ctl) {
    if (ctl->done) return;
    const double nw = sqrt(ctl->scratch[PAIR_SLOT]);
    const float inv = (float)(nw > 0.0 ? 1.0 / nw : 0.0);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) X[i] = w[i] * inv;
}

// Newton pair input X = -W R / beta0.
__global__ void __launch_bounds__(NTHREADS)
pair_stage_newton_k(Geo G, const double* __restrict__ R, float* __restrict__ X, size_t n, const Ctl* ctl) {
    const double b = ctl->beta0;
    const double inv = b > 0.0 ? 1.0 / b : 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        const int f = field_of(i, G.npt);
        X[i] = (float)(-R[i] * G.inv_scale[f] * inv);
    }
}

// Slot ctl->ncap of the store: X = staged input, T = c * corr - MX with
// c = 1 / ||w|| (Arnoldi, corr = z_j) or 1 / beta0 (Newton, corr = x_hat).
template <typename TC>
__global__ void __launch_bounds__(NTHREADS)
pair_store_k(const float* __restrict__ Xs, const TC* __restrict__ corr, const float* __restrict__ MX,
             float* __restrict__ Xbuf, float* __restrict__ Tbuf, size_t n, int cap, int arnoldi, const Ctl* ctl) {
    if (arnoldi && ctl->done) return;
    const int slot = ctl->ncap;
    if (slot < 0 || slot >= cap) return;
    const double d = arnoldi ? sqrt(ctl->scratch[PAIR_SLOT]) : ctl->beta0;
    const double c = d > 0.0 ? 1.0 / d : 0.0;
    float* X = Xbuf + (size_t)slot * n;
    float* T = Tbuf + (size_t)slot * n;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        X[i] = Xs[i];
        T[i] = (float)((double)corr[i] * c - (double)MX[i]);
    }
}

__global__ void pair_commit_k(int cap, int arnoldi, Ctl* ctl) {
    if (arnoldi && ctl->done) return;
    if (ctl->ncap < cap) ctl->ncap += 1;
}

// FD step of the next Jacobian-vector product from ||z|| once the network's
// correction has been added to z (returns at entry once the cycle is done).
__global__ void __launch_bounds__(NTHREADS)
pc_eps_k(const float* __restrict__ z, size_t n, double* part, Ctl* ctl) {
    if (ctl->done) return;
    float acc[1] = {0.f};
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) acc[0] = fmaf(z[i], z[i], acc[0]);
    block_partials<1>(acc, 1, part, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_MISC], gridDim.x)) {
        __shared__ double tot[1];
        final_sums(part, gridDim.x, 1, tot);
        if (threadIdx.x == 0) {
            const double zn = sqrt(tot[0]);
            ctl->eps_jv = zn > 0.0 ? sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2))) / zn : 0.0;
            ctl->eps_part = 0;
        }
    }
}

// ---------------------------------------------------------------- launchers

// Grids of the three passes (B and C size their reads of the previous pass's
// partials from them).  Pass C adds one block for the Givens update and keeps
// the whole grid within one wave of three CTAs per SM.
template <typename T> static int grid_a(size_t n) {
    return std::max(dot_blocks(n / V4<T>::W), reduce_blocks(n / V4<T>::W));
}
template <typename T> static int grid_b(size_t n) { return reduce_blocks(n / V4<T>::W); }
template <typename T> static int grid_c(size_t n) {
    return std::min(dot_blocks(n / V4<T>::W) + 1, MAX_DOT_BLOCKS);
}

template <typename T>
int arnoldi_a_parts(size_t n) {
    return grid_a<T>(n);
}
template int arnoldi_a_parts<float>(size_t);
template int arnoldi_a_parts<double>(size_t);

template <typename T>
cudaError_t launch_arnoldi_a(const T* V, size_t ldv, const T* w, size_t n, int nv, double* partA,
                             Ctl* ctl, cudaStream_t s) {
    const int nb = grid_a<T>(n);
    if (nv <= 8) return launch_pdl(arnoldi_a<T, 8>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, ctl);
    if (nv <= 16) return launch_pdl(arnoldi_a<T, 16>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, ctl);
    return launch_pdl(arnoldi_a<T, 32>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, ctl);
}

template <typename T>
cudaError_t launch_arnoldi_b(const T* V, size_t ldv, T* w, size_t n, int nv, const double* partA,
                             double* partB, Ctl* ctl, cudaStream_t s) {
    const int nb = grid_b<T>(n), na = grid_a<T>(n);
    if (nv <= 8) return launch_pdl(arnoldi_b<T, 8>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, na, partB, ctl, -1);
    if (nv <= 12) return launch_pdl(arnoldi_b<T, 12>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, na, partB, ctl, -1);
    if (nv <= 16) return launch_pdl(arnoldi_b<T, 16>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, na, partB, ctl, -1);
    if (nv <= 24) return launch_pdl(arnoldi_b<T, 24>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, na, partB, ctl, -1);
    return launch_pdl(arnoldi_b<T, 32>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, na, partB, ctl, -1);
}

template <typename T>
cudaError_t launch_arnoldi_c(T* V, size_t ldv, const T* w, size_t n, int nv, int m, const double* partB,
                             Ctl* ctl, cudaStream_t s) {
    const int nc = grid_c<T>(n), nb = grid_b<T>(n);
    if (nv <= 8) return launch_pdl(arnoldi_c<T, 8>, nc, NTHREADS, 0, s, V, ldv, w, n, nv, m, partB, nb, ctl);
    if (nv <= 16) return launch_pdl(arnoldi_c<T, 16>, nc, NTHREADS, 0, s, V, ldv, w, n, nv, m, partB, nb, ctl);
    return launch_pdl(arnoldi_c<T, 32>, nc, NTHREADS, 0, s, V, ldv, w, n, nv, m, partB, nb, ctl);
}

// Fused pass CA of step j (1 <= j < KMAX): the partials it leaves for pass B
// come from grid_ca_parts() blocks.
// Two CTAs per SM are resident (register use): the Givens block and the
// streaming blocks fit one wave.
constexpr int MAX_CA_BLOCKS = 2 * 152;
template <typename T> static int grid_ca(size_t n) {
    return std::min(dot_blocks(n / V4<T>::W), MAX_CA_BLOCKS - 1) + 1;
}
template <typename T>
int arnoldi_ca_parts(size_t n) {
    return grid_ca<T>(n) - 1;
}
template int arnoldi_ca_parts<float>(size_t);
template int arnoldi_ca_parts<double>(size_t);

template <typename T>
cudaError_t launch_arnoldi_ca(T* V, size_t ldv, const T* wprev, const T* w, size_t n, int j, int m,
                              const double* partB, double* partA, Ctl* ctl, cudaStream_t s) {
    const int nc = grid_ca<T>(n), nb = grid_b<T>(n);
    if (j + 1 <= 8)
        return launch_pdl(arnoldi_ca<T, 8>, nc, NTHREADS, 0, s, V, ldv, wprev, w, n, j, m, partB, nb, partA, ctl);
    if (j + 1 <= 12)
        return launch_pdl(arnoldi_ca<T, 12>, nc, NTHREADS, 0, s, V, ldv, wprev, w, n, j, m, partB, nb, partA, ctl);
    if (j + 1 <= 16)
        return launch_pdl(arnoldi_ca<T, 16>, nc, NTHREADS, 0, s, V, ldv, wprev, w, n, j, m, partB, nb, partA, ctl);
    if (j + 1 <= 24)
        return launch_pdl(arnoldi_ca<T, 24>, nc, NTHREADS, 0, s, V, ldv, wprev, w, n, j, m, partB, nb, partA, ctl);
    return launch_pdl(arnoldi_ca<T, 32>, nc, NTHREADS, 0, s, V, ldv, wprev, w, n, j, m, partB, nb, partA, ctl);
}
template cudaError_t launch_arnoldi_ca<float>(float*, size_t, const float*, const float*, size_t, int, int,
                                              const double*, double*, Ctl*, cudaStream_t);
template cudaError_t launch_arnoldi_ca<double>(double*, size_t, const double*, const double*, size_t, int, int,
                                               const double*, double*, Ctl*, cudaStream_t);

// Pass B whose h1 partials come from nblkA blocks (pass A: grid_a; pass CA: arnoldi_ca_parts).
template <typename T>
cudaError_t launch_arnoldi_b_from(const T* V, size_t ldv, T* w, size_t n, int nv, const double* partA, int nblkA,
                                  double* partB, Ctl* ctl, cudaStream_t s) {
    const int nb = grid_b<T>(n);
    const int js = nv > 1 ? nv - 1 : -1;    // step j = nv - 1 >= 1 follows pass CA: w is scaled
    if (nv <= 8) return launch_pdl(arnoldi_b<T, 8>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, nblkA, partB, ctl, js);
    if (nv <= 12) return launch_pdl(arnoldi_b<T, 12>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, nblkA, partB, ctl, js);
    if (nv <= 16) return launch_pdl(arnoldi_b<T, 16>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, nblkA, partB, ctl, js);
    if (nv <= 24) return launch_pdl(arnoldi_b<T, 24>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, nblkA, partB, ctl, js);
    return launch_pdl(arnoldi_b<T, 32>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, partA, nblkA, partB, ctl, js);
}
template cudaError_t launch_arnoldi_b_from<float>(const float*, size_t, float*, size_t, int, const double*, int,
                                                  double*, Ctl*, cudaStream_t);
template cudaError_t launch_arnoldi_b_from<double>(const double*, size_t, double*, size_t, int, const double*, int,
                                                   double*, Ctl*, cudaStream_t);

// The Hessenberg / Givens update of the last column of a cycle alone (pass C
// with its Givens block and no streaming blocks), after pass B of step nv - 1.
template <typename T>
cudaError_t launch_arnoldi_givens(size_t n, int nv, int m, const double* partB, Ctl* ctl, cudaStream_t s) {
    const int nb = grid_b<T>(n);
    T* none = nullptr;
    if (nv <= 8) return launch_pdl(arnoldi_c<T, 8>, 1, NTHREADS, 0, s, none, (size_t)0, (const T*)none, n, nv, m, partB, nb, ctl);
    if (nv <= 16) return launch_pdl(arnoldi_c<T, 16>, 1, NTHREADS, 0, s, none, (size_t)0, (const T*)none, n, nv, m, partB, nb, ctl);
    return launch_pdl(arnoldi_c<T, 32>, 1, NTHREADS, 0, s, none, (size_t)0, (const T*)none, n, nv, m, partB, nb, ctl);
}
template cudaError_t launch_arnoldi_givens<float>(size_t, int, int, const double*, Ctl*, cudaStream_t);
template cudaError_t launch_arnoldi_givens<double>(size_t, int, int, const double*, Ctl*, cudaStream_t);

template <typename T>
cudaError_t launch_update(const T* Z, size_t ldz, double* x, T* xT, size_t n, double* part,
                          Ctl* ctl, cudaStream_t s) {
    update_x<T, KMAX><<<stream_blocks(n), NTHREADS, 0, s>>>(Z, ldz, x, xT, n, part, ctl);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cycle_init(const Geo& G, const double* R, T* V0, double* x, size_t n, double eta,
                              int m, int pc_none, Ctl* ctl, cudaStream_t s) {
    cycle_init<T><<<stream_blocks(n), NTHREADS, 0, s>>>(G, R, V0, x, n, eta, m, pc_none, ctl);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restart(const Geo& G, const double* R, const T* w, T* V0, size_t n, int pc_none,
                           double* part, Ctl* ctl, cudaStream_t s, long long* launches) {
    restart_residual<T><<<stream_blocks(n), NTHREADS, 0, s>>>(G, R, w, V0, n, part, ctl);
    restart_scale<T><<<stream_blocks(n), NTHREADS, 0, s>>>(V0, n, pc_none, ctl);
    if (launches) *launches += 2;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restart_residual(const Geo& G, const double* R, const T* w, T* V0, size_t n, double* part,
                                    Ctl* ctl, cudaStream_t s) {
    restart_residual<T><<<stream_blocks(n), NTHREADS, 0, s>>>(G, R, w, V0, n, part, ctl);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_left_scale(const T* z, T* V0, size_t n, int first, Ctl* ctl, cudaStream_t s) {
    left_scale<T><<<stream_blocks(n), NTHREADS, 0, s>>>(z, V0, n, first, ctl);
    return cudaGetLastError();
}

cudaError_t launch_unit_eps(Ctl* ctl, cudaStream_t s) {
    unit_eps_k<<<1, 1, 0, s>>>(ctl);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_newton_update(const Geo& G, double* u, const double* x, T* uT, size_t n,
                                 cudaStream_t s) {
    newton_update<T><<<stream_blocks(n), NTHREADS, 0, s>>>(G, u, x, uT, n);
    return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_convert(const TI* in, TO* out, size_t n, cudaStream_t s) {
    convert_k<TI, TO><<<stream_blocks(n), NTHREADS, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_rescale(const Geo& G, const TI* in, TO* out, size_t n, int multiply, cudaStream_t s) {
    rescale_k<TI, TO><<<stream_blocks(n), NTHREADS, 0, s>>>(G, in, out, n, multiply);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_norm2(const Geo& G, const T* a, size_t n, int weighted, int slot, double* part,
                         Ctl* ctl, cudaStream_t s) {
    norm2_k<T><<<stream_blocks(n), NTHREADS, 0, s>>>(G, a, n, weighted, slot, part, ctl);
    return cudaGetLastError();
}

cudaError_t launch_set_eps(double eps, int su, int sv, Ctl* ctl, cudaStream_t s) {
    set_eps_k<<<1, 1, 0, s>>>(eps, su, sv, ctl);
    return cudaGetLastError();
}

cudaError_t launch_pair_arnoldi(const float* w, float* Xs, size_t n, double* part, Ctl* ctl, cudaStream_t s) {
    pair_norm_k<<<stream_blocks(n), NTHREADS, 0, s>>>(w, n, part, ctl);
    pair_stage_arnoldi_k<<<stream_blocks(n), NTHREADS, 0, s>>>(w, Xs, n, ctl);
    return cudaGetLastError();
}

cudaError_t launch_pair_newton(const Geo& G, const double* R, float* Xs, size_t n, const Ctl* ctl,
                               cudaStream_t s) {
    pair_stage_newton_k<<<stream_blocks(n), NTHREADS, 0, s>>>(G, R, Xs, n, ctl);
    return cudaGetLastError();
}

template <typename TC>
cudaError_t launch_pair_store(const float* Xs, const TC* corr, const float* MX, float* Xbuf, float* Tbuf, size_t n,
                              int cap, int arnoldi, Ctl* ctl, cudaStream_t s) {
    pair_store_k<TC><<<stream_blocks(n), NTHREADS, 0, s>>>(Xs, corr, MX, Xbuf, Tbuf, n, cap, arnoldi, ctl);
    pair_commit_k<<<1, 1, 0, s>>>(cap, arnoldi, ctl);
    return cudaGetLastError();
}
template cudaError_t launch_pair_store<float>(const float*, const float*, const float*, float*, float*, size_t, int,
                                              int, Ctl*, cudaStream_t);
template cudaError_t launch_pair_store<double>(const float*, const double*, const float*, float*, float*, size_t,
                                               int, int, Ctl*, cudaStream_t);

cudaError_t launch_pc_eps(const float* z, size_t n, double* part, Ctl* ctl, cudaStream_t s) {
    pc_eps_k<<<stream_blocks(n), NTHREADS, 0, s>>>(z, n, part, ctl);
    return cudaGetLastError();
}

#define JF_INST(T)                                                                                     \
    template cudaError_t launch_arnoldi_a<T>(const T*, size_t, const T*, size_t, int, double*, Ctl*,  \
                                             cudaStream_t);                                            \
    template cudaError_t launch_arnoldi_b<T>(const T*, size_t, T*, size_t, int, const double*,        \
                                             double*, Ctl*, cudaStream_t);                             \
    template cudaError_t launch_arnoldi_c<T>(T*, size_t, const T*, size_t, int, int, const double*,   \
                                             Ctl*, cudaStream_t);                                      \
    template cudaError_t launch_update<T>(const T*, size_t, double*, T*, size_t, double*, Ctl*,       \
                                          cudaStream_t);                                               \
    template cudaError_t launch_cycle_init<T>(const Geo&, const double*, T*, double*, size_t, double, \
                                              int, int, Ctl*, cudaStream_t);                           \
    template cudaError_t launch_restart<T>(const Geo&, const double*, const T*, T*, size_t, int,      \
                                           double*, Ctl*, cudaStream_t, long long*);                  \
    template cudaError_t launch_newton_update<T>(const Geo&, double*, const double*, T*, size_t,      \
                                                 cudaStream_t);                                        \
    template cudaError_t launch_restart_residual<T>(const Geo&, const double*, const T*, T*, size_t,  \
                                                    double*, Ctl*, cudaStream_t);                      \
    template cudaError_t launch_left_scale<T>(const T*, T*, size_t, int, Ctl*, cudaStream_t);         \
    template cudaError_t launch_norm2<T>(const Geo&, const T*, size_t, int, int, double*, Ctl*,       \
                                         cudaStream_t);
JF_INST(float)
JF_INST(double)

template cudaError_t launch_convert<double, float>(const double*, float*, size_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, size_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, size_t, cudaStream_t);
template cudaError_t launch_rescale<double, float>(const Geo&, const double*, float*, size_t, int, cudaStream_t);
template cudaError_t launch_rescale<double, double>(const Geo&, const double*, double*, size_t, int, cudaStream_t);
template cudaError_t launch_rescale<float, double>(const Geo&, const float*, double*, size_t, int, cudaStream_t);

}  // namespace jfnk
