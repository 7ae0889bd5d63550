// Krylov kernels of libjfnk: restarted GMRES(m) with right preconditioning in
// the flexible (stored z_j) form, classical Gram-Schmidt applied twice.
//
// One Arnoldi step j (w = J z_j already formed) is three streaming passes over
// the basis V = [v_0 .. v_j]:
//   A:  h1 = V^T w                                  (multi-dot)
//   B:  w' = w - V h1 (stored over w),  h2 = V^T w',  ||w'||^2
//       last block: h = h1 + h2, h_{j+1,j} = sqrt(||w'||^2 - ||h2||^2), Givens
//       rotation of the Hessenberg column, residual estimate |g_{j+1}|,
//       stopping test and (when the cycle ends) the triangular solve for y
//   C:  v_{j+1} = (w' - V h2) / h_{j+1,j}             (multi-axpy + scale)
// The second projection is subtracted from the stored w', as in classical
// Gram-Schmidt applied twice: the rounding of w - V h1 is then part of what
// h2 removes, and the last rounding is relative to ||w'||, not ||w||.
// Reductions are two-stage and deterministic: every block writes its partial
// sums, the last block to finish adds them in a fixed order.  A thread
// accumulates its partial dot products in the basis precision over at most
// 64 vector elements (the grid grows with n), then the block and grid
// reductions run in float64.
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
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nvec; i += stride) {
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
    block_partials<NV, T>(acc_t, nv, part, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_PASSA], gridDim.x)) {
        __shared__ double tot[NV];
        final_sums(part, gridDim.x, nv, tot);
        for (int k = threadIdx.x; k < nv; k += blockDim.x) ctl->h1[k] = tot[k];
    }
}

// ---------------------------------------------------------------- pass B
// Serial Hessenberg / Givens update for column j (one thread).
__device__ void givens_update(Ctl* c, int j, int m, const double* h2, double wn2) {
    double col[KMAX + 1];
    double hh2 = 0.0;
    for (int k = 0; k <= j; ++k) {
        const double hk = c->h1[k] + h2[k];
        c->h2[k] = h2[k];              // pass C subtracts V h2 from the stored w'
        c->Hbar[k][j] = hk;
        col[k] = hk;
        hh2 += h2[k] * h2[k];
    }
    const double hn2 = wn2 - hh2;
    const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
    c->Hbar[j + 1][j] = hn;
    col[j + 1] = hn;
    for (int i = 0; i < j; ++i) {
        const double t = c->cs[i] * col[i] + c->sn[i] * col[i + 1];
        col[i + 1] = -c->sn[i] * col[i] + c->cs[i] * col[i + 1];
        col[i] = t;
    }
    double cs = 1.0, sn = 0.0;
    if (col[j + 1] != 0.0) {
        const double rho = hypot(col[j], col[j + 1]);
        cs = col[j] / rho;
        sn = col[j + 1] / rho;
    }
    c->cs[j] = cs;
    c->sn[j] = sn;
    for (int k = 0; k < j; ++k) c->Rt[k][j] = col[k];
    c->Rt[j][j] = cs * col[j] + sn * col[j + 1];
    const double gj = c->g[j];
    c->g[j + 1] = -sn * gj;
    c->g[j] = cs * gj;
    c->gres = fabs(c->g[j + 1]);
    c->iters += 1;
    const bool finite = isfinite(hn2) && isfinite(c->g[j + 1]) && isfinite(c->Rt[j][j]);
    const bool conv = fabs(c->g[j + 1]) <= c->target;
    const bool brk = hn == 0.0;
    c->inv_hn = hn > 0.0 ? 1.0 / hn : 0.0;
    if (!finite) {
        c->nan = 1;
        c->done = 1;
        c->k = 0;
        return;
    }
    if (conv || brk || j == m - 1) {
        const int k = j + 1;
        for (int i = k - 1; i >= 0; --i) {     // back substitution R y = g
            double s = c->g[i];
            for (int l = i + 1; l < k; ++l) s -= c->Rt[i][l] * c->y[l];
            c->y[i] = s / c->Rt[i][i];
        }
        c->k = k;
        c->converged = conv || brk;
        c->breakdown = brk && !conv;
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

// Pass B, split over KS lanes per element: w' = w - V h1 (stored over w),
// ||w'||^2 and h2 = V^T w'; the last block runs the Givens update.  Each lane
// keeps its CH basis entries in registers for both uses, so every basis vector
// is read from memory once; the next element's loads are issued before the
// current one is combined (software pipeline).
template <typename T, int NV>
__global__ void __launch_bounds__(NTHREADS, 2)
arnoldi_b(const T* __restrict__ V, size_t ldv, T* __restrict__ w, size_t n, int nv, int m,
          double* part, Ctl* ctl) {
    pdl_wait();
    if (ctl->done) return;
    constexpr int KS = 4, CH = NV / KS;
    __shared__ T h1s[NV];
    __shared__ T red[NV + 1][NTHREADS / 32];
    for (int k = threadIdx.x; k < NV; k += blockDim.x) h1s[k] = k < nv ? T(ctl->h1[k]) : T(0);
    __syncthreads();
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
    VT vn[CH], wn = zerov<VT>();
    if (g0 < nvec) {
        load_b<T, VT, CH>(V, ldv, g0, nv, q, vn);
        wn = reinterpret_cast<const VT*>(w)[g0];
    }
    for (size_t i = g0; i < nvec; i += gstride) {
        VT v[CH];
#pragma unroll
        for (int c = 0; c < CH; ++c) v[c] = vn[c];
        const VT wv = wn;
        const size_t inext = i + gstride;
        if (inext < nvec) {
            load_b<T, VT, CH>(V, ldv, inext, nv, q, vn);
            wn = reinterpret_cast<const VT*>(w)[inext];
        }
        work_b<T, VT, CH, KS>(v, wv, w, i, q, h1s, acc, accn);
    }
    for (size_t i = nvec * W + g0; i < n; i += gstride) {
        T v[CH];
        load_b<T, T, CH>(V, ldv, i, nv, q, v);
        work_b<T, T, CH, KS>(v, w[i], w, i, q, h1s, acc, accn);
    }
    pdl_trigger();
    // block sums: slot 0 = ||w'||^2, slot 1 + k = v_k . w' (fixed shuffle trees; float64 across warps)
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
    const int nw = blockDim.x >> 5;
    for (int k = threadIdx.x; k < nv + 1; k += blockDim.x) {
        double t = 0.0;
        for (int ww = 0; ww < nw; ++ww) t += (double)red[k][ww];
        part[(size_t)k * gridDim.x + blockIdx.x] = t;
        __threadfence();          // publish before the block's arrival is counted
    }
    if (arrive_last(&ctl->counter[CNT_PASSB], gridDim.x)) {
        __shared__ double tot[NV + 1];
        final_sums(part, gridDim.x, nv + 1, tot);
        if (threadIdx.x == 0) givens_update(ctl, nv - 1, m, tot + 1, tot[0]);
    }
}

// ---------------------------------------------------------------- pass C
template <typename T, int NV>
__global__ void __launch_bounds__(NTHREADS, 3)
arnoldi_c(T* __restrict__ V, size_t ldv, const T* __restrict__ w, size_t n, int nv, Ctl* ctl) {
    pdl_wait();
    if (ctl->done) return;
    using VT = typename V4<T>::type;
    constexpr int W = V4<T>::W;
    __shared__ T hs[NV];
    for (int k = threadIdx.x; k < nv; k += blockDim.x) hs[k] = T(ctl->h2[k]);
    __syncthreads();
    const T inv = T(ctl->inv_hn);
    const size_t nvec = n / W;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    T* vout = V + (size_t)nv * ldv;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nvec; i += stride) {
        VT wp = reinterpret_cast<const VT*>(w)[i];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            if (k < nv) wp = axpyv(wp, hs[k], reinterpret_cast<const VT*>(V + k * ldv)[i]);
        reinterpret_cast<VT*>(vout)[i] = scalev(wp, inv);
    }
    for (size_t i = nvec * W + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        T wp = w[i];
        for (int k = 0; k < nv; ++k) wp -= hs[k] * V[k * ldv + i];
        vout[i] = wp * inv;
    }
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
        const double y = k < K ? ctl->y[k] : 0.0;
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
        if (pc_none) ctl->eps_jv = sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2)));
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
        if (pc_none) ctl->eps_jv = sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2)));
    }
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
        }
    }
}

// ---------------------------------------------------------------- launchers

template <typename T>
cudaError_t launch_arnoldi_a(const T* V, size_t ldv, const T* w, size_t n, int nv, double* part,
                             Ctl* ctl, cudaStream_t s) {
    const int nb = std::max(dot_blocks(n / V4<T>::W), reduce_blocks(n / V4<T>::W));
    if (nv <= 8) return launch_pdl(arnoldi_a<T, 8>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, part, ctl);
    if (nv <= 16) return launch_pdl(arnoldi_a<T, 16>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, part, ctl);
    return launch_pdl(arnoldi_a<T, 32>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, part, ctl);
}

template <typename T>
cudaError_t launch_arnoldi_b(const T* V, size_t ldv, T* w, size_t n, int nv, int m,
                             double* part, Ctl* ctl, cudaStream_t s) {
    const int nb = reduce_blocks(n / V4<T>::W);
    if (nv <= 8) return launch_pdl(arnoldi_b<T, 8>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, m, part, ctl);
    if (nv <= 16) return launch_pdl(arnoldi_b<T, 16>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, m, part, ctl);
    return launch_pdl(arnoldi_b<T, 32>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, m, part, ctl);
}

template <typename T>
cudaError_t launch_arnoldi_c(T* V, size_t ldv, const T* w, size_t n, int nv, Ctl* ctl,
                             cudaStream_t s) {
    const int nb = dot_blocks(n / V4<T>::W);
    if (nv <= 8) return launch_pdl(arnoldi_c<T, 8>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, ctl);
    if (nv <= 16) return launch_pdl(arnoldi_c<T, 16>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, ctl);
    return launch_pdl(arnoldi_c<T, 32>, nb, NTHREADS, 0, s, V, ldv, w, n, nv, ctl);
}

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
    template cudaError_t launch_arnoldi_b<T>(const T*, size_t, T*, size_t, int, int, double*,         \
                                             Ctl*, cudaStream_t);                                      \
    template cudaError_t launch_arnoldi_c<T>(T*, size_t, const T*, size_t, int, Ctl*, cudaStream_t);  \
    template cudaError_t launch_update<T>(const T*, size_t, double*, T*, size_t, double*, Ctl*,       \
                                          cudaStream_t);                                               \
    template cudaError_t launch_cycle_init<T>(const Geo&, const double*, T*, double*, size_t, double, \
                                              int, int, Ctl*, cudaStream_t);                           \
    template cudaError_t launch_restart<T>(const Geo&, const double*, const T*, T*, size_t, int,      \
                                           double*, Ctl*, cudaStream_t, long long*);                  \
    template cudaError_t launch_newton_update<T>(const Geo&, double*, const double*, T*, size_t,      \
                                                 cudaStream_t);                                        \
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
