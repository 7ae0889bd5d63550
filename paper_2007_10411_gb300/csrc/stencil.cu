// 2-D stencil kernels of libjfnk: F(u), R(u), the Jacobian-vector product,
// the Smagorinsky eddy field, the field-block Chebyshev preconditioner and
// the budgets.
//
// Discretisation (Hossain & Alam):
//   * Deslauriers-Dubuc collocation derivative of order p = 2 (Section 2.3):
//     the 4-point interpolating scheme gives phi'(+-1) = -+2/3, phi'(+-2) = +-1/12,
//     i.e. D f_j = [2/3 (f_{j+1} - f_{j-1}) - 1/12 (f_{j+2} - f_{j-2})] / h.
//   * skew-symmetric convection C(u)phi = 1/2 D_j(u_j phi) + 1/2 u_j D_j phi (Section 2.2)
//     for every field;
//   * Eqs. ch2_28-ch2_30 with Laplacian-form eddy diffusion sum_j D_j(K D_j phi),
//     constant K_M, K_H (Table 1) or Smagorinsky nu = (Cs Delta)^2 sqrt(2 S:S),
//     K_M = nu, K_H = nu / Pr (Section 2.4);
//   * x periodic, z cell-centred with mirror ghosts (w odd, theta and p even,
//     u even for free slip / odd for no slip); the eddy field is mirrored even.
//
// Tiling: one CTA computes a TX x TZ tile of output points.  Stage 1 stages
// the four fields with a halo of 2r = 4 points in shared memory (periodic /
// mirror index mapping, coalesced along x); stage 2 forms the first
// derivatives of u, w, theta (and nu) on the tile plus a halo of r = 2;
// stage 3 assembles the fluxes, the second application of D and the
// point-wise terms, and writes coalesced rows.  Nothing but the inputs and
// the outputs touches HBM: the eddy viscosity and the derivatives live only
// in shared memory.
#include <math.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "kernels.h"

namespace jfnk {

constexpr int R = 2;          // derivative radius for p = 2
constexpr int HALO = 2 * R;   // input halo (derivative applied twice)

template <typename T> struct Tile;
template <> struct Tile<double> { static constexpr int TX = 32, TZ = 16; };
template <> struct Tile<float>  { static constexpr int TX = 64, TZ = 16; };
// Candidate tiles of the Jacobian-product and preconditioner kernels (float32
// path); jfnk_autotune times each on the handle's workload and keeps the
// fastest (Geo::tile_jv, Geo::tile_pc).  The float64 path uses the first entry.
template <int I> struct JvTile;          // float64 Jacobian product (jv_diff2d): entry 1
template <> struct JvTile<0> { static constexpr int TX = 32, TZ = 16; };
template <> struct JvTile<1> { static constexpr int TX = 32, TZ = 8; };
template <int I> struct JvcTile;         // float32 Jacobian product (jvc2d): tile and staging buffers
template <> struct JvcTile<0> { static constexpr int TX = 32, TZ = 16, NBUF = 1; };
template <> struct JvcTile<1> { static constexpr int TX = 32, TZ = 16, NBUF = 2; };
template <> struct JvcTile<2> { static constexpr int TX = 64, TZ = 8, NBUF = 1; };
template <> struct JvcTile<3> { static constexpr int TX = 32, TZ = 8, NBUF = 1; };
template <int I> struct PcTile;
template <> struct PcTile<0> { static constexpr int TX = 64, TZ = 16; };
template <> struct PcTile<1> { static constexpr int TX = 32, TZ = 16; };
template <> struct PcTile<2> { static constexpr int TX = 64, TZ = 8; };
template <> struct PcTile<3> { static constexpr int TX = 32, TZ = 8; };

// Explicitly rounded product and fused multiply-add: expressions written with
// them round the same way in every instantiation (tile shape) of a kernel.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename T>
__device__ __forceinline__ T dd(const T* s, int i, int st, T inv_h) {
    const T d1 = s[i + st] - s[i - st], d2 = s[i + 2 * st] - s[i - 2 * st];
    return rmul(rfma(T(2.0 / 3.0), d1, rmul(T(-1.0 / 12.0), d2)), inv_h);
}

// derivative of the point-wise product a*b
template <typename T>
__device__ __forceinline__ T ddp(const T* a, const T* b, int i, int st, T inv_h) {
    const T d1 = rfma(a[i + st], b[i + st], -rmul(a[i - st], b[i - st]));
    const T d2 = rfma(a[i + 2 * st], b[i + 2 * st], -rmul(a[i - 2 * st], b[i - 2 * st]));
    return rmul(rfma(T(2.0 / 3.0), d1, rmul(T(-1.0 / 12.0), d2)), inv_h);
}

// derivative of the flux K*g where K may be a constant (Kc) or an array
template <typename T, bool KARR>
__device__ __forceinline__ T ddk(const T* K, T Kc, const T* g, int i, int st, T inv_h) {
    if (KARR) return ddp(K, g, i, st, inv_h);
    return Kc * dd(g, i, st, inv_h);
}

// Source row / sign of a ghost-extended z index.  side: 0 interior, 1 bottom, 2 top.
__device__ __forceinline__ int mirror_z(int gz, int nz, int& side) {
    side = 0;
    if (gz < 0) { side = 1; return -1 - gz; }
    if (gz >= nz) { side = 2; return 2 * nz - 1 - gz; }
    return gz;
}

__device__ __forceinline__ int wrap_x(int gx, int nx) {
    if ((unsigned)gx < (unsigned)nx) return gx;        // interior: no division
    int r = gx % nx;
    return r < 0 ? r + nx : r;
}

template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int W = 4;
    __device__ static float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static float4 fma(float a, float4 x, float4 y) {
        return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
    }
    __device__ static float4 mul(float a, float4 x) { return make_float4(a * x.x, a * x.y, a * x.z, a * x.w); }
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int W = 2;
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double2 fma(double a, double2 x, double2 y) {
        return make_double2(::fma(a, x.x, y.x), ::fma(a, x.y, y.y));
    }
    __device__ static double2 mul(double a, double2 x) { return make_double2(a * x.x, a * x.y); }
};

// True when the whole x-range [x0 - HALO, x0 - HALO + SX) of a tile is inside the
// grid and rows start on 16-byte boundaries: the tile rows load as 16-byte vectors.
template <typename T>
__device__ __forceinline__ bool rows_vectorisable(const Geo& G, int x0, int SX) {
    return x0 - HALO >= 0 && x0 - HALO + SX <= G.nx && (G.nx % Vec16<T>::W) == 0;
}

// Stage 1: s[f][SZ][SX] <- (LOADMODE 0) u, (1) u + ev*v, (2) ev*v for fields
// f0 .. f0+NF-1, ghost-extended (periodic x, signed mirror z).
template <typename T, int LOADMODE, int NF = 4>
__device__ __forceinline__ void load_fields(T* s, const T* __restrict__ u, const T* __restrict__ v,
                                            const T (&ev)[4], const Geo& G, int x0, int z0,
                                            int SX, int SZ, int f0 = 0) {
    using VT = typename Vec16<T>::type;
    constexpr int VW = Vec16<T>::W;
    if (rows_vectorisable<T>(G, x0, SX)) {
        const int nch = SX / VW;
        const int total = nch * SZ;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int iz = idx / nch, c = idx - iz * nch;
            const int gz = z0 + iz - HALO;
            int side;
            const int sz = mirror_z(gz, G.nz, side);
            const bool ok = sz >= 0 && sz < G.nz;
            const size_t off = (size_t)sz * G.nx + (x0 - HALO + c * VW);
#pragma unroll
            for (int q = 0; q < NF; ++q) {
                const int f = f0 + q;
                VT val = Vec16<T>::zero();
                if (ok) {
                    const size_t o = (size_t)f * G.npt + off;
                    if (LOADMODE == 0) val = *reinterpret_cast<const VT*>(u + o);
                    else if (LOADMODE == 1)
                        val = Vec16<T>::fma(ev[f], *reinterpret_cast<const VT*>(v + o),
                                            *reinterpret_cast<const VT*>(u + o));
                    else val = Vec16<T>::mul(ev[f], *reinterpret_cast<const VT*>(v + o));
                    if (side == 1) val = Vec16<T>::mul(T(G.pb[f]), val);
                    else if (side == 2) val = Vec16<T>::mul(T(G.pt[f]), val);
                }
                *reinterpret_cast<VT*>(s + (q * SZ + iz) * SX + c * VW) = val;
            }
        }
        return;
    }
    const int total = SX * SZ;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int iz = idx / SX, ix = idx - iz * SX;
        const int gz = z0 + iz - HALO, gx = x0 + ix - HALO;
        int side;
        const int sz = mirror_z(gz, G.nz, side);
        const int sx = wrap_x(gx, G.nx);
        const bool ok = sz >= 0 && sz < G.nz;
        const size_t off = (size_t)sz * G.nx + sx;
#pragma unroll
        for (int q = 0; q < NF; ++q) {
            const int f = f0 + q;
            T val = T(0);
            if (ok) {
                const size_t o = (size_t)f * G.npt + off;
                if (LOADMODE == 0) val = u[o];
                else if (LOADMODE == 1) val = u[o] + ev[f] * v[o];
                else val = ev[f] * v[o];
                if (side == 1) val *= T(G.pb[f]);
                else if (side == 2) val *= T(G.pt[f]);
            }
            s[(q * SZ + iz) * SX + ix] = val;
        }
    }
}

// Work item w of a QZ x QX halo region -> (qz, qx): the first 32 * (QX / 32)
// columns of every row in 32-wide blocks (a warp stays inside one row, so its
// shared-memory taps are consecutive words and free of bank conflicts), then
// the remaining QX % 32 columns of all rows.
__device__ __forceinline__ void halo_item(int w, int QX, int QZ, int& qz, int& qx) {
    const int wide = QX & ~31, main = QZ * wide;
    if (w < main) {
        qz = w / wide;
        qx = w - qz * wide;
    } else {
        const int rem = QX - wide, r = w - main;
        qz = r / rem;
        qx = wide + (r - qz * rem);
    }
}

// Stage 2: first derivatives of u, w, theta on the halo-r region.
template <typename T>
__device__ __forceinline__ void first_derivs(const T* s1, T* d, int SX, int SZ, int QX, int QZ,
                                             T idx_, T idz_) {
    const int total = QX * QZ;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        int qz, qx;
        halo_item(w, QX, QZ, qz, qx);
        const int idx = qz * QX + qx;
        const int i1 = (qz + R) * SX + qx + R;
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const T* sf = s1 + f * SZ * SX;
            d[(2 * f) * total + idx] = dd(sf, i1, 1, idx_);
            d[(2 * f + 1) * total + idx] = dd(sf, i1, SX, idz_);
        }
    }
}

// Row of the halo-r region whose eddy value a ghost row takes (even mirror); -1 if unused.
__device__ __forceinline__ int eddy_row(int qz, int z0, int nz, int QZ) {
    const int gz = z0 + qz - R;
    int iq = qz;
    if (gz < 0) iq = (-1 - gz) - z0 + R;
    else if (gz >= nz) iq = (gz < nz + R) ? (2 * nz - 1 - gz) - z0 + R : -1;
    return (iq >= 0 && iq < QZ) ? iq : -1;
}

// Deardorff heat factor s (1 + a l(s)), l = min(Delta, c_l s) (c_l < 0: l = Delta).
template <typename T>
__device__ __forceinline__ T dd_heat(T s, T a, const Geo& G) {
    const T cls = rmul(T(G.dd_cl), s);
    const T l = G.dd_cl < 0.0 ? T(G.dd_delta) : (cls < T(G.dd_delta) ? cls : T(G.dd_delta));
    return rmul(s, rfma(a, l, T(1)));
}

template <typename T>
__device__ __forceinline__ T smag_nu(T ux, T uz, T wx, T wz, T cs2) {
    const T s13 = T(0.5) * (uz + wx);
    const T ss = ux * ux + wz * wz + T(2) * s13 * s13;
    return cs2 * sqrt(T(2) * ss);
}

// ============================================================================
// F, 2u/dt + F, residual and plain forward-difference Jv
// ============================================================================
template <typename T, int MODE, int SMAG>
__global__ void __launch_bounds__(NTHREADS)
stencil2d(Geo G, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ Fu,
          const double* __restrict__ f, T* __restrict__ out, T* __restrict__ out2,
          double* __restrict__ part, Ctl* ctl, int check_done) {
    constexpr int TX = Tile<T>::TX, TZ = Tile<T>::TZ;
    constexpr int SX = TX + 2 * HALO, SZ = TZ + 2 * HALO;
    constexpr int QX = TX + 2 * R, QZ = TZ + 2 * R;
    constexpr int QN = QX * QZ;
    if (MODE == MODE_JV && check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s1 = reinterpret_cast<T*>(smem_raw);
    T* d = s1 + 4 * SZ * SX;
    T* nu = d + 6 * QN;                  // Smagorinsky nu, or the strain s (Deardorff)
    T* gh = nu + QN;                     // Deardorff: s (1 + a_h l) and s (1 + a_z l)
    T* gH = gh + QN;
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ;
    const T idx_ = T(G.inv_dx), idz_ = T(G.inv_dz);

    T ev[4] = {T(0), T(0), T(0), T(0)};
    __shared__ double cfs[4];            // 1 / (eps scale_f), computed once per block
    __shared__ T evs[4];                 // eps scale_f
    if (MODE == MODE_JV) {
        if (threadIdx.x < 4) {
            const double e = ctl->eps_jv * G.scale[threadIdx.x];
            evs[threadIdx.x] = T(e);
            cfs[threadIdx.x] = e != 0.0 ? 1.0 / e : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) ev[q] = evs[q];
        load_fields<T, 1>(s1, u, v, ev, G, x0, z0, SX, SZ);
    } else {
        load_fields<T, 0>(s1, u, v, ev, G, x0, z0, SX, SZ);
    }
    __syncthreads();
    first_derivs(s1, d, SX, SZ, QX, QZ, idx_, idz_);
    __syncthreads();
    if (SMAG) {
        const T cs2 = SMAG == 2 ? T(1) : T(G.cs2);     // Deardorff: the strain s = sqrt(2 S:S) itself
        for (int w = threadIdx.x; w < QN; w += blockDim.x) {
            int qz, qx;
            halo_item(w, QX, QZ, qz, qx);
            const int idx = qz * QX + qx;
            const int iq = eddy_row(qz, z0, G.nz, QZ);
            T val = T(0);
            if (iq >= 0) {
                const int q = iq * QX + qx;
                val = smag_nu(d[q], d[QN + q], d[2 * QN + q], d[3 * QN + q], cs2);
            }
            nu[idx] = val;
            if (SMAG == 2) {
                gh[idx] = dd_heat(val, T(G.dd_ah), G);
                gH[idx] = dd_heat(val, T(G.dd_az), G);
            }
        }
        __syncthreads();
    }

    const T* su = s1;
    const T* sw = s1 + SZ * SX;
    const T* st = s1 + 2 * SZ * SX;
    const T* sp = s1 + 3 * SZ * SX;
    const T* dux = d;
    const T* duz = d + QN;
    const T* dwx = d + 2 * QN;
    const T* dwz = d + 3 * QN;
    const T* dtx = d + 4 * QN;
    const T* dtz = d + 5 * QN;
    const T KMc = T(G.K_M), KHc = T(G.K_H), iPr = T(G.inv_Pr);
    const T th0 = T(G.theta0);

    double acc[2] = {0.0, 0.0};
    for (int idx = threadIdx.x; idx < TX * TZ; idx += blockDim.x) {
        const int tz = idx / TX, tx = idx - tz * TX;
        const int gz = z0 + tz, gx = x0 + tx;
        if (gz >= G.nz || gx >= G.nx) continue;
        const int i1 = (tz + HALO) * SX + tx + HALO;
        const int q = (tz + R) * QX + tx + R;
        const T uc = su[i1], wc = sw[i1], tc = st[i1], pc = sp[i1];
        const T px = dd(sp, i1, 1, idx_), pz = dd(sp, i1, SX, idz_);
        // skew-symmetric convection of every field
        const T cu = T(0.5) * (ddp(su, su, i1, 1, idx_) + ddp(sw, su, i1, SX, idz_)) +
                     T(0.5) * (uc * dux[q] + wc * duz[q]);
        const T cw = T(0.5) * (ddp(su, sw, i1, 1, idx_) + ddp(sw, sw, i1, SX, idz_)) +
                     T(0.5) * (uc * dwx[q] + wc * dwz[q]);
        const T ct = T(0.5) * (ddp(su, st, i1, 1, idx_) + ddp(sw, st, i1, SX, idz_)) +
                     T(0.5) * (uc * dtx[q] + wc * dtz[q]);
        const T cp = T(0.5) * (ddp(su, sp, i1, 1, idx_) + ddp(sw, sp, i1, SX, idz_)) +
                     T(0.5) * (uc * px + wc * pz);
        // eddy diffusion sum_j D_j(K D_j phi)
        T du, dw, dt_;
        if (SMAG == 2) {
            // anisotropic: D_x(K_m D_x phi) + D_z(K_M D_z phi), heat with K_h, K_H
            const T cm = T(G.dd_cm), cM = T(G.dd_cM);
            du = cm * ddp(nu, dux, q, 1, idx_) + cM * ddp(nu, duz, q, QX, idz_);
            dw = cm * ddp(nu, dwx, q, 1, idx_) + cM * ddp(nu, dwz, q, QX, idz_);
            dt_ = cm * ddp(gh, dtx, q, 1, idx_) + cM * ddp(gH, dtz, q, QX, idz_);
        } else if (SMAG) {
            du = ddp(nu, dux, q, 1, idx_) + ddp(nu, duz, q, QX, idz_);
            dw = ddp(nu, dwx, q, 1, idx_) + ddp(nu, dwz, q, QX, idz_);
            dt_ = iPr * (ddp(nu, dtx, q, 1, idx_) + ddp(nu, dtz, q, QX, idz_));
        } else {
            du = KMc * (dd(dux, q, 1, idx_) + dd(duz, q, QX, idz_));
            dw = KMc * (dd(dwx, q, 1, idx_) + dd(dwz, q, QX, idz_));
            dt_ = KHc * (dd(dtx, q, 1, idx_) + dd(dtz, q, QX, idz_));
        }
        T Fv[4];
        Fv[0] = -cu - th0 * px + du;
        Fv[1] = -cw - th0 * pz + dw + T(G.g) * tc / th0;
        Fv[2] = -ct - T(G.beta) * wc + dt_;
        if (G.heat != nullptr && gz == 0) Fv[2] += T(G.heat[gx] * G.heat_coef);
        Fv[3] = -cp - T(G.gamma_p) * (T(G.pbar) + pc) * (dux[q] + dwz[q]);

        const size_t off = (size_t)gz * G.nx + gx;
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) {
            const size_t o = (size_t)fl * G.npt + off;
            if (MODE == MODE_F) {
                out[o] = Fv[fl];
            } else if (MODE == MODE_RHS) {
                out[o] = T(G.two_over_dt * (double)u[o] + (double)Fv[fl]);
            } else if (MODE == MODE_RHSRES) {
                // at u = u^n the residual 2u/dt - F(u) - f with f = 2u/dt + F(u) is -2 F(u)
                const double uo = (double)u[o];
                const double Fd = (double)Fv[fl];
                out[o] = T(G.two_over_dt * uo + Fd);
                const double Rv = -2.0 * Fd;
                out2[o] = T(Rv);
                const double rs = Rv * G.inv_scale[fl], us = uo * G.inv_scale[fl];
                acc[0] += rs * rs;
                acc[1] += us * us;
            } else if (MODE == MODE_RES) {
                const double uo = (double)u[o];
                const double Rv = G.two_over_dt * uo - (double)Fv[fl] - f[o];
                out[o] = T(Rv);
                if (out2 != nullptr) out2[o] = Fv[fl];
                const double rs = Rv * G.inv_scale[fl], us = uo * G.inv_scale[fl];
                acc[0] += rs * rs;
                acc[1] += us * us;
            } else {  // MODE_JV: w_hat = 2 v_hat/dt - (F(u + eps V) - F(u)) / (eps scale)
                const double vh = (double)v[o];
                const double diff = (double)Fv[fl] - (double)Fu[o];
                out[o] = T(G.two_over_dt * vh - diff * cfs[fl]);
            }
        }
    }
    if (MODE == MODE_RES || MODE == MODE_RHSRES) {
        const int nblk = gridDim.x * gridDim.y;
        const int blk = blockIdx.y * gridDim.x + blockIdx.x;
        block_partials<2>(acc, 2, part, nblk, blk);
        if (arrive_last(&ctl->counter[CNT_STENCIL], nblk)) {
            __shared__ double tot[2];
            final_sums(part, nblk, 2, tot);
            if (threadIdx.x == 0) {
                ctl->res2 = tot[0];
                ctl->unorm2 = tot[1];
                ctl->nan = !(isfinite(tot[0]) && isfinite(tot[1]));
            }
        }
    }
}

// ============================================================================
// Asynchronous tile staging (cp.async, sm_80 and later): the copies of the
// next tile land in shared memory while the current tile is computed.
// 16-byte chunks for rows inside the grid, element copies at the periodic x
// seam; a source size of 0 zero-fills (rows beyond one mirror reflection).
// ============================================================================
__device__ __forceinline__ void cpa16(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
template <int B>
__device__ __forceinline__ void cpa_elem(void* dst, const void* src, int src_bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(B), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Issue the copies of the ghost-extended u and v tiles (four fields each) into
// s[0..4) and s[4..8) (planes of SZ x SX).  jv_stage_fix walks the same chunk
// -> thread assignment once the copies have landed, so a thread only touches
// what it copied itself: mirror signs on ghost rows and the eps scale on v,
// in the order load_fields applies them.
template <typename T>
__device__ __forceinline__ void jv_stage_issue(T* s, const T* __restrict__ u, const T* __restrict__ v,
                                               const Geo& G, int x0, int z0, int SX, int SZ) {
    constexpr int VW = Vec16<T>::W;
    const int plane = SZ * SX;
    if (rows_vectorisable<T>(G, x0, SX)) {
        const int nch = SX / VW;
        const int total = nch * SZ;
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int iz = idx / nch, c = idx - iz * nch;
            int side;
            const int sz = mirror_z(z0 + iz - HALO, G.nz, side);
            const bool ok = sz >= 0 && sz < G.nz;
            const size_t off = ok ? (size_t)sz * G.nx + (x0 - HALO + c * VW) : 0;
            T* d = s + iz * SX + c * VW;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                cpa16(d + f * plane, u + (size_t)f * G.npt + off, ok ? 16 : 0);
                cpa16(d + (4 + f) * plane, v + (size_t)f * G.npt + off, ok ? 16 : 0);
            }
        }
        return;
    }
    const int total = SX * SZ;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int iz = idx / SX, ix = idx - iz * SX;
        int side;
        const int sz = mirror_z(z0 + iz - HALO, G.nz, side);
        const bool ok = sz >= 0 && sz < G.nz;
        const size_t off = ok ? (size_t)sz * G.nx + wrap_x(x0 + ix - HALO, G.nx) : 0;
        T* d = s + iz * SX + ix;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            cpa_elem<sizeof(T)>(d + f * plane, u + (size_t)f * G.npt + off, ok ? (int)sizeof(T) : 0);
            cpa_elem<sizeof(T)>(d + (4 + f) * plane, v + (size_t)f * G.npt + off, ok ? (int)sizeof(T) : 0);
        }
    }
}

template <typename T>
__device__ __forceinline__ void jv_stage_fix(T* s, const T (&ev)[4], const Geo& G, int x0, int z0, int SX,
                                             int SZ) {
    using VT = typename Vec16<T>::type;
    constexpr int VW = Vec16<T>::W;
    const int plane = SZ * SX;
    const bool vec = rows_vectorisable<T>(G, x0, SX);
    const int per = vec ? SX / VW : SX;
    const int total = per * SZ;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int iz = idx / per, c = idx - iz * per;
        int side;
        const int sz = mirror_z(z0 + iz - HALO, G.nz, side);
        if (sz < 0 || sz >= G.nz) continue;       // zero-filled row
        T* d = s + iz * SX + (vec ? c * VW : c);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const T sg = side == 1 ? T(G.pb[f]) : side == 2 ? T(G.pt[f]) : T(1);
            if (vec) {
                VT* pu = reinterpret_cast<VT*>(d + f * plane);
                VT* pv = reinterpret_cast<VT*>(d + (4 + f) * plane);
                if (side) *pu = Vec16<T>::mul(sg, *pu);
                VT b = Vec16<T>::mul(ev[f], *pv);
                if (side) b = Vec16<T>::mul(sg, b);
                *pv = b;
            } else {
                if (side) d[f * plane] *= sg;
                T b = ev[f] * d[(4 + f) * plane];
                if (side) b *= sg;
                d[(4 + f) * plane] = b;
            }
        }
    }
}

// ============================================================================
// Mixed-path Jv: the forward difference F(u + eps V) - F(u) with every term
// expanded as a difference (a = u, b = eps V, a' = a + b), e.g.
//   a'_j phi' - a_j phi = a_j b_phi + b_j phi',
//   (pbar + p') div a' - (pbar + p) div a = (pbar + p') div b + b_p div a,
//   nu(a') - nu(a) = (Cs Delta)^2 2 (S':S' - S:S) / (sqrt(2 S':S') + sqrt(2 S:S)),
// so the float32 result carries float32 relative accuracy on the difference
// itself instead of on F.  Same quantity as the forward difference of Eq. fd.
// ============================================================================
//
// Persistent and pipelined (NBUF = 2): a CTA walks the tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...; the cp.async copies of tile t + gridDim.x go
// into the second staging buffer while tile t is computed, so the staging
// latency hides behind the derivative and flux stages.  NBUF = 1 stages each
// tile before computing it (one tile per CTA, the float64 path).
template <typename T, int SMAG, int TX, int TZ, int NBUF>
__global__ void __launch_bounds__(NTHREADS)
jv_diff2d(Geo G, const T* __restrict__ u, const T* __restrict__ v, T* __restrict__ out,
          const double* part, Ctl* ctl, int check_done) {
    constexpr int SX = TX + 2 * HALO, SZ = TZ + 2 * HALO;
    constexpr int QX = TX + 2 * R, QZ = TZ + 2 * R;
    constexpr int QN = QX * QZ;
    constexpr int STG = 8 * SZ * SX;
    pdl_wait();
    if (check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* stg = reinterpret_cast<T*>(smem_raw);
    T* da = stg + NBUF * STG;
    T* db = da + 6 * QN;
    T* Ka = db + 6 * QN;
    T* dK = Ka + QN;
    const int ntx = (G.nx + TX - 1) / TX;
    const int ntiles = ntx * ((G.nz + TZ - 1) / TZ);
    const T idx_ = T(G.inv_dx), idz_ = T(G.inv_dz);
    int t = blockIdx.x;
    if (t < ntiles) jv_stage_issue(stg, u, v, G, (t % ntx) * TX, (t / ntx) * TZ, SX, SZ);
    cpa_commit();
    // the step, while the first tile's copies are in flight
    const double eps = pending_eps(ctl, part);
    __shared__ T cfs[4];                 // 1 / (eps scale_f), computed once per block
    __shared__ T evs[4];                 // eps scale_f
    if (threadIdx.x < 4) {
        const double e = eps * G.scale[threadIdx.x];
        evs[threadIdx.x] = T(e);
        cfs[threadIdx.x] = T(e != 0.0 ? 1.0 / e : 0.0);
    }
    __syncthreads();
    T ev[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) ev[q] = evs[q];
    for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
    const int x0 = (t % ntx) * TX, z0 = (t / ntx) * TZ;
    T* sa = stg + (NBUF == 2 ? (it & 1) * STG : 0);
    T* sb = sa + 4 * SZ * SX;
    // the direction at this thread's outputs (consumed at the end of the tile)
    constexpr int NOUT = (TX * TZ + NTHREADS - 1) / NTHREADS;
    T vout[NOUT][4];
#pragma unroll
    for (int q = 0; q < NOUT; ++q) {
        const int idx = threadIdx.x + q * NTHREADS;
        const int tz = idx / TX, tx = idx - tz * TX;
        const int gz = z0 + tz, gx = x0 + tx;
        const bool ok = idx < TX * TZ && gz < G.nz && gx < G.nx;
#pragma unroll
        for (int fl = 0; fl < 4; ++fl)
            vout[q][fl] = ok ? v[(size_t)fl * G.npt + (size_t)gz * G.nx + gx] : T(0);
    }
    if (NBUF == 2) {
        const int tn = t + gridDim.x;
        if (tn < ntiles)
            jv_stage_issue(stg + ((it + 1) & 1) * STG, u, v, G, (tn % ntx) * TX, (tn / ntx) * TZ, SX, SZ);
        cpa_commit();
        cpa_wait<1>();
    } else {
        cpa_wait<0>();
    }
    jv_stage_fix(sa, ev, G, x0, z0, SX, SZ);
    __syncthreads();
    first_derivs(sa, da, SX, SZ, QX, QZ, idx_, idz_);
    first_derivs(sb, db, SX, SZ, QX, QZ, idx_, idz_);
    __syncthreads();
    if (SMAG) {
        const T cs2 = T(G.cs2);
        for (int w = threadIdx.x; w < QN; w += blockDim.x) {
            int qz, qx;
            halo_item(w, QX, QZ, qz, qx);
            const int idx = qz * QX + qx;
            const int iq = eddy_row(qz, z0, G.nz, QZ);
            T ka = T(0), dk = T(0);
            if (iq >= 0) {
                const int q = iq * QX + qx;
                const T aux = da[q], auz = da[QN + q], awx = da[2 * QN + q], awz = da[3 * QN + q];
                const T bux = db[q], buz = db[QN + q], bwx = db[2 * QN + q], bwz = db[3 * QN + q];
                const T a13 = T(0.5) * (auz + awx), b13 = T(0.5) * (buz + bwx);
                const T ssa = aux * aux + awz * awz + T(2) * a13 * a13;
                // S':S' - S:S = (2 S + S_b) : S_b
                const T dss = (T(2) * aux + bux) * bux + (T(2) * awz + bwz) * bwz +
                              T(2) * (T(2) * a13 + b13) * b13;
                const T na = sqrt(T(2) * ssa);
                const T np = sqrt(T(2) * (ssa + dss) > T(0) ? T(2) * (ssa + dss) : T(0));
                ka = cs2 * na;
                const T den = na + np;
                dk = den > T(0) ? cs2 * T(2) * dss / den : T(0);
            }
            Ka[idx] = ka;
            dK[idx] = dk;
        }
        __syncthreads();
    }
    const T* au = sa; const T* aw = sa + SZ * SX; const T* at = sa + 2 * SZ * SX; const T* ap = sa + 3 * SZ * SX;
    const T* bu = sb; const T* bw = sb + SZ * SX; const T* bt = sb + 2 * SZ * SX; const T* bp = sb + 3 * SZ * SX;
    const T KMc = T(G.K_M), KHc = T(G.K_H), iPr = T(G.inv_Pr), th0 = T(G.theta0);

#pragma unroll
    for (int qo = 0; qo < NOUT; ++qo) {
        const int idx = threadIdx.x + qo * NTHREADS;
        if (idx >= TX * TZ) break;
        const int tz = idx / TX, tx = idx - tz * TX;
        const int gz = z0 + tz, gx = x0 + tx;
        if (gz >= G.nz || gx >= G.nx) continue;
        const int i1 = (tz + HALO) * SX + tx + HALO;
        const int q = (tz + R) * QX + tx + R;
        const T auc = au[i1], awc = aw[i1], apc = ap[i1];
        const T buc = bu[i1], bwc = bw[i1], btc = bt[i1], bpc = bp[i1];
        const T apx = dd(ap, i1, 1, idx_), apz = dd(ap, i1, SX, idz_);
        const T bpx = dd(bp, i1, 1, idx_), bpz = dd(bp, i1, SX, idz_);
        T dF[4];
        // convection differences: 1/2 D_j(a_j b_phi + b_j phi') + 1/2 (a_j D b_phi + b_j D phi')
        const T* as[4] = {au, aw, at, ap};
        const T* bs[4] = {bu, bw, bt, bp};
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) {
            const T* A = as[fl];
            const T* B = bs[fl];
            T fx = T(0), fz = T(0);
#pragma unroll
            for (int l = 1; l <= 2; ++l) {
                const T c = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
                const int ip = i1 + l, im = i1 - l;
                const int kp = i1 + l * SX, km = i1 - l * SX;
                fx += c * ((au[ip] * B[ip] + bu[ip] * (A[ip] + B[ip])) -
                           (au[im] * B[im] + bu[im] * (A[im] + B[im])));
                fz += c * ((aw[kp] * B[kp] + bw[kp] * (A[kp] + B[kp])) -
                           (aw[km] * B[km] + bw[km] * (A[km] + B[km])));
            }
            T dax, daz, dbx, dbz;
            if (fl < 3) {
                dax = da[(2 * fl) * QN + q]; daz = da[(2 * fl + 1) * QN + q];
                dbx = db[(2 * fl) * QN + q]; dbz = db[(2 * fl + 1) * QN + q];
            } else {
                dax = apx; daz = apz; dbx = bpx; dbz = bpz;
            }
            const T adv = auc * dbx + awc * dbz + buc * (dax + dbx) + bwc * (daz + dbz);
            dF[fl] = -(T(0.5) * (fx * idx_ + fz * idz_) + T(0.5) * adv);
        }
        // diffusion differences: D_j(K_a D_j b_phi + dK D_j phi')
#pragma unroll
        for (int fl = 0; fl < 3; ++fl) {
            const T* dax = da + (2 * fl) * QN; const T* daz = da + (2 * fl + 1) * QN;
            const T* dbx = db + (2 * fl) * QN; const T* dbz = db + (2 * fl + 1) * QN;
            T sx = T(0), sz = T(0);
            const T kc = fl == 2 ? KHc : KMc;
#pragma unroll
            for (int l = 1; l <= 2; ++l) {
                const T c = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
                const int xp = q + l, xm = q - l, zp = q + l * QX, zm = q - l * QX;
                if (SMAG) {
                    sx += c * ((Ka[xp] * dbx[xp] + dK[xp] * (dax[xp] + dbx[xp])) -
                               (Ka[xm] * dbx[xm] + dK[xm] * (dax[xm] + dbx[xm])));
                    sz += c * ((Ka[zp] * dbz[zp] + dK[zp] * (daz[zp] + dbz[zp])) -
                               (Ka[zm] * dbz[zm] + dK[zm] * (daz[zm] + dbz[zm])));
                } else {
                    sx += c * (dbx[xp] - dbx[xm]);
                    sz += c * (dbz[zp] - dbz[zm]);
                }
            }
            T dif = sx * idx_ + sz * idz_;
            if (SMAG) { if (fl == 2) dif *= iPr; } else dif *= kc;
            dF[fl] += dif;
        }
        dF[0] += -th0 * bpx;
        dF[1] += -th0 * bpz + T(G.g) * btc / th0;
        dF[2] += -T(G.beta) * bwc;
        const T diva = da[q] + da[3 * QN + q];
        const T divb = db[q] + db[3 * QN + q];
        dF[3] += -T(G.gamma_p) * ((T(G.pbar) + apc + bpc) * divb + bpc * diva);

        const size_t off = (size_t)gz * G.nx + gx;
#pragma unroll
        for (int fl = 0; fl < 4; ++fl) {
            const size_t o = (size_t)fl * G.npt + off;
            // the difference dF is already free of cancellation: the quotient
            // and the 2 v/dt term need no wider type than the result
            out[o] = T(G.two_over_dt) * vout[qo][fl] - dF[fl] * cfs[fl];
        }
    }
    __syncthreads();     // staging buffer and derivative arrays are reused by the next tile
    if (NBUF == 1) {
        const int tn = t + gridDim.x;
        if (tn < ntiles) jv_stage_issue(stg, u, v, G, (tn % ntx) * TX, (tn / ntx) * TZ, SX, SZ);
        cpa_commit();
    }
    }
}

// ============================================================================
// Mixed-path Jv, compute-once form (float32 path).
//
// Same quantity as jv_diff2d, organised so that every flux is formed once per
// point and only then differentiated.  With a = u and b = eps V (per field
// eps scale_f), the difference of F(a + b) - F(a) is, term by term,
//   convection  1/2 [D_x P_phi + D_z Q_phi] + 1/2 adv_phi,
//               P_phi = a_u b_phi + b_u (a_phi + b_phi)   (x-flux difference)
//               Q_phi = a_w b_phi + b_w (a_phi + b_phi)   (z-flux difference)
//               adv_phi = a_u D_x b_phi + a_w D_z b_phi + b_u D_x phi' + b_w D_z phi'
//   diffusion   D_x Fx_phi + D_z Fz_phi,
//               Fx_phi = K_a D_x b_phi + dK D_x phi'  (dK = K(a + b) - K(a), cancellation-free),
//   point-wise  pressure gradient, buoyancy, stratification, (pbar + p) div u,
// with phi' = a_phi + b_phi.  Phase 1 stages u and the raw direction v of a
// TX x TZ tile with a halo of 4 (cp.async, the next tile's copies in flight
// while this one is computed; the eps scale is applied in registers, so only
// ghost rows need a pass over the staged planes, for the mirror signs).
// Phase 2 forms, at every point where they are differentiated, the x-fluxes
// P, Fx (tile rows, columns -2 .. TX+1) and the z-fluxes Q, Fz (rows -2 ..
// TZ+1, tile columns), and, at the tile's own points, the point-wise part S
// (kept in registers).  Phase 3 differentiates the fluxes and writes Jv.
// Phases 2 and 3 give a thread the same PPT vertically adjacent points of
// one column (warps run along x: conflict-free shared-memory rows).  Every
// value at a point is computed by the same expression whatever the tile
// shape, so all shapes give bitwise the same result.
// The eddy coefficient at a ghost row is the mirror image of the interior
// value (K mirrored even): the Smagorinsky step of a flux point in a ghost
// row is evaluated at its image row.
// ============================================================================
template <int TX, int TZ>
struct JvcShape {
    static constexpr int SX = TX + 2 * HALO, SZ = TZ + 2 * HALO;
    static constexpr int PLANE = SX * SZ;
    static constexpr int STG = 8 * PLANE;                 // u (planes 0-3) and raw v (planes 4-7)
    static constexpr int PXW = TX + 2 * R;                // x-flux rows: columns -2 .. TX+1
    static constexpr int PXN = TZ * PXW;                  // per flux field
    static constexpr int QZN = (TZ + 2 * R) * TX;         // z-flux columns: rows -2 .. TZ+1
    static constexpr int PPT = TX * TZ / NTHREADS;        // points per thread (one column, PPT rows)
    static constexpr int NARM = 4 * TX + 4 * TZ;          // z-arm items, then x-arm items
    static_assert(NTHREADS % TX == 0 && PPT * (NTHREADS / TX) == TZ && PPT >= 1, "tile / thread mapping");
    static constexpr size_t smem(int nbuf) { return sizeof(float) * ((size_t)nbuf * STG + 7 * PXN + 7 * QZN); }
};

// Tile row (in staged coordinates, relative to the tile origin) whose eddy
// value a flux point in tile row iz takes: its mirror image where the global
// row is a ghost row (-2, -1 or nz, nz+1), else itself.
__device__ __forceinline__ int jvc_smag_row(int iz, int z0, int nz) {
    const int gz = z0 + iz;
    if (gz < 0) return (-1 - gz) - z0;
    if (gz >= nz && gz <= nz + 1) return (2 * nz - 1 - gz) - z0;
    return iz;
}

struct JvcConst {
    float ev[4];        // eps scale_f: b = ev * v
    float idx, idz;
    float cs2, iPr, KM, KH;
    float cm, cM, cl, dlt, ah, az;   // Deardorff constants (Geo::dd_*)
};

// The flux and derivative arithmetic of jvc2d is written with explicitly
// rounded operations (no contraction left to the compiler), so a flux formed
// in the tile centre and the same flux formed in a neighbouring tile's arm
// are bitwise equal, and every tile shape gives the same result.
// w1 = (2/3)/h, w2 = -(1/12)/h (Geo::fx1 .. fz2)
__device__ __forceinline__ float ddf(const float* s, int i, int st, float w1, float w2) {
    const float d1 = __fsub_rn(s[i + st], s[i - st]), d2 = __fsub_rn(s[i + 2 * st], s[i - 2 * st]);
    return __fmaf_rn(w1, d1, __fmul_rn(w2, d2));
}
// a0 b + b0 (a + b): the flux difference a'_j phi' - a_j phi
__device__ __forceinline__ float flux_diff(float a0, float b0, float a, float b) {
    return __fmaf_rn(a0, b, __fmul_rn(b0, __fadd_rn(a, b)));
}
// K b' + dK (a' + b'): the diffusive flux difference
__device__ __forceinline__ float kflux_diff(float kk, float dk, float da, float db) {
    return __fmaf_rn(kk, db, __fmul_rn(dk, __fadd_rn(da, db)));
}

// The strain magnitude s = sqrt(2 S:S) at a, at a' = a + b, and their
// difference ds = s' - s in cancellation-free form, from the velocity
// gradients of a (ux, uz, wx, wz) and of b.
__device__ __forceinline__ void jvc_strain(float aux, float auz, float awx, float awz, float bux, float buz,
                                           float bwx, float bwz, float& sa, float& sp, float& ds) {
    const float a13 = __fmul_rn(0.5f, __fadd_rn(auz, awx)), b13 = __fmul_rn(0.5f, __fadd_rn(buz, bwx));
    const float ssa = __fmaf_rn(aux, aux, __fmaf_rn(awz, awz, __fmul_rn(2.f, __fmul_rn(a13, a13))));
    // S':S' - S:S = (2 S + S_b) : S_b
    const float dss = __fmaf_rn(__fmaf_rn(2.f, aux, bux), bux,
                                __fmaf_rn(__fmaf_rn(2.f, awz, bwz), bwz,
                                          __fmul_rn(2.f, __fmul_rn(__fmaf_rn(2.f, a13, b13), b13))));
    // square roots and the quotient by the special-function unit (x rsqrt(x), a / b via
    // the approximate reciprocal): a few ulp, deterministic
    const float s1 = __fmul_rn(2.f, ssa);
    sa = s1 > 0.f ? __fmul_rn(s1, rsqrtf(s1)) : 0.f;
    const float s2 = __fmul_rn(2.f, __fadd_rn(ssa, dss));
    sp = s2 > 0.f ? __fmul_rn(s2, rsqrtf(s2)) : 0.f;
    // s' - s = 2 (S':S' - S:S) / (s' + s)
    const float den = __fadd_rn(sa, sp);
    ds = den > 0.f ? __fdividef(__fmul_rn(2.f, dss), den) : 0.f;
}

// Deardorff heat factor g(s) = s (1 + a l(s)), l = min(Delta, c_l s), at s and
// its difference g(s') - g(s) = ds (1 + a l') + a s (l' - l), with l' - l = c_l ds
// where neither side is capped (0 where both are; direct where they straddle).
__device__ __forceinline__ void jvc_heat(float sa, float sp, float ds, float a, const JvcConst& k, float& g,
                                         float& dg) {
    float la = k.dlt, lp = k.dlt, dl = 0.f;
    if (k.cl >= 0.f) {
        const float ta = __fmul_rn(k.cl, sa), tp = __fmul_rn(k.cl, sp);
        la = ta < k.dlt ? ta : k.dlt;
        lp = tp < k.dlt ? tp : k.dlt;
        if (ta < k.dlt && tp < k.dlt) dl = __fmul_rn(k.cl, ds);
        else if (ta < k.dlt || tp < k.dlt) dl = __fsub_rn(lp, la);
    }
    g = __fmul_rn(sa, __fmaf_rn(a, la, 1.f));
    dg = __fmaf_rn(ds, __fmaf_rn(a, lp, 1.f), __fmul_rn(__fmul_rn(a, sa), dl));
}

// Phase 2 at one point.  i: staged index of the point; is: staged index of the
// point whose eddy coefficient it takes (its image in a ghost row).  XF: the
// x-fluxes P, Fx; ZF: the z-fluxes Q, Fz; CEN: also the point-wise part S.
template <int SMAG, bool XF, bool ZF, bool CEN, int SX, int PLANE>
__device__ __forceinline__ void jvc_point(const float* __restrict__ st, int i, int is, const JvcConst& k,
                                          const Geo& G, float (&P)[4], float (&Fx)[3], float (&Q)[4],
                                          float (&Fz)[3], float (&S)[4], float (&vraw)[4]) {
    const float* A = st;                 // a planes 0..3
    const float* V = st + 4 * PLANE;     // raw v planes 0..3
    float a[4], b[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        a[f] = A[f * PLANE + i];
        vraw[f] = V[f * PLANE + i];
        b[f] = __fmul_rn(k.ev[f], vraw[f]);
    }
    // first derivatives at the point (b-derivatives scaled by ev in registers)
    constexpr bool DXUW = XF || CEN || SMAG, DZUW = ZF || CEN || SMAG;
    constexpr bool DXT = XF || CEN, DZT = ZF || CEN;
    float dax[4] = {0.f, 0.f, 0.f, 0.f}, daz[4] = {0.f, 0.f, 0.f, 0.f};
    float dbx[4] = {0.f, 0.f, 0.f, 0.f}, dbz[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const bool wx = f < 2 ? DXUW : (f == 2 ? DXT : CEN);
        const bool wz = f < 2 ? DZUW : (f == 2 ? DZT : CEN);
        if (wx) {
            dax[f] = ddf(A + f * PLANE, i, 1, G.fx1, G.fx2);
            dbx[f] = __fmul_rn(k.ev[f], ddf(V + f * PLANE, i, 1, G.fx1, G.fx2));
        }
        if (wz) {
            daz[f] = ddf(A + f * PLANE, i, SX, G.fz1, G.fz2);
            dbz[f] = __fmul_rn(k.ev[f], ddf(V + f * PLANE, i, SX, G.fz1, G.fz2));
        }
    }
    // exchange coefficients along x and z, momentum [0] and heat [1], and their differences
    float kx[2], dkx[2], kz[2], dkz[2];
    if (SMAG) {
        float sa, sp, ds;
        if (is == i) {
            jvc_strain(dax[0], daz[0], dax[1], daz[1], dbx[0], dbz[0], dbx[1], dbz[1], sa, sp, ds);
        } else {
            jvc_strain(ddf(A, is, 1, G.fx1, G.fx2), ddf(A, is, SX, G.fz1, G.fz2), ddf(A + PLANE, is, 1, G.fx1, G.fx2),
                       ddf(A + PLANE, is, SX, G.fz1, G.fz2), __fmul_rn(k.ev[0], ddf(V, is, 1, G.fx1, G.fx2)),
                       __fmul_rn(k.ev[0], ddf(V, is, SX, G.fz1, G.fz2)),
                       __fmul_rn(k.ev[1], ddf(V + PLANE, is, 1, G.fx1, G.fx2)),
                       __fmul_rn(k.ev[1], ddf(V + PLANE, is, SX, G.fz1, G.fz2)), sa, sp, ds);
        }
        if (SMAG == 2) {
            kx[0] = __fmul_rn(k.cm, sa); dkx[0] = __fmul_rn(k.cm, ds);
            kz[0] = __fmul_rn(k.cM, sa); dkz[0] = __fmul_rn(k.cM, ds);
            float g, dg;
            jvc_heat(sa, sp, ds, k.ah, k, g, dg);
            kx[1] = __fmul_rn(k.cm, g); dkx[1] = __fmul_rn(k.cm, dg);
            jvc_heat(sa, sp, ds, k.az, k, g, dg);
            kz[1] = __fmul_rn(k.cM, g); dkz[1] = __fmul_rn(k.cM, dg);
        } else {
            const float ka = __fmul_rn(k.cs2, sa), dk = __fmul_rn(k.cs2, ds);
            kx[0] = kz[0] = ka; dkx[0] = dkz[0] = dk;
            kx[1] = kz[1] = __fmul_rn(ka, k.iPr); dkx[1] = dkz[1] = __fmul_rn(dk, k.iPr);
        }
    } else {
        kx[0] = kz[0] = k.KM; kx[1] = kz[1] = k.KH;
        dkx[0] = dkz[0] = dkx[1] = dkz[1] = 0.f;
    }
    if (XF) {
#pragma unroll
        for (int f = 0; f < 4; ++f) P[f] = flux_diff(a[0], b[0], a[f], b[f]);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const int c = f == 2 ? 1 : 0;
            Fx[f] = SMAG ? kflux_diff(kx[c], dkx[c], dax[f], dbx[f]) : __fmul_rn(kx[c], dbx[f]);
        }
    }
    if (ZF) {
#pragma unroll
        for (int f = 0; f < 4; ++f) Q[f] = flux_diff(a[1], b[1], a[f], b[f]);
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            const int c = f == 2 ? 1 : 0;
            Fz[f] = SMAG ? kflux_diff(kz[c], dkz[c], daz[f], dbz[f]) : __fmul_rn(kz[c], dbz[f]);
        }
    }
    if (CEN) {
        const float th0 = (float)G.theta0;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            // a_u D_x b + a_w D_z b + b_u D_x phi' + b_w D_z phi'
            const float adv = __fmaf_rn(a[0], dbx[f], __fmaf_rn(a[1], dbz[f],
                              __fmaf_rn(b[0], __fadd_rn(dax[f], dbx[f]), __fmul_rn(b[1], __fadd_rn(daz[f], dbz[f])))));
            S[f] = __fmul_rn(-0.5f, adv);
        }
        const float gth = (float)(G.g / G.theta0);
        S[0] = __fmaf_rn(-th0, dbx[3], S[0]);
        S[1] = __fmaf_rn(-th0, dbz[3], __fmaf_rn(gth, b[2], S[1]));
        S[2] = __fmaf_rn(-(float)G.beta, b[1], S[2]);
        const float diva = __fadd_rn(dax[0], daz[1]), divb = __fadd_rn(dbx[0], dbz[1]);
        const float pp = __fadd_rn(__fadd_rn((float)G.pbar, a[3]), b[3]);
        S[3] = __fmaf_rn(-(float)G.gamma_p, __fmaf_rn(pp, divb, __fmul_rn(b[3], diva)), S[3]);
    }
}

template <int SMAG, int TX, int TZ, int NBUF>
__global__ void __launch_bounds__(NTHREADS)
jvc2d(Geo G, const float* __restrict__ u, const float* __restrict__ v, float* __restrict__ out,
      const double* part, Ctl* ctl, int check_done) {
    using SH = JvcShape<TX, TZ>;
    constexpr int SX = SH::SX, PLANE = SH::PLANE, PXW = SH::PXW, PXN = SH::PXN, QZN = SH::QZN;
    constexpr int PPT = SH::PPT;
    pdl_wait();
    if (check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* stg = reinterpret_cast<float*>(smem_raw);
    float* PX = stg + NBUF * SH::STG;    // [4][TZ][PXW] then Fx [3][TZ][PXW]
    float* FX = PX + 4 * PXN;
    float* QZ = FX + 3 * PXN;            // [4][TZ+4][TX] then Fz [3][TZ+4][TX]
    float* FZ = QZ + 4 * QZN;
    const int ntx = (G.nx + TX - 1) / TX;
    const int ntiles = ntx * ((G.nz + TZ - 1) / TZ);
    int t = blockIdx.x;
    if (t < ntiles) jv_stage_issue(stg, u, v, G, (t % ntx) * TX, (t / ntx) * TZ, SX, SH::SZ);
    cpa_commit();
    const double eps = pending_eps(ctl, part);
    __shared__ float evs[4], cfs[4];
    if (threadIdx.x < 4) {
        const double e = eps * G.scale[threadIdx.x];
        evs[threadIdx.x] = (float)e;
        cfs[threadIdx.x] = (float)(e != 0.0 ? 1.0 / e : 0.0);
    }
    __syncthreads();
    JvcConst k;
#pragma unroll
    for (int f = 0; f < 4; ++f) k.ev[f] = evs[f];
    k.idx = (float)G.inv_dx;
    k.idz = (float)G.inv_dz;
    k.cs2 = (float)G.cs2;
    k.iPr = (float)G.inv_Pr;
    k.KM = (float)G.K_M;
    k.KH = (float)G.K_H;
    k.cm = (float)G.dd_cm;
    k.cM = (float)G.dd_cM;
    k.cl = (float)G.dd_cl;
    k.dlt = (float)G.dd_delta;
    k.ah = (float)G.dd_ah;
    k.az = (float)G.dd_az;
    const float tdt = (float)G.two_over_dt;
    const int col = threadIdx.x % TX, r0 = (threadIdx.x / TX) * PPT;
    for (int it = 0; t < ntiles; t += gridDim.x, ++it) {
        const int x0 = (t % ntx) * TX, z0 = (t / ntx) * TZ;
        float* sa = stg + (NBUF == 2 ? (it & 1) * SH::STG : 0);
        if (NBUF == 2) {
            // double buffer: the next tile's copies go out before this tile is computed
            const int tn = t + gridDim.x;
            if (tn < ntiles)
                jv_stage_issue(stg + ((it + 1) & 1) * SH::STG, u, v, G, (tn % ntx) * TX, (tn / ntx) * TZ, SX,
                               SH::SZ);
            cpa_commit();
            cpa_wait<1>();
        } else {
            cpa_wait<0>();
        }
        __syncthreads();
        if (z0 - HALO < 0 || z0 + TZ + HALO > G.nz) {
            // mirror signs of the ghost rows (u and v planes alike)
            for (int e = threadIdx.x; e < SH::SZ * SX; e += blockDim.x) {
                const int iz = e / SX;
                int side;
                const int sz = mirror_z(z0 + iz - HALO, G.nz, side);
                if (side == 0 || sz < 0 || sz >= G.nz) continue;
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const float sg = side == 1 ? (float)G.pb[f] : (float)G.pt[f];
                    if (sg != 1.f) {
                        sa[f * PLANE + e] *= sg;
                        sa[(4 + f) * PLANE + e] *= sg;
                    }
                }
            }
            __syncthreads();
        }
        // phase 2a: this thread's points (fluxes of every kind, S and the raw direction)
        float Sv[PPT][4], Vc[PPT][4];
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int iz = r0 + q;
            const int i = (iz + HALO) * SX + col + HALO;
            const int is = SMAG ? (jvc_smag_row(iz, z0, G.nz) + HALO) * SX + col + HALO : i;
            float P[4], Fx[3], Q[4], Fz[3];
            jvc_point<SMAG, true, true, true, SX, PLANE>(sa, i, is, k, G, P, Fx, Q, Fz, Sv[q], Vc[q]);
            const int ip = iz * PXW + col + R, iq = (iz + R) * TX + col;
#pragma unroll
            for (int f = 0; f < 4; ++f) { PX[f * PXN + ip] = P[f]; QZ[f * QZN + iq] = Q[f]; }
#pragma unroll
            for (int f = 0; f < 3; ++f) { FX[f * PXN + ip] = Fx[f]; FZ[f * QZN + iq] = Fz[f]; }
        }
        // phase 2b: the arms -- z-fluxes of rows -2, -1, TZ, TZ+1; x-fluxes of columns -2, -1, TX, TX+1
        for (int w = threadIdx.x; w < SH::NARM; w += blockDim.x) {
            float P[4], Fx[3], Q[4], Fz[3], S_[4], V_[4];
            if (w < 4 * TX) {
                const int a = w / TX, cx = w - a * TX;
                const int iz = a < 2 ? a - 2 : TZ + a - 2;
                const int i = (iz + HALO) * SX + cx + HALO;
                const int is = SMAG ? (jvc_smag_row(iz, z0, G.nz) + HALO) * SX + cx + HALO : i;
                jvc_point<SMAG, false, true, false, SX, PLANE>(sa, i, is, k, G, P, Fx, Q, Fz, S_, V_);
                const int iq = (iz + R) * TX + cx;
#pragma unroll
                for (int f = 0; f < 4; ++f) QZ[f * QZN + iq] = Q[f];
#pragma unroll
                for (int f = 0; f < 3; ++f) FZ[f * QZN + iq] = Fz[f];
            } else {
                const int w2 = w - 4 * TX;
                const int a = w2 / TZ, iz = w2 - a * TZ;
                const int cx = a < 2 ? a - 2 : TX + a - 2;
                const int i = (iz + HALO) * SX + cx + HALO;
                const int is = SMAG ? (jvc_smag_row(iz, z0, G.nz) + HALO) * SX + cx + HALO : i;
                jvc_point<SMAG, true, false, false, SX, PLANE>(sa, i, is, k, G, P, Fx, Q, Fz, S_, V_);
                const int ip = iz * PXW + cx + R;
#pragma unroll
                for (int f = 0; f < 4; ++f) PX[f * PXN + ip] = P[f];
#pragma unroll
                for (int f = 0; f < 3; ++f) FX[f * PXN + ip] = Fx[f];
            }
        }
        __syncthreads();
        if (NBUF == 1) {
            // single buffer: the staged planes are dead now; the next tile's copies
            // land while this one's fluxes are differentiated
            const int tn = t + gridDim.x;
            if (tn < ntiles) jv_stage_issue(stg, u, v, G, (tn % ntx) * TX, (tn / ntx) * TZ, SX, SH::SZ);
            cpa_commit();
        }
        // phase 3: differentiate the fluxes, add S, write J v = 2 v / dt - dF / (eps scale_f)
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            const int iz = r0 + q;
            const int gz = z0 + iz, gx = x0 + col;
            if (gz >= G.nz || gx >= G.nx) continue;
            const int ip = iz * PXW + col + R, iq = (iz + R) * TX + col;
            const size_t o = (size_t)gz * G.nx + gx;
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const float conv = __fadd_rn(ddf(PX + f * PXN, ip, 1, G.fx1, G.fx2),
                                             ddf(QZ + f * QZN, iq, TX, G.fz1, G.fz2));
                float dF = __fmaf_rn(-0.5f, conv, Sv[q][f]);
                if (f < 3)
                    dF = __fadd_rn(dF, __fadd_rn(ddf(FX + f * PXN, ip, 1, G.fx1, G.fx2),
                                                 ddf(FZ + f * QZN, iq, TX, G.fz1, G.fz2)));
                out[(size_t)f * G.npt + o] = __fmaf_rn(tdt, Vc[q][f], __fmul_rn(-cfs[f], dF));
            }
        }
        __syncthreads();     // staging buffer and flux arrays are reused by the next tile
    }
}

// ============================================================================
// Smagorinsky eddy field nu(u) at every point (preconditioner input) + max
// ============================================================================
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
eddy2d(Geo G, const T* __restrict__ u, T* __restrict__ nu, double* part, Ctl* ctl) {
    T mxT = T(0);
    const T idx_ = T(G.inv_dx), idz_ = T(G.inv_dz);
    const T cs2 = G.sgs == 2 ? T(1) : T(G.cs2);     // Deardorff: the strain s (coefficients follow from it)
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < G.npt; p += gridDim.x * blockDim.x) {
        const int z = p / G.nx, x = p - z * G.nx;
        T ux = T(0), uz = T(0), wx = T(0), wz = T(0);
#pragma unroll
        for (int l = 1; l <= 2; ++l) {
            const T c = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
            const int xp = wrap_x(x + l, G.nx), xm = wrap_x(x - l, G.nx);
            int sp_, sm_;
            const int zp = mirror_z(z + l, G.nz, sp_), zm = mirror_z(z - l, G.nz, sm_);
            const T sgu_p = sp_ == 2 ? T(G.pt[0]) : T(1), sgu_m = sm_ == 1 ? T(G.pb[0]) : T(1);
            const T sgw_p = sp_ == 2 ? T(G.pt[1]) : T(1), sgw_m = sm_ == 1 ? T(G.pb[1]) : T(1);
            const T* U = u;
            const T* W = u + G.npt;
            ux += c * (U[z * G.nx + xp] - U[z * G.nx + xm]);
            wx += c * (W[z * G.nx + xp] - W[z * G.nx + xm]);
            uz += c * (sgu_p * U[zp * G.nx + x] - sgu_m * U[zm * G.nx + x]);
            wz += c * (sgw_p * W[zp * G.nx + x] - sgw_m * W[zm * G.nx + x]);
        }
        const T v_ = smag_nu(ux * idx_, uz * idz_, wx * idx_, wz * idz_, cs2);
        nu[p] = v_;
        mxT = v_ > mxT ? v_ : mxT;
    }
    double mx[1] = {(double)mxT};
    block_partials_max<1>(mx, 1, part, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_EDDY], gridDim.x)) {
        __shared__ double tot[1];
        final_maxes(part, gridDim.x, 1, tot);
        if (threadIdx.x == 0) ctl->kmax = tot[0];
    }
}

// ============================================================================
// Field-block Chebyshev preconditioner (Section 2.5.2): for u, w, theta the
// block A_f = (2/dt) I - sum_j D_j(K D_j .) with K frozen at the current
// iterate; the p block is (2/dt) I.  Spectrum bounds from Gershgorin:
// [2/dt, 2/dt + (3/2)^2 K_max (1/dx^2 + 1/dz^2)] ((3/2) = sum_l |phi'(l)|).
// Sweep k (k = 1 .. s-1) of the Chebyshev semi-iteration (Saad, Alg. 12.1):
//   res = r - A x_k;  d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) res;
//   x_{k+1} = x_k + d_k,   with x_1 = d_0 = r / theta_c.
// ============================================================================
// Coefficients of every sweep of every block, computed once per Newton
// iteration from the (frozen) eddy maximum by one thread: 1/theta_c,
// rho_k rho_{k-1} and 2 rho_k / delta, with rho_0 = 1/sigma, sigma = theta_c/delta.
__global__ void pc_setup(Geo G, int sweeps, Ctl* ctl) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int fth = G.nf - 2, fp = G.nf - 1;         // theta and p
    const double h2 = G.inv_dx * G.inv_dx + G.inv_dz * G.inv_dz + (G.dim == 3 ? G.inv_dy * G.inv_dy : 0.0);
    // Deardorff: ctl->kmax is the largest strain s; every coefficient grows with s
    const double smax = ctl->kmax;
    const double lmax = G.dd_cl < 0.0 ? G.dd_delta : fmin(G.dd_delta, G.dd_cl * smax);
    const double hh2 = G.inv_dx * G.inv_dx + (G.dim == 3 ? G.inv_dy * G.inv_dy : 0.0);
    for (int f = 0; f < G.nf; ++f) {
        const double lo = G.two_over_dt;
        double kh2 = 0.0;        // sum_j max K_j / h_j^2
        if (f != fp) {
            if (G.sgs == 2) {
                const double fh = f == fth ? 1.0 + G.dd_ah * lmax : 1.0;
                const double fz = f == fth ? 1.0 + G.dd_az * lmax : 1.0;
                kh2 = G.dd_cm * smax * fh * hh2 + G.dd_cM * smax * fz * G.inv_dz * G.inv_dz;
            } else {
                kh2 = (G.smag ? ctl->kmax * (f == fth ? G.inv_Pr : 1.0) : (f == fth ? G.K_H : G.K_M)) * h2;
            }
        }
        const double hi = lo + 2.25 * kh2;
        const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
        const bool degenerate = delta <= 1e-14 * theta;
        const double sigma = degenerate ? 1.0 : theta / delta;
        double rho = 1.0 / sigma;
        ctl->cheb[f][0][0] = 1.0 / theta;
        ctl->cheb[f][0][1] = 0.0;
        ctl->cheb[f][0][2] = 0.0;
        for (int k = 1; k < sweeps && k < MAX_PC_SWEEPS; ++k) {
            const double rho_new = 1.0 / (2.0 * sigma - rho);
            ctl->cheb[f][k][0] = 1.0 / theta;
            ctl->cheb[f][k][1] = degenerate ? 0.0 : rho_new * rho;
            ctl->cheb[f][k][2] = degenerate ? 0.0 : 2.0 * rho_new / delta;
            rho = rho_new;
        }
    }
    {
        // slot 5 holds the pressure Helmholtz operator of the acoustic Schur
        // complement, H = (2/dt) I - a sum_j D_j D_j, a = gamma_p pbar theta0 dt / 2
        const double a = G.helm_a;
        const double lo = G.two_over_dt, hi = lo + 2.25 * a * h2;
        const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
        const bool degenerate = delta <= 1e-14 * theta;
        const double sigma = degenerate ? 1.0 : theta / delta;
        double rho = 1.0 / sigma;
        ctl->cheb[5][0][0] = 1.0 / theta;
        ctl->cheb[5][0][1] = 0.0;
        ctl->cheb[5][0][2] = 0.0;
        for (int k = 1; k < sweeps && k < MAX_PC_SWEEPS; ++k) {
            const double rho_new = 1.0 / (2.0 * sigma - rho);
            ctl->cheb[5][k][0] = 1.0 / theta;
            ctl->cheb[5][k][1] = degenerate ? 0.0 : rho_new * rho;
            ctl->cheb[5][k][2] = degenerate ? 0.0 : 2.0 * rho_new / delta;
            rho = rho_new;
        }
    }
}

// One CTA = one field of one TX x TZ tile; threads laid out (TX, NTHREADS/TX)
// so that every stage indexes rows and columns without divisions.  D_x z is
// formed only on the tile rows (x-halo r), D_z z only on the tile columns
// (z-halo r): exactly the taps the second application of D reads.
template <typename T, int SMAG, int FIRST, int LAST, int TX, int TZ>
__global__ void __launch_bounds__(NTHREADS, 8)
cheb2d(Geo G, int k, const T* __restrict__ r, const T* __restrict__ zin, const T* __restrict__ din,
       T* __restrict__ zout, T* __restrict__ dout, const T* __restrict__ nu, double* part, Ctl* ctl,
       int check_done) {
    constexpr int SX = TX + 2 * HALO, SZ = TZ + 2 * HALO;
    constexpr int QX = TX + 2 * R, QZ = TZ + 2 * R;
    constexpr int TY = NTHREADS / TX;              // thread rows
    static_assert(NTHREADS % TX == 0 && TZ % TY == 0, "tile must tile the block");
    pdl_wait();
    if (check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* zs = reinterpret_cast<T*>(smem_raw);      // [SZ][SX] current iterate, halo 2r
    T* gxs = zs + SZ * SX;                          // [TZ][QX] D_x z on tile rows
    T* gzs = gxs + TZ * QX;                         // [QZ][TX] D_z z on tile columns
    T* kk_ = gzs + QZ * TX;                         // [QZ][QX] eddy coefficient (along x for Deardorff)
    T* kz_ = SMAG == 2 ? kk_ + QZ * QX : kk_;       // [QZ][QX] Deardorff coefficient along z
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int fld = blockIdx.z;                     // 0 u, 1 w, 2 theta, 3 p (last sweep only)
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ;
    const T ith = T(ctl->cheb[fld][k][0]);
    const T a1 = T(ctl->cheb[fld][k][1]);
    const T a2 = T(ctl->cheb[fld][k][2]);
    const T* rf = r + (size_t)fld * G.npt;
    T* zf = zout + (size_t)fld * G.npt;
    const int gxx = x0 + tx;
    T acc[1] = {T(0)};
    if (fld == 3) {
        if (LAST && gxx < G.nx) {          // p block: (2/dt) I, exact in one step
            for (int tz = ty; tz < TZ; tz += TY) {
                const int gz = z0 + tz;
                if (gz >= G.nz) break;
                const int o = gz * G.nx + gxx;
                const T zv = rf[o] * ith;
                zf[o] = zv;
                acc[0] += zv * zv;
            }
        }
    } else {
        // per-output operands first: their latency overlaps the tile staging below
        constexpr int NR = TZ / TY;
        T rv[NR], dv[NR];
        const T* df = FIRST ? nullptr : din + (size_t)fld * G.npt;
        const bool colok = gxx < G.nx;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int gz = z0 + ty + q * TY;
            const bool ok = colok && gz < G.nz;
            const int o = gz * G.nx + gxx;
            rv[q] = ok ? rf[o] : T(0);
            dv[q] = (!FIRST && ok) ? df[o] : T(0);
        }
        // x_k with halo 2r (first sweep: x_1 = r / theta_c)
        T sc[4] = {T(0), T(0), T(0), T(0)};
        if (FIRST) {
            sc[fld] = ith;
            load_fields<T, 2, 1>(zs, nullptr, r, sc, G, x0, z0, SX, SZ, fld);
        } else {
            load_fields<T, 0, 1>(zs, zin, nullptr, sc, G, x0, z0, SX, SZ, fld);
        }
        if (SMAG == 2) {
            // Deardorff: nu holds the strain s; K_m = c_m s along x, K_M = c_M s along z,
            // heat K_h = c_m s (1 + a_h l), K_H = c_M s (1 + a_z l)
            const T cm = T(G.dd_cm), cM = T(G.dd_cM);
            for (int qz = ty; qz < QZ; qz += TY) {
                int side;
                const int szr = mirror_z(z0 + qz - R, G.nz, side);
                const bool ok = szr >= 0 && szr < G.nz;
                const T* nrow = nu + szr * G.nx;
                for (int qx = tx; qx < QX; qx += TX) {
                    const T sv = ok ? nrow[wrap_x(x0 + qx - R, G.nx)] : T(0);
                    kk_[qz * QX + qx] = rmul(cm, fld == 2 ? dd_heat(sv, T(G.dd_ah), G) : sv);
                    kz_[qz * QX + qx] = rmul(cM, fld == 2 ? dd_heat(sv, T(G.dd_az), G) : sv);
                }
            }
        } else if (SMAG) {
            const T kscale = fld == 2 ? T(G.inv_Pr) : T(1);
            for (int qz = ty; qz < QZ; qz += TY) {
                int side;
                const int szr = mirror_z(z0 + qz - R, G.nz, side);
                const bool ok = szr >= 0 && szr < G.nz;
                const T* nrow = nu + szr * G.nx;
                for (int qx = tx; qx < QX; qx += TX)
                    kk_[qz * QX + qx] = ok ? nrow[wrap_x(x0 + qx - R, G.nx)] * kscale : T(0);
            }
        }
        __syncthreads();
        const T idx_ = T(G.inv_dx), idz_ = T(G.inv_dz);
        for (int tz = ty; tz < TZ; tz += TY)              // D_x on tile rows, x-halo r
            for (int qx = tx; qx < QX; qx += TX)
                gxs[tz * QX + qx] = dd(zs, (tz + HALO) * SX + qx + R, 1, idx_);
        for (int qz = ty; qz < QZ; qz += TY)              // D_z on tile columns, z-halo r
            gzs[qz * TX + tx] = dd(zs, (qz + R) * SX + tx + HALO, SX, idz_);
        __syncthreads();
        const T Kc = T(fld == 2 ? G.K_H : G.K_M);
        const T tdt = T(G.two_over_dt);
        T* dof = LAST ? nullptr : dout + (size_t)fld * G.npt;
        if (colok) {
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const int tz = ty + q * TY;
                const int gz = z0 + tz;
                if (gz >= G.nz) break;
                const T* gxr = gxs + tz * QX + tx + R;          // centre of the x taps
                const T* gzc = gzs + (tz + R) * TX + tx;        // centre of the z taps
                // explicitly rounded (rmul / rfma): every tile shape computes the same bits
                T difx, difz;
                if (SMAG) {
                    const T* kx = kk_ + (tz + R) * QX + tx + R;
                    const T* kz = kz_ + (tz + R) * QX + tx + R;
                    const T x1 = rfma(kx[1], gxr[1], -rmul(kx[-1], gxr[-1]));
                    const T x2 = rfma(kx[2], gxr[2], -rmul(kx[-2], gxr[-2]));
                    const T z1 = rfma(kz[QX], gzc[TX], -rmul(kz[-QX], gzc[-TX]));
                    const T z2 = rfma(kz[2 * QX], gzc[2 * TX], -rmul(kz[-2 * QX], gzc[-2 * TX]));
                    difx = rfma(T(2.0 / 3.0), x1, rmul(T(-1.0 / 12.0), x2));
                    difz = rfma(T(2.0 / 3.0), z1, rmul(T(-1.0 / 12.0), z2));
                } else {
                    difx = rmul(Kc, rfma(T(2.0 / 3.0), gxr[1] - gxr[-1], rmul(T(-1.0 / 12.0), gxr[2] - gxr[-2])));
                    difz = rmul(Kc, rfma(T(2.0 / 3.0), gzc[TX] - gzc[-TX], rmul(T(-1.0 / 12.0), gzc[2 * TX] - gzc[-2 * TX])));
                }
                const T dif = rfma(difx, idx_, rmul(difz, idz_));
                const T xk = zs[(tz + HALO) * SX + tx + HALO];
                const int o = gz * G.nx + gxx;
                const T res = rv[q] - rfma(tdt, xk, -dif);
                const T dprev = FIRST ? rmul(rv[q], ith) : dv[q];
                const T dk = rfma(a1, dprev, rmul(a2, res));
                const T xn = xk + dk;
                zf[o] = xn;
                if (!LAST) dof[o] = dk;
                if (LAST) acc[0] += xn * xn;
            }
        }
    }
    pdl_trigger();
    if (LAST) {
        const int nblk = gridDim.x * gridDim.y * gridDim.z;
        const int blk = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        if constexpr (sizeof(T) == sizeof(float)) {
            // ||z||^2 stays pending, one float-float partial per block: the
            // Jacobian product that follows adds them (pending_eps), so this
            // launch ends without an arrival count and a serial tail
            block_partial_ff(acc[0], reinterpret_cast<float2*>(part), blk);
            if (blk == 0 && threadIdx.x == 0) ctl->eps_part = nblk;
        } else {
            block_partials<1, T>(acc, 1, part, nblk, blk);
            if (arrive_last(&ctl->counter[CNT_PC], nblk)) {
                __shared__ double tot[1];
                final_sums(part, nblk, 1, tot);
                if (threadIdx.x == 0) {
                    const double zn = sqrt(tot[0]);
                    ctl->eps_jv = zn > 0.0 ? sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2))) / zn : 0.0;
                    ctl->eps_part = 0;
                }
            }
        }
    }
}

// p = 1 sweep count: z = r / theta_c for every field (point-wise), + eps from ||z||
template <typename T, int SMAG>
__global__ void __launch_bounds__(NTHREADS)
pc_diag(Geo G, const T* __restrict__ r, T* __restrict__ z, size_t n, double* part, Ctl* ctl,
        int check_done) {
    if (check_done && ctl->done) return;
    T acc[1] = {T(0)};
    T inv_th[5];
    for (int f = 0; f < G.nf; ++f) inv_th[f] = T(ctl->cheb[f][0][0]);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int f = (int)(i / G.npt);
        const T zv = r[i] * inv_th[f];
        z[i] = zv;
        acc[0] += zv * zv;
    }
    block_partials<1, T>(acc, 1, part, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_PC], gridDim.x)) {
        __shared__ double tot[1];
        final_sums(part, gridDim.x, 1, tot);
        if (threadIdx.x == 0) {
            const double zn = sqrt(tot[0]);
            ctl->eps_jv = zn > 0.0 ? sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2))) / zn : 0.0;
            ctl->eps_part = 0;
        }
    }
}

// ============================================================================
// Acoustic Schur-complement preconditioner (2-D, scaled units).  Keeping only
// (2/dt) I and the pressure gradient / divergence couplings of Eqs.
// ch2_28-ch2_30 (linearised about pbar) -- the fast terms the semi-implicit
// scheme that Section 2.5 follows eliminates -- the velocities drop out:
//   H dp = v_p - c_div (D_x v_u + D_z v_w),   H = (2/dt) I - a sum_j D_j D_j,
//   z_u = (dt/2)(v_u - c_grad D_x dp),   z_w = (dt/2)(v_w - c_grad D_z dp),
// with c_div = gamma_p pbar (dt/2) s_u / s_p, c_grad = theta0 s_p / s_u and
// a = gamma_p pbar theta0 dt / 2.  H is inverted approximately by Chebyshev
// sweeps on its Gershgorin interval (coefficients ctl->cheb[5], pc_setup);
// theta gets r_theta / theta_c of its field block.
// ============================================================================
template <typename T>
__device__ __forceinline__ T plane_dx(const T* __restrict__ f, const Geo& G, int gz, int gx, T inv_h) {
    const T* row = f + (size_t)gz * G.nx;
    return (T(2.0 / 3.0) * (row[wrap_x(gx + 1, G.nx)] - row[wrap_x(gx - 1, G.nx)]) -
            T(1.0 / 12.0) * (row[wrap_x(gx + 2, G.nx)] - row[wrap_x(gx - 2, G.nx)])) * inv_h;
}

// value of plane f (field parity fld) at row gz, one mirror reflection at the walls
template <typename T>
__device__ __forceinline__ T plane_z(const T* __restrict__ f, const Geo& G, int gz, int gx, int fld) {
    int side;
    const int sz = mirror_z(gz, G.nz, side);
    const T v = f[(size_t)sz * G.nx + gx];
    return side == 1 ? T(G.pb[fld]) * v : (side == 2 ? T(G.pt[fld]) * v : v);
}

template <typename T>
__device__ __forceinline__ T plane_dz(const T* __restrict__ f, const Geo& G, int gz, int gx, int fld, T inv_h) {
    return (T(2.0 / 3.0) * (plane_z(f, G, gz + 1, gx, fld) - plane_z(f, G, gz - 1, gx, fld)) -
            T(1.0 / 12.0) * (plane_z(f, G, gz + 2, gx, fld) - plane_z(f, G, gz - 2, gx, fld))) * inv_h;
}

// rhs = v_p - c_div (D_x v_u + D_z v_w)
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
schur_rhs2d(Geo G, const T* __restrict__ r, T* __restrict__ rhs, Ctl* ctl, int check_done) {
    if (check_done && ctl->done) return;
    const T cdiv = T(G.schur_cdiv);
    const T idx_ = T(G.inv_dx), idz_ = T(G.inv_dz);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < G.npt; p += gridDim.x * blockDim.x) {
        const int gz = p / G.nx, gx = p - gz * G.nx;
        const T du = plane_dx(r, G, gz, gx, idx_);
        const T dw = plane_dz(r + G.npt, G, gz, gx, 1, idz_);
        rhs[p] = r[(size_t)3 * G.npt + p] - cdiv * (du + dw);
    }
}

// One Chebyshev sweep (k = 1 .. s-1) for H x = rhs on one plane, tiled like
// cheb2d: x_k staged with halo 2r (even mirror of p), D_x on tile rows, D_z on
// tile columns, then res = rhs - H x_k, d_k, x_{k+1} = x_k + d_k.
template <typename T, int FIRST, int LAST, int TX, int TZ>
__global__ void __launch_bounds__(NTHREADS)
helm2d(Geo G, int k, const T* __restrict__ rhs, const T* __restrict__ xin, const T* __restrict__ din,
       T* __restrict__ xout, T* __restrict__ dout, Ctl* ctl, int check_done) {
    constexpr int SX = TX + 2 * HALO, SZ = TZ + 2 * HALO;
    constexpr int QX = TX + 2 * R, QZ = TZ + 2 * R;
    constexpr int TY = NTHREADS / TX;
    static_assert(NTHREADS % TX == 0 && TZ % TY == 0, "tile must tile the block");
    if (check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* zs = reinterpret_cast<T*>(smem_raw);      // [SZ][SX]
    T* gxs = zs + SZ * SX;                          // [TZ][QX]
    T* gzs = gxs + TZ * QX;                         // [QZ][TX]
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ;
    const T ith = T(ctl->cheb[5][k][0]);
    const T a1 = T(ctl->cheb[5][k][1]);
    const T a2 = T(ctl->cheb[5][k][2]);
    const int gxx = x0 + tx;
    const bool colok = gxx < G.nx;
    constexpr int NR = TZ / TY;
    T rv[NR], dv[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
        const int gz = z0 + ty + q * TY;
        const bool ok = colok && gz < G.nz;
        const int o = gz * G.nx + gxx;
        rv[q] = ok ? rhs[o] : T(0);
        dv[q] = (!FIRST && ok) ? din[o] : T(0);
    }
    const T* src = FIRST ? rhs : xin;
    const T sc = FIRST ? ith : T(1);
    const T pb = T(G.pb[3]), pt = T(G.pt[3]);
    for (int idx = threadIdx.x; idx < SX * SZ; idx += blockDim.x) {
        const int iz = idx / SX, ix = idx - iz * SX;
        int side;
        const int sz = mirror_z(z0 + iz - HALO, G.nz, side);
        const int sx = wrap_x(x0 + ix - HALO, G.nx);
        T val = T(0);
        if (sz >= 0 && sz < G.nz) {
            val = sc * src[(size_t)sz * G.nx + sx];
            if (side == 1) val *= pb;
            else if (side == 2) val *= pt;
        }
        zs[idx] = val;
    }
    __syncthreads();
    const T idx_ = T(G.inv_dx), idz_ = T(G.inv_dz);
    for (int tz = ty; tz < TZ; tz += TY)
        for (int qx = tx; qx < QX; qx += TX) gxs[tz * QX + qx] = dd(zs, (tz + HALO) * SX + qx + R, 1, idx_);
    for (int qz = ty; qz < QZ; qz += TY) gzs[qz * TX + tx] = dd(zs, (qz + R) * SX + tx + HALO, SX, idz_);
    __syncthreads();
    const T ah = T(G.helm_a);
    const T tdt = T(G.two_over_dt);
    if (colok) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const int tz = ty + q * TY;
            const int gz = z0 + tz;
            if (gz >= G.nz) break;
            const T* gxr = gxs + tz * QX + tx + R;
            const T* gzc = gzs + (tz + R) * TX + tx;
            const T difx = T(2.0 / 3.0) * (gxr[1] - gxr[-1]) - T(1.0 / 12.0) * (gxr[2] - gxr[-2]);
            const T difz = T(2.0 / 3.0) * (gzc[TX] - gzc[-TX]) - T(1.0 / 12.0) * (gzc[2 * TX] - gzc[-2 * TX]);
            const T xk = zs[(tz + HALO) * SX + tx + HALO];
            const T res = rv[q] - (tdt * xk - ah * (difx * idx_ + difz * idz_));
            const T dprev = FIRST ? rv[q] * ith : dv[q];
            const T dk = a1 * dprev + a2 * res;
            const int o = gz * G.nx + gxx;
            xout[o] = xk + dk;
            if (!LAST) dout[o] = dk;
        }
    }
}

// Two Chebyshev sweeps (k and k+1) per launch (temporal blocking): x_k is
// staged with halo 4r, sweep k runs on the tile plus a ring of 2r points
// (ghost rows included -- the mirrored data give the mirrored result), and
// sweep k+1 on the tile from those values.  Needs nz >= 4r (one reflection).
template <typename T, int FIRST, int LAST, int TX, int TZ>
__global__ void __launch_bounds__(NTHREADS)
helm2d_x2(Geo G, int k, const T* __restrict__ rhs, const T* __restrict__ xin, const T* __restrict__ din,
          T* __restrict__ xout, T* __restrict__ dout, Ctl* ctl, int check_done) {
    constexpr int H2 = 2 * HALO;                       // staging halo (two sweeps)
    constexpr int SX = TX + 2 * H2, SZ = TZ + 2 * H2;
    constexpr int EX = TX + 2 * HALO, EZ = TZ + 2 * HALO;   // first-sweep region
    constexpr int TY = NTHREADS / TX;
    static_assert(NTHREADS % TX == 0 && TZ % TY == 0, "tile must tile the block");
    if (check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* xs = reinterpret_cast<T*>(smem_raw);   // [SZ][SX]   x_k
    T* re = xs + SZ * SX;                        // [EZ][EX]   rhs on the first-sweep region
    T* de = re + EZ * EX;                        // [EZ][EX]   d_{k-1}, then d_k
    T* x1 = de + EZ * EX;                        // [EZ][EX]   x_{k+1}
    T* gx = x1 + EZ * EX;                        // [EZ][EX + 2R]  D_x rows (reused by sweep k+1)
    T* gz = gx + EZ * (EX + 2 * R);              // [EZ + 2R][EX]  D_z columns (reused)
    const int x0 = blockIdx.x * TX, z0 = blockIdx.y * TZ;
    const T ith = T(ctl->cheb[5][k][0]);
    const T a1 = T(ctl->cheb[5][k][1]), a2 = T(ctl->cheb[5][k][2]);
    const T b1 = T(ctl->cheb[5][k + 1][1]), b2 = T(ctl->cheb[5][k + 1][2]);
    const T pb = T(G.pb[3]), pt = T(G.pt[3]);
    // staging: x_k (halo 2 HALO), rhs and d_{k-1} (halo HALO); p parity in z, periodic x
    for (int idx = threadIdx.x; idx < SX * SZ; idx += blockDim.x) {
        const int iz = idx / SX, ix = idx - iz * SX;
        int side;
        const int sz = mirror_z(z0 + iz - H2, G.nz, side);
        const int sx = wrap_x(x0 + ix - H2, G.nx);
        // rows beyond one reflection (tiles overhanging a wall) feed no output: zero
        const bool ok = sz >= 0 && sz < G.nz;
        const T sgn = side == 1 ? pb : (side == 2 ? pt : T(1));
        const size_t o = ok ? (size_t)sz * G.nx + sx : 0;
        const T xv = ok ? (FIRST ? ith * rhs[o] : xin[o]) : T(0);
        xs[idx] = sgn * xv;
        const int ez = iz - HALO, ex = ix - HALO;
        if (ez >= 0 && ez < EZ && ex >= 0 && ex < EX) {
            const T rv = ok ? sgn * rhs[o] : T(0);
            re[ez * EX + ex] = rv;
            de[ez * EX + ex] = FIRST ? ith * rv : (ok ? sgn * din[o] : T(0));
        }
    }
    __syncthreads();
    const T idx_ = T(G.inv_dx), idz_ = T(G.inv_dz);
    const T ah = T(G.helm_a), tdt = T(G.two_over_dt);
    // sweep k on the first-sweep region
    for (int i = threadIdx.x; i < EZ * (EX + 2 * R); i += blockDim.x) {
        const int ez = i / (EX + 2 * R), c = i - ez * (EX + 2 * R);
        gx[i] = dd(xs, (ez + HALO) * SX + c + R, 1, idx_);
    }
    for (int i = threadIdx.x; i < (EZ + 2 * R) * EX; i += blockDim.x) {
        const int r = i / EX, ex = i - r * EX;
        gz[i] = dd(xs, (r + R) * SX + ex + HALO, SX, idz_);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < EZ * EX; i += blockDim.x) {
        const int ez = i / EX, ex = i - ez * EX;
        const T* gxr = gx + ez * (EX + 2 * R) + ex + R;
        const T* gzc = gz + (ez + R) * EX + ex;
        const T difx = T(2.0 / 3.0) * (gxr[1] - gxr[-1]) - T(1.0 / 12.0) * (gxr[2] - gxr[-2]);
        const T difz = T(2.0 / 3.0) * (gzc[EX] - gzc[-EX]) - T(1.0 / 12.0) * (gzc[2 * EX] - gzc[-2 * EX]);
        const T xk = xs[(ez + HALO) * SX + ex + HALO];
        const T res = re[i] - (tdt * xk - ah * (difx * idx_ + difz * idz_));
        const T dk = a1 * de[i] + a2 * res;
        de[i] = dk;
        x1[i] = xk + dk;
    }
    __syncthreads();
    // sweep k+1 on the tile
    constexpr int GX2 = TX + 2 * R;
    for (int i = threadIdx.x; i < TZ * GX2; i += blockDim.x) {
        const int tz = i / GX2, c = i - tz * GX2;
        gx[i] = dd(x1, (tz + HALO) * EX + c + R, 1, idx_);
    }
    for (int i = threadIdx.x; i < (TZ + 2 * R) * TX; i += blockDim.x) {
        const int r = i / TX, tx = i - r * TX;
        gz[i] = dd(x1, (r + R) * EX + tx + HALO, EX, idz_);
    }
    __syncthreads();
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int gxx = x0 + tx;
    if (gxx < G.nx) {
#pragma unroll
        for (int q = 0; q < TZ / TY; ++q) {
            const int tz = ty + q * TY;
            const int gzz = z0 + tz;
            if (gzz >= G.nz) break;
            const T* gxr = gx + tz * GX2 + tx + R;
            const T* gzc = gz + (tz + R) * TX + tx;
            const T difx = T(2.0 / 3.0) * (gxr[1] - gxr[-1]) - T(1.0 / 12.0) * (gxr[2] - gxr[-2]);
            const T difz = T(2.0 / 3.0) * (gzc[TX] - gzc[-TX]) - T(1.0 / 12.0) * (gzc[2 * TX] - gzc[-2 * TX]);
            const int e = (tz + HALO) * EX + tx + HALO;
            const T xk = x1[e];
            const T res = re[e] - (tdt * xk - ah * (difx * idx_ + difz * idz_));
            const T dk = b1 * de[e] + b2 * res;
            const int o = gzz * G.nx + gxx;
            xout[o] = xk + dk;
            if (!LAST) dout[o] = dk;
        }
    }
}

// z_u, z_w from the pressure solution (already in plane 3 of z), z_theta, and
// the finite-difference step eps from ||z||.
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
schur_back2d(Geo G, const T* __restrict__ r, T* __restrict__ z, double* part, Ctl* ctl, int check_done) {
    if (check_done && ctl->done) return;
    const T cgrad = T(G.schur_cgrad);
    const T hdt = T(G.half_dt);
    const T ith_t = T(ctl->cheb[2][0][0]);
    const T idx_ = T(G.inv_dx), idz_ = T(G.inv_dz);
    const size_t np = (size_t)G.npt;
    const T* dp = z + 3 * np;
    T acc[1] = {T(0)};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < G.npt; p += gridDim.x * blockDim.x) {
        const int gz = p / G.nx, gx = p - gz * G.nx;
        const T zu = hdt * (r[p] - cgrad * plane_dx(dp, G, gz, gx, idx_));
        const T zw = hdt * (r[np + p] - cgrad * plane_dz(dp, G, gz, gx, 3, idz_));
        const T zt = r[2 * np + p] * ith_t;
        const T zp = dp[p];
        z[p] = zu;
        z[np + p] = zw;
        z[2 * np + p] = zt;
        acc[0] += zu * zu + zw * zw + zt * zt + zp * zp;
    }
    block_partials<1, T>(acc, 1, part, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_PC], gridDim.x)) {
        __shared__ double tot[1];
        final_sums(part, gridDim.x, 1, tot);
        if (threadIdx.x == 0) {
            const double zn = sqrt(tot[0]);
            ctl->eps_jv = zn > 0.0 ? sqrt(ctl->eps_mach * (1.0 + sqrt(ctl->unorm2))) / zn : 0.0;
            ctl->eps_part = 0;
        }
    }
}

// ============================================================================
// Budgets: E_k = 1/2 sum (u^2 + w^2) dV, E_p = sum (lz - z) theta dV (Section 3.1.3),
// sum theta dV, sum div(u) dV, max / min of every field.
// ============================================================================
__global__ void __launch_bounds__(NTHREADS)
budgets2d(Geo G, const double* __restrict__ u, double dV, double dz, double lz, double* part,
          Ctl* ctl, double* out) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    double mx[8];
    for (int f = 0; f < 4; ++f) { mx[f] = -1e300; mx[4 + f] = -1e300; }
    const double* U = u;
    const double* W = u + G.npt;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < G.npt; p += gridDim.x * blockDim.x) {
        const int z = p / G.nx, x = p - z * G.nx;
        const double zc = (z + 0.5) * dz;
        s[0] += 0.5 * (U[p] * U[p] + W[p] * W[p]);
        s[1] += (lz - zc) * u[2 * G.npt + p];
        s[2] += u[2 * G.npt + p];
        double ux = 0.0, wz = 0.0;
        for (int l = 1; l <= 2; ++l) {
            const double c = l == 1 ? 2.0 / 3.0 : -1.0 / 12.0;
            ux += c * (U[z * G.nx + wrap_x(x + l, G.nx)] - U[z * G.nx + wrap_x(x - l, G.nx)]);
            int sp_, sm_;
            const int zp = mirror_z(z + l, G.nz, sp_), zm = mirror_z(z - l, G.nz, sm_);
            const double gp = sp_ == 2 ? G.pt[1] : 1.0, gm = sm_ == 1 ? G.pb[1] : 1.0;
            wz += c * (gp * W[zp * G.nx + x] - gm * W[zm * G.nx + x]);
        }
        s[3] += ux * G.inv_dx + wz * G.inv_dz;
        for (int f = 0; f < 4; ++f) {
            const double v = u[(size_t)f * G.npt + p];
            mx[f] = max_nan(mx[f], v);
            mx[4 + f] = max_nan(mx[4 + f], -v);
        }
    }
    double* pmax = part + 4 * gridDim.x;
    block_partials<4>(s, 4, part, gridDim.x, blockIdx.x);
    block_partials_max<8>(mx, 8, pmax, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_MISC], gridDim.x)) {
        __shared__ double tot[12];
        final_sums(part, gridDim.x, 4, tot);
        final_maxes(pmax, gridDim.x, 8, tot + 4);
        if (threadIdx.x == 0) {
            for (int i = 0; i < 4; ++i) out[i] = tot[i] * dV;
            for (int f = 0; f < 4; ++f) { out[4 + f] = tot[4 + f]; out[8 + f] = -tot[8 + f]; }
        }
    }
}

// ============================================================================
// launchers
// ============================================================================
template <typename T> int stencil_blocks(const Geo& G) {
    return ((G.nx + Tile<T>::TX - 1) / Tile<T>::TX) * ((G.nz + Tile<T>::TZ - 1) / Tile<T>::TZ);
}
template int stencil_blocks<float>(const Geo&);
template int stencil_blocks<double>(const Geo&);

template <typename T, int SMAG>
static size_t stencil_smem() {
    constexpr int TX = Tile<T>::TX, TZ = Tile<T>::TZ;
    constexpr int NQ = SMAG == 2 ? 9 : 7;        // derivatives (6) + eddy field(s)
    return sizeof(T) * (4 * (TZ + 2 * HALO) * (TX + 2 * HALO) + NQ * (TX + 2 * R) * (TZ + 2 * R));
}

template <typename T, int TX, int TZ, int NBUF>
static size_t jvd_smem() {
    return sizeof(T) * (NBUF * 8 * (TZ + 2 * HALO) * (TX + 2 * HALO) + 14 * (TX + 2 * R) * (TZ + 2 * R));
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int MODE, int SMAG>
static cudaError_t launch_stencil_t(const Geo& G, const T* u, const T* v, const T* Fu,
                                    const double* f, T* out, T* out2, double* part, Ctl* ctl,
                                    int check_done, cudaStream_t s) {
    static std::atomic<bool> configured{false};   // set once; concurrent first calls are harmless
    const size_t sm = stencil_smem<T, SMAG>();
    if (!configured) {
        cudaError_t e = set_smem(stencil2d<T, MODE, SMAG>, sm);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((G.nx + Tile<T>::TX - 1) / Tile<T>::TX, (G.nz + Tile<T>::TZ - 1) / Tile<T>::TZ);
    stencil2d<T, MODE, SMAG><<<grid, NTHREADS, sm, s>>>(G, u, v, Fu, f, out, out2, part, ctl, check_done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stencil(int mode, const Geo& G, const T* u, const T* v, const T* Fu,
                           const double* f, T* out, T* out2, double* part, Ctl* ctl,
                           int check_done, cudaStream_t s) {
    if (G.dim == 3) return launch_stencil3d<T>(mode, G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
#define JF_CASE(M)                                                                           \
    case M:                                                                                  \
        return G.sgs == 2 ? launch_stencil_t<T, M, 2>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s) \
             : G.smag     ? launch_stencil_t<T, M, 1>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s) \
                          : launch_stencil_t<T, M, 0>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
    switch (mode) {
        JF_CASE(MODE_F)
        JF_CASE(MODE_RHS)
        JF_CASE(MODE_RES)
        JF_CASE(MODE_JV)
        JF_CASE(MODE_RHSRES)
        default: return cudaErrorInvalidValue;
    }
#undef JF_CASE
}
template cudaError_t launch_stencil<float>(int, const Geo&, const float*, const float*, const float*,
                                           const double*, float*, float*, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_stencil<double>(int, const Geo&, const double*, const double*, const double*,
                                            const double*, double*, double*, double*, Ctl*, int, cudaStream_t);

// float32: persistent, double-buffered (one CTA per resident slot, capped at
// the tile count); float64: one tile per CTA.
template <typename T, int SMAG, int TX, int TZ>
static cudaError_t launch_jvd_t(const Geo& G, const T* u, const T* v, T* out, const double* part, Ctl* ctl,
                                int check_done, cudaStream_t s) {
    constexpr int NBUF = sizeof(T) == sizeof(float) ? 2 : 1;
    static std::atomic<int> slots{0};   // resident CTAs on the device; set once (races are benign)
    const size_t sm = jvd_smem<T, TX, TZ, NBUF>();
    if (slots.load() == 0) {
        cudaError_t e = set_smem(jv_diff2d<T, SMAG, TX, TZ, NBUF>, sm);
        if (e != cudaSuccess) return e;
        int dev = 0, nsm = 0, per = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jv_diff2d<T, SMAG, TX, TZ, NBUF>, NTHREADS,
                                                               sm)) != cudaSuccess)
            return e;
        slots = std::max(1, nsm * per);
    }
    const int ntiles = ((G.nx + TX - 1) / TX) * ((G.nz + TZ - 1) / TZ);
    const int grid = NBUF == 2 ? std::min(ntiles, slots.load()) : ntiles;
    return launch_pdl(jv_diff2d<T, SMAG, TX, TZ, NBUF>, dim3(grid), NTHREADS, sm, s, G, u, v, out,
                      (const double*)part, ctl, check_done);
}

// float32: the compute-once kernel jvc2d, persistent (one CTA per resident
// slot, capped at the tile count), double-buffered staging.
template <int SMAG, int TX, int TZ, int NBUF>
static cudaError_t launch_jvc_t(const Geo& G, const float* u, const float* v, float* out, const double* part,
                                Ctl* ctl, int check_done, cudaStream_t s) {
    static std::atomic<int> slots{0};   // resident CTAs on the device; set once (races are benign)
    const size_t sm = JvcShape<TX, TZ>::smem(NBUF);
    if (slots.load() == 0) {
        cudaError_t e = set_smem(jvc2d<SMAG, TX, TZ, NBUF>, sm);
        if (e != cudaSuccess) return e;
        int dev = 0, nsm = 0, per = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, jvc2d<SMAG, TX, TZ, NBUF>, NTHREADS, sm)) !=
                cudaSuccess)
            return e;
        slots = std::max(1, nsm * per);
    }
    const int ntiles = ((G.nx + TX - 1) / TX) * ((G.nz + TZ - 1) / TZ);
    const int grid = std::min(ntiles, slots.load());
    return launch_pdl(jvc2d<SMAG, TX, TZ, NBUF>, dim3(grid), NTHREADS, sm, s, G, u, v, out, part, ctl, check_done);
}

template <int SMAG>
static cudaError_t launch_jvc_tile(const Geo& G, const float* u, const float* v, float* out, const double* part,
                                   Ctl* ctl, int check_done, cudaStream_t s) {
#define JF_JVC(I) launch_jvc_t<SMAG, JvcTile<I>::TX, JvcTile<I>::TZ, JvcTile<I>::NBUF>(G, u, v, out, part, ctl, \
                                                                                     check_done, s)
    switch (G.tile_jv) {
        case 1: return JF_JVC(1);
        case 2: return JF_JVC(2);
        case 3: return JF_JVC(3);
        default: return JF_JVC(0);
    }
#undef JF_JVC
}

template <typename T, int SMAG>
static cudaError_t launch_jvd_tile(const Geo& G, const T* u, const T* v, T* out, const double* part, Ctl* ctl,
                                   int check_done, cudaStream_t s) {
    if constexpr (sizeof(T) == sizeof(double)) {
        return launch_jvd_t<T, SMAG, JvTile<1>::TX, JvTile<1>::TZ>(G, u, v, out, part, ctl, check_done, s);
    } else {
        return launch_jvc_tile<SMAG>(G, u, v, out, part, ctl, check_done, s);
    }
}

template <typename T>
cudaError_t launch_jv_diff(const Geo& G, const T* u, const T* v, T* out, double* part, Ctl* ctl,
                           int check_done, cudaStream_t s) {
    if (G.dim == 3) return launch_jv_diff3d<T>(G, u, v, out, ctl, check_done, s);
    if (G.sgs == 2) {
        // Deardorff: the float32 compute-once kernel only (float64 handles take the
        // plain forward difference of stencil2d)
        if constexpr (sizeof(T) == sizeof(float)) {
            return launch_jvc_tile<2>(G, u, v, out, part, ctl, check_done, s);
        } else {
            return cudaErrorNotSupported;
        }
    }
    return G.smag ? launch_jvd_tile<T, 1>(G, u, v, out, part, ctl, check_done, s)
                  : launch_jvd_tile<T, 0>(G, u, v, out, part, ctl, check_done, s);
}
template cudaError_t launch_jv_diff<float>(const Geo&, const float*, const float*, float*, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_jv_diff<double>(const Geo&, const double*, const double*, double*, double*, Ctl*, int, cudaStream_t);

static int stream_blocks(size_t n) {
    size_t b = (n + NTHREADS - 1) / NTHREADS;
    return (int)(b < (size_t)MAX_STREAM_BLOCKS ? (b > 0 ? b : 1) : MAX_STREAM_BLOCKS);
}

template <typename T>
cudaError_t launch_eddy(const Geo& G, const T* u, T* nu, double* part, Ctl* ctl, cudaStream_t s) {
    if (G.dim == 3) return launch_eddy3d<T>(G, u, nu, part, ctl, s);
    eddy2d<T><<<stream_blocks(G.npt), NTHREADS, 0, s>>>(G, u, nu, part, ctl);
    return cudaGetLastError();
}
template cudaError_t launch_eddy<float>(const Geo&, const float*, float*, double*, Ctl*, cudaStream_t);
template cudaError_t launch_eddy<double>(const Geo&, const double*, double*, double*, Ctl*, cudaStream_t);

template <typename T, int SMAG, int TX, int TZ>
static cudaError_t launch_precond_t(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da,
                                    T* db, const T* nu, double* part, Ctl* ctl, int check_done,
                                    cudaStream_t s, long long* launches) {
    const size_t n = (size_t)G.nf * G.npt;
    if (sweeps <= 1) {
        pc_diag<T, SMAG><<<stream_blocks(n), NTHREADS, 0, s>>>(G, r, z, n, part, ctl, check_done);
        if (launches) ++*launches;
        return cudaGetLastError();
    }
    dim3 grid((G.nx + TX - 1) / TX, (G.nz + TZ - 1) / TZ, 3);
    const size_t sm = sizeof(T) * ((TZ + 2 * HALO) * (TX + 2 * HALO) + TZ * (TX + 2 * R) +
                                   (TZ + 2 * R) * TX + (SMAG == 2 ? 2 : 1) * (TX + 2 * R) * (TZ + 2 * R));
    static std::atomic<bool> configured{false};   // set once; concurrent first calls are harmless
    if (!configured) {
        cudaError_t e;
        if ((e = set_smem(cheb2d<T, SMAG, 1, 1, TX, TZ>, sm)) != cudaSuccess) return e;
        if ((e = set_smem(cheb2d<T, SMAG, 1, 0, TX, TZ>, sm)) != cudaSuccess) return e;
        if ((e = set_smem(cheb2d<T, SMAG, 0, 1, TX, TZ>, sm)) != cudaSuccess) return e;
        if ((e = set_smem(cheb2d<T, SMAG, 0, 0, TX, TZ>, sm)) != cudaSuccess) return e;
        configured = true;
    }
    const T* zin = nullptr;
    const T* din = nullptr;
    T* zbuf[2] = {za, zb};
    T* dbuf[2] = {da, db};
    for (int k = 1; k <= sweeps - 1; ++k) {
        const bool first = k == 1, last = k == sweeps - 1;
        T* zo = last ? z : zbuf[k & 1];
        T* dO = dbuf[k & 1];
        grid.z = last ? 4 : 3;            // the p block is written by the last sweep only
        cudaError_t le;
        if (first && last)
            le = launch_pdl(cheb2d<T, SMAG, 1, 1, TX, TZ>, grid, NTHREADS, sm, s, G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        else if (first)
            le = launch_pdl(cheb2d<T, SMAG, 1, 0, TX, TZ>, grid, NTHREADS, sm, s, G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        else if (last)
            le = launch_pdl(cheb2d<T, SMAG, 0, 1, TX, TZ>, grid, NTHREADS, sm, s, G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        else
            le = launch_pdl(cheb2d<T, SMAG, 0, 0, TX, TZ>, grid, NTHREADS, sm, s, G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        if (launches) ++*launches;
        if (le != cudaSuccess) return le;
        zin = zo;
        din = dO;
    }
    return cudaSuccess;
}

template <typename T, int SMAG>
static cudaError_t launch_precond_tile(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da,
                                       T* db, const T* nu, double* part, Ctl* ctl, int check_done,
                                       cudaStream_t s, long long* launches) {
#define JF_PC(I) launch_precond_t<T, SMAG, PcTile<I>::TX, PcTile<I>::TZ>(G, sweeps, r, z, za, zb, da, db, nu, \
                                                                      part, ctl, check_done, s, launches)
    if (sizeof(T) == sizeof(double)) return JF_PC(1);
    switch (G.tile_pc) {
        case 1: return JF_PC(1);
        case 2: return JF_PC(2);
        case 3: return JF_PC(3);
        default: return JF_PC(0);
    }
#undef JF_PC
}

// Acoustic Schur complement: rhs (plane 0 of da), sweeps - 1 Helmholtz
// sweeps (iterates in plane 0 of za / zb, directions in planes 0 / 1 of db,
// the last one into plane 3 of z), then the back-substitution.
template <typename T>
static cudaError_t launch_schur(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da, T* db,
                                double* part, Ctl* ctl, int check_done, cudaStream_t s, long long* launches) {
    constexpr int TX = 64, TZ = 16;
    const size_t np = (size_t)G.npt;
    const size_t sm = sizeof(T) * ((TZ + 2 * HALO) * (TX + 2 * HALO) + TZ * (TX + 2 * R) + (TZ + 2 * R) * TX);
    T* rhs = da;
    schur_rhs2d<T><<<stream_blocks(np), NTHREADS, 0, s>>>(G, r, rhs, ctl, check_done);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;
    dim3 grid((G.nx + TX - 1) / TX, (G.nz + TZ - 1) / TZ);
    T* xbuf[2] = {za, zb};
    T* dbuf[2] = {db, db + np};
    const T* xin = nullptr;
    const T* din = nullptr;
    int cur = 1;                              // buffer pair the next output goes to
    const bool pairs = G.nz >= 2 * HALO;      // fused pairs need one mirror reflection of a 2*HALO halo
    const size_t sm2 = sizeof(T) * ((TZ + 4 * HALO) * (TX + 4 * HALO) + 3 * (TZ + 2 * HALO) * (TX + 2 * HALO) +
                                    (TZ + 2 * HALO) * (TX + 2 * HALO + 2 * R) + (TZ + 2 * HALO + 2 * R) * (TX + 2 * HALO));
    static std::atomic<bool> configured{false};
    if (!configured) {
        if ((e = set_smem(helm2d_x2<T, 1, 1, TX, TZ>, sm2)) != cudaSuccess) return e;
        if ((e = set_smem(helm2d_x2<T, 1, 0, TX, TZ>, sm2)) != cudaSuccess) return e;
        if ((e = set_smem(helm2d_x2<T, 0, 1, TX, TZ>, sm2)) != cudaSuccess) return e;
        if ((e = set_smem(helm2d_x2<T, 0, 0, TX, TZ>, sm2)) != cudaSuccess) return e;
        configured = true;
    }
    for (int k = 1; k <= sweeps - 1;) {
        const bool first = k == 1;
        const bool two = pairs && k + 1 <= sweeps - 1;
        const bool last = (two ? k + 1 : k) == sweeps - 1;
        T* xo = last ? z + 3 * np : xbuf[cur];
        T* dO = dbuf[cur];
        if (two) {
            if (first && last) helm2d_x2<T, 1, 1, TX, TZ><<<grid, NTHREADS, sm2, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
            else if (first) helm2d_x2<T, 1, 0, TX, TZ><<<grid, NTHREADS, sm2, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
            else if (last) helm2d_x2<T, 0, 1, TX, TZ><<<grid, NTHREADS, sm2, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
            else helm2d_x2<T, 0, 0, TX, TZ><<<grid, NTHREADS, sm2, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
        } else {
            if (first && last) helm2d<T, 1, 1, TX, TZ><<<grid, NTHREADS, sm, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
            else if (first) helm2d<T, 1, 0, TX, TZ><<<grid, NTHREADS, sm, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
            else if (last) helm2d<T, 0, 1, TX, TZ><<<grid, NTHREADS, sm, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
            else helm2d<T, 0, 0, TX, TZ><<<grid, NTHREADS, sm, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) ++*launches;
        xin = xo;
        din = dO;
        cur ^= 1;
        k += two ? 2 : 1;
    }
    schur_back2d<T><<<stream_blocks(np), NTHREADS, 0, s>>>(G, r, z, part, ctl, check_done);
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_precond(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da, T* db,
                           const T* nu, double* part, Ctl* ctl, int check_done, cudaStream_t s,
                           long long* launches) {
    if (G.pc_schur && G.dim == 2 && sweeps > 1)
        return launch_schur<T>(G, sweeps, r, z, za, zb, da, db, part, ctl, check_done, s, launches);
    if (G.dim == 3 && sweeps > 1)
        return launch_precond3d<T>(G, sweeps, r, z, za, zb, da, db, nu, part, ctl, check_done, s, launches);
    if (G.sgs == 2)
        return launch_precond_tile<T, 2>(G, sweeps, r, z, za, zb, da, db, nu, part, ctl, check_done, s, launches);
    return G.smag ? launch_precond_tile<T, 1>(G, sweeps, r, z, za, zb, da, db, nu, part, ctl, check_done, s, launches)
                  : launch_precond_tile<T, 0>(G, sweeps, r, z, za, zb, da, db, nu, part, ctl, check_done, s, launches);
}
template cudaError_t launch_precond<float>(const Geo&, int, const float*, float*, float*, float*, float*,
                                           float*, const float*, double*, Ctl*, int, cudaStream_t, long long*);
template cudaError_t launch_precond<double>(const Geo&, int, const double*, double*, double*, double*,
                                            double*, double*, const double*, double*, Ctl*, int, cudaStream_t,
                                            long long*);

cudaError_t launch_pc_setup(const Geo& G, int sweeps, Ctl* ctl, cudaStream_t s) {
    pc_setup<<<1, 32, 0, s>>>(G, sweeps, ctl);
    return cudaGetLastError();
}

cudaError_t launch_budgets(const Geo& G, const double* u, double dx, double dz, double lz,
                           double* part, Ctl* ctl, double* out, cudaStream_t s) {
    if (G.dim == 3) return launch_budgets3d(G, u, dx * dz / G.inv_dy, dz, lz, part, ctl, out, s);
    budgets2d<<<stream_blocks(G.npt), NTHREADS, 0, s>>>(G, u, dx * dz, dz, lz, part, ctl, out);
    return cudaGetLastError();
}

}  // namespace jfnk
