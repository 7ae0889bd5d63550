// 3-D stencil kernels of libjfnk: F(u), R(u), the Jacobian-vector products,
// the Smagorinsky eddy field, the field-block Chebyshev preconditioner and the
// budgets, for fields (u, v, w, theta, p) on [z][y][x] (x, y periodic; z
// cell-centred with signed mirror ghosts: w odd, theta and p even, u and v even
// for free slip / odd for no slip; the eddy field is mirrored even).
//
// Same discretisation as the 2-D kernels (Deslauriers-Dubuc p = 2 derivative,
// Section 2.3; skew-symmetric convection of every field, Section 2.2;
// Eqs. ch2_28-ch2_30 with Laplacian-form eddy diffusion, Section 2.4), with
// the Smagorinsky filter width Delta = (dx dy dz)^(1/3) and the full 3x3 strain.
//
// Tiling: one CTA computes TX x TY x TZ outputs.  Stage 1 stages the fields in
// a box with a halo of 2r = 4 in shared memory.  Stage 2 forms the first
// derivatives only on the three "arms" the second application of D reads:
// D_x on (tile + x-halo r), D_y on (tile + y-halo r), D_z on (tile + z-halo r),
// and the eddy coefficient on the same arms (from the 9 velocity gradients at
// each arm point; a ghost z row takes the value of its mirror image).  Stage 3
// assembles fluxes, diffusion and point-wise terms for the outputs.
#include <math.h>

#include <atomic>

#include "common.cuh"
#include "kernels.h"

namespace jfnk {
namespace d3 {

constexpr int R = 2;
constexpr int HALO = 2 * R;
constexpr int MODE_F = 0, MODE_RHS = 1, MODE_RES = 2, MODE_JV = 3, MODE_RHSRES = 4;

template <typename T>
__device__ __forceinline__ T dd(const T* s, int i, int st, T ih) {
    return (T(2.0 / 3.0) * (s[i + st] - s[i - st]) - T(1.0 / 12.0) * (s[i + 2 * st] - s[i - 2 * st])) * ih;
}
template <typename T>
__device__ __forceinline__ T ddp(const T* a, const T* b, int i, int st, T ih) {
    return (T(2.0 / 3.0) * (a[i + st] * b[i + st] - a[i - st] * b[i - st]) -
            T(1.0 / 12.0) * (a[i + 2 * st] * b[i + 2 * st] - a[i - 2 * st] * b[i - 2 * st])) * ih;
}

__device__ __forceinline__ int mirror(int gz, int nz, int& side) {
    side = 0;
    if (gz < 0) { side = 1; return -1 - gz; }
    if (gz >= nz) { side = 2; return 2 * nz - 1 - gz; }
    return gz;
}
__device__ __forceinline__ int wrap(int g, int n) {
    if ((unsigned)g < (unsigned)n) return g;
    int r = g % n;
    return r < 0 ? r + n : r;
}

// Box geometry of a TX x TY x TZ tile.
template <int TX, int TY, int TZ>
struct Box {
    static constexpr int SX = TX + 2 * HALO, SY = TY + 2 * HALO, SZ = TZ + 2 * HALO;
    static constexpr int SXY = SX * SY, PL = SX * SY * SZ;
    static constexpr int QX = TX + 2 * R, QY = TY + 2 * R, QZ = TZ + 2 * R;
    static constexpr int AX = QX * TY * TZ, AY = TX * QY * TZ, AZ = TX * TY * QZ;
    static constexpr int AS = AX + AY + AZ;              // one field's three arms
    // box index of box coordinates
    __device__ static int b(int ix, int iy, int iz) { return (iz * SY + iy) * SX + ix; }
    // arm indices (centre of output (tx,ty,tz) is qx = tx + R etc.)
    __device__ static int ax(int qx, int ty, int tz) { return (tz * TY + ty) * QX + qx; }
    __device__ static int ay(int tx, int qy, int tz) { return AX + (tz * QY + qy) * TX + tx; }
    __device__ static int az(int tx, int ty, int qz) { return AX + AY + (qz * TY + ty) * TX + tx; }
};

// Stage 1: NF fields from f0 into s[q][PL]; LOADMODE 0: u, 1: u + ev v, 2: ev v.
template <typename T, int LOADMODE, int NF, int TX, int TY, int TZ>
__device__ __forceinline__ void load_box(T* s, const T* __restrict__ u, const T* __restrict__ v,
                                         const T (&ev)[5], const Geo& G, int x0, int y0, int z0,
                                         int f0) {
    using B = Box<TX, TY, TZ>;
    for (int idx = threadIdx.x; idx < B::PL; idx += blockDim.x) {
        const int ix = idx % B::SX, r1 = idx / B::SX;
        const int iy = r1 % B::SY, iz = r1 / B::SY;
        int side;
        const int sz = mirror(z0 + iz - HALO, G.nz, side);
        const int sy = wrap(y0 + iy - HALO, G.ny);
        const int sx = wrap(x0 + ix - HALO, G.nx);
        const bool ok = sz >= 0 && sz < G.nz;
        const size_t off = ((size_t)sz * G.ny + sy) * G.nx + sx;
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
            s[q * B::PL + idx] = val;
        }
    }
}

// Stage 2: derivative arms of field box s into g (one field: AS values).
template <typename T, int TX, int TY, int TZ>
__device__ __forceinline__ void arms(const T* s, T* g, T ix_, T iy_, T iz_) {
    using B = Box<TX, TY, TZ>;
    for (int idx = threadIdx.x; idx < B::AS; idx += blockDim.x) {
        int bx, by, bz, st;
        T ih;
        if (idx < B::AX) {
            const int qx = idx % B::QX, r1 = idx / B::QX;
            bx = qx + R; by = r1 % TY + HALO; bz = r1 / TY + HALO; st = 1; ih = ix_;
        } else if (idx < B::AX + B::AY) {
            const int j = idx - B::AX;
            const int tx = j % TX, r1 = j / TX;
            bx = tx + HALO; by = r1 % B::QY + R; bz = r1 / B::QY + HALO; st = B::SX; ih = iy_;
        } else {
            const int j = idx - B::AX - B::AY;
            const int tx = j % TX, r1 = j / TX;
            bx = tx + HALO; by = r1 % TY + HALO; bz = r1 / TY + R; st = B::SXY; ih = iz_;
        }
        g[idx] = dd(s, B::b(bx, by, bz), st, ih);
    }
}

// Box coordinates of arm point idx (and whether it is a z arm).
template <int TX, int TY, int TZ>
__device__ __forceinline__ void arm_point(int idx, int& bx, int& by, int& bz, bool& zarm) {
    using B = Box<TX, TY, TZ>;
    zarm = false;
    if (idx < B::AX) {
        const int qx = idx % B::QX, r1 = idx / B::QX;
        bx = qx + R; by = r1 % TY + HALO; bz = r1 / TY + HALO;
    } else if (idx < B::AX + B::AY) {
        const int j = idx - B::AX;
        const int tx = j % TX, r1 = j / TX;
        bx = tx + HALO; by = r1 % B::QY + R; bz = r1 / B::QY + HALO;
    } else {
        const int j = idx - B::AX - B::AY;
        const int tx = j % TX, r1 = j / TX;
        bx = tx + HALO; by = r1 % TY + HALO; bz = r1 / TY + R;
        zarm = true;
    }
}

// For a z-arm point in a ghost row, the box row of its mirror image (even
// reflection of the eddy field); -1 if the row is never read.
__device__ __forceinline__ int eddy_box_row(int bz, int z0, int nz) {
    const int gz = z0 + bz - HALO;
    if (gz >= 0 && gz < nz) return bz;
    if (gz < 0) return (-1 - gz) - z0 + HALO;
    if (gz < nz + R) return (2 * nz - 1 - gz) - z0 + HALO;
    return -1;
}

// Velocity gradient at box point c of boxes U, V, W: g[i][j] = D_j u_i.
template <typename T, int SX, int SXY>
__device__ __forceinline__ void grad3(const T* U, const T* V, const T* W, int c, T ix_, T iy_, T iz_,
                                      T (&g)[3][3]) {
    const T* comp[3] = {U, V, W};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        g[i][0] = dd(comp[i], c, 1, ix_);
        g[i][1] = dd(comp[i], c, SX, iy_);
        g[i][2] = dd(comp[i], c, SXY, iz_);
    }
}

// Deardorff coefficient along an arm (Section 2.4, Eq. KmM) from the strain s:
// momentum c s with c = K_m / s along x and y, K_M / s along z; heat times
// 1 + a l(s), a = 2 / sqrt(dx dy) horizontally, 2 / dz vertically.
template <typename T>
__device__ __forceinline__ T dd3_coef(T s, bool zarm, bool heat, const Geo& G) {
    const T c = T(zarm ? G.dd_cM : G.dd_cm);
    if (!heat) return c * s;
    const T cls = T(G.dd_cl) * s;
    const T l = G.dd_cl < 0.0 ? T(G.dd_delta) : (cls < T(G.dd_delta) ? cls : T(G.dd_delta));
    return c * (s * (T(1) + T(zarm ? G.dd_az : G.dd_ah) * l));
}

template <typename T>
__device__ __forceinline__ T strain_sq(const T (&g)[3][3]) {    // S_ij S_ij
    T ss = T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const T s = T(0.5) * (g[i][j] + g[j][i]);
            ss += s * s;
        }
    return ss;
}

// ============================================================================
// F, 2u/dt + F, residual and plain forward-difference Jv
// ============================================================================
template <typename T, int MODE, int SMAG, int TX, int TY, int TZ>
__global__ void __launch_bounds__(NTHREADS)
stencil3d(Geo G, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ Fu,
          const double* __restrict__ f, T* __restrict__ out, T* __restrict__ out2,
          double* __restrict__ part, Ctl* ctl, int check_done) {
    using B = Box<TX, TY, TZ>;
    if (MODE == MODE_JV && check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s1 = reinterpret_cast<T*>(smem_raw);        // [5][PL]
    T* g = s1 + 5 * B::PL;                          // [4][AS] derivative arms of u, v, w, theta
    T* nu = g + 4 * B::AS;                          // [AS] eddy coefficient on the arms
    T* kh = nu + B::AS;                             // [AS] Deardorff: heat coefficient on the arms
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const T ix_ = T(G.inv_dx), iy_ = T(G.inv_dy), iz_ = T(G.inv_dz);
    __shared__ double cfs[5];
    __shared__ T evs[5];
    T ev[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (MODE == MODE_JV) {
        if (threadIdx.x < 5) {
            const double e = ctl->eps_jv * G.scale[threadIdx.x];
            evs[threadIdx.x] = T(e);
            cfs[threadIdx.x] = e != 0.0 ? 1.0 / e : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 5; ++q) ev[q] = evs[q];
        load_box<T, 1, 5, TX, TY, TZ>(s1, u, v, ev, G, x0, y0, z0, 0);
    } else {
        load_box<T, 0, 5, TX, TY, TZ>(s1, u, v, ev, G, x0, y0, z0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) arms<T, TX, TY, TZ>(s1 + q * B::PL, g + q * B::AS, ix_, iy_, iz_);
    if (SMAG) {
        const T cs2 = T(G.cs2);
        for (int idx = threadIdx.x; idx < B::AS; idx += blockDim.x) {
            int bx, by, bz;
            bool zarm;
            arm_point<TX, TY, TZ>(idx, bx, by, bz, zarm);
            T val = T(0);
            const int bzz = zarm ? eddy_box_row(bz, z0, G.nz) : bz;
            T hv = T(0);
            if (bzz >= 0) {
                T gr[3][3];
                grad3<T, B::SX, B::SXY>(s1, s1 + B::PL, s1 + 2 * B::PL, B::b(bx, by, bzz), ix_, iy_, iz_, gr);
                if (SMAG == 2) {
                    // Deardorff: the arm's own direction picks K_m / K_M and K_h / K_H
                    const T sv = sqrt(T(2) * strain_sq(gr));
                    val = dd3_coef(sv, zarm, false, G);
                    hv = dd3_coef(sv, zarm, true, G);
                } else {
                    val = cs2 * sqrt(T(2) * strain_sq(gr));
                }
            }
            nu[idx] = val;
            if (SMAG == 2) kh[idx] = hv;
        }
    }
    __syncthreads();

    const T* U = s1;
    const T* Vv = s1 + B::PL;
    const T* W = s1 + 2 * B::PL;
    const T* P = s1 + 4 * B::PL;
    const T KMc = T(G.K_M), KHc = T(G.K_H), iPr = T(G.inv_Pr), th0 = T(G.theta0);
    double acc[2] = {0.0, 0.0};
    for (int idx = threadIdx.x; idx < TX * TY * TZ; idx += blockDim.x) {
        const int tx = idx % TX, r1 = idx / TX;
        const int ty = r1 % TY, tz = r1 / TY;
        const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
        if (gx >= G.nx || gy >= G.ny || gz >= G.nz) continue;
        const int c = B::b(tx + HALO, ty + HALO, tz + HALO);
        const int cx = B::ax(tx + R, ty, tz), cy = B::ay(tx, ty + R, tz), cz = B::az(tx, ty, tz + R);
        const T uc = U[c], vc = Vv[c], wc = W[c];
        const T px = dd(P, c, 1, ix_), py = dd(P, c, B::SX, iy_), pz = dd(P, c, B::SXY, iz_);
        T Fv[5];
#pragma unroll
        for (int fl = 0; fl < 5; ++fl) {
            const T* Ph = s1 + fl * B::PL;
            T dxp, dyp, dzp;
            if (fl < 4) {
                const T* gf = g + fl * B::AS;
                dxp = gf[cx]; dyp = gf[cy]; dzp = gf[cz];
            } else {
                dxp = px; dyp = py; dzp = pz;
            }
            const T conv = T(0.5) * (ddp(U, Ph, c, 1, ix_) + ddp(Vv, Ph, c, B::SX, iy_) + ddp(W, Ph, c, B::SXY, iz_)) +
                           T(0.5) * (uc * dxp + vc * dyp + wc * dzp);
            T dif = T(0);
            if (fl < 4) {
                const T* gf = g + fl * B::AS;
                if (SMAG == 2) {
                    const T* kf = fl == 3 ? kh : nu;
                    dif = ddp(kf, gf, cx, 1, ix_) + ddp(kf, gf, cy, TX, iy_) + ddp(kf, gf, cz, TX * TY, iz_);
                } else if (SMAG) {
                    dif = ddp(nu, gf, cx, 1, ix_) + ddp(nu, gf, cy, TX, iy_) + ddp(nu, gf, cz, TX * TY, iz_);
                    if (fl == 3) dif *= iPr;
                } else {
                    dif = (fl == 3 ? KHc : KMc) * (dd(gf, cx, 1, ix_) + dd(gf, cy, TX, iy_) + dd(gf, cz, TX * TY, iz_));
                }
            }
            Fv[fl] = -conv + dif;
        }
        const T div = g[cx] + g[B::AS + cy] + g[2 * B::AS + cz];
        Fv[0] += -th0 * px;
        Fv[1] += -th0 * py;
        Fv[2] += -th0 * pz + T(G.g) * s1[3 * B::PL + c] / th0;
        Fv[3] += -T(G.beta) * wc;
        if (G.heat != nullptr && gz == 0) Fv[3] += T(G.heat[(size_t)gy * G.nx + gx] * G.heat_coef);
        Fv[4] += -T(G.gamma_p) * (T(G.pbar) + P[c]) * div;
        const size_t off = ((size_t)gz * G.ny + gy) * G.nx + gx;
#pragma unroll
        for (int fl = 0; fl < 5; ++fl) {
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
            } else {
                const double vh = (double)v[o];
                const double diff = (double)Fv[fl] - (double)Fu[o];
                out[o] = T(G.two_over_dt * vh - diff * cfs[fl]);
            }
        }
    }
    if (MODE == MODE_RES || MODE == MODE_RHSRES) {
        const int nblk = gridDim.x * gridDim.y * gridDim.z;
        const int blk = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
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
// Mixed-path Jv in difference form (a = u, b = eps V, a' = a + b): every term
// of F(a') - F(a) expanded as a difference, as in the 2-D kernel.
// ============================================================================
template <typename T, int SMAG, int TX, int TY, int TZ>
__global__ void __launch_bounds__(NTHREADS)
jv_diff3d(Geo G, const T* __restrict__ u, const T* __restrict__ v, T* __restrict__ out, Ctl* ctl,
          int check_done) {
    using B = Box<TX, TY, TZ>;
    if (check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sa = reinterpret_cast<T*>(smem_raw);        // [5][PL]
    T* sb = sa + 5 * B::PL;                         // [5][PL]
    T* ga = sb + 5 * B::PL;                         // [4][AS]
    T* gb = ga + 4 * B::AS;                         // [4][AS]
    T* Ka = gb + 4 * B::AS;                         // [AS]
    T* dK = Ka + B::AS;                             // [AS]
    T* Kh = dK + B::AS;                             // [AS] Deardorff: heat coefficient and its difference
    T* dKh = Kh + B::AS;                            // [AS]
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * TZ;
    const T ix_ = T(G.inv_dx), iy_ = T(G.inv_dy), iz_ = T(G.inv_dz);
    __shared__ T cfs[5];
    __shared__ T evs[5];
    if (threadIdx.x < 5) {
        const double e = ctl->eps_jv * G.scale[threadIdx.x];
        evs[threadIdx.x] = T(e);
        cfs[threadIdx.x] = T(e != 0.0 ? 1.0 / e : 0.0);
    }
    __syncthreads();
    T ev[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) ev[q] = evs[q];
    load_box<T, 0, 5, TX, TY, TZ>(sa, u, v, ev, G, x0, y0, z0, 0);
    load_box<T, 2, 5, TX, TY, TZ>(sb, u, v, ev, G, x0, y0, z0, 0);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        arms<T, TX, TY, TZ>(sa + q * B::PL, ga + q * B::AS, ix_, iy_, iz_);
        arms<T, TX, TY, TZ>(sb + q * B::PL, gb + q * B::AS, ix_, iy_, iz_);
    }
    if (SMAG) {
        const T cs2 = T(G.cs2);
        for (int idx = threadIdx.x; idx < B::AS; idx += blockDim.x) {
            int bx, by, bz;
            bool zarm;
            arm_point<TX, TY, TZ>(idx, bx, by, bz, zarm);
            T ka = T(0), dk = T(0), kh_ = T(0), dkh_ = T(0);
            const int bzz = zarm ? eddy_box_row(bz, z0, G.nz) : bz;
            if (bzz >= 0) {
                const int c = B::b(bx, by, bzz);
                T gA[3][3], gB[3][3];
                grad3<T, B::SX, B::SXY>(sa, sa + B::PL, sa + 2 * B::PL, c, ix_, iy_, iz_, gA);
                grad3<T, B::SX, B::SXY>(sb, sb + B::PL, sb + 2 * B::PL, c, ix_, iy_, iz_, gB);
                T ssa = T(0), dss = T(0);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const T sA = T(0.5) * (gA[i][j] + gA[j][i]);
                        const T sB = T(0.5) * (gB[i][j] + gB[j][i]);
                        ssa += sA * sA;
                        dss += (T(2) * sA + sB) * sB;       // S':S' - S:S
                    }
                const T na = sqrt(T(2) * ssa);
                const T tp = T(2) * (ssa + dss);
                const T np = sqrt(tp > T(0) ? tp : T(0));
                const T den = na + np;
                const T ds = den > T(0) ? T(2) * dss / den : T(0);     // s' - s, cancellation-free
                if (SMAG == 2) {
                    // Deardorff: the arm's direction picks the coefficient; heat by its difference
                    // form g(s') - g(s) = ds (1 + a l') + a s (l' - l) (l' - l = c_l ds below the cap)
                    ka = dd3_coef(na, zarm, false, G);
                    dk = dd3_coef(ds, zarm, false, G);
                    const T c = T(zarm ? G.dd_cM : G.dd_cm), a = T(zarm ? G.dd_az : G.dd_ah);
                    T la = T(G.dd_delta), lp = T(G.dd_delta), dl = T(0);
                    if (G.dd_cl >= 0.0) {
                        const T ta = T(G.dd_cl) * na, tq = T(G.dd_cl) * np;
                        la = ta < T(G.dd_delta) ? ta : T(G.dd_delta);
                        lp = tq < T(G.dd_delta) ? tq : T(G.dd_delta);
                        if (ta < T(G.dd_delta) && tq < T(G.dd_delta)) dl = T(G.dd_cl) * ds;
                        else if (ta < T(G.dd_delta) || tq < T(G.dd_delta)) dl = lp - la;
                    }
                    kh_ = c * (na * (T(1) + a * la));
                    dkh_ = c * (ds * (T(1) + a * lp) + a * na * dl);
                } else {
                    ka = cs2 * na;
                    dk = cs2 * ds;
                }
            }
            Ka[idx] = ka;
            dK[idx] = dk;
            if (SMAG == 2) {
                Kh[idx] = kh_;
                dKh[idx] = dkh_;
            }
        }
    }
    __syncthreads();
    const T KMc = T(G.K_M), KHc = T(G.K_H), iPr = T(G.inv_Pr), th0 = T(G.theta0);
    const T* AU[3] = {sa, sa + B::PL, sa + 2 * B::PL};
    const T* BU[3] = {sb, sb + B::PL, sb + 2 * B::PL};
    const int sts[3] = {1, B::SX, B::SXY};
    const T ihs[3] = {ix_, iy_, iz_};
    for (int idx = threadIdx.x; idx < TX * TY * TZ; idx += blockDim.x) {
        const int tx = idx % TX, r1 = idx / TX;
        const int ty = r1 % TY, tz = r1 / TY;
        const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
        if (gx >= G.nx || gy >= G.ny || gz >= G.nz) continue;
        const int c = B::b(tx + HALO, ty + HALO, tz + HALO);
        const int ca[3] = {B::ax(tx + R, ty, tz), B::ay(tx, ty + R, tz), B::az(tx, ty, tz + R)};
        const int ast[3] = {1, TX, TX * TY};       // arm strides along x, y, z
        T dapc[3], dbpc[3];
        const T* AP = sa + 4 * B::PL;
        const T* BP = sb + 4 * B::PL;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            dapc[j] = dd(AP, c, sts[j], ihs[j]);
            dbpc[j] = dd(BP, c, sts[j], ihs[j]);
        }
        T dF[5];
#pragma unroll
        for (int fl = 0; fl < 5; ++fl) {
            const T* A = sa + fl * B::PL;
            const T* Bf = sb + fl * B::PL;
            T flux = T(0), adv = T(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const T* aj = AU[j];
                const T* bj = BU[j];
                const int st = sts[j];
                T fj = T(0);
#pragma unroll
                for (int l = 1; l <= 2; ++l) {
                    const T cl = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
                    const int ip = c + l * st, im = c - l * st;
                    fj += cl * ((aj[ip] * Bf[ip] + bj[ip] * (A[ip] + Bf[ip])) -
                                (aj[im] * Bf[im] + bj[im] * (A[im] + Bf[im])));
                }
                flux += fj * ihs[j];
                T daj, dbj;
                if (fl < 4) { daj = ga[fl * B::AS + ca[j]]; dbj = gb[fl * B::AS + ca[j]]; }
                else { daj = dapc[j]; dbj = dbpc[j]; }
                adv += aj[c] * dbj + bj[c] * (daj + dbj);
            }
            dF[fl] = -(T(0.5) * flux + T(0.5) * adv);
            if (fl < 4) {
                const T* gaf = ga + fl * B::AS;
                const T* gbf = gb + fl * B::AS;
                T dif = T(0);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const int q = ca[j], st = ast[j];
                    T sj = T(0);
#pragma unroll
                    for (int l = 1; l <= 2; ++l) {
                        const T cl = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
                        const int p1 = q + l * st, m1 = q - l * st;
                        if (SMAG) {
                            const T* K1 = (SMAG == 2 && fl == 3) ? Kh : Ka;
                            const T* d1 = (SMAG == 2 && fl == 3) ? dKh : dK;
                            sj += cl * ((K1[p1] * gbf[p1] + d1[p1] * (gaf[p1] + gbf[p1])) -
                                        (K1[m1] * gbf[m1] + d1[m1] * (gaf[m1] + gbf[m1])));
                        } else {
                            sj += cl * (gbf[p1] - gbf[m1]);
                        }
                    }
                    dif += sj * ihs[j];
                }
                if (SMAG == 1) { if (fl == 3) dif *= iPr; } else if (!SMAG) dif *= (fl == 3 ? KHc : KMc);
                dF[fl] += dif;
            }
        }
        dF[0] += -th0 * dbpc[0];
        dF[1] += -th0 * dbpc[1];
        dF[2] += -th0 * dbpc[2] + T(G.g) * sb[3 * B::PL + c] / th0;
        dF[3] += -T(G.beta) * sb[2 * B::PL + c];
        const T diva = ga[ca[0]] + ga[B::AS + ca[1]] + ga[2 * B::AS + ca[2]];
        const T divb = gb[ca[0]] + gb[B::AS + ca[1]] + gb[2 * B::AS + ca[2]];
        dF[4] += -T(G.gamma_p) * ((T(G.pbar) + AP[c] + BP[c]) * divb + BP[c] * diva);
        const size_t off = ((size_t)gz * G.ny + gy) * G.nx + gx;
#pragma unroll
        for (int fl = 0; fl < 5; ++fl) {
            const size_t o = (size_t)fl * G.npt + off;
            out[o] = T(G.two_over_dt) * v[o] - dF[fl] * cfs[fl];
        }
    }
}

// ============================================================================
// Smagorinsky eddy field at every point (preconditioner input) and its maximum
// ============================================================================
template <typename T>
__global__ void __launch_bounds__(NTHREADS)
eddy3d(Geo G, const T* __restrict__ u, T* __restrict__ nu, double* part, Ctl* ctl) {
    T mxT = T(0);
    const T ih[3] = {T(G.inv_dx), T(G.inv_dy), T(G.inv_dz)};
    const T cs2 = G.sgs == 2 ? T(1) : T(G.cs2);     // Deardorff: the strain s itself
    const int nxy = G.nx * G.ny;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < G.npt; p += gridDim.x * blockDim.x) {
        const int z = p / nxy, rem = p - z * nxy;
        const int y = rem / G.nx, x = rem - y * G.nx;
        T gr[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const T* C = u + (size_t)i * G.npt;
            T dxv = T(0), dyv = T(0), dzv = T(0);
#pragma unroll
            for (int l = 1; l <= 2; ++l) {
                const T cl = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
                dxv += cl * (C[(size_t)z * nxy + y * G.nx + wrap(x + l, G.nx)] -
                             C[(size_t)z * nxy + y * G.nx + wrap(x - l, G.nx)]);
                dyv += cl * (C[(size_t)z * nxy + wrap(y + l, G.ny) * G.nx + x] -
                             C[(size_t)z * nxy + wrap(y - l, G.ny) * G.nx + x]);
                int sp_, sm_;
                const int zp = mirror(z + l, G.nz, sp_), zm = mirror(z - l, G.nz, sm_);
                const T gp = sp_ == 2 ? T(G.pt[i]) : T(1), gm = sm_ == 1 ? T(G.pb[i]) : T(1);
                dzv += cl * (gp * C[(size_t)zp * nxy + y * G.nx + x] - gm * C[(size_t)zm * nxy + y * G.nx + x]);
            }
            gr[i][0] = dxv * ih[0];
            gr[i][1] = dyv * ih[1];
            gr[i][2] = dzv * ih[2];
        }
        const T val = cs2 * sqrt(T(2) * strain_sq(gr));
        nu[p] = val;
        mxT = val > mxT ? val : mxT;
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
// Field-block Chebyshev sweep (same recurrence as the 2-D kernel, Section 2.5.2):
// one CTA = one field of one tile; p (field 4) is written by the last sweep.
// ============================================================================
template <typename T, int SMAG, int FIRST, int LAST, int TX, int TY, int TZ>
__global__ void __launch_bounds__(NTHREADS)
cheb3d(Geo G, int k, const T* __restrict__ r, const T* __restrict__ zin, const T* __restrict__ din,
       T* __restrict__ zout, T* __restrict__ dout, const T* __restrict__ nu, double* part, Ctl* ctl,
       int check_done) {
    using B = Box<TX, TY, TZ>;
    if (check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* zs = reinterpret_cast<T*>(smem_raw);      // [PL]
    T* g = zs + B::PL;                              // [AS] derivative arms of x_k
    T* kk = g + B::AS;                              // [AS] eddy coefficient on the arms
    const int fld = blockIdx.z % 5;
    const int zt = blockIdx.z / 5;                  // z tile
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = zt * TZ;
    const T ith = T(ctl->cheb[fld][k][0]);
    const T a1 = T(ctl->cheb[fld][k][1]);
    const T a2 = T(ctl->cheb[fld][k][2]);
    const size_t foff = (size_t)fld * G.npt;
    T acc[1] = {T(0)};
    if (fld == 4) {
        if (LAST) {
            for (int idx = threadIdx.x; idx < TX * TY * TZ; idx += blockDim.x) {
                const int tx = idx % TX, r1 = idx / TX;
                const int ty = r1 % TY, tz = r1 / TY;
                const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
                if (gx >= G.nx || gy >= G.ny || gz >= G.nz) continue;
                const size_t o = foff + ((size_t)gz * G.ny + gy) * G.nx + gx;
                const T zv = r[o] * ith;
                zout[o] = zv;
                acc[0] += zv * zv;
            }
        }
    } else {
        T sc[5] = {T(0), T(0), T(0), T(0), T(0)};
        if (FIRST) {
            sc[fld] = ith;
            load_box<T, 2, 1, TX, TY, TZ>(zs, nullptr, r, sc, G, x0, y0, z0, fld);
        } else {
            load_box<T, 0, 1, TX, TY, TZ>(zs, zin, nullptr, sc, G, x0, y0, z0, fld);
        }
        if (SMAG) {
            const T kscale = fld == 3 ? T(G.inv_Pr) : T(1);
            for (int idx = threadIdx.x; idx < B::AS; idx += blockDim.x) {
                int bx, by, bz;
                bool zarm;
                arm_point<TX, TY, TZ>(idx, bx, by, bz, zarm);
                int side;
                const int sz = mirror(z0 + bz - HALO, G.nz, side);    // even mirror of nu
                const int sy = wrap(y0 + by - HALO, G.ny), sx = wrap(x0 + bx - HALO, G.nx);
                const T nv = (sz >= 0 && sz < G.nz) ? nu[((size_t)sz * G.ny + sy) * G.nx + sx] : T(0);
                // Deardorff: nu holds the strain and the arm's direction picks the coefficient
                kk[idx] = SMAG == 2 ? dd3_coef(nv, zarm, fld == 3, G) : nv * kscale;
            }
        }
        __syncthreads();
        arms<T, TX, TY, TZ>(zs, g, T(G.inv_dx), T(G.inv_dy), T(G.inv_dz));
        __syncthreads();
        const T Kc = T(fld == 3 ? G.K_H : G.K_M);
        const T tdt = T(G.two_over_dt);
        const T ihs[3] = {T(G.inv_dx), T(G.inv_dy), T(G.inv_dz)};
        for (int idx = threadIdx.x; idx < TX * TY * TZ; idx += blockDim.x) {
            const int tx = idx % TX, r1 = idx / TX;
            const int ty = r1 % TY, tz = r1 / TY;
            const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
            if (gx >= G.nx || gy >= G.ny || gz >= G.nz) continue;
            const int ca[3] = {B::ax(tx + R, ty, tz), B::ay(tx, ty + R, tz), B::az(tx, ty, tz + R)};
            const int ast[3] = {1, TX, TX * TY};
            T dif = T(0);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (SMAG) dif += ddp(kk, g, ca[j], ast[j], ihs[j]);
                else dif += Kc * dd(g, ca[j], ast[j], ihs[j]);
            }
            const T xk = zs[B::b(tx + HALO, ty + HALO, tz + HALO)];
            const size_t o = foff + ((size_t)gz * G.ny + gy) * G.nx + gx;
            const T rv = r[o];
            const T res = rv - (tdt * xk - dif);
            const T dprev = FIRST ? rv * ith : din[o];
            const T dk = a1 * dprev + a2 * res;
            const T xn = xk + dk;
            zout[o] = xn;
            if (!LAST) dout[o] = dk;
            if (LAST) acc[0] += xn * xn;
        }
    }
    if (LAST) {
        const int nblk = gridDim.x * gridDim.y * gridDim.z;
        const int blk = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
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

// ============================================================================
// Budgets: E_k = 1/2 sum (u^2+v^2+w^2) dV, E_p = sum (lz - z) theta dV,
// sum theta dV, sum div(u) dV, max / min of the five fields.
// ============================================================================
__global__ void __launch_bounds__(NTHREADS)
budgets3d(Geo G, const double* __restrict__ u, double dV, double dz, double lz, double* part,
          Ctl* ctl, double* out) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    double mx[10];
    for (int f = 0; f < 10; ++f) mx[f] = -1e300;
    const int nxy = G.nx * G.ny;
    const double* U = u;
    const double* Vv = u + G.npt;
    const double* W = u + 2 * (size_t)G.npt;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < G.npt; p += gridDim.x * blockDim.x) {
        const int z = p / nxy, rem = p - z * nxy;
        const int y = rem / G.nx, x = rem - y * G.nx;
        const double zc = (z + 0.5) * dz;
        s[0] += 0.5 * (U[p] * U[p] + Vv[p] * Vv[p] + W[p] * W[p]);
        s[1] += (lz - zc) * u[3 * (size_t)G.npt + p];
        s[2] += u[3 * (size_t)G.npt + p];
        double ux = 0.0, vy = 0.0, wz = 0.0;
        for (int l = 1; l <= 2; ++l) {
            const double c = l == 1 ? 2.0 / 3.0 : -1.0 / 12.0;
            ux += c * (U[(size_t)z * nxy + y * G.nx + wrap(x + l, G.nx)] - U[(size_t)z * nxy + y * G.nx + wrap(x - l, G.nx)]);
            vy += c * (Vv[(size_t)z * nxy + wrap(y + l, G.ny) * G.nx + x] - Vv[(size_t)z * nxy + wrap(y - l, G.ny) * G.nx + x]);
            int sp_, sm_;
            const int zp = mirror(z + l, G.nz, sp_), zm = mirror(z - l, G.nz, sm_);
            const double gp = sp_ == 2 ? -1.0 : 1.0, gm = sm_ == 1 ? -1.0 : 1.0;   // w odd at both walls
            wz += c * (gp * W[(size_t)zp * nxy + y * G.nx + x] - gm * W[(size_t)zm * nxy + y * G.nx + x]);
        }
        s[3] += ux * G.inv_dx + vy * G.inv_dy + wz * G.inv_dz;
        for (int f = 0; f < 5; ++f) {
            const double val = u[(size_t)f * G.npt + p];
            mx[f] = max_nan(mx[f], val);
            mx[5 + f] = max_nan(mx[5 + f], -val);
        }
    }
    double* pmax = part + 4 * gridDim.x;
    block_partials<4>(s, 4, part, gridDim.x, blockIdx.x);
    block_partials_max<10>(mx, 10, pmax, gridDim.x, blockIdx.x);
    if (arrive_last(&ctl->counter[CNT_MISC], gridDim.x)) {
        __shared__ double tot[14];
        final_sums(part, gridDim.x, 4, tot);
        final_maxes(pmax, gridDim.x, 10, tot + 4);
        if (threadIdx.x == 0) {
            for (int i = 0; i < 4; ++i) out[i] = tot[i] * dV;
            for (int f = 0; f < 5; ++f) { out[4 + f] = tot[4 + f]; out[9 + f] = -tot[9 + f]; }
        }
    }
}

// ------------------------------------------------------------------ tiles
template <typename T> struct FTile;          // F / residual / plain Jv
template <> struct FTile<float>  { static constexpr int TX = 16, TY = 8, TZ = 4; };
template <> struct FTile<double> { static constexpr int TX = 8, TY = 8, TZ = 4; };
template <typename T> struct DTile;          // difference-form Jv (two states staged)
template <> struct DTile<float>  { static constexpr int TX = 8, TY = 8, TZ = 4; };
template <> struct DTile<double> { static constexpr int TX = 4, TY = 4, TZ = 4; };
template <typename T> struct CTile;          // Chebyshev sweep (one field)
template <> struct CTile<float>  { static constexpr int TX = 16, TY = 8, TZ = 4; };
template <> struct CTile<double> { static constexpr int TX = 16, TY = 8, TZ = 4; };

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// ---------------------------------------------------------------------------
// Acoustic Schur-complement preconditioner in 3-D (scaled units): the 2-D
// construction with three velocity components,
//   H dp = v_p - c_div (D_x v_u + D_y v_v + D_z v_w),  H = (2/dt) I - a sum_j D_j D_j,
//   z_i = (dt/2)(v_i - c_grad D_i dp),  z_theta = v_theta / theta_c,
// with H applied point-wise as the composite stencil of the first derivative
// taken twice along each axis (coefficients c_s = sum_{a+b=s} w_a w_b: -65/72,
// 1/9, 4/9, -1/9, 1/144 for |s| = 0..4) on the ghost-extended plane (p even
// at the walls), which equals D_j applied to D_j dp evaluated with its ghosts.
// Fields: 0 u, 1 v, 2 w, 3 theta, 4 p; planes [z][y][x].
template <typename T>
__device__ __forceinline__ T pz(const T* __restrict__ f, const Geo& G, int gz, int gy, int gx, int fld) {
    int side;
    const int sz = mirror(gz, G.nz, side);
    const T v = f[((size_t)sz * G.ny + gy) * G.nx + gx];
    return side == 1 ? T(G.pb[fld]) * v : (side == 2 ? T(G.pt[fld]) * v : v);
}

template <typename T>
__device__ __forceinline__ T d1x(const T* __restrict__ f, const Geo& G, int gz, int gy, int gx, T ih) {
    const T* row = f + ((size_t)gz * G.ny + gy) * G.nx;
    return (T(2.0 / 3.0) * (row[wrap(gx + 1, G.nx)] - row[wrap(gx - 1, G.nx)]) -
            T(1.0 / 12.0) * (row[wrap(gx + 2, G.nx)] - row[wrap(gx - 2, G.nx)])) * ih;
}
template <typename T>
__device__ __forceinline__ T d1y(const T* __restrict__ f, const Geo& G, int gz, int gy, int gx, T ih) {
    const T* pl = f + (size_t)gz * G.ny * G.nx + gx;
    return (T(2.0 / 3.0) * (pl[(size_t)wrap(gy + 1, G.ny) * G.nx] - pl[(size_t)wrap(gy - 1, G.ny) * G.nx]) -
            T(1.0 / 12.0) * (pl[(size_t)wrap(gy + 2, G.ny) * G.nx] - pl[(size_t)wrap(gy - 2, G.ny) * G.nx])) * ih;
}
template <typename T>
__device__ __forceinline__ T d1z(const T* __restrict__ f, const Geo& G, int gz, int gy, int gx, int fld, T ih) {
    return (T(2.0 / 3.0) * (pz(f, G, gz + 1, gy, gx, fld) - pz(f, G, gz - 1, gy, gx, fld)) -
            T(1.0 / 12.0) * (pz(f, G, gz + 2, gy, gx, fld) - pz(f, G, gz - 2, gy, gx, fld))) * ih;
}

// sum_j D_j D_j x at (gz, gy, gx), x taken as sc * f (p parity in z)
template <typename T>
__device__ __forceinline__ T lap_dd(const T* __restrict__ f, const Geo& G, int gz, int gy, int gx, T sc, T ix2,
                                    T iy2, T iz2) {
    const T c[5] = {T(-65.0 / 72.0), T(1.0 / 9.0), T(4.0 / 9.0), T(-1.0 / 9.0), T(1.0 / 144.0)};
    const T* row = f + ((size_t)gz * G.ny + gy) * G.nx;
    const T* pl = f + (size_t)gz * G.ny * G.nx + gx;
    const T ctr = row[gx];
    T lx = c[0] * ctr, ly = c[0] * ctr, lz = c[0] * ctr;
#pragma unroll
    for (int k = 1; k <= 4; ++k) {
        lx += c[k] * (row[wrap(gx + k, G.nx)] + row[wrap(gx - k, G.nx)]);
        ly += c[k] * (pl[(size_t)wrap(gy + k, G.ny) * G.nx] + pl[(size_t)wrap(gy - k, G.ny) * G.nx]);
        lz += c[k] * (pz(f, G, gz + k, gy, gx, 4) + pz(f, G, gz - k, gy, gx, 4));
    }
    return sc * (lx * ix2 + ly * iy2 + lz * iz2);
}

template <typename T>
__device__ __forceinline__ void unflat(const Geo& G, int p, int& gz, int& gy, int& gx) {
    const int pxy = G.nx * G.ny;
    gz = p / pxy;
    const int rem = p - gz * pxy;
    gy = rem / G.nx;
    gx = rem - gy * G.nx;
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
schur_rhs3d(Geo G, const T* __restrict__ r, T* __restrict__ rhs, Ctl* ctl, int check_done) {
    if (check_done && ctl->done) return;
    const T cdiv = T(G.schur_cdiv);
    const T ix = T(G.inv_dx), iy = T(G.inv_dy), iz = T(G.inv_dz);
    const size_t np = (size_t)G.npt;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < G.npt; p += gridDim.x * blockDim.x) {
        int gz, gy, gx;
        unflat<T>(G, p, gz, gy, gx);
        const T div = d1x(r, G, gz, gy, gx, ix) + d1y(r + np, G, gz, gy, gx, iy) + d1z(r + 2 * np, G, gz, gy, gx, 2, iz);
        rhs[p] = r[4 * np + p] - cdiv * div;
    }
}

// one Chebyshev sweep k for H x = rhs (FIRST: x_k = rhs / theta_c, d_{k-1} = x_k)
template <typename T, int FIRST, int LAST>
__global__ void __launch_bounds__(NTHREADS)
helm3d(Geo G, int k, const T* __restrict__ rhs, const T* __restrict__ xin, const T* __restrict__ din,
       T* __restrict__ xout, T* __restrict__ dout, Ctl* ctl, int check_done) {
    if (check_done && ctl->done) return;
    const T ith = T(ctl->cheb[5][k][0]);
    const T a1 = T(ctl->cheb[5][k][1]), a2 = T(ctl->cheb[5][k][2]);
    const T ah = T(G.helm_a), tdt = T(G.two_over_dt);
    const T ix2 = T(G.inv_dx * G.inv_dx), iy2 = T(G.inv_dy * G.inv_dy), iz2 = T(G.inv_dz * G.inv_dz);
    const T* src = FIRST ? rhs : xin;
    const T sc = FIRST ? ith : T(1);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < G.npt; p += gridDim.x * blockDim.x) {
        int gz, gy, gx;
        unflat<T>(G, p, gz, gy, gx);
        const T xk = sc * src[p];
        const T rv = rhs[p];
        const T res = rv - (tdt * xk - ah * lap_dd(src, G, gz, gy, gx, sc, ix2, iy2, iz2));
        const T dprev = FIRST ? rv * ith : din[p];
        const T dk = a1 * dprev + a2 * res;
        xout[p] = xk + dk;
        if (!LAST) dout[p] = dk;
    }
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS)
schur_back3d(Geo G, const T* __restrict__ r, T* __restrict__ z, double* part, Ctl* ctl, int check_done) {
    if (check_done && ctl->done) return;
    const T cgrad = T(G.schur_cgrad), hdt = T(G.half_dt);
    const T ith_t = T(ctl->cheb[3][0][0]);
    const T ix = T(G.inv_dx), iy = T(G.inv_dy), iz = T(G.inv_dz);
    const size_t np = (size_t)G.npt;
    const T* dp = z + 4 * np;
    T acc[1] = {T(0)};
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < G.npt; p += gridDim.x * blockDim.x) {
        int gz, gy, gx;
        unflat<T>(G, p, gz, gy, gx);
        const T zu = hdt * (r[p] - cgrad * d1x(dp, G, gz, gy, gx, ix));
        const T zv = hdt * (r[np + p] - cgrad * d1y(dp, G, gz, gy, gx, iy));
        const T zw = hdt * (r[2 * np + p] - cgrad * d1z(dp, G, gz, gy, gx, 4, iz));
        const T zt = r[3 * np + p] * ith_t;
        const T zp = dp[p];
        z[p] = zu;
        z[np + p] = zv;
        z[2 * np + p] = zw;
        z[3 * np + p] = zt;
        acc[0] += zu * zu + zv * zv + zw * zw + zt * zt + zp * zp;
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

static int stream_blocks3(size_t n) {
    size_t b = (n + NTHREADS - 1) / NTHREADS;
    return (int)(b < (size_t)MAX_STREAM_BLOCKS ? (b > 0 ? b : 1) : MAX_STREAM_BLOCKS);
}

}  // namespace d3

// ------------------------------------------------------------------ launchers
int stencil3d_part_blocks(const Geo& G) {
    // largest reduction grid any 3-D kernel launches (Chebyshev: 5 field slices)
    using namespace d3;
    const int a = ((G.nx + 7) / 8) * ((G.ny + 7) / 8) * ((G.nz + 3) / 4);
    const int c = ((G.nx + 15) / 16) * ((G.ny + 7) / 8) * ((G.nz + 3) / 4) * 5;
    return a > c ? a : c;
}

template <typename T, int MODE, int SMAG>
static cudaError_t launch_s3(const Geo& G, const T* u, const T* v, const T* Fu, const double* f, T* out,
                             T* out2, double* part, Ctl* ctl, int check_done, cudaStream_t s) {
    using namespace d3;
    constexpr int TX = FTile<T>::TX, TY = FTile<T>::TY, TZ = FTile<T>::TZ;
    using B = Box<TX, TY, TZ>;
    const size_t sm = sizeof(T) * (5 * B::PL + (SMAG == 2 ? 6 : 5) * B::AS);
    static std::atomic<bool> configured{false};   // set once; concurrent first calls are harmless
    if (!configured) {
        cudaError_t e = set_smem(stencil3d<T, MODE, SMAG, TX, TY, TZ>, sm);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((G.nx + TX - 1) / TX, (G.ny + TY - 1) / TY, (G.nz + TZ - 1) / TZ);
    stencil3d<T, MODE, SMAG, TX, TY, TZ><<<grid, NTHREADS, sm, s>>>(G, u, v, Fu, f, out, out2, part, ctl, check_done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stencil3d(int mode, const Geo& G, const T* u, const T* v, const T* Fu, const double* f,
                             T* out, T* out2, double* part, Ctl* ctl, int check_done, cudaStream_t s) {
#define JF3(M)                                                                                         \
    case M:                                                                                            \
        return G.sgs == 2 ? launch_s3<T, M, 2>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s)   \
             : G.smag     ? launch_s3<T, M, 1>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s)   \
                          : launch_s3<T, M, 0>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
    switch (mode) {
        JF3(d3::MODE_F)
        JF3(d3::MODE_RHS)
        JF3(d3::MODE_RES)
        JF3(d3::MODE_JV)
        JF3(d3::MODE_RHSRES)
        default: return cudaErrorInvalidValue;
    }
#undef JF3
}
template cudaError_t launch_stencil3d<float>(int, const Geo&, const float*, const float*, const float*,
                                             const double*, float*, float*, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_stencil3d<double>(int, const Geo&, const double*, const double*, const double*,
                                              const double*, double*, double*, double*, Ctl*, int, cudaStream_t);

template <typename T, int SMAG>
static cudaError_t launch_jvd3(const Geo& G, const T* u, const T* v, T* out, Ctl* ctl, int check_done,
                               cudaStream_t s) {
    using namespace d3;
    constexpr int TX = DTile<T>::TX, TY = DTile<T>::TY, TZ = DTile<T>::TZ;
    using B = Box<TX, TY, TZ>;
    const size_t sm = sizeof(T) * (10 * B::PL + (SMAG == 2 ? 12 : 10) * B::AS);
    static std::atomic<bool> configured{false};   // set once; concurrent first calls are harmless
    if (!configured) {
        cudaError_t e = set_smem(jv_diff3d<T, SMAG, TX, TY, TZ>, sm);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 grid((G.nx + TX - 1) / TX, (G.ny + TY - 1) / TY, (G.nz + TZ - 1) / TZ);
    jv_diff3d<T, SMAG, TX, TY, TZ><<<grid, NTHREADS, sm, s>>>(G, u, v, out, ctl, check_done);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_jv_diff3d(const Geo& G, const T* u, const T* v, T* out, Ctl* ctl, int check_done,
                             cudaStream_t s) {
    if (G.sgs == 2) return launch_jvd3<T, 2>(G, u, v, out, ctl, check_done, s);
    return G.smag ? launch_jvd3<T, 1>(G, u, v, out, ctl, check_done, s)
                  : launch_jvd3<T, 0>(G, u, v, out, ctl, check_done, s);
}
template cudaError_t launch_jv_diff3d<float>(const Geo&, const float*, const float*, float*, Ctl*, int, cudaStream_t);
template cudaError_t launch_jv_diff3d<double>(const Geo&, const double*, const double*, double*, Ctl*, int, cudaStream_t);

template <typename T>
cudaError_t launch_eddy3d(const Geo& G, const T* u, T* nu, double* part, Ctl* ctl, cudaStream_t s) {
    d3::eddy3d<T><<<d3::stream_blocks3(G.npt), NTHREADS, 0, s>>>(G, u, nu, part, ctl);
    return cudaGetLastError();
}
template cudaError_t launch_eddy3d<float>(const Geo&, const float*, float*, double*, Ctl*, cudaStream_t);
template cudaError_t launch_eddy3d<double>(const Geo&, const double*, double*, double*, Ctl*, cudaStream_t);

template <typename T, int SMAG>
static cudaError_t launch_pc3(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da, T* db,
                              const T* nu, double* part, Ctl* ctl, int check_done, cudaStream_t s,
                              long long* launches) {
    using namespace d3;
    constexpr int TX = CTile<T>::TX, TY = CTile<T>::TY, TZ = CTile<T>::TZ;
    using B = Box<TX, TY, TZ>;
    const size_t sm = sizeof(T) * (B::PL + 2 * B::AS);
    static std::atomic<bool> configured{false};   // set once; concurrent first calls are harmless
    if (!configured) {
        cudaError_t e;
        if ((e = set_smem(cheb3d<T, SMAG, 1, 1, TX, TY, TZ>, sm)) != cudaSuccess) return e;
        if ((e = set_smem(cheb3d<T, SMAG, 1, 0, TX, TY, TZ>, sm)) != cudaSuccess) return e;
        if ((e = set_smem(cheb3d<T, SMAG, 0, 1, TX, TY, TZ>, sm)) != cudaSuccess) return e;
        if ((e = set_smem(cheb3d<T, SMAG, 0, 0, TX, TY, TZ>, sm)) != cudaSuccess) return e;
        configured = true;
    }
    const int ntz = (G.nz + TZ - 1) / TZ;
    dim3 grid((G.nx + TX - 1) / TX, (G.ny + TY - 1) / TY, ntz * 5);
    const T* zin = nullptr;
    const T* din = nullptr;
    T* zbuf[2] = {za, zb};
    T* dbuf[2] = {da, db};
    for (int k = 1; k <= sweeps - 1; ++k) {
        const bool first = k == 1, last = k == sweeps - 1;
        T* zo = last ? z : zbuf[k & 1];
        T* dO = dbuf[k & 1];
        if (first && last)
            cheb3d<T, SMAG, 1, 1, TX, TY, TZ><<<grid, NTHREADS, sm, s>>>(G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        else if (first)
            cheb3d<T, SMAG, 1, 0, TX, TY, TZ><<<grid, NTHREADS, sm, s>>>(G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        else if (last)
            cheb3d<T, SMAG, 0, 1, TX, TY, TZ><<<grid, NTHREADS, sm, s>>>(G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        else
            cheb3d<T, SMAG, 0, 0, TX, TY, TZ><<<grid, NTHREADS, sm, s>>>(G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        if (launches) ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        zin = zo;
        din = dO;
    }
    return cudaSuccess;
}

// Acoustic Schur complement (3-D): rhs in da, iterates in za / zb, directions
// in db and db + npt, the last sweep into the p plane of z, back-substitution.
template <typename T>
static cudaError_t launch_schur3d(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da, T* db,
                                  double* part, Ctl* ctl, int check_done, cudaStream_t s, long long* launches) {
    const size_t np = (size_t)G.npt;
    const int nb = d3::stream_blocks3(np);
    T* rhs = da;
    d3::schur_rhs3d<T><<<nb, NTHREADS, 0, s>>>(G, r, rhs, ctl, check_done);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (launches) ++*launches;
    T* xbuf[2] = {za, zb};
    T* dbuf[2] = {db, db + np};
    const T* xin = nullptr;
    const T* din = nullptr;
    for (int k = 1; k <= sweeps - 1; ++k) {
        const bool first = k == 1, last = k == sweeps - 1;
        T* xo = last ? z + 4 * np : xbuf[k & 1];
        T* dO = dbuf[k & 1];
        if (first && last) d3::helm3d<T, 1, 1><<<nb, NTHREADS, 0, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
        else if (first) d3::helm3d<T, 1, 0><<<nb, NTHREADS, 0, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
        else if (last) d3::helm3d<T, 0, 1><<<nb, NTHREADS, 0, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
        else d3::helm3d<T, 0, 0><<<nb, NTHREADS, 0, s>>>(G, k, rhs, xin, din, xo, dO, ctl, check_done);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (launches) ++*launches;
        xin = xo;
        din = dO;
    }
    d3::schur_back3d<T><<<nb, NTHREADS, 0, s>>>(G, r, z, part, ctl, check_done);
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_precond3d(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da, T* db,
                             const T* nu, double* part, Ctl* ctl, int check_done, cudaStream_t s,
                             long long* launches) {
    if (G.pc_schur) return launch_schur3d<T>(G, sweeps, r, z, za, zb, da, db, part, ctl, check_done, s, launches);
    if (G.sgs == 2) return launch_pc3<T, 2>(G, sweeps, r, z, za, zb, da, db, nu, part, ctl, check_done, s, launches);
    return G.smag ? launch_pc3<T, 1>(G, sweeps, r, z, za, zb, da, db, nu, part, ctl, check_done, s, launches)
                  : launch_pc3<T, 0>(G, sweeps, r, z, za, zb, da, db, nu, part, ctl, check_done, s, launches);
}
template cudaError_t launch_precond3d<float>(const Geo&, int, const float*, float*, float*, float*, float*,
                                             float*, const float*, double*, Ctl*, int, cudaStream_t, long long*);
template cudaError_t launch_precond3d<double>(const Geo&, int, const double*, double*, double*, double*,
                                              double*, double*, const double*, double*, Ctl*, int, cudaStream_t,
                                              long long*);

cudaError_t launch_budgets3d(const Geo& G, const double* u, double dV, double dz, double lz, double* part,
                             Ctl* ctl, double* out, cudaStream_t s) {
    d3::budgets3d<<<d3::stream_blocks3(G.npt), NTHREADS, 0, s>>>(G, u, dV, dz, lz, part, ctl, out);
    return cudaGetLastError();
}

}  // namespace jfnk
