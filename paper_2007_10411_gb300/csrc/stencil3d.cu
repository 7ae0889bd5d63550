// 3-D stencil kernels of libjfnk: F(u), R(u), the Jacobian-vector products,
// the eddy field, the field-block Chebyshev preconditioner, the acoustic
// Schur complement and the budgets, for fields (u, v, w, theta, p) on
// [z][y][x] (x, y periodic; z cell-centred with signed mirror ghosts: w odd,
// theta and p even, u and v even for free slip / odd for no slip; the eddy
// field is mirrored even).
//
// Same discretisation as the 2-D kernels (Deslauriers-Dubuc p = 2 derivative,
// Section 2.3; skew-symmetric convection of every field, Section 2.2;
// Eqs. ch2_28-ch2_30 with Laplacian-form eddy diffusion, Section 2.4), with
// the filter width Delta = (dx dy dz)^(1/3) and the full 3x3 strain.
//
// Every term of F is a sum over the three axes of a one-dimensional stencil
// once the eddy coefficient is known at each point (convection flux and
// advective form along j, D_j(K D_j phi), the pressure gradient and the
// divergence of the pressure equation), plus point-wise terms.  The operator
// is therefore evaluated in three passes that each stage only what their axis
// needs:
//   strain  |S| (and, for the difference-form Jacobian product, |S(a+b)| - |S(a)|
//           without cancellation) at every point: a plane tile with a halo of
//           r = 2 in x, y in shared memory, z neighbours read directly;
//   plane   the x and y terms and the point-wise ones for a TX x TY tile of one
//           plane: the fields with a halo of 2r = 4 in x and y, the first
//           derivatives on the x / y arms (tile + r) computed once, the eddy
//           coefficients on the arms from the strain pass; writes the partial sum;
//   slab    the z terms for a TX x TZ slab of one y row: the fields with a halo
//           of 4 in z (mirror ghosts), z derivatives on the z arms, then the
//           partial sum of the plane pass is added and the mode's output
//           (F, 2u/dt + F, the residual with its norms, or the Jacobian product)
//           written.
// Loads are coalesced along x in every pass; the halos are re-read from L2.
//
// Difference form (float32 Jacobian product): with a = u and b = eps v every
// term of F(a + b) - F(a) is written as a difference (products a_j b_phi +
// b_j (a_phi + b_phi), K(a) D b + (K(a + b) - K(a)) D(a + b)), so no O(1)
// quantity is cancelled in float32.  The other modes evaluate F(b) with
// a = 0 (b = u, or b = u + eps v for the plain forward difference), for
// which the same formulas reduce to F term by term.
#include <math.h>

#include <atomic>

#include "common.cuh"
#include "kernels.h"

namespace jfnk {
namespace d3 {

constexpr int R = 2;
constexpr int HALO = 2 * R;
constexpr int MODE_F = 0, MODE_RHS = 1, MODE_RES = 2, MODE_JV = 3, MODE_RHSRES = 4, MODE_DJV = 5;

template <int MODE>
struct Two { static constexpr bool v = MODE == MODE_DJV; };   // two states a, b (else a = 0)

template <typename T>
__device__ __forceinline__ T dd(const T* s, int i, int st, T ih) {
    return (T(2.0 / 3.0) * (s[i + st] - s[i - st]) - T(1.0 / 12.0) * (s[i + 2 * st] - s[i - 2 * st])) * ih;
}
// D f from the four neighbours f(-2), f(-1), f(+1), f(+2)
template <typename T>
__device__ __forceinline__ T d5(T m2, T m1, T p1, T p2, T ih) {
    return (T(2.0 / 3.0) * (p1 - m1) - T(1.0 / 12.0) * (p2 - m2)) * ih;
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
// even mirror of a row of the eddy field (-1: beyond one reflection, never read)
__device__ __forceinline__ int eddy_row(int gz, int nz) {
    if (gz >= 0 && gz < nz) return gz;
    if (gz < 0) return -1 - gz < nz ? -1 - gz : -1;
    return 2 * nz - 1 - gz >= 0 ? 2 * nz - 1 - gz : -1;
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

// Coefficient pair (K(a), K(a + b) - K(a)) of one field at an arm point from
// na = |S(a)| and ds = |S(a + b)| - |S(a)| (na = 0: the coefficient K(b) of
// the one-state modes in the second slot).  SMAG 1: Smagorinsky (the caller
// applies 1/Pr for theta); SMAG 2: Deardorff, the arm's direction and the
// field (momentum / heat) picking the coefficient.
template <typename T, int SMAG>
__device__ __forceinline__ void kpair(const Geo& G, T na, T ds, bool zarm, bool heat, T& k, T& dk) {
    if (SMAG == 1) {
        const T c = T(G.cs2);
        k = c * na;
        dk = c * ds;
        return;
    }
    const T c = T(zarm ? G.dd_cM : G.dd_cm);
    if (!heat) {
        k = c * na;
        dk = c * ds;
        return;
    }
    // heat: g(s) = c s (1 + a l(s)); g(s') - g(s) = ds (1 + a l') + a s (l' - l),
    // l' - l = c_l ds while both are below the cap
    const T a = T(zarm ? G.dd_az : G.dd_ah);
    const T dl_cap = T(G.dd_delta);
    T la = dl_cap, lp = dl_cap, dl = T(0);
    if (G.dd_cl >= 0.0) {
        const T ta = T(G.dd_cl) * na, tq = T(G.dd_cl) * (na + ds);
        la = ta < dl_cap ? ta : dl_cap;
        lp = tq < dl_cap ? tq : dl_cap;
        if (ta < dl_cap && tq < dl_cap) dl = T(G.dd_cl) * ds;
        else if (ta < dl_cap || tq < dl_cap) dl = lp - la;
    }
    k = c * (na * (T(1) + a * la));
    dk = c * (ds * (T(1) + a * lp) + a * na * dl);
}

// The two states of field f at flat index o: DJV a = u, b = eps_f v;
// JV a = 0, b = u + eps_f v; other modes a = 0, b = u.
template <typename T, int MODE>
__device__ __forceinline__ void load_ab(const T* __restrict__ u, const T* __restrict__ v, T ev, size_t o, T& a,
                                        T& b) {
    if constexpr (MODE == MODE_DJV) {
        a = u[o];
        b = ev * v[o];
    } else if constexpr (MODE == MODE_JV) {
        a = T(0);
        b = u[o] + ev * v[o];
    } else {
        a = T(0);
        b = u[o];
    }
}

// eps_f = eps_jv * scale_f (Jacobian-product modes)
template <typename T>
__device__ __forceinline__ T eps_field(const Ctl* ctl, const Geo& G, int f) {
    return T(ctl->eps_jv * G.scale[f]);
}

// ------------------------------------------------------------------ tiles
constexpr int PX = 32, PY = 8;                 // plane tile (one output per thread)
constexpr int KX = 32, KY = 8;                 // strain tile
template <typename T> struct SlabT;            // slab tile TX x TZ
template <> struct SlabT<float>  { static constexpr int TX = 32, TZ = 16; };
template <> struct SlabT<double> { static constexpr int TX = 32, TZ = 8; };
static_assert(PX * PY == NTHREADS && KX * KY == NTHREADS, "one output per thread");

// ============================================================================
// Strain pass: s = sqrt(2 S:S) of b (one-state modes) or, for the difference
// form, sa = |S(a)| and ds = |S(a + b)| - |S(a)| = (S':S' - S:S) * 2 / (s + s')
// at every point.  EDDY: the eddy field of u instead (nu = cs2 s, Deardorff:
// s itself), with its maximum.  One CTA marches up a KX x KY column of SZB
// planes: each thread keeps its point's velocity components at z-2 .. z+2 in
// registers (one new plane per step); the plane itself is staged with a halo
// of r = 2 in x and y for the horizontal derivatives.
// ============================================================================
constexpr int SZB = 16;      // planes per CTA of the strain pass

template <typename T, int MODE, int EDDY>
__global__ void __launch_bounds__(NTHREADS)
strain3d(Geo G, const T* __restrict__ u, const T* __restrict__ v, T* __restrict__ s0, T* __restrict__ s1,
         double* part, Ctl* ctl, int check_done) {
    constexpr bool TWO = Two<MODE>::v;
    constexpr int SX = KX + 2 * R, SY = KY + 2 * R, SP = SX * SY;
    constexpr int NA = TWO ? 6 : 3;               // (b u, b v, b w) [, (a u, a v, a w)]
    constexpr int XS = (SP + NTHREADS - 1) / NTHREADS;
    if ((MODE == MODE_JV || MODE == MODE_DJV) && check_done && ctl->done) return;
    __shared__ T st[NA][SP];
    const int x0 = blockIdx.x * KX, y0 = blockIdx.y * KY;
    const int z0 = blockIdx.z * SZB, z1 = min(z0 + SZB, G.nz);
    const T ix = T(G.inv_dx), iy = T(G.inv_dy), iz = T(G.inv_dz);
    T ev[3] = {T(0), T(0), T(0)};
    if (MODE == MODE_JV || MODE == MODE_DJV) {
#pragma unroll
        for (int f = 0; f < 3; ++f) ev[f] = eps_field<T>(ctl, G, f);
    }
    const size_t nxy = (size_t)G.ny * G.nx;
    int xoff[XS];
#pragma unroll
    for (int q = 0; q < XS; ++q) {
        const int idx = threadIdx.x + q * NTHREADS;
        xoff[q] = idx < SP ? wrap(y0 + idx / SX - R, G.ny) * G.nx + wrap(x0 + idx % SX - R, G.nx) : -1;
    }
    const int tx = threadIdx.x % KX, ty = threadIdx.x / KX;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool inside = gx < G.nx && gy < G.ny;
    const size_t own = inside ? (size_t)gy * G.nx + gx : 0;
    // the column's components at z-2 .. z+2 (mirror ghosts with each component's parity)
    T wb[3][5], wa[3][5];
    auto col = [&](int z, int f, T& a, T& b) {
        int side;
        const int sz = mirror(z, G.nz, side);
        load_ab<T, MODE>(u, v, ev[f], (size_t)f * G.npt + (size_t)sz * nxy + own, a, b);
        const T sg = side == 1 ? T(G.pb[f]) : (side == 2 ? T(G.pt[f]) : T(1));
        a *= sg;
        b *= sg;
    };
    if (inside) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int f = 0; f < 3; ++f) col(z0 - 2 + q, f, wa[f][q], wb[f][q]);
    }
    T mx = T(0);
    for (int z = z0; z < z1; ++z) {
        const size_t pz = (size_t)z * nxy;
#pragma unroll
        for (int q = 0; q < XS; ++q) {
            if (xoff[q] < 0) continue;
            const size_t o = pz + xoff[q];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                T a, b;
                load_ab<T, MODE>(u, v, ev[f], (size_t)f * G.npt + o, a, b);
                st[f][threadIdx.x + q * NTHREADS] = b;
                if (TWO) st[3 + f][threadIdx.x + q * NTHREADS] = a;
            }
        }
        __syncthreads();
        if (inside) {
#pragma unroll
            for (int f = 0; f < 3; ++f) col(z + 2, f, wa[f][4], wb[f][4]);
            const int c = (ty + R) * SX + tx + R;
            T gB[3][3], gA[3][3];
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                gB[f][0] = dd(st[f], c, 1, ix);
                gB[f][1] = dd(st[f], c, SX, iy);
                gB[f][2] = d5(wb[f][0], wb[f][1], wb[f][3], wb[f][4], iz);
                if (TWO) {
                    gA[f][0] = dd(st[3 + f], c, 1, ix);
                    gA[f][1] = dd(st[3 + f], c, SX, iy);
                    gA[f][2] = d5(wa[f][0], wa[f][1], wa[f][3], wa[f][4], iz);
                }
            }
            const size_t p = pz + own;
            if (TWO) {
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
                s0[p] = na;
                s1[p] = den > T(0) ? T(2) * dss / den : T(0);
            } else {
                T ss = T(0);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const T sB = T(0.5) * (gB[i][j] + gB[j][i]);
                        ss += sB * sB;
                    }
                const T sv = sqrt(T(2) * ss);
                if (EDDY) {
                    const T val = (G.sgs == 2 ? T(1) : T(G.cs2)) * sv;
                    s1[p] = val;
                    mx = val > mx ? val : mx;
                } else {
                    s1[p] = sv;
                }
            }
#pragma unroll
            for (int f = 0; f < 3; ++f)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    wb[f][q] = wb[f][q + 1];
                    wa[f][q] = wa[f][q + 1];
                }
        }
        __syncthreads();      // the next plane overwrites the staged one
    }
    if (EDDY) {
        double m1[1] = {(double)mx};
        const int nblk = gridDim.x * gridDim.y * gridDim.z;
        const int blk = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        block_partials_max<1>(m1, 1, part, nblk, blk);
        if (arrive_last(&ctl->counter[CNT_EDDY], nblk)) {
            __shared__ double tot[1];
            final_maxes(part, nblk, 1, tot);
            if (threadIdx.x == 0) ctl->kmax = tot[0];
        }
    }
}

// ============================================================================
// Plane pass: x and y terms of every field and the point-wise terms, for a
// PX x PY tile of plane z = blockIdx.z; writes their sum to P.
// ============================================================================
template <typename T, int MODE, int SMAG>
__global__ void __launch_bounds__(NTHREADS)
plane3d(Geo G, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ s0,
        const T* __restrict__ s1, T* __restrict__ P, Ctl* ctl, int check_done) {
    constexpr bool TWO = Two<MODE>::v;
    constexpr int SX = PX + 2 * HALO, SY = PY + 2 * HALO, SP = SX * SY;
    constexpr int AXN = (PX + 2 * R) * PY, AYN = PX * (PY + 2 * R), AN = AXN + AYN;   // x arms, y arms
    constexpr int NS = TWO ? 2 : 1;                  // states staged (b [, a])
    if ((MODE == MODE_JV || MODE == MODE_DJV) && check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* st = reinterpret_cast<T*>(smem_raw);          // [NS][5][SP]: b fields, then a fields
    T* ga = st + NS * 5 * SP;                        // [NS][4][AN] first derivatives on the arms
    T* ks = ga + NS * 4 * AN;                        // [NS][AN] strain on the arms (SMAG)
    const int x0 = blockIdx.x * PX, y0 = blockIdx.y * PY, gz = blockIdx.z;
    const T ix = T(G.inv_dx), iy = T(G.inv_dy);
    T ev[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (MODE == MODE_JV || MODE == MODE_DJV) {
#pragma unroll
        for (int f = 0; f < 5; ++f) ev[f] = eps_field<T>(ctl, G, f);
    }
    const size_t plane = (size_t)gz * G.ny * G.nx;
    for (int idx = threadIdx.x; idx < SP; idx += NTHREADS) {
        const int ixl = idx % SX, iyl = idx / SX;
        const size_t o = plane + (size_t)wrap(y0 + iyl - HALO, G.ny) * G.nx + wrap(x0 + ixl - HALO, G.nx);
#pragma unroll
        for (int f = 0; f < 5; ++f) {
            T a, b;
            load_ab<T, MODE>(u, v, ev[f], (size_t)f * G.npt + o, a, b);
            st[f * SP + idx] = b;
            if (TWO) st[(5 + f) * SP + idx] = a;
        }
    }
    if (SMAG) {
        for (int idx = threadIdx.x; idx < AN; idx += NTHREADS) {
            int qx, qy;
            if (idx < AXN) { qx = idx % (PX + 2 * R) - R; qy = idx / (PX + 2 * R); }
            else { const int j = idx - AXN; qx = j % PX; qy = j / PX - R; }
            const size_t o = plane + (size_t)wrap(y0 + qy, G.ny) * G.nx + wrap(x0 + qx, G.nx);
            ks[idx] = s1[o];
            if (TWO) ks[AN + idx] = s0[o];
        }
    }
    __syncthreads();
    // first derivatives of u, v, w, theta (each state) on the arms
    for (int idx = threadIdx.x; idx < AN; idx += NTHREADS) {
        int c, stp;
        T ih;
        if (idx < AXN) {
            const int qx = idx % (PX + 2 * R), qy = idx / (PX + 2 * R);
            c = (qy + HALO) * SX + qx + R;
            stp = 1;
            ih = ix;
        } else {
            const int j = idx - AXN;
            const int qx = j % PX, qy = j / PX;
            c = (qy + R) * SX + qx + HALO;
            stp = SX;
            ih = iy;
        }
#pragma unroll
        for (int q = 0; q < NS * 4; ++q) {
            const int arr = q < 4 ? q : 5 + (q - 4);          // b: fields 0..3, a: fields 0..3
            ga[q * AN + idx] = dd(st + arr * SP, c, stp, ih);
        }
    }
    __syncthreads();
    const int tx = threadIdx.x % PX, ty = threadIdx.x / PX;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx >= G.nx || gy >= G.ny) return;
    const int c = (ty + HALO) * SX + tx + HALO;
    const int cax = ty * (PX + 2 * R) + tx + R;               // x arm at the output point
    const int cay = AXN + (ty + R) * PX + tx;                 // y arm at the output point
    const int astr[2] = {1, PX};
    const int carm[2] = {cax, cay};
    const int sst[2] = {1, SX};
    const T ihs[2] = {ix, iy};
    const T* Bf = st;                                         // b fields
    const T* Af = st + 5 * SP;                                // a fields (TWO)
    T dF[5];
    T dbp[2], dap[2];                                         // D_j of p (b, a) at the point
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        dbp[j] = dd(Bf + 4 * SP, c, sst[j], ihs[j]);
        dap[j] = TWO ? dd(Af + 4 * SP, c, sst[j], ihs[j]) : T(0);
    }
#pragma unroll
    for (int fl = 0; fl < 5; ++fl) {
        const T* B = Bf + fl * SP;
        const T* A = Af + fl * SP;
        T flux = T(0), adv = T(0);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const T* bj = Bf + j * SP;                        // b_u (x) or b_v (y)
            const T* aj = Af + j * SP;
            const int s = sst[j];
            T fj = T(0);
#pragma unroll
            for (int l = 1; l <= 2; ++l) {
                const T cl = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
                const int ip = c + l * s, im = c - l * s;
                if (TWO)
                    fj += cl * ((aj[ip] * B[ip] + bj[ip] * (A[ip] + B[ip])) - (aj[im] * B[im] + bj[im] * (A[im] + B[im])));
                else
                    fj += cl * (bj[ip] * B[ip] - bj[im] * B[im]);
            }
            flux += fj * ihs[j];
            T daj, dbj;
            if (fl < 4) {
                dbj = ga[fl * AN + carm[j]];
                daj = TWO ? ga[(4 + fl) * AN + carm[j]] : T(0);
            } else {
                dbj = dbp[j];
                daj = dap[j];
            }
            adv += TWO ? (aj[c] * dbj + bj[c] * (daj + dbj)) : bj[c] * dbj;
        }
        dF[fl] = -(T(0.5) * flux + T(0.5) * adv);
        if (fl < 4) {
            const T* gb = ga + fl * AN;
            const T* gA = ga + (4 + fl) * AN;
            T dif = T(0);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int q = carm[j], s = astr[j];
                T sj = T(0);
#pragma unroll
                for (int l = 1; l <= 2; ++l) {
                    const T cl = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
                    const int p1 = q + l * s, m1 = q - l * s;
                    if (SMAG) {
                        T kp, dkp, km, dkm;
                        kpair<T, SMAG>(G, TWO ? ks[AN + p1] : T(0), ks[p1], false, fl == 3, kp, dkp);
                        kpair<T, SMAG>(G, TWO ? ks[AN + m1] : T(0), ks[m1], false, fl == 3, km, dkm);
                        if (TWO)
                            sj += cl * ((kp * gb[p1] + dkp * (gA[p1] + gb[p1])) - (km * gb[m1] + dkm * (gA[m1] + gb[m1])));
                        else
                            sj += cl * (dkp * gb[p1] - dkm * gb[m1]);
                    } else {
                        sj += cl * (gb[p1] - gb[m1]);
                    }
                }
                dif += sj * ihs[j];
            }
            if (SMAG == 1) {
                if (fl == 3) dif *= T(G.inv_Pr);
            } else if (!SMAG) {
                dif *= T(fl == 3 ? G.K_H : G.K_M);
            }
            dF[fl] += dif;
        }
    }
    const T th0 = T(G.theta0);
    dF[0] += -th0 * dbp[0];
    dF[1] += -th0 * dbp[1];
    dF[2] += T(G.g) * Bf[3 * SP + c] / th0;
    dF[3] += -T(G.beta) * Bf[2 * SP + c];
    if (MODE != MODE_DJV && G.heat != nullptr && gz == 0)
        dF[3] += T(G.heat[(size_t)gy * G.nx + gx] * G.heat_coef);
    {   // pressure equation, x and y parts of the divergence
        const T divb = ga[cax] + ga[AN + cay];
        const T pa = TWO ? Af[4 * SP + c] : T(0), pb = Bf[4 * SP + c];
        T t = (T(G.pbar) + pa + pb) * divb;
        if (TWO) t += pb * (ga[4 * AN + cax] + ga[5 * AN + cay]);
        dF[4] += -T(G.gamma_p) * t;
    }
    const size_t off = plane + (size_t)gy * G.nx + gx;
#pragma unroll
    for (int fl = 0; fl < 5; ++fl) P[(size_t)fl * G.npt + off] = dF[fl];
}

// ============================================================================
// Slab pass: z terms for a TX x TZ slab of row y = blockIdx.z (z tiles along
// blockIdx.x so that consecutive CTAs share their z halos in L2), plus the
// plane pass's sum; writes the mode's output.
// ============================================================================
template <typename T, int MODE, int SMAG>
__global__ void __launch_bounds__(NTHREADS)
slab3d(Geo G, const T* __restrict__ u, const T* __restrict__ v, const T* __restrict__ Fu,
       const double* __restrict__ f, const T* __restrict__ s0, const T* __restrict__ s1,
       const T* __restrict__ P, T* __restrict__ out, T* __restrict__ out2, double* __restrict__ part, Ctl* ctl,
       int check_done) {
    constexpr bool TWO = Two<MODE>::v;
    constexpr int TX = SlabT<T>::TX, TZ = SlabT<T>::TZ;
    constexpr int SZ = TZ + 2 * HALO, SP = TX * SZ;          // staged rows [row][x]
    constexpr int QZ = TZ + 2 * R, AN = TX * QZ;             // z arms
    constexpr int NS = TWO ? 2 : 1;
    constexpr int PER = TX * TZ / NTHREADS;                  // outputs per thread
    if ((MODE == MODE_JV || MODE == MODE_DJV) && check_done && ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* st = reinterpret_cast<T*>(smem_raw);                  // [NS][5][SP]
    T* ga = st + NS * 5 * SP;                                // [NS][4][AN]
    T* ks = ga + NS * 4 * AN;                                // [NS][AN] strain on the z arms (SMAG)
    const int z0 = blockIdx.x * TZ, x0 = blockIdx.y * TX, gy = blockIdx.z;
    const T iz = T(G.inv_dz);
    T ev[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (MODE == MODE_JV || MODE == MODE_DJV) {
#pragma unroll
        for (int q = 0; q < 5; ++q) ev[q] = eps_field<T>(ctl, G, q);
    }
    const size_t row = (size_t)gy * G.nx;
    for (int idx = threadIdx.x; idx < SP; idx += NTHREADS) {
        const int xl = idx % TX, rl = idx / TX;
        int side;
        const int sz = mirror(z0 + rl - HALO, G.nz, side);
        const bool ok = sz >= 0 && sz < G.nz;
        const size_t o = (size_t)sz * G.ny * G.nx + row + wrap(x0 + xl, G.nx);
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            T a = T(0), b = T(0);
            if (ok) {
                load_ab<T, MODE>(u, v, ev[q], (size_t)q * G.npt + o, a, b);
                const T sg = side == 1 ? T(G.pb[q]) : (side == 2 ? T(G.pt[q]) : T(1));
                a *= sg;
                b *= sg;
            }
            st[q * SP + idx] = b;
            if (TWO) st[(5 + q) * SP + idx] = a;
        }
    }
    if (SMAG) {
        for (int idx = threadIdx.x; idx < AN; idx += NTHREADS) {
            const int xl = idx % TX, ql = idx / TX;
            const int sz = eddy_row(z0 + ql - R, G.nz);
            T kv1 = T(0), kv0 = T(0);
            if (sz >= 0) {
                const size_t o = (size_t)sz * G.ny * G.nx + row + wrap(x0 + xl, G.nx);
                kv1 = s1[o];
                if (TWO) kv0 = s0[o];
            }
            ks[idx] = kv1;
            if (TWO) ks[AN + idx] = kv0;
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < AN; idx += NTHREADS) {
        const int xl = idx % TX, ql = idx / TX;
        const int c = (ql + R) * TX + xl;
#pragma unroll
        for (int q = 0; q < NS * 4; ++q) {
            const int arr = q < 4 ? q : 5 + (q - 4);
            ga[q * AN + idx] = dd(st + arr * SP, c, TX, iz);
        }
    }
    __syncthreads();
    const T th0 = T(G.theta0);
    double acc[2] = {0.0, 0.0};
    const T* Bf = st;
    const T* Af = st + 5 * SP;
    double cf[5] = {0.0, 0.0, 0.0, 0.0, 0.0};          // 1 / eps_f of the Jacobian-product modes
    if (MODE == MODE_JV || MODE == MODE_DJV) {
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const double e = ctl->eps_jv * G.scale[q];
            cf[q] = e != 0.0 ? 1.0 / e : 0.0;
        }
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int idx = threadIdx.x + k * NTHREADS;
        const int xl = idx % TX, zl = idx / TX;
        const int gx = x0 + xl, gz = z0 + zl;
        if (gx >= G.nx || gz >= G.nz) continue;
        const int c = (zl + HALO) * TX + xl;
        const int ca = (zl + R) * TX + xl;                 // z arm at the output point
        const T* bw = Bf + 2 * SP;
        const T* aw = Af + 2 * SP;
        const T dbpz = dd(Bf + 4 * SP, c, TX, iz);
        const T dapz = TWO ? dd(Af + 4 * SP, c, TX, iz) : T(0);
        T dF[5];
#pragma unroll
        for (int fl = 0; fl < 5; ++fl) {
            const T* B = Bf + fl * SP;
            const T* A = Af + fl * SP;
            T fj = T(0);
#pragma unroll
            for (int l = 1; l <= 2; ++l) {
                const T cl = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
                const int ip = c + l * TX, im = c - l * TX;
                if (TWO)
                    fj += cl * ((aw[ip] * B[ip] + bw[ip] * (A[ip] + B[ip])) - (aw[im] * B[im] + bw[im] * (A[im] + B[im])));
                else
                    fj += cl * (bw[ip] * B[ip] - bw[im] * B[im]);
            }
            const T flux = fj * iz;
            T daz, dbz;
            if (fl < 4) {
                dbz = ga[fl * AN + ca];
                daz = TWO ? ga[(4 + fl) * AN + ca] : T(0);
            } else {
                dbz = dbpz;
                daz = dapz;
            }
            const T adv = TWO ? (aw[c] * dbz + bw[c] * (daz + dbz)) : bw[c] * dbz;
            dF[fl] = -(T(0.5) * flux + T(0.5) * adv);
            if (fl < 4) {
                const T* gb = ga + fl * AN;
                const T* gA = ga + (4 + fl) * AN;
                T sj = T(0);
#pragma unroll
                for (int l = 1; l <= 2; ++l) {
                    const T cl = l == 1 ? T(2.0 / 3.0) : T(-1.0 / 12.0);
                    const int p1 = ca + l * TX, m1 = ca - l * TX;
                    if (SMAG) {
                        T kp, dkp, km, dkm;
                        kpair<T, SMAG>(G, TWO ? ks[AN + p1] : T(0), ks[p1], true, fl == 3, kp, dkp);
                        kpair<T, SMAG>(G, TWO ? ks[AN + m1] : T(0), ks[m1], true, fl == 3, km, dkm);
                        if (TWO)
                            sj += cl * ((kp * gb[p1] + dkp * (gA[p1] + gb[p1])) - (km * gb[m1] + dkm * (gA[m1] + gb[m1])));
                        else
                            sj += cl * (dkp * gb[p1] - dkm * gb[m1]);
                    } else {
                        sj += cl * (gb[p1] - gb[m1]);
                    }
                }
                T dif = sj * iz;
                if (SMAG == 1) {
                    if (fl == 3) dif *= T(G.inv_Pr);
                } else if (!SMAG) {
                    dif *= T(fl == 3 ? G.K_H : G.K_M);
                }
                dF[fl] += dif;
            }
        }
        dF[2] += -th0 * dbpz;
        {
            const T pa = TWO ? Af[4 * SP + c] : T(0), pb = Bf[4 * SP + c];
            T t = (T(G.pbar) + pa + pb) * ga[2 * AN + ca];
            if (TWO) t += pb * ga[6 * AN + ca];
            dF[4] += -T(G.gamma_p) * t;
        }
        const size_t off = (size_t)gz * G.ny * G.nx + row + gx;
#pragma unroll
        for (int fl = 0; fl < 5; ++fl) {
            const size_t o = (size_t)fl * G.npt + off;
            const T Fv = P[o] + dF[fl];
            if (MODE == MODE_DJV) {
                out[o] = T(G.two_over_dt) * v[o] - Fv * T(cf[fl]);
            } else if (MODE == MODE_F) {
                out[o] = Fv;
            } else if (MODE == MODE_RHS) {
                out[o] = T(G.two_over_dt * (double)u[o] + (double)Fv);
            } else if (MODE == MODE_RHSRES) {
                // at u = u^n the residual 2u/dt - F(u) - f with f = 2u/dt + F(u) is -2 F(u)
                const double uo = (double)u[o];
                const double Fd = (double)Fv;
                out[o] = T(G.two_over_dt * uo + Fd);
                const double Rv = -2.0 * Fd;
                out2[o] = T(Rv);
                const double rs = Rv * G.inv_scale[fl], us = uo * G.inv_scale[fl];
                acc[0] += rs * rs;
                acc[1] += us * us;
            } else if (MODE == MODE_RES) {
                const double uo = (double)u[o];
                const double Rv = G.two_over_dt * uo - (double)Fv - f[o];
                out[o] = T(Rv);
                if (out2 != nullptr) out2[o] = Fv;
                const double rs = Rv * G.inv_scale[fl], us = uo * G.inv_scale[fl];
                acc[0] += rs * rs;
                acc[1] += us * us;
            } else {   // MODE_JV: plain forward difference against F(u)
                const double diff = (double)Fv - (double)Fu[o];
                out[o] = T(G.two_over_dt * (double)v[o] - diff * cf[fl]);
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
// Field-block Chebyshev sweep (same recurrence as the 2-D kernel, Section 2.5.2).
// One CTA = one field of a PX x PY column of ZB planes: blockIdx.z = zblock * 5
// + field.  The CTA marches up its planes; each thread owns one (x, y) column
// and keeps, in registers, the iterate at z-4 .. z+4 and the vertical fluxes
// K D_z x at z-2 .. z+2 (each computed once, when its plane enters the
// window).  Per plane the iterate is staged with a halo of 4 in x and y and
// the eddy field with a halo of 2; the horizontal fluxes K D_x x, K D_y x are
// formed once per arm point in shared memory.  The staging offsets are
// computed once per CTA.  p (field 4) is written by the last sweep.
// ============================================================================
constexpr int CZB = 16;      // planes per CTA of the Chebyshev sweep

template <typename T, int SMAG, int FIRST, int LAST>
__global__ void __launch_bounds__(NTHREADS)
cheb3d(Geo G, int k, const T* __restrict__ r, const T* __restrict__ zin, const T* __restrict__ din,
       T* __restrict__ zout, T* __restrict__ dout, const T* __restrict__ nu, double* part, Ctl* ctl,
       int check_done) {
    constexpr int SX = PX + 2 * HALO, SY = PY + 2 * HALO, SP = SX * SY;      // iterate plane
    constexpr int NX = PX + 2 * R, NY = PY + 2 * R, NP = NX * NY;            // eddy plane
    constexpr int AXN = (PX + 2 * R) * PY, AYN = PX * (PY + 2 * R), AN = AXN + AYN;
    constexpr int XS = (SP + NTHREADS - 1) / NTHREADS;    // staging slots per thread
    constexpr int NS = (NP + NTHREADS - 1) / NTHREADS;
    constexpr int AS = (AN + NTHREADS - 1) / NTHREADS;
    if (check_done && ctl->done) return;
    __shared__ T xs[SP];
    __shared__ T ns[SMAG ? NP : 1];
    __shared__ T kg[AN];       // K D_x x on the x arms, K D_y x on the y arms (D only when K is constant)
    const int fld = blockIdx.z % 5;
    const int z0 = (blockIdx.z / 5) * CZB;
    const int z1 = min(z0 + CZB, G.nz);
    const int x0 = blockIdx.x * PX, y0 = blockIdx.y * PY;
    const T ith = T(ctl->cheb[fld][k][0]);
    const T a1 = T(ctl->cheb[fld][k][1]);
    const T a2 = T(ctl->cheb[fld][k][2]);
    const size_t nxy = (size_t)G.ny * G.nx;
    const T* fr = r + (size_t)fld * G.npt;
    const T* fsrc = (FIRST ? r : zin) + (size_t)fld * G.npt;
    const T* fdin = FIRST ? nullptr : din + (size_t)fld * G.npt;
    T* fzo = zout + (size_t)fld * G.npt;
    T* fdo = dout + (size_t)fld * G.npt;
    const T sc = FIRST ? ith : T(1);
    const int tx = threadIdx.x % PX, ty = threadIdx.x / PX;
    const int gx = x0 + tx, gy = y0 + ty;
    const bool inside = gx < G.nx && gy < G.ny;
    const size_t own = inside ? (size_t)gy * G.nx + gx : 0;       // in-plane offset of the thread's column
    T acc[1] = {T(0)};
    if (fld == 4) {
        if (LAST && inside) {
            for (int z = z0; z < z1; ++z) {
                const size_t o = (size_t)z * nxy + own;
                const T zv = fr[o] * ith;
                fzo[o] = zv;
                acc[0] += zv * zv;
            }
        }
    } else {
        // in-plane offsets of this thread's staging slots (-1: unused slot)
        int xoff[XS], noff[NS], acen[AS], anu[AS];
#pragma unroll
        for (int q = 0; q < XS; ++q) {
            const int idx = threadIdx.x + q * NTHREADS;
            xoff[q] = idx < SP ? wrap(y0 + idx / SX - HALO, G.ny) * G.nx + wrap(x0 + idx % SX - HALO, G.nx) : -1;
        }
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int idx = threadIdx.x + q * NTHREADS;
            noff[q] = (SMAG && idx < NP) ? wrap(y0 + idx / NX - R, G.ny) * G.nx + wrap(x0 + idx % NX - R, G.nx) : -1;
        }
#pragma unroll
        for (int q = 0; q < AS; ++q) {
            const int idx = threadIdx.x + q * NTHREADS;
            if (idx < AXN) {
                const int qx = idx % NX, qy = idx / NX;          // x arm at tile (qx - R, qy)
                acen[q] = (qy + HALO) * SX + qx + R;
                anu[q] = (qy + R) * NX + qx;
            } else if (idx < AN) {
                const int j = idx - AXN;
                const int qx = j % PX, qy = j / PX;               // y arm at tile (qx, qy - R)
                acen[q] = -((qy + R) * SX + qx + HALO) - 1;       // negative: a y arm
                anu[q] = qy * NX + qx + R;
            } else {
                acen[q] = 0;
                anu[q] = -1;
            }
        }
        const T kscale = fld == 3 ? T(G.inv_Pr) : T(1);
        const T ix = T(G.inv_dx), iy = T(G.inv_dy), iz = T(G.inv_dz);
        const T Kc = T(fld == 3 ? G.K_H : G.K_M);
        auto xval = [&](int z) -> T {          // iterate at row z of the column (mirror ghosts)
            int side;
            const int sz = mirror(z, G.nz, side);
            const T sg = side == 1 ? T(G.pb[fld]) : (side == 2 ? T(G.pt[fld]) : T(1));
            return sg * sc * fsrc[(size_t)sz * nxy + own];
        };
        auto zflux = [&](T d, int z) -> T {    // K D_z x at row z (eddy field mirrored even)
            if (!SMAG) return d;
            const int sz = eddy_row(z, G.nz);
            const T nv = sz >= 0 ? nu[(size_t)sz * nxy + own] : T(0);
            return (SMAG == 2 ? dd3_coef(nv, true, fld == 3, G) : nv * kscale) * d;
        };
        T xw[9], fw[5];
        if (inside) {
#pragma unroll
            for (int q = 0; q < 8; ++q) xw[q] = xval(z0 - 4 + q);
#pragma unroll
            for (int q = 0; q < 4; ++q) fw[q] = zflux(d5(xw[q], xw[q + 1], xw[q + 3], xw[q + 4], iz), z0 - 2 + q);
        }
        // every global value a plane needs (its staged tile and eddy plane, the
        // point's r, d, the iterate at z+4 and the eddy field at z+2) is loaded one
        // plane ahead into registers, so that the latency overlaps the previous
        // plane's arithmetic
        T px[XS], pn[NS];
        T pr = T(0), pd = T(0), px4 = T(0), pnu2 = T(0);
        auto prefetch = [&](int z) {
            const size_t pz = (size_t)z * nxy;
#pragma unroll
            for (int q = 0; q < XS; ++q) px[q] = xoff[q] >= 0 ? fsrc[pz + xoff[q]] : T(0);
#pragma unroll
            for (int q = 0; q < NS; ++q) pn[q] = (SMAG && noff[q] >= 0) ? nu[pz + noff[q]] : T(0);
            if (inside) {
                pr = fr[pz + own];
                if (!FIRST) pd = fdin[pz + own];
                px4 = xval(z + 4);
                if (SMAG) {
                    const int sz = eddy_row(z + 2, G.nz);
                    pnu2 = sz >= 0 ? nu[(size_t)sz * nxy + own] : T(0);
                }
            }
        };
        prefetch(z0);
        for (int z = z0; z < z1; ++z) {
            const size_t pz = (size_t)z * nxy;
#pragma unroll
            for (int q = 0; q < XS; ++q)
                if (xoff[q] >= 0) xs[threadIdx.x + q * NTHREADS] = sc * px[q];
            if (SMAG) {
#pragma unroll
                for (int q = 0; q < NS; ++q)
                    if (noff[q] >= 0) ns[threadIdx.x + q * NTHREADS] = pn[q];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < AS; ++q) {
                if (anu[q] < 0) continue;
                const bool xarm = acen[q] >= 0;
                const int c = xarm ? acen[q] : -acen[q] - 1;
                const T d = xarm ? dd(xs, c, 1, ix) : dd(xs, c, SX, iy);
                T kv = T(1);
                if (SMAG) {
                    const T nv = ns[anu[q]];
                    kv = SMAG == 2 ? dd3_coef(nv, false, fld == 3, G) : nv * kscale;
                }
                kg[threadIdx.x + q * NTHREADS] = SMAG ? kv * d : d;
            }
            __syncthreads();
            const T rv = pr, dv = pd, nu2 = pnu2;
            xw[8] = px4;
            if (z + 1 < z1) prefetch(z + 1);
            if (inside) {
                {
                    const T dz2 = d5(xw[4], xw[5], xw[7], xw[8], iz);
                    fw[4] = SMAG ? (SMAG == 2 ? dd3_coef(nu2, true, fld == 3, G) : nu2 * kscale) * dz2 : dz2;
                }
                const int cax = ty * NX + tx + R;
                const int cay = AXN + (ty + R) * PX + tx;
                T dif;
                if (SMAG) {
                    dif = dd(kg, cax, 1, ix) + dd(kg, cay, PX, iy) +
                          (T(2.0 / 3.0) * (fw[3] - fw[1]) - T(1.0 / 12.0) * (fw[4] - fw[0])) * iz;
                } else {
                    dif = Kc * dd(kg, cax, 1, ix) + Kc * dd(kg, cay, PX, iy) + Kc * d5(fw[0], fw[1], fw[3], fw[4], iz);
                }
                const T xk = xw[4];
                const size_t o = pz + own;
                const T res = rv - (T(G.two_over_dt) * xk - dif);
                const T dprev = FIRST ? rv * ith : dv;
                const T dk = a1 * dprev + a2 * res;
                const T xn = xk + dk;
                fzo[o] = xn;
                if (!LAST) fdo[o] = dk;
                if (LAST) acc[0] += xn * xn;
#pragma unroll
                for (int q = 0; q < 8; ++q) xw[q] = xw[q + 1];
#pragma unroll
                for (int q = 0; q < 4; ++q) fw[q] = fw[q + 1];
            }
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


// ------------------------------------------------------------------ launchers
template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int MODE>
constexpr size_t plane_smem(int smag) {
    constexpr int SP = (PX + 2 * HALO) * (PY + 2 * HALO);
    constexpr int AN = (PX + 2 * R) * PY + PX * (PY + 2 * R);
    constexpr int NS = Two<MODE>::v ? 2 : 1;
    return sizeof(T) * ((size_t)NS * 5 * SP + (size_t)NS * 4 * AN + (smag ? (size_t)NS * AN : 0));
}

template <typename T, int MODE>
constexpr size_t slab_smem(int smag) {
    constexpr int TX = SlabT<T>::TX, TZ = SlabT<T>::TZ;
    constexpr int SP = TX * (TZ + 2 * HALO), AN = TX * (TZ + 2 * R);
    constexpr int NS = Two<MODE>::v ? 2 : 1;
    return sizeof(T) * ((size_t)NS * 5 * SP + (size_t)NS * 4 * AN + (smag ? (size_t)NS * AN : 0));
}

static int stream_blocks3(size_t n) {
    size_t b = (n + NTHREADS - 1) / NTHREADS;
    return (int)(b < (size_t)MAX_STREAM_BLOCKS ? (b > 0 ? b : 1) : MAX_STREAM_BLOCKS);
}

// Scratch of the split passes inside G.s3 (7 npt values of T): the plane
// pass's partial sums (5 npt), then the strain values s1, s0 (npt each).
template <typename T>
struct S3 {
    T *P, *s1, *s0;
    explicit S3(const Geo& G) {
        T* b = reinterpret_cast<T*>(G.s3);
        P = b;
        s1 = b + 5 * (size_t)G.npt;
        s0 = b + 6 * (size_t)G.npt;
    }
};

template <typename T, int MODE, int SMAG>
static cudaError_t launch_split(const Geo& G, const T* u, const T* v, const T* Fu, const double* f, T* out,
                                T* out2, double* part, Ctl* ctl, int check_done, cudaStream_t s) {
    if (G.s3 == nullptr) return cudaErrorInvalidValue;
    S3<T> sc(G);
    const size_t smp = plane_smem<T, MODE>(SMAG), sms = slab_smem<T, MODE>(SMAG);
    static std::atomic<bool> configured{false};   // set once; concurrent first calls are harmless
    if (!configured) {
        cudaError_t e = set_smem(plane3d<T, MODE, SMAG>, smp);
        if (e != cudaSuccess) return e;
        if ((e = set_smem(slab3d<T, MODE, SMAG>, sms)) != cudaSuccess) return e;
        configured = true;
    }
    if (SMAG) {
        dim3 gk((G.nx + KX - 1) / KX, (G.ny + KY - 1) / KY, (G.nz + SZB - 1) / SZB);
        strain3d<T, MODE, 0><<<gk, NTHREADS, 0, s>>>(G, u, v, sc.s0, sc.s1, part, ctl, check_done);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    dim3 gp((G.nx + PX - 1) / PX, (G.ny + PY - 1) / PY, G.nz);
    plane3d<T, MODE, SMAG><<<gp, NTHREADS, smp, s>>>(G, u, v, sc.s0, sc.s1, sc.P, ctl, check_done);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    constexpr int TX = SlabT<T>::TX, TZ = SlabT<T>::TZ;
    dim3 gs((G.nz + TZ - 1) / TZ, (G.nx + TX - 1) / TX, G.ny);
    slab3d<T, MODE, SMAG><<<gs, NTHREADS, sms, s>>>(G, u, v, Fu, f, sc.s0, sc.s1, sc.P, out, out2, part, ctl,
                                                     check_done);
    return cudaGetLastError();
}

template <typename T, int MODE>
static cudaError_t launch_split_m(const Geo& G, const T* u, const T* v, const T* Fu, const double* f, T* out,
                                  T* out2, double* part, Ctl* ctl, int check_done, cudaStream_t s) {
    if (G.sgs == 2) return launch_split<T, MODE, 2>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
    return G.smag ? launch_split<T, MODE, 1>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s)
                  : launch_split<T, MODE, 0>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
}

// ---------------------------------------------------------------------------
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

}  // namespace d3

// ------------------------------------------------------------------ entry points
int stencil3d_part_blocks(const Geo& G) {
    // largest reduction grid any 3-D kernel launches
    using namespace d3;
    const long long slab = (long long)((G.nz + SlabT<float>::TZ - 1) / SlabT<float>::TZ) *
                           ((G.nx + SlabT<float>::TX - 1) / SlabT<float>::TX) * G.ny;
    const long long slab64 = (long long)((G.nz + SlabT<double>::TZ - 1) / SlabT<double>::TZ) *
                             ((G.nx + SlabT<double>::TX - 1) / SlabT<double>::TX) * G.ny;
    const long long cheb = (long long)((G.nx + PX - 1) / PX) * ((G.ny + PY - 1) / PY) * G.nz * 5;
    const long long strain = (long long)((G.nx + KX - 1) / KX) * ((G.ny + KY - 1) / KY) * G.nz;
    long long m = slab > slab64 ? slab : slab64;
    if (cheb > m) m = cheb;
    if (strain > m) m = strain;
    return (int)m;
}

size_t stencil3d_scratch_bytes(const Geo& G) { return 7 * (size_t)G.npt * sizeof(double); }

template <typename T>
cudaError_t launch_stencil3d(int mode, const Geo& G, const T* u, const T* v, const T* Fu, const double* f,
                             T* out, T* out2, double* part, Ctl* ctl, int check_done, cudaStream_t s) {
    using namespace d3;
    switch (mode) {
        case d3::MODE_F: return launch_split_m<T, d3::MODE_F>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
        case d3::MODE_RHS: return launch_split_m<T, d3::MODE_RHS>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
        case d3::MODE_RES: return launch_split_m<T, d3::MODE_RES>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
        case d3::MODE_JV: return launch_split_m<T, d3::MODE_JV>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
        case d3::MODE_RHSRES:
            return launch_split_m<T, d3::MODE_RHSRES>(G, u, v, Fu, f, out, out2, part, ctl, check_done, s);
        default: return cudaErrorInvalidValue;
    }
}
template cudaError_t launch_stencil3d<float>(int, const Geo&, const float*, const float*, const float*,
                                             const double*, float*, float*, double*, Ctl*, int, cudaStream_t);
template cudaError_t launch_stencil3d<double>(int, const Geo&, const double*, const double*, const double*,
                                              const double*, double*, double*, double*, Ctl*, int, cudaStream_t);

template <typename T>
cudaError_t launch_jv_diff3d(const Geo& G, const T* u, const T* v, T* out, Ctl* ctl, int check_done,
                             cudaStream_t s) {
    using namespace d3;
    return launch_split_m<T, d3::MODE_DJV>(G, u, v, nullptr, nullptr, out, nullptr, nullptr, ctl, check_done, s);
}
template cudaError_t launch_jv_diff3d<float>(const Geo&, const float*, const float*, float*, Ctl*, int, cudaStream_t);
template cudaError_t launch_jv_diff3d<double>(const Geo&, const double*, const double*, double*, Ctl*, int, cudaStream_t);

template <typename T>
cudaError_t launch_eddy3d(const Geo& G, const T* u, T* nu, double* part, Ctl* ctl, cudaStream_t s) {
    using namespace d3;
    dim3 gk((G.nx + KX - 1) / KX, (G.ny + KY - 1) / KY, (G.nz + SZB - 1) / SZB);
    strain3d<T, d3::MODE_F, 1><<<gk, NTHREADS, 0, s>>>(G, u, nullptr, nullptr, nu, part, ctl, 0);
    return cudaGetLastError();
}
template cudaError_t launch_eddy3d<float>(const Geo&, const float*, float*, double*, Ctl*, cudaStream_t);
template cudaError_t launch_eddy3d<double>(const Geo&, const double*, double*, double*, Ctl*, cudaStream_t);

template <typename T, int SMAG>
static cudaError_t launch_pc3(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da, T* db,
                              const T* nu, double* part, Ctl* ctl, int check_done, cudaStream_t s,
                              long long* launches) {
    using namespace d3;
    dim3 grid((G.nx + PX - 1) / PX, (G.ny + PY - 1) / PY, ((G.nz + CZB - 1) / CZB) * 5);
    const T* zin = nullptr;
    const T* din = nullptr;
    T* zbuf[2] = {za, zb};
    T* dbuf[2] = {da, db};
    for (int k = 1; k <= sweeps - 1; ++k) {
        const bool first = k == 1, last = k == sweeps - 1;
        T* zo = last ? z : zbuf[k & 1];
        T* dO = dbuf[k & 1];
        if (first && last)
            cheb3d<T, SMAG, 1, 1><<<grid, NTHREADS, 0, s>>>(G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        else if (first)
            cheb3d<T, SMAG, 1, 0><<<grid, NTHREADS, 0, s>>>(G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        else if (last)
            cheb3d<T, SMAG, 0, 1><<<grid, NTHREADS, 0, s>>>(G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
        else
            cheb3d<T, SMAG, 0, 0><<<grid, NTHREADS, 0, s>>>(G, k, r, zin, din, zo, dO, nu, part, ctl, check_done);
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
