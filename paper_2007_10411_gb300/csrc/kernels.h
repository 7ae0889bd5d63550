// Host-side launchers of the libjfnk kernels (internal to the library).
#pragma once

#include "common.cuh"

namespace jfnk {

enum StencilMode { MODE_F = 0, MODE_RHS = 1, MODE_RES = 2, MODE_JV = 3,
                   MODE_RHSRES = 4 };   // f = 2u/dt + F(u) into out and R(u) = -2 F(u) into out2, with norms

// Number of blocks of the 2-D stencil grid for element type T.
template <typename T> int stencil_blocks(const Geo& G);

// F / 2u/dt + F / residual / plain forward-difference Jv (see stencil.cu).
template <typename T>
cudaError_t launch_stencil(int mode, const Geo& G, const T* u, const T* v, const T* Fu,
                           const double* f, T* out, T* out2, double* part, Ctl* ctl,
                           int check_done, cudaStream_t s);

// Mixed-path Jv: difference F(u + eps V) - F(u) formed without cancellation.
template <typename T>
cudaError_t launch_jv_diff(const Geo& G, const T* u, const T* v, T* out, double* part, Ctl* ctl,
                           int check_done, cudaStream_t s);

// Smagorinsky nu at every point of u, and its maximum into ctl->kmax.
template <typename T>
cudaError_t launch_eddy(const Geo& G, const T* u, T* nu, double* part, Ctl* ctl, cudaStream_t s);

// Field-block Chebyshev preconditioner z = M^{-1} r (sweeps >= 1); sets ctl->eps_jv from ||z||.
template <typename T>
cudaError_t launch_precond(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da, T* db,
                           const T* nu, double* part, Ctl* ctl, int check_done, cudaStream_t s,
                           long long* launches);

// Chebyshev coefficients of the preconditioner blocks from ctl->kmax (or the constant K).
cudaError_t launch_pc_setup(const Geo& G, int sweeps, Ctl* ctl, cudaStream_t s);

// Budgets (E_k, E_p, sum theta, sum div, max/min per field) into out[0..4+2nf).
cudaError_t launch_budgets(const Geo& G, const double* u, double dx, double dz, double lz,
                           double* part, Ctl* ctl, double* out, cudaStream_t s);

// ------------------------------------------------------------ 3-D stencils
int stencil3d_part_blocks(const Geo& G);
size_t stencil3d_scratch_bytes(const Geo& G);
template <typename T>
cudaError_t launch_stencil3d(int mode, const Geo& G, const T* u, const T* v, const T* Fu, const double* f,
                             T* out, T* out2, double* part, Ctl* ctl, int check_done, cudaStream_t s);
template <typename T>
cudaError_t launch_jv_diff3d(const Geo& G, const T* u, const T* v, T* out, Ctl* ctl, int check_done,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_eddy3d(const Geo& G, const T* u, T* nu, double* part, Ctl* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_precond3d(const Geo& G, int sweeps, const T* r, T* z, T* za, T* zb, T* da, T* db,
                             const T* nu, double* part, Ctl* ctl, int check_done, cudaStream_t s,
                             long long* launches);
cudaError_t launch_budgets3d(const Geo& G, const double* u, double dV, double dz, double lz, double* part,
                             Ctl* ctl, double* out, cudaStream_t s);

// ------------------------------------------------------------ Krylov kernels
// One Arnoldi step over v_0 .. v_{nv-1}: A writes its partial sums to partA,
// B reads them and writes its own to partB (a separate buffer), C reads partB
// and, in one extra block, updates the Hessenberg / Givens state in ctl.
template <typename T>
cudaError_t launch_arnoldi_a(const T* V, size_t ldv, const T* w, size_t n, int nv, double* partA,
                             Ctl* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_arnoldi_b(const T* V, size_t ldv, T* w, size_t n, int nv, const double* partA,
                             double* partB, Ctl* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_arnoldi_c(T* V, size_t ldv, const T* w, size_t n, int nv, int m, const double* partB,
                             Ctl* ctl, cudaStream_t s);
// Right-preconditioned path, lagged second projection: pass CA of step j
// forms v_j from w'_{j-1} (wprev) and pass B's partials of step j-1, runs the
// Givens update of column j-1, and leaves h1 = [v_0..v_j]^T w_j as partials of
// arnoldi_ca_parts(n) blocks for launch_arnoldi_b_from.
template <typename T>
cudaError_t launch_arnoldi_ca(T* V, size_t ldv, const T* wprev, const T* w, size_t n, int j, int m,
                              const double* partB, double* partA, Ctl* ctl, cudaStream_t s);
template <typename T>
int arnoldi_ca_parts(size_t n);
template <typename T>
cudaError_t launch_arnoldi_b_from(const T* V, size_t ldv, T* w, size_t n, int nv, const double* partA, int nblkA,
                                  double* partB, Ctl* ctl, cudaStream_t s);
template <typename T>
int arnoldi_a_parts(size_t n);
// Givens update of column nv - 1 alone (the last column of a full cycle).
template <typename T>
cudaError_t launch_arnoldi_givens(size_t n, int nv, int m, const double* partB, Ctl* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_update(const T* Z, size_t ldz, double* x, T* xT, size_t n, double* part,
                          Ctl* ctl, cudaStream_t s);
// Left preconditioning: r = b - w unnormalised into V0 (||r||^2 in scratch[1]);
// v_0 = z / ||z|| with ||z||^2 in scratch[1] and the cycle's g_0 (first: the
// Newton solve's preconditioned ||b||); the unit-vector finite-difference step.
template <typename T>
cudaError_t launch_restart_residual(const Geo& G, const double* R, const T* w, T* V0, size_t n, double* part,
                                    Ctl* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_left_scale(const T* z, T* V0, size_t n, int first, Ctl* ctl, cudaStream_t s);
cudaError_t launch_unit_eps(Ctl* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_cycle_init(const Geo& G, const double* R, T* V0, double* x, size_t n, double eta,
                              int m, int pc_none, Ctl* ctl, cudaStream_t s);
template <typename T>
cudaError_t launch_restart(const Geo& G, const double* R, const T* w, T* V0, size_t n, int pc_none,
                           double* part, Ctl* ctl, cudaStream_t s, long long* launches);
template <typename T>
cudaError_t launch_newton_update(const Geo& G, double* u, const double* x, T* uT, size_t n,
                                 cudaStream_t s);

// ------------------------------------------------------- vector utilities
template <typename TI, typename TO>
cudaError_t launch_convert(const TI* in, TO* out, size_t n, cudaStream_t s);
// out = in * (scale ? scale_f : 1/scale_f) per field
template <typename TI, typename TO>
cudaError_t launch_rescale(const Geo& G, const TI* in, TO* out, size_t n, int multiply, cudaStream_t s);
// ctl->scratch[slot] = ||W a||^2 (weighted = 1) or ||a||^2
template <typename T>
cudaError_t launch_norm2(const Geo& G, const T* a, size_t n, int weighted, int slot, double* part,
                         Ctl* ctl, cudaStream_t s);
// ctl->eps_jv = eps > 0 ? eps : sqrt(eps_mach (1 + sqrt(scratch[su]))) / sqrt(scratch[sv])
cudaError_t launch_set_eps(double eps, int su, int sv, Ctl* ctl, cudaStream_t s);

// ------------------------------------------------- learned preconditioner
// Training pairs.  Arnoldi step (skipped once ctl->done is set): stage
// Xs = w / ||w||.  Newton correction: stage Xs = -W R / beta0.  Then, after
// the caller's MX = M^-1 Xs, store slot ctl->ncap (< cap) of the pair buffers:
// X = Xs, T = corr / ||w|| - MX (arnoldi, corr = z_j) or corr / beta0 - MX
// (Newton, corr = x_hat), and advance ctl->ncap.
cudaError_t launch_pair_arnoldi(const float* w, float* Xs, size_t n, double* part, Ctl* ctl, cudaStream_t s);
cudaError_t launch_pair_newton(const Geo& G, const double* R, float* Xs, size_t n, const Ctl* ctl,
                               cudaStream_t s);
template <typename TC>
cudaError_t launch_pair_store(const float* Xs, const TC* corr, const float* MX, float* Xbuf, float* Tbuf, size_t n,
                              int cap, int arnoldi, Ctl* ctl, cudaStream_t s);
// ctl->eps_jv from ||z|| (skipped once ctl->done is set).
cudaError_t launch_pc_eps(const float* z, size_t n, double* part, Ctl* ctl, cudaStream_t s);

}  // namespace jfnk
