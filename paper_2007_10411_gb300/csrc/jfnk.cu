// C ABI of libjfnk: handle management, argument validation, the per-call
// entry points and the implicit-step driver (inexact Newton, Section 2.5.1,
// around restarted GMRES(m) on the device).
//
// The host only sequences kernels and reads the device control block once
// per GMRES cycle and once per Newton correction; every vector operation of
// the step runs in this library's kernels.  The end of a cycle is detected
// with a pipelined poll: after enqueueing Arnoldi step j the host waits for
// step j - LAG (j - 1 with the Schur-complement preconditioner) and stops
// enqueueing once that step reports the cycle done (steps enqueued after the
// finish return at entry).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "common.cuh"
#include "kernels.h"
#include "unet.h"

using namespace jfnk;

namespace {
constexpr int LAG = 2;
// A GMRES cycle with the learned preconditioner that reduces the residual by
// less than this factor hands the rest of the solve to the field-block one.
constexpr double UNET_MIN_CYCLE_REDUCTION = 0.5;
constexpr int KT_RING = 256;   // outstanding timed launches before a drain
}

struct jfnk_handle {
    jfnk_grid grid;
    jfnk_strat strat;
    jfnk_sgs sgs;
    jfnk_opts opts;
    cudaStream_t stream;
    Geo G;
    size_t npt, n, ld;
    int mixed, m;
    // float64 buffers
    double *un, *f, *R, *Fu64, *x, *tmp64, *udev, *heat, *budg;
    // stencil-precision buffers (double for FP64, float for MIXED)
    void *V, *Z, *w, *uT, *xT, *za, *zb, *da, *db, *nu, *tA, *tB;
    void* w2;        // second Jacobian-product buffer (right preconditioning: w'_{j-1} and w_j coexist)
    void* s3;        // 3-D: scratch of the split stencil passes
    double* part;
    double* partB;   // second partial-sum area (Arnoldi pass B), inside the part allocation
    Ctl* ctl;
    Ctl* hctl;       // pinned mirror of the control header
    int* hdone;      // pinned ring of per-step "done" flags
    cudaEvent_t ev[KMAX];
    long long launches;
    // kernel-family timing (roofline reports)
    unsigned int kt_mask;
    bool kt_ready;
    cudaEvent_t kt_start[KT_RING], kt_stop[KT_RING];
    int kt_fam[KT_RING];
    int kt_stepi[KT_RING];        // Krylov step of the timed launch (-1: outside a cycle)
    double kt_b[KT_RING];
    int kt_head, kt_count, kt_open;
    int kt_step;                  // Krylov step being enqueued (-1: outside a cycle)
    int kt_every;                 // in-cycle launches are timed at steps j = kt_every / 2 mod kt_every
    // timing inside captured cycles: one event pair per (step, family), recorded
    // by event nodes of the graph and read after each cycle
    bool gkt_ready, gcapturing;
    cudaEvent_t gkt_start[KMAX][JFNK_KF_COUNT], gkt_stop[KMAX][JFNK_KF_COUNT];
    double gkt_b[KMAX][JFNK_KF_COUNT];
    jfnk_kernel_time kt_acc[JFNK_KF_COUNT];
    // learned preconditioner: network and recorded training pairs
    UNet* net;
    float *capX, *capT;
    int cap_cap, cap_kinds;
    // graph-captured Krylov steps of a cycle: gseg steps per segment (-1: the
    // default of the cycle's kind, see cycle_segment)
    // (0: one stream launch per kernel), captured on a private stream and
    // keyed on everything the captured launches read from the host
    int gseg, gnseg;
    cudaStream_t gstream;
    cudaGraphExec_t gexec[KMAX];
    long long gnl[KMAX];          // kernel launches per segment
    Geo gG;
    int gsweeps, gseg_key;
    unsigned int gkt_mask;
    int gkt_every, gprecond, glearned;
    unsigned long long gnet_ver;  // network version a learned capture holds
    unsigned int gwarm_modes;     // preconditioner modes whose cycles have run once as stream launches
    const void *guT, *gZ, *gw2;
};

#define CK(call)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            fprintf(stderr, "libjfnk: %s failed: %s (%s:%d)\n", #call,            \
                    cudaGetErrorString(e_), __FILE__, __LINE__);                  \
            return JFNK_ERR_CUDA;                                                 \
        }                                                                         \
    } while (0)

static const size_t CTL_HEAD = offsetof(Ctl, h1);

// ------------------------------------------------------------------ helpers
static bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

static jfnk_status validate(const jfnk_grid* g, const jfnk_strat* s, const jfnk_sgs* q,
                            const jfnk_opts* o) {
    if (!g || !s || !q || !o) return JFNK_ERR_INVALID_ARG;
    if (g->dim != 2 && g->dim != 3) return JFNK_ERR_INVALID_ARG;
    if (g->nx < 1 || g->nz < 1 || (g->dim == 3 && g->ny < 1)) return JFNK_ERR_INVALID_ARG;
    if (!finite_pos(g->lx) || !finite_pos(g->lz) || (g->dim == 3 && !finite_pos(g->ly)))
        return JFNK_ERR_INVALID_ARG;
    if ((g->bc_bottom != JFNK_FREESLIP && g->bc_bottom != JFNK_NOSLIP) ||
        (g->bc_top != JFNK_FREESLIP && g->bc_top != JFNK_NOSLIP))
        return JFNK_ERR_INVALID_ARG;
    if (!finite_pos(s->theta0) || !isfinite(s->beta) || !isfinite(s->pbar) || !isfinite(s->g) ||
        !isfinite(s->gamma_p) || !finite_pos(s->rho0) || !finite_pos(s->cp))
        return JFNK_ERR_INVALID_ARG;
    if (q->mode != JFNK_SGS_CONST && q->mode != JFNK_SGS_SMAGORINSKY && q->mode != JFNK_SGS_DEARDORFF)
        return JFNK_ERR_INVALID_ARG;
    if (!(q->K_M >= 0.0) || !(q->K_H >= 0.0) || !(q->Cs >= 0.0) || !finite_pos(q->Pr) ||
        !isfinite(q->K_M) || !isfinite(q->K_H) || !isfinite(q->Cs))
        return JFNK_ERR_INVALID_ARG;
    if (o->precision != JFNK_FP64 && o->precision != JFNK_MIXED) return JFNK_ERR_INVALID_ARG;
    if (o->krylov_m < 1 || o->krylov_m > JFNK_MAX_KRYLOV) return JFNK_ERR_INVALID_ARG;
    if (o->precond != JFNK_PC_NONE && o->precond != JFNK_PC_BLOCK && o->precond != JFNK_PC_UNET &&
        o->precond != JFNK_PC_SCHUR && o->precond != JFNK_PC_NONLINEAR)
        return JFNK_ERR_INVALID_ARG;
    if (o->pc_sweeps < 1 || o->pc_sweeps > MAX_PC_SWEEPS) return JFNK_ERR_INVALID_ARG;
    if (!finite_pos(o->newton_rtol) || !(o->newton_atol_factor >= 0.0) ||
        !(o->eta > 0.0 && o->eta < 1.0))
        return JFNK_ERR_INVALID_ARG;
    if (o->max_newton < 0 || o->max_newton > JFNK_MAX_NEWTON || o->max_restarts < 0)
        return JFNK_ERR_INVALID_ARG;
    if (!finite_pos(o->dt) || !finite_pos(o->scale_u) || !finite_pos(o->scale_theta) ||
        !finite_pos(o->scale_p))
        return JFNK_ERR_INVALID_ARG;
    if (o->wavelet_p < 1) return JFNK_ERR_INVALID_ARG;
    // implemented subset
    if (o->wavelet_p != 2) return JFNK_ERR_UNSUPPORTED;
    if (g->nz < 4) return JFNK_ERR_INVALID_ARG;      // one mirror reflection covers the halo
    if (o->precond == JFNK_PC_UNET &&
        (o->precision != JFNK_MIXED || !unet_grid_ok(g->dim, g->nx, g->dim == 3 ? g->ny : 1, g->nz)))
        return JFNK_ERR_UNSUPPORTED;
    if (o->precond == JFNK_PC_SCHUR && o->pc_sweeps < 2) return JFNK_ERR_UNSUPPORTED;
    return JFNK_OK;
}

// The learned preconditioner is implemented for float32-basis handles on the
// grids unet_grid_ok accepts (2-D: nx, nz multiples of 32; 3-D: nx of 32, ny of
// 64, nz of 4).
static bool unet_supported(const jfnk_handle* h) {
    return h->mixed && unet_grid_ok(h->G.dim, h->grid.nx, h->G.ny, h->grid.nz);
}

static void free_all(jfnk_handle* h) {
    void* dev[] = {h->un, h->f, h->R, h->Fu64, h->x, h->tmp64, h->udev, h->heat, h->budg,
                   h->V, h->Z, h->w, h->w2, h->s3, h->uT, h->xT, h->za, h->zb, h->da, h->db, h->nu,
                   h->tA, h->tB, h->part, h->ctl};
    for (void* p : dev)
        if (p) cudaFree(p);
    if (h->net) unet_destroy(h->net);
    if (h->capX) cudaFree(h->capX);
    if (h->capT) cudaFree(h->capT);
    if (h->hctl) cudaFreeHost(h->hctl);
    if (h->hdone) cudaFreeHost(h->hdone);
    for (int i = 0; i < KMAX; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    for (int i = 0; i < KMAX; ++i)
        if (h->gexec[i]) cudaGraphExecDestroy(h->gexec[i]);
    if (h->gstream) cudaStreamDestroy(h->gstream);
    if (h->kt_ready)
        for (int i = 0; i < KT_RING; ++i) {
            cudaEventDestroy(h->kt_start[i]);
            cudaEventDestroy(h->kt_stop[i]);
        }
    if (h->gkt_ready)
        for (int j = 0; j < KMAX; ++j)
            for (int f = 0; f < JFNK_KF_COUNT; ++f) {
                cudaEventDestroy(h->gkt_start[j][f]);
                cudaEventDestroy(h->gkt_stop[j][f]);
            }
}

// ------------------------------------------------------------ kernel timing
static void kt_add(jfnk_handle* h, int fam, cudaEvent_t e0, cudaEvent_t e1, double bytes) {
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        jfnk_kernel_time& a = h->kt_acc[fam];
        a.launches += 1;
        a.ms += ms;
        a.bytes += bytes;
    } else {
        cudaGetLastError();
    }
}

// Whether the timed launch of family fam in Krylov step `step` did its work in
// a cycle that processed `cols` Hessenberg columns.  Every kernel of a step
// returns at entry once the cycle has ended, so launches past the end take
// no time and move no bytes and are left out of the averages.  In the
// fused cycle the preconditioner and Jacobian product of step cols still run
// (the cycle ends inside that step's pass CA); elsewhere the end comes with
// the Givens update of step cols - 1.
static bool kt_valid(int fam, int step, int cols, bool fused) {
    if (step < 0) return true;
    if (fused && (fam == JFNK_KF_PRECOND || fam == JFNK_KF_JV || fam == JFNK_KF_UNET)) return step <= cols;
    return step < cols;
}

static void kt_drain_cycle(jfnk_handle* h, int cols, bool fused) {
    for (int c = 0; c < h->kt_count; ++c) {
        const int i = (h->kt_head + c) % KT_RING;
        if (cols < 0 || kt_valid(h->kt_fam[i], h->kt_stepi[i], cols, fused))
            kt_add(h, h->kt_fam[i], h->kt_start[i], h->kt_stop[i], h->kt_b[i]);
        else
            cudaEventSynchronize(h->kt_stop[i]);
    }
    h->kt_head = 0;
    h->kt_count = 0;
}

static void kt_drain(jfnk_handle* h) { kt_drain_cycle(h, -1, false); }

// Timings of a captured cycle's steps (valid launches only), after the cycle.
static void kt_drain_graph(jfnk_handle* h, int cols, bool fused) {
    if (!h->gkt_mask) return;
    for (int j = 0; j <= std::min(cols, h->m - 1); ++j)
        for (int f = 0; f < JFNK_KF_COUNT; ++f)
            if (((h->gkt_mask >> f) & 1u) && j % h->gkt_every == h->gkt_every / 2 && kt_valid(f, j, cols, fused))
                kt_add(h, f, h->gkt_start[j][f], h->gkt_stop[j][f], h->gkt_b[j][f]);
}

static inline bool kt_on(const jfnk_handle* h, int fam) {
    return ((h->kt_mask >> fam) & 1u) && (h->kt_step < 0 || h->kt_step % h->kt_every == h->kt_every / 2);
}

static void kt_begin(jfnk_handle* h, int fam) {
    if (!kt_on(h, fam)) return;
    if (h->gcapturing) {   // an event node of the graph being captured
        cudaEventRecordWithFlags(h->gkt_start[h->kt_step][fam], h->stream, cudaEventRecordExternal);
        return;
    }
    if (h->kt_count == KT_RING) kt_drain(h);
    const int i = (h->kt_head + h->kt_count) % KT_RING;
    cudaEventRecord(h->kt_start[i], h->stream);
    h->kt_open = i;
}

static void kt_end(jfnk_handle* h, int fam, double bytes) {
    if (!kt_on(h, fam)) return;
    if (h->gcapturing) {
        cudaEventRecordWithFlags(h->gkt_stop[h->kt_step][fam], h->stream, cudaEventRecordExternal);
        h->gkt_b[h->kt_step][fam] = bytes;
        return;
    }
    const int i = h->kt_open;
    cudaEventRecord(h->kt_stop[i], h->stream);
    h->kt_fam[i] = fam;
    h->kt_stepi[i] = h->kt_step;
    h->kt_b[i] = bytes;
    h->kt_count += 1;
}

// Algorithmic HBM bytes of one preconditioner apply (every input read once,
// every output written once, per field plane).
static double pc_bytes(const jfnk_handle* h) {
    const double P = (double)h->npt * (h->mixed ? 4.0 : 8.0);
    const int s = h->opts.pc_sweeps;
    if (h->G.pc_schur) {
        // rhs: velocities and v_p -> rhs; each Helmholtz launch (one sweep, or two
        // in 2-D where nz >= 8) reads x (rhs on the first), rhs and d and writes x
        // and d (not on the last); back: velocities, v_theta, dp -> z but z_p
        const int nf = h->G.nf;
        double b = nf + (2.0 * nf - 1.0);     // rhs kernel + back-substitution
        const bool pairs = h->G.dim == 2 && h->G.nz >= 8;
        for (int k = 1; k <= s - 1;) {
            const bool two = pairs && k + 1 <= s - 1;
            const bool first = k == 1, last = (two ? k + 1 : k) == s - 1;
            b += (first ? 1.0 : 3.0) + (last ? 1.0 : 2.0);
            k += two ? 2 : 1;
        }
        return b * P;
    }
    if (s <= 1) return 2.0 * 4.0 * P;
    double b = 0.0;
    for (int k = 1; k <= s - 1; ++k) {
        const bool first = k == 1, last = k == s - 1;
        b += 3.0 * P * (1.0 + (first ? 0.0 : 2.0) + 1.0 + (last ? 0.0 : 1.0) + (h->G.smag ? 1.0 : 0.0));
    }
    return b + 2.0 * P;
}

// Blocks of the largest stencil grid any tile candidate can launch (4 field slices).
static int stencil_part_blocks(const Geo& G) {
    return ((G.nx + 15) / 16) * ((G.nz + 7) / 8) * 4;
}

// ------------------------------------------------------------------ create
extern "C" jfnk_status jfnk_create(const jfnk_grid* grid, const jfnk_strat* strat,
                                   const jfnk_sgs* sgs, const jfnk_opts* opts, void* cuda_stream,
                                   jfnk_handle** out) {
    if (!out) return JFNK_ERR_INVALID_ARG;
    *out = nullptr;
    jfnk_status st = validate(grid, strat, sgs, opts);
    if (st != JFNK_OK) return st;
    jfnk_handle* h = new (std::nothrow) jfnk_handle;
    if (!h) return JFNK_ERR_OOM;
    memset(h, 0, sizeof(*h));
    h->grid = *grid;
    h->strat = *strat;
    h->sgs = *sgs;
    h->opts = *opts;
    h->stream = (cudaStream_t)cuda_stream;
    h->mixed = opts->precision == JFNK_MIXED;
    h->m = opts->krylov_m;
    h->kt_step = -1;
    h->kt_every = 1;
    h->gseg = JFNK_CYCLE_GRAPH_AUTO;
    const int dim = grid->dim;
    const int ny = dim == 3 ? grid->ny : 1;
    const int nf = dim == 3 ? 5 : 4;
    h->npt = (size_t)grid->nx * ny * grid->nz;
    h->n = (size_t)nf * h->npt;
    h->ld = (h->n + 63) / 64 * 64;

    Geo& G = h->G;
    memset(&G, 0, sizeof(G));
    G.dim = dim;
    G.nx = grid->nx;
    G.ny = ny;
    G.nz = grid->nz;
    G.npt = (int)h->npt;
    G.nf = nf;
    const int sb = grid->bc_bottom == JFNK_FREESLIP ? 1 : -1;
    const int stp = grid->bc_top == JFNK_FREESLIP ? 1 : -1;
    // parities: horizontal velocities follow the wall condition, w is odd, theta and p even
    for (int f = 0; f < nf; ++f) {
        const bool horiz = f < nf - 3;
        const bool wv = f == nf - 3;
        G.pb[f] = horiz ? sb : (wv ? -1 : 1);
        G.pt[f] = horiz ? stp : (wv ? -1 : 1);
    }
    const double dx = grid->lx / grid->nx, dz = grid->lz / grid->nz;
    const double dy = dim == 3 ? grid->ly / ny : 1.0;
    G.inv_dx = 1.0 / dx;
    G.inv_dy = 1.0 / dy;
    G.inv_dz = 1.0 / dz;
    G.fx1 = (float)(2.0 / 3.0 / dx);
    G.fx2 = (float)(-1.0 / 12.0 / dx);
    G.fz1 = (float)(2.0 / 3.0 / dz);
    G.fz2 = (float)(-1.0 / 12.0 / dz);
    G.theta0 = strat->theta0;
    G.beta = strat->beta;
    G.pbar = strat->pbar;
    G.g = strat->g;
    G.gamma_p = strat->gamma_p;
    G.heat_coef = 1.0 / (strat->rho0 * strat->cp * dz);
    G.sgs = sgs->mode;
    G.smag = sgs->mode != JFNK_SGS_CONST;
    G.K_M = G.smag ? 0.0 : sgs->K_M;
    G.K_H = G.smag ? 0.0 : sgs->K_H;
    const double delta = dim == 3 ? cbrt(dx * dy * dz) : sqrt(dx * dz);
    G.cs2 = (sgs->Cs * delta) * (sgs->Cs * delta);
    {
        // Deardorff (Section 2.4, Eq. KmM): eps^(1/3) = (cs2 / 2)^(1/3) s, so every
        // coefficient is a constant times s (times 1 + 2l/h for heat)
        const double dyh = dim == 3 ? dy : dx;              // dy reads as dx in 2-D
        const double c = pow(sgs->Cs, 4.0 / 3.0) * cbrt(0.5 * G.cs2);
        G.dd_cm = c * pow(dx * dyh, 2.0 / 3.0);
        G.dd_cM = c * pow(dz, 4.0 / 3.0);
        G.dd_delta = delta;
        const double n2 = strat->g * strat->beta / strat->theta0;
        // l = 0.75 sqrt(e) / N with sqrt(e) = nu / (0.1 Delta) = cs2 s / (0.1 Delta)
        G.dd_cl = n2 > 0.0 ? 0.75 * G.cs2 / (0.1 * delta) / sqrt(n2) : -1.0;
        G.dd_ah = 2.0 / sqrt(dx * dyh);
        G.dd_az = 2.0 / dz;
    }
    G.inv_Pr = 1.0 / sgs->Pr;
    G.two_over_dt = 2.0 / opts->dt;
    for (int f = 0; f < nf; ++f) {
        G.scale[f] = f < nf - 2 ? opts->scale_u : (f == nf - 2 ? opts->scale_theta : opts->scale_p);
        G.inv_scale[f] = 1.0 / G.scale[f];
    }
    G.heat = nullptr;
    G.tile_jv = 0;
    G.tile_pc = 0;
    G.pc_schur = opts->precond == JFNK_PC_SCHUR;
    G.half_dt = 0.5 * opts->dt;
    G.helm_a = strat->gamma_p * strat->pbar * strat->theta0 * G.half_dt;
    G.schur_cdiv = strat->gamma_p * strat->pbar * G.half_dt * G.scale[0] * G.inv_scale[nf - 1];
    G.schur_cgrad = strat->theta0 * G.scale[nf - 1] * G.inv_scale[0];

    const size_t eT = h->mixed ? sizeof(float) : sizeof(double);
    const size_t nb8 = h->ld * sizeof(double);
    const size_t nbT = h->ld * eT;
    const int m = h->m;
    int maxblk = std::max(MAX_STREAM_BLOCKS, MAX_DOT_BLOCKS);
    maxblk = std::max(maxblk, dim == 3 ? stencil3d_part_blocks(G) : stencil_part_blocks(G));
    {   // multi-dot grids: up to n / (4 * NTHREADS * 64) CTAs
        const size_t rb = h->n / ((size_t)NTHREADS * 64) + 1;
        maxblk = std::max(maxblk, (int)std::min(rb, (size_t)MAX_REDUCE_BLOCKS));
    }
    const size_t partA_len = (size_t)maxblk * (KMAX + 2) + 16 * (size_t)MAX_STREAM_BLOCKS;
    const size_t part_len = partA_len + (size_t)maxblk * (KMAX + 2);

#define ALLOC(ptr, bytes)                                                         \
    do {                                                                          \
        if (cudaMalloc((void**)&(ptr), (bytes)) != cudaSuccess) {                 \
            cudaGetLastError();                                                   \
            free_all(h);                                                          \
            delete h;                                                             \
            return JFNK_ERR_OOM;                                                  \
        }                                                                         \
    } while (0)
    ALLOC(h->un, nb8);
    ALLOC(h->f, nb8);
    ALLOC(h->R, nb8);
    if (!h->mixed) ALLOC(h->Fu64, nb8);
    ALLOC(h->x, nb8);
    ALLOC(h->tmp64, nb8);
    ALLOC(h->udev, nb8);
    ALLOC(h->heat, (size_t)grid->nx * ny * sizeof(double));
    ALLOC(h->budg, 64 * sizeof(double));
    ALLOC(h->V, (size_t)(m + 1) * nbT);
    if (opts->precond != JFNK_PC_NONE) ALLOC(h->Z, (size_t)m * nbT);
    ALLOC(h->w, nbT);
    if (opts->precond != JFNK_PC_NONE && opts->precond != JFNK_PC_NONLINEAR) ALLOC(h->w2, nbT);
    if (h->mixed) {
        ALLOC(h->uT, nbT);
        ALLOC(h->xT, nbT);
    }
    ALLOC(h->za, nbT);
    ALLOC(h->zb, nbT);
    ALLOC(h->da, nbT);
    ALLOC(h->db, nbT);
    ALLOC(h->nu, h->npt * eT);
    if (dim == 3) {
        ALLOC(h->s3, stencil3d_scratch_bytes(G));
        G.s3 = h->s3;
    }
    ALLOC(h->tA, nbT);
    ALLOC(h->tB, nbT);
    ALLOC(h->part, part_len * sizeof(double));
    h->partB = h->part + partA_len;
    ALLOC(h->ctl, sizeof(Ctl));
#undef ALLOC
    if (cudaMallocHost((void**)&h->hctl, sizeof(Ctl)) != cudaSuccess ||
        cudaMallocHost((void**)&h->hdone, KMAX * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        free_all(h);
        delete h;
        return JFNK_ERR_OOM;
    }
    memset(h->hctl, 0, sizeof(Ctl));
    for (int i = 0; i < KMAX; ++i) {
        if (cudaEventCreateWithFlags(&h->ev[i], cudaEventDisableTiming) != cudaSuccess) {
            free_all(h);
            delete h;
            return JFNK_ERR_CUDA;
        }
    }
    Ctl init;
    memset(&init, 0, sizeof(init));
    // Both paths use the float64 unit roundoff in the step rule: the mixed
    // path forms F(u + eps V) - F(u) in difference form, without cancellation,
    // so its step need not grow with the float32 roundoff.
    init.eps_mach = ldexp(1.0, -52);
    init.m = m;
    if (cudaMemcpy(h->ctl, &init, sizeof(Ctl), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(h->part, 0, part_len * sizeof(double)) != cudaSuccess ||
        cudaMemset(h->x, 0, nb8) != cudaSuccess) {
        free_all(h);
        delete h;
        return JFNK_ERR_CUDA;
    }
    *out = h;
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_destroy(jfnk_handle* h) {
    if (!h) return JFNK_OK;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_set_surface_flux(jfnk_handle* h, const double* H) {
    if (!h) return JFNK_ERR_INVALID_ARG;
    if (H == nullptr) {
        h->G.heat = nullptr;
        return JFNK_OK;
    }
    CK(cudaMemcpyAsync(h->heat, H, (size_t)h->grid.nx * h->G.ny * sizeof(double),
                       cudaMemcpyDeviceToDevice, h->stream));
    h->G.heat = h->heat;
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_kernel_timing(jfnk_handle* h, unsigned int mask) {
    return jfnk_kernel_timing_sampled(h, mask, 1);
}

extern "C" jfnk_status jfnk_kernel_timing_sampled(jfnk_handle* h, unsigned int mask, int every) {
    if (!h || every < 1) return JFNK_ERR_INVALID_ARG;
    if (mask != 0 && !h->kt_ready) {
        for (int i = 0; i < KT_RING; ++i) {
            CK(cudaEventCreate(&h->kt_start[i]));
            CK(cudaEventCreate(&h->kt_stop[i]));
        }
        h->kt_ready = true;
    }
    if (h->kt_count) kt_drain(h);
    h->kt_mask = mask;
    h->kt_every = every;
    memset(h->kt_acc, 0, sizeof(h->kt_acc));
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_kernel_timing_read(jfnk_handle* h, jfnk_kernel_time* out) {
    if (!h || !out) return JFNK_ERR_INVALID_ARG;
    kt_drain(h);
    memcpy(out, h->kt_acc, sizeof(h->kt_acc));
    return JFNK_OK;
}

// Time every tile candidate of the float32 Jacobian-product and preconditioner
// kernels on this handle's grid (inputs: u and a direction built from it) and
// keep the fastest; tiles[0..1] (may be NULL) receive the chosen indices.
template <typename T>
static jfnk_status autotune_impl(jfnk_handle* h, const double* u, int* tiles) {
    cudaStream_t s = h->stream;
    Geo& G = h->G;
    T* uT = (T*)h->uT;
    T* dir = (T*)h->tA;
    CK((launch_convert<double, T>(u, uT, h->n, s)));
    CK((launch_rescale<double, T>(G, u, dir, h->n, 0, s)));
    CK(launch_norm2<double>(G, u, h->n, 1, 2, h->part, h->ctl, s));
    CK(launch_set_eps(1e-6, 2, 3, h->ctl, s));
    CK(launch_norm2<double>(G, u, h->n, 1, 2, h->part, h->ctl, s));
    if (G.smag) CK(launch_eddy<T>(G, uT, (T*)h->nu, h->part, h->ctl, s));
    CK(launch_pc_setup(G, h->opts.pc_sweeps, h->ctl, s));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int reps = 16;
    float best_jv = 1e30f, best_pc = 1e30f;
    int arg_jv = 0, arg_pc = 0;
    for (int c = 0; c < NUM_TILE_SHAPES; ++c) {
        G.tile_jv = c;
        G.tile_pc = c;
        for (int pass = 0; pass < 4; ++pass) {          // pass 0 warms up (and sets shared-memory limits)
            CK(cudaEventRecord(e0, s));
            for (int r = 0; r < reps; ++r) CK(launch_jv_diff<T>(G, uT, dir, (T*)h->w, h->part, h->ctl, 0, s));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (pass > 0 && ms < best_jv) { best_jv = ms; arg_jv = c; }   // best of three timings
        }
        if (h->opts.precond != JFNK_PC_NONE && h->opts.pc_sweeps > 1) {
            for (int pass = 0; pass < 4; ++pass) {
                CK(cudaEventRecord(e0, s));
                for (int r = 0; r < reps; ++r)
                    CK(launch_precond<T>(G, h->opts.pc_sweeps, dir, (T*)h->tB, (T*)h->za, (T*)h->zb,
                                         (T*)h->da, (T*)h->db, (const T*)h->nu, h->part, h->ctl, 0, s,
                                         nullptr));
                CK(cudaEventRecord(e1, s));
                CK(cudaEventSynchronize(e1));
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, e0, e1));
                if (pass > 0 && ms < best_pc) { best_pc = ms; arg_pc = c; }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    G.tile_jv = arg_jv;
    G.tile_pc = arg_pc;
    if (tiles) { tiles[0] = arg_jv; tiles[1] = arg_pc; }
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_autotune(jfnk_handle* h, const double* u, int* tiles) {
    if (!h || !u) return JFNK_ERR_INVALID_ARG;
    if (!h->mixed) {                       // the float64 kernels have a single tile shape
        if (tiles) { tiles[0] = h->G.tile_jv; tiles[1] = h->G.tile_pc; }
        return JFNK_OK;
    }
    return autotune_impl<float>(h, u, tiles);
}

extern "C" jfnk_status jfnk_set_tiles(jfnk_handle* h, int tile_jv, int tile_pc) {
    if (!h || tile_jv < 0 || tile_jv >= NUM_TILE_SHAPES || tile_pc < 0 || tile_pc >= NUM_TILE_SHAPES)
        return JFNK_ERR_INVALID_ARG;
    h->G.tile_jv = tile_jv;
    h->G.tile_pc = tile_pc;
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_set_cycle_graph(jfnk_handle* h, int steps) {
    if (!h || steps < JFNK_CYCLE_GRAPH_AUTO) return JFNK_ERR_INVALID_ARG;
    h->gseg = steps < 0 ? JFNK_CYCLE_GRAPH_AUTO : std::min(steps, h->m);
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_get_launch_count(jfnk_handle* h, long long* out) {
    if (!h || !out) return JFNK_ERR_INVALID_ARG;
    *out = h->launches;
    return JFNK_OK;
}

// ------------------------------------------------------------ per-call ABI
template <typename T>
static jfnk_status rhs_impl(jfnk_handle* h, const double* u, double* F) {
    cudaStream_t s = h->stream;
    if (sizeof(T) == sizeof(double)) {
        CK(launch_stencil<double>(MODE_F, h->G, u, nullptr, nullptr, nullptr, F, nullptr, h->part,
                                  h->ctl, 0, s));
        h->launches += 1;
        return JFNK_OK;
    }
    T* uT = (T*)h->tA;
    T* FT = (T*)h->tB;
    CK((launch_convert<double, T>(u, uT, h->n, s)));
    CK(launch_stencil<T>(MODE_F, h->G, uT, nullptr, nullptr, nullptr, FT, nullptr, h->part, h->ctl,
                         0, s));
    CK((launch_convert<T, double>(FT, F, h->n, s)));
    h->launches += 3;
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_rhs(jfnk_handle* h, const double* u, double* F) {
    if (!h || !u || !F) return JFNK_ERR_INVALID_ARG;
    return h->mixed ? rhs_impl<float>(h, u, F) : rhs_impl<double>(h, u, F);
}

extern "C" jfnk_status jfnk_residual(jfnk_handle* h, const double* u_n, const double* u, double* R) {
    if (!h || !u_n || !u || !R) return JFNK_ERR_INVALID_ARG;
    cudaStream_t s = h->stream;
    CK(launch_stencil<double>(MODE_RHS, h->G, u_n, nullptr, nullptr, nullptr, h->tmp64, nullptr,
                              h->part, h->ctl, 0, s));
    CK(launch_stencil<double>(MODE_RES, h->G, u, nullptr, nullptr, h->tmp64, R, nullptr, h->part,
                              h->ctl, 0, s));
    h->launches += 2;
    return JFNK_OK;
}

template <typename T>
static jfnk_status jv_impl(jfnk_handle* h, const double* u, const double* F_u, const double* v,
                           double eps, double* Jv) {
    cudaStream_t s = h->stream;
    const Geo& G = h->G;
    CK(launch_norm2<double>(G, u, h->n, 1, 2, h->part, h->ctl, s));
    CK(launch_norm2<double>(G, v, h->n, 1, 3, h->part, h->ctl, s));
    CK(launch_set_eps(eps, 2, 3, h->ctl, s));
    T* vh = (T*)h->tA;
    T* wh = (T*)h->tB;
    CK((launch_rescale<double, T>(G, v, vh, h->n, 0, s)));
    h->launches += 4;
    if (sizeof(T) == sizeof(double)) {
        const double* Fu = F_u;
        if (!Fu) {
            CK(launch_stencil<double>(MODE_F, G, u, nullptr, nullptr, nullptr, h->tmp64, nullptr,
                                      h->part, h->ctl, 0, s));
            Fu = h->tmp64;
            h->launches += 1;
        }
        CK(launch_stencil<double>(MODE_JV, G, u, (const double*)vh, Fu, nullptr, (double*)wh,
                                  nullptr, h->part, h->ctl, 0, s));
    } else {
        T* uT = (T*)h->uT;
        CK((launch_convert<double, T>(u, uT, h->n, s)));
        CK(launch_jv_diff<T>(G, uT, vh, wh, h->part, h->ctl, 0, s));
        h->launches += 1;
    }
    CK((launch_rescale<T, double>(G, wh, Jv, h->n, 1, s)));
    h->launches += 2;
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_jv(jfnk_handle* h, const double* u, const double* F_u, const double* v,
                               double eps, double* Jv, double* eps_out) {
    if (!h || !u || !v || !Jv || !isfinite(eps)) return JFNK_ERR_INVALID_ARG;
    jfnk_status st = h->mixed ? jv_impl<float>(h, u, F_u, v, eps, Jv) : jv_impl<double>(h, u, F_u, v, eps, Jv);
    if (st != JFNK_OK) return st;
    if (eps_out) {
        CK(cudaMemcpyAsync(h->hctl, h->ctl, CTL_HEAD, cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        *eps_out = h->hctl->eps_jv;
    }
    return JFNK_OK;
}

template <typename T>
static jfnk_status precond_impl(jfnk_handle* h, const double* u, const double* r, double* z) {
    cudaStream_t s = h->stream;
    const Geo& G = h->G;
    if (h->opts.precond == JFNK_PC_NONE) {
        CK(cudaMemcpyAsync(z, r, h->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return JFNK_OK;
    }
    const T* uT;
    const T* rT;
    T* zT;
    if (sizeof(T) == sizeof(double)) {
        uT = (const T*)u;
        rT = (const T*)r;
        zT = (T*)z;
    } else {
        CK((launch_convert<double, T>(u, (T*)h->uT, h->n, s)));
        CK((launch_convert<double, T>(r, (T*)h->tA, h->n, s)));
        h->launches += 2;
        uT = (const T*)h->uT;
        rT = (const T*)h->tA;
        zT = (T*)h->tB;
    }
    if (G.smag) {
        CK(launch_eddy<T>(G, uT, (T*)h->nu, h->part, h->ctl, s));
        h->launches += 1;
    }
    CK(launch_pc_setup(G, h->opts.pc_sweeps, h->ctl, s));
    h->launches += 1;
    CK(launch_precond<T>(G, h->opts.pc_sweeps, rT, zT, (T*)h->za, (T*)h->zb, (T*)h->da, (T*)h->db,
                         (const T*)h->nu, h->part, h->ctl, 0, s, &h->launches));
    if constexpr (sizeof(T) == sizeof(float)) {
        if (h->opts.precond == JFNK_PC_UNET && h->net) {
            CK(unet_apply(h->net, rT, zT, 1, nullptr, s));
            h->launches += unet_launches_per_apply();
        }
    }
    if (sizeof(T) != sizeof(double)) {
        CK((launch_convert<T, double>(zT, z, h->n, s)));
        h->launches += 1;
    }
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_precond_apply(jfnk_handle* h, const double* u, const double* r, double* z) {
    if (!h || !u || !r || !z) return JFNK_ERR_INVALID_ARG;
    return h->mixed ? precond_impl<float>(h, u, r, z) : precond_impl<double>(h, u, r, z);
}

// ------------------------------------------------------------------- step
// Pair recording requested for these kinds and, as of the last control-block
// read, room left in the store (the device makes the final check).
static bool capturing(const jfnk_handle* h, int kinds) {
    return (h->cap_kinds & kinds) && h->capX != nullptr && h->hctl->ncap < h->cap_cap;
}

static jfnk_status read_ctl(jfnk_handle* h) {
    CK(cudaMemcpyAsync(h->hctl, h->ctl, CTL_HEAD, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return JFNK_OK;
}

// Jacobian-vector product of the Newton system in scaled units: w = J_hat z.
template <typename T>
static jfnk_status apply_jv(jfnk_handle* h, const T* uT, const T* z, T* w, int check_done) {
    kt_begin(h, JFNK_KF_JV);
    if (sizeof(T) == sizeof(double)) {
        CK(launch_stencil<double>(MODE_JV, h->G, (const double*)uT, (const double*)z, h->Fu64,
                                  nullptr, (double*)w, nullptr, h->part, h->ctl, check_done, h->stream));
    } else {
        CK(launch_jv_diff<T>(h->G, uT, z, w, h->part, h->ctl, check_done, h->stream));
    }
    kt_end(h, JFNK_KF_JV, (double)h->n * (h->mixed ? 3.0 * 4.0 : 4.0 * 8.0));
    h->launches += 1;
    return JFNK_OK;
}

// One Krylov step of the fused cycle (right preconditioner but the Schur
// complement), with the second projection of CGS2 lagged behind the next
// Jacobian product (Arnoldi passes CA and B per step, see arnoldi_ca): step j
// takes the direction d_j = v_0 (j = 0) or w'_{j-1}, z_j = M^{-1} d_j
// (+ N(d_j) for the learned correction), w_j = J z_j; pass CA forms v_j,
// updates column j-1 of the Hessenberg / Givens state and projects w_j once;
// pass B projects it again into w'_j.  The w'_{j-1} / w_j buffers alternate
// between w and w2.
template <typename T>
static jfnk_status fused_step(jfnk_handle* h, const T* uT, bool learned, bool arnoldi_pairs, int j) {
    cudaStream_t s = h->stream;
    const Geo& G = h->G;
    const size_t n = h->n, ld = h->ld;
    const int m = h->m;
    T* V = (T*)h->V;
    T* Z = (T*)h->Z;
    T* wb[2] = {(T*)h->w, (T*)h->w2};
    const double vb = (double)n * sizeof(T);
    h->kt_step = j;
    const T* dj = j == 0 ? V : wb[(j - 1) & 1];
    T* zj = Z + (size_t)j * ld;
    T* wj = wb[j & 1];
    kt_begin(h, JFNK_KF_PRECOND);
    CK(launch_precond<T>(G, h->opts.pc_sweeps, dj, zj, (T*)h->za, (T*)h->zb, (T*)h->da, (T*)h->db,
                         (const T*)h->nu, h->part, h->ctl, 1, s, &h->launches));
    kt_end(h, JFNK_KF_PRECOND, pc_bytes(h));
    if constexpr (sizeof(T) == sizeof(float)) {
        if (learned) {   // z_j += N(d_j), then the FD step for the new ||z_j||
            kt_begin(h, JFNK_KF_UNET);
            CK(unet_apply(h->net, (const float*)dj, (float*)zj, 1, &h->ctl->done, s));
            kt_end(h, JFNK_KF_UNET, 3.0 * (double)n * sizeof(float));
            CK(launch_pc_eps(zj, n, h->part, h->ctl, s));
            h->launches += unet_launches_per_apply() + 1;
        }
    }
    jfnk_status st = apply_jv<T>(h, uT, zj, wj, 1);
    if (st != JFNK_OK) return st;
    if constexpr (sizeof(T) == sizeof(float)) {
        if (arnoldi_pairs) {   // (J z_j, z_j) is an exact inverse pair
            CK(launch_pair_arnoldi(wj, (float*)h->tA, n, h->part, h->ctl, s));
            CK(launch_precond<float>(G, h->opts.pc_sweeps, (const float*)h->tA, (float*)h->tB,
                                     (float*)h->za, (float*)h->zb, (float*)h->da, (float*)h->db,
                                     (const float*)h->nu, h->part, h->ctl, 1, s, &h->launches));
            CK(launch_pair_store<float>((const float*)h->tA, zj, (const float*)h->tB, h->capX, h->capT, n,
                                        h->cap_cap, 1, h->ctl, s));
            h->launches += 4;
        }
    }
    kt_begin(h, JFNK_KF_ARNOLDI_A);
    int nblkA;
    if (j == 0) {
        CK(launch_arnoldi_a<T>(V, ld, wj, n, 1, h->part, h->ctl, s));
        nblkA = arnoldi_a_parts<T>(n);
        kt_end(h, JFNK_KF_ARNOLDI_A, 2 * vb);
    } else {
        CK(launch_arnoldi_ca<T>(V, ld, wb[(j - 1) & 1], wj, n, j, m, h->partB, h->part, h->ctl, s));
        nblkA = arnoldi_ca_parts<T>(n);
        kt_end(h, JFNK_KF_ARNOLDI_A, (j + 3) * vb);   // reads v_0..v_{j-1}, w'_{j-1}, w_j; writes v_j
    }
    kt_begin(h, JFNK_KF_ARNOLDI_B);
    CK(launch_arnoldi_b_from<T>(V, ld, wj, n, j + 1, h->part, nblkA, h->partB, h->ctl, s));
    kt_end(h, JFNK_KF_ARNOLDI_B, (j + 3) * vb);      // reads v_0..v_j, w_j; writes w'_j
    h->launches += 2;
    return JFNK_OK;
}

// One Krylov step of the three-pass cycle (no preconditioner, the Schur
// complement, or nonlinear preconditioning from the left): z_j = M^{-1} v_j
// (right) or v_j, w = J z_j (left: w <- M^{-1} w), pass A h1 = V^T w, pass B
// w' = w - V h1 and h2 = V^T w', pass C (block 0: Hessenberg / Givens update
// of column j) v_{j+1} = (w' - V h2) / h_{j+1,j}.
template <typename T>
static jfnk_status plain_step(jfnk_handle* h, const T* uT, bool learned, bool arnoldi_pairs, int j) {
    cudaStream_t s = h->stream;
    const Geo& G = h->G;
    const size_t n = h->n, ld = h->ld;
    const int m = h->m;
    const bool left = h->opts.precond == JFNK_PC_NONLINEAR;
    const bool pc = h->opts.precond != JFNK_PC_NONE && !left;
    T* V = (T*)h->V;
    T* Z = pc ? (T*)h->Z : V;
    T* w = (T*)h->w;
    h->kt_step = j;
    T* vj = V + (size_t)j * ld;
    T* zj = Z + (size_t)j * ld;
    if (pc) {
        kt_begin(h, JFNK_KF_PRECOND);
        CK(launch_precond<T>(G, h->opts.pc_sweeps, vj, zj, (T*)h->za, (T*)h->zb, (T*)h->da, (T*)h->db,
                             (const T*)h->nu, h->part, h->ctl, 1, s, &h->launches));
        kt_end(h, JFNK_KF_PRECOND, pc_bytes(h));
    }
    if constexpr (sizeof(T) == sizeof(float)) {
        if (learned) {   // z_j += N(v_j), then the FD step for the new ||z_j||
            kt_begin(h, JFNK_KF_UNET);
            CK(unet_apply(h->net, vj, zj, 1, &h->ctl->done, s));
            kt_end(h, JFNK_KF_UNET, 3.0 * (double)n * sizeof(float));
            CK(launch_pc_eps(zj, n, h->part, h->ctl, s));
            h->launches += unet_launches_per_apply() + 1;
        }
    }
    jfnk_status st = apply_jv<T>(h, uT, zj, w, 1);
    if (st != JFNK_OK) return st;
    T* wa = w;                      // the vector the Arnoldi step orthogonalises
    if (left) {                     // w <- M^{-1} J v_j
        kt_begin(h, JFNK_KF_PRECOND);
        CK(launch_precond<T>(G, h->opts.pc_sweeps, w, (T*)h->tB, (T*)h->za, (T*)h->zb, (T*)h->da, (T*)h->db,
                             (const T*)h->nu, h->part, h->ctl, 1, s, &h->launches));
        kt_end(h, JFNK_KF_PRECOND, pc_bytes(h));
        CK(launch_unit_eps(h->ctl, s));      // the next product acts on the unit vector v_{j+1}
        h->launches += 1;
        wa = (T*)h->tB;
    }
    if constexpr (sizeof(T) == sizeof(float)) {
        if (arnoldi_pairs) {   // (J z_j, z_j) is an exact inverse pair
            CK(launch_pair_arnoldi(w, (float*)h->tA, n, h->part, h->ctl, s));
            CK(launch_precond<float>(G, h->opts.pc_sweeps, (const float*)h->tA, (float*)h->tB, (float*)h->za,
                                     (float*)h->zb, (float*)h->da, (float*)h->db, (const float*)h->nu, h->part,
                                     h->ctl, 1, s, &h->launches));
            CK(launch_pair_store<float>((const float*)h->tA, zj, (const float*)h->tB, h->capX, h->capT, n,
                                        h->cap_cap, 1, h->ctl, s));
            h->launches += 4;
        }
    }
    const double vb = (double)n * sizeof(T);
    kt_begin(h, JFNK_KF_ARNOLDI_A);
    CK(launch_arnoldi_a<T>(V, ld, wa, n, j + 1, h->part, h->ctl, s));
    kt_end(h, JFNK_KF_ARNOLDI_A, (j + 2) * vb);
    kt_begin(h, JFNK_KF_ARNOLDI_B);
    CK(launch_arnoldi_b<T>(V, ld, wa, n, j + 1, h->part, h->partB, h->ctl, s));
    kt_end(h, JFNK_KF_ARNOLDI_B, (j + 3) * vb);   // reads v_0..v_j, w; writes w'
    kt_begin(h, JFNK_KF_ARNOLDI_C);
    CK(launch_arnoldi_c<T>(V, ld, wa, n, j + 1, m, h->partB, h->ctl, s));
    kt_end(h, JFNK_KF_ARNOLDI_C, (j + 3) * vb);
    h->launches += 3;
    return JFNK_OK;
}

// Krylov steps per captured segment.  By default one for the Schur
// complement (a solve takes a few steps, and a longer segment runs its
// expensive steps past the end), two with the learned correction (eight
// network launches per step), otherwise JFNK_CYCLE_GRAPH_SEGMENT on grids up
// to JFNK_CYCLE_GRAPH_SEGMENT_POINTS points and the whole cycle above, where
// the steps are long enough that those past the end cost little.
static int cycle_segment(const jfnk_handle* h, bool learned) {
    if (h->gseg >= 0) return h->gseg;
    if (h->G.pc_schur) return 1;
    if (learned) return std::min(h->m, 2);
    return h->npt <= (size_t)JFNK_CYCLE_GRAPH_SEGMENT_POINTS ? std::min(h->m, JFNK_CYCLE_GRAPH_SEGMENT) : h->m;
}

static void graph_release(jfnk_handle* h) {
    if (h->gnseg > 0) cudaStreamSynchronize(h->stream);   // no launch of them in flight
    for (int k = 0; k < KMAX; ++k)
        if (h->gexec[k]) {
            cudaGraphExecDestroy(h->gexec[k]);
            h->gexec[k] = nullptr;
        }
    h->gnseg = 0;
}

// Capture the cycle's m Krylov steps as segments of cycle_segment() steps.
// Every kernel of a step returns at entry once the device has ended the cycle
// (ctl->done), so a segment launched past the end leaves the state untouched,
// and the captured launches depend on the host only through the Geo, the
// sweep count, the preconditioner, the buffer pointers, the timing settings
// and (learned cycles) the network's weight version: the key a later cycle
// compares (graph_current).
template <typename T>
static jfnk_status graph_capture(jfnk_handle* h, const T* uT, bool fused, bool learned) {
    graph_release(h);
    if (!h->gstream) CK(cudaStreamCreateWithFlags(&h->gstream, cudaStreamNonBlocking));
    if (h->kt_mask && !h->gkt_ready) {
        for (int j = 0; j < KMAX; ++j)
            for (int f = 0; f < JFNK_KF_COUNT; ++f) {
                CK(cudaEventCreate(&h->gkt_start[j][f]));
                CK(cudaEventCreate(&h->gkt_stop[j][f]));
            }
        h->gkt_ready = true;
    }
    const int m = h->m, S = cycle_segment(h, learned);
    const int nseg = (m + S - 1) / S;
    cudaStream_t user = h->stream;
    h->stream = h->gstream;
    h->gcapturing = true;
    jfnk_status st = JFNK_OK;
    for (int k = 0; k < nseg && st == JFNK_OK; ++k) {
        const long long l0 = h->launches;
        cudaError_t e = cudaStreamBeginCapture(h->gstream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) {
            st = JFNK_ERR_CUDA;
            break;
        }
        for (int j = k * S; j < std::min(m, (k + 1) * S) && st == JFNK_OK; ++j)
            st = fused ? fused_step<T>(h, uT, learned, false, j) : plain_step<T>(h, uT, learned, false, j);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(h->gstream, &g);
        h->gnl[k] = h->launches - l0;
        h->launches = l0;
        if (st == JFNK_OK && e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec[k], g, 0);
        if (g) cudaGraphDestroy(g);
        if (st == JFNK_OK && e != cudaSuccess) {
            fprintf(stderr, "libjfnk: cycle capture failed: %s\n", cudaGetErrorString(e));
            st = JFNK_ERR_CUDA;
        }
    }
    h->stream = user;
    h->gcapturing = false;
    h->kt_step = -1;
    if (st != JFNK_OK) {
        cudaGetLastError();
        graph_release(h);
        return st;
    }
    h->gnseg = nseg;
    memcpy(&h->gG, &h->G, sizeof(Geo));
    h->gsweeps = h->opts.pc_sweeps;
    h->gseg_key = S;
    h->guT = uT;
    h->gZ = h->Z;
    h->gw2 = h->w2;
    h->gkt_mask = h->kt_mask;
    h->gkt_every = h->kt_every;
    h->gprecond = h->opts.precond;
    h->glearned = learned;
    h->gnet_ver = learned ? unet_version(h->net) : 0;
    return JFNK_OK;
}

template <typename T>
static bool graph_current(const jfnk_handle* h, const T* uT, bool learned) {
    return h->gnseg > 0 && h->gseg_key == cycle_segment(h, learned) && h->gsweeps == h->opts.pc_sweeps && h->guT == uT &&
           h->gZ == h->Z && h->gw2 == h->w2 && h->gkt_mask == h->kt_mask &&
           h->gkt_every == h->kt_every && h->gprecond == h->opts.precond &&
           h->glearned == (int)learned && (!learned || h->gnet_ver == unet_version(h->net)) &&
           memcmp(&h->gG, &h->G, sizeof(Geo)) == 0;
}

// One GMRES cycle: fused steps (fused_step; the last column of a full cycle
// then gets its Givens update alone) or three-pass steps (plain_step).  The
// host learns that the cycle ended from a copy of ctl->done made after each
// step (stream launches) or each captured segment of steps (graph launches),
// read with a lag so that the GPU never waits for it.
template <typename T>
static jfnk_status run_cycle(jfnk_handle* h, const T* uT, bool fused, bool learned, bool arnoldi_pairs, int lag,
                             bool* used_graph) {
    cudaStream_t s = h->stream;
    const int m = h->m;
    // the first cycle of each preconditioner mode (with and without the learned
    // correction) runs as stream launches (one-time kernel attribute set-up happens
    // outside any capture); later ones may use graphs
    const unsigned int mode_bit = 1u << (2 * h->opts.precond + (learned ? 1 : 0));
    const bool graph = cycle_segment(h, learned) > 0 && (h->gwarm_modes & mode_bit) && !arnoldi_pairs;
    h->gwarm_modes |= mode_bit;
    *used_graph = graph;
    int ncol = m;   // columns the closing Givens update of a fused cycle may cover
    if (graph) {
        if constexpr (sizeof(T) == sizeof(float)) {
            if (learned) CK(unet_prepare(h->net, s));   // weights composed outside the capture
        }
        if (!graph_current<T>(h, uT, learned)) {
            jfnk_status st = graph_capture<T>(h, uT, fused, learned);
            if (st != JFNK_OK) return st;
        }
        for (int k = 0; k < h->gnseg; ++k) {
            CK(cudaGraphLaunch(h->gexec[k], s));
            h->launches += h->gnl[k];
            CK(cudaMemcpyAsync(&h->hdone[k], &h->ctl->done, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaEventRecord(h->ev[k], s));
            if (k >= 1) {
                CK(cudaEventSynchronize(h->ev[k - 1]));
                if (h->hdone[k - 1]) break;
            }
        }
    } else {
        int j = 0;
        for (; j < m; ++j) {
            jfnk_status st = fused ? fused_step<T>(h, uT, learned, arnoldi_pairs, j)
                                   : plain_step<T>(h, uT, learned, arnoldi_pairs, j);
            if (st != JFNK_OK) return st;
            CK(cudaMemcpyAsync(&h->hdone[j], &h->ctl->done, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaEventRecord(h->ev[j], s));
            if (j >= lag) {
                CK(cudaEventSynchronize(h->ev[j - lag]));
                if (h->hdone[j - lag]) break;
            }
        }
        ncol = std::min(j + 1, m);
        h->kt_step = -1;
    }
    if (fused) {   // Givens update of the last column (returns at once when the cycle ended earlier)
        CK(launch_arnoldi_givens<T>(h->n, ncol, m, h->partB, h->ctl, s));
        h->launches += 1;
    }
    return JFNK_OK;
}

// Restarted GMRES(m) on J_hat x = -W R from x = 0 (cycle_init already enqueued).
// Nonlinear preconditioning (left): v_0 <- M^{-1} v_0 / ||M^{-1} v_0|| and the
// cycle's g_0, after cycle_init (first) or restart_residual left r in v_0.
template <typename T>
static jfnk_status left_cycle_start(jfnk_handle* h, int first) {
    cudaStream_t s = h->stream;
    const Geo& G = h->G;
    T* V0 = (T*)h->V;
    T* z = (T*)h->tA;
    CK(launch_precond<T>(G, h->opts.pc_sweeps, V0, z, (T*)h->za, (T*)h->zb, (T*)h->da, (T*)h->db,
                         (const T*)h->nu, h->part, h->ctl, 0, s, &h->launches));
    CK(launch_norm2<T>(G, z, h->n, 0, 1, h->part, h->ctl, s));
    CK(launch_left_scale<T>(z, V0, h->n, first, h->ctl, s));
    h->launches += 2;
    return JFNK_OK;
}

template <typename T>
static jfnk_status gmres_solve(jfnk_handle* h, const T* uT, int* iters, int* restarts, int* conv, int* switched) {
    cudaStream_t s = h->stream;
    const Geo& G = h->G;
    const size_t n = h->n, ld = h->ld;
    const int m = h->m;
    const bool left = h->opts.precond == JFNK_PC_NONLINEAR;      // M^{-1} J from the left
    const bool pc = h->opts.precond != JFNK_PC_NONE && !left;     // right preconditioner (stored z_j)
    bool learned = h->opts.precond == JFNK_PC_UNET && h->net != nullptr;
    // A Schur-preconditioned step is long enough (tens of launches) for the host
    // to stay ahead with a lag of one, which halves the steps enqueued past a finish.
    const int lag = h->G.pc_schur ? 1 : LAG;
    const bool arnoldi_pairs = !left && sizeof(T) == sizeof(float) && capturing(h, JFNK_PAIRS_ARNOLDI);
    T* V = (T*)h->V;
    T* Z = pc ? (T*)h->Z : V;
    T* w = (T*)h->w;
    T* xT = h->mixed ? (T*)h->xT : (T*)h->x;
    *restarts = 0;
    *conv = 0;
    *switched = 0;
    // Two-pass Arnoldi steps (fused_step) pay for themselves where a solve runs
    // many Krylov steps per expensive preconditioner apply; the Schur-complement
    // preconditioner converges in a few steps per solve, where the lagged scheme's
    // one extra (speculative) preconditioner apply and Jacobian product per cycle
    // cost more than the basis passes it saves: it keeps three passes.
    const bool fused = pc && !h->G.pc_schur;
    int iters_before = 0;
    for (int cycle = 0;; ++cycle) {
        bool graph = false;
        jfnk_status st0 = run_cycle<T>(h, uT, fused, learned, arnoldi_pairs, lag, &graph);
        if (st0 != JFNK_OK) return st0;
        h->kt_step = -1;
        CK(launch_update<T>(Z, ld, h->x, h->mixed ? xT : nullptr, n, h->part, h->ctl, s));
        h->launches += 1;
        jfnk_status st = read_ctl(h);
        if (st != JFNK_OK) return st;
        const Ctl& c = *h->hctl;
        *iters = c.iters;
        if (h->kt_mask) {   // this cycle's timed launches, those past its end left out
            const int cols = c.iters - iters_before;
            if (graph) kt_drain_graph(h, cols, fused);
            kt_drain_cycle(h, cols, fused);
        }
        iters_before = c.iters;
        if (c.nan) return JFNK_ERR_NAN;
        if (c.converged) {
            *conv = 1;
            return JFNK_OK;
        }
        if (cycle >= h->opts.max_restarts) return JFNK_OK;
        if (learned && c.gres > UNET_MIN_CYCLE_REDUCTION * c.gstart) {
            // the learned directions stalled: finish this solve with the field-block
            // preconditioner, restarting from the correction reached so far
            learned = false;
            *switched = 1;
        }
        *restarts = cycle + 1;
        st = apply_jv<T>(h, uT, xT, w, 0);
        if (st != JFNK_OK) return st;
        if (left) {
            CK(launch_restart_residual<T>(G, h->R, w, V, n, h->part, h->ctl, s));
            h->launches += 1;
            st = left_cycle_start<T>(h, 0);
            if (st != JFNK_OK) return st;
        } else {
            CK(launch_restart<T>(G, h->R, w, V, n, pc ? 0 : 1, h->part, h->ctl, s, &h->launches));
        }
    }
}

template <typename T>
static jfnk_status residual_eval(jfnk_handle* h, const double* u) {
    kt_begin(h, JFNK_KF_RESIDUAL);
    CK(launch_stencil<double>(MODE_RES, h->G, u, nullptr, nullptr, h->f, h->R, h->mixed ? nullptr : h->Fu64,
                              h->part, h->ctl, 0, h->stream));
    kt_end(h, JFNK_KF_RESIDUAL, (double)h->n * 8.0 * (h->mixed ? 3.0 : 4.0));
    h->launches += 1;
    return read_ctl(h);
}

template <typename T>
static jfnk_status step_impl(jfnk_handle* h, double* u, jfnk_stats* out) {
    cudaStream_t s = h->stream;
    const Geo& G = h->G;
    const size_t n = h->n;
    jfnk_stats stats;
    memset(&stats, 0, sizeof(stats));
    CK(cudaMemcpyAsync(h->un, u, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    T* uT = h->mixed ? (T*)h->uT : (T*)u;
    if (h->mixed) {
        CK((launch_convert<double, T>(u, uT, n, s)));
        h->launches += 1;
    }
    jfnk_status st;
    if (h->mixed) {
        // f = 2u^n/dt + F(u^n) and the first residual R(u^n) = -2 F(u^n) in one float64 pass
        kt_begin(h, JFNK_KF_RESIDUAL);
        CK(launch_stencil<double>(MODE_RHSRES, G, h->un, nullptr, nullptr, nullptr, h->f, h->R, h->part,
                                  h->ctl, 0, s));
        kt_end(h, JFNK_KF_RESIDUAL, (double)n * 8.0 * 3.0);
        h->launches += 1;
        st = read_ctl(h);
    } else {
        CK(launch_stencil<double>(MODE_RHS, G, h->un, nullptr, nullptr, nullptr, h->f, nullptr, h->part,
                                  h->ctl, 0, s));
        h->launches += 1;
        st = residual_eval<T>(h, u);
    }
    if (st != JFNK_OK) return st;
    if (h->hctl->nan) return JFNK_ERR_NAN;
    const double r0 = sqrt(h->hctl->res2);
    const double tol = fmax(h->opts.newton_rtol * r0,
                            h->opts.newton_atol_factor * G.two_over_dt * sqrt(h->hctl->unorm2));
    stats.res0 = r0;
    stats.tol = tol;
    stats.res_hist[0] = r0;
    double res = r0;
    int k = 0;
    const bool capture = sizeof(T) == sizeof(float) && capturing(h, JFNK_PAIRS_NEWTON | JFNK_PAIRS_ARNOLDI);
    while (res > tol && k < h->opts.max_newton) {
        if (h->opts.precond != JFNK_PC_NONE || capture) {
            if (G.smag) {
                CK(launch_eddy<T>(G, uT, (T*)h->nu, h->part, h->ctl, s));
                h->launches += 1;
            }
            CK(launch_pc_setup(G, h->opts.pc_sweeps, h->ctl, s));
            h->launches += 1;
        }
        const bool left = h->opts.precond == JFNK_PC_NONLINEAR;
        CK(launch_cycle_init<T>(G, h->R, (T*)h->V, h->x, n, h->opts.eta, h->m,
                                h->opts.precond == JFNK_PC_NONE || left, h->ctl, s));
        h->launches += 1;
        if (left) {
            st = left_cycle_start<T>(h, 1);
            if (st != JFNK_OK) return st;
        }
        int it = 0, rs = 0, cv = 0, sw = 0;
        st = gmres_solve<T>(h, uT, &it, &rs, &cv, &sw);
        if (st != JFNK_OK) return st;
        stats.pc_switches += sw;
        stats.gmres_per_newton[k] = it;
        stats.gmres_iters += it;
        stats.restarts += rs;
        if constexpr (sizeof(T) == sizeof(float)) {
            if (cv && capturing(h, JFNK_PAIRS_NEWTON)) {   // training pair of this correction
                CK(launch_pair_newton(G, h->R, (float*)h->tA, n, h->ctl, s));
                CK(launch_precond<float>(G, h->opts.pc_sweeps, (const float*)h->tA, (float*)h->tB, (float*)h->za,
                                         (float*)h->zb, (float*)h->da, (float*)h->db, (const float*)h->nu, h->part,
                                         h->ctl, 0, s, &h->launches));
                CK(launch_pair_store<double>((const float*)h->tA, h->x, (const float*)h->tB, h->capX, h->capT, n,
                                             h->cap_cap, 0, h->ctl, s));
                h->launches += 3;
            }
        }
        CK(launch_newton_update<T>(G, u, h->x, h->mixed ? uT : nullptr, n, s));
        h->launches += 1;
        st = residual_eval<T>(h, u);
        if (st != JFNK_OK) return st;
        if (h->hctl->nan) return JFNK_ERR_NAN;
        res = sqrt(h->hctl->res2);
        ++k;
        stats.res_hist[k] = res;
    }
    stats.newton_iters = k;
    stats.res_final = res;
    stats.converged = res <= tol;
    if (out) *out = stats;
    return stats.converged ? JFNK_OK : JFNK_ERR_NOT_CONVERGED;
}

extern "C" jfnk_status jfnk_step(jfnk_handle* h, double* u, jfnk_stats* out) {
    if (!h || !u) return JFNK_ERR_INVALID_ARG;
    if (!h->mixed) return step_impl<double>(h, u, out);
    jfnk_status st = step_impl<float>(h, u, out);
    if (h->opts.precond == JFNK_PC_UNET && h->net &&
        (st == JFNK_ERR_NOT_CONVERGED || st == JFNK_ERR_BREAKDOWN || st == JFNK_ERR_NAN)) {
        // the learned preconditioner failed: redo the step from u^n with the block one
        CK(cudaMemcpyAsync(u, h->un, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        h->opts.precond = JFNK_PC_BLOCK;
        st = step_impl<float>(h, u, out);
        h->opts.precond = JFNK_PC_UNET;
        if (out) out->pc_fallback = 1;
    }
    return st;
}

// ------------------------------------------------- learned preconditioner
extern "C" jfnk_status jfnk_unet_init(jfnk_handle* h, unsigned long long seed) {
    if (!h) return JFNK_ERR_INVALID_ARG;
    if (!unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    CK(cudaStreamSynchronize(h->stream));
    if (h->net) {
        unet_destroy(h->net);
        h->net = nullptr;
    }
    // balanced units: the linearised acoustic and buoyancy couplings become skew-adjoint
    const double su = h->opts.scale_u;
    // (velocity components 1, theta factor, p factor)
    const int nf = h->G.dim == 2 ? 4 : 5;
    double bal[5] = {1.0, 1.0, 1.0, 1.0, 1.0};
    if (h->strat.beta != 0.0 && h->strat.g > 0.0)
        bal[nf - 2] = h->opts.scale_theta / (su * sqrt(fabs(h->strat.beta) * h->strat.theta0 / h->strat.g));
    if (h->strat.gamma_p * h->strat.pbar > 0.0)
        bal[nf - 1] = h->opts.scale_p / (su * sqrt(h->strat.gamma_p * h->strat.pbar / h->strat.theta0));
    cudaError_t e = cudaSuccess;
    h->net = unet_create(h->G.dim, h->grid.nx, h->G.ny, h->grid.nz, bal, seed, &e);
    if (!h->net) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? JFNK_ERR_OOM : JFNK_ERR_CUDA;
    }
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_num_weights(jfnk_handle* h, size_t* count) {
    if (!h || !count) return JFNK_ERR_INVALID_ARG;
    if (!unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    if (!h->net) return JFNK_ERR_INVALID_ARG;
    *count = unet_num_weights(h->net);
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_get_weights(jfnk_handle* h, float* host, size_t count) {
    if (!h || !host) return JFNK_ERR_INVALID_ARG;
    if (!unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    if (!h->net || count != unet_num_weights(h->net)) return JFNK_ERR_INVALID_ARG;
    CK(unet_get_weights(h->net, host, h->stream));
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_set_weights(jfnk_handle* h, const float* host, size_t count) {
    if (!h || !host) return JFNK_ERR_INVALID_ARG;
    if (!unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    if (!h->net || count != unet_num_weights(h->net)) return JFNK_ERR_INVALID_ARG;
    for (size_t i = 0; i < count; ++i)
        if (!isfinite(host[i])) return JFNK_ERR_INVALID_ARG;
    CK(unet_set_weights(h->net, host, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_capture(jfnk_handle* h, int capacity, int kinds) {
    if (!h || capacity < 0 || (kinds & ~(JFNK_PAIRS_NEWTON | JFNK_PAIRS_ARNOLDI)) != 0) return JFNK_ERR_INVALID_ARG;
    if (!unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    CK(cudaStreamSynchronize(h->stream));
    if (h->capX) cudaFree(h->capX);
    if (h->capT) cudaFree(h->capT);
    h->capX = h->capT = nullptr;
    h->cap_cap = 0;
    h->cap_kinds = 0;
    const int zero = 0;
    CK(cudaMemcpy(&h->ctl->ncap, &zero, sizeof(int), cudaMemcpyHostToDevice));
    h->hctl->ncap = 0;
    if (capacity == 0 || kinds == 0) return JFNK_OK;
    const size_t bytes = (size_t)capacity * h->n * sizeof(float);
    if (cudaMalloc((void**)&h->capX, bytes) != cudaSuccess || cudaMalloc((void**)&h->capT, bytes) != cudaSuccess) {
        cudaGetLastError();
        if (h->capX) cudaFree(h->capX);
        h->capX = nullptr;
        return JFNK_ERR_OOM;
    }
    h->cap_cap = capacity;
    h->cap_kinds = kinds;
    return JFNK_OK;
}

static jfnk_status pair_count(jfnk_handle* h, int* count) {
    int c = 0;
    CK(cudaMemcpyAsync(&c, &h->ctl->ncap, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    *count = std::min(c, h->cap_cap);
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_pair_count(jfnk_handle* h, int* count) {
    if (!h || !count) return JFNK_ERR_INVALID_ARG;
    return pair_count(h, count);
}

extern "C" jfnk_status jfnk_unet_get_pair(jfnk_handle* h, int i, float* X, float* T) {
    if (!h || !X || !T || i < 0) return JFNK_ERR_INVALID_ARG;
    int c = 0;
    jfnk_status st = pair_count(h, &c);
    if (st != JFNK_OK) return st;
    if (i >= c) return JFNK_ERR_INVALID_ARG;
    const size_t bytes = h->n * sizeof(float);
    CK(cudaMemcpyAsync(X, h->capX + (size_t)i * h->n, bytes, cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaMemcpyAsync(T, h->capT + (size_t)i * h->n, bytes, cudaMemcpyDeviceToDevice, h->stream));
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_train(jfnk_handle* h, int epochs, float lr, double* loss_hist) {
    if (!h || epochs < 0 || !(lr > 0.0f) || !isfinite(lr)) return JFNK_ERR_INVALID_ARG;
    if (!unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    int c = 0;
    jfnk_status st = pair_count(h, &c);
    if (st != JFNK_OK) return st;
    if (!h->net || c < 1) return JFNK_ERR_INVALID_ARG;
    const cudaError_t e = unet_train(h->net, h->capX, h->capT, c, epochs, lr, loss_hist, h->stream);
    if (e == cudaErrorLaunchTimeout) return JFNK_ERR_TIMEOUT;
    CK(e);
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_forward(jfnk_handle* h, const float* x, float* y) {
    if (!h || !x || !y) return JFNK_ERR_INVALID_ARG;
    if (!unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    if (!h->net) return JFNK_ERR_INVALID_ARG;
    CK(unet_apply(h->net, x, y, 0, nullptr, h->stream));
    h->launches += unet_launches_per_apply();
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_loss_grad(jfnk_handle* h, const float* x, const float* t, double* loss,
                                           float* grads) {
    if (!h || !x || !t || !loss) return JFNK_ERR_INVALID_ARG;
    if (!unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    if (!h->net) return JFNK_ERR_INVALID_ARG;
    const cudaError_t e = unet_loss_grad(h->net, x, t, loss, grads, h->stream);
    if (e == cudaErrorLaunchTimeout) return JFNK_ERR_TIMEOUT;
    CK(e);
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_set_engine(jfnk_handle* h, int engine) {
    if (!h || (engine != JFNK_UNET_TCGEN05 && engine != JFNK_UNET_MMA_SYNC)) return JFNK_ERR_INVALID_ARG;
    if (!unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    if (!h->net) return JFNK_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(h->stream));
    CK(unet_set_engine(h->net, engine));
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_unet_status(jfnk_handle* h) {
    if (!h) return JFNK_ERR_INVALID_ARG;
    if (!h->net) return JFNK_OK;
    const cudaError_t e = unet_check(h->net, h->stream);
    if (e == cudaErrorLaunchTimeout) return JFNK_ERR_TIMEOUT;
    CK(e);
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_set_precond(jfnk_handle* h, int precond) {
    if (!h) return JFNK_ERR_INVALID_ARG;
    if (precond != JFNK_PC_NONE && precond != JFNK_PC_BLOCK && precond != JFNK_PC_UNET &&
        precond != JFNK_PC_SCHUR && precond != JFNK_PC_NONLINEAR)
        return JFNK_ERR_INVALID_ARG;
    if (precond == JFNK_PC_UNET && !unet_supported(h)) return JFNK_ERR_UNSUPPORTED;
    if (precond == JFNK_PC_SCHUR && h->opts.pc_sweeps < 2) return JFNK_ERR_UNSUPPORTED;
    const size_t eT = h->mixed ? sizeof(float) : sizeof(double);
    if (precond != JFNK_PC_NONE && !h->Z) {
        CK(cudaStreamSynchronize(h->stream));
        if (cudaMalloc(&h->Z, (size_t)h->m * h->ld * eT) != cudaSuccess) {
            cudaGetLastError();
            h->Z = nullptr;
            return JFNK_ERR_OOM;
        }
    }
    // the right-preconditioned cycle keeps w'_{j-1} and w_j in two buffers
    if (precond != JFNK_PC_NONE && precond != JFNK_PC_NONLINEAR && !h->w2) {
        CK(cudaStreamSynchronize(h->stream));
        if (cudaMalloc(&h->w2, h->ld * eT) != cudaSuccess) {
            cudaGetLastError();
            h->w2 = nullptr;
            return JFNK_ERR_OOM;
        }
    }
    h->opts.precond = precond;
    h->G.pc_schur = precond == JFNK_PC_SCHUR;
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_step_host(jfnk_handle* h, double* u_host, jfnk_stats* out) {
    if (!h || !u_host) return JFNK_ERR_INVALID_ARG;
    const size_t bytes = h->n * sizeof(double);
    CK(cudaMemcpyAsync(h->udev, u_host, bytes, cudaMemcpyHostToDevice, h->stream));
    jfnk_status st = jfnk_step(h, h->udev, out);
    if (st != JFNK_OK && st != JFNK_ERR_NOT_CONVERGED) return st;
    CK(cudaMemcpyAsync(u_host, h->udev, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return st;
}

extern "C" jfnk_status jfnk_budgets(jfnk_handle* h, const double* u, jfnk_budget* out) {
    if (!h || !u || !out) return JFNK_ERR_INVALID_ARG;
    const double dx = h->grid.lx / h->grid.nx, dz = h->grid.lz / h->grid.nz;
    CK(launch_budgets(h->G, u, dx, dz, h->grid.lz, h->part, h->ctl, h->budg, h->stream));   // 3-D: dV includes dy
    h->launches += 1;
    double b[14];
    const int nf = h->G.nf;
    CK(cudaMemcpyAsync(b, h->budg, (4 + 2 * nf) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    memset(out, 0, sizeof(*out));
    out->E_k = b[0];
    out->E_p = b[1];
    out->sum_theta = b[2];
    out->sum_div = b[3];
    for (int f = 0; f < nf; ++f) {
        out->max[f] = b[4 + f];
        out->min[f] = b[4 + nf + f];
    }
    return JFNK_OK;
}

extern "C" const char* jfnk_status_str(jfnk_status s) {
    switch (s) {
        case JFNK_OK: return "ok";
        case JFNK_ERR_INVALID_ARG: return "invalid argument";
        case JFNK_ERR_CUDA: return "CUDA runtime error";
        case JFNK_ERR_OOM: return "device memory allocation failed";
        case JFNK_ERR_NOT_CONVERGED: return "Newton iteration did not converge";
        case JFNK_ERR_BREAKDOWN: return "GMRES breakdown";
        case JFNK_ERR_NAN: return "non-finite residual";
        case JFNK_ERR_TIMEOUT: return "device loop iteration cap reached";
        case JFNK_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}
