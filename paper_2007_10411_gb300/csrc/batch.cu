// Batched solver: many independent grids (e.g. heat-island instances of
// uneven sizes and surface fluxes) stepped together on one GPU.
//
// Every instance owns a handle and a non-blocking stream; jfnk_step_batch runs
// the instances' Newton / GMRES sequences concurrently from a pool of host
// threads (one per instance), so the GPU overlaps their kernels -- small
// grids alone cannot fill 152 SMs.  The caller's stream is forked into the
// instance streams before the step and joined after it, so the batch step is
// ordered on the caller's stream like any other call.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <thread>
#include <vector>

#include "../../include/jfnk.h"

struct jfnk_batch {
    int n;
    cudaStream_t parent;
    cudaEvent_t fork;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    std::vector<jfnk_handle*> h;
};

static void destroy_parts(jfnk_batch* b) {
    for (jfnk_handle* h : b->h)
        if (h) jfnk_destroy(h);
    for (cudaStream_t s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->joins)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
}

extern "C" jfnk_status jfnk_create_batch(int n, const jfnk_grid* grids, const jfnk_strat* strats,
                                         const jfnk_sgs* sgs, const jfnk_opts* opts, void* cuda_stream,
                                         jfnk_batch** out) {
    if (!out) return JFNK_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 1 || n > JFNK_MAX_BATCH || !grids || !strats || !sgs || !opts) return JFNK_ERR_INVALID_ARG;
    jfnk_batch* b = new (std::nothrow) jfnk_batch;
    if (!b) return JFNK_ERR_OOM;
    b->n = n;
    b->parent = (cudaStream_t)cuda_stream;
    b->fork = nullptr;
    b->streams.assign(n, nullptr);
    b->joins.assign(n, nullptr);
    b->h.assign(n, nullptr);
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        destroy_parts(b);
        delete b;
        return JFNK_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i) {
        if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming) != cudaSuccess) {
            destroy_parts(b);
            delete b;
            return JFNK_ERR_CUDA;
        }
        const jfnk_status st = jfnk_create(&grids[i], &strats[i], &sgs[i], &opts[i], b->streams[i], &b->h[i]);
        if (st != JFNK_OK) {
            destroy_parts(b);
            delete b;
            return st;
        }
        // Concurrent instances keep the GPU busy between one instance's launches,
        // and graph segments would run Krylov steps past a cycle's end that take
        // time from the other instances: stream launches by default.
        jfnk_set_cycle_graph(b->h[i], 0);
    }
    *out = b;
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_destroy_batch(jfnk_batch* b) {
    if (!b) return JFNK_OK;
    destroy_parts(b);
    delete b;
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_batch_handle(jfnk_batch* b, int i, jfnk_handle** out) {
    if (!b || !out || i < 0 || i >= b->n) return JFNK_ERR_INVALID_ARG;
    *out = b->h[i];
    return JFNK_OK;
}

extern "C" jfnk_status jfnk_step_batch(jfnk_batch* b, double* const* u, jfnk_stats* stats,
                                       jfnk_status* status) {
    if (!b || !u) return JFNK_ERR_INVALID_ARG;
    for (int i = 0; i < b->n; ++i)
        if (!u[i]) return JFNK_ERR_INVALID_ARG;
    if (cudaEventRecord(b->fork, b->parent) != cudaSuccess) return JFNK_ERR_CUDA;
    for (int i = 0; i < b->n; ++i)
        if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) return JFNK_ERR_CUDA;
    std::vector<jfnk_status> st(b->n, JFNK_OK);
    std::vector<jfnk_stats> sv(b->n);
    {
        std::vector<std::thread> pool;
        pool.reserve(b->n);
        for (int i = 0; i < b->n; ++i)
            pool.emplace_back([&, i]() { st[i] = jfnk_step(b->h[i], u[i], &sv[i]); });
        for (std::thread& t : pool) t.join();
    }
    for (int i = 0; i < b->n; ++i) {
        if (cudaEventRecord(b->joins[i], b->streams[i]) != cudaSuccess ||
            cudaStreamWaitEvent(b->parent, b->joins[i], 0) != cudaSuccess)
            return JFNK_ERR_CUDA;
    }
    jfnk_status worst = JFNK_OK;
    for (int i = 0; i < b->n; ++i) {
        if (stats) stats[i] = sv[i];
        if (status) status[i] = st[i];
        if (st[i] != JFNK_OK && (worst == JFNK_OK || worst == JFNK_ERR_NOT_CONVERGED)) worst = st[i];
    }
    return worst;
}
