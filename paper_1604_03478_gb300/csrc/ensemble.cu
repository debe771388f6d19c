// ensemble.cu -- a batch of independent cavities of uneven sizes and
// parameters advanced by ONE persistent kernel launch (the batched form of
// the melting step of Li, Yang & Zhang, arXiv:1604.03478, section 2).
//
// The launch walks a work list: per step, phase 1 covers every node of every
// cavity in items of (block size x nodes per thread) nodes, handed out one
// by one from an atomic counter (fused stream-collide, Eqs. 1-5), phase 2
// every column of every cavity in
// items of one block (front update, Eq. 6), phase 3 the same columns (phase
// flip).  Phases are separated by a grid-wide barrier; the launch is
// cooperative (all blocks resident) and every barrier wait is bounded: a
// block that waits too long raises an error flag and the whole launch
// returns, which the host reports as LBM_ETIMEOUT.  The launch (with the
// barrier reset) is captured once in a CUDA graph and replayed.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/lbm_melt.h"
#include "handle.h"
#include "kernels.cuh"
#include "launch.h"

#define LBM_API extern "C" __attribute__((visibility("default")))

#include "ensemble_kernel.cuh"

using lbm::CavDesc;
using lbm::EnsWork;

struct lbm_ensemble {
    int n;
    std::vector<lbm_melt *> cav;
    cudaStream_t user;    // the caller's stream (ordering only)
    cudaStream_t stream;  // own non-blocking stream: capturable, unlike the legacy default stream
    cudaEvent_t ev_in, ev_out;
    int precision;
    int block, K, grid;
    long long max_spins;
    unsigned int *bar_dev;
    long long items[lbm::kMaxCavities + 1], cols[lbm::kMaxCavities + 1];
    std::vector<CavDesc> desc;
    cudaGraphExec_t graph;
    int graph_steps;
    long long steps;
    char err[512];
};

namespace {

lbm_status ens_err(lbm_ensemble *e, lbm_status st, const char *fmt, ...) {
    if (e) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(e->err, sizeof e->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

#define ECK(call, where)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return ens_err(e, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", \
                           where, cudaGetErrorString(e_));                                       \
    } while (0)

const void *kernel_ptr(int precision, int K) {
    if (precision == 1) {
        if (K == 1) return lbm::ens_kernel_f16_k1();
        if (K == 2) return lbm::ens_kernel_f16_k2();
        if (K == 4) return lbm::ens_kernel_f16_k4();
        return lbm::ens_kernel_f16_k8();
    }
    if (K == 1) return lbm::ens_kernel_f32_k1();
    if (K == 2) return lbm::ens_kernel_f32_k2();
    if (K == 4) return lbm::ens_kernel_f32_k4();
    return lbm::ens_kernel_f32_k8();
}

// Tile of a cavity for the block size: a power of two from 32 to 128 wide
// along x, the one that leaves the fewest idle lanes over a row
// (block_width), the rest of the block along y.
void tile(const lbm::KP &p, int block, int &bxs, int &by) {
    const int bx = lbm::block_width(p.nx, block);
    bxs = 0;
    while ((1 << bxs) < bx) ++bxs;
    by = block / bx;
}

void fill_desc(lbm_melt *h, CavDesc &d, int block) {
    std::memset(&d, 0, sizeof d);
    tile(h->kp, block, d.bxs, d.by);
    d.gx = (h->kp.nx + (1 << d.bxs) - 1) >> d.bxs;
    d.gxy = d.gx * ((h->kp.ny + d.by - 1) / d.by);
    d.p = h->kp;
    d.face = h->face;
    d.cur0 = h->cur;
    d.inflight0 = h->inflight;
    d.F = h->F;
    d.G = h->G;
    for (int k = 0; k < 2; ++k) { d.js[k] = h->js[k]; d.nb[k] = h->nb[k]; d.s[k] = h->s[k]; }
    d.gpost = h->gpost;
    d.thw = h->thw_cur;
    d.thw_rd0 = h->thw_pending ? h->thw_prev : h->thw_cur;
    d.status = h->status_dev;
    d.jmax = h->jmax_dev;
    d.cut = h->kp.skip_deep;
}

// Work-list prefix sums and the co-resident grid for the launch shape.
lbm_status plan(lbm_ensemble *e) {
    e->items[0] = e->cols[0] = 0;
    for (int k = 0; k < e->n; ++k) {
        const lbm::KP &p = e->cav[k]->kp;
        int bxs, by;
        tile(p, e->block, bxs, by);
        const long long gx = (p.nx + (1 << bxs) - 1) >> bxs, gy = (p.ny + by - 1) / by;
        const long long gz = (p.nz + e->K - 1) / e->K;
        e->items[k + 1] = e->items[k] + gx * gy * gz;
        e->cols[k + 1] = e->cols[k] + (p.ncols + e->block - 1) / e->block;
    }
    int dev = 0, sms = 0, per_sm = 0;
    ECK(cudaGetDevice(&dev), "device");
    ECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    ECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_ptr(e->precision, e->K), e->block, 0),
        "occupancy");
    if (per_sm < 1) return ens_err(e, LBM_EINVAL, "block size %d does not fit on an SM", e->block);
    e->grid = (int)std::min<long long>((long long)per_sm * sms, std::max(e->items[e->n], e->cols[e->n]));
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    return LBM_OK;
}

// Descriptors from the members' current phases; a change invalidates the
// captured graph (its kernel parameters hold the descriptors by value).
void refresh_desc(lbm_ensemble *e) {
    for (int k = 0; k < e->n; ++k) fill_desc(e->cav[k], e->desc[k], e->block);
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
}

lbm_status launch(lbm_ensemble *e, int nsteps, int skip_block) {
    EnsWork *w = new (std::nothrow) EnsWork();
    if (!w) return LBM_ENOMEM;
    w->ncav = e->n;
    w->nodes_per_item = e->block * e->K;
    for (int k = 0; k <= e->n; ++k) {
        w->item_begin[k] = e->items[k];
        w->col_begin[k] = e->cols[k];
    }
    for (int k = 0; k < e->n; ++k) w->desc[k] = e->desc[k];
    w->bar = e->bar_dev;
    w->max_spins = e->max_spins;
    w->skip_arrival_block = skip_block;
    void *args[] = {w, &nsteps};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(e->grid);
    cfg.blockDim = dim3(e->block);
    cfg.stream = e->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t err = cudaMemsetAsync(e->bar_dev, 0, 8 * sizeof(unsigned int), e->stream);
    if (err == cudaSuccess) err = cudaLaunchKernelExC(&cfg, kernel_ptr(e->precision, e->K), args);
    delete w;
    ECK(err, "ensemble launch");
    return LBM_OK;
}

void advance_handles(lbm_ensemble *e, long long n) {
    for (lbm_melt *h : e->cav) {
        h->steps += n;
        if (n & 1) { h->cur ^= 1; h->inflight ^= 1; }
        if (n > 0) { h->thw_pending = 0; h->thw_last_prev = 0; }
        h->exec_steps += n;  // the launch kept the running maximum: host read-backs stay bounds
    }
    e->steps += n;
}

bool desc_current(lbm_ensemble *e) {
    for (int k = 0; k < e->n; ++k) {
        const lbm_melt *h = e->cav[k];
        const CavDesc &d = e->desc[k];
        if (d.cur0 != h->cur || d.inflight0 != h->inflight ||
            d.thw_rd0 != (h->thw_pending ? h->thw_prev : h->thw_cur))
            return false;
    }
    return true;
}

}  // namespace

LBM_API lbm_status lbm_ensemble_create(int n, const lbm_melt_case *cases, void *cuda_stream, lbm_ensemble **out) {
    if (!out || n < 1 || n > lbm::kMaxCavities || !cases) return LBM_EINVAL;
    *out = nullptr;
    lbm_ensemble *e = new (std::nothrow) lbm_ensemble();
    if (!e) return LBM_ENOMEM;
    e->n = n;
    e->user = (cudaStream_t)cuda_stream;
    e->block = 128;
    e->K = 2;
    e->max_spins = 1LL << 24;  // with 64 ns sleeps: about a second
    e->graph_steps = 8;
    e->desc.resize(n);
    auto fail = [&](lbm_status st) {
        for (lbm_melt *h : e->cav) lbm_melt_destroy(h);
        cudaFree(e->bar_dev);
        if (e->ev_in) cudaEventDestroy(e->ev_in);
        if (e->ev_out) cudaEventDestroy(e->ev_out);
        if (e->stream) cudaStreamDestroy(e->stream);
        delete e;
        return st;
    };
    if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_out, cudaEventDisableTiming) != cudaSuccess)
        return fail(LBM_ECUDA);
    // members run on the ensemble's stream, after what the caller queued so far
    if (cudaEventRecord(e->ev_in, e->user) != cudaSuccess || cudaStreamWaitEvent(e->stream, e->ev_in, 0) != cudaSuccess)
        return fail(LBM_ECUDA);
    for (int k = 0; k < n; ++k) {
        const lbm_melt_case &c = cases[k];
        lbm_melt *h = nullptr;
        lbm_status st = lbm_melt_create(&c.grid, c.Ra, c.Pr, c.Ste, c.Th, c.Tc, c.Tm, &c.rates, (void *)e->stream, &h);
        if (st != LBM_OK) return fail(st);
        h->member = 1;
        e->cav.push_back(h);
        // the persistent kernel's even step indexes a member's state in 32 bits
        if (19LL * h->kp.ld >= (1LL << 32)) return fail(LBM_EINVAL);
        if (k == 0) e->precision = h->precision;
        else if (h->precision != e->precision) return fail(LBM_EINVAL);
    }
    // 8 barrier words, then the phase timers (4 x u64), zeroed here only
    if (cudaMalloc(&e->bar_dev, 16 * sizeof(unsigned int)) != cudaSuccess ||
        cudaMemset(e->bar_dev, 0, 16 * sizeof(unsigned int)) != cudaSuccess)
        return fail(LBM_ENOMEM);
    refresh_desc(e);
    if (plan(e) != LBM_OK) return fail(LBM_ECUDA);
    if (cudaStreamSynchronize(e->stream) != cudaSuccess) return fail(LBM_ECUDA);
    *out = e;
    return LBM_OK;
}

LBM_API void lbm_ensemble_destroy(lbm_ensemble *e) {
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    for (lbm_melt *h : e->cav) lbm_melt_destroy(h);
    cudaFree(e->bar_dev);
    cudaEventDestroy(e->ev_in);
    cudaEventDestroy(e->ev_out);
    cudaStreamDestroy(e->stream);
    delete e;
}

LBM_API const char *lbm_ensemble_last_error(const lbm_ensemble *e) { return e ? e->err : "null ensemble"; }

LBM_API lbm_status lbm_ensemble_set_launch(lbm_ensemble *e, int block, int nodes_per_thread, int graph_steps) {
    if (!e) return LBM_EINVAL;
    if (block != 64 && block != 128 && block != 256)
        return ens_err(e, LBM_EINVAL, "block must be 64, 128 or 256");
    if (nodes_per_thread != 1 && nodes_per_thread != 2 && nodes_per_thread != 4 && nodes_per_thread != 8)
        return ens_err(e, LBM_EINVAL, "nodes_per_thread must be 1, 2, 4 or 8");
    if (graph_steps < 2 || (graph_steps & 1)) return ens_err(e, LBM_EINVAL, "graph_steps must be even and >= 2");
    e->block = block;
    e->K = nodes_per_thread;
    e->graph_steps = graph_steps;
    refresh_desc(e);
    lbm_status st = plan(e);
    if (st == LBM_OK) ECK(cudaStreamSynchronize(e->stream), "synchronize");
    return st;
}

LBM_API lbm_status lbm_ensemble_set_barrier_timeout(lbm_ensemble *e, long long max_spins) {
    if (!e || max_spins < 1) return LBM_EINVAL;
    e->max_spins = max_spins;
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    return LBM_OK;
}

LBM_API lbm_status lbm_ensemble_step(lbm_ensemble *e, long long nsteps) {
    if (!e || nsteps < 0) return LBM_EINVAL;
    if (nsteps == 0) return LBM_OK;
    // stream order: after the caller's queued work, and the caller's later
    // work after this
    ECK(cudaEventRecord(e->ev_in, e->user), "event");
    ECK(cudaStreamWaitEvent(e->stream, e->ev_in, 0), "wait");
    if (!desc_current(e)) refresh_desc(e);
    long long left = nsteps;
    const long long G = e->graph_steps;
    if (left >= G) {
        if (!e->graph) {
            cudaGraph_t g;
            ECK(cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal), "capture");
            lbm_status st = launch(e, (int)G, -1);
            cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
            if (st != LBM_OK) return st;
            ECK(ce, "end capture");
            ce = cudaGraphInstantiate(&e->graph, g, 0);
            cudaGraphDestroy(g);
            ECK(ce, "instantiate");
        }
        // G is even: every replay starts from the same AA phase, so the
        // descriptors stay valid across replays
        while (left >= G) {
            ECK(cudaGraphLaunch(e->graph, e->stream), "graph launch");
            left -= G;
        }
    }
    if (left > 0) {
        lbm_status st = launch(e, (int)left, -1);
        if (st != LBM_OK) return st;
    }
    advance_handles(e, nsteps);
    if (left & 1) refresh_desc(e);  // the members' phases moved on
    ECK(cudaEventRecord(e->ev_out, e->stream), "event");
    ECK(cudaStreamWaitEvent(e->user, e->ev_out, 0), "wait");
    return LBM_OK;
}

// Test hook: one launch of one step in which block `block` never arrives at
// the first barrier; the bounded waits must end the launch with
// LBM_ETIMEOUT.  The ensemble's state is not meaningful afterwards.
LBM_API lbm_status lbm_ensemble_inject_barrier_fault(lbm_ensemble *e, int block) {
    if (!e || block < 0 || block >= e->grid) return LBM_EINVAL;
    if (!desc_current(e)) refresh_desc(e);
    lbm_status st = launch(e, 1, block);
    if (st != LBM_OK) return st;
    advance_handles(e, 1);
    refresh_desc(e);
    return LBM_OK;
}

LBM_API lbm_status lbm_ensemble_sync(lbm_ensemble *e) {
    if (!e) return LBM_EINVAL;
    unsigned int bar[3] = {0, 0, 0};
    ECK(cudaMemcpyAsync(bar, e->bar_dev, sizeof bar, cudaMemcpyDeviceToHost, e->stream), "barrier read");
    ECK(cudaStreamSynchronize(e->stream), "synchronize");
    if (bar[2]) return ens_err(e, LBM_ETIMEOUT, "a grid-barrier wait gave up (bounded spin exhausted)");
    for (int k = 0; k < e->n; ++k) {
        lbm_status st = lbm_melt_sync(e->cav[k]);
        if (st != LBM_OK) return ens_err(e, st, "cavity %d: %s", k, lbm_melt_last_error(e->cav[k]));
    }
    return LBM_OK;
}

LBM_API lbm_status lbm_ensemble_phase_times(lbm_ensemble *e, int reset, double *us_per_step, long long *steps) {
    if (!e) return LBM_EINVAL;
    unsigned long long acc[4] = {0, 0, 0, 0};
    ECK(cudaMemcpyAsync(acc, e->bar_dev + 8, sizeof acc, cudaMemcpyDeviceToHost, e->stream), "timer read");
    if (reset) ECK(cudaMemsetAsync(e->bar_dev + 8, 0, sizeof acc, e->stream), "timer reset");
    ECK(cudaStreamSynchronize(e->stream), "synchronize");
    if (us_per_step)
        for (int i = 0; i < 3; ++i) us_per_step[i] = acc[3] ? (double)acc[i] * 1e-3 / (double)acc[3] : 0.0;
    if (steps) *steps = (long long)acc[3];
    return LBM_OK;
}

LBM_API lbm_melt *lbm_ensemble_member(lbm_ensemble *e, int i) {
    if (!e || i < 0 || i >= e->n) return nullptr;
    return e->cav[i];
}

LBM_API lbm_status lbm_ensemble_info(lbm_ensemble *e, long long *n_nodes, int *grid, int *block, int *nodes_per_thread) {
    if (!e) return LBM_EINVAL;
    long long tot = 0;
    for (lbm_melt *h : e->cav) tot += h->kp.N;
    if (n_nodes) *n_nodes = tot;
    if (grid) *grid = e->grid;
    if (block) *block = e->block;
    if (nodes_per_thread) *nodes_per_thread = e->K;
    return LBM_OK;
}
