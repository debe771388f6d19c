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

// Launch-bound occupancy target of the persistent kernel (blocks of 256
// per SM: 3 caps it at 80 registers a thread, with under 100 bytes of
// spills) and whether the node variants are out-of-line functions.  Measured
// on the 48-cavity workload over 100 steps (before the dynamic tile
// distribution): 3 blocks 14.5 k MLUPS, 2 blocks (up to 128 registers, no
// spills) 13.3 k.
#ifndef LBM_ENS_MINB
#define LBM_ENS_MINB 3
#endif
#ifndef LBM_ENS_NOINLINE
#define LBM_ENS_NOINLINE 0
#endif
#if LBM_ENS_NOINLINE
#define ENS_FN __device__ __noinline__
#else
#define ENS_FN __device__ __forceinline__
#endif

namespace lbm {

struct CavDesc {
    KP p;
    int face, cur0, inflight0;
    int bxs, by, gx, gxy;         // tile: 1 << bxs by by threads; tiles per row and per plane
    void *F, *G;
    int *js[2], *nb[2];
    double *s[2];
    float *gpost, *thw, *thw_rd0;
    int *status;
    int *jmax;                    // running maximum of the liquid counts (kept by phase 2)
    int cut;                      // nodes at heights >= *jmax + 3 are deep solid (Tc == Tm)
};

// Everything the launch needs, passed as one __grid_constant__ kernel
// parameter: the descriptors are read through the constant bank (uniform
// per block, no aliasing with the distributions being written).
constexpr int kMaxCavities = 64;
struct EnsWork {
    int ncav;
    int nodes_per_item;
    long long item_begin[kMaxCavities + 1];  // prefix sums of node items
    long long col_begin[kMaxCavities + 1];   // prefix sums of column items
    CavDesc desc[kMaxCavities];
    unsigned int *bar;            // {arrived, generation, timed out, -, item counters (2 x u64)}
    long long max_spins;
    int skip_arrival_block;       // fault injection for tests: this block never arrives (-1: none)
};

// Grid-wide barrier with a bounded wait.  Returns false once any block has
// given up (then every block leaves the launch).
__device__ __forceinline__ bool grid_barrier(const EnsWork &w, unsigned int nblocks) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vb = w.bar;
        if (vb[2]) {
            ok = 0;
        } else if ((int)blockIdx.x == w.skip_arrival_block) {
            // injected fault: this block does not arrive; it waits like the
            // others so that every block leaves through the timeout
            long long spins = 0;
            while (!vb[2] && ++spins <= w.max_spins) __nanosleep(256);
            atomicExch(w.bar + 2, 1u);
            ok = 0;
        } else {
            const unsigned int gen = vb[1];
            __threadfence();
            const unsigned int arrived = atomicAdd(w.bar, 1u) + 1u;
            if (arrived == nblocks) {
                atomicExch(w.bar, 0u);
                __threadfence();
                atomicAdd(w.bar + 1, 1u);
            } else {
                long long spins = 0;
                while (vb[1] == gen) {
                    if (vb[2] || ++spins > w.max_spins) {
                        atomicExch(w.bar + 2, 1u);
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
        }
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ int find_cavity(const long long *begin, int n, long long item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One node of phase 1.  Each (face, parity) variant is its own out-of-line
// function so that the variants do not share one register allocation.
template <typename ST, int FACE>
ENS_FN void ens_even(const CavDesc &d, int cur, int x, int y, int z) {
    even_node<ST, FACE>(d.p, (ST *)d.F, (ST *)d.G, d.js[cur], d.nb[cur], d.gpost, x, y, z);
}
template <typename ST, int FACE>
ENS_FN void ens_odd(const CavDesc &d, int cur, const float *trd, int x, int y, int z) {
    odd_node<ST, FACE, false>(d.p, nullptr, (ST *)d.F, (ST *)d.G, d.js[cur], d.nb[cur], d.gpost, trd, d.thw, x, y, z);
}

// One column of phase 2 (front update; returns the new liquid count) or 3
// (flip; returns -1).
template <typename ST>
ENS_FN int ens_column(const CavDesc &d, int cur, int inflight, int phase, int col) {
    if (phase == 2) {
        const ST *F = (const ST *)d.F, *G = (const ST *)d.G;
        if (d.face == 0)
            return front_column<ST, 0, false>(d.p, F, G, d.js[cur], d.js[1 - cur], d.s[cur], d.s[1 - cur], d.gpost, d.thw,
                                       inflight, 1, d.status, col);
        return front_column<ST, 1, false>(d.p, F, G, d.js[cur], d.js[1 - cur], d.s[cur], d.s[1 - cur], d.gpost, d.thw,
                                   inflight, 1, d.status, col);
    } else {
        ST *F = (ST *)d.F;
        if (d.face == 0) flip_column<ST, 0>(d.p, F, d.js[cur], d.js[1 - cur], d.nb[1 - cur], inflight, 1, col);
        else flip_column<ST, 1>(d.p, F, d.js[cur], d.js[1 - cur], d.nb[1 - cur], inflight, 1, col);
        return -1;
    }
}

template <typename ST, int K>
__global__ void __launch_bounds__(256, LBM_ENS_MINB) k_ensemble(const __grid_constant__ EnsWork w, int nsteps) {
    const long long items1 = w.item_begin[w.ncav], items2 = w.col_begin[w.ncav];
    __shared__ int top[kMaxCavities];  // per cavity: first height at which every node is deep solid
    __shared__ long long next;         // first item of the block's next chunk
    // per-step item counters (alternating), zeroed with the barrier words
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(w.bar + 4);
    constexpr int kChunk = 1;  // measured: 1, 2, 4 items -> 19.3, 18.7, 18.5 k MLUPS
    for (int t = 0; t < nsteps; ++t) {
        for (int k = threadIdx.x; k < w.ncav; k += blockDim.x) {
            const CavDesc &d = w.desc[k];
            top[k] = d.cut ? *(volatile int *)d.jmax + 3 : 1 << 30;
        }
        if (threadIdx.x == 0) next = (long long)atomicAdd(ctr + (t & 1), (unsigned long long)kChunk);
        __syncthreads();
        // phase 1: fused stream-collide of every node of every cavity; an
        // item is one (1 << bxs) x by tile of K consecutive z-planes; tiles
        // wholly above the liquid (deep solid) are skipped.  Blocks take
        // chunks of kChunk items from the step's counter (tiles differ in
        // work: deep-solid ones are skipped), asking for the next chunk
        // before working on the current one.
        for (long long base = next; base < items1; base = next) {
            __syncthreads();  // every thread has read `next`
            if (threadIdx.x == 0) next = (long long)atomicAdd(ctr + (t & 1), (unsigned long long)kChunk);
            const long long stop = base + kChunk < items1 ? base + kChunk : items1;
            for (long long it = base; it < stop; ++it) {
            const int k = find_cavity(w.item_begin, w.ncav, it);
            const CavDesc &d = w.desc[k];
            const int li = (int)(it - w.item_begin[k]);
            const int zc = li / d.gxy, r = li - zc * d.gxy;
            const int iy = r / d.gx, ix = r - iy * d.gx;
            if ((d.face == 0 ? iy * d.by : zc * K) >= top[k]) continue;
            const int cur = d.cur0 ^ (t & 1), odd = d.inflight0 ^ (t & 1);
            const float *trd = t == 0 ? d.thw_rd0 : d.thw;
            const int x = (ix << d.bxs) + (threadIdx.x & ((1 << d.bxs) - 1));
            const int y = iy * d.by + (threadIdx.x >> d.bxs);
            if (x >= d.p.nx || y >= d.p.ny) continue;
#pragma unroll 1
            for (int j = 0; j < K; ++j) {
                const int z = zc * K + j;
                if (z >= d.p.nz) break;
                if (d.face == 0) {
                    if (odd) ens_odd<ST, 0>(d, cur, trd, x, y, z);
                    else ens_even<ST, 0>(d, cur, x, y, z);
                } else {
                    if (odd) ens_odd<ST, 1>(d, cur, trd, x, y, z);
                    else ens_even<ST, 1>(d, cur, x, y, z);
                }
            }
            }
            __syncthreads();  // `next` holds the following chunk
        }
        // the other counter serves the next step; it was last used by the
        // step before, which every block has left
        if (blockIdx.x == 0 && threadIdx.x == 0) ctr[(t + 1) & 1] = 0ull;
        if (!grid_barrier(w, gridDim.x)) return;
        // phases 2 and 3: front update (Eq. 6), then flip, of every column
        for (int phase = 2; phase <= 3; ++phase) {
            for (long long it = blockIdx.x; it < items2; it += gridDim.x) {
                const int k = find_cavity(w.col_begin, w.ncav, it);
                const CavDesc &d = w.desc[k];
                const int cur = d.cur0 ^ (t & 1), inflight = 1 - (d.inflight0 ^ (t & 1));
                const int col = (int)((it - w.col_begin[k]) * blockDim.x + threadIdx.x);
                const int jn = col < d.p.ncols ? ens_column<ST>(d, cur, inflight, phase, col) : -1;
                if (phase == 2) {  // an item is one cavity's columns: whole warps
                    const int m = __reduce_max_sync(0xffffffffu, jn);
                    if ((threadIdx.x & 31) == 0 && m >= 0) atomicMax(d.jmax, m);
                }
            }
            if (!grid_barrier(w, gridDim.x)) return;
        }
    }
}

}  // namespace lbm

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
        if (K == 1) return (const void *)lbm::k_ensemble<__half, 1>;
        if (K == 2) return (const void *)lbm::k_ensemble<__half, 2>;
        return (const void *)lbm::k_ensemble<__half, 4>;
    }
    if (K == 1) return (const void *)lbm::k_ensemble<float, 1>;
    if (K == 2) return (const void *)lbm::k_ensemble<float, 2>;
    return (const void *)lbm::k_ensemble<float, 4>;
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
        if (n > 0) h->thw_pending = 0;
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
        e->cav.push_back(h);
        if (k == 0) e->precision = h->precision;
        else if (h->precision != e->precision) return fail(LBM_EINVAL);
    }
    if (cudaMalloc(&e->bar_dev, 8 * sizeof(unsigned int)) != cudaSuccess) return fail(LBM_ENOMEM);
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
    if (nodes_per_thread != 1 && nodes_per_thread != 2 && nodes_per_thread != 4)
        return ens_err(e, LBM_EINVAL, "nodes_per_thread must be 1, 2 or 4");
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
