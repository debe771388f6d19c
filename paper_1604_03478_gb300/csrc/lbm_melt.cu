// lbm_melt.cu -- host side of the C ABI declared in include/lbm_melt.h:
// argument checking, the lattice parameters of section 1 / Eq. 7, the
// initial state, device memory, the per-step launch sequence and I/O.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/lbm_melt.h"
#include "handle.h"
#include "launch.h"

#define LBM_API extern "C" __attribute__((visibility("default")))

using lbm::Bufs;
using lbm::KP;

namespace {

const double CS2T = 0.25;  // D3Q7 pseudo sound speed squared (w0 = 1/4)
const int kRedBlocks = 608;  // partial blocks of the FP64 totals (4 per SM of a GB300)
// Step graphs: steps per replay, and the largest cavity that uses them by
// default (a 160^3 step takes about as long on the GPU as its three launches
// take the host; larger cavities are bound by the GPU).
const int kGraphSteps = 16;
const long long kGraphMaxNodes = 160LL * 160 * 160;



// Root of lambda exp(lambda^2) erf(lambda) = Ste / sqrt(pi) (the one-phase
// Neumann solution of conduction melting with zero subcooling, section 3.1),
// by bisection on [0, hi].
double neumann_lambda(double Ste) {
    if (!(Ste > 0.0)) return 0.0;
    const double rhs = Ste / std::sqrt(M_PI);
    double lo = 0.0, hi = 1.0;
    while (hi * std::exp(hi * hi) * std::erf(hi) < rhs) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid * std::exp(mid * mid) * std::erf(mid) < rhs) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// The two-phase Neumann solution of conduction melting against a solid
// initially at Tc < Tm (conductivity ratio kappa = k_s / k_l, equal rho c,
// so alpha_s = kappa alpha): the front is s = 2 lambda sqrt(alpha t), and the
// one-dimensional interface balance (Eq. 6 without slopes) gives
//   lambda sqrt(pi) / Ste = e^(-lambda^2) / erf(lambda)
//                           - theta sqrt(kappa) e^(-lambda^2 / kappa) / erfc(lambda / sqrt(kappa)),
// theta = (Tm - Tc) / (Th - Tm).  The left side grows and the right side
// falls with lambda: bisection.  theta = 0 is neumann_lambda's equation.
double neumann_lambda_two_phase(double Ste, double theta, double kappa) {
    if (!(Ste > 0.0) || !(kappa > 0.0)) return 0.0;
    const double rk = std::sqrt(kappa);
    auto excess = [&](double l) {  // left side minus right side
        return l * std::sqrt(M_PI) / Ste - std::exp(-l * l) / std::erf(l) +
               theta * rk * std::exp(-l * l / kappa) / std::erfc(l / rk);
    };
    double lo = 0.0, hi = 1.0;
    while (excess(hi) < 0.0) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (excess(mid) < 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

double pick(double v, double dflt) { return v > 0.0 ? v : dflt; }

lbm_status derive(const lbm_melt_grid *g, double Ra, double Pr, double Ste, double Th, double Tc, double Tm,
                  const lbm_melt_rates *r, Derived &d, char *err, size_t errlen) {
    auto fail = [&](const char *fmt, ...) {
        if (err && errlen) {
            va_list ap;
            va_start(ap, fmt);
            vsnprintf(err, errlen, fmt, ap);
            va_end(ap);
        }
        return LBM_EINVAL;
    };
    if (!g || !r) return fail("null grid or rates");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return fail("cavity edges must be >= 1");
    if (g->heated_face != 0 && g->heated_face != 1) return fail("heated_face must be 0 (y = 0) or 1 (z = 0)");
    if (g->precision != 0 && g->precision != 1) return fail("precision must be 0 (fp32) or 1 (fp16)");
    d.H = g->heated_face == 0 ? g->ny : g->nz;
    d.P1 = g->nx;
    d.P2 = g->heated_face == 0 ? g->nz : g->ny;
    if (d.H < 4) return fail("cavity length along the heating axis must be >= 4");
    if (d.H > 32767) return fail("cavity length along the heating axis must be <= 32767");
    d.N = (long long)g->nx * g->ny * g->nz;
    d.ncols = (long long)d.P1 * d.P2;
    if (d.N > (1LL << 31) - 1) return fail("too many nodes");
    if (!(Th > Tm)) return fail("Th must exceed Tm");
    if (!(Tc <= Tm)) return fail("Tc must not exceed Tm");
    if (!(Ste >= 0.0)) return fail("Ste must be >= 0");
    if (!(Ra >= 0.0)) return fail("Ra must be >= 0");
    if (r->derive_from_Ra) {
        if (!(Ra > 0.0)) return fail("derive_from_Ra needs Ra > 0");
        if (!(Pr > 0.0)) return fail("Pr must be > 0");
        if (!(g->Ma > 0.0 && g->Ma <= 0.3)) return fail("Ma must be in (0, 0.3]");
        const double U0 = g->Ma / std::sqrt(3.0);
        d.nu = U0 * d.H * std::sqrt(Pr / Ra);
        d.alpha = d.nu / Pr;
        d.s_nu = 1.0 / (3.0 * d.nu + 0.5);
        d.s_alpha = 1.0 / (d.alpha / CS2T + 0.5);
    } else {
        if (!(r->s_nu > 0.0 && r->s_nu < 2.0)) return fail("s_nu must be in (0, 2)");
        if (!(r->s_alpha > 0.0 && r->s_alpha < 2.0)) return fail("s_alpha must be in (0, 2)");
        d.s_nu = r->s_nu;
        d.s_alpha = r->s_alpha;
        d.nu = (1.0 / d.s_nu - 0.5) / 3.0;
        d.alpha = CS2T * (1.0 / d.s_alpha - 0.5);
    }
    if (!(3.0 * d.nu + 0.5 > 0.5 + 1e-4)) return fail("tau_nu = %.6g is too close to 1/2", 3.0 * d.nu + 0.5);
    if (!(d.s_alpha > 0.0 && d.s_alpha < 2.0)) return fail("s_alpha = %.6g outside (0, 2)", d.s_alpha);
    d.gbeta = Ra > 0.0 ? Ra * d.nu * d.alpha / ((Th - Tm) * std::pow((double)d.H, 3)) : 0.0;
    d.s_e = pick(r->s_e, 1.19);
    d.s_eps = pick(r->s_eps, 1.4);
    d.s_q = pick(r->s_q, 1.2);
    d.s_pi = pick(r->s_pi, 1.4);
    d.s_m = pick(r->s_m, 1.98);
    d.s_g4 = pick(r->s_g4, 1.0);
    d.s_g5 = pick(r->s_g5, 1.0);
    const double rs[7] = {d.s_e, d.s_eps, d.s_q, d.s_pi, d.s_m, d.s_g4, d.s_g5};
    for (double v : rs)
        if (!(v < 2.0)) return fail("relaxation rates must be below 2");
    d.s0 = g->s0 > 0.0 ? g->s0 : 1.0;
    if (!(d.s0 >= 0.5 && d.s0 <= d.H)) return fail("s0 must be in [0.5, H]");
    d.lambda = neumann_lambda(Ste);
    d.t0 = Ste > 0.0 ? d.s0 * d.s0 / (4.0 * d.lambda * d.lambda * d.alpha) : 0.0;
    return LBM_OK;
}

}  // namespace



namespace {

lbm_status set_err(lbm_melt *h, lbm_status st, const char *fmt, ...) {
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof h->err, fmt, ap);
        va_end(ap);
    }
    return st;
}

lbm_status cuda_err(lbm_melt *h, cudaError_t e, const char *where) {
    return set_err(h, e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", where,
                   cudaGetErrorString(e));
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_err(h, e_, where); \
    } while (0)

// Two nodes per thread in the stream-collide (an even nx): chosen for
// cavities above 160^3, whose grids are large enough to keep the GPU busy
// with half the threads (256^3: 0.2245 against 0.234 ms per launch in FP32,
// 0.145 against 0.19 ms in FP16); smaller cavities with a thin liquid layer
// are latency bound and run faster with one node per thread (96^3 adjoint
// forward 54 against 61 ms, 128^3 convection 33 against 35 us per step).
bool use_pairs(const lbm_melt *h) {
    if (h->kp.nx % 2 != 0) return false;
    return h->pairs_mode < 0 ? h->d.N > kGraphMaxNodes : h->pairs_mode == 1;
}

// Buffers of a step from phase (cur, inflight) with the handle's wall fields.
Bufs bufs_at(lbm_melt *h, int cur, int inflight) {
    Bufs b;
    b.F = h->F;
    b.G = h->G;
    b.js = h->js[cur];
    b.js_next = h->js[1 - cur];
    b.nb = h->nb[cur];
    b.nb_next = h->nb[1 - cur];
    b.s = h->s[cur];
    b.s_next = h->s[1 - cur];
    b.gpost = h->gpost;
    b.thw_rd = h->thw_pending ? h->thw_prev : h->thw_cur;
    b.thw_wr = h->thw_cur;
    b.status = h->status_dev;
    b.lk = &h->lk;
    b.cblk = h->cblk;
    b.jmax = h->jmax_dev;
    b.k1_height = h->kp.H;
    // the wall field of the last streaming: in flight, the one the pending
    // reads will apply; in the natural layout, the one the last odd step
    // wrote with, unless a new field has been set since
    b.thw_nu = inflight ? b.thw_rd : (h->thw_last_prev ? h->thw_prev : h->thw_cur);
    b.nu = h->nu_dev;
    b.nu_scale = (double)h->kp.H / (h->d.alpha * (h->Th - h->Tm));
    b.spost = h->spost;
    b.pairs = use_pairs(h) ? 1 : 0;
    return b;
}

Bufs bufs(lbm_melt *h) { return bufs_at(h, h->cur, h->inflight); }

#define LAUNCH(h, method, ...)                                                       \
    ((h)->precision == 1 ? lbm::Launch<__half>::method(__VA_ARGS__)                  \
                         : lbm::Launch<float>::method(__VA_ARGS__))

// Prepare js from s, its 3x3 bounds and the ghost nodes from the state
// (front held, no flip).
lbm_status refresh_front(lbm_melt *h) {
    Bufs b = bufs(h);
    CK(LAUNCH(h, front, h->kp, h->face, h->inflight, 0, b, h->stream), "front refresh");
    CK(LAUNCH(h, flip, h->kp, h->face, h->inflight, 0, b, h->stream), "neighbour bounds");
    h->cur ^= 1;
    return LBM_OK;
}

lbm_status copy_in(lbm_melt *h, void *dst, const void *src, size_t bytes, int ptr_kind) {
    CK(cudaMemcpyAsync(dst, src, bytes, ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream),
       "copy in");
    return LBM_OK;
}

lbm_status check_status(lbm_melt *h) {
    int st = 0;
    CK(cudaMemcpyAsync(&st, h->status_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "status read");
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    if (st & 2) return set_err(h, LBM_ENAN, "non-finite temperature at the front");
    if (st & 1) return set_err(h, LBM_EUNSTABLE, "the front moved more than half a cell in one step");
    return LBM_OK;
}

void free_all(lbm_melt *h) {
    cudaFree(h->F);
    cudaFree(h->G);
    for (int k = 0; k < 2; ++k) { cudaFree(h->js[k]); cudaFree(h->nb[k]); cudaFree(h->s[k]); }
    cudaFree(h->gpost);
    cudaFree(h->thw_cur);
    cudaFree(h->thw_prev);
    cudaFree(h->status_dev);
    cudaFree(h->sum_dev);
    cudaFree(h->ticket);
    cudaFree(h->red_part);
    cudaFree(h->totals_dev);
    cudaFree(h->nu_dev);
    cudaFree(h->report);
    cudaFree(h->jmax_dev);
    cudaFree(h->spost);
    if (h->rb_val) cudaFreeHost(h->rb_val);
    for (int k = 0; k < lbm_melt::kRbRing; ++k)
        if (h->rb_ev[k]) cudaEventDestroy(h->rb_ev[k]);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    for (auto &row : h->graphs)
        for (auto &g : row)
            if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
}

// Height bound of the next stream-collide grid (see lbm_melt::kRbLag): all
// heights while no valid read-back old enough exists, or when deep solid
// nodes are updated (Tc below Tm).
lbm_status k1_height(lbm_melt *h, int *out) {
    const int H = h->kp.H;
    *out = H;
    if (!h->kp.skip_deep) return LBM_OK;
    const long long want = h->exec_steps - lbm_melt::kRbLag;
    const long long oldest = std::max(h->rb_valid_from, h->rb_next - lbm_melt::kRbRing);
    for (long long k = h->rb_next - 1; k >= oldest; --k) {
        const int slot = (int)(k % lbm_melt::kRbRing);
        if (h->rb_step[slot] > want && k > h->rb_synced) continue;  // too recent to wait for
        if (k > h->rb_synced) {
            CK(cudaEventSynchronize(h->rb_ev[slot]), "read-back wait");
            h->rb_synced = k;
        }
        // the copy followed step rb_step (0-based): counts of the state the
        // coming step reads exceed it by at most the steps in between
        const long long b = (long long)h->rb_val[slot] + (h->exec_steps - h->rb_step[slot] - 1) + 3;
        *out = b < H ? (int)b : H;
        return LBM_OK;
    }
    return LBM_OK;
}

// A read-back taken now, synchronously (after create and set_state, so that
// the first steps of a run are bounded too).
lbm_status seed_readback(lbm_melt *h) {
    if (!h->kp.skip_deep) return LBM_OK;
    const int slot = (int)(h->rb_next % lbm_melt::kRbRing);
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    CK(cudaMemcpy(h->rb_val + slot, h->jmax_dev, sizeof(int), cudaMemcpyDeviceToHost), "read-back");
    h->rb_step[slot] = h->exec_steps - 1;
    h->rb_synced = h->rb_next;
    h->rb_next++;
    return LBM_OK;
}

// After every kRbEvery-th step (or now, with force): copy the running
// maximum into the next ring slot.
lbm_status jmax_readback(lbm_melt *h, bool force = false) {
    if (!h->kp.skip_deep || (!force && h->exec_steps % lbm_melt::kRbEvery)) return LBM_OK;
    const int slot = (int)(h->rb_next % lbm_melt::kRbRing);
    CK(cudaMemcpyAsync(h->rb_val + slot, h->jmax_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read-back");
    CK(cudaEventRecord(h->rb_ev[slot], h->stream), "read-back event");
    h->rb_step[slot] = h->exec_steps - 1;
    h->rb_next++;
    return LBM_OK;
}

// scale * (sum of the n values v) in one launch, deterministic for a given
// n and block count: block b adds the b-th contiguous chunk in a fixed order
// in strides of the block size, then a tree; the block that finishes last
// (atomic ticket) adds the partials in block order, writes the result and
// resets the ticket.
__global__ void k_sum_once(const double *__restrict__ v, long long n, long long chunk, double scale,
                           double *part, unsigned int *ticket, double *__restrict__ out) {
    __shared__ double sh[256];
    __shared__ bool last;
    const long long lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
    double acc = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) acc += v[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[blockIdx.x] = sh[0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) acc += __ldcg(part + b);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *out = sh[0] * scale;
        *ticket = 0u;
    }
}

__global__ void k_fill_f(float *p, long long n, float v) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

__global__ void k_fill_d(double *p, long long n, double v) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Launch shape of the stream-collide.
// Launch shape of the stream-collide: the caller's (lbm_melt_set_launch),
// else 128 threads x-major, the width fitted to the threads of a row (nx / 2
// with two nodes per thread; at most 64 wide with FP16 pairs, 0.141 against
// 0.145 ms at 256^3 with 128).
dim3 sc_block(const lbm_melt *h) {
    if (h->bx) return dim3(h->bx, h->by, 1);
    if (!use_pairs(h)) return lbm::node_block(h->kp);
    const int bx = lbm::block_width(h->kp.nx / 2, h->precision == 1 ? 64 : 128);
    return dim3(bx, 128 / bx, 1);
}

// Enqueue one step from phase (cur, inflight) on stream st with the
// stream-collide grid cut at `height`; returns the phase after it.
cudaError_t enqueue_step(lbm_melt *h, int &cur, int &inflight, int height, dim3 blk, cudaStream_t st) {
    Bufs b = bufs_at(h, cur, inflight);
    b.k1_height = height;
    const int odd = inflight;
    cudaError_t e = LAUNCH(h, stream_collide, h->kp, h->face, odd, b, blk, st);
    if (e != cudaSuccess) return e;
    inflight = !odd;
    b = bufs_at(h, cur, inflight);
    e = LAUNCH(h, front, h->kp, h->face, inflight, 1, b, st);
    if (e == cudaSuccess) e = LAUNCH(h, flip, h->kp, h->face, inflight, 1, b, st);
    cur ^= 1;
    return e;
}

// The graph of graph_steps steps from the handle's phase with the
// stream-collide grid cut at `height` or higher: the cached one when it was
// captured for this phase and block shape at a height from `height` to
// height + 32, else a new capture (heights rounded up to a multiple of 8).
// The replays are bit-identical to single steps: the extra blocks of a
// higher grid find only deep solid nodes and return at once.
lbm_status step_graph(lbm_melt *h, int height, cudaGraphExec_t *out) {
    const dim3 blk = sc_block(h);
    lbm_melt::StepGraph &g = h->graphs[h->cur][h->inflight];
    if (g.exec && g.bx == (int)blk.x && g.by == (int)blk.y && g.height >= height && g.height <= height + 32) {
        *out = g.exec;
        return LBM_OK;
    }
    const int H = h->kp.H;
    int hc = std::min(H, (height + 7) / 8 * 8);
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "capture stream");
    CK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    int cur = h->cur, inflight = h->inflight;
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < h->graph_steps && e == cudaSuccess; ++k) e = enqueue_step(h, cur, inflight, hc, blk, h->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && g.exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(g.exec, graph, &info) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
    }
    if (e == cudaSuccess && !g.exec) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g.exec = nullptr;
        return cuda_err(h, e, "step graph");
    }
    g.height = hc;
    g.bx = (int)blk.x;
    g.by = (int)blk.y;
    *out = g.exec;
    return LBM_OK;
}

// Whether the next graph_steps steps may be replayed from a graph: no timed
// launches, no wall field pending (the graphs read the walls of thw_cur), no
// report row due within them.
bool graph_eligible(const lbm_melt *h, long long left) {
    const long long G = h->graph_steps;
    if (G <= 0 || left < G || h->timing || h->thw_pending) return false;
    if (h->report_every > 0 && (h->steps + G) / h->report_every != h->steps / h->report_every) return false;
    return true;
}

}  // namespace

lbm_status lbm_check_status(lbm_melt *h) { return check_status(h); }

cudaError_t lbm_enqueue_step(lbm_melt *h, int &cur, int &inflight, int height, cudaStream_t st) {
    return enqueue_step(h, cur, inflight, height, sc_block(h), st);
}



namespace {

// The initial state (reading of the paper's initial condition: a front at s0
// with the liquid below at the Neumann temperature of that front; with heat
// conduction in a subcooled solid, the two-phase Neumann solution, the solid
// above the front at its temperature), the liquid counts, 3x3 bounds and
// ghost nodes of that state.  Synchronises.
cudaError_t initial_state(lbm_melt *h) {
    const Derived &d = h->d;
    const KP &p = h->kp;
    const double Th = h->Th, Tc = h->Tc, Tm = h->Tm, Ste = h->Ste;
    const size_t nc = (size_t)d.ncols;
    const size_t es = h->precision == 1 ? sizeof(__half) : sizeof(float);
    const size_t nF = 19 * (size_t)p.ld * es, nG = 7 * (size_t)p.ld * es;
    const bool subcooled = p.cond && Tc < Tm;
    const double rk = std::sqrt(p.cond ? h->ks_kl : 1.0);
    std::vector<float> Tprof(d.H);
    for (int j = 0; j < d.H; ++j) {
        const double a = j + 0.5;
        double T = Tm;
        if (a < d.s0) {
            if (Ste > 0.0) T = Th - (Th - Tm) * std::erf(a / (2.0 * std::sqrt(d.alpha * d.t0))) / std::erf(d.lambda);
        } else if (subcooled) {
            // T = Tc + (Tm - Tc) erfc(a / (2 sqrt(alpha_s t0))) / erfc(lambda sqrt(alpha / alpha_s)),
            // with alpha_s t0 = kappa s0^2 / (4 lambda^2)
            T = Ste > 0.0 ? Tc + (Tm - Tc) * std::erfc(d.lambda * a / (rk * d.s0)) / std::erfc(d.lambda / rk) : Tc;
        }
        Tprof[j] = (float)T;
    }
    float *Tprof_dev = nullptr;
    cudaError_t e = cudaMalloc(&Tprof_dev, sizeof(float) * d.H);
    if (e != cudaSuccess) return e;
    const int nb = (int)((nc + 255) / 256);
    e = cudaMemcpyAsync(Tprof_dev, Tprof.data(), sizeof(float) * d.H, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->F, 0, nF, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->G, 0, nG, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->js[0], 0, nc * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->nb[0], 0, nc * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->nb[1], 0, nc * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->gpost, 0, 7 * nc * 4, h->stream);
    if (e == cudaSuccess && h->spost) e = cudaMemsetAsync(h->spost, 0, 7 * nc * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->status_dev, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->jmax_dev, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->ticket, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) {
        k_fill_d<<<nb, 256, 0, h->stream>>>(h->s[0], (long long)nc, d.s0);
        k_fill_f<<<nb, 256, 0, h->stream>>>(h->thw_cur, (long long)nc, (float)Th);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        // liquid counts of the initial front (front held), then the initial
        // distributions, then the ghost nodes of that state
        h->cur = 0;
        h->inflight = 0;
        Bufs b = bufs(h);
        e = LAUNCH(h, front, p, h->face, 0, 0, b, h->stream);
        if (e == cudaSuccess) {
            h->cur = 1;
            b = bufs(h);
            e = LAUNCH(h, init, p, h->face, b, Tprof_dev, h->stream);
        }
    }
    if (e == cudaSuccess && refresh_front(h) != LBM_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(Tprof_dev);
    return e;
}

}  // namespace

LBM_API const char *lbm_melt_version(void) { return "lbm_melt 0.1 (sm_103a)"; }

LBM_API lbm_status lbm_melt_derive(const lbm_melt_grid *grid, double Ra, double Pr, double Ste, double Th,
                                   double Tc, double Tm, const lbm_melt_rates *rates, lbm_melt_info *info) {
    Derived d;
    lbm_status st = derive(grid, Ra, Pr, Ste, Th, Tc, Tm, rates, d, nullptr, 0);
    if (st != LBM_OK || !info) return st;
    std::memset(info, 0, sizeof *info);
    info->nu = d.nu;
    info->alpha = d.alpha;
    info->gbeta = d.gbeta;
    info->tau_nu = 3.0 * d.nu + 0.5;
    info->s_nu = d.s_nu;
    info->s_alpha = d.s_alpha;
    info->lambda = d.lambda;
    info->t0 = d.t0;
    info->H = d.H;
    info->n_cells = d.N;
    info->n_columns = d.ncols;
    return LBM_OK;
}

// Validation message of lbm_melt_derive's rejection (static buffer, not
// thread-safe; for diagnostics).
LBM_API const char *lbm_melt_derive_error(const lbm_melt_grid *grid, double Ra, double Pr, double Ste, double Th,
                                          double Tc, double Tm, const lbm_melt_rates *rates) {
    static char msg[256];
    Derived d;
    msg[0] = 0;
    derive(grid, Ra, Pr, Ste, Th, Tc, Tm, rates, d, msg, sizeof msg);
    return msg;
}

LBM_API lbm_status lbm_melt_create(const lbm_melt_grid *grid, double Ra, double Pr, double Ste, double Th,
                                   double Tc, double Tm, const lbm_melt_rates *rates, void *cuda_stream,
                                   lbm_melt **out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    Derived d;
    lbm_status st = derive(grid, Ra, Pr, Ste, Th, Tc, Tm, rates, d, nullptr, 0);
    if (st != LBM_OK) return st;
    lbm_melt *h = new (std::nothrow) lbm_melt();
    if (!h) return LBM_ENOMEM;
    h->d = d;
    h->face = grid->heated_face;
    h->precision = grid->precision;
    h->Ste = Ste; h->Th = Th; h->Tc = Tc; h->Tm = Tm;
    h->Ra = Ra;
    h->derived_from_Ra = rates->derive_from_Ra ? 1 : 0;
    h->stream = (cudaStream_t)cuda_stream;
    KP &p = h->kp;
    p.nx = grid->nx; p.ny = grid->ny; p.nz = grid->nz;
    p.H = d.H; p.P1 = d.P1; p.P2 = d.P2; p.ncols = (int)d.ncols;
    p.N = d.N;
    p.ld = (d.N + 127) / 128 * 128;  // 256-byte aligned direction arrays (fp16) / 512 (fp32)
    p.Tm = (float)Tm; p.Tc = (float)Tc; p.gbeta = (float)d.gbeta;
    p.s_e = (float)d.s_e; p.s_eps = (float)d.s_eps; p.s_q = (float)d.s_q; p.s_nu = (float)d.s_nu;
    p.s_pi = (float)d.s_pi; p.s_m = (float)d.s_m;
    p.s_alpha = (float)d.s_alpha; p.s_g4 = (float)d.s_g4; p.s_g5 = (float)d.s_g5;
    p.Tm_d = Tm; p.Th_d = Th;
    // storage shift of the energy populations: Tm, or the mid temperature
    // for FP16 storage (halves the largest stored value)
    p.Ts = h->precision == 1 ? (float)(0.5 * (Th + Tm)) : (float)Tm;
    p.dTms = (float)Tm - p.Ts;
    p.coef = Ste > 0.0 ? d.alpha * Ste / (Th - Tm) : 0.0;
    p.coef_f = (float)p.coef;
    p.skip_deep = (Tc == Tm) ? 1 : 0;
    p.cond = 0;  // the solid held at Tm until lbm_melt_set_solid_conduction
    p.kappa = 1.0f;
    p.s_alpha_s = p.s_alpha;
    {
        const long long sy = p.nx, sz = (long long)p.nx * p.ny;
        for (int i = 0; i < 19; ++i) {
            const long long off = lbm::ex(i) + lbm::ey(i) * sy + lbm::ez(i) * sz;
            h->lk.fin[i] = lbm::opp(i) * p.ld - off;
            h->lk.fout[i] = i * p.ld + off;
        }
        for (int i = 0; i < 7; ++i) {
            const long long off = lbm::tx(i) + lbm::ty(i) * sy + lbm::tz(i) * sz;
            h->lk.gin[i] = lbm::opp7(i) * p.ld - off;
            h->lk.gout[i] = i * p.ld + off;
        }
    }
    auto fail = [&](lbm_status s) { free_all(h); delete h; return s; };
    if (cudaGetDevice(&h->device) != cudaSuccess) return fail(LBM_ECUDA);
    {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess || sms < 1)
            return fail(LBM_ECUDA);
        h->cblk = lbm::col_block(h->kp.ncols, sms);
        h->sms = sms;
    }
    h->rb_synced = -1;
    // small cavities are launch bound: replay their steps from graphs
    h->graph_steps = d.N <= kGraphMaxNodes ? kGraphSteps : 0;
    h->pairs_mode = -1;
    if (cudaMallocHost(&h->rb_val, lbm_melt::kRbRing * sizeof(int)) != cudaSuccess) return fail(LBM_ENOMEM);
    for (int k = 0; k < lbm_melt::kRbRing; ++k)
        if (cudaEventCreateWithFlags(&h->rb_ev[k], cudaEventDisableTiming) != cudaSuccess) return fail(LBM_ECUDA);
    const size_t es = h->precision == 1 ? sizeof(__half) : sizeof(float);
    const size_t nF = 19 * (size_t)p.ld * es, nG = 7 * (size_t)p.ld * es;
    const size_t nc = (size_t)d.ncols;
    struct { void **p; size_t b; } allocs[] = {
        {&h->F, nF}, {&h->G, nG}, {(void **)&h->js[0], nc * 4}, {(void **)&h->js[1], nc * 4},
        {(void **)&h->nb[0], nc * 4}, {(void **)&h->nb[1], nc * 4},
        {(void **)&h->s[0], nc * 8}, {(void **)&h->s[1], nc * 8}, {(void **)&h->gpost, 7 * nc * 4},
        {(void **)&h->thw_cur, nc * 4}, {(void **)&h->thw_prev, nc * 4}, {(void **)&h->status_dev, 4},
        {(void **)&h->sum_dev, 8}, {(void **)&h->ticket, 8}, {(void **)&h->red_part, kRedBlocks * 4 * 8}, {(void **)&h->totals_dev, 7 * 8},
        {(void **)&h->jmax_dev, sizeof(int)}, {(void **)&h->nu_dev, nc * 8}};
    h->nred = kRedBlocks;
    for (auto &a : allocs) {
        cudaError_t e = cudaMalloc(a.p, a.b);
        if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA);
        h->bytes += a.b;
    }
    const cudaError_t e = initial_state(h);
    if (e != cudaSuccess) return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA);
    if (seed_readback(h) != LBM_OK) return fail(LBM_ECUDA);
    *out = h;
    return LBM_OK;
}

LBM_API void lbm_melt_destroy(lbm_melt *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    lbm_tape_free(h);
    free_all(h);
    delete h;
}

LBM_API const char *lbm_melt_last_error(const lbm_melt *h) { return h ? h->err : "null handle"; }

LBM_API lbm_status lbm_melt_step(lbm_melt *h, long long n) {
    if (!h) return LBM_EINVAL;
    if (n < 0) return set_err(h, LBM_EINVAL, "negative step count");
    const dim3 blk = sc_block(h);
    for (long long t = 0; t < n; ++t) {
        if (graph_eligible(h, n - t)) {
            // graph_steps steps in one replay; the grid height bound of the
            // first of them grows by one node per step over the replay
            int height = 0;
            lbm_status hs = k1_height(h, &height);
            if (hs != LBM_OK) return hs;
            cudaGraphExec_t exec = nullptr;
            if ((hs = step_graph(h, std::min(h->kp.H, height + h->graph_steps), &exec)) != LBM_OK) return hs;
            CK(cudaGraphLaunch(exec, h->stream), "step graph launch");
            const int G = h->graph_steps;
            if (G & 1) { h->cur ^= 1; h->inflight ^= 1; }
            h->thw_last_prev = 0;
            h->steps += G;
            h->exec_steps += G;
            if ((hs = jmax_readback(h, true)) != LBM_OK) return hs;
            t += G - 1;
            continue;
        }
        Bufs b = bufs(h);
        lbm_status hs = k1_height(h, &b.k1_height);
        if (hs != LBM_OK) return hs;
        const int odd = h->inflight;
        cudaEvent_t *evp = nullptr;
        if (h->timing) {
            if (h->ev_used + 2 > h->ev.size()) {
                for (int k = 0; k < 64; ++k) {
                    cudaEvent_t ev;
                    CK(cudaEventCreate(&ev), "event create");
                    h->ev.push_back(ev);
                }
            }
            evp = &h->ev[h->ev_used];
            h->ev_used += 2;
            CK(cudaEventRecord(evp[0], h->stream), "event record");
        }
        CK(LAUNCH(h, stream_collide, h->kp, h->face, odd, b, blk, h->stream), "stream-collide");
        if (evp) CK(cudaEventRecord(evp[1], h->stream), "event record");
        h->inflight = !odd;
        if (odd) h->thw_pending = 0;
        h->thw_last_prev = 0;
        b = bufs(h);
        CK(LAUNCH(h, front, h->kp, h->face, h->inflight, 1, b, h->stream), "front");
        CK(LAUNCH(h, flip, h->kp, h->face, h->inflight, 1, b, h->stream), "flip");
        h->cur ^= 1;
        h->steps++;
        h->exec_steps++;
        if ((hs = jmax_readback(h)) != LBM_OK) return hs;
        if (h->report_every > 0 && h->steps % h->report_every == 0) {
            double *row = h->report + 8 * (h->report_rows % h->report_cap);
            b = bufs(h);
            CK(LAUNCH(h, totals, h->kp, h->face, h->inflight, b, h->red_part, h->nred, (double)h->steps, row,
                      h->stream), "report totals");
            h->report_rows++;
        }
    }
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_totals(lbm_melt *h, double *out, int ptr_kind) {
    if (!h || !out) return LBM_EINVAL;
    Bufs b = bufs(h);
    CK(LAUNCH(h, totals, h->kp, h->face, h->inflight, b, h->red_part, h->nred, -1.0, h->totals_dev, h->stream),
       "totals");
    CK(cudaMemcpyAsync(out, h->totals_dev, 7 * 8, ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       h->stream), "copy totals");
    return check_status(h);
}

LBM_API lbm_status lbm_melt_set_report(lbm_melt *h, long long every, long long capacity) {
    if (!h || every < 0 || (every > 0 && capacity < 1)) return LBM_EINVAL;
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    cudaFree(h->report);
    h->report = nullptr;
    h->report_every = 0;
    h->report_cap = 0;
    h->report_rows = 0;
    if (every == 0) return LBM_OK;
    CK(cudaMalloc(&h->report, (size_t)capacity * 8 * 8), "alloc report");
    h->report_every = every;
    h->report_cap = capacity;
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_get_report(lbm_melt *h, double *rows, long long max_rows, long long *n_rows) {
    if (!h || !n_rows) return LBM_EINVAL;
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    const long long avail = h->report_rows < h->report_cap ? h->report_rows : h->report_cap;
    if (!rows) {  // query: how many rows are kept
        *n_rows = avail;
        return LBM_OK;
    }
    const long long n = avail < max_rows ? avail : max_rows;
    *n_rows = n;
    if (n == 0) return LBM_OK;
    // the oldest kept row first
    const long long first = h->report_rows - avail;
    for (long long r = 0; r < n; ++r) {
        const long long slot = (first + r) % h->report_cap;
        CK(cudaMemcpy(rows + 8 * r, h->report + 8 * slot, 8 * 8, cudaMemcpyDeviceToHost), "copy report");
    }
    return LBM_OK;
}

// scale * (sum of the ncols column values v), into dst on the handle's
// stream: one launch of k_sum_once (chunks of at least 1024 columns per
// block, fixed order), then a copy.
lbm_status enqueue_column_sum(lbm_melt *h, const double *v, double scale, double *dst, int ptr_kind) {
    const long long nc = h->kp.ncols;
    const long long nb = std::max<long long>(1, std::min<long long>(kRedBlocks, (nc + 1023) / 1024));
    const long long chunk = (nc + nb - 1) / nb;
    k_sum_once<<<(int)nb, 256, 0, h->stream>>>(v, nc, chunk, scale, h->red_part, h->ticket, h->sum_dev);
    CK(cudaGetLastError(), "sum");
    CK(cudaMemcpyAsync(dst, h->sum_dev, 8, ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream),
       "copy sum");
    return LBM_OK;
}

// Liquid fraction = mean front height over H (Σ s / (H ncols)).
lbm_status enqueue_liquid_fraction(lbm_melt *h, double *dst, int ptr_kind) {
    return enqueue_column_sum(h, h->s[h->cur], 1.0 / ((double)h->kp.H * (double)h->kp.ncols), dst, ptr_kind);
}

LBM_API lbm_status lbm_melt_sync(lbm_melt *h) {
    if (!h) return LBM_EINVAL;
    return check_status(h);
}

LBM_API lbm_status lbm_melt_get(lbm_melt *h, float *T, float *u, double *S, double *liquid_fraction, int ptr_kind) {
    if (!h) return LBM_EINVAL;
    const KP &p = h->kp;
    const size_t N = (size_t)p.N, nc = (size_t)p.ncols;
    float *Td = nullptr, *ud = nullptr;
    if (T || u) {
        if (ptr_kind) { Td = T; ud = u; }
        else {
            if (T) CK(cudaMalloc(&Td, N * 4), "alloc T");
            if (u) CK(cudaMalloc(&ud, 3 * N * 4), "alloc u");
        }
        Bufs b = bufs(h);
        CK(LAUNCH(h, macro, p, h->face, h->inflight, b, Td, ud, h->stream), "macro");
        if (!ptr_kind) {
            if (T) CK(cudaMemcpyAsync(T, Td, N * 4, cudaMemcpyDeviceToHost, h->stream), "copy T");
            if (u) CK(cudaMemcpyAsync(u, ud, 3 * N * 4, cudaMemcpyDeviceToHost, h->stream), "copy u");
        }
    }
    if (S) CK(cudaMemcpyAsync(S, h->s[h->cur], nc * 8, ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              h->stream), "copy S");
    if (liquid_fraction) {
        const lbm_status st = enqueue_liquid_fraction(h, liquid_fraction, ptr_kind);
        if (st != LBM_OK) return st;
    }
    lbm_status st = check_status(h);
    if (!ptr_kind) { cudaFree(Td); cudaFree(ud); }
    return st;
}

LBM_API lbm_status lbm_melt_get_async(lbm_melt *h, double *S, double *liquid_fraction, int ptr_kind) {
    if (!h) return LBM_EINVAL;
    if (S)
        CK(cudaMemcpyAsync(S, h->s[h->cur], (size_t)h->kp.ncols * 8,
                           ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream), "copy S");
    if (liquid_fraction) return enqueue_liquid_fraction(h, liquid_fraction, ptr_kind);
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_get_state(lbm_melt *h, float *f, float *g, double *S, int ptr_kind) {
    if (!h) return LBM_EINVAL;
    const KP &p = h->kp;
    const size_t N = (size_t)p.N, nc = (size_t)p.ncols;
    float *fd = nullptr, *gd = nullptr;
    if (f || g) {
        if (ptr_kind) { fd = f; gd = g; }
        else {
            if (f) CK(cudaMalloc(&fd, 19 * N * 4), "alloc f");
            if (g) CK(cudaMalloc(&gd, 7 * N * 4), "alloc g");
        }
        Bufs b = bufs(h);
        CK(LAUNCH(h, state_out, p, h->face, h->inflight, b, fd, gd, h->stream), "state out");
        if (!ptr_kind) {
            if (f) CK(cudaMemcpyAsync(f, fd, 19 * N * 4, cudaMemcpyDeviceToHost, h->stream), "copy f");
            if (g) CK(cudaMemcpyAsync(g, gd, 7 * N * 4, cudaMemcpyDeviceToHost, h->stream), "copy g");
        }
    }
    if (S) CK(cudaMemcpyAsync(S, h->s[h->cur], nc * 8, ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              h->stream), "copy S");
    lbm_status st = check_status(h);
    if (!ptr_kind) { cudaFree(fd); cudaFree(gd); }
    return st;
}

LBM_API lbm_status lbm_melt_set_state(lbm_melt *h, const float *f, const float *g, const double *S, int ptr_kind) {
    if (!h) return LBM_EINVAL;
    if (S && (!f || !g)) return set_err(h, LBM_EINVAL, "a new front needs f and g too");
    const KP &p = h->kp;
    const size_t N = (size_t)p.N, nc = (size_t)p.ncols;
    // Bring the layout to natural first, so that kept parts stay valid.
    if (h->inflight && (!f || !g)) {
        float *fd = nullptr, *gd = nullptr;
        CK(cudaMalloc(&fd, 19 * N * 4), "alloc f");
        CK(cudaMalloc(&gd, 7 * N * 4), "alloc g");
        Bufs b = bufs(h);
        CK(LAUNCH(h, state_out, p, h->face, 1, b, fd, gd, h->stream), "state out");
        CK(LAUNCH(h, state_in, p, h->face, b, fd, gd, h->stream), "state in");
        CK(cudaStreamSynchronize(h->stream), "synchronize");
        cudaFree(fd);
        cudaFree(gd);
    }
    h->inflight = 0;
    h->thw_pending = 0;
    if (S) {
        lbm_status st = copy_in(h, h->s[h->cur], S, nc * 8, ptr_kind);
        if (st != LBM_OK) return st;
        // liquid counts from the new fronts, front held; their maximum anew
        CK(cudaMemsetAsync(h->jmax_dev, 0, sizeof(int), h->stream), "reset maximum");
        if ((st = refresh_front(h)) != LBM_OK) return st;
        h->rb_valid_from = h->rb_next;  // earlier copies may lie below the new counts
        if ((st = seed_readback(h)) != LBM_OK) return st;
    }
    const float *fd = f, *gd = g;
    float *tf = nullptr, *tg = nullptr;
    if (!ptr_kind) {
        if (f) { CK(cudaMalloc(&tf, 19 * N * 4), "alloc f"); CK(cudaMemcpyAsync(tf, f, 19 * N * 4, cudaMemcpyHostToDevice, h->stream), "copy f"); fd = tf; }
        if (g) { CK(cudaMalloc(&tg, 7 * N * 4), "alloc g"); CK(cudaMemcpyAsync(tg, g, 7 * N * 4, cudaMemcpyHostToDevice, h->stream), "copy g"); gd = tg; }
    }
    if (f || g) {
        Bufs b = bufs(h);
        CK(LAUNCH(h, state_in, p, h->face, b, fd, gd, h->stream), "state in");
    }
    lbm_status st = refresh_front(h);
    if (st == LBM_OK) st = check_status(h);
    cudaFree(tf);
    cudaFree(tg);
    return st;
}

LBM_API lbm_status lbm_melt_set_hot_wall(lbm_melt *h, const float *T_h_field, int ptr_kind) {
    if (!h || !T_h_field) return LBM_EINVAL;
    const size_t nc = (size_t)h->kp.ncols;
    if (h->inflight && !h->thw_pending) {
        // the pending odd step must still read the walls with the field of
        // the step that produced the in-flight values
        CK(cudaMemcpyAsync(h->thw_prev, h->thw_cur, nc * 4, cudaMemcpyDeviceToDevice, h->stream), "copy wall");
        h->thw_pending = 1;
    } else if (!h->inflight && !h->thw_last_prev) {
        // keep the field of the last streaming for the Nusselt number until
        // the next step (the next step, an even one, reads no wall)
        CK(cudaMemcpyAsync(h->thw_prev, h->thw_cur, nc * 4, cudaMemcpyDeviceToDevice, h->stream), "copy wall");
        h->thw_last_prev = 1;
    }
    h->thw_gen++;
    return copy_in(h, h->thw_cur, T_h_field, nc * 4, ptr_kind);
}

LBM_API lbm_status lbm_melt_get_nusselt(lbm_melt *h, double *Nu, double *Nu_mean, int ptr_kind) {
    if (!h) return LBM_EINVAL;
    if (Nu || Nu_mean) {
        Bufs b = bufs(h);
        CK(LAUNCH(h, nusselt, h->kp, h->face, h->inflight, b, h->stream), "nusselt");
        if (Nu)
            CK(cudaMemcpyAsync(Nu, h->nu_dev, (size_t)h->kp.ncols * 8,
                               ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream), "copy Nu");
        if (Nu_mean) {
            const lbm_status st = enqueue_column_sum(h, h->nu_dev, 1.0 / (double)h->kp.ncols, Nu_mean, ptr_kind);
            if (st != LBM_OK) return st;
        }
    }
    return check_status(h);
}

LBM_API lbm_status lbm_melt_get_info(lbm_melt *h, lbm_melt_info *info) {
    if (!h || !info) return LBM_EINVAL;
    std::memset(info, 0, sizeof *info);
    const Derived &d = h->d;
    info->nu = d.nu;
    info->alpha = d.alpha;
    info->gbeta = d.gbeta;
    info->tau_nu = 3.0 * d.nu + 0.5;
    info->s_nu = d.s_nu;
    info->s_alpha = d.s_alpha;
    info->lambda = d.lambda;
    info->t0 = d.t0;
    info->H = d.H;
    info->n_cells = d.N;
    info->n_columns = d.ncols;
    info->steps = h->steps;
    info->device_bytes = h->bytes;
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_set_launch(lbm_melt *h, int bx, int by) {
    if (!h) return LBM_EINVAL;
    if (bx == 0 && by == 0) { h->bx = h->by = 0; return LBM_OK; }
    if (bx < 32 || bx % 32 || by < 1 || bx * by > 128)
        return set_err(h, LBM_EINVAL, "block shape must be a multiple of 32 along x with at most 128 threads");
    h->bx = bx;
    h->by = by;
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_set_graph_steps(lbm_melt *h, int steps) {
    if (!h) return LBM_EINVAL;
    if (steps < 0 || steps > 256) return set_err(h, LBM_EINVAL, "graph steps must be in [0, 256]");
    if (steps != h->graph_steps) {
        CK(cudaStreamSynchronize(h->stream), "synchronize");
        for (auto &row : h->graphs)
            for (auto &g : row)
                if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
        h->graph_steps = steps;
    }
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_set_node_pairs(lbm_melt *h, int mode) {
    if (!h) return LBM_EINVAL;
    if (mode < -1 || mode > 1) return set_err(h, LBM_EINVAL, "node-pair mode must be -1, 0 or 1");
    if (mode == 1 && h->kp.nx % 2 != 0) return set_err(h, LBM_EINVAL, "two nodes per thread need an even nx");
    if (mode != h->pairs_mode) {
        CK(cudaStreamSynchronize(h->stream), "synchronize");
        for (auto &row : h->graphs)
            for (auto &g : row)
                if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
        h->pairs_mode = mode;
    }
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_set_solid_conduction(lbm_melt *h, double ks_kl) {
    if (!h) return LBM_EINVAL;
    if (h->member) return set_err(h, LBM_EINVAL, "an ensemble member keeps its solid at Tm");
    if (h->steps != 0 || h->exec_steps != 0)
        return set_err(h, LBM_EINVAL, "heat conduction in the solid is chosen before the first step");
    if (!(ks_kl >= 0.0 && ks_kl <= 1e6))
        return set_err(h, LBM_EINVAL, "k_s / k_l must be in (0, 1e6] (0 turns conduction in the solid off)");
    const bool on = ks_kl > 0.0;
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    if (on && !h->spost) {
        const size_t b = 7 * (size_t)h->kp.ncols * 4;
        CK(cudaMalloc(&h->spost, b), "alloc solid ghosts");
        h->bytes += b;
    }
    KP &p = h->kp;
    const double alpha_s = on ? ks_kl * h->d.alpha : h->d.alpha;
    p.cond = on ? 1 : 0;
    p.kappa = (float)(on ? ks_kl : 1.0);
    p.s_alpha_s = (float)(1.0 / (alpha_s / CS2T + 0.5));
    p.skip_deep = (!on && h->Tc == h->Tm) ? 1 : 0;
    h->ks_kl = on ? ks_kl : 0.0;
    // the initial front's Neumann constant: two-phase against a subcooled solid
    Derived &d = h->d;
    d.lambda = (on && h->Tc < h->Tm)
                   ? neumann_lambda_two_phase(h->Ste, (h->Tm - h->Tc) / (h->Th - h->Tm), ks_kl)
                   : neumann_lambda(h->Ste);
    d.t0 = h->Ste > 0.0 ? d.s0 * d.s0 / (4.0 * d.lambda * d.lambda * d.alpha) : 0.0;
    for (auto &row : h->graphs)
        for (auto &g : row)
            if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    h->rb_valid_from = h->rb_next;  // earlier read-backs bound another run
    h->thw_pending = 0;
    h->thw_last_prev = 0;
    const cudaError_t e = initial_state(h);
    if (e != cudaSuccess) return cuda_err(h, e, "initial state");
    return seed_readback(h);
}

LBM_API lbm_status lbm_melt_set_timing(lbm_melt *h, int enable) {
    if (!h) return LBM_EINVAL;
    h->timing = enable ? 1 : 0;
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_kernel_time(lbm_melt *h, double *ms, long long *launches, int reset) {
    if (!h) return LBM_EINVAL;
    CK(cudaStreamSynchronize(h->stream), "synchronize");
    double tot = 0.0;
    for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, h->ev[k], h->ev[k + 1]), "event elapsed");
        tot += t;
    }
    if (ms) *ms = tot;
    if (launches) *launches = (long long)(h->ev_used / 2);
    if (reset) h->ev_used = 0;
    return LBM_OK;
}

// ------------------------------------------------------------------------
// Read-back without allocation.
//
// lbm_melt_get stages host-bound T and u in device buffers it allocates per
// call.  Some callers cannot let a library allocate: a real-time driver loop
// in which a cudaMalloc would synchronise the device, or an application that
// gives all device memory to its own pool allocator.  lbm_melt_get_noalloc
// stages through the fixed array below instead.  The array lives in every GPU
// that loads the library until the process exits.  All calls share it, so
// calls whose work overlaps on the GPU race with each other.
static const long long kNoallocMaxNodes = 2097152;  // 128^3: 16 bytes per node (T and u)
static __device__ __align__(256) unsigned char g_noalloc_stage[kNoallocMaxNodes * 16];

namespace {
const int kMaxDevices = 64;
// Device address of the array per device, looked up once (with that device
// current) under a once-flag, so that concurrent first calls from several
// host threads do the set-up once.  A reset of the device (cudaDeviceReset)
// invalidates the address, as it does every handle made before it.
void *g_noalloc_dev[kMaxDevices];
cudaError_t g_noalloc_err[kMaxDevices];
std::once_flag g_noalloc_once[kMaxDevices];
}  // namespace

LBM_API lbm_status lbm_melt_get_noalloc(lbm_melt *h, float *T, float *u, double *S, double *liquid_fraction,
                                        int ptr_kind) {
    if (!h) return LBM_EINVAL;
    const KP &p = h->kp;
    const size_t N = (size_t)p.N, nc = (size_t)p.ncols;
    if (p.N > kNoallocMaxNodes)
        return set_err(h, LBM_EINVAL, "lbm_melt_get_noalloc stages at most %lld nodes; this cavity has %lld",
                       kNoallocMaxNodes, p.N);
    int dev = -1;
    CK(cudaGetDevice(&dev), "get device");
    if (dev != h->device || dev < 0 || dev >= kMaxDevices)
        return set_err(h, LBM_EINVAL, "make the handle's device (%d) current before lbm_melt_get_noalloc", h->device);
    // one-time set-up on this device (the device is current): the host-side
    // name of the array is only a stand-in, so look up its device address
    std::call_once(g_noalloc_once[dev], [dev]() {
        void *ptr = nullptr;
        g_noalloc_err[dev] = cudaGetSymbolAddress(&ptr, g_noalloc_stage);
        g_noalloc_dev[dev] = ptr;
    });
    CK(g_noalloc_err[dev], "staging array address");
    unsigned char *stage = (unsigned char *)g_noalloc_dev[dev];
    float *Td = ptr_kind ? T : (float *)stage;
    float *ud = ptr_kind ? u : (float *)(stage + N * 4);
    if (T || u) {
        Bufs b = bufs(h);
        CK(LAUNCH(h, macro, p, h->face, h->inflight, b, T ? Td : nullptr, u ? ud : nullptr, h->stream), "macro");
        if (!ptr_kind) {
            if (T) CK(cudaMemcpyAsync(T, Td, N * 4, cudaMemcpyDeviceToHost, h->stream), "copy T");
            if (u) CK(cudaMemcpyAsync(u, ud, 3 * N * 4, cudaMemcpyDeviceToHost, h->stream), "copy u");
        }
    }
    if (S) CK(cudaMemcpyAsync(S, h->s[h->cur], nc * 8, ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                              h->stream), "copy S");
    if (liquid_fraction) {
        // the handle's own reduction buffers, allocated at create: the same
        // two-pass sum as lbm_melt_get
        const lbm_status st = enqueue_liquid_fraction(h, liquid_fraction, ptr_kind);
        if (st != LBM_OK) return st;
    }
    return check_status(h);
}
