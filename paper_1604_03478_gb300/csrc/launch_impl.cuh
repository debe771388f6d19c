// launch_impl.cuh -- definitions of Launch<ST>; included by exactly one
// translation unit per storage type.
#pragma once

#include "kernels.cuh"
#include "launch.h"

namespace lbm {

// The step's kernels (stream-collide, front, flip) are launched with
// programmatic stream serialization (see step_launch_wait) when LBM_PDL.
#ifndef LBM_PDL
#define LBM_PDL 1
#endif
template <typename... KArgs, typename... Args>
static cudaError_t launch_step_kernel(void (*kern)(KArgs...), dim3 grd, dim3 blk, cudaStream_t st, Args... args) {
#if LBM_PDL
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grd;
    cfg.blockDim = blk;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
#else
    kern<<<grd, blk, 0, st>>>(args...);
    return cudaGetLastError();
#endif
}

template <typename ST, typename IXE>
static cudaError_t launch_sc(const KP &p, int face, int odd, const Bufs &b, dim3 grd, dim3 blk, cudaStream_t st) {
    const int *jm = p.skip_deep ? b.jmax : nullptr;
    ST *F = (ST *)b.F, *G = (ST *)b.G;
    if (face == 0) {
        if (odd) return launch_step_kernel(k_odd<ST, 0>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, jm);
        else return launch_step_kernel(k_even<ST, 0, IXE>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, jm);
    } else {
        if (odd) return launch_step_kernel(k_odd<ST, 1>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, jm);
        else return launch_step_kernel(k_even<ST, 1, IXE>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, jm);
    }
}

#ifndef LBM_PAIR_ODD_IX
#define LBM_PAIR_ODD_IX unsigned
#endif
// An even nx: two nodes per thread (k_even_pair / k_odd_pair), the grid's x
// extent covering nx / 2 threads.
template <typename ST, typename IXE, typename IXO>
static cudaError_t launch_sc_pair(const KP &p, int face, int odd, const Bufs &b, dim3 blk, cudaStream_t st) {
    const int *jm = p.skip_deep ? b.jmax : nullptr;
    ST *F = (ST *)b.F, *G = (ST *)b.G;
    KP half_x = p;
    half_x.nx = p.nx / 2;
    dim3 grd = k1_grid(half_x, blk, face, b.k1_height);
    if (face == 0) {
        if (odd) return launch_step_kernel(k_odd_pair<ST, 0, IXO>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, jm);
        else return launch_step_kernel(k_even_pair<ST, 0, IXE>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, jm);
    } else {
        if (odd) return launch_step_kernel(k_odd_pair<ST, 1, IXO>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, jm);
        else return launch_step_kernel(k_even_pair<ST, 1, IXE>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, jm);
    }
}

// The even step indexes in 32 bits whenever every index of the 19 direction
// arrays of F fits (19 ld < 2^32: cavities up to about 2.2e8 nodes), else in
// 64 bits (FP16 storage 2% faster at 256^3; the odd step ran slower with
// 32-bit indices, 0.258 against 0.245 ms in FP32, and keeps 64-bit ones).
template <typename ST>
cudaError_t Launch<ST>::stream_collide(const KP &p, int face, int odd, const Bufs &b, dim3 blk, cudaStream_t st) {
    if (p.cond) return LaunchCond<ST>::stream_collide(p, face, odd, b, blk, st);
    if (b.pairs && p.nx % 2 == 0) {
        if (19LL * p.ld < (1LL << 32)) return launch_sc_pair<ST, unsigned, LBM_PAIR_ODD_IX>(p, face, odd, b, blk, st);
        return launch_sc_pair<ST, long long, long long>(p, face, odd, b, blk, st);
    }
    const dim3 grd = k1_grid(p, blk, face, b.k1_height);
    if (19LL * p.ld < (1LL << 32)) return launch_sc<ST, unsigned>(p, face, odd, b, grd, blk, st);
    return launch_sc<ST, long long>(p, face, odd, b, grd, blk, st);
}

template <typename ST>
cudaError_t Launch<ST>::front(const KP &p, int face, int inflight, int move, const Bufs &b, cudaStream_t st) {
    if (p.cond) return LaunchCond<ST>::front(p, face, inflight, move, b, st);
    const dim3 blk(b.cblk), grd = col_grid(p.ncols, b.cblk);
    const ST *F = (const ST *)b.F, *G = (const ST *)b.G;
    if (face == 0)
        return launch_step_kernel(k_front<ST, 0>, grd, blk, st, p, F, G, b.js, b.js_next, b.s, b.s_next, b.gpost, b.thw_wr, inflight, move, b.status, b.jmax);
    return launch_step_kernel(k_front<ST, 1>, grd, blk, st, p, F, G, b.js, b.js_next, b.s, b.s_next, b.gpost, b.thw_wr, inflight, move, b.status, b.jmax);
}

template <typename ST>
cudaError_t Launch<ST>::flip(const KP &p, int face, int inflight, int do_flip, const Bufs &b, cudaStream_t st) {
    const dim3 blk(b.cblk), grd = col_grid(p.ncols, b.cblk);
    ST *F = (ST *)b.F;
    if (face == 0) return launch_step_kernel(k_flip<ST, 0>, grd, blk, st, p, F, b.js, b.js_next, b.nb_next, inflight, do_flip);
    return launch_step_kernel(k_flip<ST, 1>, grd, blk, st, p, F, b.js, b.js_next, b.nb_next, inflight, do_flip);
}

template <typename ST>
cudaError_t Launch<ST>::macro(const KP &p, int face, int inflight, const Bufs &b, float *T, float *u, cudaStream_t st) {
    dim3 blk = node_block(p), grd = node_grid(p, blk);
    const ST *F = (const ST *)b.F, *G = (const ST *)b.G;
    if (face == 0) k_macro<ST, 0><<<grd, blk, 0, st>>>(p, F, G, b.js, b.thw_rd, inflight, T, u);
    else k_macro<ST, 1><<<grd, blk, 0, st>>>(p, F, G, b.js, b.thw_rd, inflight, T, u);
    return cudaGetLastError();
}

template <typename ST>
cudaError_t Launch<ST>::state_out(const KP &p, int face, int inflight, const Bufs &b, float *f, float *g, cudaStream_t st) {
    dim3 blk = node_block(p), grd = node_grid(p, blk);
    const ST *F = (const ST *)b.F, *G = (const ST *)b.G;
    if (face == 0) k_state_out<ST, 0><<<grd, blk, 0, st>>>(p, F, G, b.js, b.nb, b.thw_rd, inflight, f, g);
    else k_state_out<ST, 1><<<grd, blk, 0, st>>>(p, F, G, b.js, b.nb, b.thw_rd, inflight, f, g);
    return cudaGetLastError();
}

template <typename ST>
cudaError_t Launch<ST>::state_in(const KP &p, int face, const Bufs &b, const float *f, const float *g, cudaStream_t st) {
    dim3 blk = node_block(p), grd = node_grid(p, blk);
    ST *F = (ST *)b.F, *G = (ST *)b.G;
    if (face == 0) k_state_in<ST, 0><<<grd, blk, 0, st>>>(p, F, G, b.js, f, g);
    else k_state_in<ST, 1><<<grd, blk, 0, st>>>(p, F, G, b.js, f, g);
    return cudaGetLastError();
}

template <typename ST>
cudaError_t Launch<ST>::init(const KP &p, int face, const Bufs &b, const float *Tprof, cudaStream_t st) {
    dim3 blk = node_block(p), grd = node_grid(p, blk);
    ST *F = (ST *)b.F, *G = (ST *)b.G;
    if (face == 0) k_init<ST, 0><<<grd, blk, 0, st>>>(p, F, G, b.js, Tprof);
    else k_init<ST, 1><<<grd, blk, 0, st>>>(p, F, G, b.js, Tprof);
    return cudaGetLastError();
}

template <typename ST>
cudaError_t Launch<ST>::totals(const KP &p, int face, int inflight, const Bufs &b, double *part, int nparts,
                               double t, double *out, cudaStream_t st) {
    const ST *F = (const ST *)b.F, *G = (const ST *)b.G;
    if (face == 0) k_totals_part<ST, 0><<<nparts, 256, 0, st>>>(p, F, G, b.js, b.thw_rd, inflight, part);
    else k_totals_part<ST, 1><<<nparts, 256, 0, st>>>(p, F, G, b.js, b.thw_rd, inflight, part);
    const cudaError_t e = nusselt(p, face, inflight, b, st);
    if (e != cudaSuccess) return e;
    k_totals_final<<<1, 256, 0, st>>>(part, nparts, b.s, b.nu, p.ncols, (double)p.H, t, out);
    return cudaGetLastError();
}

template <typename ST>
cudaError_t Launch<ST>::nusselt(const KP &p, int face, int inflight, const Bufs &b, cudaStream_t st) {
    const dim3 blk(b.cblk), grd = col_grid(p.ncols, b.cblk);
    const ST *G = (const ST *)b.G;
    if (face == 0) k_nusselt<ST, 0><<<grd, blk, 0, st>>>(p, G, b.thw_nu, inflight, b.nu_scale, b.nu);
    else k_nusselt<ST, 1><<<grd, blk, 0, st>>>(p, G, b.thw_nu, inflight, b.nu_scale, b.nu);
    return cudaGetLastError();
}

}  // namespace lbm
