// k_cond.cu -- the stream-collide and front kernels with heat conduction in
// the solid (Eq. 6's k_s term), for both storage types, one or two nodes per
// thread.  Every node is updated (no deep-solid skip, no height bound on the
// grid).
#include "kernels.cuh"
#include "launch.h"

namespace lbm {

// ------------------------------------------------- two nodes per thread
// The D3Q7 conduction collision of two solid nodes (collide_solid on the
// lanes of float2 values, packed FP32x2 arithmetic).
__device__ __forceinline__ void collide_solid2(const KP &p, float2 (&g)[7]) {
    const float2 g12 = add2(g[1], g[2]), g34 = add2(g[3], g[4]), g56 = add2(g[5], g[6]);
    const float2 Th = add2(g[0], add2(g12, add2(g34, g56)));
    constexpr float i1 = 1.0f / (float)nnorm(1), i4 = 1.0f / (float)nnorm(4);
    constexpr float i5 = 1.0f / (float)nnorm(5), i6 = 1.0f / (float)nnorm(6);
    const float sa = p.s_alpha_s, s4 = p.s_g4, s5 = p.s_g5;
    const float2 c1 = smul2(-sa * i1, sub2(g[1], g[2]));
    const float2 c2 = smul2(-sa * i1, sub2(g[3], g[4]));
    const float2 c3 = smul2(-sa * i1, sub2(g[5], g[6]));
    const float2 mc4 = smul2(s4 * i4, sfma2(7.0f, g[0], smul2(-1.75f, Th)));  // -cn[4]
    const float2 c5 = smul2(-s5 * i5, sub2(smul2(2.0f, g12), add2(g34, g56)));
    const float2 c6 = smul2(-s5 * i6, sub2(g34, g56));
    g[0] = sfma2(-6.0f, mc4, g[0]);
    const float2 ex4 = sfma2(2.0f, c5, mc4), yz4 = sub2(mc4, c5);
    g[1] = add2(g[1], add2(ex4, c1));
    g[2] = add2(g[2], sub2(ex4, c1));
    const float2 ey = add2(yz4, c6), ez = sub2(yz4, c6);
    g[3] = add2(g[3], add2(ey, c2));
    g[4] = add2(g[4], sub2(ey, c2));
    g[5] = add2(g[5], add2(ez, c3));
    g[6] = add2(g[6], sub2(ez, c3));
}

// Even step, pair (x, x + 1): two liquid nodes whose 3x3 columns are liquid
// one node above (no link crosses the phase boundary) collide as in the
// held-solid pair kernel; two solid nodes above every neighbouring liquid
// count (no link crosses it either) conduct as a pair; any other pair takes
// the one-node conduction code node by node.
template <typename ST, int FACE, typename IX>
__device__ __forceinline__ void even_pair_cond(const KP &p, ST *__restrict__ F, ST *__restrict__ G,
                                               const int *__restrict__ js, const int *__restrict__ nb,
                                               const float *__restrict__ gpost, const float *__restrict__ spost,
                                               int x, int y, int z) {
    const int a = axial<FACE>(x, y, z);
    const int col = column<FACE>(p, x, y, z);
    const int nb0 = __ldg(nb + col), nb1 = __ldg(nb + col + 1);
    const IX c = (IX)node_index(p, x, y, z);
    if (a + 1 < (nb0 >> 16) && a + 1 < (nb1 >> 16)) {
        even_pair_liquid<ST, IX>(p, F, G, c);
    } else if (a > (nb0 & 0xffff) && a > (nb1 & 0xffff)) {
        float2 g[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) g[i] = ld_pair(elem<IX>(G, c, i * p.ld));
        collide_solid2(p, g);
#pragma unroll
        for (int i = 0; i < 7; ++i) st_pair(elem<IX>(G, c, opp7(i) * p.ld), g[i]);
    } else {
        even_node<ST, FACE, long long, true>(p, F, G, js, nb, gpost, x, y, z, spost);
        even_node<ST, FACE, long long, true>(p, F, G, js, nb, gpost, x + 1, y, z, spost);
    }
}

template <typename ST, int FACE, typename IX>
__global__ void __launch_bounds__(128, pair_min_blocks<ST>()) k_even_pair_cond(
    const __grid_constant__ KP p, ST *__restrict__ F, ST *__restrict__ G, const int *__restrict__ js,
    const int *__restrict__ nb, const float *__restrict__ gpost, const float *__restrict__ spost) {
    step_launch_wait();
    int x, y, z;
    if (k1_pair<FACE>(p, nullptr, x, y, z)) even_pair_cond<ST, FACE, IX>(p, F, G, js, nb, gpost, spost, x, y, z);
}

// Odd step, pair: off the walls of the heating axis and of the other
// in-plane axis, a liquid pair as odd_pair_liquid, a solid pair above every
// neighbouring liquid count pulls, conducts and pushes its g as a pair (the x
// walls are adiabatic: bounce-back from / into the node's own slots); any
// other pair the one-node conduction code.
template <typename ST, int FACE, typename IX>
__device__ __forceinline__ void odd_pair_cond(const KP &p, const Links *lk, ST *__restrict__ F,
                                              ST *__restrict__ G, const int *__restrict__ js,
                                              const int *__restrict__ nb, const float *__restrict__ gpost,
                                              const float *__restrict__ thw_rd, const float *__restrict__ thw_wr,
                                              const float *__restrict__ spost, int x, int y, int z) {
    const int a = axial<FACE>(x, y, z);
    const int col = column<FACE>(p, x, y, z);
    const int q = FACE == 0 ? z : y, nq = FACE == 0 ? p.nz : p.ny;
    const bool off_qa = q >= 1 && q <= nq - 2 && a >= 1 && a <= p.H - 2;
    const int nb0 = __ldg(nb + col), nb1 = __ldg(nb + col + 1);
    if (off_qa && a + 1 < (nb0 >> 16) && a + 1 < (nb1 >> 16)) {
        odd_pair_liquid<ST, FACE, IX>(p, lk, F, G, x, y, z);
        return;
    }
    if (!(off_qa && a > (nb0 & 0xffff) && a > (nb1 & 0xffff))) {
        odd_node<ST, FACE, true, true>(p, lk, F, G, js, nb, gpost, thw_rd, thw_wr, x, y, z, spost);
        odd_node<ST, FACE, true, true>(p, lk, F, G, js, nb, gpost, thw_rd, thw_wr, x + 1, y, z, spost);
        return;
    }
    const IX c = (IX)node_index(p, x, y, z), c1 = c + 1;
    const bool xlo = x == 0, xhi = x + 1 == p.nx - 1;
    float2 g[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        if (tx(i) == 0) {
            g[i] = ld_pair(elem<IX>(G, c, lk->gin[i]));
        } else {
            g[i].x = Store<ST>::ld(elem<IX>(G, c, tx(i) > 0 && xlo ? i * p.ld : lk->gin[i]));
            g[i].y = Store<ST>::ld(elem<IX>(G, c1, tx(i) < 0 && xhi ? i * p.ld : lk->gin[i]));
        }
    }
    collide_solid2(p, g);
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        if (tx(i) == 0) {
            st_pair(elem<IX>(G, c, lk->gout[i]), g[i]);
        } else {
            Store<ST>::st_stream(elem<IX>(G, c, tx(i) < 0 && xlo ? opp7(i) * p.ld : lk->gout[i]), g[i].x);
            Store<ST>::st_stream(elem<IX>(G, c1, tx(i) > 0 && xhi ? opp7(i) * p.ld : lk->gout[i]), g[i].y);
        }
    }
}

template <typename ST, int FACE, typename IX>
__global__ void __launch_bounds__(128, pair_min_blocks<ST>()) k_odd_pair_cond(
    const __grid_constant__ KP p, ST *__restrict__ F, ST *__restrict__ G, const int *__restrict__ js,
    const int *__restrict__ nb, const float *__restrict__ gpost, const float *__restrict__ thw_rd,
    const float *__restrict__ thw_wr, const __grid_constant__ Links lk, const float *__restrict__ spost) {
    step_launch_wait();
    int x, y, z;
    if (k1_pair<FACE>(p, nullptr, x, y, z))
        odd_pair_cond<ST, FACE, IX>(p, &lk, F, G, js, nb, gpost, thw_rd, thw_wr, spost, x, y, z);
}

// The conduction step's kernels are launched like the plain step's, with
// programmatic stream serialization (see step_launch_wait).
template <typename... KArgs, typename... Args>
static cudaError_t launch_cond_kernel(void (*kern)(KArgs...), dim3 grd, dim3 blk, cudaStream_t st, Args... args) {
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
}

// Two nodes per thread, element indices in IX (32 bits whenever all fit).
template <typename ST, typename IX>
static cudaError_t launch_pair_cond(const KP &p, int face, int odd, const Bufs &b, dim3 g2, dim3 blk, cudaStream_t st) {
    ST *F = (ST *)b.F, *G = (ST *)b.G;
    if (face == 0) {
        if (odd) return launch_cond_kernel(k_odd_pair_cond<ST, 0, IX>, g2, blk, st, p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, b.spost);
        else return launch_cond_kernel(k_even_pair_cond<ST, 0, IX>, g2, blk, st, p, F, G, b.js, b.nb, b.gpost, b.spost);
    } else {
        if (odd) return launch_cond_kernel(k_odd_pair_cond<ST, 1, IX>, g2, blk, st, p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, b.spost);
        else return launch_cond_kernel(k_even_pair_cond<ST, 1, IX>, g2, blk, st, p, F, G, b.js, b.nb, b.gpost, b.spost);
    }
}

template <typename ST>
cudaError_t LaunchCond<ST>::stream_collide(const KP &p, int face, int odd, const Bufs &b, dim3 blk, cudaStream_t st) {
    ST *F = (ST *)b.F, *G = (ST *)b.G;
    if (b.pairs && p.nx % 2 == 0) {
        KP half_x = p;
        half_x.nx = p.nx / 2;
        const dim3 g2 = k1_grid(half_x, blk, face, p.H);
        if (19LL * p.ld < (1LL << 32)) return launch_pair_cond<ST, unsigned>(p, face, odd, b, g2, blk, st);
        return launch_pair_cond<ST, long long>(p, face, odd, b, g2, blk, st);
    }
    const dim3 grd = k1_grid(p, blk, face, p.H);
    if (face == 0) {
        if (odd) return launch_cond_kernel(k_odd_cond<ST, 0>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, b.spost);
        else return launch_cond_kernel(k_even_cond<ST, 0>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, b.spost);
    } else {
        if (odd) return launch_cond_kernel(k_odd_cond<ST, 1>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, b.spost);
        else return launch_cond_kernel(k_even_cond<ST, 1>, grd, blk, st, p, F, G, b.js, b.nb, b.gpost, b.spost);
    }
}

template <typename ST>
cudaError_t LaunchCond<ST>::front(const KP &p, int face, int inflight, int move, const Bufs &b, cudaStream_t st) {
    const dim3 blk(b.cblk), grd = col_grid(p.ncols, b.cblk);
    const ST *F = (const ST *)b.F, *G = (const ST *)b.G;
    if (face == 0)
        return launch_cond_kernel(k_front_cond<ST, 0>, grd, blk, st, p, F, G, b.js, b.js_next, b.s, b.s_next, b.gpost,
                                  b.spost, b.thw_wr, inflight, move, b.status);
    return launch_cond_kernel(k_front_cond<ST, 1>, grd, blk, st, p, F, G, b.js, b.js_next, b.s, b.s_next, b.gpost, b.spost,
                              b.thw_wr, inflight, move, b.status);
}

template struct LaunchCond<float>;
template struct LaunchCond<__half>;

}  // namespace lbm
