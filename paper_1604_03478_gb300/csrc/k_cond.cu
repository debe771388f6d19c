// k_cond.cu -- the stream-collide and front kernels with heat conduction in
// the solid (Eq. 6's k_s term), for both storage types.  Every node is
// updated (no deep-solid skip, no height bound on the grid).
#include "kernels.cuh"
#include "launch.h"

namespace lbm {

template <typename ST>
cudaError_t LaunchCond<ST>::stream_collide(const KP &p, int face, int odd, const Bufs &b, dim3 blk, cudaStream_t st) {
    const dim3 grd = k1_grid(p, blk, face, p.H);
    ST *F = (ST *)b.F, *G = (ST *)b.G;
    if (face == 0) {
        if (odd) k_odd_cond<ST, 0><<<grd, blk, 0, st>>>(p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, b.spost);
        else k_even_cond<ST, 0><<<grd, blk, 0, st>>>(p, F, G, b.js, b.nb, b.gpost, b.spost);
    } else {
        if (odd) k_odd_cond<ST, 1><<<grd, blk, 0, st>>>(p, F, G, b.js, b.nb, b.gpost, b.thw_rd, b.thw_wr, *b.lk, b.spost);
        else k_even_cond<ST, 1><<<grd, blk, 0, st>>>(p, F, G, b.js, b.nb, b.gpost, b.spost);
    }
    return cudaGetLastError();
}

template <typename ST>
cudaError_t LaunchCond<ST>::front(const KP &p, int face, int inflight, int move, const Bufs &b, cudaStream_t st) {
    const dim3 blk(b.cblk), grd = col_grid(p.ncols, b.cblk);
    const ST *F = (const ST *)b.F, *G = (const ST *)b.G;
    if (face == 0)
        k_front_cond<ST, 0><<<grd, blk, 0, st>>>(p, F, G, b.js, b.js_next, b.s, b.s_next, b.gpost, b.spost, b.thw_wr,
                                                 inflight, move, b.status);
    else
        k_front_cond<ST, 1><<<grd, blk, 0, st>>>(p, F, G, b.js, b.js_next, b.s, b.s_next, b.gpost, b.spost, b.thw_wr,
                                                 inflight, move, b.status);
    return cudaGetLastError();
}

template struct LaunchCond<float>;
template struct LaunchCond<__half>;

}  // namespace lbm
