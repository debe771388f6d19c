// launch.h -- host-side launchers of the kernels, one instantiation per
// storage type (k_f32.cu: float, k_f16.cu: __half).  Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "lbm_core.cuh"

namespace lbm {

struct Bufs {
    void *F, *G;                 // shifted distributions, 19 and 7 arrays of ld elements
    const int *js;               // liquid-node count per column (current flags)
    int *js_next;
    const int *nb;               // 3x3 min/max of js (min << 16 | max), current
    int *nb_next;
    const double *s;             // front per column (current)
    double *s_next;
    float *gpost;                // ghost-node post-collision g, 7 x ncols
    const float *thw_rd, *thw_wr;
    int *status;
    const Links *lk;             // interior link offsets of the odd step
    int cblk;                    // threads per block of the per-column kernels (col_block)
    int *jmax;                   // running maximum of the liquid counts (k_front), or null
    int k1_height;               // the stream-collide grid covers heights < k1_height (the rest is deep solid)
    const float *thw_nu;         // heated-wall field of the last streaming (Nusselt number)
    double *nu;                  // per-column Nusselt numbers (ncols)
    double nu_scale;             // H / (alpha (Th - Tm))
    float *spost;                // solid-side ghost populations, 7 x ncols (heat conduction in the solid)
    int pairs;                   // stream-collide with two nodes per thread (even nx)
};

// The stream-collide and front kernels with heat conduction in the solid
// (KP::cond), in a translation unit of their own (k_cond.cu); Launch
// forwards to them.
template <typename ST> struct LaunchCond {
    static cudaError_t stream_collide(const KP &p, int face, int odd, const Bufs &b, dim3 blk, cudaStream_t st);
    static cudaError_t front(const KP &p, int face, int inflight, int move, const Bufs &b, cudaStream_t st);
};

template <typename ST> struct Launch {
    static cudaError_t stream_collide(const KP &p, int face, int odd, const Bufs &b, dim3 blk, cudaStream_t st);
    static cudaError_t front(const KP &p, int face, int inflight, int move, const Bufs &b, cudaStream_t st);
    static cudaError_t flip(const KP &p, int face, int inflight, int do_flip, const Bufs &b, cudaStream_t st);
    static cudaError_t macro(const KP &p, int face, int inflight, const Bufs &b, float *T, float *u, cudaStream_t st);
    static cudaError_t state_out(const KP &p, int face, int inflight, const Bufs &b, float *f, float *g, cudaStream_t st);
    static cudaError_t state_in(const KP &p, int face, const Bufs &b, const float *f, const float *g, cudaStream_t st);
    static cudaError_t init(const KP &p, int face, const Bufs &b, const float *Tprof, cudaStream_t st);
    static cudaError_t totals(const KP &p, int face, int inflight, const Bufs &b, double *part, int nparts,
                              double t, double *out, cudaStream_t st);
    static cudaError_t nusselt(const KP &p, int face, int inflight, const Bufs &b, cudaStream_t st);
};

// Threads per block of the per-column kernels (front, flip and their
// adjoints): the largest of 128, 64 and 32 that still gives two blocks per
// SM, so that a small front (96 x 96 columns) spreads its FP64 arithmetic
// over all SMs instead of half of them.
inline int col_block(long long ncols, int sms) {
    for (int b = 128; b > 32; b >>= 1)
        if ((ncols + b - 1) / b >= 2LL * sms) return b;
    return 32;
}
inline dim3 col_grid(long long ncols, int b) { return dim3((unsigned)((ncols + b - 1) / b)); }

// Block shape for the per-node kernels: 128 threads, x-major.
// Width along x of a block of `block` threads: the power of two from 32 to
// min(block, 128) that leaves the fewest idle lanes over a row of nx nodes
// (the widest on a tie): 160 -> 32, 96 -> 32, 48 -> 64, 256 -> 128.
inline int block_width(int nx, int block) {
    int best = 32;
    long long best_waste = -1;
    for (int bx = 32; bx <= block && bx <= 128; bx *= 2) {
        const long long waste = (long long)((nx + bx - 1) / bx) * bx - nx;
        if (best_waste < 0 || waste <= best_waste) {
            best = bx;
            best_waste = waste;
        }
    }
    return best;
}
inline dim3 node_block(const KP &p) {
    const int bx = block_width(p.nx, 128);
    return dim3(bx, 128 / bx, 1);
}
inline dim3 node_grid(const KP &p, dim3 b) {
    return dim3((p.nx + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, p.nz);
}
// Grid of the stream-collide (k1_node): x tiles, the in-plane tiles, then
// the heights along the heating axis (slowest).
inline dim3 k1_grid(const KP &p, dim3 b, int face, int height) {
    const unsigned gx = (p.nx + b.x - 1) / b.x;
    if (height < 1) height = 1;
    if (face == 0) {
        const unsigned gz = (unsigned)((height + (int)b.y - 1) / (int)b.y), full = (p.ny + b.y - 1) / b.y;
        return dim3(gx, p.nz, gz < full ? gz : full);
    }
    return dim3(gx, (p.ny + b.y - 1) / b.y, (unsigned)(height < p.nz ? height : p.nz));
}

// node_grid cut to the heights a < abound along the heating axis (y for
// face 0, z for face 1).
inline dim3 node_grid_axial(const KP &p, dim3 b, int face, int abound) {
    dim3 g = node_grid(p, b);
    if (abound < 1) abound = 1;
    if (face == 0) {
        const unsigned gy = (unsigned)((abound + (int)b.y - 1) / (int)b.y);
        if (gy < g.y) g.y = gy;
    } else if ((unsigned)abound < g.z) {
        g.z = (unsigned)abound;
    }
    return g;
}

}  // namespace lbm
