// ensemble_kernel.cuh -- the persistent kernel of the batched form (see
// ensemble.cu): its work list, bounded grid barrier and phases.  Included by
// ensemble.cu (host side) and by the ens_*.cu files, which instantiate one
// kernel each so that they compile in parallel.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "kernels.cuh"

// Launch-bound occupancy target of the persistent kernel (blocks of 256
// per SM: 3 caps it at 80 registers a thread, with under 100 bytes of
// spills) and whether the node variants are out-of-line functions.  Measured
// on the 48-cavity workload over 100 steps (before the dynamic tile
// distribution): 3 blocks 14.5 k MLUPS, 2 blocks (up to 128 registers, no
// spills) 13.3 k.  With 8 z-planes per item over 2000 steps: 3 blocks 23.9 k,
// 4 blocks (64 registers, 308 bytes of spills) 23.1 k, a cap of 72
// registers (7 blocks of 128) 23.8 k.
#ifndef LBM_ENS_MINB
#define LBM_ENS_MINB 3
#endif
// LBM_ENS_MAXNREG, when defined, caps the registers directly instead.
#ifdef LBM_ENS_MAXNREG
#define ENS_BOUNDS __maxnreg__(LBM_ENS_MAXNREG)
#else
#define ENS_BOUNDS __launch_bounds__(256, LBM_ENS_MINB)
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
    unsigned int *bar;            // {arrived, generation, timed out, -, item counters (2 x u64),
                                  //  phase times in ns and steps (4 x u64)}
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

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int find_cavity(const long long *begin, int n, long long item) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (begin[mid] <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One node of phase 1, one function per (face, parity) variant (inlined;
// out of line, so that the variants do not share one register allocation,
// when LBM_ENS_NOINLINE is set).  The even step indexes in 32 bits (lbm_ensemble_create admits members whose
// indices fit): 23.4 k against 22.8 k MLUPS over 1000 steps of the 48-cavity
// workload.
template <typename ST, int FACE>
ENS_FN void ens_even(const CavDesc &d, int cur, int x, int y, int z) {
    even_node<ST, FACE, unsigned>(d.p, (ST *)d.F, (ST *)d.G, d.js[cur], d.nb[cur], d.gpost, x, y, z);
}
template <typename ST, int FACE>
ENS_FN void ens_odd(const CavDesc &d, int cur, const float *trd, int x, int y, int z) {
    odd_node<ST, FACE, false>(d.p, nullptr, (ST *)d.F, (ST *)d.G, d.js[cur], d.nb[cur], d.gpost, trd, d.thw, x, y, z);
}

// One column of phase 2 (front update; returns the new liquid count) or 3
// (flip; returns -1).  The front update does not load the ghost's likely
// source node with the gradient stencil (as k_front does): under this
// kernel's register cap that spilled 1.3 KB a thread and slowed every phase
// (19.8 k against 23.2 k MLUPS on the 48-cavity workload).
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
__global__ void ENS_BOUNDS k_ensemble(const __grid_constant__ EnsWork w, int nsteps) {
    const long long items1 = w.item_begin[w.ncav], items2 = w.col_begin[w.ncav];
    __shared__ int top[kMaxCavities];  // per cavity: first height at which every node is deep solid
    __shared__ long long next;         // first item of the block's next chunk
    // per-step item counters (alternating), zeroed with the barrier words
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(w.bar + 4);
    constexpr int kChunk = 1;  // measured: 1, 2, 4 items -> 19.3, 18.7, 18.5 k MLUPS
    int kc = 0;  // cavity of the block's last item (items are handed out in increasing order)
    // Block 0 times the phases on the global timer: each phase ends when
    // block 0 leaves the grid barrier after it (accumulated, with the step
    // count, in the barrier words 8..15 for lbm_ensemble_phase_times).
    unsigned long long *phase_ns = reinterpret_cast<unsigned long long *>(w.bar + 8);
    const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long tp = timer ? global_ns() : 0ull;
    for (int t = 0; t < nsteps; ++t) {
        kc = 0;
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
            if (it >= w.item_begin[kc + 1]) kc += find_cavity(w.item_begin + kc, w.ncav - kc, it);
            const int k = kc;
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
        if (timer) { const unsigned long long tn = global_ns(); phase_ns[0] += tn - tp; tp = tn; }
        // phases 2 and 3: front update (Eq. 6), then flip, of every column.
        // Items are dealt round-robin: consecutive items, which hold
        // neighbouring columns and so much the same amount of flip work, go
        // to different blocks (one contiguous range per block ran the flip
        // phase 67 against 37 us a step on the 48-cavity workload).
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
            if (timer) {
                const unsigned long long tn = global_ns();
                phase_ns[phase - 1] += tn - tp;
                tp = tn;
                if (phase == 3) phase_ns[3] += 1ull;
            }
        }
    }
}

}  // namespace lbm

// One translation unit per instantiation (ens_*.cu) compiles the kernel and
// hands its address to the host code of ensemble.cu.
namespace lbm {
const void *ens_kernel_f32_k1();
const void *ens_kernel_f32_k2();
const void *ens_kernel_f32_k4();
const void *ens_kernel_f32_k8();
const void *ens_kernel_f16_k1();
const void *ens_kernel_f16_k2();
const void *ens_kernel_f16_k4();
const void *ens_kernel_f16_k8();
}  // namespace lbm
