// adjoint.cu -- hand-written adjoint of the melting step (Li, Yang & Zhang,
// arXiv:1604.03478, Eqs. 1-6) for gradients of a function of the final
// front S with respect to the heated-wall temperature field and Ra.
//
// The step is differentiated with the phase flags held at their forward
// values (the map is smooth between flips).  Forward: one step maps the
// natural state (f, g, s) at t to t+1 by collision (Eqs. 1-5; the first
// solid node of each column takes the ghost populations prepared from the
// state at t), pull streaming with the wall rules, the front update (Eq. 6)
// and the flip (a newly liquid node's f is reset to a constant).  Reverse
// step t, from the adjoint at t+1 to the adjoint at t:
//   k_adj_front  Eq. 6 backwards: lambda_s(t+1) -> lambda_s(t), the T of
//                the two stencil nodes at t+1, the wall field, d/d coef;
//   k_adj_node   streaming transposed (a push becomes a gather under the
//                flags of t) and the collision Jacobian transposed, FP32,
//                with d/d s_nu, s_alpha, g*beta in FP64 block partials;
//   k_adj_ghost  the ghost populations of the state at t backwards, and the
//                in-plane slope terms of Eq. 6 gathered from the neighbours.
// k_adj_ghost_front runs the ghost adjoint of t and the front adjoint of
// the step before in one launch.  The forward is recorded with
// sqrt(N)-style checkpoints; each segment is recomputed forward with a
// natural-layout snapshot per step, then reversed.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
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

namespace lbm {

// -------------------------------------------------------------- snapshot
// Natural shifted state of one time level: fh (19 x N, zero at solid nodes)
// then gh (7 x N), FP32, with copies of the fronts s, the liquid counts and
// their 3x3 ranges.  Nodes two or more above the largest liquid count of
// their 3x3 neighbour columns are not written: the reverse sweep reads the
// snapshot of a level only below the liquid count of that level or of the
// level before, which differ by at most one.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_snapshot(const __grid_constant__ KP p, const ST *__restrict__ F, const ST *__restrict__ G,
                                                  const int *__restrict__ js, const int *__restrict__ nb,
                                                  const double *__restrict__ s, const float *__restrict__ thw,
                                                  int inflight, float *__restrict__ out, double *__restrict__ out_s,
                                                  int *__restrict__ out_js, int *__restrict__ out_nb) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z), col = column<FACE>(p, x, y, z);
    const int nbv = nb[col];
    if (a == 0) {  // the column's front, liquid count and neighbourhood range
        out_s[col] = s[col];
        out_js[col] = js[col];
        out_nb[col] = nbv;
    }
    if (a >= (nbv & 0xffff) + 2) return;
    float g[7], f[19];
    gather_g<ST, FACE>(p, G, x, y, z, inflight != 0, thw, g);
    const bool liq = a < js[col];
    if (liq) gather_f<ST, FACE>(p, F, js, x, y, z, inflight != 0, f);
#pragma unroll
    for (int i = 0; i < 19; ++i) out[i * p.N + c] = liq ? f[i] : 0.0f;
#pragma unroll
    for (int i = 0; i < 7; ++i) out[(19 + i) * p.N + c] = g[i];
}

// ------------------------------------------------- collision, transposed
// Given the state (fh, gh) of a liquid node and the adjoint of its
// post-collision populations (lf, lg), return the adjoint of the
// pre-collision populations (of, og) and add d/d s_nu, s_alpha, g*beta.
__device__ __forceinline__ void collide_adjoint(const KP &p, const float (&f)[19], const float (&g)[7],
                                                const float (&lf)[19], const float (&lg)[7], float (&of)[19],
                                                float (&og)[7], float &dsnu, float &dsal, float &dgb) {
    // forward quantities
    const float Th = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
    const float T = Th + p.Ts;
    const float Fz = p.gbeta * (Th - p.dTms);
    float S[9], D[9], m[19];
#pragma unroll
    for (int P = 0; P < 9; ++P) {
        S[P] = f[pf(P)] + f[opp(pf(P))];
        D[P] = f[pf(P)] - f[opp(pf(P))];
    }
    moments_pairs<0>(f[0], S, D, m);
    const float ux = m[3], uy = m[5], uz = m[7] + 0.5f * Fz;
    const float uzF = uz * Fz;
    const float pxx = 2.0f * ux * ux - uy * uy - uz * uz;
    const float pww = uy * uy - uz * uz;
    // adjoint of the moment deltas: A_k = (M lf)_k / |row k|^2
    float Sl[9], Dl[9], Ml[19], A[19];
#pragma unroll
    for (int P = 0; P < 9; ++P) {
        Sl[P] = lf[pf(P)] + lf[opp(pf(P))];
        Dl[P] = lf[pf(P)] - lf[opp(pf(P))];
    }
    moments_pairs<0>(lf[0], Sl, Dl, Ml);
    scale_by_inverse_norms<0>(Ml, A);
    const float se = p.s_e, seps = p.s_eps, sq = p.s_q, snu = p.s_nu, spi = p.s_pi, sm = p.s_m;
    float lm[19];
    lm[1] = -se * A[1];
    lm[2] = -seps * A[2];
    lm[4] = -sq * A[4];
    lm[6] = -sq * A[6];
    lm[8] = -sq * A[8];
    lm[9] = -snu * A[9];
    lm[10] = -spi * A[10];
    lm[11] = -snu * A[11];
    lm[12] = -spi * A[12];
    lm[13] = -snu * A[13];
    lm[14] = -snu * A[14];
    lm[15] = -snu * A[15];
    lm[16] = -sm * A[16];
    lm[17] = -sm * A[17];
    lm[18] = -sm * A[18];
    const float lrho = -11.0f * se * A[1] + 3.0f * seps * A[2];
    const float luu = 19.0f * se * A[1] - 5.5f * seps * A[2];
    const float luzF = 38.0f * (1.0f - 0.5f * se) * A[1] - 11.0f * (1.0f - 0.5f * seps) * A[2] -
                       2.0f * (1.0f - 0.5f * snu) * (A[9] + A[11]) + (1.0f - 0.5f * spi) * (A[10] + A[12]);
    const float lpxx = snu * A[9] - 0.5f * spi * A[10];
    const float lpww = snu * A[11] - 0.5f * spi * A[12];
    const float lxy = snu * A[13], lyz = snu * A[14], lxz = snu * A[15];
    const float lyF = (1.0f - 0.5f * snu) * A[14], lxF = (1.0f - 0.5f * snu) * A[15];
    float lux = -(2.0f / 3.0f) * sq * A[4] + 2.0f * ux * luu + 4.0f * ux * lpxx + uy * lxy + uz * lxz + Fz * lxF;
    float luy = -(2.0f / 3.0f) * sq * A[6] + 2.0f * uy * luu - 2.0f * uy * lpxx + 2.0f * uy * lpww + ux * lxy +
                uz * lyz + Fz * lyF;
    float luz = -(2.0f / 3.0f) * sq * A[8] + 2.0f * uz * luu - 2.0f * uz * lpxx - 2.0f * uz * lpww + uy * lyz +
                ux * lxz + Fz * luzF;
    float lFz = A[7] - (2.0f / 3.0f) * (1.0f - 0.5f * sq) * A[8] + uz * luzF + uy * lyF + ux * lxF;
    dsnu += A[9] * (-(m[9] - pxx) + uzF) + A[11] * (-(m[11] - pww) + uzF) - A[13] * (m[13] - ux * uy) +
            A[14] * (-(m[14] - uy * uz) - 0.5f * uy * Fz) + A[15] * (-(m[15] - ux * uz) - 0.5f * ux * Fz);
    // D3Q7: B_k = (N lg)_k / |row k|^2
    const float n1 = g[1] - g[2], n2 = g[3] - g[4], n3 = g[5] - g[6];
    constexpr float i1 = 1.0f / (float)nnorm(1), i4 = 1.0f / (float)nnorm(4);
    constexpr float i5 = 1.0f / (float)nnorm(5), i6 = 1.0f / (float)nnorm(6);
    const float B1 = (lg[1] - lg[2]) * i1, B2 = (lg[3] - lg[4]) * i1, B3 = (lg[5] - lg[6]) * i1;
    const float B4 = (6.0f * lg[0] - (lg[1] + lg[2] + lg[3] + lg[4] + lg[5] + lg[6])) * i4;
    const float B5 = (2.0f * (lg[1] + lg[2]) - (lg[3] + lg[4] + lg[5] + lg[6])) * i5;
    const float B6 = ((lg[3] + lg[4]) - (lg[5] + lg[6])) * i6;
    const float sa = p.s_alpha;
    float ln[7];
    ln[1] = -sa * B1;
    ln[2] = -sa * B2;
    ln[3] = -sa * B3;
    ln[4] = -p.s_g4 * B4;
    ln[5] = -p.s_g5 * B5;
    ln[6] = -p.s_g5 * B6;
    lux += sa * T * B1;
    luy += sa * T * B2;
    luz += sa * T * B3;
    float lTh = sa * (ux * B1 + uy * B2 + uz * B3) + 0.75f * p.s_g4 * B4;
    dsal += -((n1 - ux * T) * B1 + (n2 - uy * T) * B2 + (n3 - uz * T) * B3);
    // through u_z = j_z + F/2 and F = g beta (T - Tm)
    lFz += 0.5f * luz;
    lTh += p.gbeta * lFz;
    dgb += (Th - p.dTms) * lFz;
    lm[0] = lrho;
    lm[3] = lux;
    lm[5] = luy;
    lm[7] = luz;
    ln[0] = lTh;
#pragma unroll
    for (int i = 0; i < 19; ++i) of[i] = lf[i];
    of[0] = pcol_all<0, 0, false>(lm, of[0]);
    add_back_pairs_all<0>(of, lm);
#pragma unroll
    for (int i = 0; i < 7; ++i) og[i] = lg[i];
    add_back7_all<0>(og, ln);
}

// Temperature of node j of column col in a snapshot; cn receives its index.
// Summed in FP32 in the order of the forward's front update (the snapshot
// holds the values it read), so the recomputed gradient is the forward's.
template <int FACE>
__device__ __forceinline__ float snap_T(const KP &p, const float *snap, int col, int j, long long &cn) {
    int x, y, z;
    column_node<FACE>(p, col, j, x, y, z);
    cn = node_index(p, x, y, z);
    float t = 0.0f;
    for (int i = 0; i < 7; ++i) t += snap[(19 + i) * p.N + cn];
    return p.Ts + t;
}

// The slopes s_p, s_q of column c' read the fronts of its neighbours (with a
// mirror at the side walls); the sum of their d/d s for column col.
__device__ __forceinline__ double slope_terms(const KP &p, const double *__restrict__ wp,
                                              const double *__restrict__ wq, int col) {
    const int P1 = p.P1, P2 = p.P2;
    const int pp = col % P1, q = col / P1;
    double acc = 0.0;
    if (P1 > 1) {
        if (pp >= 1) acc += 0.5 * wp[col - 1];       // column pp-1 reads s[pp] as its upper neighbour
        if (pp <= P1 - 2) acc -= 0.5 * wp[col + 1];  // column pp+1 reads s[pp] as its lower neighbour
        if (pp == 0) acc -= 0.5 * wp[col];           // mirror: s[-1] = s[0]
        if (pp == P1 - 1) acc += 0.5 * wp[col];      // mirror: s[P1] = s[P1-1]
    }
    if (P2 > 1) {
        if (q >= 1) acc += 0.5 * wq[col - P1];
        if (q <= P2 - 2) acc -= 0.5 * wq[col + P1];
        if (q == 0) acc -= 0.5 * wq[col];
        if (q == P2 - 1) acc += 0.5 * wq[col];
    }
    return acc;
}

// ----------------------------------------- streaming and collision, reversed
// The adjoint of a solid node other than the ghost node is zero.  Nodes three
// or more above the largest liquid count of their 3x3 neighbour columns are
// not written: the buffer already holds zero there.  It was zeroed before the
// sweep and then holds the adjoint of two levels later (or zero, by the same
// argument), which is nonzero only up to the liquid count of that level
// (ghost node) or one above the count of the level between (front terms);
// liquid counts change by at most one per step (|ds| <= 1/2, else the run
// stops as unstable), so both bounds lie below the skipped nodes.
template <int FACE>
__global__ void __launch_bounds__(128) k_adj_node(const __grid_constant__ KP p, const float *__restrict__ snap, const int *__restrict__ js,
                                                  const int *__restrict__ nb, const float *__restrict__ lam1,
                                                  float *__restrict__ lam0, float *__restrict__ lgpost,
                                                  double *__restrict__ lthw, double *__restrict__ part) {
    __shared__ double sh[3][128];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    float dsnu = 0.0f, dsal = 0.0f, dgb = 0.0f;
    int liquid = 0;
    if (x < p.nx && y < p.ny) {
        const long long c = node_index(p, x, y, z);
        const long long N = p.N;
        const int a = axial<FACE>(x, y, z), col = column<FACE>(p, x, y, z);
        const int jsc = js[col];
        liquid = a < jsc;
        // heated-wall link: the node next to the wall receives
        // -g*_opp + 2 w (Tw - Tm) along the heating axis
        if (a == 0) {
            const int iin = FACE == 0 ? 3 : 5;
            lthw[col] += 2.0 * (double)w7(iin) * (double)lam1[(19 + iin) * N + c];
        }
        if (a > jsc) {
            if (a < (nb[col] & 0xffff) + 3) {
#pragma unroll
                for (int i = 0; i < 26; ++i) lam0[i * N + c] = 0.0f;
            }
        } else {
            // g*: every node streams g; the transpose of the pull is a gather
            float lg[7];
            lg[0] = lam1[19 * N + c];
#pragma unroll
            for (int i = 1; i < 7; ++i) {
                if (inside(p, x + tx(i), y + ty(i), z + tz(i))) {
                    lg[i] = lam1[(19 + i) * N + c + off7<FACE>(p, i)];
                } else {
                    const int w = wall_of_link<FACE>(i);
                    const float v = lam1[(19 + opp7(i)) * N + c];
                    lg[i] = w == 3 ? v : -v;
                }
            }
            if (a == jsc) {  // ghost node: its post-collision g came from the ghost rule
#pragma unroll
                for (int i = 0; i < 7; ++i) lgpost[(long long)i * p.ncols + col] = lg[i];
#pragma unroll
                for (int i = 0; i < 26; ++i) lam0[i * N + c] = 0.0f;
            } else {
                float lf[19], f[19], g[7], of[19], og[7];
                lf[0] = lam1[c];
#pragma unroll
                for (int i = 1; i < 19; ++i) {
                    if (liquid_at<FACE>(p, js, x + ex(i), y + ey(i), z + ez(i)))
                        lf[i] = lam1[i * N + c + off19<FACE>(p, i)];
                    else
                        lf[i] = lam1[opp(i) * N + c];
                }
#pragma unroll
                for (int i = 0; i < 19; ++i) f[i] = snap[i * N + c];
#pragma unroll
                for (int i = 0; i < 7; ++i) g[i] = snap[(19 + i) * N + c];
                collide_adjoint(p, f, g, lf, lg, of, og, dsnu, dsal, dgb);
#pragma unroll
                for (int i = 0; i < 19; ++i) lam0[i * N + c] = of[i];
#pragma unroll
                for (int i = 0; i < 7; ++i) lam0[(19 + i) * N + c] = og[i];
            }
        }
    }
    // blocks without a liquid node add nothing to the rate partials
    if (!__syncthreads_or(liquid)) return;
    sh[0][tid] = dsnu;
    sh[1][tid] = dsal;
    sh[2][tid] = dgb;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (tid < w) {
            sh[0][tid] += sh[0][tid + w];
            sh[1][tid] += sh[1][tid + w];
            sh[2][tid] += sh[2][tid + w];
        }
        __syncthreads();
    }
    if (tid < 3) {
        const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        part[b * 3 + tid] += sh[tid][0];
    }
}

// ------------------------------------- column adjoints (Eq. 6, ghost node)
// Two per-column pieces of a reverse step, run in one thread:
//
// ghost (level t): g*_ghost = w (T_ghost - Tm) + N^T D^-1 (I - Q)(n_L -
// n^eq_L), with T_ghost on the line through (s, Tm) and the guarded node (or
// the wall), taken backwards; also the in-plane slope terms of Eq. 6 that
// the neighbour columns computed, gathered into lambda_s(t).
//
// front (step t-1 -> t): Eq. 6 backwards, lambda_s(t) -> lambda_s(t-1), the
// temperature adjoint of the two stencil nodes at t, the slope partials
// wp/wq (d/d s of the neighbours' slopes), the wall field and d/d coef.
//
// All loads that depend only on the column, the fronts and the liquid count
// are issued before the first store; the population adjoint of every node
// touched (ghost source, guarded node, two stencil nodes; some may coincide)
// is read once, the contributions for that node summed, and stored.
struct ColIn {
    // ghost
    int jn, kg;
    double sn, slope;
    float lTG;
    float lgp[7];
    long long ck, cL;
    float Tk;
    float fL[19], gL[7];
    // front
    int k;
    double sc;
    float sp, sq, y0, y1;
    long long c1, c0;
};

template <int FACE, bool GHOST, bool FRONT>
__device__ __forceinline__ void adj_column(const KP &p, int col, const float *__restrict__ snap,
                                           const int *__restrict__ js, const double *__restrict__ s,
                                           const double *__restrict__ s_prev, const float *__restrict__ thw,
                                           const float *__restrict__ lgpost, float *__restrict__ lam,
                                           double *__restrict__ lams, double *__restrict__ lams_prev,
                                           double *__restrict__ lthw, double *__restrict__ lsal,
                                           double *__restrict__ lgb, double *__restrict__ lcoef,
                                           const double *__restrict__ wp, const double *__restrict__ wq,
                                           double *__restrict__ wp_prev, double *__restrict__ wq_prev) {
    const int H = p.H, P1 = p.P1, P2 = p.P2;
    const long long N = p.N;
    // FP32 arithmetic as in the forward front update; the adjoint of the
    // front (lambda_s) and the parameter and wall sums accumulate in FP64
    const float Tm = p.Tm, Tw = thw[col];
    const int pp = col % P1, q = col / P1;
    ColIn in;
    in.jn = H;
    in.kg = -1;
    in.ck = in.cL = -1;
    in.k = -1;
    in.c1 = in.c0 = -1;
    // ---- loads (everything this column reads, issued before the first
    // store: the compiler cannot move a load of lam or of a per-column sum
    // above a store through another pointer, and each such wait is a
    // memory round trip of a latency-bound kernel)
    const double lams_in = lams[col];
    const double lsal0 = GHOST ? lsal[col] : 0.0, lgb0 = GHOST ? lgb[col] : 0.0;
    const double lcoef0 = FRONT ? lcoef[col] : 0.0, lthw0 = lthw[col];
    float lamf[19];
    // stage 1: what depends on the column only
    if (GHOST) {
        in.slope = slope_terms(p, wp, wq, col);
        in.jn = js[col];
        in.sn = s[col];
        in.lTG = 0.0f;
#pragma unroll
        for (int i = 0; i < 7; ++i) {
            in.lgp[i] = lgpost[(long long)i * p.ncols + col];
            in.lTG = __fmaf_rn(w7(i), in.lgp[i], in.lTG);
        }
    }
    if (FRONT) {
        in.sc = s_prev[col];
        in.sp = 0.5f * (float)(s_prev[q * P1 + (pp + 1 < P1 ? pp + 1 : pp)] - s_prev[q * P1 + (pp > 0 ? pp - 1 : pp)]);
        in.sq = 0.5f * (float)(s_prev[(q + 1 < P2 ? q + 1 : q) * P1 + pp] - s_prev[(q > 0 ? q - 1 : q) * P1 + pp]);
    }
    // stage 2: the nodes the column touches (ghost source, guarded node, two
    // stencil nodes), all loads issued unconditionally from indices clamped
    // into the column (a node that is not needed is read and ignored), so
    // that no load waits behind a branch
    const bool g_on = GHOST && in.jn < H;
    if (g_on) in.kg = guarded_node(in.sn, H);
    if (FRONT) in.k = guarded_node(in.sc, H);
    const bool hasL = g_on && in.jn >= 1, hasK = g_on && in.kg >= 0;
    const bool has1 = FRONT && in.k >= 0, has0 = FRONT && in.k >= 1;
    auto node_of = [&](int j) {
        int x, y, z;
        column_node<FACE>(p, col, j < 0 ? 0 : j, x, y, z);
        return node_index(p, x, y, z);
    };
    const long long eL = node_of(in.jn - 1), eK = node_of(in.kg), e1 = node_of(in.k), e0 = node_of(in.k - 1);
    float gK[7], g1[7], g0[7];
    if (GHOST) {
#pragma unroll
        for (int i = 0; i < 7; ++i) in.gL[i] = snap[(19 + i) * N + eL];
#pragma unroll
        for (int i = 0; i < 19; ++i) in.fL[i] = snap[i * N + eL];
#pragma unroll
        for (int i = 0; i < 19; ++i) lamf[i] = lam[i * N + eL];
#pragma unroll
        for (int i = 0; i < 7; ++i) gK[i] = snap[(19 + i) * N + eK];
    }
    if (FRONT) {
#pragma unroll
        for (int i = 0; i < 7; ++i) g1[i] = snap[(19 + i) * N + e1];
#pragma unroll
        for (int i = 0; i < 7; ++i) g0[i] = snap[(19 + i) * N + e0];
    }
    // the g adjoint of the four nodes (clamped as above)
    const long long eff[4] = {eL, eK, e1, e0};
    float base[4][7];
#pragma unroll
    for (int e = 0; e < 4; ++e)
        if (e < 2 ? GHOST : FRONT) {
#pragma unroll
            for (int i = 0; i < 7; ++i) base[e][i] = lam[(19 + i) * N + eff[e]];
        }
    // temperatures summed in the order of the forward's front update
    auto tsum = [&](const float (&g)[7]) {
        float t = 0.0f;
#pragma unroll
        for (int i = 0; i < 7; ++i) t += g[i];
        return p.Ts + t;
    };
    if (hasL) in.cL = eL;
    if (hasK) { in.ck = eK; in.Tk = tsum(gK); }
    in.y0 = Tw;
    if (has1) { in.c1 = e1; in.y1 = tsum(g1); }
    if (has0) { in.c0 = e0; in.y0 = tsum(g0); }
    long long nd[4] = {in.cL, in.ck, in.c1, in.c0};
    float add[4][7];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int i = 0; i < 7; ++i) add[e][i] = 0.0f;
    float fadd[19];
    double dthw = 0.0;
    double Ls = lams_in;  // lambda_s of level t, completed below
    // ---- ghost, backwards
    if (GHOST) {
        Ls += in.slope;
        if (in.jn < H) {
            const double sn = in.sn, yg = in.jn + 0.5;
            const float lTG = in.lTG, dy = (float)(yg - sn);
            if (in.kg < 0) {
                const float is = __fdiv_rn(1.0f, (float)sn);
                dthw += (double)(-__fmul_rn(__fmul_rn(dy, is), lTG));
                Ls += (double)__fmul_rn(__fmul_rn(__fsub_rn(Tm, Tw), __fmul_rn(__fmul_rn(-(float)yg, is), is)), lTG);
            } else {
                const double yk = in.kg + 0.5;
                const float id = __fdiv_rn(1.0f, (float)(sn - yk)), r = __fmul_rn(dy, id);
                const float lTk = -__fmul_rn(r, lTG);
#pragma unroll
                for (int i = 0; i < 7; ++i) add[1][i] = lTk;
                Ls += (double)__fmul_rn(__fmul_rn(__fsub_rn(Tm, in.Tk), __fmul_rn(__fmul_rn(-(float)(yg - yk), id), id)),
                                        lTG);
            }
            if (in.jn >= 1) {
                const float *gL = in.gL, *fL = in.fL, *lgp = in.lgp;
                float Th = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
                for (int i = 0; i < 7; ++i) Th += gL[i];
#pragma unroll
                for (int i = 0; i < 19; ++i) { jx += ex(i) * fL[i]; jy += ey(i) * fL[i]; jz += ez(i) * fL[i]; }
                const float TL = Th + p.Ts;
                const float ux = jx, uy = jy, uz = jz + 0.5f * p.gbeta * (Th - p.dTms);
                constexpr float i1 = 1.0f / (float)nnorm(1), i4 = 1.0f / (float)nnorm(4);
                constexpr float i5 = 1.0f / (float)nnorm(5), i6 = 1.0f / (float)nnorm(6);
                const float Nl1 = lgp[1] - lgp[2], Nl2 = lgp[3] - lgp[4], Nl3 = lgp[5] - lgp[6];
                const float Nl4 = 6.0f * lgp[0] - (lgp[1] + lgp[2] + lgp[3] + lgp[4] + lgp[5] + lgp[6]);
                const float Nl5 = 2.0f * (lgp[1] + lgp[2]) - (lgp[3] + lgp[4] + lgp[5] + lgp[6]);
                const float Nl6 = (lgp[3] + lgp[4]) - (lgp[5] + lgp[6]);
                // rounded one by one (no contraction): the kernels running this
                // part (with and without the front part) agree bit for bit
                const float d1 = __fsub_rn(gL[1] - gL[2], __fmul_rn(ux, TL));
                const float d2 = __fsub_rn(gL[3] - gL[4], __fmul_rn(uy, TL));
                const float d3 = __fsub_rn(gL[5] - gL[6], __fmul_rn(uz, TL));
                lsal[col] = lsal0 + -(double)__fmul_rn(
                    i1, __fadd_rn(__fadd_rn(__fmul_rn(Nl1, d1), __fmul_rn(Nl2, d2)), __fmul_rn(Nl3, d3)));
                const float ra = 1.0f - p.s_alpha, r4 = 1.0f - p.s_g4, r5 = 1.0f - p.s_g5;
                float mu[7];
                mu[0] = 0.0f;
                mu[1] = ra * i1 * Nl1;
                mu[2] = ra * i1 * Nl2;
                mu[3] = ra * i1 * Nl3;
                mu[4] = r4 * i4 * Nl4;
                mu[5] = r5 * i5 * Nl5;
                mu[6] = r5 * i6 * Nl6;
                const float lux = -mu[1] * TL, luy = -mu[2] * TL, luz = -mu[3] * TL;
                const float lTh = __fadd_rn(
                    __fsub_rn(-__fadd_rn(__fadd_rn(__fmul_rn(mu[1], ux), __fmul_rn(mu[2], uy)), __fmul_rn(mu[3], uz)),
                              __fmul_rn(0.75f, mu[4])),
                    __fmul_rn(__fmul_rn(0.5f, p.gbeta), luz));
                lgb[col] = __dadd_rn(lgb0, __dmul_rn(0.5 * (double)(Th - p.dTms), (double)luz));
                float og[7];
#pragma unroll
                for (int i = 0; i < 7; ++i) og[i] = lTh;
                add_back7_all<0>(og, mu);
#pragma unroll
                for (int i = 0; i < 7; ++i) add[0][i] = og[i];
#pragma unroll
                for (int i = 0; i < 19; ++i) fadd[i] = ex(i) * lux + ey(i) * luy + ez(i) * luz;
            }
        }
        lams[col] = Ls;
    }
    // ---- front of the step before, backwards (lambda_s of level t = Ls)
    if (FRONT) {
        const double sc = in.sc;
        const float sp = in.sp, sq = in.sq;
        const int k = in.k;
        // G and the speed exactly as the forward computes them (the clamp
        // test below must agree with the forward's); the derivatives through
        // reciprocals.  Operations rounded one by one here too: the kernels
        // that run this (with and without the ghost part) then agree.
        const float G = front_gradient(k, sc, in.y0, in.y1, Tm, Tw);
        float dGds, dGdy0 = 0.0f, dGdy1 = 0.0f, dGdTw = 0.0f;
        if (k < 0) {
            const float is = __fdiv_rn(1.0f, (float)sc);
            dGds = __fmul_rn(__fmul_rn(-__fsub_rn(Tm, Tw), is), is);
            dGdTw = -is;
        } else {
            const float y1 = in.y1, y0 = in.y0;
            const double x1 = k + 0.5;
            const double x0 = k >= 1 ? k - 0.5 : 0.0;
            const float d1 = (float)(sc - x1), d0 = (float)(sc - x0);
            const float ih = k >= 1 ? 1.0f : 2.0f;  // h is 1 or 1/2
            const float i0 = __fdiv_rn(1.0f, d0), i1 = __fdiv_rn(1.0f, d1);
            dGdy0 = __fmul_rn(__fmul_rn(d1, ih), i0);
            dGdy1 = -__fmul_rn(__fmul_rn(d0, ih), i1);
            dGds = __fadd_rn(__fmul_rn(__fmul_rn(__fsub_rn(y0, Tm), i0), i0),
                             __fmul_rn(__fmul_rn(__fsub_rn(y1, Tm), i1), i1));
        }
        const float fac = front_slope_factor(sp, sq);
        const float v = front_speed(p, fac, G);
        const double sn = sc + (double)v;
        if (!(sn >= 0.5) || sn > (double)H) {  // clamped: s(t) does not depend on anything
            lams_prev[col] = 0.0;
            wp_prev[col] = 0.0;
            wq_prev[col] = 0.0;
            nd[2] = nd[3] = -1;
        } else {
            const float af = __fmul_rn(p.coef_f, fac);  // d v / d(-G)
            const float La = __fmul_rn((float)Ls, af);  // lambda times that
            const float vG = __fmul_rn(__fmul_rn(p.coef_f, -G), 2.0f);
            lams_prev[col] = __dsub_rn(Ls, __dmul_rn(Ls, (double)__fmul_rn(af, dGds)));
            wp_prev[col] = Ls * (double)__fmul_rn(vG, sp);
            wq_prev[col] = Ls * (double)__fmul_rn(vG, sq);
            lcoef[col] = __dadd_rn(lcoef0, __dmul_rn(Ls, (double)__fmul_rn(fac, -G)));
            if (k >= 0) {
                const float lT1 = -__fmul_rn(La, dGdy1);
#pragma unroll
                for (int i = 0; i < 7; ++i) add[2][i] = lT1;
                if (k >= 1) {
                    const float lT0 = -__fmul_rn(La, dGdy0);
#pragma unroll
                    for (int i = 0; i < 7; ++i) add[3][i] = lT0;
                } else {
                    dthw += (double)(-__fmul_rn(La, dGdy0));
                }
            } else {
                dthw += (double)(-__fmul_rn(La, dGdTw));
            }
        }
    }
    // ---- stores: each touched node gets its base plus every contribution
    // aimed at it (coinciding entries store the same value)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        if (nd[e] < 0) continue;
        float v[7];
#pragma unroll
        for (int i = 0; i < 7; ++i) v[i] = base[e][i];
#pragma unroll
        for (int o = 0; o < 4; ++o)
            if (nd[o] == nd[e]) {
#pragma unroll
                for (int i = 0; i < 7; ++i) v[i] += add[o][i];
            }
#pragma unroll
        for (int i = 0; i < 7; ++i) lam[(19 + i) * N + nd[e]] = v[i];
    }
    if (GHOST && in.cL >= 0) {
#pragma unroll
        for (int i = 0; i < 19; ++i) lam[i * N + in.cL] = lamf[i] + fadd[i];
    }
    if (dthw != 0.0) lthw[col] = lthw0 + dthw;
}

// Front adjoint of the step t -> t+1 alone (top of a segment): snap and lam
// of level t+1, lambda_s(t+1) in lams1, lambda_s(t) and the slope partials
// of level t out.
template <int FACE>
__global__ void __launch_bounds__(128) k_adj_front(const __grid_constant__ KP p, const float *__restrict__ snap1,
                                                   const double *__restrict__ s, const float *__restrict__ thw,
                                                   double *__restrict__ lams1, double *__restrict__ lams0,
                                                   double *__restrict__ wp, double *__restrict__ wq,
                                                   float *__restrict__ lam1, double *__restrict__ lthw,
                                                   double *__restrict__ lcoef) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= p.ncols) return;
    adj_column<FACE, false, true>(p, col, snap1, nullptr, nullptr, s, thw, nullptr, lam1, lams1, lams0, lthw, nullptr,
                                  nullptr, lcoef, nullptr, nullptr, wp, wq);
}

// Ghost adjoint of level t alone (t = 0 of a segment).
template <int FACE>
__global__ void __launch_bounds__(128) k_adj_ghost(const __grid_constant__ KP p, const float *__restrict__ snap,
                                                   const int *__restrict__ js, const double *__restrict__ s,
                                                   const float *__restrict__ thw, const float *__restrict__ lgpost,
                                                   float *__restrict__ lam0, double *__restrict__ lams0,
                                                   double *__restrict__ lthw, double *__restrict__ lsal,
                                                   double *__restrict__ lgb, const double *__restrict__ wp,
                                                   const double *__restrict__ wq) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= p.ncols) return;
    adj_column<FACE, true, false>(p, col, snap, js, s, nullptr, thw, lgpost, lam0, lams0, nullptr, lthw, lsal, lgb,
                                  nullptr, wp, wq, nullptr, nullptr);
}

// The ghost adjoint of level t, then the front adjoint of the step t-1 -> t
// for the same column: the latter needs lambda_s of level t only in its own
// column, adds to the level-t population adjoint only in its own column and
// writes its slope partials to the other of two buffers (the neighbours'
// ghost adjoints still read the level-t ones), so one launch does both.
template <int FACE>
__global__ void __launch_bounds__(128) k_adj_ghost_front(
    const __grid_constant__ KP p, const float *__restrict__ snap, const int *__restrict__ js,
    const double *__restrict__ s, const double *__restrict__ s_prev, const float *__restrict__ thw,
    const float *__restrict__ lgpost, float *__restrict__ lam0, double *__restrict__ lams0,
    double *__restrict__ lams_prev, double *__restrict__ lthw, double *__restrict__ lsal, double *__restrict__ lgb,
    double *__restrict__ lcoef, const double *__restrict__ wp, const double *__restrict__ wq,
    double *__restrict__ wp_prev, double *__restrict__ wq_prev) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= p.ncols) return;
    adj_column<FACE, true, true>(p, col, snap, js, s, s_prev, thw, lgpost, lam0, lams0, lams_prev, lthw, lsal, lgb,
                                 lcoef, wp, wq, wp_prev, wq_prev);
}

// Deterministic FP64 sum of n values (one block), times scale, added to *out.
__global__ void __launch_bounds__(256) k_sum_into(const double *__restrict__ v, long long n, long long stride,
                                                  double *__restrict__ out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) acc += v[i * stride];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out += sh[0];
}

// Checkpoint copy of a state whose deep solid nodes are skipped (Tc = Tm):
// only the heights below the running maximum liquid count + 3 are copied
// (every node that is not deep, and so every slot the method reads, lies
// there; the slots above are never read until they have been written again
// by the steps that follow), with the small per-column arrays.  dir = 0
// saves (the bound from *jmax, recorded at `bound` in the checkpoint), dir =
// 1 restores with the recorded bound.  F and G live at offsets offF, offG of
// the checkpoint, the small arrays at off[k] (byte sizes sz[k]).
struct CkptSmall {
    unsigned char *dev[7];
    size_t off[7], sz[7];
};
template <typename ST, int FACE>
__global__ void __launch_bounds__(256) k_ckpt_move(const __grid_constant__ KP p, ST *__restrict__ F,
                                                   ST *__restrict__ G, unsigned char *__restrict__ buf,
                                                   size_t offF, size_t offG, const __grid_constant__ CkptSmall sm,
                                                   const int *__restrict__ jmax, int *__restrict__ bound, int dir) {
    int b;
    if (dir == 0) {
        b = *jmax + 3;
        b = b > p.H ? p.H : (b < 1 ? 1 : b);
        if (blockIdx.x == 0 && threadIdx.x == 0) *bound = b;
    } else {
        b = *bound;
    }
    ST *cF = (ST *)(buf + offF), *cG = (ST *)(buf + offG);
    const long long plane = FACE == 0 ? (long long)b * p.nx : (long long)b * p.nx * p.ny;  // per z-plane (face 0) or prefix
    const long long per_dir = FACE == 0 ? plane * p.nz : plane;
    const long long total = 26 * per_dir;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int i = (int)(e / per_dir);
        const long long r = e - (long long)i * per_dir;
        const long long node = FACE == 0 ? (r / plane) * (long long)p.ny * p.nx + r % plane : r;
        ST *st = i < 19 ? F + (long long)i * p.ld + node : G + (long long)(i - 19) * p.ld + node;
        ST *ck = i < 19 ? cF + (long long)i * p.ld + node : cG + (long long)(i - 19) * p.ld + node;
        if (dir == 0) *ck = *st;
        else *st = *ck;
    }
    for (int k = 0; k < 7; ++k) {
        unsigned int *a = (unsigned int *)sm.dev[k], *c = (unsigned int *)(buf + sm.off[k]);
        const long long n = (long long)(sm.sz[k] / 4);
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
            if (dir == 0) c[e] = a[e];
            else a[e] = c[e];
        }
    }
}

}  // namespace lbm

// ------------------------------------------------------------------ tape

struct lbm_tape {
    long long T, C, nseg;
    long long thw_gen;               // the handle's wall-field generation when recorded
    size_t ck_bytes, ck_bound_off;
    std::vector<void *> ck;          // device checkpoints, one per segment (in the workspace's pool)
    std::vector<int> ck_cur, ck_inflight;
    std::vector<long long> ck_steps;
};

// The adjoint's device buffers, kept with the handle from one gradient to
// the next (a loop of gradients of one run length allocates once): the
// checkpoint pool of the recorded run and the work buffers of the backward,
// by slot.  A slot is reallocated when a request's size differs; released by
// lbm_melt_tape_clear and lbm_melt_destroy.
struct AdjWorkspace {
    static const int kSlots = 32;
    void *p[kSlots] = {};
    size_t b[kSlots] = {};
};

namespace {

AdjWorkspace *workspace(lbm_melt *h) {
    if (!h->adj_ws) h->adj_ws = new (std::nothrow) AdjWorkspace();
    return (AdjWorkspace *)h->adj_ws;
}

// Device buffer of `bytes` in workspace slot k (the cached one when it has
// that size).
cudaError_t ws_alloc(lbm_melt *h, int k, size_t bytes, void **out) {
    AdjWorkspace *w = workspace(h);
    if (!w) return cudaErrorMemoryAllocation;
    if (w->p[k] && w->b[k] == bytes) {
        *out = w->p[k];
        return cudaSuccess;
    }
    if (w->p[k]) {
        cudaFree(w->p[k]);
        w->p[k] = nullptr;
        w->b[k] = 0;
    }
    const cudaError_t e = cudaMalloc(&w->p[k], bytes);
    if (e != cudaSuccess) {
        w->p[k] = nullptr;
        *out = nullptr;
        return e;
    }
    w->b[k] = bytes;
    *out = w->p[k];
    return cudaSuccess;
}

void free_workspace(lbm_melt *h) {
    AdjWorkspace *w = (AdjWorkspace *)h->adj_ws;
    if (!w) return;
    cudaStreamSynchronize(h->stream);
    for (int k = 0; k < AdjWorkspace::kSlots; ++k)
        if (w->p[k]) cudaFree(w->p[k]);
    delete w;
    h->adj_ws = nullptr;
}

// Workspace slots: 0 the checkpoint pool, 1.. the backward's buffers.
const int kSlotCheckpoints = 0, kSlotBackward = 1;

lbm_status tape_err(lbm_melt *h, lbm_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof h->err, fmt, ap);
    va_end(ap);
    return st;
}

#define TCK(call, where)                                                                                   \
    do {                                                                                                   \
        cudaError_t e_ = (call);                                                                           \
        if (e_ != cudaSuccess)                                                                             \
            return tape_err(h, e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", where,  \
                            cudaGetErrorString(e_));                                                       \
    } while (0)

// Layout of a checkpoint: the nine state arrays of a handle, each starting
// on a 256-byte boundary.  Returns the total size; dev/sz/off describe them.
size_t state_layout(const lbm_melt *h, void *dev[9], size_t sz[9], size_t off[9]) {
    const size_t es = h->precision == 1 ? 2 : 4, nc = (size_t)h->kp.ncols;
    void *d[9] = {h->F, h->G, h->js[0], h->js[1], h->nb[0], h->nb[1], h->s[0], h->s[1], h->gpost};
    const size_t b[9] = {19 * (size_t)h->kp.ld * es, 7 * (size_t)h->kp.ld * es, nc * 4, nc * 4, nc * 4, nc * 4,
                         nc * 8, nc * 8, 7 * nc * 4};
    size_t o = 0;
    for (int k = 0; k < 9; ++k) {
        if (dev) dev[k] = d[k];
        if (sz) sz[k] = b[k];
        if (off) off[k] = o;
        o += (b[k] + 255) / 256 * 256;
    }
    return o;
}

// copy the handle's state to (dir = 0) or from (dir = 1) a checkpoint buffer
lbm_status move_state(lbm_melt *h, unsigned char *buf, int dir) {
    void *dev[9];
    size_t sz[9], off[9];
    state_layout(h, dev, sz, off);
    for (int k = 0; k < 9; ++k) {
        void *a = dev[k], *b = buf + off[k];
        TCK(cudaMemcpyAsync(dir ? a : b, dir ? b : a, sz[k], cudaMemcpyDeviceToDevice, h->stream), "state copy");
    }
    return LBM_OK;
}

// Save (dir = 0) or restore (dir = 1) a checkpoint: with the deep solid
// skipped (Tc = Tm), one kernel copying the heights below the running
// maximum liquid count + 3 (k_ckpt_move; the bound is recorded at byte
// `boff` of the checkpoint); else the whole state.
lbm_status move_checkpoint(lbm_melt *h, unsigned char *buf, size_t boff, int dir) {
    if (!h->kp.skip_deep) return move_state(h, buf, dir);
    void *dev[9];
    size_t sz[9], off[9];
    state_layout(h, dev, sz, off);
    lbm::CkptSmall sm;
    for (int k = 0; k < 7; ++k) {
        sm.dev[k] = (unsigned char *)dev[2 + k];
        sm.off[k] = off[2 + k];
        sm.sz[k] = sz[2 + k];
    }
    const int blocks = 4 * h->sms;
    int *bound = (int *)(buf + boff);
    if (h->precision == 1) {
        __half *F = (__half *)h->F, *G = (__half *)h->G;
        if (h->face == 0)
            lbm::k_ckpt_move<__half, 0><<<blocks, 256, 0, h->stream>>>(h->kp, F, G, buf, off[0], off[1], sm, h->jmax_dev, bound, dir);
        else
            lbm::k_ckpt_move<__half, 1><<<blocks, 256, 0, h->stream>>>(h->kp, F, G, buf, off[0], off[1], sm, h->jmax_dev, bound, dir);
    } else {
        float *F = (float *)h->F, *G = (float *)h->G;
        if (h->face == 0)
            lbm::k_ckpt_move<float, 0><<<blocks, 256, 0, h->stream>>>(h->kp, F, G, buf, off[0], off[1], sm, h->jmax_dev, bound, dir);
        else
            lbm::k_ckpt_move<float, 1><<<blocks, 256, 0, h->stream>>>(h->kp, F, G, buf, off[0], off[1], sm, h->jmax_dev, bound, dir);
    }
    TCK(cudaGetLastError(), "checkpoint copy");
    return LBM_OK;
}

void free_tape(lbm_melt *h) {
    lbm_tape *t = (lbm_tape *)h->tape;
    if (!t) return;
    cudaStreamSynchronize(h->stream);
    delete t;
    h->tape = nullptr;
}

}  // namespace

void lbm_tape_free(lbm_melt *h) {
    free_tape(h);
    free_workspace(h);
}

LBM_API lbm_status lbm_melt_tape_forward(lbm_melt *h, long long steps, long long ckpt_every) {
    if (!h) return LBM_EINVAL;
    if (steps < 1) return tape_err(h, LBM_EINVAL, "steps must be >= 1");
    if (h->kp.cond)
        return tape_err(h, LBM_EINVAL, "the adjoint differentiates the method with the solid held at Tm "
                                       "(no heat conduction in the solid)");
    if (h->thw_pending)
        return tape_err(h, LBM_EINVAL, "set the heated-wall field before recording (no change may be pending)");
    if (ckpt_every <= 0) {
        // about sqrt(steps), rounded up to whole step graphs (lbm_melt_step
        // replays graph_steps steps at a time; a remainder runs step by step)
        ckpt_every = (long long)std::ceil(std::sqrt((double)steps));
        const long long G = h->graph_steps;
        if (G > 1 && ckpt_every < steps) ckpt_every = std::min(steps, (ckpt_every + G - 1) / G * G);
    }
    free_tape(h);
    lbm_tape *t = new (std::nothrow) lbm_tape();
    if (!t) return LBM_ENOMEM;
    h->tape = t;
    t->T = steps;
    t->C = ckpt_every;
    t->thw_gen = h->thw_gen;
    t->nseg = (steps + ckpt_every - 1) / ckpt_every;
    t->ck_bound_off = state_layout(h, nullptr, nullptr, nullptr);
    t->ck_bytes = t->ck_bound_off + 256;  // + the recorded height bound
    void *pool = nullptr;
    {
        const cudaError_t e = ws_alloc(h, kSlotCheckpoints, (size_t)t->nseg * t->ck_bytes, &pool);
        if (e != cudaSuccess) {
            free_tape(h);
            return tape_err(h, LBM_ENOMEM, "%lld checkpoints: %s", t->nseg, cudaGetErrorString(e));
        }
    }
    for (long long sgm = 0; sgm < t->nseg; ++sgm) {
        void *buf = (unsigned char *)pool + (size_t)sgm * t->ck_bytes;
        t->ck.push_back(buf);
        t->ck_cur.push_back(h->cur);
        t->ck_inflight.push_back(h->inflight);
        t->ck_steps.push_back(h->steps);
        lbm_status st = move_checkpoint(h, (unsigned char *)buf, t->ck_bound_off, 0);
        if (st != LBM_OK) return st;
        const long long n = std::min(ckpt_every, steps - sgm * ckpt_every);
        st = lbm_melt_step(h, n);
        if (st != LBM_OK) return st;
    }
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_tape_clear(lbm_melt *h) {
    if (!h) return LBM_EINVAL;
    free_tape(h);
    free_workspace(h);
    return LBM_OK;
}

LBM_API lbm_status lbm_melt_tape_backward(lbm_melt *h, const double *seed, double *dL_dTh, double *dL_dparams,
                                          int ptr_kind) {
    if (!h || !seed) return LBM_EINVAL;
    lbm_tape *t = (lbm_tape *)h->tape;
    if (!t) return tape_err(h, LBM_EINVAL, "no recorded run (call lbm_melt_tape_forward first)");
    if (t->thw_gen != h->thw_gen)
        return tape_err(h, LBM_EINVAL, "the heated-wall field changed after the recorded run; record it again");
    // the sweep relies on fronts that move at most half a node per step
    {
        const lbm_status s0 = lbm_check_status(h);
        if (s0 != LBM_OK) return s0;
    }
    const lbm::KP &p = h->kp;
    const size_t N = (size_t)p.N, nc = (size_t)p.ncols;
    const long long C = t->C;
    const dim3 blk = lbm::node_block(p);
    const dim3 grd_all = lbm::node_grid(p, blk);
    const size_t nblk = (size_t)grd_all.x * grd_all.y * grd_all.z;
    // Every level of the recorded run has liquid counts at most the running
    // maximum; the snapshot and the node adjoint touch nothing three or more
    // nodes above it (deep solid), so their grids stop there.
    int abound = p.H;
    if (p.skip_deep) {
        int jm = 0;
        if (cudaMemcpy(&jm, h->jmax_dev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return tape_err(h, LBM_ECUDA, "liquid-count maximum");
        abound = std::min(p.H, jm + 3);
    }
    const dim3 grd = lbm::node_grid_axial(p, blk, h->face, abound);
    const int cb = h->cblk;
    const dim3 cgrid = lbm::col_grid((long long)nc, cb);
    // buffers; the snapshots of a segment twice, so that one segment's
    // recomputation fills one set while the previous segment's reverse sweep
    // reads the other
    unsigned char *fin = nullptr;
    float *snapb[2] = {nullptr, nullptr}, *lam[2] = {nullptr, nullptr}, *lgpost = nullptr;
    double *snap_sb[2] = {nullptr, nullptr}, *lams[2] = {nullptr, nullptr}, *wp[2] = {nullptr, nullptr},
           *wq[2] = {nullptr, nullptr};
    double *lthw = nullptr;
    double *part = nullptr, *lsal = nullptr, *lgb = nullptr, *lcoef = nullptr, *acc = nullptr;
    int *snap_jsb[2] = {nullptr, nullptr}, *snap_nbb[2] = {nullptr, nullptr};
    struct Alloc { void **p; size_t b; } al[] = {
        {(void **)&fin, t->ck_bytes}, {(void **)&snapb[0], (size_t)(C + 1) * 26 * N * 4},
        {(void **)&snap_sb[0], (size_t)(C + 1) * nc * 8}, {(void **)&snap_jsb[0], (size_t)(C + 1) * nc * 4},
        {(void **)&snap_nbb[0], (size_t)(C + 1) * nc * 4},
        {(void **)&lam[0], 26 * N * 4}, {(void **)&lam[1], 26 * N * 4}, {(void **)&lgpost, 7 * nc * 4},
        {(void **)&lams[0], nc * 8}, {(void **)&lams[1], nc * 8}, {(void **)&wp[0], nc * 8}, {(void **)&wq[0], nc * 8},
        {(void **)&wp[1], nc * 8}, {(void **)&wq[1], nc * 8},
        {(void **)&lthw, nc * 8}, {(void **)&part, nblk * 3 * 8}, {(void **)&lsal, nc * 8},
        {(void **)&lgb, nc * 8}, {(void **)&lcoef, nc * 8}, {(void **)&acc, 4 * 8}};
    lbm_status st = LBM_OK;
    // the buffers stay in the handle's workspace for the next gradient; on
    // an error they are released
    auto cleanup = [&]() {};
    const int nal = (int)(sizeof al / sizeof al[0]);
    for (int k = 0; k < nal; ++k) {
        cudaError_t e = ws_alloc(h, kSlotBackward + k, al[k].b, al[k].p);
        if (e != cudaSuccess) {
            free_workspace(h);
            return tape_err(h, LBM_ENOMEM, "adjoint buffers: %s", cudaGetErrorString(e));
        }
    }
    // the second snapshot set if the device has room for it (else the
    // segments run one after another through the first)
    int nsets = 2;
    {
        const int k2 = kSlotBackward + nal;
        if (ws_alloc(h, k2, (size_t)(C + 1) * 26 * N * 4, (void **)&snapb[1]) != cudaSuccess ||
            ws_alloc(h, k2 + 1, (size_t)(C + 1) * nc * 8, (void **)&snap_sb[1]) != cudaSuccess ||
            ws_alloc(h, k2 + 2, (size_t)(C + 1) * nc * 4, (void **)&snap_jsb[1]) != cudaSuccess ||
            ws_alloc(h, k2 + 3, (size_t)(C + 1) * nc * 4, (void **)&snap_nbb[1]) != cudaSuccess) {
            (void)cudaGetLastError();
            AdjWorkspace *w = workspace(h);
            for (int k = k2; k < k2 + 4; ++k)
                if (w->p[k]) { cudaFree(w->p[k]); w->p[k] = nullptr; w->b[k] = 0; }
            snapb[1] = nullptr;
            snap_sb[1] = nullptr;
            snap_jsb[1] = nullptr;
            snap_nbb[1] = nullptr;
            nsets = 1;
        }
    }
#define BCK(call, where)                                                             \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            cleanup();                                                               \
            return tape_err(h, LBM_ECUDA, "%s: %s", where, cudaGetErrorString(e_));  \
        }                                                                            \
    } while (0)
    // the final state is restored at the end
    const int fin_cur = h->cur, fin_inflight = h->inflight;
    const long long fin_steps = h->steps;
    if ((st = move_state(h, fin, 0)) != LBM_OK) { cleanup(); return st; }
    for (auto &a : al)
        if (a.p != (void **)&fin && a.p != (void **)&snapb[0] && a.p != (void **)&snapb[1])
            BCK(cudaMemsetAsync(*a.p, 0, a.b, h->stream), "zero");
    if (nsets == 2) {
        BCK(cudaMemsetAsync(snap_sb[1], 0, (size_t)(C + 1) * nc * 8, h->stream), "zero");
        BCK(cudaMemsetAsync(snap_jsb[1], 0, (size_t)(C + 1) * nc * 4, h->stream), "zero");
        BCK(cudaMemsetAsync(snap_nbb[1], 0, (size_t)(C + 1) * nc * 4, h->stream), "zero");
    }
    BCK(cudaMemcpyAsync(lams[1], seed, nc * 8, ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        h->stream), "seed");
    // A segment's recomputation: snapshot of its first level, then the
    // recomputed steps with a snapshot after each, into snapshot set b, on
    // stream sm from phase (cur, inflight), the stream-collide grids cut at
    // the run's height bound.  It reads and writes the handle's state.
    const float *thw = h->thw_cur;
    auto enqueue_recompute = [&](long long len, int cur, int inflight, int b, cudaStream_t sm) -> cudaError_t {
        float *snap = snapb[b];
        double *snap_s = snap_sb[b];
        int *snap_js = snap_jsb[b], *snap_nb = snap_nbb[b];
        auto snapshot = [&](long long j) {
            float *out = snap + (size_t)j * 26 * N;
            double *os = snap_s + (size_t)j * nc;
            int *ojs = snap_js + (size_t)j * nc, *onb = snap_nb + (size_t)j * nc;
            const int *js = h->js[cur], *nbv = h->nb[cur];
            const double *sv = h->s[cur];
            if (h->precision == 1) {
                const __half *F = (const __half *)h->F, *G = (const __half *)h->G;
                if (h->face == 0) lbm::k_snapshot<__half, 0><<<grd, blk, 0, sm>>>(p, F, G, js, nbv, sv, thw, inflight, out, os, ojs, onb);
                else lbm::k_snapshot<__half, 1><<<grd, blk, 0, sm>>>(p, F, G, js, nbv, sv, thw, inflight, out, os, ojs, onb);
            } else {
                const float *F = (const float *)h->F, *G = (const float *)h->G;
                if (h->face == 0) lbm::k_snapshot<float, 0><<<grd, blk, 0, sm>>>(p, F, G, js, nbv, sv, thw, inflight, out, os, ojs, onb);
                else lbm::k_snapshot<float, 1><<<grd, blk, 0, sm>>>(p, F, G, js, nbv, sv, thw, inflight, out, os, ojs, onb);
            }
            return cudaGetLastError();
        };
        cudaError_t e = snapshot(0);
        for (long long j = 1; j <= len && e == cudaSuccess; ++j) {
            e = lbm_enqueue_step(h, cur, inflight, abound, sm);
            if (e == cudaSuccess) e = snapshot(j);
        }
        return e;
    };
    // A segment's reverse sweep over its levels from snapshot set b, on
    // stream sm; it reads only the snapshots and the adjoint buffers, which
    // alternate as the levels go by.
    auto enqueue_reverse = [&](long long len, int b, cudaStream_t sm, float *(&lm)[2], double *(&lms)[2]) -> cudaError_t {
        const float *snap = snapb[b];
        const double *snap_s = snap_sb[b];
        const int *snap_js = snap_jsb[b], *snap_nb = snap_nbb[b];
        cudaError_t e = cudaSuccess;
        for (long long j = len - 1; j >= 0 && e == cudaSuccess; --j) {
            const float *s1 = snap + (size_t)(j + 1) * 26 * N, *s0 = snap + (size_t)j * 26 * N;
            const double *st_s = snap_s + (size_t)j * nc;
            const int *st_js = snap_js + (size_t)j * nc;
            const int *st_nb = snap_nb + (size_t)j * nc;
            // Level j: the front adjoint of step j -> j+1 (run by the
            // previous iteration's fused launch, except at the top of the
            // segment), the node adjoint, then the ghost adjoint fused with
            // the front adjoint of step j-1 -> j (alone at j = 0).
            const int pj = (int)(j & 1), pm = pj ^ 1;
            const double *st_s_prev = j > 0 ? snap_s + (size_t)(j - 1) * nc : nullptr;
            if (h->face == 0) {
                if (j == len - 1)
                    lbm::k_adj_front<0><<<cgrid, cb, 0, sm>>>(p, s1, st_s, thw, lms[1], lms[0], wp[pj], wq[pj], lm[1], lthw, lcoef);
                lbm::k_adj_node<0><<<grd, blk, 0, sm>>>(p, s0, st_js, st_nb, lm[1], lm[0], lgpost, lthw, part);
                if (j > 0)
                    lbm::k_adj_ghost_front<0><<<cgrid, cb, 0, sm>>>(p, s0, st_js, st_s, st_s_prev, thw, lgpost, lm[0], lms[0], lms[1], lthw, lsal, lgb, lcoef, wp[pj], wq[pj], wp[pm], wq[pm]);
                else
                    lbm::k_adj_ghost<0><<<cgrid, cb, 0, sm>>>(p, s0, st_js, st_s, thw, lgpost, lm[0], lms[0], lthw, lsal, lgb, wp[pj], wq[pj]);
            } else {
                if (j == len - 1)
                    lbm::k_adj_front<1><<<cgrid, cb, 0, sm>>>(p, s1, st_s, thw, lms[1], lms[0], wp[pj], wq[pj], lm[1], lthw, lcoef);
                lbm::k_adj_node<1><<<grd, blk, 0, sm>>>(p, s0, st_js, st_nb, lm[1], lm[0], lgpost, lthw, part);
                if (j > 0)
                    lbm::k_adj_ghost_front<1><<<cgrid, cb, 0, sm>>>(p, s0, st_js, st_s, st_s_prev, thw, lgpost, lm[0], lms[0], lms[1], lthw, lsal, lgb, lcoef, wp[pj], wq[pj], wp[pm], wq[pm]);
                else
                    lbm::k_adj_ghost<1><<<cgrid, cb, 0, sm>>>(p, s0, st_js, st_s, thw, lgpost, lm[0], lms[0], lthw, lsal, lgb, wp[pj], wq[pj]);
            }
            e = cudaGetLastError();
            std::swap(lm[0], lm[1]);
            std::swap(lms[0], lms[1]);
        }
        return e;
    };
    // The recomputation of a segment (stream A: the handle's stream, which
    // owns the state) and the reverse sweep of the segment after it (stream
    // B) do not share data, so they run at the same time on the two snapshot
    // sets; events order each set's writer after its previous reader.
    // Full-length segments run the same launches from the same phase (and
    // the same parity of the alternating adjoint buffers), so each
    // combination is captured into a CUDA graph once and replayed: the
    // host's launches would otherwise bound small cavities.
    struct SegGraph { int kind, a, b, c; cudaGraphExec_t exec; };
    std::vector<SegGraph> seg_graphs;
    float *const lam0_first = lam[0];
    cudaStream_t sB = nullptr;
    cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr}, ev_set = nullptr;
    auto free_graphs = [&]() {
        for (auto &g : seg_graphs) cudaGraphExecDestroy(g.exec);
        seg_graphs.clear();
        for (int i = 0; i < 2; ++i) {
            if (ev_rec[i]) cudaEventDestroy(ev_rec[i]);
            if (ev_rev[i]) cudaEventDestroy(ev_rev[i]);
        }
        if (ev_set) cudaEventDestroy(ev_set);
        if (sB) cudaStreamDestroy(sB);
    };
    if (!h->cap_stream) BCK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "capture stream");
    BCK(cudaStreamCreateWithFlags(&sB, cudaStreamNonBlocking), "reverse stream");
    for (int i = 0; i < 2; ++i) {
        BCK(cudaEventCreateWithFlags(&ev_rec[i], cudaEventDisableTiming), "event");
        BCK(cudaEventCreateWithFlags(&ev_rev[i], cudaEventDisableTiming), "event");
    }
    BCK(cudaEventCreateWithFlags(&ev_set, cudaEventDisableTiming), "event");
    // the reverse stream starts after the zeroed buffers and the seed
    BCK(cudaEventRecord(ev_set, h->stream), "event");
    BCK(cudaStreamWaitEvent(sB, ev_set, 0), "wait");
    // a cached graph for (kind, a, b, c), else capture it from enqueue()
    auto graph_of = [&](int kind, int a, int b, int c, const auto &enqueue, cudaGraphExec_t *out) -> cudaError_t {
        for (auto &g : seg_graphs)
            if (g.kind == kind && g.a == a && g.b == b && g.c == c) { *out = g.exec; return cudaSuccess; }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            e = enqueue(h->cap_stream);
            const cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &graph);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e == cudaSuccess) seg_graphs.push_back({kind, a, b, c, *out});
        return e;
    };
    bool used[2] = {false, false};
    for (long long sgm = t->nseg - 1; sgm >= 0 && st == LBM_OK; --sgm) {
        const long long len = std::min(C, t->T - sgm * C);
        const int b = nsets == 2 ? (int)(sgm & 1) : 0;
        const bool full = len == C && t->nseg > 2;
        cudaError_t e = cudaSuccess;
        // stream A: the set's previous reader done, restore the checkpoint,
        // recompute into the set
        if (used[b]) e = cudaStreamWaitEvent(h->stream, ev_rev[b], 0);
        if (e == cudaSuccess && (st = move_checkpoint(h, (unsigned char *)t->ck[sgm], t->ck_bound_off, 1)) != LBM_OK)
            break;
        const int cur0 = t->ck_cur[sgm], infl0 = t->ck_inflight[sgm];
        h->steps = t->ck_steps[sgm];
        if (e == cudaSuccess) {
            if (full) {
                cudaGraphExec_t exec = nullptr;
                e = graph_of(0, cur0, infl0, b,
                             [&](cudaStream_t sm) { return enqueue_recompute(len, cur0, infl0, b, sm); }, &exec);
                if (e == cudaSuccess) e = cudaGraphLaunch(exec, h->stream);
            } else {
                e = enqueue_recompute(len, cur0, infl0, b, h->stream);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_rec[b], h->stream);
        // stream B: reverse the segment once its snapshots are in
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sB, ev_rec[b], 0);
        if (e == cudaSuccess) {
            if (full) {
                const int par = lam[0] == lam0_first ? 0 : 1;
                cudaGraphExec_t exec = nullptr;
                e = graph_of(1, par, b, 0,
                             [&](cudaStream_t sm) {
                                 float *lm[2] = {lam[0], lam[1]};
                                 double *lms[2] = {lams[0], lams[1]};
                                 return enqueue_reverse(len, b, sm, lm, lms);
                             }, &exec);
                if (e == cudaSuccess) e = cudaGraphLaunch(exec, sB);
                if (len & 1) {
                    std::swap(lam[0], lam[1]);
                    std::swap(lams[0], lams[1]);
                }
            } else {
                e = enqueue_reverse(len, b, sB, lam, lams);
            }
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_rev[b], sB);
        used[b] = true;
        if (e != cudaSuccess) st = tape_err(h, LBM_ECUDA, "adjoint segment: %s", cudaGetErrorString(e));
    }
    // the sums below run on stream A after the last reverse sweep
    if (st == LBM_OK) {
        cudaError_t e = cudaEventRecord(ev_set, sB);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, ev_set, 0);
        if (e != cudaSuccess) st = tape_err(h, LBM_ECUDA, "adjoint join: %s", cudaGetErrorString(e));
    }
    if (st == LBM_OK) {
        // parameter sensitivities: acc = {d/ds_nu, d/ds_alpha, d/dcoef, d/dgbeta}
        lbm::k_sum_into<<<1, 256, 0, h->stream>>>(part, (long long)nblk, 3, acc);
        lbm::k_sum_into<<<1, 256, 0, h->stream>>>(part + 1, (long long)nblk, 3, acc + 1);
        lbm::k_sum_into<<<1, 256, 0, h->stream>>>(lsal, (long long)nc, 1, acc + 1);
        lbm::k_sum_into<<<1, 256, 0, h->stream>>>(lcoef, (long long)nc, 1, acc + 2);
        lbm::k_sum_into<<<1, 256, 0, h->stream>>>(part + 2, (long long)nblk, 3, acc + 3);
        lbm::k_sum_into<<<1, 256, 0, h->stream>>>(lgb, (long long)nc, 1, acc + 3);
        double a[4] = {0, 0, 0, 0};
        cudaError_t e = cudaMemcpyAsync(a, acc, sizeof a, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && dL_dTh)
            e = cudaMemcpyAsync(dL_dTh, lthw, nc * 8, ptr_kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = tape_err(h, LBM_ECUDA, "adjoint outputs: %s", cudaGetErrorString(e));
        if (st == LBM_OK && dL_dparams) {
            // chain to Ra: with derive_from_Ra, nu = U0 H sqrt(Pr/Ra), alpha = nu/Pr,
            // s_nu = 1/(3 nu + 1/2), s_alpha = 1/(4 alpha + 1/2), coef = alpha Ste/(Th - Tm)
            // and g beta = U0^2 / (H (Th - Tm)) does not depend on Ra; with given
            // rates only g beta = Ra nu alpha / ((Th - Tm) H^3) does.
            const Derived &d = h->d;
            double dRa = 0.0;
            if (h->derived_from_Ra) {
                const double Ra = h->Ra;
                dRa = a[0] * 3.0 * d.s_nu * d.s_nu * d.nu / (2.0 * Ra) + a[1] * 2.0 * d.s_alpha * d.s_alpha * d.alpha / Ra -
                      a[2] * p.coef / (2.0 * Ra);
            } else if (h->Ra > 0.0) {
                dRa = a[3] * d.gbeta / h->Ra;
            }
            const double out[5] = {dRa, a[0], a[1], a[2], a[3]};
            if (ptr_kind) {
                if (cudaMemcpy(dL_dparams, out, sizeof out, cudaMemcpyHostToDevice) != cudaSuccess)
                    st = tape_err(h, LBM_ECUDA, "copy parameters");
            } else {
                std::memcpy(dL_dparams, out, sizeof out);
            }
        }
    }
    // restore the final state (after everything on both streams)
    if (sB) cudaStreamSynchronize(sB);
    lbm_status st2 = move_state(h, fin, 1);
    h->cur = fin_cur;
    h->inflight = fin_inflight;
    h->steps = fin_steps;
    cudaStreamSynchronize(h->stream);
    free_graphs();
    cleanup();
    return st != LBM_OK ? st : st2;
}
