// kernels.cuh -- the device kernels of one time step and of the state I/O,
// templated on the storage type (float or __half) and the heated face.
//
// One step of the method (Li, Yang & Zhang, arXiv:1604.03478, section 2):
//   k_even / k_odd : fused stream + collide of f (D3Q19 MRT, Eqs. 1-3) and
//                    g (D3Q7 MRT, Eqs. 4-5), in place by the AA pattern;
//   k_front        : interfacial tracking, Eq. 6, one thread per column, FP64;
//   k_flip         : phase flip of the nodes the front crossed.
//
// AA pattern.  A step that starts from the natural layout (slot i of node x
// holds f_i(x), "even") reads and writes only node x: the post-collision
// f*_i goes to slot opp(i) of x.  The next step ("odd") pulls f_i(x) from
// slot opp(i) of x - e_i and pushes f*_i to slot i of x + e_i, which brings
// the layout back to natural.  Walls and liquid/solid links are handled on
// the odd step's reads and writes: a missing upstream node means halfway
// bounce-back (read slot i of x itself), a missing downstream node means the
// value stays at x in slot opp(i).  Every node reads and writes the same set
// of slots in a step, so the update is race-free in place.
//
// Between an even and an odd step the post-collision values are "in flight"
// (their streaming is deferred to the odd step).  If the front flips a node
// there, the odd step would read the in-flight values with the new flags;
// k_flip rewrites the two slots of every link touching a flipped node so that
// the new-flag reads deliver exactly what the old flags (and the re-initialised
// f = f^eq(1, 0) of a newly liquid node) prescribe.
#pragma once

#include "lbm_core.cuh"

namespace lbm {

template <int FACE> __device__ __forceinline__ long long off19(const KP &p, int i) {
    return (long long)ex(i) + (long long)ey(i) * p.nx + (long long)ez(i) * p.nx * p.ny;
}
template <int FACE> __device__ __forceinline__ long long off7(const KP &p, int i) {
    return (long long)tx(i) + (long long)ty(i) * p.nx + (long long)tz(i) * p.nx * p.ny;
}

// Post-collision shifted g of a solid node: the ghost node (first solid node
// of its column) takes the populations prepared by k_front; deeper nodes are
// at rest at Tm, i.e. zero.
__device__ __forceinline__ void solid_post(const KP &p, bool ghost, const float *gpost, int col, float (&g)[7]) {
#pragma unroll
    for (int i = 0; i < 7; ++i) g[i] = ghost ? __ldg(gpost + (long long)i * p.ncols + col) : 0.0f;
}

// ------------------------------------------------------------- even step
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_even(KP p, ST *__restrict__ F, ST *__restrict__ G,
                                              const int *__restrict__ js, const float *__restrict__ gpost) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z);
    const int col = column<FACE>(p, x, y, z);
    const int jsc = __ldg(js + col);
    float g[7];
    if (a < jsc) {
        float f[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) f[i] = Store<ST>::ld(F + i * p.ld + c);
#pragma unroll
        for (int i = 0; i < 7; ++i) g[i] = Store<ST>::ld(G + i * p.ld + c);
        collide(p, f, g);
#pragma unroll
        for (int i = 0; i < 19; ++i) Store<ST>::st(F + opp(i) * p.ld + c, f[i]);
    } else {
        solid_post(p, a == jsc, gpost, col, g);
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) Store<ST>::st(G + opp7(i) * p.ld + c, g[i]);
}

// -------------------------------------------------------------- odd step
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_odd(KP p, ST *__restrict__ F, ST *__restrict__ G,
                                             const int *__restrict__ js, const float *__restrict__ gpost,
                                             const float *__restrict__ thw_rd, const float *__restrict__ thw_wr) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z);
    const int col = column<FACE>(p, x, y, z);
    const int jsc = __ldg(js + col);
    float g[7];
    if (a < jsc) {
        float f[19];
        f[0] = Store<ST>::ld(F + c);
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            if (liquid_at<FACE>(p, js, x - ex(i), y - ey(i), z - ez(i)))
                f[i] = Store<ST>::ld(F + opp(i) * p.ld + (c - off19<FACE>(p, i)));
            else  // halfway bounce-back: f*_opp(i) of this node, parked in slot i
                f[i] = Store<ST>::ld(F + i * p.ld + c);
        }
        g[0] = Store<ST>::ld(G + c);
#pragma unroll
        for (int i = 1; i < 7; ++i) {
            if (inside(p, x - tx(i), y - ty(i), z - tz(i))) {
                g[i] = Store<ST>::ld(G + opp7(i) * p.ld + (c - off7<FACE>(p, i)));
            } else {
                const int w = wall_of_link<FACE>(opp7(i));
                const float own = Store<ST>::ld(G + i * p.ld + c);
                if (w == 3) g[i] = own;  // adiabatic: bounce-back
                else g[i] = -own + 2.0f * w7(i) * ((w == 1 ? __ldg(thw_rd + col) : p.Tc) - p.Tm);
            }
        }
        collide(p, f, g);
#pragma unroll
        for (int i = 1; i < 19; ++i) {
            if (liquid_at<FACE>(p, js, x + ex(i), y + ey(i), z + ez(i)))
                Store<ST>::st(F + i * p.ld + (c + off19<FACE>(p, i)), f[i]);
            else
                Store<ST>::st(F + opp(i) * p.ld + c, f[i]);
        }
        Store<ST>::st(F + c, f[0]);
    } else {
        solid_post(p, a == jsc, gpost, col, g);
    }
    Store<ST>::st(G + c, g[0]);
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        if (inside(p, x + tx(i), y + ty(i), z + tz(i))) {
            Store<ST>::st(G + i * p.ld + (c + off7<FACE>(p, i)), g[i]);
        } else {
            const int w = wall_of_link<FACE>(i);
            if (w == 3) Store<ST>::st(G + opp7(i) * p.ld + c, g[i]);
            else Store<ST>::st(G + opp7(i) * p.ld + c,
                               -g[i] + 2.0f * w7(i) * ((w == 1 ? __ldg(thw_wr + col) : p.Tc) - p.Tm));
        }
    }
}

// -------------------------------------------------- state gathers (natural)
// Shifted pre-collision g of node (x,y,z).  In flight: pull from the
// neighbours' slots (walls by their rules with wall field thw); natural:
// the node's own slots.
template <typename ST, int FACE>
__device__ __forceinline__ void gather_g(const KP &p, const ST *G, int x, int y, int z, bool inflight,
                                         const float *thw, float (&g)[7]) {
    const long long c = node_index(p, x, y, z);
    g[0] = Store<ST>::ld(G + c);
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        if (!inflight) {
            g[i] = Store<ST>::ld(G + i * p.ld + c);
        } else if (inside(p, x - tx(i), y - ty(i), z - tz(i))) {
            g[i] = Store<ST>::ld(G + opp7(i) * p.ld + (c - off7<FACE>(p, i)));
        } else {
            const int w = wall_of_link<FACE>(opp7(i));
            const float own = Store<ST>::ld(G + i * p.ld + c);
            g[i] = (w == 3) ? own
                            : -own + 2.0f * w7(i) * ((w == 1 ? thw[column<FACE>(p, x, y, z)] : p.Tc) - p.Tm);
        }
    }
}

// Shifted pre-collision f of a liquid node, with the liquid flags js that
// the in-flight values were produced under.
template <typename ST, int FACE>
__device__ __forceinline__ void gather_f(const KP &p, const ST *F, const int *js, int x, int y, int z,
                                         bool inflight, float (&f)[19]) {
    const long long c = node_index(p, x, y, z);
    f[0] = Store<ST>::ld(F + c);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        if (!inflight) f[i] = Store<ST>::ld(F + i * p.ld + c);
        else if (liquid_at<FACE>(p, js, x - ex(i), y - ey(i), z - ez(i)))
            f[i] = Store<ST>::ld(F + opp(i) * p.ld + (c - off19<FACE>(p, i)));
        else f[i] = Store<ST>::ld(F + i * p.ld + c);
    }
}

template <typename ST, int FACE>
__device__ __forceinline__ double node_T(const KP &p, const ST *G, int col, int j, bool inflight, const float *thw) {
    int x, y, z;
    column_node<FACE>(p, col, j, x, y, z);
    float g[7];
    gather_g<ST, FACE>(p, G, x, y, z, inflight, thw, g);
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < 7; ++i) t += (double)g[i];
    return p.Tm_d + t;
}

// Highest node at least half a cell below s (centre j + 1/2 <= s - 1/2).
__device__ __forceinline__ int guarded_node(double s, int H) {
    int k = (int)floor(s - 1.0);
    return k > H - 1 ? H - 1 : (k < 0 ? -1 : k);
}

// ------------------------------------------------------------ front (Eq. 6)
// One thread per column.  From the state after a step (T of the liquid at
// t + 1, front s_t): the one-sided quadratic gradient at the front, the
// in-plane slopes from the old fronts of the neighbour columns (mirror at
// the side walls), ds/dt = coef (1 + s_p^2 + s_q^2)(-dT/da), the new front
// clamped to [1/2, H], its liquid-node count, and the ghost node of the new
// front: g*_ghost = g^eq(T_ghost, 0) + (g*_L - g^eq(T_L, u_L)).
// move = 0 keeps the front (used to prepare the ghost after a state upload).
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_front(KP p, const ST *__restrict__ F, const ST *__restrict__ G,
                                               const int *__restrict__ js, int *__restrict__ js_next,
                                               const double *__restrict__ s, double *__restrict__ s_next,
                                               float *__restrict__ gpost, const float *__restrict__ thw,
                                               int inflight, int move, int *__restrict__ status) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= p.ncols) return;
    const int P1 = p.P1, P2 = p.P2, H = p.H;
    const int pp = col % P1, q = col / P1;
    const double sc = s[col];
    const double Tm = p.Tm_d;
    const double Tw = (double)thw[col];
    const bool infl = inflight != 0;
    double sn = sc;
    if (move) {
        const double sp = 0.5 * (s[q * P1 + (pp + 1 < P1 ? pp + 1 : pp)] - s[q * P1 + (pp > 0 ? pp - 1 : pp)]);
        const double sq = 0.5 * (s[(q + 1 < P2 ? q + 1 : q) * P1 + pp] - s[(q > 0 ? q - 1 : q) * P1 + pp]);
        const int k = guarded_node(sc, H);
        double Gr;
        if (k < 0) {
            Gr = (Tm - Tw) / sc;
        } else {
            const double x1 = k + 0.5, y1 = node_T<ST, FACE>(p, G, col, k, infl, thw), x2 = sc, y2 = Tm;
            double x0, y0;
            if (k >= 1) { x0 = k - 0.5; y0 = node_T<ST, FACE>(p, G, col, k - 1, infl, thw); }
            else        { x0 = 0.0; y0 = Tw; }
            Gr = y0 * (x2 - x1) / ((x0 - x1) * (x0 - x2)) + y1 * (x2 - x0) / ((x1 - x0) * (x1 - x2))
               + y2 * (2.0 * x2 - x0 - x1) / ((x2 - x0) * (x2 - x1));
        }
        const double v = p.coef * (1.0 + sp * sp + sq * sq) * (-Gr);
        if (!isfinite(Gr)) atomicOr(status, 2);
        else if (!(fabs(v) <= 0.5)) atomicOr(status, 1);
        sn = sc + v;
        if (!(sn >= 0.5)) sn = 0.5;  // also catches NaN
        if (sn > (double)H) sn = (double)H;
    }
    s_next[col] = sn;
    int jn = (int)ceil(sn - 0.5);
    jn = jn < 0 ? 0 : (jn > H ? H : jn);
    js_next[col] = jn;
    if (jn >= H) return;  // fully liquid column: no ghost node
    const double yg = jn + 0.5;
    const int kg = guarded_node(sn, H);
    double Tg;
    if (kg < 0) Tg = Tm + (Tm - Tw) * (yg - sn) / sn;
    else Tg = Tm + (Tm - node_T<ST, FACE>(p, G, col, kg, infl, thw)) * (yg - sn) / (sn - (kg + 0.5));
    double gh[7];
#pragma unroll
    for (int i = 0; i < 7; ++i) gh[i] = (double)w7(i) * (Tg - Tm);
    if (jn >= 1) {
        int x, y, z;
        column_node<FACE>(p, col, jn - 1, x, y, z);
        float gL[7], fL[19];
        gather_g<ST, FACE>(p, G, x, y, z, infl, thw, gL);
        const bool newly_liquid = (jn - 1) >= js[col];
        if (newly_liquid) {
#pragma unroll
            for (int i = 0; i < 19; ++i) fL[i] = 0.0f;
        } else {
            gather_f<ST, FACE>(p, F, js, x, y, z, infl, fL);
        }
        double Th = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
        for (int i = 0; i < 7; ++i) Th += (double)gL[i];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            jx += ex(i) * (double)fL[i];
            jy += ey(i) * (double)fL[i];
            jz += ez(i) * (double)fL[i];
        }
        const double TL = Th + Tm;
        const double ux = jx, uy = jy, uz = jz + 0.5 * (double)p.gbeta * Th;
        double dn[7];
        dn[0] = 0.0;
        dn[1] = ((double)gL[1] - gL[2] - ux * TL) * (1.0 - p.s_alpha) / nnorm(1);
        dn[2] = ((double)gL[3] - gL[4] - uy * TL) * (1.0 - p.s_alpha) / nnorm(2);
        dn[3] = ((double)gL[5] - gL[6] - uz * TL) * (1.0 - p.s_alpha) / nnorm(3);
        dn[4] = (6.0 * gL[0] - ((double)gL[1] + gL[2] + gL[3] + gL[4] + gL[5] + gL[6]) - 0.75 * Th)
              * (1.0 - p.s_g4) / nnorm(4);
        dn[5] = (2.0 * ((double)gL[1] + gL[2]) - ((double)gL[3] + gL[4] + gL[5] + gL[6])) * (1.0 - p.s_g5) / nnorm(5);
        dn[6] = (((double)gL[3] + gL[4]) - ((double)gL[5] + gL[6])) * (1.0 - p.s_g5) / nnorm(6);
#pragma unroll
        for (int i = 0; i < 7; ++i)
#pragma unroll
            for (int kk = 1; kk < 7; ++kk) gh[i] += npoly(kk, i) * dn[kk];
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) gpost[(long long)i * p.ncols + col] = (float)gh[i];
}

// ------------------------------------------------------------------ flip
// Nodes of a column between the old and the new liquid counts changed phase.
// Natural layout: a newly liquid node gets fh = 0 (f = f^eq(1, 0)).
// In flight: every link (x, x - e_i) touching a flipped node has its two
// slots P = slot opp(i) of x - e_i and Q = slot i of x rewritten so that the
// odd step's reads under the new flags deliver the values prescribed by the
// old flags (streaming if the upstream node was liquid, bounce-back if not)
// and zero to a newly liquid node.  A link whose two ends both flipped is
// handled once, by the end with the lower node index.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_flip(KP p, ST *__restrict__ F, const int *__restrict__ js_old,
                                              const int *__restrict__ js_new, int inflight) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= p.ncols) return;
    const int jo = js_old[col], jn = js_new[col];
    if (jo == jn) return;
    const int lo = jo < jn ? jo : jn, hi = jo < jn ? jn : jo;
    for (int j = lo; j < hi; ++j) {
        int x, y, z;
        column_node<FACE>(p, col, j, x, y, z);
        const long long c = node_index(p, x, y, z);
        const bool lx_t = j < jo, lx_n = j < jn;
        if (!inflight) {
            if (lx_n && !lx_t)
                for (int i = 0; i < 19; ++i) Store<ST>::st(F + i * p.ld + c, 0.0f);
            continue;
        }
        if (lx_n && !lx_t) Store<ST>::st(F + c, 0.0f);
        for (int i = 1; i < 19; ++i) {
            const int xn = x - ex(i), yn = y - ey(i), zn = z - ez(i);
            const bool yin = inside(p, xn, yn, zn);
            bool ly_t = false, ly_n = false;
            long long cy = 0;
            if (yin) {
                const int cc = column<FACE>(p, xn, yn, zn), an = axial<FACE>(xn, yn, zn);
                ly_t = an < js_old[cc];
                ly_n = an < js_new[cc];
                cy = node_index(p, xn, yn, zn);
                if (ly_t != ly_n && cy < c) continue;  // the other end owns this link
            }
            ST *Ps = F + opp(i) * p.ld + cy;
            ST *Qs = F + i * p.ld + c;
            const float P = yin ? Store<ST>::ld(Ps) : 0.0f;
            const float Q = Store<ST>::ld(Qs);
            const float dx = !lx_t ? 0.0f : (ly_t ? P : Q);
            const float dy = !ly_t ? 0.0f : (lx_t ? Q : P);
            if (lx_n && ly_n) { Store<ST>::st(Ps, dx); Store<ST>::st(Qs, dy); }
            else if (lx_n) Store<ST>::st(Qs, dx);
            else if (ly_n) Store<ST>::st(Ps, dy);
        }
    }
}

// ----------------------------------------------------- outputs and inputs
// T and u per node (solid: Tm and 0), natural values.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_macro(KP p, const ST *__restrict__ F, const ST *__restrict__ G,
                                               const int *__restrict__ js, const float *__restrict__ thw,
                                               int inflight, float *__restrict__ T, float *__restrict__ u) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z), col = column<FACE>(p, x, y, z);
    float Tc = p.Tm, ux = 0.0f, uy = 0.0f, uz = 0.0f;
    if (a < js[col]) {
        float g[7], f[19];
        gather_g<ST, FACE>(p, G, x, y, z, inflight != 0, thw, g);
        gather_f<ST, FACE>(p, F, js, x, y, z, inflight != 0, f);
        float Th = 0.0f;
#pragma unroll
        for (int i = 0; i < 7; ++i) Th += g[i];
#pragma unroll
        for (int i = 0; i < 19; ++i) { ux += ex(i) * f[i]; uy += ey(i) * f[i]; uz += ez(i) * f[i]; }
        uz += 0.5f * p.gbeta * Th;
        Tc = p.Tm + Th;
    }
    if (T) T[c] = Tc;
    if (u) { u[3 * c] = ux; u[3 * c + 1] = uy; u[3 * c + 2] = uz; }
}

// Natural (unshifted) distributions out, direction-major with stride N.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_state_out(KP p, const ST *__restrict__ F, const ST *__restrict__ G,
                                                   const int *__restrict__ js, const float *__restrict__ thw,
                                                   int inflight, float *__restrict__ fo, float *__restrict__ go) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z), col = column<FACE>(p, x, y, z);
    if (go) {
        float g[7];
        gather_g<ST, FACE>(p, G, x, y, z, inflight != 0, thw, g);
#pragma unroll
        for (int i = 0; i < 7; ++i) go[i * p.N + c] = g[i] + w7(i) * p.Tm;
    }
    if (fo) {
        float f[19];
        const bool liq = a < js[col];
        if (liq) gather_f<ST, FACE>(p, F, js, x, y, z, inflight != 0, f);
#pragma unroll
        for (int i = 0; i < 19; ++i) fo[i * p.N + c] = liq ? f[i] + w19(i) : 0.0f;
    }
}

// Natural distributions in; leaves the natural layout.  Solid nodes get
// fh = 0.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_state_in(KP p, ST *__restrict__ F, ST *__restrict__ G,
                                                  const int *__restrict__ js, const float *__restrict__ fi,
                                                  const float *__restrict__ gi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z), col = column<FACE>(p, x, y, z);
    if (gi)
#pragma unroll
        for (int i = 0; i < 7; ++i) Store<ST>::st(G + i * p.ld + c, gi[i * p.N + c] - w7(i) * p.Tm);
    if (fi) {
        const bool liq = a < js[col];
#pragma unroll
        for (int i = 0; i < 19; ++i) Store<ST>::st(F + i * p.ld + c, liq ? fi[i * p.N + c] - w19(i) : 0.0f);
    }
}

// Initial state: fh = 0 everywhere (rest, rho = 1); gh = w (T(a) - Tm) with
// the given profile below the front, 0 above.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_init(KP p, ST *__restrict__ F, ST *__restrict__ G,
                                              const int *__restrict__ js, const float *__restrict__ Tprof) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z), col = column<FACE>(p, x, y, z);
    const float dT = a < js[col] ? Tprof[a] - p.Tm : 0.0f;
#pragma unroll
    for (int i = 0; i < 19; ++i) Store<ST>::st(F + i * p.ld + c, 0.0f);
#pragma unroll
    for (int i = 0; i < 7; ++i) Store<ST>::st(G + i * p.ld + c, w7(i) * dT);
}

}  // namespace lbm
