// kernels.cuh -- the device kernels of one time step and of the state I/O,
// templated on the storage type (float or __half) and the heated face.
//
// One step of the method (Li, Yang & Zhang, arXiv:1604.03478, section 2):
//   k_even / k_odd : fused stream + collide of f (D3Q19 MRT, Eqs. 1-3) and
//                    g (D3Q7 MRT, Eqs. 4-5), in place by the AA pattern, one
//                    node per thread (k_even_pair / k_odd_pair: two
//                    x-adjacent nodes per thread in packed FP32x2 arithmetic);
//   k_front        : interfacial tracking, Eq. 6, one thread per column (FP64
//                    fronts, FP32 gradient and speed);
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

// Programmatic dependent launch: the kernels of a step are launched so that
// the next one may be scheduled while the previous one drains; each waits
// for its predecessor's completion (and memory) before its first access,
// then lets its own successor be scheduled.  Both are no-ops for a kernel
// launched without the attribute.
__device__ __forceinline__ void step_launch_wait() {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <int FACE> __device__ __forceinline__ long long off19(const KP &p, int i) {
    return (long long)ex(i) + (long long)ey(i) * p.nx + (long long)ez(i) * p.nx * p.ny;
}
template <int FACE> __device__ __forceinline__ long long off7(const KP &p, int i) {
    return (long long)tx(i) + (long long)ty(i) * p.nx + (long long)tz(i) * p.nx * p.ny;
}

// Element offsets of the odd step's interior links: from the table lk (a
// kernel parameter) when TAB, else from the extents.
template <int FACE, bool TAB> __device__ __forceinline__ long long fin_off(const KP &p, const Links *lk, int i) {
    return TAB ? lk->fin[i] : opp(i) * p.ld - off19<FACE>(p, i);
}
template <int FACE, bool TAB> __device__ __forceinline__ long long fout_off(const KP &p, const Links *lk, int i) {
    return TAB ? lk->fout[i] : i * p.ld + off19<FACE>(p, i);
}
template <int FACE, bool TAB> __device__ __forceinline__ long long gin_off(const KP &p, const Links *lk, int i) {
    return TAB ? lk->gin[i] : opp7(i) * p.ld - off7<FACE>(p, i);
}
template <int FACE, bool TAB> __device__ __forceinline__ long long gout_off(const KP &p, const Links *lk, int i) {
    return TAB ? lk->gout[i] : i * p.ld + off7<FACE>(p, i);
}

// Element base[c + off] with the index arithmetic done in IX: unsigned (32
// bits, for states whose every element index fits) or long long.  With
// 32-bit indices a link offset enters the address as one 32-bit add of a
// kernel-parameter operand.
template <typename IX, typename ST>
__device__ __forceinline__ ST *elem(ST *base, IX c, long long off) {
    return base + (IX)(c + (IX)off);
}

// Post-collision shifted g of a solid node: the ghost node (first solid node
// of its column) takes the populations prepared by k_front; deeper nodes are
// at rest at Tm (gh = w (Tm - Ts), zero with FP32 storage).
__device__ __forceinline__ void solid_post(const KP &p, bool ghost, const float *gpost, int col, float (&g)[7]) {
#pragma unroll
    for (int i = 0; i < 7; ++i) g[i] = ghost ? __ldg(gpost + (long long)i * p.ncols + col) : w7(i) * p.dTms;
}

// A solid node at least two nodes above its column's first solid node and
// above every 3x3-neighbour column's first solid node ("deep") has only
// solid neighbours that are not ghost nodes.  Nothing reads its slots while
// it is deep, and one step before the front can reach it, it is no longer
// deep (the 3x3 maximum includes its own column), so with Tc = Tm (the cold
// wall then returns zero too) its update can be skipped exactly.
__device__ __forceinline__ bool deep_solid(const KP &p, int a, int nbv) {
    return p.skip_deep && a >= (nbv & 0xffff) + 2;
}

// ------------------------------------------------- conduction in the solid
// Bit i (1..6): the D3Q7 link leaving node x along t_i ends inside the
// cavity on a node of the other phase (liq: x is liquid).
template <int FACE>
__device__ __forceinline__ unsigned other_phase7(const KP &p, const int *__restrict__ js, int x, int y, int z,
                                                 bool liq) {
    unsigned m = 0;
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        const int xn = x + tx(i), yn = y + ty(i), zn = z + tz(i);
        if (inside(p, xn, yn, zn) && (axial<FACE>(xn, yn, zn) < __ldg(js + column<FACE>(p, xn, yn, zn))) != liq)
            m |= 1u << i;
    }
    return m;
}

// With heat conduction in the solid, a population leaving node x towards a
// node of the other phase (bits of `other`) is not x's own post-collision
// value: it is the ghost population of x's column for the receiving phase
// when x is that ghost (ghost: the first solid node towards the liquid, with
// the liquid side's ghost populations gbuf; the last liquid node towards the
// solid, with the solid side's), else the rest state at Tm.
__device__ __forceinline__ void cross_phase(const KP &p, unsigned other, bool ghost, const float *__restrict__ gbuf,
                                            int col, float (&g)[7]) {
#pragma unroll
    for (int i = 1; i < 7; ++i)
        if ((other >> i) & 1u) g[i] = ghost ? __ldg(gbuf + (long long)i * p.ncols + col) : w7(i) * p.dTms;
}

// ------------------------------------------------------------- even step
// COND: heat conduction in the solid (the solid collides its own g at u = 0
// and the links across the phase boundary carry the ghost or rest values of
// cross_phase; spost holds the solid side's ghost populations).
template <typename ST, int FACE, typename IX = long long, bool COND = false>
__device__ __forceinline__ void even_node(const KP &p, ST *__restrict__ F, ST *__restrict__ G, const int *__restrict__ js,
                                          const int *__restrict__ nb, const float *__restrict__ gpost, int x, int y,
                                          int z, const float *__restrict__ spost = nullptr) {
    const IX c = (IX)node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z);
    const int col = column<FACE>(p, x, y, z);
    const int jsc = __ldg(js + col);
    float g[7];
    if (a < jsc) {
        float f[19];
#pragma unroll
        for (int i = 0; i < 19; ++i) f[i] = Store<ST>::ld(elem<IX>(F, c, i * p.ld));
#pragma unroll
        for (int i = 0; i < 7; ++i) g[i] = Store<ST>::ld(elem<IX>(G, c, i * p.ld));
        collide(p, f, g);
#pragma unroll
        for (int i = 0; i < 19; ++i) Store<ST>::st_stream(elem<IX>(F, c, opp(i) * p.ld), f[i]);
        if (COND && a + 1 >= (__ldg(nb + col) >> 16)) {
            const unsigned other = other_phase7<FACE>(p, js, x, y, z, true);
            if (other) cross_phase(p, other, a == jsc - 1, spost, col, g);
        }
    } else if (COND) {
#pragma unroll
        for (int i = 0; i < 7; ++i) g[i] = Store<ST>::ld(elem<IX>(G, c, i * p.ld));
        collide_solid(p, g);
        if (a <= (__ldg(nb + col) & 0xffff)) {
            const unsigned other = other_phase7<FACE>(p, js, x, y, z, false);
            if (other) cross_phase(p, other, a == jsc, gpost, col, g);
        }
    } else {
        if (deep_solid(p, a, __ldg(nb + col))) return;
        solid_post(p, a == jsc, gpost, col, g);
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) Store<ST>::st_stream(elem<IX>(G, c, opp7(i) * p.ld), g[i]);
}

// Stream-collide grid: blocks of blockDim.x x blockDim.y nodes of one plane
// across the heating axis, with the height along that axis slowest
// (blockIdx.z), so that the blocks near the heated wall are dispatched
// first.  jmax (null: no bound) is the running maximum of the liquid counts,
// written by the previous front update: nodes two or more above every
// neighbouring count are deep solid and do nothing, so a block whose heights
// are all >= jmax + 3 returns at once.
template <int FACE>
__device__ __forceinline__ bool k1_node(const KP &p, const int *jmax, int &x, int &y, int &z) {
    const int a0 = (int)blockIdx.z * (FACE == 0 ? (int)blockDim.y : 1);  // lowest height of the block
    if (jmax && a0 >= *jmax + 3) return false;
    x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (FACE == 0) {
        y = a0 + (int)threadIdx.y;
        z = (int)blockIdx.y;
    } else {
        y = (int)(blockIdx.y * blockDim.y + threadIdx.y);
        z = (int)blockIdx.z;
    }
    return x < p.nx && y < p.ny;
}

// Resident blocks of 128 the stream-collide asks for: 8 (64 registers, a
// few bytes of spills) for FP16 storage, whose warps move half the bytes and
// need more of them in flight (+1.3%); none for FP32 (72 registers, 7
// blocks, no spills; forced to 8 it loses 1%).
template <typename ST> constexpr int k1_min_blocks() { return sizeof(ST) == 2 ? 8 : 0; }

template <typename ST, int FACE, typename IX>
__global__ void __launch_bounds__(128, k1_min_blocks<ST>()) k_even(const __grid_constant__ KP p, ST *__restrict__ F, ST *__restrict__ G,
                                              const int *__restrict__ js, const int *__restrict__ nb,
                                              const float *__restrict__ gpost, const int *jmax) {
    step_launch_wait();
    int x, y, z;
    if (k1_node<FACE>(p, jmax, x, y, z)) even_node<ST, FACE, IX>(p, F, G, js, nb, gpost, x, y, z);
}

// The even step with heat conduction in the solid (every node updated).
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_even_cond(const __grid_constant__ KP p, ST *__restrict__ F, ST *__restrict__ G,
                                                   const int *__restrict__ js, const int *__restrict__ nb,
                                                   const float *__restrict__ gpost, const float *__restrict__ spost) {
    step_launch_wait();
    int x, y, z;
    if (k1_node<FACE>(p, nullptr, x, y, z)) even_node<ST, FACE, long long, true>(p, F, G, js, nb, gpost, x, y, z, spost);
}


// -------------------------------------------------------------- odd step
// Bit i (1..18) of the link mask: node x - e_i is inside and liquid, i.e.
// f_i streams in from there (else halfway bounce-back).  Since x + e_i =
// x - e_opp(i), bit opp(i) tells whether f*_i streams out to x + e_i.
template <int FACE>
__device__ __forceinline__ unsigned link_mask(const KP &p, const int *js, int x, int y, int z) {
    unsigned m = 0;
#pragma unroll
    for (int i = 1; i < 19; ++i)
        if (liquid_at<FACE>(p, js, x - ex(i), y - ey(i), z - ez(i))) m |= 1u << i;
    return m;
}
// Bit i (1..6): node x - t_i is inside (else the link crosses a wall).
__device__ __forceinline__ unsigned inside_mask(const KP &p, int x, int y, int z) {
    unsigned m = 0;
#pragma unroll
    for (int i = 1; i < 7; ++i)
        if (inside(p, x - tx(i), y - ty(i), z - tz(i))) m |= 1u << i;
    return m;
}

// Wall rule for a D3Q7 population leaving along link direction `dir`
// across a wall: adiabatic bounce-back keeps it, the isothermal walls return
// -v + 2 w (Tw - Ts) (anti-bounce-back, shifted populations).
template <int FACE>
__device__ __forceinline__ float wall_value(const KP &p, int dir, float v, float Th_col) {
    const int w = wall_of_link<FACE>(dir);
    return w == 3 ? v : -v + 2.0f * w7(dir) * ((w == 1 ? Th_col : p.Tc) - p.Ts);
}

// Across an x wall (x = 0 for e_x = +1 upstream, x = nx - 1 for e_x = -1):
// the only walls a warp's nodes (32 consecutive x at one height and plane)
// do not all share.
__device__ __forceinline__ bool xwall(int ex_up, bool xlo, bool xhi) {
    return ex_up > 0 ? xlo : (ex_up < 0 ? xhi : false);
}

// TAB: take the interior link offsets from the precomputed tables of KP
// (kernel parameters: constant-bank operands); false computes them from the
// extents, which keeps them out of registers when KP lives in shared memory.
//
// Fast path: a liquid node off the walls of the heating axis and of the
// other in-plane axis and at least one node below the lowest first-solid
// node of its 3x3 neighbour columns, so that every link streams except those
// across an x wall, which bounce back (no-slip for f, adiabatic for g).  The
// x walls are taken by selects inside the fast path, so that the warps that
// hold x = 0 or x = nx - 1 do not split between two paths.
//
// COND: heat conduction in the solid (see even_node).
template <typename ST, int FACE, bool TAB = true, bool COND = false>
__device__ __forceinline__ void odd_node(const KP &p, const Links *lk, ST *__restrict__ F, ST *__restrict__ G, const int *__restrict__ js,
                                         const int *__restrict__ nb, const float *__restrict__ gpost,
                                         const float *__restrict__ thw_rd, const float *__restrict__ thw_wr, int x,
                                         int y, int z, const float *__restrict__ spost = nullptr) {
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z);
    const int col = column<FACE>(p, x, y, z);
    const int jsc = __ldg(js + col);
    const int nbv = __ldg(nb + col);
    const int q = FACE == 0 ? z : y, nq = FACE == 0 ? p.nz : p.ny;
    const bool off_qa = q >= 1 && q <= nq - 2 && a >= 1 && a <= p.H - 2;
    const bool off_walls = off_qa && x >= 1 && x <= p.nx - 2;
    const bool xlo = x == 0, xhi = x == p.nx - 1;
    ST *const Fc = F + c;
    ST *const Gc = G + c;
    float g[7];
    if (a < jsc) {
        const bool fast = off_qa && a + 1 < (nbv >> 16);
        float f[19];
        unsigned lm = 0x7fffeu, im = 0x7eu;
        if (fast) {
#pragma unroll
            for (int i = 0; i < 19; ++i) f[i] = Store<ST>::ld(Fc + fin_off<FACE, TAB>(p, lk, i));
#pragma unroll
            for (int i = 0; i < 7; ++i) g[i] = Store<ST>::ld(Gc + gin_off<FACE, TAB>(p, lk, i));
            // Across an x wall the pull above read the neighbouring row's
            // node instead (an in-bounds element of the same direction array:
            // the node is off the walls of the other two axes); bounce-back
            // replaces it with the value parked in the node's own slot i
            // (no-slip for f, adiabatic for g).
            if (xlo | xhi) {
#pragma unroll
                for (int i = 1; i < 19; ++i)
                    if (xwall(ex(i), xlo, xhi)) f[i] = Store<ST>::ld(Fc + i * p.ld);
#pragma unroll
                for (int i = 1; i < 7; ++i)
                    if (xwall(tx(i), xlo, xhi)) g[i] = Store<ST>::ld(Gc + i * p.ld);
            }
        } else {
            lm = link_mask<FACE>(p, js, x, y, z);
            im = inside_mask(p, x, y, z);
            const float th_rd = __ldg(thw_rd + col);
            f[0] = Store<ST>::ld(Fc);
#pragma unroll
            for (int i = 1; i < 19; ++i)  // else bounce-back: f*_opp(i) parked in slot i
                f[i] = Store<ST>::ld(((lm >> i) & 1u) ? Fc + fin_off<FACE, TAB>(p, lk, i) : Fc + i * p.ld);
            g[0] = Store<ST>::ld(Gc);
#pragma unroll
            for (int i = 1; i < 7; ++i) {
                const bool in = (im >> i) & 1u;
                const float v = Store<ST>::ld(in ? Gc + gin_off<FACE, TAB>(p, lk, i) : Gc + i * p.ld);
                g[i] = in ? v : wall_value<FACE>(p, opp7(i), v, th_rd);
            }
        }
        collide(p, f, g);
        if (fast) {
            Store<ST>::st_stream(Fc, f[0]);
#pragma unroll
            for (int i = 1; i < 19; ++i)  // towards an x wall: stays in slot opp(i)
                Store<ST>::st_stream(xwall(-ex(i), xlo, xhi) ? Fc + opp(i) * p.ld : Fc + fout_off<FACE, TAB>(p, lk, i),
                                     f[i]);
            Store<ST>::st_stream(Gc, g[0]);
#pragma unroll
            for (int i = 1; i < 7; ++i)
                Store<ST>::st_stream(xwall(-tx(i), xlo, xhi) ? Gc + opp7(i) * p.ld : Gc + gout_off<FACE, TAB>(p, lk, i),
                                     g[i]);
            return;
        }
        Store<ST>::st_stream(Fc, f[0]);
#pragma unroll
        for (int i = 1; i < 19; ++i)
            Store<ST>::st_stream(((lm >> opp(i)) & 1u) ? Fc + fout_off<FACE, TAB>(p, lk, i) : Fc + opp(i) * p.ld, f[i]);
        if (COND) {
            // x + t_i = x - e_opp(i): inside (bit opp(i) of im) and solid (bit opp(i) of lm clear)
            unsigned other = 0;
#pragma unroll
            for (int i = 1; i < 7; ++i)
                if (((im >> opp7(i)) & 1u) && !((lm >> opp(i)) & 1u)) other |= 1u << i;
            if (other) cross_phase(p, other, a == jsc - 1, spost, col, g);
        }
    } else if (COND) {
        // the solid's own g: pulled as for a liquid node, collided at u = 0
        const unsigned ims = off_walls ? 0x7eu : inside_mask(p, x, y, z);
        const float th_rd = __ldg(thw_rd + col);
        g[0] = Store<ST>::ld(Gc);
#pragma unroll
        for (int i = 1; i < 7; ++i) {
            const bool in = (ims >> i) & 1u;
            const float v = Store<ST>::ld(in ? Gc + gin_off<FACE, TAB>(p, lk, i) : Gc + i * p.ld);
            g[i] = in ? v : wall_value<FACE>(p, opp7(i), v, th_rd);
        }
        collide_solid(p, g);
        if (a <= (nbv & 0xffff)) {
            const unsigned other = other_phase7<FACE>(p, js, x, y, z, false);
            if (other) cross_phase(p, other, a == jsc, gpost, col, g);
        }
    } else {
        if (deep_solid(p, a, nbv)) return;
        solid_post(p, a == jsc, gpost, col, g);
    }
    const unsigned im = off_walls ? 0x7eu : inside_mask(p, x, y, z);
    const float th_wr = __ldg(thw_wr + col);
    Store<ST>::st_stream(Gc, g[0]);
#pragma unroll
    for (int i = 1; i < 7; ++i) {
        const bool out = (im >> opp7(i)) & 1u;
        Store<ST>::st_stream(out ? Gc + gout_off<FACE, TAB>(p, lk, i) : Gc + opp7(i) * p.ld,
                      out ? g[i] : wall_value<FACE>(p, i, g[i], th_wr));
    }
}

template <typename ST, int FACE>
__global__ void __launch_bounds__(128, k1_min_blocks<ST>()) k_odd(const __grid_constant__ KP p, ST *__restrict__ F, ST *__restrict__ G,
                                             const int *__restrict__ js, const int *__restrict__ nb,
                                             const float *__restrict__ gpost, const float *__restrict__ thw_rd,
                                             const float *__restrict__ thw_wr, const __grid_constant__ Links lk,
                                             const int *jmax) {
    step_launch_wait();
    int x, y, z;
    if (k1_node<FACE>(p, jmax, x, y, z)) odd_node<ST, FACE>(p, &lk, F, G, js, nb, gpost, thw_rd, thw_wr, x, y, z);
}

// The odd step with heat conduction in the solid (every node updated).
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_odd_cond(const __grid_constant__ KP p, ST *__restrict__ F, ST *__restrict__ G,
                                                  const int *__restrict__ js, const int *__restrict__ nb,
                                                  const float *__restrict__ gpost, const float *__restrict__ thw_rd,
                                                  const float *__restrict__ thw_wr, const __grid_constant__ Links lk,
                                                  const float *__restrict__ spost) {
    step_launch_wait();
    int x, y, z;
    if (k1_node<FACE>(p, nullptr, x, y, z))
        odd_node<ST, FACE, true, true>(p, &lk, F, G, js, nb, gpost, thw_rd, thw_wr, x, y, z, spost);
}


// ------------------------------------------- two nodes per thread (FP16)
// With FP16 storage and an even nx, a thread of the stream-collide takes the
// nodes x0 = 2k and x0 + 1 of a row.  Their slots of a direction are
// adjacent and 4-byte aligned (c = index of x0 is even, ld a multiple of 128,
// and a link offset is even unless the link has an x component), so a pair
// of liquid nodes moves its populations as half2 words and collides in
// packed FP32x2 arithmetic (collide2): about half the instructions per node
// of the one-node kernels, whose FP32 arithmetic, not HBM, bounds them with
// 2-byte populations.  A pair that meets the interface (or, in the odd step,
// a wall of the heating axis or of the other in-plane axis) takes the
// one-node code for each of its nodes.
// Resident blocks of 128 the pair kernels ask for (the register budget of a
// thread is 65536 / (128 x this)): 5, 96 registers and under 90 bytes of
// spills, ran the 256^3 FP16 stream-collide in 0.148 ms against 0.158 ms with
// 4 (128 registers, no spills) and 0.164 ms with 6 (80 registers, up to
// 256 bytes of spills).
#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 5
#endif
#ifndef LBM_PAIR_MIN_BLOCKS_F32
#define LBM_PAIR_MIN_BLOCKS_F32 5
#endif
template <typename ST> constexpr int pair_min_blocks() {
    return sizeof(ST) == 2 ? LBM_PAIR_MIN_BLOCKS : LBM_PAIR_MIN_BLOCKS_F32;
}

template <int FACE>
__device__ __forceinline__ bool k1_pair(const KP &p, const int *jmax, int &x, int &y, int &z) {
    const int a0 = (int)blockIdx.z * (FACE == 0 ? (int)blockDim.y : 1);
    if (jmax && a0 >= *jmax + 3) return false;
    x = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (FACE == 0) {
        y = a0 + (int)threadIdx.y;
        z = (int)blockIdx.y;
    } else {
        y = (int)(blockIdx.y * blockDim.y + threadIdx.y);
        z = (int)blockIdx.z;
    }
    return x < p.nx && y < p.ny;
}

// The two adjacent populations of a pair (an aligned half2 or float2 word).
__device__ __forceinline__ float2 ld_pair(const __half *q) { return __half22float2(*(const __half2 *)q); }
__device__ __forceinline__ float2 ld_pair(const float *q) { return *(const float2 *)q; }
__device__ __forceinline__ void st_pair(__half *q, float2 v) { __stcs((__half2 *)q, __floats2half2_rn(v.x, v.y)); }
__device__ __forceinline__ void st_pair(float *q, float2 v) { __stcs((float2 *)q, v); }

// The even step of a pair of liquid nodes (both collide, no phase test).
template <typename ST, typename IX>
__device__ __forceinline__ void even_pair_liquid(const KP &p, ST *__restrict__ F, ST *__restrict__ G, IX c) {
    float2 f[19], g[7];
#pragma unroll
    for (int i = 0; i < 19; ++i) f[i] = ld_pair(elem<IX>(F, c, i * p.ld));
#pragma unroll
    for (int i = 0; i < 7; ++i) g[i] = ld_pair(elem<IX>(G, c, i * p.ld));
    collide2(p, f, g);
#pragma unroll
    for (int i = 0; i < 19; ++i) st_pair(elem<IX>(F, c, opp(i) * p.ld), f[i]);
#pragma unroll
    for (int i = 0; i < 7; ++i) st_pair(elem<IX>(G, c, opp7(i) * p.ld), g[i]);
}

template <typename ST, int FACE, typename IX>
__device__ __forceinline__ void even_pair(const KP &p, ST *__restrict__ F, ST *__restrict__ G,
                                          const int *__restrict__ js, const int *__restrict__ nb,
                                          const float *__restrict__ gpost, int x, int y, int z) {
    const int a = axial<FACE>(x, y, z);
    const int col = column<FACE>(p, x, y, z);  // x + 1 is in column col + 1
    if (a < __ldg(js + col) && a < __ldg(js + col + 1)) {
        even_pair_liquid<ST, IX>(p, F, G, (IX)node_index(p, x, y, z));
    } else {
        even_node<ST, FACE, IX>(p, F, G, js, nb, gpost, x, y, z);
        even_node<ST, FACE, IX>(p, F, G, js, nb, gpost, x + 1, y, z);
    }
}

template <typename ST, int FACE, typename IX>
__global__ void __launch_bounds__(128, pair_min_blocks<ST>()) k_even_pair(const __grid_constant__ KP p, ST *__restrict__ F,
                                                      ST *__restrict__ G, const int *__restrict__ js,
                                                      const int *__restrict__ nb, const float *__restrict__ gpost,
                                                      const int *jmax) {
    step_launch_wait();
    int x, y, z;
    if (k1_pair<FACE>(p, jmax, x, y, z)) even_pair<ST, FACE, IX>(p, F, G, js, nb, gpost, x, y, z);
}

// The odd step of a pair on the fast path (both liquid, off the walls of the
// heating axis and of the other in-plane axis, every link streaming but
// those across an x wall).  Links without an x component move as half2 /
// float2 words; the others node by node, with the x walls (x0 = 0 for lane
// x, x0 + 1 = nx - 1 for lane y) taken as in odd_node.
template <typename ST, int FACE, typename IX>
__device__ __forceinline__ void odd_pair_liquid(const KP &p, const Links *lk, ST *__restrict__ F,
                                                ST *__restrict__ G, int x, int y, int z) {
    const IX c = (IX)node_index(p, x, y, z), c1 = c + 1;
    const bool xlo = x == 0, xhi = x + 1 == p.nx - 1;
    float2 f[19], g[7];
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        if (ex(i) == 0) {
            f[i] = ld_pair(elem<IX>(F, c, lk->fin[i]));
        } else {
            // across an x wall: bounce-back from the node's own slot i
            f[i].x = Store<ST>::ld(elem<IX>(F, c, ex(i) > 0 && xlo ? i * p.ld : lk->fin[i]));
            f[i].y = Store<ST>::ld(elem<IX>(F, c1, ex(i) < 0 && xhi ? i * p.ld : lk->fin[i]));
        }
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) {
        if (tx(i) == 0) {
            g[i] = ld_pair(elem<IX>(G, c, lk->gin[i]));
        } else {
            g[i].x = Store<ST>::ld(elem<IX>(G, c, tx(i) > 0 && xlo ? i * p.ld : lk->gin[i]));
            g[i].y = Store<ST>::ld(elem<IX>(G, c1, tx(i) < 0 && xhi ? i * p.ld : lk->gin[i]));
        }
    }
    collide2(p, f, g);
#pragma unroll
    for (int i = 0; i < 19; ++i) {
        if (ex(i) == 0) {
            st_pair(elem<IX>(F, c, lk->fout[i]), f[i]);
        } else {
            // towards an x wall: stays in the node's slot opp(i)
            Store<ST>::st_stream(elem<IX>(F, c, ex(i) < 0 && xlo ? opp(i) * p.ld : lk->fout[i]), f[i].x);
            Store<ST>::st_stream(elem<IX>(F, c1, ex(i) > 0 && xhi ? opp(i) * p.ld : lk->fout[i]), f[i].y);
        }
    }
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

// The odd step for a pair: both nodes on the one-node fast path (liquid, off
// the walls of the heating axis and of the other in-plane axis, one node
// below the lowest first-solid node of their 3x3 columns) take
// odd_pair_liquid, any other pair the one-node code node by node.
template <typename ST, int FACE, typename IX>
__device__ __forceinline__ void odd_pair(const KP &p, const Links *lk, ST *__restrict__ F,
                                         ST *__restrict__ G, const int *__restrict__ js,
                                         const int *__restrict__ nb, const float *__restrict__ gpost,
                                         const float *__restrict__ thw_rd, const float *__restrict__ thw_wr, int x,
                                         int y, int z) {
    const int a = axial<FACE>(x, y, z);
    const int col = column<FACE>(p, x, y, z);
    const int q = FACE == 0 ? z : y, nq = FACE == 0 ? p.nz : p.ny;
    const bool off_qa = q >= 1 && q <= nq - 2 && a >= 1 && a <= p.H - 2;
    const bool fast = off_qa && a + 1 < (__ldg(nb + col) >> 16) && a + 1 < (__ldg(nb + col + 1) >> 16);
    if (!fast) {
        odd_node<ST, FACE>(p, lk, F, G, js, nb, gpost, thw_rd, thw_wr, x, y, z);
        odd_node<ST, FACE>(p, lk, F, G, js, nb, gpost, thw_rd, thw_wr, x + 1, y, z);
        return;
    }
    odd_pair_liquid<ST, FACE, IX>(p, lk, F, G, x, y, z);
}

template <typename ST, int FACE, typename IX>
__global__ void __launch_bounds__(128, pair_min_blocks<ST>()) k_odd_pair(const __grid_constant__ KP p, ST *__restrict__ F,
                                                     ST *__restrict__ G, const int *__restrict__ js,
                                                     const int *__restrict__ nb, const float *__restrict__ gpost,
                                                     const float *__restrict__ thw_rd,
                                                     const float *__restrict__ thw_wr,
                                                     const __grid_constant__ Links lk, const int *jmax) {
    step_launch_wait();
    int x, y, z;
    if (k1_pair<FACE>(p, jmax, x, y, z)) odd_pair<ST, FACE, IX>(p, &lk, F, G, js, nb, gpost, thw_rd, thw_wr, x, y, z);
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
                            : -own + 2.0f * w7(i) * ((w == 1 ? thw[column<FACE>(p, x, y, z)] : p.Tc) - p.Ts);
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

// Liquid counts of the 3x3 columns around column (pp, q), 0 outside the
// cavity; entry (dq + 1) * 3 + dp + 1.
__device__ __forceinline__ void load_js9(const KP &p, const int *__restrict__ js, int pp, int q, int (&js9)[9]) {
#pragma unroll
    for (int dq = -1; dq <= 1; ++dq)
#pragma unroll
        for (int dp = -1; dp <= 1; ++dp) {
            const int p2 = pp + dp, q2 = q + dq;
            const bool in = (unsigned)p2 < (unsigned)p.P1 && (unsigned)q2 < (unsigned)p.P2;
            js9[(dq + 1) * 3 + dp + 1] = in ? __ldg(js + q2 * p.P1 + p2) : 0;
        }
}

// gather_f in flight for the node at height a of the middle column, with
// the liquid tests read from js9 (load_js9) instead of memory.
template <typename ST, int FACE>
__device__ __forceinline__ void gather_f9(const KP &p, const ST *F, const int (&js9)[9], int x, int y, int z, int a,
                                          float (&f)[19]) {
    const long long c = node_index(p, x, y, z);
    f[0] = Store<ST>::ld(F + c);
#pragma unroll
    for (int i = 1; i < 19; ++i) {
        // the upstream node x - e_i: in-plane column offset and height
        const int dp = -ex(i), dq = FACE == 0 ? -ez(i) : -ey(i), da = FACE == 0 ? -ey(i) : -ez(i);
        const int an = a + da;
        const bool liq = an >= 0 && an < js9[(dq + 1) * 3 + dp + 1];
        if (liq) f[i] = Store<ST>::ld(F + opp(i) * p.ld + (c - off19<FACE>(p, i)));
        else f[i] = Store<ST>::ld(F + i * p.ld + c);
    }
}

// Ts + the sum of the shifted g (the temperature the front reads; FP32, the
// precision the populations are held in).
__device__ __forceinline__ float sum_T(const KP &p, const float (&g)[7]) {
    float t = 0.0f;
#pragma unroll
    for (int i = 0; i < 7; ++i) t += g[i];
    return p.Ts + t;
}

template <typename ST, int FACE>
__device__ __forceinline__ float node_T(const KP &p, const ST *G, int col, int j, bool inflight, const float *thw) {
    int x, y, z;
    column_node<FACE>(p, col, j, x, y, z);
    float g[7];
    gather_g<ST, FACE>(p, G, x, y, z, inflight, thw, g);
    return sum_T(p, g);
}

// The Eq. 6 gradient dT/da at the front a = s (R8: the one-sided quadratic
// through (s, Tm) and the guarded node k with the node below it, or the
// heated wall (0, Tw) for a missing node; linear through the wall when k <
// 0), and the front speed ds/dt = coef (1 + s_p^2 + s_q^2)(-dT/da).  FP32
// with every operation rounded on its own (no contraction into FMAs), so that
// each kernel that evaluates them (the front update, the ensemble, the
// adjoint's recomputation) gets the same bits.  With h = x1 - x0,
// d1 = s - x1, d0 = s - x0: p'(s) = (y0 d1^2 - y1 d0^2 + Tm h (d0 + d1)) /
// (h d0 d1).
__device__ __forceinline__ float front_gradient(int k, double sc, float y0, float y1, float Tm, float Tw) {
    if (k < 0) return __fdiv_rn(__fsub_rn(Tm, Tw), (float)sc);
    const double x1 = k + 0.5, x0 = k >= 1 ? k - 0.5 : 0.0;
    const float h = (float)(x1 - x0), d1 = (float)(sc - x1), d0 = (float)(sc - x0);
    const float num = __fadd_rn(__fsub_rn(__fmul_rn(__fmul_rn(y0, d1), d1), __fmul_rn(__fmul_rn(y1, d0), d0)),
                                __fmul_rn(__fmul_rn(Tm, h), __fadd_rn(d0, d1)));
    return __fdiv_rn(num, __fmul_rn(__fmul_rn(h, d0), d1));
}
__device__ __forceinline__ float front_slope_factor(float sp, float sq) {
    return __fadd_rn(__fadd_rn(1.0f, __fmul_rn(sp, sp)), __fmul_rn(sq, sq));
}
__device__ __forceinline__ float front_speed(const KP &p, float fac, float G) {
    return __fmul_rn(__fmul_rn(p.coef_f, fac), -G);
}

// Highest node at least half a cell below s (centre j + 1/2 <= s - 1/2).
__device__ __forceinline__ int guarded_node(double s, int H) {
    int k = (int)floor(s - 1.0);
    return k > H - 1 ? H - 1 : (k < 0 ? -1 : k);
}

// Lowest node at least half a cell above s (centre j + 1/2 >= s + 1/2, i.e.
// j = ceil(s)), or H when there is none.
__device__ __forceinline__ int guarded_solid_node(double s, int H) {
    const int k = (int)ceil(s);
    return k > H ? H : k;
}

// Solid-side dT/da at the front a = s (the k_s dT_s/da term of Eq. 6, heat
// conduction in the solid): the mirror of front_gradient, the one-sided
// quadratic through (s, Tm), the guarded solid node ks and the node above
// it, the cold wall (H, Tc) standing in for a missing node; linear through
// (s, Tm) and (H, Tc) when ks = H.  Y1, Y2: the temperatures of nodes ks and
// ks + 1 (or the wall) minus Tm, so that a solid at Tm gives exactly zero.
__device__ __forceinline__ float solid_gradient(int ks, int H, double sc, float Y1, float Y2, float Tm, float Tc) {
    if (ks >= H) return (Tc - Tm) / (float)((double)H - sc);
    const double x1 = ks + 0.5, x2 = ks + 1 < H ? ks + 1.5 : (double)H;
    return Y1 * (float)(sc - x2) / ((float)(x1 - sc) * (float)(x1 - x2)) +
           Y2 * (float)(sc - x1) / ((float)(x2 - sc) * (float)(x2 - x1));
}

// ------------------------------------------------------------ front (Eq. 6)
// One thread per column.  From the state after a step (T of the liquid at
// t + 1, front s_t): the one-sided quadratic gradient at the front, the
// in-plane slopes from the old fronts of the neighbour columns (mirror at
// the side walls), ds/dt = coef (1 + s_p^2 + s_q^2)(-dT/da), the new front
// clamped to [1/2, H], its liquid-node count, and the ghost node of the new
// front: g*_ghost = g^eq(T_ghost, 0) + (g*_L - g^eq(T_L, u_L)).
// move = 0 keeps the front (used to prepare the ghost after a state upload).
// SPEC: load the ghost's likely source node together with the gradient
// stencil (two dependent load stages instead of three; more registers).
//
// Precision: the front heights are accumulated in FP64 (s + ds, and the
// distances from s to the stencil nodes and the ghost are FP64 differences);
// the gradient, the speed and the ghost temperature are FP32 arithmetic, the
// precision of the temperatures they are made of.  GB300 issues FP64 at a
// small fraction of its FP32 rate, and the FP64 divisions of an all-FP64
// version made this kernel FP64-pipe bound.
//
// COND (heat conduction in the solid): Eq. 6 gains kappa dT_s/da from
// solid_gradient at s_t, and the solid side's ghost populations of the new
// front are written to spost: at the last liquid node, g^eq(T_sghost, 0)
// plus the non-equilibrium part of the first solid node collided at u = 0,
// with T_sghost on the line through (s, Tm) and the guarded solid node (or
// the cold wall); the rest state at Tm in a column without both phases.
template <typename ST, int FACE, bool SPEC = true, bool COND = false>
__device__ __forceinline__ int front_column(const KP &p, const ST *__restrict__ F, const ST *__restrict__ G,
                                           const int *__restrict__ js, int *__restrict__ js_next,
                                           const double *__restrict__ s, double *__restrict__ s_next,
                                           float *__restrict__ gpost, const float *__restrict__ thw, int inflight,
                                           int move, int *__restrict__ status, int col,
                                           float *__restrict__ spost = nullptr) {
    const int P1 = p.P1, P2 = p.P2, H = p.H;
    const int pp = col % P1, q = col / P1;
    const bool infl = inflight != 0;
    // Load stage 1: what depends on the column only.
    const double sc = s[col];
    const float Tm = p.Tm;
    const float Tw = thw[col];
    const int jsc = js[col];
    int js9[9];
    if (SPEC && infl) load_js9(p, js, pp, q, js9);
    float sp = 0.0f, sq = 0.0f;
    if (move) {
        sp = 0.5f * (float)(s[q * P1 + (pp + 1 < P1 ? pp + 1 : pp)] - s[q * P1 + (pp > 0 ? pp - 1 : pp)]);
        sq = 0.5f * (float)(s[(q + 1 < P2 ? q + 1 : q) * P1 + pp] - s[(q > 0 ? q - 1 : q) * P1 + pp]);
    }
    // Load stage 2: the gradient stencil of s_t and, speculatively, the node
    // below the current front, which is the ghost's source node whenever the
    // liquid count does not change (all but a few columns per step).
    const int k = move ? guarded_node(sc, H) : -2;
    float y1 = 0.0f, y0 = Tw;
    if (k >= 0) {
        y1 = node_T<ST, FACE>(p, G, col, k, infl, thw);
        if (k >= 1) y0 = node_T<ST, FACE>(p, G, col, k - 1, infl, thw);
    }
    const int L = jsc - 1;
    const bool spec = SPEC && L >= 0 && jsc < H;
    float gL[7], fL[19];
    if (spec) {
        int x, y, z;
        column_node<FACE>(p, col, L, x, y, z);
        gather_g<ST, FACE>(p, G, x, y, z, infl, thw, gL);
        if (infl) gather_f9<ST, FACE>(p, F, js9, x, y, z, L, fL);
        else gather_f<ST, FACE>(p, F, js, x, y, z, false, fL);
    }
    // The solid side of the front (conduction in the solid, a column with a
    // solid node): temperatures of the guarded solid node and the one above.
    int ks = H;
    float Ts1 = Tm, Ts2 = Tm, Gs = 0.0f;
    if (COND && move && jsc < H) {
        ks = guarded_solid_node(sc, H);
        if (ks < H) {
            Ts1 = node_T<ST, FACE>(p, G, col, ks, infl, thw);
            Ts2 = ks + 1 < H ? node_T<ST, FACE>(p, G, col, ks + 1, infl, thw) : p.Tc;
        }
        Gs = p.kappa * solid_gradient(ks, H, sc, Ts1 - Tm, Ts2 - Tm, Tm, p.Tc);
    }
    // Then Eq. 6.
    double sn = sc;
    if (move) {
        const float Gr = front_gradient(k, sc, y0, y1, Tm, Tw);
        const float v = front_speed(p, front_slope_factor(sp, sq), COND ? Gr - Gs : Gr);
        if (!isfinite(Gr) || (COND && !isfinite(Gs))) atomicOr(status, 2);
        else if (!(fabsf(v) <= 0.5f)) atomicOr(status, 1);
        sn = sc + (double)v;
        if (!(sn >= 0.5)) sn = 0.5;  // also catches NaN
        if (sn > (double)H) sn = (double)H;
    }
    s_next[col] = sn;
    int jn = (int)ceil(sn - 0.5);
    jn = jn < 0 ? 0 : (jn > H ? H : jn);
    js_next[col] = jn;
    if (COND) {
        // the solid side's ghost populations at the last liquid node jn - 1
        float sg[7];
        if (jn >= 1 && jn < H) {
            const double yg = jn - 0.5;
            const int ks2 = guarded_solid_node(sn, H);
            float Tsg;
            if (ks2 >= H) {
                Tsg = Tm + (p.Tc - Tm) * (float)((yg - sn) / ((double)H - sn));
            } else {
                float Tk;
                if (move && jsc < H && ks2 == ks) Tk = Ts1;
                else if (move && jsc < H && ks2 == ks + 1 && ks + 1 < H) Tk = Ts2;
                else Tk = node_T<ST, FACE>(p, G, col, ks2, infl, thw);
                Tsg = Tm + (Tk - Tm) * (float)((yg - sn) / ((ks2 + 0.5) - sn));
            }
            float gS[7];
            int x, y, z;
            column_node<FACE>(p, col, jn, x, y, z);
            gather_g<ST, FACE>(p, G, x, y, z, infl, thw, gS);
            const float Th = gS[0] + gS[1] + gS[2] + gS[3] + gS[4] + gS[5] + gS[6];
            const float dTg = Tsg - p.Ts;
#pragma unroll
            for (int i = 0; i < 7; ++i) sg[i] = w7(i) * dTg;
            // N^-1 (I - Q)(n - n^eq) of the solid node at u = 0
            constexpr float i1 = 1.0f / (float)nnorm(1), i4 = 1.0f / (float)nnorm(4);
            constexpr float i5 = 1.0f / (float)nnorm(5), i6 = 1.0f / (float)nnorm(6);
            const float ra = 1.0f - p.s_alpha_s, r4 = 1.0f - p.s_g4, r5 = 1.0f - p.s_g5;
            float cn[7];
            cn[0] = 0.0f;
            cn[1] = ra * (gS[1] - gS[2]) * i1;
            cn[2] = ra * (gS[3] - gS[4]) * i1;
            cn[3] = ra * (gS[5] - gS[6]) * i1;
            cn[4] = r4 * (6.0f * gS[0] - (gS[1] + gS[2] + gS[3] + gS[4] + gS[5] + gS[6]) - 0.75f * Th) * i4;
            cn[5] = r5 * (2.0f * (gS[1] + gS[2]) - (gS[3] + gS[4] + gS[5] + gS[6])) * i5;
            cn[6] = r5 * ((gS[3] + gS[4]) - (gS[5] + gS[6])) * i6;
            add_back7<0>(sg, cn);
        } else {
#pragma unroll
            for (int i = 0; i < 7; ++i) sg[i] = w7(i) * p.dTms;
        }
#pragma unroll
        for (int i = 0; i < 7; ++i) spost[(long long)i * p.ncols + col] = sg[i];
    }
    if (jn >= H) return jn;  // fully liquid column: no ghost node
    const double yg = jn + 0.5;
    const int kg = guarded_node(sn, H);
    float Tg;
    if (kg < 0) {
        Tg = Tm + (Tm - Tw) * ((float)(yg - sn) / (float)sn);
    } else {
        float Tk;
        if (kg == k) Tk = y1;
        else if (kg == k - 1 && k >= 1) Tk = y0;
        else if (spec && kg == L) Tk = sum_T(p, gL);
        else Tk = node_T<ST, FACE>(p, G, col, kg, infl, thw);
        Tg = Tm + (Tm - Tk) * ((float)(yg - sn) / (float)(sn - (kg + 0.5)));
    }
    // ghost populations (FP32, like the collision): rest equilibrium at the
    // ghost temperature plus the non-equilibrium part N^-1 (I - Q)(n - n^eq)
    // of the post-collision populations of the liquid node below
    float gh[7];
    const float dTg = Tg - p.Ts;
#pragma unroll
    for (int i = 0; i < 7; ++i) gh[i] = w7(i) * dTg;
    if (jn >= 1) {
        if (!(spec && jn == jsc)) {  // the count changed: the source node moved
            int x, y, z;
            column_node<FACE>(p, col, jn - 1, x, y, z);
            gather_g<ST, FACE>(p, G, x, y, z, infl, thw, gL);
            const bool newly_liquid = (jn - 1) >= jsc;
            if (newly_liquid) {
#pragma unroll
                for (int i = 0; i < 19; ++i) fL[i] = 0.0f;
            } else {
                gather_f<ST, FACE>(p, F, js, x, y, z, infl, fL);
            }
        }
        float Th = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
        for (int i = 0; i < 7; ++i) Th += gL[i];
#pragma unroll
        for (int i = 0; i < 19; ++i) {
            jx += ex(i) * fL[i];
            jy += ey(i) * fL[i];
            jz += ez(i) * fL[i];
        }
        const float TL = Th + p.Ts;
        const float ux = jx, uy = jy, uz = jz + 0.5f * p.gbeta * (Th - p.dTms);
        constexpr float i1 = 1.0f / (float)nnorm(1), i4 = 1.0f / (float)nnorm(4);
        constexpr float i5 = 1.0f / (float)nnorm(5), i6 = 1.0f / (float)nnorm(6);
        const float ra = 1.0f - p.s_alpha, r4 = 1.0f - p.s_g4, r5 = 1.0f - p.s_g5;
        float cn[7];
        cn[0] = 0.0f;
        cn[1] = ra * ((gL[1] - gL[2]) - ux * TL) * i1;
        cn[2] = ra * ((gL[3] - gL[4]) - uy * TL) * i1;
        cn[3] = ra * ((gL[5] - gL[6]) - uz * TL) * i1;
        cn[4] = r4 * (6.0f * gL[0] - (gL[1] + gL[2] + gL[3] + gL[4] + gL[5] + gL[6]) - 0.75f * Th) * i4;
        cn[5] = r5 * (2.0f * (gL[1] + gL[2]) - (gL[3] + gL[4] + gL[5] + gL[6])) * i5;
        cn[6] = r5 * ((gL[3] + gL[4]) - (gL[5] + gL[6])) * i6;
        add_back7<0>(gh, cn);
    }
#pragma unroll
    for (int i = 0; i < 7; ++i) gpost[(long long)i * p.ncols + col] = gh[i];
    return jn;
}

// jmax (may be null): running maximum of the liquid counts, one atomic per
// warp; the host reads it back now and then to bound the height of the
// stream-collide grid (nodes two above every neighbouring count are deep
// solid and do nothing).
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_front(const __grid_constant__ KP p, const ST *__restrict__ F, const ST *__restrict__ G,
                                               const int *__restrict__ js, int *__restrict__ js_next,
                                               const double *__restrict__ s, double *__restrict__ s_next,
                                               float *__restrict__ gpost, const float *__restrict__ thw,
                                               int inflight, int move, int *__restrict__ status,
                                               int *__restrict__ jmax) {
    step_launch_wait();
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    int jn = -1;
    if (col < p.ncols) jn = front_column<ST, FACE>(p, F, G, js, js_next, s, s_next, gpost, thw, inflight, move, status, col);
    // blocks are whole warps and every thread of the grid reaches this point
    const int m = __reduce_max_sync(0xffffffffu, jn);
    if (jmax && (threadIdx.x & 31) == 0 && m >= 0) atomicMax(jmax, m);
}

// The front update with heat conduction in the solid.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_front_cond(const __grid_constant__ KP p, const ST *__restrict__ F,
                                                    const ST *__restrict__ G, const int *__restrict__ js,
                                                    int *__restrict__ js_next, const double *__restrict__ s,
                                                    double *__restrict__ s_next, float *__restrict__ gpost,
                                                    float *__restrict__ spost, const float *__restrict__ thw,
                                                    int inflight, int move, int *__restrict__ status) {
    step_launch_wait();
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col < p.ncols)
        front_column<ST, FACE, true, true>(p, F, G, js, js_next, s, s_next, gpost, thw, inflight, move, status, col,
                                           spost);
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
//
// Every column also records the minimum and maximum of the new liquid counts
// over its 3x3 neighbourhood (min << 16 | max) for the interior and
// deep-solid tests of the next stream-collide.  do_flip = 0 only records.
// The links I0 .. I0 + 8 of a flipped node c = (x, y, z) (see flip_column).
// The 18 links of one node touch 36 distinct slots (slot i of c, slot opp(i)
// of c - e_i), so every phase flag and slot of the nine is loaded before the
// first store: the loads are in flight together, where a link-by-link loop
// waits two dependent memory round trips per link (the compiler cannot move
// a load above a store into the same array).  Same values, same stores.
template <typename ST, int FACE, int I0>
__device__ __forceinline__ void flip_links(const KP &p, ST *__restrict__ F, const int *__restrict__ js_old,
                                           const int *__restrict__ js_new, int x, int y, int z, long long c,
                                           bool lx_t, bool lx_n) {
    bool yin[9], ly_t[9], ly_n[9], own[9];
    long long cy[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = I0 + k;
        const int xn = x - ex(i), yn = y - ey(i), zn = z - ez(i);
        yin[k] = inside(p, xn, yn, zn);
        ly_t[k] = ly_n[k] = false;
        cy[k] = 0;
        if (yin[k]) {
            const int cc = column<FACE>(p, xn, yn, zn), an = axial<FACE>(xn, yn, zn);
            ly_t[k] = an < js_old[cc];
            ly_n[k] = an < js_new[cc];
            cy[k] = node_index(p, xn, yn, zn);
        }
        own[k] = !(ly_t[k] != ly_n[k] && cy[k] < c);  // else the other end owns this link
    }
    float P[9], Q[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = I0 + k;
        P[k] = own[k] && yin[k] ? Store<ST>::ld(F + opp(i) * p.ld + cy[k]) : 0.0f;
        Q[k] = own[k] ? Store<ST>::ld(F + i * p.ld + c) : 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        if (!own[k]) continue;
        const int i = I0 + k;
        ST *Ps = F + opp(i) * p.ld + cy[k];
        ST *Qs = F + i * p.ld + c;
        const float dx = !lx_t ? 0.0f : (ly_t[k] ? P[k] : Q[k]);
        const float dy = !ly_t[k] ? 0.0f : (lx_t ? Q[k] : P[k]);
        if (lx_n && ly_n[k]) { Store<ST>::st(Ps, dx); Store<ST>::st(Qs, dy); }
        else if (lx_n) Store<ST>::st(Qs, dx);
        else if (ly_n[k]) Store<ST>::st(Ps, dy);
    }
}

template <typename ST, int FACE>
__device__ __forceinline__ void flip_column(const KP &p, ST *__restrict__ F, const int *__restrict__ js_old,
                                          const int *__restrict__ js_new, int *__restrict__ nb_new, int inflight,
                                          int do_flip, int col) {
    {
        const int pp = col % p.P1, q = col / p.P1;
        int mn = 1 << 15, mx = 0;
        for (int dq = -1; dq <= 1; ++dq)
            for (int dp = -1; dp <= 1; ++dp) {
                const int p2 = pp + dp, q2 = q + dq;
                if (p2 < 0 || p2 >= p.P1 || q2 < 0 || q2 >= p.P2) continue;
                const int v = js_new[q2 * p.P1 + p2];
                mn = v < mn ? v : mn;
                mx = v > mx ? v : mx;
            }
        nb_new[col] = (mn << 16) | mx;
    }
    const int jo = js_old[col], jn = js_new[col];
    if (!do_flip || jo == jn) return;
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
        flip_links<ST, FACE, 1>(p, F, js_old, js_new, x, y, z, c, lx_t, lx_n);
        flip_links<ST, FACE, 10>(p, F, js_old, js_new, x, y, z, c, lx_t, lx_n);
    }
}

// 4 blocks of 128 a multiprocessor (up to 128 registers: flip_links holds
// nine links' flags and slots; 608 blocks cover a 256 x 256 front at once).
template <typename ST, int FACE>
__global__ void __launch_bounds__(128, 4) k_flip(const __grid_constant__ KP p, ST *__restrict__ F, const int *__restrict__ js_old,
                                              const int *__restrict__ js_new, int *__restrict__ nb_new,
                                              int inflight, int do_flip) {
    step_launch_wait();
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= p.ncols) return;
    flip_column<ST, FACE>(p, F, js_old, js_new, nb_new, inflight, do_flip, col);
}


// ----------------------------------------------------- outputs and inputs
// T and u per node (solid: Tm, or its own temperature with heat conduction
// in the solid, and u = 0), natural values.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_macro(const __grid_constant__ KP p, const ST *__restrict__ F, const ST *__restrict__ G,
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
        uz += 0.5f * p.gbeta * (Th - p.dTms);
        Tc = p.Ts + Th;
    } else if (p.cond) {
        float g[7];
        gather_g<ST, FACE>(p, G, x, y, z, inflight != 0, thw, g);
        Tc = sum_T(p, g);
    }
    if (T) T[c] = Tc;
    if (u) { u[3 * c] = ux; u[3 * c + 1] = uy; u[3 * c + 2] = uz; }
}

// Natural (unshifted) distributions out, direction-major with stride N.
// Solid nodes report f = 0; deep solid nodes (see deep_solid) report g at
// rest at Tm, the value their slots would hold if they were updated.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_state_out(const __grid_constant__ KP p, const ST *__restrict__ F, const ST *__restrict__ G,
                                                   const int *__restrict__ js, const int *__restrict__ nb,
                                                   const float *__restrict__ thw, int inflight,
                                                   float *__restrict__ fo, float *__restrict__ go) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z), col = column<FACE>(p, x, y, z);
    if (go) {
        float g[7];
        if (a >= js[col] && deep_solid(p, a, nb[col])) {
#pragma unroll
            for (int i = 0; i < 7; ++i) g[i] = w7(i) * p.dTms;
        } else {
            gather_g<ST, FACE>(p, G, x, y, z, inflight != 0, thw, g);
        }
#pragma unroll
        for (int i = 0; i < 7; ++i) go[i * p.N + c] = g[i] + w7(i) * p.Ts;
    }
    if (fo) {
        float f[19];
        const bool liq = a < js[col];
        if (liq) gather_f<ST, FACE>(p, F, js, x, y, z, inflight != 0, f);
#pragma unroll
        for (int i = 0; i < 19; ++i) fo[i * p.N + c] = liq ? f[i] + w19(i) : 0.0f;
    }
}

// Natural distributions in; leaves the natural layout.  A solid node's own
// populations never enter the method (its post-collision values are reset
// every step), so solid nodes are stored at rest: fh = 0 and gh = 0
// (g at rest at Tm); with heat conduction in the solid they keep their g.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_state_in(const __grid_constant__ KP p, ST *__restrict__ F, ST *__restrict__ G,
                                                  const int *__restrict__ js, const float *__restrict__ fi,
                                                  const float *__restrict__ gi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z), col = column<FACE>(p, x, y, z);
    const bool liq = a < js[col];
    if (gi)
#pragma unroll
        for (int i = 0; i < 7; ++i)
            Store<ST>::st(G + i * p.ld + c, (liq || p.cond) ? gi[i * p.N + c] - w7(i) * p.Ts : w7(i) * p.dTms);
    if (fi)
#pragma unroll
        for (int i = 0; i < 19; ++i) Store<ST>::st(F + i * p.ld + c, liq ? fi[i * p.N + c] - w19(i) : 0.0f);
}

// Initial state: fh = 0 everywhere (rest, rho = 1); g at rest at the given
// profile T(a) below the front and at Tm above (at the profile everywhere
// with heat conduction in the solid).
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_init(const __grid_constant__ KP p, ST *__restrict__ F, ST *__restrict__ G,
                                              const int *__restrict__ js, const float *__restrict__ Tprof) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = node_index(p, x, y, z);
    const int a = axial<FACE>(x, y, z), col = column<FACE>(p, x, y, z);
    const float dT = (a < js[col] || p.cond) ? Tprof[a] - p.Ts : p.dTms;
#pragma unroll
    for (int i = 0; i < 19; ++i) Store<ST>::st(F + i * p.ld + c, 0.0f);
#pragma unroll
    for (int i = 0; i < 7; ++i) Store<ST>::st(G + i * p.ld + c, w7(i) * dT);
}

// ---------------------------------------------------------- Nusselt number
// Heat-surface Nusselt number per column (section 3.2, Fig. 4(b)):
// Nu = -H (dT/da at the heated wall) / (Th - Tm), from the heat the last
// streaming carried through the wall link of the column's first node,
// q = in - out = -alpha dT/da, times scale = H / (alpha (Th - Tm)).  The
// link is anti-bounce-back, in = -out + 2 w (Tw - Tm) in shifted values, so
// slot +a of the node gives q alone: in the natural layout it holds `in`
// (q = 2 (in - w (Tw - Tm))); in flight it still holds `out`, the node's
// post-collision population towards the wall (q = 2 (w (Tw - Tm) - out)).
// Tw is the wall field of that streaming.  FP64 from the stored value.
template <typename ST, int FACE>
__global__ void __launch_bounds__(128) k_nusselt(const __grid_constant__ KP p, const ST *__restrict__ G,
                                                 const float *__restrict__ thw, int inflight, double scale,
                                                 double *__restrict__ nu) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= p.ncols) return;
    int x, y, z;
    column_node<FACE>(p, col, 0, x, y, z);
    constexpr int up = FACE == 0 ? 3 : 5;  // the D3Q7 direction leaving the heated wall
    const double v = (double)Store<ST>::ld(G + up * p.ld + node_index(p, x, y, z));
    const double wt = (double)w7(up) * ((double)thw[col] - (double)p.Ts);
    nu[col] = (inflight ? 2.0 * (wt - v) : 2.0 * (v - wt)) * scale;
}

// ------------------------------------------------------ FP64 reductions
// Block partials of the liquid-node totals: sum (T - Tm), sum (rho - 1),
// count, max |u|^2.  Fixed block and thread order: deterministic.
template <typename ST, int FACE>
__global__ void __launch_bounds__(256) k_totals_part(const __grid_constant__ KP p, const ST *__restrict__ F, const ST *__restrict__ G,
                                                     const int *__restrict__ js, const float *__restrict__ thw,
                                                     int inflight, double *__restrict__ part) {
    __shared__ double sh[4][256];
    double sT = 0.0, sr = 0.0, n = 0.0, umax = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < p.N; c += stride) {
        const int x = (int)(c % p.nx), y = (int)((c / p.nx) % p.ny), z = (int)(c / ((long long)p.nx * p.ny));
        if (axial<FACE>(x, y, z) >= js[column<FACE>(p, x, y, z)]) continue;
        float g[7], f[19];
        gather_g<ST, FACE>(p, G, x, y, z, inflight != 0, thw, g);
        gather_f<ST, FACE>(p, F, js, x, y, z, inflight != 0, f);
        float Th = 0.0f, rh = 0.0f, ux = 0.0f, uy = 0.0f, uz = 0.0f;
#pragma unroll
        for (int i = 0; i < 7; ++i) Th += g[i];
#pragma unroll
        for (int i = 0; i < 19; ++i) { rh += f[i]; ux += ex(i) * f[i]; uy += ey(i) * f[i]; uz += ez(i) * f[i]; }
        uz += 0.5f * p.gbeta * (Th - p.dTms);
        sT += Th - p.dTms;
        sr += rh;
        n += 1.0;
        const double u2 = (double)ux * ux + (double)uy * uy + (double)uz * uz;
        umax = u2 > umax ? u2 : umax;
    }
    sh[0][threadIdx.x] = sT; sh[1][threadIdx.x] = sr; sh[2][threadIdx.x] = n; sh[3][threadIdx.x] = umax;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) part[blockIdx.x * 4 + threadIdx.x] = sh[threadIdx.x][0];
}

// Final pass in one block: out = {liquid fraction, sum (T - Tm), sum (rho - 1),
// liquid nodes, max |u|, sum s, mean Nusselt number over the heated wall
// (of the per-column values nu)}; with t >= 0 also writes the time first.
static __global__ void __launch_bounds__(256) k_totals_final(const double *__restrict__ part, int nparts,
                                                      const double *__restrict__ s,
                                                      const double *__restrict__ nu, int ncols, double H,
                                                      double t, double *__restrict__ out) {
    __shared__ double sh[6][256];
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, ss = 0.0, sn = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        a0 += part[b * 4];
        a1 += part[b * 4 + 1];
        a2 += part[b * 4 + 2];
        a3 = fmax(a3, part[b * 4 + 3]);
    }
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        ss += s[c];
        sn += nu[c];
    }
    sh[0][threadIdx.x] = a0; sh[1][threadIdx.x] = a1; sh[2][threadIdx.x] = a2; sh[3][threadIdx.x] = a3;
    sh[4][threadIdx.x] = ss; sh[5][threadIdx.x] = sn;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
            sh[2][threadIdx.x] += sh[2][threadIdx.x + w];
            sh[3][threadIdx.x] = fmax(sh[3][threadIdx.x], sh[3][threadIdx.x + w]);
            sh[4][threadIdx.x] += sh[4][threadIdx.x + w];
            sh[5][threadIdx.x] += sh[5][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *o = out;
        if (t >= 0.0) *o++ = t;
        o[0] = sh[4][0] / (H * (double)ncols);
        o[1] = sh[0][0];
        o[2] = sh[1][0];
        o[3] = sh[2][0];
        o[4] = sqrt(sh[3][0]);
        o[5] = sh[4][0];
        o[6] = sh[5][0] / (double)ncols;
    }
}

}  // namespace lbm
