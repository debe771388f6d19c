// lbm_core.cuh -- lattice constants, kernel parameters and the per-node
// double-MRT collision (Li, Yang & Zhang, arXiv:1604.03478, Eqs. 1-5).
//
// Storage convention: every distribution is held SHIFTED by a rest
// equilibrium, fh_i = f_i - w_i rho0 (rho0 = 1) and gh_i = g_i - w_i Ts, so
// that the stored numbers are small (FP16 storage keeps its precision for
// them).  Ts is Tm with FP32 storage (a liquid node at rest and a solid node
// at Tm are all zeros) and the mid temperature (Th + Tm) / 2 with FP16
// storage, which halves the largest stored energy population (|T - Ts| <=
// (Th - Tm) / 2 instead of Th - Tm).
// Arrays are direction-major: direction i of node c lives at base[i*ld + c].
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ---------------------------------------------------------------- lattices
// D3Q19 velocities in the order printed in Eq. 3: rest, +-x, +-y, +-z, then
// the xy, xz and yz diagonals.
__host__ __device__ constexpr int ex(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int ey(int i) {
    return (i == 3 || i == 7 || i == 8 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 9 || i == 10 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int ez(int i) {
    return (i == 5 || i == 11 || i == 12 || i == 15 || i == 16) ? 1
         : (i == 6 || i == 13 || i == 14 || i == 17 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int e2(int i) { return ex(i) * ex(i) + ey(i) * ey(i) + ez(i) * ez(i); }
__host__ __device__ constexpr int opp(int i) {
    int r = 0;
    for (int j = 0; j < 19; ++j)
        if (ex(j) == -ex(i) && ey(j) == -ey(i) && ez(j) == -ez(i)) r = j;
    return r;
}
__host__ __device__ constexpr float w19(int i) {
    return e2(i) == 0 ? 1.0f / 3.0f : (e2(i) == 1 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

// D3Q7 velocities in the order of Eq. 5.
__host__ __device__ constexpr int tx(int i) { return i == 1 ? 1 : (i == 2 ? -1 : 0); }
__host__ __device__ constexpr int ty(int i) { return i == 3 ? 1 : (i == 4 ? -1 : 0); }
__host__ __device__ constexpr int tz(int i) { return i == 5 ? 1 : (i == 6 ? -1 : 0); }
__host__ __device__ constexpr int opp7(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// w0 = 1/4, so the D3Q7 pseudo sound speed squared is (1 - w0)/3 = 1/4.
__host__ __device__ constexpr float w7(int i) { return i == 0 ? 0.25f : 0.125f; }

// Row k of the D3Q19 moment basis (d'Humieres et al. 2002) at velocity i;
// integer-valued on the lattice.
__host__ __device__ constexpr int mpoly(int k, int i) {
    const int x = ex(i), y = ey(i), z = ez(i), q = e2(i);
    return k == 0 ? 1
         : k == 1 ? 19 * q - 30
         : k == 2 ? (21 * q * q - 53 * q + 24) / 2
         : k == 3 ? x
         : k == 4 ? (5 * q - 9) * x
         : k == 5 ? y
         : k == 6 ? (5 * q - 9) * y
         : k == 7 ? z
         : k == 8 ? (5 * q - 9) * z
         : k == 9 ? 3 * x * x - q
         : k == 10 ? (3 * q - 5) * (3 * x * x - q)
         : k == 11 ? y * y - z * z
         : k == 12 ? (3 * q - 5) * (y * y - z * z)
         : k == 13 ? x * y
         : k == 14 ? y * z
         : k == 15 ? x * z
         : k == 16 ? (y * y - z * z) * x
         : k == 17 ? (z * z - x * x) * y
         : (x * x - y * y) * z;
}
// |row k|^2; the rows are orthogonal, so M^-1 = M^T diag(1/norm).
__host__ __device__ constexpr int mnorm(int k) {
    int s = 0;
    for (int i = 0; i < 19; ++i) s += mpoly(k, i) * mpoly(k, i);
    return s;
}

// Row k of the D3Q7 basis: 1, e_x, e_y, e_z, 6 - 7|e|^2, 3e_x^2 - |e|^2,
// e_y^2 - e_z^2.
__host__ __device__ constexpr int npoly(int k, int i) {
    const int x = tx(i), y = ty(i), z = tz(i), q = x * x + y * y + z * z;
    return k == 0 ? 1 : k == 1 ? x : k == 2 ? y : k == 3 ? z
         : k == 4 ? 6 - 7 * q : k == 5 ? 3 * x * x - q : y * y - z * z;
}
__host__ __device__ constexpr int nnorm(int k) {
    int s = 0;
    for (int i = 0; i < 7; ++i) s += npoly(k, i) * npoly(k, i);
    return s;
}

// --------------------------------------------------------- kernel params
// Kernels take KP as a const __grid_constant__ parameter, so its fields are
// read in place from the parameter bank; passed as a plain by-value struct
// of this size the compiler may keep a copy in registers (the even step then
// needed 112 instead of 70 registers a thread).
struct KP {
    int nx, ny, nz;   // cavity
    int H;            // length along the heating axis
    int P1, P2;       // column grid: P1 = nx, P2 = nz (face 0) or ny (face 1)
    int ncols;
    long long N;      // nodes
    long long ld;     // distance between direction arrays (elements)
    float Tm, Tc, gbeta;
    float Ts;         // storage shift of g: gh = g - w Ts
    float dTms;       // Tm - Ts: a node at rest at Tm holds gh = w dTms
    float s_e, s_eps, s_q, s_nu, s_pi, s_m;
    float s_alpha, s_g4, s_g5;
    double Tm_d, Th_d;
    double coef;      // alpha Ste / (Th - Tm): Eq. 6 front speed per unit -dT/da
    float coef_f;     // the same in FP32 (the front speed is FP32 arithmetic)
    int skip_deep;    // Tc == Tm and no conduction in the solid: deep solid nodes need no update
    // Heat conduction in the solid (Eq. 6's k_s term; off: the solid is held
    // at Tm, the zero-subcooling case the paper solves): the solid runs the
    // D3Q7 collision at u = 0 with the flux rate s_alpha_s of alpha_s =
    // kappa alpha (equal rho c in both phases), kappa = k_s / k_l.
    int cond;
    float s_alpha_s, kappa;
};

// Element offsets of the interior odd step, relative to node c: f_i is
// pulled from slot opp(i) of c - e_i and pushed to slot i of c + e_i (g
// likewise).  Passed as a kernel parameter so that they are constant-bank
// operands.
struct Links {
    long long fin[19], fout[19], gin[7], gout[7];
};

// ------------------------------------------------------------ load/store
template <typename ST> struct Store;
// st_stream: a store of the stream-collide, marked evict-first (the state is
// far larger than L2 and is next read a whole step later).
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p) { return *p; }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
    static __device__ __forceinline__ void st_stream(float *p, float v) { __stcs(p, v); }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ void st_stream(__half *p, float v) { __stcs(p, __float2half_rn(v)); }
};

// ----------------------------------------------- compile-time transforms
// The 18 moving velocities form 9 opposite pairs (i, opp(i)); pair P has
// first member pf(P).  A moment row is even or odd in e, so it sees a pair
// only through S = f_i + f_opp(i) (even rows) or D = f_i - f_opp(i) (odd
// rows), which halves the work of m = M f and of f += M^T c.
__host__ __device__ constexpr int pf(int P) {
    return P == 0 ? 1 : P == 1 ? 3 : P == 2 ? 5 : P == 3 ? 7 : P == 4 ? 8 : P == 5 ? 11 : P == 6 ? 12
         : P == 7 ? 15 : 16;
}
__host__ __device__ constexpr bool row_odd(int k) {
    return (k >= 3 && k <= 8) || k >= 16;
}

// acc + sum over pairs of mpoly(K, pf(P)) v[P], nonzero coefficients only.
template <int K, int P>
__device__ __forceinline__ float prow(const float (&v)[9], float acc) {
    if constexpr (P == 9) {
        return acc;
    } else {
        constexpr int m = mpoly(K, pf(P));
        if constexpr (m == 0) return prow<K, P + 1>(v, acc);
        else if constexpr (m == 1) return prow<K, P + 1>(v, acc + v[P]);
        else if constexpr (m == -1) return prow<K, P + 1>(v, acc - v[P]);
        else return prow<K, P + 1>(v, fmaf((float)m, v[P], acc));
    }
}

// m[K] for all rows from the rest population and the pair sums/differences.
template <int K>
__device__ __forceinline__ void moments_pairs(float f0, const float (&S)[9], const float (&D)[9], float (&m)[19]) {
    if constexpr (K < 19) {
        if constexpr (row_odd(K)) m[K] = prow<K, 0>(D, -0.0f);
        else m[K] = prow<K, 0>(S, (float)mpoly(K, 0) * f0);
        moments_pairs<K + 1>(f0, S, D, m);
    }
}

// Sum over rows K.. of mpoly(k, I) c[k] restricted to rows of parity ODD,
// skipping rows whose update is identically zero (mass; x and y momentum).
template <int I, int K, bool ODD>
__device__ __forceinline__ float pcol(const float (&c)[19], float acc) {
    if constexpr (K == 19) {
        return acc;
    } else {
        constexpr int m = mpoly(K, I);
        if constexpr (m == 0 || K == 0 || K == 3 || K == 5 || row_odd(K) != ODD) return pcol<I, K + 1, ODD>(c, acc);
        else if constexpr (m == 1) return pcol<I, K + 1, ODD>(c, acc + c[K]);
        else if constexpr (m == -1) return pcol<I, K + 1, ODD>(c, acc - c[K]);
        else return pcol<I, K + 1, ODD>(c, fmaf((float)m, c[K], acc));
    }
}

// Sum over ALL rows K.. of parity ODD of mpoly(k, I) c[k] (adjoint use: no
// row is identically zero there).
template <int I, int K, bool ODD>
__device__ __forceinline__ float pcol_all(const float (&c)[19], float acc) {
    if constexpr (K == 19) {
        return acc;
    } else {
        constexpr int m = mpoly(K, I);
        if constexpr (m == 0 || row_odd(K) != ODD) return pcol_all<I, K + 1, ODD>(c, acc);
        else if constexpr (m == 1) return pcol_all<I, K + 1, ODD>(c, acc + c[K]);
        else if constexpr (m == -1) return pcol_all<I, K + 1, ODD>(c, acc - c[K]);
        else return pcol_all<I, K + 1, ODD>(c, fmaf((float)m, c[K], acc));
    }
}

// out += M^T c over all rows.
template <int P>
__device__ __forceinline__ void add_back_pairs_all(float (&out)[19], const float (&c)[19]) {
    if constexpr (P < 9) {
        constexpr int i = pf(P), j = opp(pf(P));
        const float E = pcol_all<i, 0, false>(c, -0.0f);
        const float O = pcol_all<i, 0, true>(c, -0.0f);
        out[i] += E + O;
        out[j] += E - O;
        add_back_pairs_all<P + 1>(out, c);
    }
}

// f += M^T c, pair by pair: f_i += E + O, f_opp(i) += E - O.
template <int P>
__device__ __forceinline__ void add_back_pairs(float (&f)[19], const float (&c)[19]) {
    if constexpr (P < 9) {
        constexpr int i = pf(P), j = opp(pf(P));
        const float E = pcol<i, 0, false>(c, -0.0f);
        const float O = pcol<i, 0, true>(c, -0.0f);
        f[i] += E + O;
        f[j] += E - O;
        add_back_pairs<P + 1>(f, c);
    }
}

// c[k] = d[k] / |row k|^2 with the reciprocal formed at compile time.
template <int K>
__device__ __forceinline__ void scale_by_inverse_norms(const float (&d)[19], float (&c)[19]) {
    if constexpr (K < 19) {
        constexpr float inv = 1.0f / (float)mnorm(K);
        c[K] = d[K] * inv;
        scale_by_inverse_norms<K + 1>(d, c);
    }
}

template <int K, int I>
__device__ __forceinline__ float nrow(const float (&v)[7], float acc) {
    if constexpr (I == 7) {
        return acc;
    } else {
        constexpr int m = npoly(K, I);
        if constexpr (m == 0) return nrow<K, I + 1>(v, acc);
        else if constexpr (m == 1) return nrow<K, I + 1>(v, acc + v[I]);
        else if constexpr (m == -1) return nrow<K, I + 1>(v, acc - v[I]);
        else return nrow<K, I + 1>(v, fmaf((float)m, v[I], acc));
    }
}

template <int I, int K>
__device__ __forceinline__ float ncol(const float (&c)[7], float acc) {
    if constexpr (K == 7) {
        return acc;
    } else {
        constexpr int m = npoly(K, I);
        if constexpr (m == 0 || K == 0) return ncol<I, K + 1>(c, acc);
        else if constexpr (m == 1) return ncol<I, K + 1>(c, acc + c[K]);
        else if constexpr (m == -1) return ncol<I, K + 1>(c, acc - c[K]);
        else return ncol<I, K + 1>(c, fmaf((float)m, c[K], acc));
    }
}

// acc + sum over ALL rows k of npoly(k, I) c[k].
template <int I, int K>
__device__ __forceinline__ float ncol_all(const float (&c)[7], float acc) {
    if constexpr (K == 7) {
        return acc;
    } else {
        constexpr int m = npoly(K, I);
        if constexpr (m == 0) return ncol_all<I, K + 1>(c, acc);
        else if constexpr (m == 1) return ncol_all<I, K + 1>(c, acc + c[K]);
        else if constexpr (m == -1) return ncol_all<I, K + 1>(c, acc - c[K]);
        else return ncol_all<I, K + 1>(c, fmaf((float)m, c[K], acc));
    }
}

template <int I>
__device__ __forceinline__ void add_back7_all(float (&g)[7], const float (&c)[7]) {
    if constexpr (I < 7) {
        g[I] = ncol_all<I, 0>(c, g[I]);
        add_back7_all<I + 1>(g, c);
    }
}

template <int I>
__device__ __forceinline__ void add_back7(float (&g)[7], const float (&c)[7]) {
    if constexpr (I < 7) {
        g[I] = ncol<I, 0>(c, g[I]);
        add_back7<I + 1>(g, c);
    }
}

// ------------------------------------- transforms with shared sub-sums
// m = M f and f += M^T c written out by hand over the pair sums S and
// differences D, sharing the partial sums that several rows (or, for the
// back-transform, several pairs) have in common: about 140 additions and
// multiplications for both instead of about 240 when every row and every
// pair is summed on its own.  Pair order: x, y, z axes, then the diagonals
// with first members 7 (1,1,0), 8 (-1,1,0), 11 (1,0,1), 12 (-1,0,1),
// 15 (0,1,1), 16 (0,-1,1).  The coefficients are the d'Humieres rows of
// mpoly at those first members.
__host__ __device__ __forceinline__ void moments_shared(float f0, const float (&S)[9], const float (&D)[9],
                                                        float (&m)[19]) {
    const float Sx = S[0], Sy = S[1], Sz = S[2], S7 = S[3], S8 = S[4], S11 = S[5], S12 = S[6], S15 = S[7], S16 = S[8];
    const float Dx = D[0], Dy = D[1], Dz = D[2], D7 = D[3], D8 = D[4], D11 = D[5], D12 = D[6], D15 = D[7], D16 = D[8];
    const float Sxy = S7 + S8, Sxz = S11 + S12, Syz = S15 + S16;
    const float Sax = Sx + Sy + Sz, Sdg = Sxy + Sxz + Syz;
    m[0] = f0 + Sax + Sdg;
    m[1] = fmaf(8.0f, Sdg, fmaf(-11.0f, Sax, -30.0f * f0));
    m[2] = fmaf(-4.0f, Sax, fmaf(12.0f, f0, Sdg));
    const float a9 = fmaf(2.0f, Sx, -Sy) - Sz, d9 = fmaf(-2.0f, Syz, Sxy + Sxz);
    m[9] = a9 + d9;
    m[10] = fmaf(-2.0f, a9, d9);
    const float a11 = Sy - Sz, d11 = Sxy - Sxz;
    m[11] = a11 + d11;
    m[12] = fmaf(-2.0f, a11, d11);
    m[13] = S7 - S8;
    m[14] = S15 - S16;
    m[15] = S11 - S12;
    const float A = D7 - D8, B = D11 - D12, Xd = A + B;
    m[3] = Dx + Xd;
    m[4] = fmaf(-4.0f, Dx, Xd);
    m[16] = A - B;
    const float C = D7 + D8, E = D15 - D16, Yd = C + E;
    m[5] = Dy + Yd;
    m[6] = fmaf(-4.0f, Dy, Yd);
    m[17] = E - C;
    const float G = D11 + D12, H = D15 + D16, Zd = G + H;
    m[7] = Dz + Zd;
    m[8] = fmaf(-4.0f, Dz, Zd);
    m[18] = G - H;
}

// f += M^T c for c with c[0] = c[3] = c[5] = 0 (mass and in-plane momentum
// are not changed; c[7], the z momentum, carries the force).
__host__ __device__ __forceinline__ void add_back_shared(float (&f)[19], const float (&c)[19]) {
    f[0] = fmaf(12.0f, c[2], fmaf(-30.0f, c[1], f[0]));
    // even rows
    const float Kax = fmaf(-4.0f, c[2], -11.0f * c[1]), Kdg = fmaf(8.0f, c[1], c[2]);
    const float b1 = fmaf(-2.0f, c[10], c[9]), b2 = c[9] + c[10];
    const float b3 = fmaf(-2.0f, c[12], c[11]), b4 = c[11] + c[12];
    const float Ex = fmaf(2.0f, b1, Kax), Ky = Kax - b1, Ey = Ky + b3, Ez = Ky - b3;
    const float K1 = Kdg + b2, K2 = K1 + b4, K3 = K1 - b4, K4 = fmaf(-2.0f, b2, Kdg);
    const float E7 = K2 + c[13], E8 = K2 - c[13], E11 = K3 + c[15], E12 = K3 - c[15];
    const float E15 = K4 + c[14], E16 = K4 - c[14];
    // odd rows
    const float Ox = -4.0f * c[4], Oy = -4.0f * c[6], Oz = fmaf(-4.0f, c[8], c[7]);
    const float P = c[4] + c[16], Q = c[6] - c[17], Pp = c[4] - c[16], Qp = c[6] + c[17];
    const float c78 = c[7] + c[8], R = c78 + c[18], Rp = c78 - c[18];
    const float O7 = P + Q, O8 = Q - P, O11 = Pp + R, O12 = R - Pp, O15 = Qp + Rp, O16 = Rp - Qp;
    // pairs (first member, opposite): (1,2) (3,4) (5,6) (7,10) (8,9) (11,14) (12,13) (15,18) (16,17)
    f[1] += Ex + Ox;   f[2] += Ex - Ox;
    f[3] += Ey + Oy;   f[4] += Ey - Oy;
    f[5] += Ez + Oz;   f[6] += Ez - Oz;
    f[7] += E7 + O7;   f[10] += E7 - O7;
    f[8] += E8 + O8;   f[9] += E8 - O8;
    f[11] += E11 + O11; f[14] += E11 - O11;
    f[12] += E12 + O12; f[13] += E12 - O12;
    f[15] += E15 + O15; f[18] += E15 - O15;
    f[16] += E16 + O16; f[17] += E16 - O16;
}

// --------------------------------------------------- two-lane arithmetic
// Two nodes per thread (lane x and lane y of a float2): every operation is
// one packed FP32x2 instruction of sm_100 and later (add/mul/fma .f32x2,
// each lane rounded to nearest like the scalar FP32 instruction), so two
// nodes cost about the arithmetic instructions of one.  The host versions
// (for checks on the CPU) do the same lane by lane.
__host__ __device__ __forceinline__ float2 v2(float s) { return make_float2(s, s); }
__host__ __device__ __forceinline__ float2 add2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    return __fadd2_rn(a, b);
#else
    return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 mul2(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    return __fmul2_rn(a, b);
#else
    return make_float2(a.x * b.x, a.y * b.y);
#endif
}
__host__ __device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
#ifdef __CUDA_ARCH__
    return __ffma2_rn(a, b, c);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}
// a - b as fma(b, -1, a): one rounding, the exact difference rounded
__host__ __device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(b, v2(-1.0f), a); }
// s b + c and s b with a scalar (uniform) coefficient
__host__ __device__ __forceinline__ float2 sfma2(float s, float2 b, float2 c) { return fma2(v2(s), b, c); }
__host__ __device__ __forceinline__ float2 smul2(float s, float2 b) { return mul2(v2(s), b); }

// moments_shared for two nodes.
__host__ __device__ __forceinline__ void moments_shared2(float2 f0, const float2 (&S)[9], const float2 (&D)[9],
                                                         float2 (&m)[19]) {
    const float2 Sx = S[0], Sy = S[1], Sz = S[2], S7 = S[3], S8 = S[4], S11 = S[5], S12 = S[6], S15 = S[7],
                 S16 = S[8];
    const float2 Dx = D[0], Dy = D[1], Dz = D[2], D7 = D[3], D8 = D[4], D11 = D[5], D12 = D[6], D15 = D[7],
                 D16 = D[8];
    const float2 Sxy = add2(S7, S8), Sxz = add2(S11, S12), Syz = add2(S15, S16);
    const float2 Sax = add2(add2(Sx, Sy), Sz), Sdg = add2(add2(Sxy, Sxz), Syz);
    m[0] = add2(add2(f0, Sax), Sdg);
    m[1] = sfma2(8.0f, Sdg, sfma2(-11.0f, Sax, smul2(-30.0f, f0)));
    m[2] = sfma2(-4.0f, Sax, sfma2(12.0f, f0, Sdg));
    const float2 a9 = sub2(smul2(2.0f, Sx), add2(Sy, Sz));
    const float2 d9 = sfma2(-2.0f, Syz, add2(Sxy, Sxz));
    m[9] = add2(a9, d9);
    m[10] = sfma2(-2.0f, a9, d9);
    const float2 a11 = sub2(Sy, Sz), d11 = sub2(Sxy, Sxz);
    m[11] = add2(a11, d11);
    m[12] = sfma2(-2.0f, a11, d11);
    m[13] = sub2(S7, S8);
    m[14] = sub2(S15, S16);
    m[15] = sub2(S11, S12);
    const float2 A = sub2(D7, D8), B = sub2(D11, D12), Xd = add2(A, B);
    m[3] = add2(Dx, Xd);
    m[4] = sfma2(-4.0f, Dx, Xd);
    m[16] = sub2(A, B);
    const float2 C = add2(D7, D8), E = sub2(D15, D16), Yd = add2(C, E);
    m[5] = add2(Dy, Yd);
    m[6] = sfma2(-4.0f, Dy, Yd);
    m[17] = sub2(E, C);
    const float2 G = add2(D11, D12), H = add2(D15, D16), Zd = add2(G, H);
    m[7] = add2(Dz, Zd);
    m[8] = sfma2(-4.0f, Dz, Zd);
    m[18] = sub2(G, H);
}

// add_back_shared for two nodes (c[0] = c[3] = c[5] = 0).
__host__ __device__ __forceinline__ void add_back_shared2(float2 (&f)[19], const float2 (&c)[19]) {
    f[0] = sfma2(12.0f, c[2], sfma2(-30.0f, c[1], f[0]));
    const float2 Kax = sfma2(-4.0f, c[2], smul2(-11.0f, c[1])), Kdg = sfma2(8.0f, c[1], c[2]);
    const float2 b1 = sfma2(-2.0f, c[10], c[9]), b2 = add2(c[9], c[10]);
    const float2 b3 = sfma2(-2.0f, c[12], c[11]), b4 = add2(c[11], c[12]);
    const float2 Ex = sfma2(2.0f, b1, Kax), Ky = sub2(Kax, b1), Ey = add2(Ky, b3), Ez = sub2(Ky, b3);
    const float2 K1 = add2(Kdg, b2), K2 = add2(K1, b4), K3 = sub2(K1, b4), K4 = sfma2(-2.0f, b2, Kdg);
    const float2 E7 = add2(K2, c[13]), E8 = sub2(K2, c[13]), E11 = add2(K3, c[15]), E12 = sub2(K3, c[15]);
    const float2 E15 = add2(K4, c[14]), E16 = sub2(K4, c[14]);
    const float2 Ox = smul2(-4.0f, c[4]), Oy = smul2(-4.0f, c[6]), Oz = sfma2(-4.0f, c[8], c[7]);
    const float2 P = add2(c[4], c[16]), Q = sub2(c[6], c[17]), Pp = sub2(c[4], c[16]), Qp = add2(c[6], c[17]);
    const float2 c78 = add2(c[7], c[8]), R = add2(c78, c[18]), Rp = sub2(c78, c[18]);
    const float2 O7 = add2(P, Q), O8 = sub2(Q, P), O11 = add2(Pp, R), O12 = sub2(R, Pp), O15 = add2(Qp, Rp),
                 O16 = sub2(Rp, Qp);
    f[1] = add2(f[1], add2(Ex, Ox));    f[2] = add2(f[2], sub2(Ex, Ox));
    f[3] = add2(f[3], add2(Ey, Oy));    f[4] = add2(f[4], sub2(Ey, Oy));
    f[5] = add2(f[5], add2(Ez, Oz));    f[6] = add2(f[6], sub2(Ez, Oz));
    f[7] = add2(f[7], add2(E7, O7));    f[10] = add2(f[10], sub2(E7, O7));
    f[8] = add2(f[8], add2(E8, O8));    f[9] = add2(f[9], sub2(E8, O8));
    f[11] = add2(f[11], add2(E11, O11)); f[14] = add2(f[14], sub2(E11, O11));
    f[12] = add2(f[12], add2(E12, O12)); f[13] = add2(f[13], sub2(E12, O12));
    f[15] = add2(f[15], add2(E15, O15)); f[18] = add2(f[18], sub2(E15, O15));
    f[16] = add2(f[16], add2(E16, O16)); f[17] = add2(f[17], sub2(E16, O16));
}

// -------------------------------------------------------------- collision
// One liquid node: shifted populations in, shifted post-collision out.
//   T = Ts + sum gh;  F = g beta (T - Tm) z-hat (Boussinesq, gravity -z);
//   u = sum fh e + F/2 (rho0 = 1);
//   D3Q19 (Eq. 2 with the Guo source): m* - m = -S (m - m^eq) + (I - S/2) M F~,
//   f* = f + M^T D^-1 (m* - m);
//   D3Q7 (Eq. 4): n* - n = -Q (n - n^eq), n^eq = (T, u T, 3T/4, 0, 0),
//   g* = g + N^T D^-1 (n* - n).
// m^eq and M F~ are the closed forms of the incompressible equilibrium and
// Guo's source for a force along z.  Writes u (for diagnostics) to uout.
__device__ __forceinline__ void collide(const KP &p, float (&f)[19], float (&g)[7], float *uout = nullptr) {
    float Th = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
    const float T = Th + p.Ts;
    const float Fz = p.gbeta * (Th - p.dTms);  // g beta (T - Tm)
    float m[19], S[9], D[9];
#pragma unroll
    for (int P = 0; P < 9; ++P) {
        S[P] = f[pf(P)] + f[opp(pf(P))];
        D[P] = f[pf(P)] - f[opp(pf(P))];
    }
    moments_shared(f[0], S, D, m);
    const float rho_h = m[0];
    const float ux = m[3], uy = m[5], uz = m[7] + 0.5f * Fz;
    const float uu = ux * ux + uy * uy + uz * uz;
    const float uzF = uz * Fz;
    const float pxx = 2.0f * ux * ux - uy * uy - uz * uz;
    const float pww = uy * uy - uz * uz;
    float d[19];
    d[0] = 0.0f; d[3] = 0.0f; d[5] = 0.0f;
    d[1] = -p.s_e * (m[1] - (-11.0f * rho_h + 19.0f * uu)) + (1.0f - 0.5f * p.s_e) * (38.0f * uzF);
    d[2] = -p.s_eps * (m[2] - (3.0f * rho_h - 5.5f * uu)) + (1.0f - 0.5f * p.s_eps) * (-11.0f * uzF);
    d[4] = -p.s_q * (m[4] + (2.0f / 3.0f) * ux);
    d[6] = -p.s_q * (m[6] + (2.0f / 3.0f) * uy);
    d[7] = Fz;
    d[8] = -p.s_q * (m[8] + (2.0f / 3.0f) * uz) + (1.0f - 0.5f * p.s_q) * (-(2.0f / 3.0f) * Fz);
    d[9] = -p.s_nu * (m[9] - pxx) + (1.0f - 0.5f * p.s_nu) * (-2.0f * uzF);
    d[10] = -p.s_pi * (m[10] + 0.5f * pxx) + (1.0f - 0.5f * p.s_pi) * uzF;
    d[11] = -p.s_nu * (m[11] - pww) + (1.0f - 0.5f * p.s_nu) * (-2.0f * uzF);
    d[12] = -p.s_pi * (m[12] + 0.5f * pww) + (1.0f - 0.5f * p.s_pi) * uzF;
    d[13] = -p.s_nu * (m[13] - ux * uy);
    d[14] = -p.s_nu * (m[14] - uy * uz) + (1.0f - 0.5f * p.s_nu) * (uy * Fz);
    d[15] = -p.s_nu * (m[15] - ux * uz) + (1.0f - 0.5f * p.s_nu) * (ux * Fz);
    d[16] = -p.s_m * m[16];
    d[17] = -p.s_m * m[17];
    d[18] = -p.s_m * m[18];
    float c[19];
    scale_by_inverse_norms<0>(d, c);
    add_back_shared(f, c);

    float n1 = g[1] - g[2], n2 = g[3] - g[4], n3 = g[5] - g[6];
    float n4 = 6.0f * g[0] - (g[1] + g[2] + g[3] + g[4] + g[5] + g[6]);
    float n5 = 2.0f * (g[1] + g[2]) - (g[3] + g[4] + g[5] + g[6]);
    float n6 = (g[3] + g[4]) - (g[5] + g[6]);
    constexpr float i1 = 1.0f / (float)nnorm(1), i4 = 1.0f / (float)nnorm(4);
    constexpr float i5 = 1.0f / (float)nnorm(5), i6 = 1.0f / (float)nnorm(6);
    float cn[7];
    cn[0] = 0.0f;
    cn[1] = -p.s_alpha * (n1 - ux * T) * i1;
    cn[2] = -p.s_alpha * (n2 - uy * T) * i1;
    cn[3] = -p.s_alpha * (n3 - uz * T) * i1;
    cn[4] = -p.s_g4 * (n4 - 0.75f * Th) * i4;
    cn[5] = -p.s_g5 * n5 * i5;
    cn[6] = -p.s_g5 * n6 * i6;
    add_back7<0>(g, cn);
    if (uout) { uout[0] = ux; uout[1] = uy; uout[2] = uz; }
}

// collide for two liquid nodes at once (lane x and lane y), packed FP32x2
// arithmetic: the same equations, with each row's rate and inverse norm
// folded into uniform coefficients (c[k] = d[k] / |row k|^2 formed
// directly).
__device__ __forceinline__ void collide2(const KP &p, float2 (&f)[19], float2 (&g)[7]) {
    const float2 g12 = add2(g[1], g[2]), g34 = add2(g[3], g[4]), g56 = add2(g[5], g[6]);
    const float2 Th = add2(g[0], add2(g12, add2(g34, g56)));      // T - Ts
    const float2 T = add2(Th, v2(p.Ts));
    const float2 Fz = sfma2(p.gbeta, Th, v2(-p.gbeta * p.dTms));  // g beta (T - Tm)
    float2 m[19], S[9], D[9];
#pragma unroll
    for (int P = 0; P < 9; ++P) {
        S[P] = add2(f[pf(P)], f[opp(pf(P))]);
        D[P] = sub2(f[pf(P)], f[opp(pf(P))]);
    }
    moments_shared2(f[0], S, D, m);
    const float2 rho_h = m[0];
    const float2 ux = m[3], uy = m[5], uz = sfma2(0.5f, Fz, m[7]);
    const float2 ux2 = mul2(ux, ux), uy2 = mul2(uy, uy), uz2 = mul2(uz, uz);
    const float2 uu = add2(ux2, add2(uy2, uz2));
    const float2 uzF = mul2(uz, Fz);
    const float2 pxx = sub2(smul2(3.0f, ux2), uu);  // 2 ux^2 - uy^2 - uz^2
    const float2 pww = sub2(uy2, uz2);
    constexpr float n1 = 1.0f / (float)mnorm(1), n2 = 1.0f / (float)mnorm(2), n4 = 1.0f / (float)mnorm(4);
    constexpr float n7 = 1.0f / (float)mnorm(7), n9 = 1.0f / (float)mnorm(9), n10 = 1.0f / (float)mnorm(10);
    constexpr float n11 = 1.0f / (float)mnorm(11), n12 = 1.0f / (float)mnorm(12), n13 = 1.0f / (float)mnorm(13);
    constexpr float n16 = 1.0f / (float)mnorm(16);
    const float se = p.s_e, sps = p.s_eps, sq = p.s_q, snu = p.s_nu, spi = p.s_pi, sm = p.s_m;
    float2 c[19];
    // d1 = -s_e (m1 + 11 rho - 19 u^2) + (1 - s_e/2) 38 uz F
    c[1] = sfma2(-se * n1, m[1], sfma2(-11.0f * se * n1, rho_h,
                 sfma2(19.0f * se * n1, uu, smul2(38.0f * (1.0f - 0.5f * se) * n1, uzF))));
    // d2 = -s_eps (m2 - 3 rho + 5.5 u^2) - 11 (1 - s_eps/2) uz F
    c[2] = sfma2(-sps * n2, m[2], sfma2(3.0f * sps * n2, rho_h,
                 sfma2(-5.5f * sps * n2, uu, smul2(-11.0f * (1.0f - 0.5f * sps) * n2, uzF))));
    c[0] = v2(0.0f);
    c[3] = v2(0.0f);
    c[5] = v2(0.0f);
    // d4, d6 = -s_q (m + 2/3 u);  d8 adds -(2/3)(1 - s_q/2) F
    c[4] = sfma2(-sq * n4, m[4], smul2(-(2.0f / 3.0f) * sq * n4, ux));
    c[6] = sfma2(-sq * n4, m[6], smul2(-(2.0f / 3.0f) * sq * n4, uy));
    c[7] = smul2(n7, Fz);
    c[8] = sfma2(-sq * n4, m[8], sfma2(-(2.0f / 3.0f) * sq * n4, uz,
                 smul2(-(2.0f / 3.0f) * (1.0f - 0.5f * sq) * n4, Fz)));
    // viscous rows
    const float knu = 1.0f - 0.5f * snu, kpi = 1.0f - 0.5f * spi;
    c[9] = sfma2(-snu * n9, sub2(m[9], pxx), smul2(-2.0f * knu * n9, uzF));
    c[10] = sfma2(-spi * n10, sfma2(0.5f, pxx, m[10]), smul2(kpi * n10, uzF));
    c[11] = sfma2(-snu * n11, sub2(m[11], pww), smul2(-2.0f * knu * n11, uzF));
    c[12] = sfma2(-spi * n12, sfma2(0.5f, pww, m[12]), smul2(kpi * n12, uzF));
    c[13] = smul2(-snu * n13, sub2(m[13], mul2(ux, uy)));
    c[14] = sfma2(-snu * n13, sub2(m[14], mul2(uy, uz)), smul2(knu * n13, mul2(uy, Fz)));
    c[15] = sfma2(-snu * n13, sub2(m[15], mul2(ux, uz)), smul2(knu * n13, mul2(ux, Fz)));
    c[16] = smul2(-sm * n16, m[16]);
    c[17] = smul2(-sm * n16, m[17]);
    c[18] = smul2(-sm * n16, m[18]);
    add_back_shared2(f, c);

    // D3Q7: n* - n = -Q (n - n^eq), n^eq = (T, u T, 3T/4, 0, 0)
    constexpr float i1 = 1.0f / (float)nnorm(1), i4 = 1.0f / (float)nnorm(4);
    constexpr float i5 = 1.0f / (float)nnorm(5), i6 = 1.0f / (float)nnorm(6);
    const float sa = p.s_alpha, s4 = p.s_g4, s5 = p.s_g5;
    float2 cn[7];
    cn[1] = sfma2(-sa * i1, sub2(g[1], g[2]), smul2(sa * i1, mul2(ux, T)));
    cn[2] = sfma2(-sa * i1, sub2(g[3], g[4]), smul2(sa * i1, mul2(uy, T)));
    cn[3] = sfma2(-sa * i1, sub2(g[5], g[6]), smul2(sa * i1, mul2(uz, T)));
    // n4 = 6 g0 - (g1 + ... + g6) = 7 g0 - Th; n4^eq (shifted) = 3 Th / 4;
    // mc4 = -cn[4]
    const float2 mc4 = smul2(s4 * i4, sfma2(7.0f, g[0], smul2(-1.75f, Th)));
    cn[5] = smul2(-s5 * i5, sub2(smul2(2.0f, g12), add2(g34, g56)));
    cn[6] = smul2(-s5 * i6, sub2(g34, g56));
    // g += N^T cn (row 0 carries nothing): rows 4 and 5 weigh the rest
    // population 6, 0, the x links -1, 2, the y and z links -1, -1
    g[0] = sfma2(-6.0f, mc4, g[0]);
    const float2 ex4 = sfma2(2.0f, cn[5], mc4);
    const float2 yz4 = sub2(mc4, cn[5]);
    g[1] = add2(g[1], add2(ex4, cn[1]));
    g[2] = add2(g[2], sub2(ex4, cn[1]));
    const float2 ey = add2(yz4, cn[6]), ez = sub2(yz4, cn[6]);
    g[3] = add2(g[3], add2(ey, cn[2]));
    g[4] = add2(g[4], sub2(ey, cn[2]));
    g[5] = add2(g[5], add2(ez, cn[3]));
    g[6] = add2(g[6], sub2(ez, cn[3]));
}

// Heat conduction in a solid node: the D3Q7 collision of Eq. 4 at u = 0 with
// the solid's flux rate, n^eq = (T, 0, 0, 0, 3T/4, 0, 0); shifted
// populations in and out.
__device__ __forceinline__ void collide_solid(const KP &p, float (&g)[7]) {
    const float Th = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
    const float n1 = g[1] - g[2], n2 = g[3] - g[4], n3 = g[5] - g[6];
    const float n4 = 6.0f * g[0] - (g[1] + g[2] + g[3] + g[4] + g[5] + g[6]);
    const float n5 = 2.0f * (g[1] + g[2]) - (g[3] + g[4] + g[5] + g[6]);
    const float n6 = (g[3] + g[4]) - (g[5] + g[6]);
    constexpr float i1 = 1.0f / (float)nnorm(1), i4 = 1.0f / (float)nnorm(4);
    constexpr float i5 = 1.0f / (float)nnorm(5), i6 = 1.0f / (float)nnorm(6);
    float cn[7];
    cn[0] = 0.0f;
    cn[1] = -p.s_alpha_s * n1 * i1;
    cn[2] = -p.s_alpha_s * n2 * i1;
    cn[3] = -p.s_alpha_s * n3 * i1;
    cn[4] = -p.s_g4 * (n4 - 0.75f * Th) * i4;
    cn[5] = -p.s_g5 * n5 * i5;
    cn[6] = -p.s_g5 * n6 * i6;
    add_back7<0>(g, cn);
}

// ------------------------------------------------------------- geometry
template <int FACE> __device__ __forceinline__ int axial(int x, int y, int z) {
    (void)x;
    return FACE == 0 ? y : z;
}
template <int FACE> __device__ __forceinline__ int column(const KP &p, int x, int y, int z) {
    return FACE == 0 ? z * p.nx + x : y * p.nx + x;
}
// Node of column col at height j.
template <int FACE> __device__ __forceinline__ void column_node(const KP &p, int col, int j, int &x, int &y, int &z) {
    x = col % p.nx;
    int q = col / p.nx;
    if (FACE == 0) { y = j; z = q; } else { y = q; z = j; }
}
__device__ __forceinline__ long long node_index(const KP &p, int x, int y, int z) {
    return ((long long)z * p.ny + y) * p.nx + x;
}
__device__ __forceinline__ bool inside(const KP &p, int x, int y, int z) {
    return (unsigned)x < (unsigned)p.nx && (unsigned)y < (unsigned)p.ny && (unsigned)z < (unsigned)p.nz;
}
template <int FACE> __device__ __forceinline__ bool liquid_at(const KP &p, const int *js, int x, int y, int z) {
    return inside(p, x, y, z) && axial<FACE>(x, y, z) < __ldg(js + column<FACE>(p, x, y, z));
}

// Wall crossed by the D3Q7 link that leaves node (x,y,z) along direction i
// (i.e. x + t_i is outside): 1 heated wall, 2 opposite isothermal wall,
// 3 adiabatic wall.  Only meaningful when x + t_i is outside.
template <int FACE> __host__ __device__ constexpr int wall_of_link(int i) {
    // the heating axis is y (directions 3, 4) or z (5, 6); the heated wall is
    // at coordinate 0, reached going in the negative direction
    return FACE == 0 ? (i == 4 ? 1 : (i == 3 ? 2 : 3)) : (i == 6 ? 1 : (i == 5 ? 2 : 3));
}

}  // namespace lbm
