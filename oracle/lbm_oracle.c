/*
 * lbm_oracle.c -- plain CPU FP64 oracle of the double-MRT lattice Boltzmann
 * method with interfacial tracking for 3-D melting
 * (Li, Yang, Zhang, "Lattice Boltzmann method simulation of 3-D melting using
 * double MRT model with interfacial tracking method", arXiv:1604.03478).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct restatement
 * of the method that the CUDA library is checked against.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg load it.  It shares no
 * code, header, table or constant with the CUDA library, and the library never
 * calls it.
 *
 * What it computes, one time step (section 2 of the paper):
 *   1. per liquid node: rho, T, the Boussinesq force and the D3Q19 MRT
 *      collision with forcing (Eqs. 1-3) and the D3Q7 MRT collision (Eqs. 4-5);
 *      per solid node: the energy distribution is reset to its rest equilibrium
 *      at the node's imposed temperature;
 *   2. streaming by a double-buffered pull, with halfway bounce-back of f at the
 *      walls and at liquid->solid links, anti-bounce-back of g at the two
 *      isothermal walls and bounce-back of g at the adiabatic walls (section 1);
 *   3. the interfacial-tracking front update from the interface energy balance
 *      (Eq. 6), Jacobi in the columns, in FP64;
 *   4. the phase flip of nodes crossed by the front and the ghost temperature
 *      of the first solid node of each column.
 *
 * Layout: cell index c = (z*ny + y)*nx + x; f[c*19 + i], g[c*7 + i] (cell
 * major).  The exchange format of orc_get_state/orc_set_state is direction
 * major, f[i*N + c], g[i*N + c].
 *
 * Points where the paper defers to other work or is silent, and the reading
 * taken here (each also stated where it is used):
 *   - M, S, m^eq: the Gram-Schmidt D3Q19 moment basis of d'Humieres et al.
 *     (2002); m^eq is obtained as M times the incompressible (rho0 = 1) BGK
 *     equilibrium; the rates are s_nu for the five viscous-stress moments,
 *     s_e, s_eps, s_q, s_pi, s_m for the others, 1 for the conserved ones.
 *   - N, Q, n^eq for D3Q7: the orthogonal basis 1, e_x, e_y, e_z, 6-7|e|^2..,
 *     n^eq = N g^eq with g^eq_i = w_i T (1 + e_i.u / cs2T), w_0 = 1/4,
 *     w_1..6 = 1/8, cs2T = 1/4, so alpha = cs2T (1/s_alpha - 1/2).
 *   - Forcing: Guo's scheme; the velocity is shifted by F/2 and the source
 *     enters moment space as (I - S/2) M F~.
 *   - Gravity along -z, Boussinesq reference temperature T_m.
 *   - The front is a Dirichlet T = T_m surface at sub-grid height s, imposed
 *     on the first solid node of each column (the ghost node) by
 *     non-equilibrium extrapolation: its post-collision energy populations are
 *     the rest equilibrium at a ghost temperature, linearly extrapolated
 *     through (s, T_m), plus the non-equilibrium part of the post-collision
 *     populations of the liquid node directly below it.  Deeper solid nodes
 *     are held at T_m.
 *   - Front gradient: one-sided quadratic through (s, T_m) and the two nearest
 *     liquid nodes at least half a cell below s; the heated wall stands in for
 *     a missing node; linear through wall and front when no node qualifies.
 *   - s_x, s_z: central differences with a mirror ghost at the side walls.
 *   - A node whose centre equals s is solid.  A node newly crossed by the
 *     front gets f = f^eq(rho0 = 1, u = 0); g is carried through a flip
 *     unchanged (every node, solid or liquid, holds and streams g).
 *   - The initial front sits at s0 (one lattice unit by default) with the
 *     liquid at the analytic conduction (Neumann) temperature of that front.
 *
 * Solid-phase conduction (cfg.solid = 1; the paper solves only Tc = Tm,
 * where the solid stays at Tm and the k_s term of Eq. 6 vanishes):
 *   - rho_s c_s = rho_l c_l, so the solid diffusivity is alpha_s =
 *     (k_s / k_l) alpha; a solid node runs the D3Q7 MRT collision at u = 0
 *     with that diffusivity, and its populations stream among solid nodes
 *     and against the walls like the liquid's.
 *   - The interface is imposed on each side by the mirror of the liquid-side
 *     ghost rule: the last liquid node of a column is the solid side's ghost,
 *     with the temperature extrapolated through (s, Tm) and the lowest solid
 *     node at least half a cell above s (the cold wall (H, Tc) standing in
 *     for a missing one), plus the non-equilibrium part of the solid node
 *     above it.  A population that crosses the phase boundary from a node
 *     of the other phase is that node's ghost population when the node is
 *     its column's ghost for the receiving phase, else the rest state at Tm.
 *   - Eq. 6 gains k_s dT_s/dy: the solid-side gradient at s is the one-sided
 *     quadratic through (s, Tm) and the two lowest solid nodes at least half
 *     a cell above s (the cold wall standing in for a missing one), linear
 *     through (s, Tm) and (H, Tc) when none qualifies, and zero in a column
 *     with no solid node.
 *   - The initial solid is at the two-phase Neumann temperature of the front
 *     s0 (a solid initially at Tc); with Tc = Tm everything reduces to the
 *     method above.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Arithmetic type of the method.  The default build computes in double.
   Built with -DORC_COMPLEX the same source computes in double _Complex: a
   perturbation i*h*v of the heated-wall field or of Ra then carries the
   directional derivative of every quantity in its imaginary part (complex-
   step differentiation, a tangent-linear evaluation without cancellation);
   every branch (phase flags, guarded nodes, clamps, stability check) is
   taken on real parts, so the flags are those of the unperturbed run. */
#ifdef ORC_COMPLEX
#include <complex.h>
typedef double _Complex real;
#define RE(x) creal(x)
#define RSQRT(x) csqrt(x)
#else
typedef double real;
#define RE(x) (x)
#define RSQRT(x) sqrt(x)
#endif

#define Q19 19
#define Q7 7

/* Eq. 3: the 19 discrete velocities, columns of the printed 3 x 19 matrix. */
static const int EX[Q19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[Q19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[Q19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};

/* Eq. 5: the 7 discrete velocities of the energy distribution. */
static const int TX[Q7] = {0, 1, -1, 0, 0, 0, 0};
static const int TY[Q7] = {0, 0, 0, 1, -1, 0, 0};
static const int TZ[Q7] = {0, 0, 0, 0, 0, 1, -1};

static const double CS2T = 0.25; /* D3Q7 pseudo sound speed squared, (1 - w0)/3 */

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_EUNSTABLE = -4 };

typedef struct orc_cfg {
    int nx, ny, nz;
    int face;   /* 0: heated wall y = 0 (front columns over x,z); 1: heated wall z = 0 (columns over x,y) */
    double Ra, Pr, Ste, Th, Tc, Tm, Ma;
    double s0;  /* initial front height above the heated wall, lattice units */
    double s_nu, s_e, s_eps, s_q, s_pi, s_m;
    double s_alpha, s_g4, s_g5;
    int derive; /* 1: s_nu and s_alpha from Ra, Pr, Ma and H; 0: as given */
    int solid;    /* 0: solid held at Tm (zero subcooling); 1: heat conduction in the solid */
    double ks_kl; /* k_s / k_l, the solid's conductivity ratio (solid = 1) */
} orc_cfg;

typedef struct orc_sim {
    orc_cfg cfg;
    int H;           /* cavity length along the heating axis */
    int P1, P2;      /* sizes of the two in-plane (column) axes */
    long N, ncols;
    real nu, alpha, gbeta, s_nu_r, s_alpha_r;
    double lambda, t0, Ra_im;
    double M[Q19 * Q19], Minv[Q19 * Q19], Nm[Q7 * Q7], Ninv[Q7 * Q7];
    real S[Q19], Qr[Q7];
    real alpha_s, Qs[Q7];       /* solid diffusivity and D3Q7 rates (solid = 1) */
    real *f, *g, *fs, *gs;     /* current (post-streaming) and post-collision */
    real *s, *snew, *Tghost, *Thw;
    real *Gpost;                /* ghost-node post-collision g, 7 per column */
    real *Spost;                /* solid-side ghost post-collision g, 7 per column (solid = 1) */
    int *js;                      /* number of liquid nodes per column */
    unsigned char *liq;
    long steps;
    real q_hot, q_cold;         /* heat that entered through the isothermal walls, summed over steps */
    int status;
    char err[256];
} orc_sim;

/* ------------------------------------------------------------------ lattice */

static int e2_19(int i) { return EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i]; }

/* D3Q19 weights: 1/3 rest, 1/18 axis, 1/36 diagonal. */
static double w19(int i) {
    int e2 = e2_19(i);
    return e2 == 0 ? 1.0 / 3.0 : (e2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

/* D3Q7 weights (reading: w0 = 1/4 so that cs2T = 1/4). */
static double w7(int i) { return i == 0 ? 0.25 : 0.125; }

static int opp19(int i) {
    for (int j = 0; j < Q19; ++j)
        if (EX[j] == -EX[i] && EY[j] == -EY[i] && EZ[j] == -EZ[i]) return j;
    return -1;
}

static int opp7(int i) {
    for (int j = 0; j < Q7; ++j)
        if (TX[j] == -TX[i] && TY[j] == -TY[i] && TZ[j] == -TZ[i]) return j;
    return -1;
}

/* Row k of the D3Q19 transform M (Eq. 2), the d'Humieres polynomial in e. */
static double m_row_poly(int k, int ex, int ey, int ez) {
    double x = ex, y = ey, z = ez, e2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return 19.0 * e2 - 30.0;
    case 2: return (21.0 * e2 * e2 - 53.0 * e2 + 24.0) / 2.0;
    case 3: return x;
    case 4: return (5.0 * e2 - 9.0) * x;
    case 5: return y;
    case 6: return (5.0 * e2 - 9.0) * y;
    case 7: return z;
    case 8: return (5.0 * e2 - 9.0) * z;
    case 9: return 3.0 * x * x - e2;
    case 10: return (3.0 * e2 - 5.0) * (3.0 * x * x - e2);
    case 11: return y * y - z * z;
    case 12: return (3.0 * e2 - 5.0) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    case 18: return (x * x - y * y) * z;
    }
    return 0.0;
}

/* Row k of the D3Q7 transform N (Eq. 4). */
static double n_row_poly(int k, int ex, int ey, int ez) {
    double x = ex, y = ey, z = ez, e2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return 6.0 - 7.0 * e2;
    case 5: return 3.0 * x * x - e2;
    case 6: return y * y - z * z;
    }
    return 0.0;
}

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success. */
static int invert(int n, const double *A, double *Ainv) {
    double a[Q19 * 2 * Q19];
    int w = 2 * n;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < w; ++c)
            a[r * w + c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r * w + col]) > fabs(a[piv * w + col])) piv = r;
        if (fabs(a[piv * w + col]) < 1e-300) return -1;
        if (piv != col)
            for (int c = 0; c < w; ++c) {
                double t = a[col * w + c];
                a[col * w + c] = a[piv * w + c];
                a[piv * w + c] = t;
            }
        double p = a[col * w + col];
        for (int c = 0; c < w; ++c) a[col * w + c] /= p;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double fac = a[r * w + col];
            if (fac == 0.0) continue;
            for (int c = 0; c < w; ++c) a[r * w + c] -= fac * a[col * w + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r * w + n + c];
    return 0;
}

static void build_M(double *M) {
    for (int k = 0; k < Q19; ++k)
        for (int i = 0; i < Q19; ++i) M[k * Q19 + i] = m_row_poly(k, EX[i], EY[i], EZ[i]);
}

static void build_N(double *Nm) {
    for (int k = 0; k < Q7; ++k)
        for (int i = 0; i < Q7; ++i) Nm[k * Q7 + i] = n_row_poly(k, TX[i], TY[i], TZ[i]);
}

static void matvec(int n, const double *A, const real *x, real *y) {
    for (int r = 0; r < n; ++r) {
        real acc = 0.0;
        for (int c = 0; c < n; ++c) acc += A[r * n + c] * x[c];
        y[r] = acc;
    }
}

/* ------------------------------------------------------------ equilibria */

/* Incompressible D3Q19 BGK equilibrium with rho0 = 1 (the textbook second-order
   polynomial); its moments M f^eq are the m^eq of Eq. 2. */
static void feq19(real rho, const real *u, real *out) {
    real uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q19; ++i) {
        real eu = EX[i] * u[0] + EY[i] * u[1] + EZ[i] * u[2];
        out[i] = w19(i) * (rho + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* D3Q7 equilibrium, linear in u: g^eq_i = w_i T (1 + e_i.u / cs2T). */
static void geq7(real T, const real *u, real *out) {
    for (int i = 0; i < Q7; ++i) {
        real eu = TX[i] * u[0] + TY[i] * u[1] + TZ[i] * u[2];
        out[i] = w7(i) * T * (1.0 + eu / CS2T);
    }
}

/* Guo's discrete forcing term F~_i = w_i [3 (e_i - u).F + 9 (e_i.u)(e_i.F)]
   (the F_i of Eq. 1 before the (I - S/2) moment-space factor). */
static void guo19(const real *u, const real *F, real *out) {
    for (int i = 0; i < Q19; ++i) {
        real e[3] = {EX[i], EY[i], EZ[i]};
        real emuF = (e[0] - u[0]) * F[0] + (e[1] - u[1]) * F[1] + (e[2] - u[2]) * F[2];
        real eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
        real eF = e[0] * F[0] + e[1] * F[1] + e[2] * F[2];
        out[i] = w19(i) * (3.0 * emuF + 9.0 * eu * eF);
    }
}

/* ------------------------------------------------------------- collisions */

/* Eqs. 1-2 with forcing: m = M f; u = (sum f e + F/2)/rho0;
   m* = m - S (m - m^eq) + (I - S/2) M F~;  f* = M^-1 m*.  Writes u too. */
static void collide_f(const double *M, const double *Minv, const real *S,
                      const real *f, const real *F, real *fout, real *u) {
    real m[Q19], meq[Q19], mF[Q19], fe[Q19], Fi[Q19], ms[Q19];
    matvec(Q19, M, f, m);
    real rho = m[0];
    u[0] = m[3] + 0.5 * F[0];
    u[1] = m[5] + 0.5 * F[1];
    u[2] = m[7] + 0.5 * F[2];
    feq19(rho, u, fe);
    matvec(Q19, M, fe, meq);
    guo19(u, F, Fi);
    matvec(Q19, M, Fi, mF);
    for (int k = 0; k < Q19; ++k) ms[k] = m[k] - S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * S[k]) * mF[k];
    matvec(Q19, Minv, ms, fout);
}

/* Eq. 4: n = N g; n* = n - Q (n - n^eq); g* = N^-1 n*. */
static void collide_g(const double *Nm, const double *Ninv, const real *Qr,
                      const real *g, const real *u, real *gout) {
    real n[Q7], neq[Q7], ge[Q7], ns[Q7];
    real T = 0.0;
    for (int i = 0; i < Q7; ++i) T += g[i];
    matvec(Q7, Nm, g, n);
    geq7(T, u, ge);
    matvec(Q7, Nm, ge, neq);
    for (int k = 0; k < Q7; ++k) ns[k] = n[k] - Qr[k] * (n[k] - neq[k]);
    matvec(Q7, Ninv, ns, gout);
}

/* ---------------------------------------------------- front (Eq. 6) rules */

/* Root of lambda exp(lambda^2) erf(lambda) = Ste/sqrt(pi), the one-phase
   Neumann (Stefan) solution for melting with zero subcooling (section 3.1),
   by bisection. */
double orc_neumann_lambda(double Ste) {
    if (!(Ste > 0.0)) return 0.0;
    double rhs = Ste / sqrt(M_PI), lo = 0.0, hi = 1.0;
    while (hi * exp(hi * hi) * erf(hi) < rhs) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid * exp(mid * mid) * erf(mid) < rhs) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Two-phase Neumann solution of conduction melting (a solid initially at
   Tc < Tm; conductivity ratio kappa = k_s / k_l and equal rho c in both
   phases, so alpha_s = kappa alpha_l): the front is s = 2 lambda
   sqrt(alpha_l t), and the interface energy balance (Eq. 6 in one dimension)
   fixes lambda as the root of
       lambda sqrt(pi) / Ste = exp(-lambda^2) / erf(lambda)
           - theta sqrt(kappa) exp(-lambda^2 / kappa) / erfc(lambda / sqrt(kappa))
   with theta = (Tm - Tc) / (Th - Tm).  The right side falls and the left
   rises with lambda, so the root is unique; bisection.  theta = 0 gives the
   one-phase equation of orc_neumann_lambda. */
static double neumann2_residual(double l, double Ste, double theta, double kappa) {
    double r = sqrt(kappa);
    return l * sqrt(M_PI) / Ste - exp(-l * l) / erf(l) + theta * r * exp(-l * l / kappa) / erfc(l / r);
}

double orc_neumann_lambda2(double Ste, double theta, double kappa) {
    if (!(Ste > 0.0) || !(kappa > 0.0)) return 0.0;
    double lo = 0.0, hi = 1.0;
    while (neumann2_residual(hi, Ste, theta, kappa) < 0.0) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (neumann2_residual(mid, Ste, theta, kappa) < 0.0) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Highest node k (centre k + 1/2) at least half a cell below s, or -1. */
static int guarded_node(real s, int n) {
    int k = (int)floor(RE(s) - 1.0);
    if (k > n - 1) k = n - 1;
    return k < 0 ? -1 : k;
}

/* Liquid-side dT/da at the front a = s of one column (the k_l dT_l/dy term of
   Eq. 6).  Tcol holds T at node centres a = j + 1/2; Tw is the heated-wall
   temperature at a = 0.  Quadratic through (y_{k-1}, T_{k-1}), (y_k, T_k),
   (s, Tm), with (0, Tw) standing in for node k-1 when k = 0; linear through
   (0, Tw) and (s, Tm) when no node is at least half a cell below s. */
static real front_gradient(const real *Tcol, int n, real s, real Tw, real Tm) {
    int k = guarded_node(s, n);
    if (k < 0) return (Tm - Tw) / s;
    real x0, y0, x1 = k + 0.5, y1 = Tcol[k], x2 = s, y2 = Tm;
    if (k >= 1) { x0 = k - 0.5; y0 = Tcol[k - 1]; }
    else        { x0 = 0.0;     y0 = Tw; }
    return y0 * (x2 - x1) / ((x0 - x1) * (x0 - x2))
         + y1 * (x2 - x0) / ((x1 - x0) * (x1 - x2))
         + y2 * (2.0 * x2 - x0 - x1) / ((x2 - x0) * (x2 - x1));
}

/* Number of liquid nodes in a column: node j is liquid iff j + 1/2 < s. */
static int n_liquid(real s, int n) {
    int c = 0;
    for (int j = 0; j < n; ++j)
        if (j + 0.5 < RE(s)) ++c;
    return c;
}

/* Ghost temperature of the first solid node of a column: the line through the
   guarded liquid node (or the heated wall) and (s, Tm), evaluated at that
   node's centre.  Returns Tm when the column has no solid node. */
static real ghost_T(const real *Tcol, int n, real s, real Tw, real Tm) {
    int js = n_liquid(s, n);
    if (js >= n) return Tm;
    real yg = js + 0.5;
    int k = guarded_node(s, n);
    if (k < 0) return Tm + (Tm - Tw) * (yg - s) / s;
    return Tm + (Tm - Tcol[k]) * (yg - s) / (s - (k + 0.5));
}

/* Lowest node k (centre k + 1/2) at least half a cell above s, i.e. the
   smallest k >= s; n when there is none. */
static int guarded_solid_node(real s, int n) {
    int k = (int)ceil(RE(s));
    return k > n ? n : k;
}

/* Solid-side dT/da at the front a = s of one column (the k_s dT_s/dy term of
   Eq. 6), the mirror of front_gradient: quadratic through (s, Tm) and the
   guarded solid node k with the node above it, the cold wall (n, Tc)
   standing in for node k + 1 = n; linear through (s, Tm) and (n, Tc) when no
   node is at least half a cell above s.  The caller takes it only in a
   column with a solid node (s <= n - 1/2).  Written with the deviations
   from Tm, so that a solid at Tm gives exactly zero. */
static real solid_gradient(const real *Tcol, int n, real s, real Tc, real Tm) {
    int k = guarded_solid_node(s, n);
    if (k >= n) return (Tc - Tm) / (n - s);
    real x1 = k + 0.5, Y1 = Tcol[k] - Tm, x2, Y2;
    if (k + 1 < n) { x2 = k + 1.5; Y2 = Tcol[k + 1] - Tm; }
    else           { x2 = n;       Y2 = Tc - Tm; }
    return Y1 * (s - x2) / ((x1 - s) * (x1 - x2)) + Y2 * (s - x1) / ((x2 - s) * (x2 - x1));
}

/* Ghost temperature of the solid side at the last liquid node of a column
   (centre js - 1/2): the line through (s, Tm) and the guarded solid node (or
   the cold wall), evaluated there.  Tm when the column has no liquid or no
   solid node. */
static real solid_ghost_T(const real *Tcol, int n, real s, real Tc, real Tm) {
    int js = n_liquid(s, n);
    if (js < 1 || js >= n) return Tm;
    real yg = js - 0.5;
    int k = guarded_solid_node(s, n);
    if (k >= n) return Tm + (Tc - Tm) * (yg - s) / (n - s);
    return Tm + (Tcol[k] - Tm) * (yg - s) / ((k + 0.5) - s);
}

/* ------------------------------------------------------------- geometry */

static void coords(const orc_sim *S, long c, int *x, int *y, int *z) {
    int nx = S->cfg.nx, ny = S->cfg.ny;
    *x = (int)(c % nx);
    *y = (int)((c / nx) % ny);
    *z = (int)(c / ((long)nx * ny));
}

static long cell_index(const orc_sim *S, int x, int y, int z) {
    return ((long)z * S->cfg.ny + y) * S->cfg.nx + x;
}

/* Column index and height along the heating axis of a node. */
static long column_of(const orc_sim *S, int x, int y, int z) {
    return S->cfg.face == 0 ? (long)z * S->cfg.nx + x : (long)y * S->cfg.nx + x;
}

static int axial_of(const orc_sim *S, int x, int y, int z) {
    (void)x;
    return S->cfg.face == 0 ? y : z;
}

/* Cell index of the node at height j of column col. */
static long column_cell(const orc_sim *S, long col, int j) {
    int p = (int)(col % S->cfg.nx), q = (int)(col / S->cfg.nx);
    return S->cfg.face == 0 ? cell_index(S, p, j, q) : cell_index(S, p, q, j);
}

static int inside(const orc_sim *S, int x, int y, int z) {
    return x >= 0 && y >= 0 && z >= 0 && x < S->cfg.nx && y < S->cfg.ny && z < S->cfg.nz;
}

static real cell_T(const orc_sim *S, long c) {
    real T = 0.0;
    for (int i = 0; i < Q7; ++i) T += S->g[c * Q7 + i];
    return T;
}

static void column_T(const orc_sim *S, long col, real *Tcol) {
    for (int j = 0; j < S->H; ++j) Tcol[j] = cell_T(S, column_cell(S, col, j));
}

static void refresh_flags(orc_sim *S) {
    for (long col = 0; col < S->ncols; ++col) S->js[col] = n_liquid(S->s[col], S->H);
    for (long c = 0; c < S->N; ++c) {
        int x, y, z;
        coords(S, c, &x, &y, &z);
        S->liq[c] = (axial_of(S, x, y, z) + 0.5 < RE(S->s[column_of(S, x, y, z)])) ? 1 : 0;
    }
}

/* Force-shifted velocity of a liquid node, u = sum f e + F/2 (rho0 = 1). */
static void cell_u(const orc_sim *S, long c, real T, real *u) {
    const real *f = S->f + c * Q19;
    u[0] = u[1] = u[2] = 0.0;
    for (int i = 0; i < Q19; ++i) {
        u[0] += f[i] * EX[i];
        u[1] += f[i] * EY[i];
        u[2] += f[i] * EZ[i];
    }
    u[2] += 0.5 * S->gbeta * (T - S->cfg.Tm);
}

/* Ghost temperature and ghost-node post-collision populations of every
   column, from the current state: g*_ghost = g^eq(T_ghost, 0) +
   (g*_L - g^eq(T_L, u_L)), L the liquid node below the ghost (none: the
   equilibrium alone).  With solid conduction also the solid side's ghost at
   the last liquid node: g^eq(T_sghost, 0) + (g*_S - g^eq(T_S, 0)), S the
   solid node above it (collided at u = 0 with the solid's rates). */
static void refresh_ghosts(orc_sim *S) {
    real *Tcol = (real *)malloc(sizeof(real) * S->H);
    real zero[3] = {0.0, 0.0, 0.0};
    for (long col = 0; col < S->ncols; ++col) {
        column_T(S, col, Tcol);
        real Tg = ghost_T(Tcol, S->H, S->s[col], S->Thw[col], S->cfg.Tm);
        S->Tghost[col] = Tg;
        real *gp = S->Gpost + col * Q7;
        geq7(Tg, zero, gp);
        int js = S->js[col];
        if (js >= 1 && js < S->H) {
            long L = column_cell(S, col, js - 1);
            real uL[3], gsL[Q7], geL[Q7];
            cell_u(S, L, Tcol[js - 1], uL);
            collide_g(S->Nm, S->Ninv, S->Qr, S->g + L * Q7, uL, gsL);
            geq7(Tcol[js - 1], uL, geL);
            for (int i = 0; i < Q7; ++i) gp[i] += gsL[i] - geL[i];
        }
        if (S->cfg.solid) {
            real *sp = S->Spost + col * Q7;
            geq7(solid_ghost_T(Tcol, S->H, S->s[col], S->cfg.Tc, S->cfg.Tm), zero, sp);
            if (js >= 1 && js < S->H) {
                long Sn = column_cell(S, col, js);
                real gsS[Q7], geS[Q7];
                collide_g(S->Nm, S->Ninv, S->Qs, S->g + Sn * Q7, zero, gsS);
                geq7(Tcol[js], zero, geS);
                for (int i = 0; i < Q7; ++i) sp[i] += gsS[i] - geS[i];
            }
        }
    }
    free(Tcol);
}

/* ------------------------------------------------------------- creation */

static int set_err(orc_sim *S, const char *msg) {
    snprintf(S->err, sizeof S->err, "%s", msg);
    return ORC_EINVAL;
}

/* Lattice parameters (section 1 and Eq. 7).  With U0 = Ma c_s, c_s = 1/sqrt(3):
   nu = U0 H sqrt(Pr/Ra), alpha = nu/Pr; otherwise nu and alpha follow from the
   given rates.  g*beta = Ra nu alpha / ((Th - Tm) H^3) in both cases. */
static int derive(orc_sim *S) {
    orc_cfg *c = &S->cfg;
    S->H = c->face == 0 ? c->ny : c->nz;
    S->P1 = c->nx;
    S->P2 = c->face == 0 ? c->nz : c->ny;
    if (c->nx < 1 || c->ny < 1 || c->nz < 1 || S->H < 4) return set_err(S, "grid too small");
    if (c->face != 0 && c->face != 1) return set_err(S, "face must be 0 or 1");
    if (!(c->Th > c->Tm)) return set_err(S, "Th must exceed Tm");
    if (c->Tc > c->Tm) return set_err(S, "Tc must not exceed Tm");
    if (!(c->Ste >= 0.0)) return set_err(S, "Ste must be >= 0");
    if (!(c->Ra >= 0.0)) return set_err(S, "Ra must be >= 0");
    /* Ra carries the complex-step perturbation in the complex build */
    real Ra = c->Ra;
#ifdef ORC_COMPLEX
    Ra += I * S->Ra_im;
#endif
    if (c->derive) {
        if (!(c->Ra > 0.0) || !(c->Pr > 0.0) || !(c->Ma > 0.0)) return set_err(S, "derive needs Ra, Pr, Ma > 0");
        real U0 = c->Ma / sqrt(3.0);
        S->nu = U0 * S->H * RSQRT(c->Pr / Ra);
        S->alpha = S->nu / c->Pr;
        S->s_nu_r = 1.0 / (3.0 * S->nu + 0.5);
        S->s_alpha_r = 1.0 / (S->alpha / CS2T + 0.5);
    } else {
        S->s_nu_r = c->s_nu;
        S->s_alpha_r = c->s_alpha;
        S->nu = (1.0 / c->s_nu - 0.5) / 3.0;
        S->alpha = CS2T * (1.0 / c->s_alpha - 0.5);
    }
    S->gbeta = c->Ra > 0.0 ? Ra * S->nu * S->alpha / ((c->Th - c->Tm) * pow((double)S->H, 3)) : 0.0;
    double s0 = c->s0 > 0.0 ? c->s0 : 1.0;
    if (s0 < 0.5 || s0 > S->H) return set_err(S, "s0 outside [0.5, H]");
    c->s0 = s0;
    /* D3Q19 rates by moment row: conserved rows 0, 3, 5, 7 are inert (1). */
    real sr[Q19] = {1.0, c->s_e, c->s_eps, 1.0, c->s_q, 1.0, c->s_q, 1.0, c->s_q,
                      S->s_nu_r, c->s_pi, S->s_nu_r, c->s_pi, S->s_nu_r, S->s_nu_r, S->s_nu_r,
                      c->s_m, c->s_m, c->s_m};
    memcpy(S->S, sr, sizeof sr);
    real qr[Q7] = {1.0, S->s_alpha_r, S->s_alpha_r, S->s_alpha_r, c->s_g4, c->s_g5, c->s_g5};
    memcpy(S->Qr, qr, sizeof qr);
    /* Solid conduction: alpha_s = (k_s / k_l) alpha (equal rho c), the same
       D3Q7 basis and higher-order rates. */
    if (c->solid != 0 && c->solid != 1) return set_err(S, "solid must be 0 or 1");
    if (c->solid && !(c->ks_kl > 0.0)) return set_err(S, "ks_kl must be > 0");
    S->alpha_s = c->solid ? c->ks_kl * S->alpha : S->alpha;
    real sas = 1.0 / (S->alpha_s / CS2T + 0.5);
    real qs[Q7] = {1.0, sas, sas, sas, c->s_g4, c->s_g5, c->s_g5};
    memcpy(S->Qs, qs, sizeof qs);
    return ORC_OK;
}

orc_sim *orc_create(const orc_cfg *cfg, char *err, int errlen) {
    orc_sim *S = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!S) return NULL;
    S->cfg = *cfg;
    if (derive(S) != ORC_OK) {
        if (err) snprintf(err, errlen, "%s", S->err);
        free(S);
        return NULL;
    }
    build_M(S->M);
    build_N(S->Nm);
    invert(Q19, S->M, S->Minv);
    invert(Q7, S->Nm, S->Ninv);
    S->N = (long)cfg->nx * cfg->ny * cfg->nz;
    S->ncols = (long)S->P1 * S->P2;
    S->f = (real *)calloc((size_t)S->N * Q19, sizeof(real));
    S->fs = (real *)calloc((size_t)S->N * Q19, sizeof(real));
    S->g = (real *)calloc((size_t)S->N * Q7, sizeof(real));
    S->gs = (real *)calloc((size_t)S->N * Q7, sizeof(real));
    S->s = (real *)calloc(S->ncols, sizeof(real));
    S->snew = (real *)calloc(S->ncols, sizeof(real));
    S->Tghost = (real *)calloc(S->ncols, sizeof(real));
    S->Thw = (real *)calloc(S->ncols, sizeof(real));
    S->js = (int *)calloc(S->ncols, sizeof(int));
    S->Gpost = (real *)calloc((size_t)S->ncols * Q7, sizeof(real));
    S->Spost = (real *)calloc((size_t)S->ncols * Q7, sizeof(real));
    S->liq = (unsigned char *)calloc(S->N, 1);
    if (!S->f || !S->fs || !S->g || !S->gs || !S->s || !S->snew || !S->Tghost || !S->Thw || !S->js ||
        !S->Gpost || !S->Spost || !S->liq) {
        if (err) snprintf(err, errlen, "out of memory");
        free(S->f); free(S->fs); free(S->g); free(S->gs); free(S->s); free(S->snew);
        free(S->Tghost); free(S->Thw); free(S->js); free(S->Gpost); free(S->Spost); free(S->liq); free(S);
        return NULL;
    }
    const orc_cfg *c = &S->cfg;
    /* Initial state: front at s0; liquid at the Neumann temperature of that
       front, T = Th - (Th - Tm) erf(a / (2 sqrt(alpha t0))) / erf(lambda) with
       t0 = s0^2 / (4 lambda^2 alpha); at rest, rho = 1.  With Ste = 0 (front
       held fixed) the liquid starts at Tm.  Solid at Tm; with solid
       conduction and Tc < Tm, lambda is the two-phase one and the solid is at
       T = Tc + (Tm - Tc) erfc(a / (2 sqrt(alpha_s t0))) / erfc(lambda /
       sqrt(kappa)) (at Tc when Ste = 0). */
    const int subcooled = c->solid && c->Tc < c->Tm;
    const double kappa = c->solid ? c->ks_kl : 1.0;
    S->lambda = subcooled ? orc_neumann_lambda2(c->Ste, (c->Tm - c->Tc) / (c->Th - c->Tm), kappa)
                          : orc_neumann_lambda(c->Ste);
    S->t0 = c->Ste > 0.0 ? c->s0 * c->s0 / (4.0 * S->lambda * S->lambda * RE(S->alpha)) : 0.0;
    for (long col = 0; col < S->ncols; ++col) {
        S->s[col] = c->s0;
        S->Thw[col] = c->Th;
    }
    refresh_flags(S);
    real zero[3] = {0.0, 0.0, 0.0};
    for (long cc = 0; cc < S->N; ++cc) {
        int x, y, z;
        coords(S, cc, &x, &y, &z);
        double a = axial_of(S, x, y, z) + 0.5;
        real T = c->Tm;
        if (S->liq[cc]) {
            /* alpha t0 = s0^2 / (4 lambda^2) does not depend on alpha */
            if (c->Ste > 0.0)
                T = c->Th - (c->Th - c->Tm) * erf(a / (2.0 * sqrt(RE(S->alpha) * S->t0))) / erf(S->lambda);
            feq19(1.0, zero, S->f + cc * Q19);
        } else if (subcooled) {
            /* alpha_s t0 = kappa s0^2 / (4 lambda^2) */
            T = c->Tc;
            if (c->Ste > 0.0) {
                double r = sqrt(kappa);
                T = c->Tc + (c->Tm - c->Tc) * erfc(S->lambda * a / (r * c->s0)) / erfc(S->lambda / r);
            }
        }
        geq7(T, zero, S->g + cc * Q7);
    }
    refresh_ghosts(S);
    return S;
}

void orc_destroy(orc_sim *S) {
    if (!S) return;
    free(S->f); free(S->fs); free(S->g); free(S->gs); free(S->s); free(S->snew);
    free(S->Tghost); free(S->Thw); free(S->js); free(S->Gpost); free(S->Spost); free(S->liq);
    free(S);
}

/* ---------------------------------------------------------------- stepping */

static void collide_all(orc_sim *S) {
    const real Tm = S->cfg.Tm;
    #pragma omp parallel for schedule(static)
    for (long c = 0; c < S->N; ++c) {
        int x, y, z;
        coords(S, c, &x, &y, &z);
        if (S->liq[c]) {
            const real *g = S->g + c * Q7;
            real T = 0.0;
            for (int i = 0; i < Q7; ++i) T += g[i];
            /* Boussinesq buoyancy, gravity along -z, reference temperature Tm. */
            real F[3] = {0.0, 0.0, S->gbeta * (T - Tm)};
            real u[3];
            collide_f(S->M, S->Minv, S->S, S->f + c * Q19, F, S->fs + c * Q19, u);
            collide_g(S->Nm, S->Ninv, S->Qr, g, u, S->gs + c * Q7);
        } else if (S->cfg.solid) {
            /* heat conduction in the solid: D3Q7 MRT at u = 0 */
            real zero[3] = {0.0, 0.0, 0.0};
            collide_g(S->Nm, S->Ninv, S->Qs, S->g + c * Q7, zero, S->gs + c * Q7);
            for (int i = 0; i < Q19; ++i) S->fs[c * Q19 + i] = 0.0;
        } else {
            long col = column_of(S, x, y, z);
            int j = axial_of(S, x, y, z);
            real zero[3] = {0.0, 0.0, 0.0};
            if (j == S->js[col]) /* ghost node */
                memcpy(S->gs + c * Q7, S->Gpost + col * Q7, sizeof(real) * Q7);
            else
                geq7(Tm, zero, S->gs + c * Q7);
            for (int i = 0; i < Q19; ++i) S->fs[c * Q19 + i] = 0.0;
        }
    }
}

/* Which wall a D3Q7 link from node (x,y,z) against direction i crosses:
   returns 1 for the heated wall, 2 for the opposite isothermal wall, 3 for an
   adiabatic wall, 0 if the upstream node is inside. */
static int wall_kind7(const orc_sim *S, int x, int y, int z, int i) {
    int ux = x - TX[i], uy = y - TY[i], uz = z - TZ[i];
    if (inside(S, ux, uy, uz)) return 0;
    int axis = TX[i] != 0 ? 0 : (TY[i] != 0 ? 1 : 2);
    int heat_axis = S->cfg.face == 0 ? 1 : 2;
    if (axis != heat_axis) return 3;
    int up = axis == 1 ? uy : uz;
    return up < 0 ? 1 : 2;
}

/* With solid conduction: the D3Q7 population that streams from node u to
   its neighbour c along direction i.  Within a phase it is u's own
   post-collision value; across the phase boundary it is u's ghost
   population for c's phase when u is its column's ghost for that phase (the
   first solid node for a liquid c, the last liquid node for a solid c), else
   the rest state at Tm. */
static real crossing_g(const orc_sim *S, long u, long c, int i) {
    if (S->liq[u] == S->liq[c]) return S->gs[u * Q7 + i];
    int x, y, z;
    coords(S, u, &x, &y, &z);
    long col = column_of(S, x, y, z);
    int j = axial_of(S, x, y, z);
    if (S->liq[u]) /* a solid c */
        return j == S->js[col] - 1 ? S->Spost[col * Q7 + i] : w7(i) * S->cfg.Tm;
    return j == S->js[col] ? S->Gpost[col * Q7 + i] : w7(i) * S->cfg.Tm;
}

static void stream_all(orc_sim *S) {
    #pragma omp parallel for schedule(static)
    for (long c = 0; c < S->N; ++c) {
        int x, y, z;
        coords(S, c, &x, &y, &z);
        real *fn = S->f + c * Q19;
        if (S->liq[c]) {
            for (int i = 0; i < Q19; ++i) {
                int ux = x - EX[i], uy = y - EY[i], uz = z - EZ[i];
                if (inside(S, ux, uy, uz) && S->liq[cell_index(S, ux, uy, uz)])
                    fn[i] = S->fs[cell_index(S, ux, uy, uz) * Q19 + i];
                else /* halfway bounce-back at a wall or a solid node */
                    fn[i] = S->fs[c * Q19 + opp19(i)];
            }
        } else {
            for (int i = 0; i < Q19; ++i) fn[i] = 0.0;
        }
        real *gn = S->g + c * Q7;
        long col = column_of(S, x, y, z);
        for (int i = 0; i < Q7; ++i) {
            int kind = wall_kind7(S, x, y, z, i);
            if (kind == 0) {
                long u = cell_index(S, x - TX[i], y - TY[i], z - TZ[i]);
                gn[i] = S->cfg.solid ? crossing_g(S, u, c, i) : S->gs[u * Q7 + i];
            } else if (kind == 3) { /* adiabatic wall: bounce-back */
                gn[i] = S->gs[c * Q7 + opp7(i)];
            } else { /* isothermal wall: anti-bounce-back -g*_opp + 2 w_i Tw */
                real Tw = kind == 1 ? S->Thw[col] : S->cfg.Tc;
                gn[i] = -S->gs[c * Q7 + opp7(i)] + 2.0 * w7(i) * Tw;
            }
        }
    }
    /* Heat that entered through the isothermal walls this step (diagnostic):
       (incoming - outgoing) population on each wall link. */
    for (long col = 0; col < S->ncols; ++col) {
        for (int end = 0; end < 2; ++end) {
            long c = column_cell(S, col, end == 0 ? 0 : S->H - 1);
            int x, y, z;
            coords(S, c, &x, &y, &z);
            for (int i = 0; i < Q7; ++i) {
                int kind = wall_kind7(S, x, y, z, i);
                if (kind == 1 || kind == 2) {
                    real in = S->g[c * Q7 + i], out = S->gs[c * Q7 + opp7(i)];
                    if (kind == 1) S->q_hot += in - out; else S->q_cold += in - out;
                }
            }
        }
    }
}

/* Eq. 6 with k_s = k_l, a solid held at Tm (zero subcooling, so the solid-side
   gradient vanishes) and rho_l h_sl / k_l = Ste / (alpha (Th - Tm)) in lattice
   units:  ds/dt = alpha Ste / (Th - Tm) (1 + s_p^2 + s_q^2) (-dT_l/da).
   With solid conduction the solid side's term enters:
   ds/dt = alpha Ste / (Th - Tm) (1 + s_p^2 + s_q^2) (kappa dT_s/da - dT_l/da).
   In-plane slopes by central differences, mirror ghost at the side walls.
   All columns read the old s (Jacobi). */
static int front_update(orc_sim *S) {
    const orc_cfg *c = &S->cfg;
    int P1 = S->P1, P2 = S->P2, bad = 0;
    /* Ste = 0 (infinite latent heat) holds the front in place. */
    real coef = c->Ste > 0.0 ? S->alpha * c->Ste / (c->Th - c->Tm) : 0.0;
    real *Tcol = (real *)malloc(sizeof(real) * S->H);
    for (long col = 0; col < S->ncols; ++col) {
        int p = (int)(col % P1), q = (int)(col / P1);
        real sp_hi = S->s[(long)q * P1 + (p + 1 < P1 ? p + 1 : p)];
        real sp_lo = S->s[(long)q * P1 + (p - 1 >= 0 ? p - 1 : p)];
        real sq_hi = S->s[(long)(q + 1 < P2 ? q + 1 : q) * P1 + p];
        real sq_lo = S->s[(long)(q - 1 >= 0 ? q - 1 : q) * P1 + p];
        real sp = 0.5 * (sp_hi - sp_lo), sq = 0.5 * (sq_hi - sq_lo);
        column_T(S, col, Tcol);
        real G = front_gradient(Tcol, S->H, S->s[col], S->Thw[col], c->Tm);
        /* solid conduction: + (k_s / k_l) dT_s/da, in a column with a solid node */
        real Gs = 0.0;
        if (c->solid && n_liquid(S->s[col], S->H) < S->H)
            Gs = c->ks_kl * solid_gradient(Tcol, S->H, S->s[col], c->Tc, c->Tm);
        real v = c->solid ? coef * (1.0 + sp * sp + sq * sq) * (Gs - G) : coef * (1.0 + sp * sp + sq * sq) * (-G);
        if (!(fabs(RE(v)) <= 0.5)) bad = 1;
        real sn = S->s[col] + v;
        if (RE(sn) < 0.5) sn = 0.5;
        if (RE(sn) > S->H) sn = S->H;
        S->snew[col] = sn;
    }
    free(Tcol);
    real *t = S->s; S->s = S->snew; S->snew = t;
    return bad ? ORC_EUNSTABLE : ORC_OK;
}

/* Phase flip: a node the front passed becomes liquid with f = f^eq(1, 0); a
   node the front receded over becomes solid (its f is dropped).  g is kept. */
static void flip(orc_sim *S) {
    real zero[3] = {0.0, 0.0, 0.0}, fe[Q19];
    feq19(1.0, zero, fe);
    for (long c = 0; c < S->N; ++c) {
        int x, y, z;
        coords(S, c, &x, &y, &z);
        unsigned char now = (axial_of(S, x, y, z) + 0.5 < RE(S->s[column_of(S, x, y, z)])) ? 1 : 0;
        if (now && !S->liq[c]) memcpy(S->f + c * Q19, fe, sizeof fe);
        if (!now && S->liq[c]) memset(S->f + c * Q19, 0, sizeof fe);
        S->liq[c] = now;
    }
    for (long col = 0; col < S->ncols; ++col) S->js[col] = n_liquid(S->s[col], S->H);
}

int orc_step(orc_sim *S, long nsteps) {
    for (long t = 0; t < nsteps; ++t) {
        if (S->status != ORC_OK) return S->status;
        collide_all(S);
        /* stream_all overwrites the pre-collision arrays with the new state */
        stream_all(S);
        int st = front_update(S);
        flip(S);
        refresh_ghosts(S);
        S->steps++;
        if (st != ORC_OK) {
            S->status = st;
            snprintf(S->err, sizeof S->err, "front moved more than half a cell in one step");
            return st;
        }
    }
    return ORC_OK;
}

/* --------------------------------------------------------------- outputs */

/* T and u per node (liquid: T = sum g, u = (sum f e + F/2)/rho0; solid:
   T = Tm, or sum g with solid conduction, u = 0), the front heights, and the
   liquid fraction sum(s)/(H ncols). */
void orc_get(const orc_sim *S, double *T, double *u, double *s, double *lf) {
    for (long c = 0; c < S->N; ++c) {
        real Tc = S->cfg.solid ? cell_T(S, c) : S->cfg.Tm, uc[3] = {0.0, 0.0, 0.0};
        if (S->liq[c]) {
            Tc = cell_T(S, c);
            const real *f = S->f + c * Q19;
            for (int i = 0; i < Q19; ++i) {
                uc[0] += f[i] * EX[i];
                uc[1] += f[i] * EY[i];
                uc[2] += f[i] * EZ[i];
            }
            uc[2] += 0.5 * S->gbeta * (Tc - S->cfg.Tm);
        }
        if (T) T[c] = RE(Tc);
        if (u) { u[3 * c] = RE(uc[0]); u[3 * c + 1] = RE(uc[1]); u[3 * c + 2] = RE(uc[2]); }
    }
    if (s)
        for (long col = 0; col < S->ncols; ++col) s[col] = RE(S->s[col]);
    if (lf) {
        real acc = 0.0;
        for (long col = 0; col < S->ncols; ++col) acc += S->s[col];
        *lf = RE(acc / ((double)S->H * (double)S->ncols));
    }
}

/* Local Nusselt number on the heated wall (the heat-surface diagnostic of
   section 3.2, Fig. 4(b)): Nu = -H (dT/da at the wall) / (Th - Tm), the
   conduction flux through the wall expressed against the scalar Th.  The
   flux is the heat the last step's streaming carried through each wall link
   of the column, incoming population minus the outgoing post-collision one
   (in - out on the anti-bounce-back link of the first node), and equals
   -alpha dT/da there.  Per column (column order of S) and the mean over the
   wall.  Defined after at least one step. */
void orc_nusselt(const orc_sim *S, double *Nu, double *Nu_mean) {
    int up = S->cfg.face == 0 ? 3 : 5; /* the D3Q7 direction pointing away from the heated wall */
    int down = opp7(up);
    double scale = (double)S->H / (RE(S->alpha) * (S->cfg.Th - S->cfg.Tm));
    double acc = 0.0;
    for (long col = 0; col < S->ncols; ++col) {
        long c = column_cell(S, col, 0);
        double q = RE(S->g[c * Q7 + up]) - RE(S->gs[c * Q7 + down]);
        double nu = q * scale;
        if (Nu) Nu[col] = nu;
        acc += nu;
    }
    if (Nu_mean) *Nu_mean = acc / (double)S->ncols;
}

/* Natural (post-streaming, pre-collision) distributions, direction major. */
void orc_get_state(const orc_sim *S, double *f, double *g, double *s) {
    if (f)
        for (long c = 0; c < S->N; ++c)
            for (int i = 0; i < Q19; ++i) f[(long)i * S->N + c] = RE(S->f[c * Q19 + i]);
    if (g)
        for (long c = 0; c < S->N; ++c)
            for (int i = 0; i < Q7; ++i) g[(long)i * S->N + c] = RE(S->g[c * Q7 + i]);
    if (s)
        for (long col = 0; col < S->ncols; ++col) s[col] = RE(S->s[col]);
}

/* Replace the state; flags and ghost nodes are recomputed from s and g.  A
   solid node's own populations never enter the method (its post-collision
   values are reset every step), so solid nodes are stored at rest: f = 0,
   g = g^eq(Tm, 0).  With solid conduction a solid node keeps the given g
   (f = 0). */
void orc_set_state(orc_sim *S, const double *f, const double *g, const double *s) {
    if (s)
        for (long col = 0; col < S->ncols; ++col) S->s[col] = s[col];
    refresh_flags(S);
    real zero[3] = {0.0, 0.0, 0.0}, gm[Q7];
    geq7(S->cfg.Tm, zero, gm);
    if (f)
        for (long c = 0; c < S->N; ++c)
            for (int i = 0; i < Q19; ++i) S->f[c * Q19 + i] = S->liq[c] ? f[(long)i * S->N + c] : 0.0;
    if (g)
        for (long c = 0; c < S->N; ++c)
            for (int i = 0; i < Q7; ++i)
                S->g[c * Q7 + i] = (S->liq[c] || S->cfg.solid) ? g[(long)i * S->N + c] : gm[i];
    refresh_ghosts(S);
}

/* Heated-wall temperature per column (overrides the scalar Th at the wall).
   It takes effect at the next step's streaming; the ghost nodes of the
   current state were prepared with the field of the step that produced it. */
void orc_set_hot_wall(orc_sim *S, const double *Thw) {
    for (long col = 0; col < S->ncols; ++col) S->Thw[col] = Thw[col];
}

/* info[0..]: nu, alpha, gbeta, lambda, t0, s_nu, s_alpha, H, steps, q_hot,
   q_cold, liquid mass (sum rho over liquid nodes), liquid node count,
   sum of T over liquid nodes, sum of T over solid nodes (Tm each without
   solid conduction), alpha_s. */
void orc_info(const orc_sim *S, double *info) {
    double mass = 0.0, nl = 0.0, eT = 0.0, eS = 0.0;
    for (long c = 0; c < S->N; ++c) {
        if (!S->liq[c]) {
            eS += S->cfg.solid ? RE(cell_T(S, c)) : S->cfg.Tm;
            continue;
        }
        for (int i = 0; i < Q19; ++i) mass += RE(S->f[c * Q19 + i]);
        eT += RE(cell_T(S, c));
        nl += 1.0;
    }
    double v[16] = {RE(S->nu), RE(S->alpha), RE(S->gbeta), S->lambda, S->t0, RE(S->s_nu_r), RE(S->s_alpha_r),
                    (double)S->H, (double)S->steps, RE(S->q_hot), RE(S->q_cold), mass, nl, eT, eS,
                    RE(S->alpha_s)};
    memcpy(info, v, sizeof v);
}

const char *orc_error(const orc_sim *S) { return S->err; }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops from now on (a timing knob; no effect on the
   results, which do not depend on the thread count). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ----------------------------------------------------- unit-level exports */
#ifndef ORC_COMPLEX

void orc_lattice19(int *ex, int *ey, int *ez, real *w, int *opp) {
    for (int i = 0; i < Q19; ++i) {
        ex[i] = EX[i]; ey[i] = EY[i]; ez[i] = EZ[i]; w[i] = w19(i); opp[i] = opp19(i);
    }
}

void orc_lattice7(int *ex, int *ey, int *ez, real *w, int *opp) {
    for (int i = 0; i < Q7; ++i) {
        ex[i] = TX[i]; ey[i] = TY[i]; ez[i] = TZ[i]; w[i] = w7(i); opp[i] = opp7(i);
    }
}

void orc_matrices(real *M, real *Minv, real *Nm, real *Ninv) {
    real a[Q19 * Q19], b[Q7 * Q7];
    build_M(a);
    build_N(b);
    if (M) memcpy(M, a, sizeof a);
    if (Minv) invert(Q19, a, Minv);
    if (Nm) memcpy(Nm, b, sizeof b);
    if (Ninv) invert(Q7, b, Ninv);
}

void orc_feq19(real rho, const real *u, real *out) { feq19(rho, u, out); }
void orc_geq7(real T, const real *u, real *out) { geq7(T, u, out); }
void orc_guo19(const real *u, const real *F, real *out) { guo19(u, F, out); }

/* One D3Q19 collision with the given 19 rates and force; u receives the
   force-shifted velocity. */
void orc_collide_f(const real *f, const real *S19, const real *F, real *fout, real *u) {
    real M[Q19 * Q19], Minv[Q19 * Q19];
    build_M(M);
    invert(Q19, M, Minv);
    collide_f(M, Minv, S19, f, F, fout, u);
}

void orc_collide_g(const real *g, const real *Q, const real *u, real *gout) {
    real Nm[Q7 * Q7], Ninv[Q7 * Q7];
    build_N(Nm);
    invert(Q7, Nm, Ninv);
    collide_g(Nm, Ninv, Q, g, u, gout);
}

/* Liquid-side front gradient and ghost temperature of one column (the
   Eq. 6 stencil and the interface ghost rule), for unit tests. */
double orc_front_gradient(const double *Tcol, int n, double s, double Tw, double Tm) {
    return front_gradient(Tcol, n, s, Tw, Tm);
}

double orc_ghost_T(const double *Tcol, int n, double s, double Tw, double Tm) {
    return ghost_T(Tcol, n, s, Tw, Tm);
}

/* Solid-side front gradient and ghost temperature of one column. */
double orc_solid_gradient(const double *Tcol, int n, double s, double Tc, double Tm) {
    return solid_gradient(Tcol, n, s, Tc, Tm);
}

double orc_solid_ghost_T(const double *Tcol, int n, double s, double Tc, double Tm) {
    return solid_ghost_T(Tcol, n, s, Tc, Tm);
}
#else
/* --------------------------------------------- complex-step (tangent) API */

/* Perturb Ra by i*h*dRa and the heated-wall field by i*h*dTw (h folded into
   the caller's direction), re-deriving the lattice parameters; the state
   keeps its real part.  Call right after orc_create. */
int orc_cs_perturb(orc_sim *S, double Ra_im, const double *Thw_im) {
    S->Ra_im = Ra_im;
    if (derive(S) != ORC_OK) return ORC_EINVAL;
    if (Thw_im)
        for (long col = 0; col < S->ncols; ++col) S->Thw[col] = RE(S->Thw[col]) + I * Thw_im[col];
    refresh_ghosts(S);
    return ORC_OK;
}

/* Real and imaginary parts of the front heights and of the liquid fraction. */
void orc_cs_get_s(const orc_sim *S, double *re, double *im, double *lf_re, double *lf_im) {
    real acc = 0.0;
    for (long col = 0; col < S->ncols; ++col) {
        if (re) re[col] = creal(S->s[col]);
        if (im) im[col] = cimag(S->s[col]);
        acc += S->s[col];
    }
    acc /= ((double)S->H * (double)S->ncols);
    if (lf_re) *lf_re = creal(acc);
    if (lf_im) *lf_im = cimag(acc);
}
#endif
