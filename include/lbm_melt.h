/*
 * lbm_melt.h -- C ABI of the GB300 (sm_103a) double-MRT lattice Boltzmann
 * library for 3-D melting with interfacial tracking.
 *
 * Method: Li, Yang & Zhang, "Lattice Boltzmann method simulation of 3-D
 * melting using double MRT model with interfacial tracking method",
 * arXiv:1604.03478 -- section 1 (problem statement: a cubic cavity of edge H
 * heated to Th on one wall, the opposite wall at Tc <= Tm, the others
 * adiabatic, no-slip everywhere), section 2 (Eqs. 1-3: D3Q19 MRT flow with a
 * body force; Eqs. 4-5: D3Q7 MRT energy; Eq. 6: the front velocity from the
 * interface energy balance) and Eq. 7 (Fourier number).
 *
 * Conventions
 *   - Every call returns an lbm_status; nothing throws across the ABI.  On an
 *     error, lbm_melt_last_error() gives a message.
 *   - Node (x, y, z), 0 <= x < nx etc., has its centre at (x+1/2, y+1/2,
 *     z+1/2); the walls are at 0 and n on each axis.  Per-node arrays are
 *     row-major (z, y, x) with x fastest: index (z*ny + y)*nx + x.
 *   - The heating axis a is y (heated_face 0: heated wall y = 0) or z
 *     (heated_face 1: heated wall z = 0); gravity is always -z.  The front is
 *     a height field s over the two other axes ("columns"): column index
 *     z*nx + x for heated_face 0, y*nx + x for heated_face 1.  Node j of a
 *     column is liquid iff j + 1/2 < s.
 *   - ptr_kind 0: host pointers; 1: device pointers (on the handle's device).
 *     Outputs are caller-owned.  The handle owns all of its device memory.
 *   - lbm_melt_step is asynchronous on the handle's stream; a front that
 *     moved more than half a cell in a step (LBM_EUNSTABLE) or a non-finite
 *     temperature (LBM_ENAN) is reported by the next call that synchronises
 *     (lbm_melt_get, lbm_melt_get_state, lbm_melt_sync).
 */
#ifndef LBM_MELT_H
#define LBM_MELT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_melt lbm_melt; /* opaque handle */

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,    /* an argument is out of range */
    LBM_ENOMEM = -2,    /* device or host allocation failed */
    LBM_ECUDA = -3,     /* a CUDA call failed (message in last_error) */
    LBM_EUNSTABLE = -4, /* the front moved more than half a cell in one step */
    LBM_ETIMEOUT = -5,  /* a bounded device-side wait gave up */
    LBM_ENAN = -6       /* a non-finite temperature reached the front */
} lbm_status;

/* Cavity and storage.  heated_face: 0 = wall y = 0 (side-heated), 1 = wall
   z = 0 (bottom-heated).  precision: 0 = FP32 storage, 1 = FP16 storage of
   the shifted distributions f - w rho0 and g - w Tm (FP32 arithmetic in both;
   the front and the reductions in FP64).  Ma: Mach number U0 / c_s (Eq. 7;
   any value below 0.3).  s0: initial front height above the heated wall in
   lattice units (0 selects 1.0); the liquid below it starts at the analytic
   conduction-melting temperature of that front, at rest. */
typedef struct {
    int nx, ny, nz;
    int heated_face;
    int precision;
    double Ma;
    double s0;
} lbm_melt_grid;

/* Relaxation rates (Eqs. 2 and 4).  D3Q19 (moment basis of d'Humieres et al.
   2002): s_nu on the five viscous-stress moments, s_e energy, s_eps energy
   square, s_q heat flux, s_pi the two 4th-order stress moments, s_m the three
   3rd-order moments.  D3Q7: s_alpha on the three flux moments (alpha =
   (1/s_alpha - 1/2)/4), s_g4 and s_g5 on the higher ones.  derive_from_Ra = 1:
   s_nu and s_alpha follow from Ra, Pr, Ma and the cavity length H along the
   heating axis (nu = Ma/sqrt(3) H sqrt(Pr/Ra), alpha = nu/Pr); 0: as given.
   In both cases g*beta = Ra nu alpha / ((Th - Tm) H^3), zero for Ra = 0.
   A rate <= 0 among s_e .. s_m, s_g4, s_g5 selects its default (1.19, 1.4,
   1.2, 1.4, 1.98, 1, 1). */
typedef struct {
    double s_nu, s_e, s_eps, s_q, s_pi, s_m;
    double s_alpha, s_g4, s_g5;
    int derive_from_Ra;
} lbm_melt_rates;

/* Derived lattice quantities of a handle (or of a would-be handle, see
   lbm_melt_derive). */
typedef struct {
    double nu, alpha, gbeta;     /* lattice viscosity, diffusivity, g*beta */
    double tau_nu;               /* 3 nu + 1/2 */
    double s_nu, s_alpha;        /* rates in effect */
    double lambda;               /* Neumann root: lambda e^(lambda^2) erf(lambda) = Ste/sqrt(pi) */
    double t0;                   /* lattice time of the initial front, s0^2 / (4 lambda^2 alpha) */
    double H;                    /* cavity length along the heating axis */
    long long n_cells, n_columns;
    long long steps;             /* steps taken */
    size_t device_bytes;         /* device memory held by the handle */
} lbm_melt_info;

/* Validate the arguments and fill *info with the derived lattice parameters,
   without touching the GPU.  Rejects: a cavity edge < 1 or a heating-axis
   length < 4, heated_face or precision out of range, Th <= Tm, Tc > Tm,
   Ste < 0 (Ste = 0 holds the front in place), Ra < 0, Ra = 0 with
   derive_from_Ra, Ma outside (0, 0.3] when deriving,
   tau_nu <= 0.5 + 1e-4, any rate outside (0, 2), s0 outside [0.5, H]. */
lbm_status lbm_melt_derive(const lbm_melt_grid *grid, double Ra, double Pr, double Ste,
                           double Th, double Tc, double Tm, const lbm_melt_rates *rates,
                           lbm_melt_info *info);

/* The message explaining why lbm_melt_derive rejects these arguments ("" if
   it accepts them).  Returns a static buffer (not thread-safe). */
const char *lbm_melt_derive_error(const lbm_melt_grid *grid, double Ra, double Pr, double Ste,
                                  double Th, double Tc, double Tm, const lbm_melt_rates *rates);

/* Create a cavity on the current CUDA device, in its initial state.
   cuda_stream: the cudaStream_t the handle launches on (NULL: the legacy
   default stream).  On success *out receives the handle; on failure *out is
   NULL and the status says why (the message is lost with the handle: use
   lbm_melt_derive to see validation messages). */
lbm_status lbm_melt_create(const lbm_melt_grid *grid, double Ra, double Pr, double Ste,
                           double Th, double Tc, double Tm, const lbm_melt_rates *rates,
                           void *cuda_stream, lbm_melt **out);

/* Advance n >= 0 time steps (Eqs. 1-6 per step: stream-collide, front
   update, phase flip).  Asynchronous, with one exception: with Tc == Tm the
   stream-collide grid stops above the liquid (deep solid nodes have no
   work), at a height taken from a copy of the running maximum liquid count
   that the device posts every 4 steps; before a step the host uses the newest
   copy already complete, else waits for one 16 steps old.  So the host blocks
   only while it is more than ~16 steps ahead of the device (no effect on the
   results). */
lbm_status lbm_melt_step(lbm_melt *h, long long n);

/* Macroscopic outputs, any of them NULL to skip: T per node (solid nodes
   report Tm), u per node as 3 interleaved floats (force-shifted velocity,
   zero in solid nodes), S per column (the front height above the heated
   wall), liquid_fraction = sum(S) / (H * columns).  Synchronises. */
lbm_status lbm_melt_get(lbm_melt *h, float *T, float *u, double *S, double *liquid_fraction,
                        int ptr_kind);

/* The front S and the liquid fraction of the current state (the quantities
   the paper follows in §3, Figs. 2-4), enqueued on the handle's stream
   without waiting (either may be NULL): the values land in
   the caller's buffers when the stream reaches the copies, so they may be
   read only after lbm_melt_sync (or another synchronising call).  A loop of
   step + get_async keeps the device busy while earlier results travel; for
   the copies to overlap, host buffers must be page-locked (pageable ones make
   the copy wait), and a buffer must not be reused before the copy into it is
   complete.  Status flags (LBM_EUNSTABLE, LBM_ENAN) surface at the sync. */
lbm_status lbm_melt_get_async(lbm_melt *h, double *S, double *liquid_fraction, int ptr_kind);

/* Same outputs as lbm_melt_get, without allocating anything.  The paper has
   no counterpart: this serves callers that cannot let a library allocate
   device memory (a time-critical loop in which a cudaMalloc would synchronise
   the device, or an application whose own pool allocator owns all device
   memory).  Host-bound results are staged through a fixed array that the
   library holds on every GPU that loads it until the process exits, sized
   for at most 2097152 nodes (128^3, 32 MiB); a larger cavity is rejected
   with LBM_EINVAL.  The liquid fraction is reduced in the handle's own
   buffers (allocated at create), so every output equals lbm_melt_get's bit
   for bit.  The handle's device must be current.  The first call on a
   device performs a one-time set-up (it looks up the array's device
   address); make that first call before any stream capture.  A device reset
   (cudaDeviceReset) invalidates that set-up, as it invalidates every handle
   made before it: do not call this entry point in a process after a reset.
   Every call shares the array: calls whose work overlaps on the GPU race.
   Calls no cudaMalloc, cudaFree or allocating library routine.
   Synchronises. */
lbm_status lbm_melt_get_noalloc(lbm_melt *h, float *T, float *u, double *S, double *liquid_fraction,
                                int ptr_kind);

/* Distributions in natural form (post-streaming, pre-collision; f_i and g_i,
   not shifted), direction-major: f[i*N + node], g[i*N + node]; solid nodes
   report f = 0, and solid nodes whose neighbourhood is all solid report g at
   rest at Tm.  Any pointer may be NULL.  Synchronises. */
lbm_status lbm_melt_get_state(lbm_melt *h, float *f, float *g, double *S, int ptr_kind);

/* Replace the state with natural-form distributions and front heights (same
   layout as lbm_melt_get_state).  Solid nodes are stored at rest (f and g of
   solid nodes are ignored: a solid node's own populations never enter the
   method, its post-collision values being reset every step).  f or g may be
   NULL to keep that part; a new S needs both f and g.  The phase flags and
   the ghost nodes are recomputed from the new state. */
lbm_status lbm_melt_set_state(lbm_melt *h, const float *f, const float *g, const double *S,
                              int ptr_kind);

/* Heated-wall temperature per column (overrides the scalar Th on the wall;
   the scalar Th still defines the Stefan number).  Takes effect for the
   next step's streaming. */
lbm_status lbm_melt_set_hot_wall(lbm_melt *h, const float *T_h_field, int ptr_kind);

/* FP64 totals of the current state (paper §3.1 and Fig. 4(d): the liquid
   fraction; energy and mass balances; §3.2, Fig. 4(b): the heat-surface
   Nusselt number): out[0] liquid fraction, out[1] sum over liquid nodes of
   (T - Tm), out[2] sum over liquid nodes of (rho - 1), out[3] number of
   liquid nodes, out[4] max |u| over liquid nodes, out[5] sum of S over
   columns, out[6] mean Nusselt number over the heated wall (as
   lbm_melt_get_nusselt).  The heat content relative to solid at Tm is
   out[1] + (Th - Tm) / Ste * out[5].  Deterministic (fixed reduction order).
   Synchronises. */
lbm_status lbm_melt_totals(lbm_melt *h, double *out, int ptr_kind);

/* Heat-surface Nusselt number (paper §3.2, Fig. 4(b) and the Case 1 / Case
   2 comparison of Fig. 5): Nu = -H (dT/da at the heated wall) / (Th - Tm)
   per column, from the heat that the last step's streaming carried through
   the heated-wall link of the column's first node (incoming minus outgoing
   population on that anti-bounce-back link, which equals -alpha dT/da),
   with the wall field of that streaming and the scalar Th.  Nu: ncols
   doubles in the column order of S (NULL: not wanted); Nu_mean: one double,
   the mean over the wall by a fixed-order FP64 sum (NULL: not wanted).
   Meaningful after at least one step (after create or set_state it is
   computed from the uploaded populations).  Synchronises. */
lbm_status lbm_melt_get_nusselt(lbm_melt *h, double *Nu, double *Nu_mean, int ptr_kind);

/* Record the totals every `every` steps (0 turns recording off) into a ring
   of `capacity` rows of 8 doubles {steps, out[0..6] of lbm_melt_totals},
   filled on the device inside lbm_melt_step.  Clears earlier rows. */
lbm_status lbm_melt_set_report(lbm_melt *h, long long every, long long capacity);

/* Copy up to max_rows recorded rows (oldest kept first) to host memory;
   *n_rows receives how many.  rows = NULL asks how many rows are kept.
   Synchronises. */
lbm_status lbm_melt_get_report(lbm_melt *h, double *rows, long long max_rows, long long *n_rows);

/* Derived quantities and counters of a handle. */
lbm_status lbm_melt_get_info(lbm_melt *h, lbm_melt_info *info);

/* Wait for the handle's stream; report a device-side error flag. */
lbm_status lbm_melt_sync(lbm_melt *h);

/* Block shape (bx threads along x, a multiple of 32; by along y; bx*by <=
   128) of the stream-collide kernels; (0, 0) restores the default.  The
   autotuner in the Python package picks it per cavity size and precision. */
lbm_status lbm_melt_set_launch(lbm_melt *h, int bx, int by);

/* Kernel timing: when enabled, each stream-collide launch is bracketed by
   CUDA events; lbm_melt_kernel_time returns (after synchronising) the summed
   milliseconds and the number of timed launches since the last reset. */
lbm_status lbm_melt_set_timing(lbm_melt *h, int enable);
lbm_status lbm_melt_kernel_time(lbm_melt *h, double *ms, long long *launches, int reset);

/* Replay lbm_melt_step's steps from CUDA graphs of `steps` steps each (0:
   launch every step on its own).  A step is three kernels; on a small
   cavity the host's launches take longer than the GPU's work, so by default
   cavities of at most 160^3 nodes replay 16 steps per graph and larger ones
   launch step by step.  A graph is captured once per starting phase of the
   in-place streaming (and again when the front outgrows the grid it was
   captured for) and replayed on the handle's stream; results are
   bit-identical to step-by-step launches.  Steps that carry a report row,
   follow a heated-wall change still pending, or are timed
   (lbm_melt_set_timing) run step by step.  steps in [0, 256]. */
lbm_status lbm_melt_set_graph_steps(lbm_melt *h, int steps);

/* Nodes per thread of the stream-collide (the same method and results up to
   FP32 rounding): -1 (default) chooses two for cavities above 160^3 nodes
   with an even nx and one otherwise; 0 one node per thread; 1 two nodes per
   thread (x-adjacent nodes as the two lanes of packed FP32x2 arithmetic,
   their populations moved as float2/half2 words where aligned; needs an
   even nx, else LBM_EINVAL).  Two nodes
   per thread pay about half the instructions per node and win where the
   grid is large; small grids with a thin liquid layer are latency bound
   and run faster with one. */
lbm_status lbm_melt_set_node_pairs(lbm_melt *h, int mode);

/* Heat conduction in the solid: the k_s dT_s/da term of Eq. 6, for a cold
   wall below the melting point (Tc < Tm, a subcooled solid; the paper
   solves only zero subcooling, where the solid stays at Tm and the term
   vanishes -- the default).  ks_kl = k_s / k_l > 0 turns it on, 0 turns it
   off.  With it on:
   - the solid (equal rho c in both phases, so alpha_s = ks_kl alpha) runs
     the D3Q7 collision of Eq. 4 at u = 0 with that diffusivity, and its
     populations stream among solid nodes and against the walls like the
     liquid's (Tc at the cold wall);
   - the front is a T = Tm surface on both sides: the solid side's ghost is
     the last liquid node of a column, at the temperature extrapolated
     through (s, Tm) and the lowest solid node at least half a cell above s
     (the cold wall standing in), plus the non-equilibrium part of the solid
     node above it; a population crossing the phase boundary from a node
     that is not its column's ghost for the receiving phase is the rest
     state at Tm;
   - Eq. 6 reads ds/dt = alpha Ste / (Th - Tm) (1 + s_x^2 + s_z^2)
     (ks_kl dT_s/da - dT_l/da), with dT_s/da the one-sided quadratic through
     (s, Tm) and the two lowest solid nodes at least half a cell above s (the
     cold wall standing in for a missing one);
   - lbm_melt_get reports the solid's own temperature; lbm_melt_set_state
     keeps the g given for solid nodes; every node is updated every step
     (no deep-solid skip).
   Only before the first step: the call re-initialises the state, the
   liquid below s0 and the solid above it at the two-phase Neumann solution
   of conduction melting against a solid initially at Tc (lambda and t0 of
   lbm_melt_get_info follow it), and resets the heated-wall field to the
   scalar Th.  Rejected (LBM_EINVAL) for an ensemble member; the adjoint
   (lbm_melt_tape_forward) rejects a handle with conduction on.
   Synchronises. */
lbm_status lbm_melt_set_solid_conduction(lbm_melt *h, double ks_kl);

const char *lbm_melt_last_error(const lbm_melt *h);
void lbm_melt_destroy(lbm_melt *h);

/* ----------------------------------------------------------------- adjoint
   Gradients of a function of the final front S with respect to the
   heated-wall temperature field and Ra, by a hand-written adjoint of the
   step (Eqs. 1-6) with the phase flags held at their recorded values.

   lbm_melt_tape_forward advances the handle by `steps` steps (as
   lbm_melt_step) and keeps a checkpoint of the state every ckpt_every steps
   (<= 0: ceil(sqrt(steps)) rounded up to a multiple of the step-graph length
   when steps are replayed from graphs).  The heated-wall field must be set before (no
   change pending) and stays fixed during the recorded run.

   lbm_melt_tape_backward takes seed_dL_dS = dL/dS of the final front (one
   value per column) and returns dL_dTh = dL/d(heated-wall temperature) per
   column and dL_dparams[5] = {dL/dRa, dL/ds_nu, dL/ds_alpha, dL/dcoef,
   dL/d(g beta)} (coef = alpha Ste / (Th - Tm), the Eq. 6 factor; dL/dRa
   chains these through the parameter map of lbm_melt_derive).  Segments are
   recomputed from their checkpoints with one snapshot per step, then
   reversed; the handle is back in its final state afterwards.  Synchronises.
   Returns LBM_EUNSTABLE (or LBM_ENAN) without computing anything when the
   front status of the handle is flagged: the reverse sweep relies on fronts
   that moved at most half a node per step; and LBM_EINVAL when the
   heated-wall field was set after the recorded run (the sweep recomputes
   the run with it).  The recomputation of a segment and the reverse sweep
   of the segment after it run concurrently on the handle's stream and an
   internal one (two snapshot sets when the device has room for them; full
   segments replayed from CUDA graphs). */
lbm_status lbm_melt_tape_forward(lbm_melt *h, long long steps, long long ckpt_every);
lbm_status lbm_melt_tape_backward(lbm_melt *h, const double *seed_dL_dS, double *dL_dTh, double *dL_dparams,
                                  int ptr_kind);
/* Release the recorded run and the adjoint's device buffers.  The
   checkpoints of a recorded run and the work buffers of the backward are
   kept with the handle from one gradient to the next (a loop of gradients
   of one run length allocates once); this call, or lbm_melt_destroy, gives
   them back. */
lbm_status lbm_melt_tape_clear(lbm_melt *h);

/* ------------------------------------------------------------------ ensemble
   A batch of independent cavities of uneven sizes and parameters advanced in
   lockstep by one persistent kernel launch per run of steps: each step covers
   the nodes of all cavities (fused stream-collide), then all their columns
   (front update, Eq. 6), then the phase flips, separated by grid-wide
   barriers whose waits are bounded (an exhausted wait ends the launch;
   lbm_ensemble_sync then returns LBM_ETIMEOUT).  The launch is captured once
   in a CUDA graph (graph_steps steps per replay) and replayed. */
typedef struct lbm_ensemble lbm_ensemble;

/* One member cavity: the arguments of lbm_melt_create. */
typedef struct {
    lbm_melt_grid grid;
    double Ra, Pr, Ste, Th, Tc, Tm;
    lbm_melt_rates rates;
} lbm_melt_case;

/* Create n cavities (all with the same storage precision, n <= 64, each
   with fewer than 2^32 / 19 stored elements per direction array, about
   2.2e8 nodes) on the current device; LBM_EINVAL otherwise.  The ensemble
   runs on a stream of its own, ordered after the work queued on cuda_stream
   at each call and before the work queued there afterwards. */
lbm_status lbm_ensemble_create(int n, const lbm_melt_case *cases, void *cuda_stream, lbm_ensemble **out);

/* Advance every member by nsteps steps.  Asynchronous. */
lbm_status lbm_ensemble_step(lbm_ensemble *e, long long nsteps);

/* Launch shape: threads per block (64, 128 or 256; a block covers an x-y
   tile of one cavity), nodes per thread in the stream-collide phase (1, 2,
   4 or 8 consecutive z-planes) and steps per graph replay (even, >= 2).  The grid
   is the co-resident maximum for that shape. */
lbm_status lbm_ensemble_set_launch(lbm_ensemble *e, int block, int nodes_per_thread, int graph_steps);

/* Bound of a barrier wait, in polls (default 2^24, about a second). */
lbm_status lbm_ensemble_set_barrier_timeout(lbm_ensemble *e, long long max_spins);

/* Test hook for failure detection: one step in which block `block` never
   arrives at the first barrier, so that the bounded waits of the others run
   out and the launch returns; lbm_ensemble_sync then reports LBM_ETIMEOUT.
   The members' states are not meaningful afterwards. */
lbm_status lbm_ensemble_inject_barrier_fault(lbm_ensemble *e, int block);

/* Phase timers of the persistent kernel: block 0 reads the GPU's global
   timer each time it leaves a grid barrier, so a step splits into the fused
   stream-collide of every cavity (phase 1), the front update of every column
   (Eq. 6, phase 2) and the phase flip (phase 3), each with the barrier that
   ends it.  us_per_step (3 doubles, may be NULL): the mean microseconds per
   step of each phase since the ensemble was created or last reset; steps
   (may be NULL): the steps timed.  reset != 0 zeroes the timers after the
   read.  Synchronizes the ensemble's stream (call it between steps, not
   while a capture is open).  LBM_EINVAL for a NULL ensemble, LBM_ECUDA if
   the read fails. */
lbm_status lbm_ensemble_phase_times(lbm_ensemble *e, int reset, double *us_per_step, long long *steps);

/* Wait for the ensemble; report a barrier timeout or a member's error. */
lbm_status lbm_ensemble_sync(lbm_ensemble *e);

/* Member i as a cavity handle (for lbm_melt_get, _totals, _set_hot_wall ...;
   owned by the ensemble, not to be destroyed by the caller).  NULL if out of
   range. */
lbm_melt *lbm_ensemble_member(lbm_ensemble *e, int i);

/* Total nodes and the launch shape in use. */
lbm_status lbm_ensemble_info(lbm_ensemble *e, long long *n_nodes, int *grid, int *block, int *nodes_per_thread);

const char *lbm_ensemble_last_error(const lbm_ensemble *e);
void lbm_ensemble_destroy(lbm_ensemble *e);

/* Library version string. */
const char *lbm_melt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_MELT_H */
