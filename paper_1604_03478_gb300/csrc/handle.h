// handle.h -- internal definition of the cavity handle (opaque in the C ABI),
// shared by the single-cavity entry points and the ensemble.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/lbm_melt.h"
#include "lbm_core.cuh"

// Lattice parameters derived from the problem statement (section 1, Eq. 7).
struct Derived {
    int H, P1, P2;
    long long N, ncols;
    double nu, alpha, gbeta, s_nu, s_alpha, lambda, t0, s0;
    double s_e, s_eps, s_q, s_pi, s_m, s_g4, s_g5;
};

struct lbm_melt {
    lbm::KP kp;
    lbm::Links lk;     // interior link offsets of the odd step
    Derived d;
    int face, precision;
    double Ste, Th, Tc, Tm;
    cudaStream_t stream;
    int device;
    void *F, *G;
    int *js[2];
    int *nb[2];
    double *s[2];
    int cur;
    float *gpost;
    float *thw_cur, *thw_prev;
    int thw_pending;   // set_hot_wall happened while values were in flight
    int *status_dev;
    double *sum_dev;
    double *red_part;  // scratch: per-block partials of the FP64 totals
    int nred;          // number of partial blocks
    double *totals_dev;  // 6 doubles
    double *report;    // ring of report rows (7 doubles: t, totals)
    long long report_every, report_cap, report_rows;
    int inflight;      // last stream-collide was an even (local) step
    long long steps;
    size_t bytes;
    int timing;
    int bx, by;        // block shape of the per-node kernels (0: default)
    int cblk;          // threads per block of the per-column kernels
    // Height bound of the stream-collide grid (solid nodes two above every
    // liquid count of their neighbourhood do nothing): k_front keeps a
    // running maximum of the liquid counts on the device, read back
    // asynchronously every few steps; a count grows by at most one a step.
    int *jmax_dev;
    int *jmax_host;    // pinned landing slot of the read-back
    cudaEvent_t jmax_ev;
    int jmax_pending;  // a read-back is in flight
    int jmax_stale;    // jmax_dev may be below the counts (advanced elsewhere)
    long long jmax_pending_at;  // exec_steps when it was enqueued
    int ab_known;      // last maximum read, -1: unknown
    long long ab_at;   // exec_steps at which ab_known held
    long long exec_steps;  // steps this handle executed (never rewound)
    double Ra;         // as given to create
    int derived_from_Ra;
    void *tape;        // recorded run for the adjoint (adjoint.cu)
    std::vector<cudaEvent_t> ev;  // start/stop pairs of timed launches
    size_t ev_used;
    char err[512];
};

// Release a handle's recorded run (defined with the adjoint).
void lbm_tape_free(lbm_melt *h);
// Reads the sticky front status on the handle's stream (synchronises):
// LBM_EUNSTABLE after a step with |ds| > 1/2, LBM_ENAN after a non-finite
// front temperature, else LBM_OK.
lbm_status lbm_check_status(lbm_melt *h);
// Forget the host's view of the liquid-count maximum: after the state was
// advanced by other code (the ensemble) or replaced.
void lbm_jmax_invalidate(lbm_melt *h);
