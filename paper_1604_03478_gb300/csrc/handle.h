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
    long long thw_gen; // number of set_hot_wall calls (a recorded run keeps the field of its record)
    int thw_last_prev; // set_hot_wall since the last step in the natural layout: thw_prev holds the
                       // field of the last streaming (the Nusselt number's wall value)
    double *nu_dev;    // per-column Nusselt numbers (ncols)
    int *status_dev;
    double *sum_dev;
    unsigned int *ticket;  // last-block ticket of the one-launch column sum (k_sum_once)
    double *red_part;  // scratch: per-block partials of the FP64 totals
    int nred;          // number of partial blocks
    double *totals_dev;  // 7 doubles
    double *report;    // ring of report rows (8 doubles: t, totals)
    long long report_every, report_cap, report_rows;
    int inflight;      // last stream-collide was an even (local) step
    long long steps;
    size_t bytes;
    int timing;
    int bx, by;        // block shape of the per-node kernels (0: default)
    int cblk;          // threads per block of the per-column kernels
    int sms;           // SMs of the device
    // Running maximum of the liquid counts, kept by k_front on the device;
    // stream-collide blocks at heights >= it + 3 (all deep solid) return at
    // once.  It is also copied every kRbEvery steps into a ring of pinned
    // slots; before a stream-collide the host takes the newest copy at least
    // kRbLag steps old (waiting for it only when it runs that far ahead of
    // the device) and launches no block above it + its age + 2 (a count
    // grows by at most one node per step).
    static const int kRbRing = 32, kRbLag = 16, kRbEvery = 4;
    int *jmax_dev;
    int *rb_val;       // pinned ring of read-backs
    cudaEvent_t rb_ev[kRbRing];
    long long rb_step[kRbRing];  // exec step after which each copy was taken
    long long rb_next;           // read-backs enqueued so far
    long long rb_valid_from;     // read-backs before this one are not bounds any more
    long long rb_synced;         // newest read-back known complete (its value read)
    long long exec_steps;        // steps this handle executed (never rewound)
    double Ra;         // as given to create
    int derived_from_Ra;
    // Heat conduction in the solid (lbm_melt_set_solid_conduction): the
    // conductivity ratio k_s / k_l (0: off, the solid held at Tm) and the
    // solid side's ghost populations of each column (7 x ncols).
    double ks_kl;
    float *spost;
    int member;        // owned by an ensemble (whose kernel holds the solid at Tm)
    void *tape;        // recorded run for the adjoint (adjoint.cu)
    void *adj_ws;      // the adjoint's device buffers, kept between gradients (adjoint.cu)
    // Steps replayed from CUDA graphs (lbm_melt_step): graph_steps steps per
    // replay (0: every step launched on its own).  One instantiated graph per
    // starting (cur, inflight) phase; each records the stream-collide grid
    // height and block shape it was captured with.
    int graph_steps;
    // Nodes per thread of the stream-collide: -1 chooses (two for cavities
    // above 160^3 with an even nx, one otherwise), 0 one, 1 two (even nx).
    int pairs_mode;
    cudaStream_t cap_stream;     // private stream the graphs are captured on
    struct StepGraph {
        cudaGraphExec_t exec;
        int height, bx, by;
    } graphs[2][2];              // [cur][inflight]
    std::vector<cudaEvent_t> ev;  // start/stop pairs of timed launches
    size_t ev_used;
    char err[512];
};

// Release a handle's recorded run and the adjoint's buffers (defined with
// the adjoint).
void lbm_tape_free(lbm_melt *h);
// Enqueue one step (stream-collide, front, flip) from phase (cur, inflight)
// on stream st, the stream-collide grid cut at `height`; advances cur and
// inflight.  No host bookkeeping (step counters, read-backs, report rows).
cudaError_t lbm_enqueue_step(lbm_melt *h, int &cur, int &inflight, int height, cudaStream_t st);
// Reads the sticky front status on the handle's stream (synchronises):
// LBM_EUNSTABLE after a step with |ds| > 1/2, LBM_ENAN after a non-finite
// front temperature, else LBM_OK.
lbm_status lbm_check_status(lbm_melt *h);

