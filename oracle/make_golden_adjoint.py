"""Write the expected gradients of the 96^3 adjoint workload to
``tests/golden/adjoint_96cube_4000steps.txt``, from the FP64 oracle alone.

TEST INFRASTRUCTURE: this script calls only ``oracle/`` (and the seeded
random draws of ``paper_1604_03478_gb300/inputs.py``, loaded by path without
the package, which holds none of the method's arithmetic).

Workload: the 96^3 cube heated at y = 0, Ra 1e5, Pr 0.02, Ste 0.1, Ma 0.1,
front from s0 = 1, 4000 steps, heated wall at 1 + N(0, 0.01^2) per column
(seed 5).  Stored values, all derivatives of that run's final state:

* d lf / dRa and d lf / dv for two seeded wall directions v (N(0, 1) per
  column, seeds 7 and 8), lf = final liquid fraction (Eq. 6 front heights
  summed, over H times the number of columns), by complex step (the oracle's
  tangent-linear build, flags of the unperturbed run);
* central differences of lf along the seed-7 direction with the real oracle,
  eps = 1e-9, and the number of columns whose final liquid count differs
  between the two perturbed runs (0: no node changed phase at the end);
* the L2 front mismatch L = sum (S - S*)^2 to the final front S* of a run
  whose wall is 1 + N(0, 0.01^2) with seed 11 (a reachable target), and its
  derivatives along dRa and the seed-7 direction, 2 (S - S*) . dS.

Command (about an hour on 8 host cores; with --cache DIR each run's result
is kept in DIR and a rerun resumes from there):
    python oracle/make_golden_adjoint.py [--cache DIR]
"""
from __future__ import annotations

import importlib.util
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "adjoint_96cube_4000steps.txt")
N, STEPS, EPS = 96, 4000, 1e-9
CASE = dict(face=0, Ra=1e5, Pr=0.02, Ste=0.1, Ma=0.1, s0=1.0, derive=True)
SEEDS = dict(wall=5, v1=7, v2=8, target=11)


def _inputs():
    spec = importlib.util.spec_from_file_location(
        "_seeded_inputs", os.path.join(ROOT, "paper_1604_03478_gb300", "inputs.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _real_run(wall):
    o = oracle.Oracle(N, N, N, **CASE)
    o.set_hot_wall(wall)
    o.step(STEPS)
    _, _, S, lf = o.get()
    o.close()
    return S.ravel(), lf


def _cached(cache, name, fn):
    """fn() -> tuple of arrays/floats, stored under cache/name.npz."""
    if cache:
        path = os.path.join(cache, name + ".npz")
        if os.path.exists(path):
            d = np.load(path)
            return tuple(d["v%d" % i] for i in range(len(d.files)))
    out = tuple(np.asarray(v) for v in fn())
    if cache:
        os.makedirs(cache, exist_ok=True)
        np.savez(os.path.join(cache, name + ".npz"), **{"v%d" % i: v for i, v in enumerate(out)})
    return out


def main():
    cache = sys.argv[sys.argv.index("--cache") + 1] if "--cache" in sys.argv else None
    inp = _inputs()
    oracle.build()
    ncols = N * N
    wall = 1.0 + inp.gaussian_field(ncols, 0.01, SEEDS["wall"])
    v1 = inp.gaussian_field(ncols, 1.0, SEEDS["v1"])
    v2 = inp.gaussian_field(ncols, 1.0, SEEDS["v2"])
    target_wall = 1.0 + inp.gaussian_field(ncols, 0.01, SEEDS["target"])
    t0 = time.time()

    def log(msg):
        print("[%6.0f s] %s" % (time.time() - t0, msg), flush=True)

    S, dS_ra, lf, dlf_ra = _cached(cache, "tl_ra", lambda: oracle.tangent(N, N, N, STEPS, dRa=1.0, wall=wall, **CASE))
    S, dS_ra, lf, dlf_ra = S.ravel(), dS_ra.ravel(), float(lf), float(dlf_ra)
    log("tangent along Ra: lf %.12g, dlf %.12g" % (lf, dlf_ra))
    _, dS_v1, _, dlf_v1 = _cached(cache, "tl_v1", lambda: oracle.tangent(N, N, N, STEPS, dThw=v1, wall=wall, **CASE))
    dS_v1, dlf_v1 = dS_v1.ravel(), float(dlf_v1)
    log("tangent along v1: dlf %.12g" % dlf_v1)
    _, _, _, dlf_v2 = _cached(cache, "tl_v2", lambda: oracle.tangent(N, N, N, STEPS, dThw=v2, wall=wall, **CASE))
    dlf_v2 = float(dlf_v2)
    log("tangent along v2: dlf %.12g" % dlf_v2)
    Sp, lfp = _cached(cache, "fd_plus", lambda: _real_run(wall + EPS * v1))
    Sm, lfm = _cached(cache, "fd_minus", lambda: _real_run(wall - EPS * v1))
    lfp, lfm = float(lfp), float(lfm)
    fd = (lfp - lfm) / (2.0 * EPS)
    js = lambda s: np.clip(np.ceil(s - 0.5), 0, N).astype(np.int64)  # noqa: E731
    flips = int(np.count_nonzero(js(Sp) != js(Sm))) + int(np.count_nonzero(js(Sp) != js(S)))
    log("central differences along v1: %.12g (columns with another final count: %d)" % (fd, flips))
    St, _ = _cached(cache, "target", lambda: _real_run(target_wall))
    r = S - St
    L2 = float(r @ r)
    dL2_ra = float(2.0 * r @ dS_ra)
    dL2_v1 = float(2.0 * r @ dS_v1)
    log("mismatch %.12g, along Ra %.12g, along v1 %.12g" % (L2, dL2_ra, dL2_v1))
    rows = [("liquid_fraction", lf), ("dlf_dRa", dlf_ra), ("dlf_dv1", dlf_v1), ("dlf_dv2", dlf_v2),
            ("fd_dlf_dv1", fd), ("fd_count_changes", flips), ("fd_eps", EPS),
            ("mismatch_L2", L2), ("dL2_dRa", dL2_ra), ("dL2_dv1", dL2_v1)]
    with open(OUT, "w") as f:
        f.write("# Gradients of the 96^3 adjoint workload (heated at y = 0, Ra 1e5, Pr 0.02, Ste 0.1, Ma 0.1,\n"
                "# s0 = 1, %d steps, heated wall 1 + N(0, 0.01^2) per column, seed %d) from the FP64 oracle:\n"
                "# complex-step tangent-linear derivatives of the final liquid fraction (Eq. 6 fronts) along\n"
                "# dRa = 1 and the wall directions v1, v2 = N(0, 1) per column (seeds %d, %d); central\n"
                "# differences along v1; the L2 mismatch to the final front of a run with wall seed %d.\n"
                "# Written by: python oracle/make_golden_adjoint.py\n"
                % (STEPS, SEEDS["wall"], SEEDS["v1"], SEEDS["v2"], SEEDS["target"]))
        for k, v in rows:
            f.write("%s %.17g\n" % (k, v))
    log("wrote %s" % OUT)


if __name__ == "__main__":
    main()
