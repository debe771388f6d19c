"""Benchmark of the double-MRT melting step on GB300.

Workload (the precision-study configuration, side-heated variant): a 256^3
cavity heated at y = 0, Ra = 1e6, Pr = 0.02, Ste = 0.05, Ma = 0.1, FP32
storage, the front started flat at s0 = 0.4 H so that the liquid fraction is
mid-cavity while timing.  One step = the whole hot path: the fused
stream-collide (D3Q19 + D3Q7 MRT, AA pattern), the FP64 front update (Eq. 6)
and the phase flip.

Prints ONE JSON line.  ``value`` is liquid-node updates per second (MLUPS,
the fluid-node convention) with the state resident in HBM; ``e2e`` is the
same metric through the C ABI with host buffers, every step uploading the
heated-wall field from pinned host memory and reading the front and the
liquid fraction back.  ``--impl reference`` times the CPU FP64 oracle on the
same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "double-MRT melting MLUPS & % HBM roofline at 256³; adjoint/forward time ratio"
N_EDGE = 256
CASE = dict(face=0, Ra=1e6, Pr=0.02, Ste=0.05, Ma=0.1, s0=0.4 * N_EDGE, derive=True)
WORKLOAD = ("256^3 cavity heated at y=0, Ra 1e6, Pr 0.02, Ste 0.05, Ma 0.1, FP32 storage, "
            "front started flat at s0 = 0.4 H")
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--edge", type=int, default=N_EDGE,
                    help="cavity edge (256 is the benchmark workload; smaller edges for profiling captures)")
    ap.add_argument("--precision", type=int, default=0, help="0: FP32 storage, 1: shifted FP16 storage")
    ap.add_argument("--skip-extra", action="store_true",
                    help="skip the FP16, ensemble and adjoint legs (profiling runs)")
    ap.add_argument("--leg", choices=["precision", "ensemble", "adjoint", "convection", "table1", "solid"],
                    help="run one of the extra legs alone and print its JSON (profiling runs)")
    ap.add_argument("--leg-steps", type=int, default=0, help="steps of that leg (0: its default)")
    ap.add_argument("--dump-dir", default=None, help="directory for the convection leg's final front map (.npy)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers

def dist_setup(n):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_across_ranks(ms, units, dist=None, device="cpu"):
    """Max of the timed region and sum of the work over ranks (one process
    per GPU, each advancing its own replica: no data-path collective)."""
    if dist is None:
        return ms, units
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# Sources of the stream-collide kernels and their launchers: a recorded DRAM
# traffic figure holds only while they are unchanged.
K1_SOURCES = ("paper_1604_03478_gb300/csrc/kernels.cuh", "paper_1604_03478_gb300/csrc/lbm_core.cuh",
              "paper_1604_03478_gb300/csrc/launch.h", "paper_1604_03478_gb300/csrc/launch_impl.cuh",
              "paper_1604_03478_gb300/csrc/k_f32.cu")
TRAFFIC_RECORD = "profiles/stream_collide_256cube_fp32_traffic.md"


def k1_source_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in K1_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes (read + write) per stream-collide launch of the 256^3 FP32
    workload, from the committed ncu record, or None when the record is
    missing or the kernel sources changed since it was taken."""
    try:
        rec = {}
        with open(os.path.join(ROOT, TRAFFIC_RECORD)) as f:
            for ln in f:
                if ":" in ln and ln.split(":", 1)[0].strip() in ("source_sha256", "bytes_per_launch"):
                    k, v = ln.split(":", 1)
                    rec[k.strip()] = v.strip().strip("`")
        if rec.get("source_sha256") != k1_source_hash():
            return None
        return float(rec["bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for k in ("hbm_gbs", "hbm_GBs", "hbm"):
            if k in d and d[k]:
                v = d[k]
                if isinstance(v, dict):
                    v = v.get("value") or v.get("gbs")
                return float(v), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, TypeError):
        pass
    return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def liquid_counts(S, H):
    """Liquid nodes and the solid nodes the stream-collide still updates
    (solid nodes below the 3x3-neighbourhood maximum first-solid index + 2;
    deeper ones are provably unchanged and skipped)."""
    js = np.clip(np.ceil(S - 0.5), 0, H).astype(np.int64)
    pad = np.pad(js, 1, mode="edge")
    mx = np.max(np.stack([pad[1 + di:1 + di + js.shape[0], 1 + dj:1 + dj + js.shape[1]]
                          for di in (-1, 0, 1) for dj in (-1, 0, 1)]), axis=0)
    n_liq = int(js.sum())
    n_solid_active = int(np.minimum(mx + 2, H).sum() - n_liq)
    return n_liq, max(n_solid_active, 0)


# --------------------------------------------------------------- CPU oracle

def oracle_sample(steps, warm=0, n=N_EDGE, single_steps=0):
    """Time the FP64 oracle on the workload (edge n, same parameters, front
    at 0.4 n) on this host's cores; with single_steps > 0, then time that
    many more steps on one thread.  Returns (MLUPS, seconds, threads) and,
    for the single-thread sample, (MLUPS, seconds) or None."""
    import oracle
    oracle.build()
    case = dict(CASE, s0=0.4 * n)
    o = oracle.Oracle(n, n, n, **case)
    threads = oracle.num_threads()
    if warm:
        o.step(warm)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    n_liq = o.info()["n_liquid"]  # after the steps; the front moves < 1 cell
    single = None
    if single_steps > 0:
        oracle.set_num_threads(1)
        t0 = time.perf_counter()
        o.step(single_steps)
        dt1 = time.perf_counter() - t0
        oracle.set_num_threads(threads)
        single = (n_liq * single_steps / dt1 / 1e6, dt1)
    o.close()
    if single_steps > 0:
        return n_liq * steps / dt / 1e6, dt, threads, single
    return n_liq * steps / dt / 1e6, dt, threads


def run_reference(args):
    rank, world, local = dist_setup(args.gpus)
    if rank != 0:
        return 0
    # each step is one oracle step of a downscaled twin of the workload, its
    # edge chosen so that the whole run stays near 90 s of host time
    import oracle
    oracle.build()
    threads = oracle.num_threads()
    per_step = 90.0 / max(1, args.steps + args.warmup)
    n = int((per_step * threads / 1.5e-6) ** (1.0 / 3.0)) // 16 * 16
    n = max(32, min(N_EDGE, n))
    value, dt, cores = oracle_sample(args.steps, warm=args.warmup, n=n)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "implementation": "CPU FP64 oracle (OpenMP)",
                                           "sample_edge": n},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": "%d oracle steps (after %d warm-up steps) of a %d^3 twin of the workload "
                                   "(same Ra, Pr, Ste, Ma, front at 0.4 H)" % (args.steps, args.warmup, n)},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------ extra legs

def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def precision_leg(steps=200, twin_steps=(400, 1000, 2000)):
    """The precision study: FP32 and FP16 storage at 256^3 with the heated
    wall at the side (y = 0, the benchmark workload) and at the bottom
    (z = 0, Rayleigh-Benard-like), throughput and roofline of each, and the
    error of each storage against the FP64 oracle on a 64^3 twin."""
    import torch
    import oracle
    from paper_1604_03478_gb300 import Cavity
    stream = torch.cuda.current_stream()
    peak, _ = hbm_peak()

    def throughput(face, prec):
        cav = Cavity(N_EDGE, N_EDGE, N_EDGE, precision=prec, stream=stream.cuda_stream, **dict(CASE, face=face))
        cav.step(10)
        cav.sync()
        cav.set_timing(True)
        cav.kernel_time(reset=True)
        e0, e1 = _events()
        e0.record(stream)
        cav.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        k1, nk = cav.kernel_time(reset=True)
        S = cav.get(T=False, u=False)[2]
        n_liq, n_sol = liquid_counts(S, cav.H)
        cav.close()
        per_liq, per_sol = (208.0, 28.0) if prec == 0 else (104.0, 14.0)
        alg = per_liq * n_liq + per_sol * n_sol
        gbs = alg / (k1 / nk * 1e-3) / 1e9
        return n_liq * steps / (ms * 1e-3) / 1e6, {"achieved": gbs, "frac": gbs / peak, "unit": "GB/s",
                                                    "bytes_per_liquid_node": per_liq}

    def twin(face):
        """Errors of both storages against the oracle on a 64^3 twin at
        several horizons, the largest split by region: the liquid nodes next
        to the heated wall (3 layers), those within 3 nodes below the front,
        and the bulk between."""
        n = 64
        case = dict(CASE, face=face, s0=0.4 * n)
        o = oracle.Oracle(n, n, n, **case)
        gpu = {prec: Cavity(n, n, n, precision=prec, stream=stream.cuda_stream, **case) for prec in (0, 1)}
        err = {"fp32_twin_error": {}, "fp16_twin_error": {}}
        done = 0
        for horizon in twin_steps:
            o.step(horizon - done)
            for c in gpu.values():
                c.step(horizon - done)
            done = horizon
            To, uo, So, lfo = o.get()
            H = n
            a = (np.arange(n)[None, :, None] if face == 0 else np.arange(n)[:, None, None]) * np.ones(To.shape)
            s_node = (So[:, None, :] if face == 0 else So[None, :, :]) * np.ones(To.shape)
            liq = a + 0.5 < s_node
            regions = {"wall_layer": liq & (a < 3), "front_layer": liq & (a + 0.5 >= s_node - 3.0),
                       "bulk": liq & (a >= 3) & (a + 0.5 < s_node - 3.0)}
            for prec, name in ((0, "fp32"), (1, "fp16")):
                Tg, ug, Sg, lfg = gpu[prec].get()
                dT = np.abs(Tg - To)
                e = {"max_abs_dT": float(dT.max()), "max_abs_du": float(np.abs(ug - uo).max()),
                     "abs_d_liquid_fraction": abs(lfg - lfo)}
                e["max_abs_dT_by_region"] = {k: float(dT[m].max()) if m.any() else 0.0 for k, m in regions.items()}
                err["%s_twin_error" % name]["%d_steps" % horizon] = e
        o.close()
        for c in gpu.values():
            c.close()
        return err

    out = {}
    out["fp16_mlups"], out["fp16_roofline"] = throughput(0, 1)
    out.update(twin(0))
    bottom = {}
    bottom["fp32_mlups"], bottom["fp32_roofline"] = throughput(1, 0)
    bottom["fp16_mlups"], bottom["fp16_roofline"] = throughput(1, 1)
    bottom.update(twin(1))
    out["bottom_heated"] = bottom
    out["twin"] = ("64^3 twin of each workload (same parameters, front at 0.4 H), %s steps from the same initial "
                   "state, against the FP64 oracle; FP16 stores g shifted by the mid temperature (Th + Tm) / 2"
                   % ", ".join(str(t) for t in twin_steps))
    out["full_horizon"] = full_horizon()
    return out


def full_horizon(steps=50000):
    """The precision workload over its configured 50000 steps at 256^3, for
    both heated faces: FP16 storage against FP32 storage run side by side
    (the oracle's FP64 run of that length would take hours on the host; FP32
    stays within 2e-7 of it on the 64^3 twin over the horizons checked), the
    liquid fraction each reaches, and a control: FP32 against FP32 with the
    one-node kernels (the same arithmetic rounded differently, differences
    of 1e-7 per step), which shows how far the convecting flow itself carries
    rounding differences over that horizon."""
    import torch
    from paper_1604_03478_gb300 import Cavity
    stream = torch.cuda.current_stream()
    res = {"steps": steps}
    for face, name in ((0, "side_heated"), (1, "bottom_heated")):
        cav = {prec: Cavity(N_EDGE, N_EDGE, N_EDGE, precision=prec % 2, stream=stream.cuda_stream,
                            **dict(CASE, face=face)) for prec in (0, 1, 2)}
        cav[2].set_node_pairs(0)
        ms = {}
        for prec, c in cav.items():
            e0, e1 = _events()
            torch.cuda.synchronize()
            e0.record(stream)
            c.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms[prec] = e0.elapsed_time(e1)
        T32, u32, S32, lf32 = cav[0].get()
        T16, u16, S16, lf16 = cav[1].get()
        Tc, uc, Sc, lfc = cav[2].get()
        for c in cav.values():
            c.close()
        res[name] = {"fp32_control_max_abs_dT": float(np.abs(Tc - T32).max()),
                     "fp32_control_max_abs_dS": float(np.abs(Sc - S32).max()),
                     "fp32_control_d_liquid_fraction": abs(lfc - lf32),
                     "fp16_vs_fp32_max_abs_dT": float(np.abs(T16 - T32).max()),
                     "fp16_vs_fp32_max_abs_du": float(np.abs(u16 - u32).max()),
                     "fp16_vs_fp32_max_abs_dS": float(np.abs(S16 - S32).max()),
                     "liquid_fraction_fp32": lf32, "liquid_fraction_fp16": lf16,
                     "s_fp32": ms[0] * 1e-3, "s_fp16": ms[1] * 1e-3}
    return res


def convection_leg(steps=20000, n=128, every=500, dump_dir=None):
    """Convection-controlled melting in a 128^3 cavity heated at y = 0 (Ra
    1e5, Pr 0.02, Ste 0.1, Ma 0.1, front from s0 = 1), the whole 20000-step
    run: liquid and all-node MLUPS, the stream-collide's HBM roofline
    fraction over the run (algorithmic bytes of the liquid and active solid
    nodes of each step over the stream-collide time), the liquid fraction
    and the mean heat-surface Nusselt number against time from the
    on-device report ring (FP64 totals every `every` steps) and summaries of
    the final front S(x, z) and Nusselt number Nu(x, z).  The run goes in
    chunks of `every` steps with the front read back between them (for the
    node counts); only the chunks are timed.  Steps are replayed from CUDA
    graphs except the last two of each chunk, whose stream-collide launches
    are timed with CUDA events: their mean stands for the chunk's launches
    in the roofline (launch timing needs step-by-step launches)."""
    import torch
    from paper_1604_03478_gb300 import Cavity
    stream = torch.cuda.current_stream()
    peak, _ = hbm_peak()
    cav = Cavity(n, n, n, stream=stream.cuda_stream, face=0, Ra=1e5, Pr=0.02, Ste=0.1, Ma=0.1, s0=1.0, derive=True)
    cav.set_report(every, steps // every + 1)
    S = cav.get(T=False, u=False)[2]
    counts = [liquid_counts(S, cav.H)]
    ms = 0.0
    k1 = 0.0
    done = 0
    while done < steps:
        k = min(every, steps - done)
        e0, e1 = _events()
        torch.cuda.synchronize()
        e0.record(stream)
        cav.step(k - 2)
        cav.set_timing(True)
        cav.kernel_time(reset=True)
        cav.step(2)
        cav.set_timing(False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        sc_ms, sc_n = cav.kernel_time(reset=True)
        k1 += sc_ms / sc_n * k
        done += k
        S = cav.get(T=False, u=False)[2]
        counts.append(liquid_counts(S, cav.H))
    nk = steps
    rows = cav.get_report()
    info = cav.info()
    nu, nu_mean = cav.nusselt()
    cav.close()
    # node-steps by the trapezoid rule over the chunks (counts change by at
    # most one node per column and step)
    c = np.asarray(counts, dtype=np.float64)
    w = np.diff(np.concatenate([[0], np.minimum(np.arange(1, len(c)) * every, steps)]))
    liq_steps = float(np.sum(0.5 * (c[1:, 0] + c[:-1, 0]) * w))
    sol_steps = float(np.sum(0.5 * (c[1:, 1] + c[:-1, 1]) * w))
    alg = 208.0 * liq_steps + 28.0 * sol_steps
    gbs = alg / (k1 * 1e-3) / 1e9
    mid = n // 2
    if dump_dir:
        os.makedirs(dump_dir, exist_ok=True)
        np.save(os.path.join(dump_dir, "convection_128cube_front.npy"), S)
        np.save(os.path.join(dump_dir, "convection_128cube_nusselt.npy"), nu)
    return {"cube": n, "steps": steps, "ms_per_step": ms / steps,
            "liquid_mlups": liq_steps / (ms * 1e-3) / 1e6,
            "all_node_mlups": n ** 3 * steps / (ms * 1e-3) / 1e6,
            "stream_collide_ms_per_launch": k1 / nk,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "kernel": "fused stream-collide, averaged over the run (2 timed launches per chunk)",
                         "algorithmic_bytes": alg, "stream_collide_ms": k1},
            "stream_collide_share_of_step": k1 / ms,
            "fourier_number_at_end": info["alpha"] * (info["t0"] + steps) / float(n * n),
            "liquid_fraction_vs_step": [[int(r[0]), float(r[1])] for r in rows],
            "nusselt_mean_vs_step": [[int(r[0]), float(r[7])] for r in rows],
            "nusselt": {"mean": nu_mean, "at_mid_x_vs_z": [[int(z), float(nu[z, mid])] for z in range(0, n, 16)],
                        "mean_over_z_vs_x": [[int(x), float(nu[:, x].mean())] for x in range(0, n, 16)],
                        "layout": "Nu[z, x] on the heated wall y = 0, -H dT/dy / (Th - Tm)"},
            "front": {"mean": float(S.mean()), "min": float(S.min()), "max": float(S.max()),
                      "at_mid_x_vs_z": [[int(z), float(S[z, mid])] for z in range(0, n, 8)] + [[n - 1, float(S[n - 1, mid])]],
                      "layout": "S[z, x], heights above the heated wall y = 0 in lattice units"},
            "workload": "128^3 heated at y=0, Ra 1e5, Pr 0.02, Ste 0.1, Ma 0.1, front from s0 = 1, FP32"}


def table1_leg(n=96):
    """The paper's two convection-melting cases (section 3.2, Table 1): Pr
    0.02, Ste 0.1, Ra 25000 to Fo 1.00 and Ra 10000 to Fo 1.57 (the same
    lattice time by Eq. 7), n^3 heated at y = 0, Ma 0.1, front from s0 = 1:
    the quantities the paper discusses with Figs. 4 and 5 (liquid fraction,
    heat-surface Nusselt number, front across x, temperature against
    height) and the run's throughput."""
    import torch
    from paper_1604_03478_gb300 import Cavity
    stream = torch.cuda.current_stream()
    cases = [(1, 0.02, 25000.0, 0.1, 1.00), (2, 0.02, 10000.0, 0.1, 1.57)]
    out = {}
    for case, Pr, Ra, Ste, Fo in cases:
        cav = Cavity(n, n, n, stream=stream.cuda_stream, face=0, Ra=Ra, Pr=Pr, Ste=Ste, Ma=0.1, s0=1.0, derive=True)
        info = cav.info()
        steps = int(round(Fo * n * n / info["alpha"] - info["t0"]))
        cav.set_report(max(1, steps // 10), 16)
        steps_fo1 = int(round(1.0 * n * n / info["alpha"] - info["t0"]))
        e0, e1 = _events()
        torch.cuda.synchronize()
        e0.record(stream)
        cav.step(steps_fo1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        lf_fo1 = cav.get(T=False, u=False)[3]
        e0.record(stream)
        cav.step(steps - steps_fo1)
        e1.record(stream)
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
        T, u, S, lf = cav.get()
        nu, nu_mean = cav.nusselt()
        rows = cav.get_report()
        cav.close()
        zmid = slice(n // 2 - 8, n // 2 + 8)
        out["case%d" % case] = {
            "Ra": Ra, "Fo": Fo, "steps": steps, "lattice_time": info["t0"] + steps, "ms": ms,
            "us_per_step": ms * 1e3 / steps, "liquid_fraction": lf, "liquid_fraction_at_Fo_1": lf_fo1,
            "nusselt_mean": nu_mean,
            "nusselt_over_z_vs_x": [[int(x), float(nu[:, x].mean())] for x in range(0, n, 8)],
            "front_over_z_vs_x": [[int(x), float(S[:, x].mean())] for x in range(0, n, 8)],
            "front_std_across_x_at_mid_height": float(S[zmid, :].std(axis=1).mean()),
            "T_near_wall_vs_z": [[int(z), float(T[z, 2, :].mean())] for z in range(0, n, 8)],
            "liquid_fraction_vs_Fo": [[float(info["alpha"] * (info["t0"] + r[0]) / (n * n)), float(r[1])]
                                      for r in rows],
            "nusselt_mean_vs_Fo": [[float(info["alpha"] * (info["t0"] + r[0]) / (n * n)), float(r[7])]
                                   for r in rows]}
    out["workload"] = ("%d^3 heated at y=0, Pr 0.02, Ste 0.1, Ma 0.1, front from s0 = 1, FP32; case 1 Ra 25000 "
                       "to Fo 1.00, case 2 Ra 10000 to Fo 1.57" % n)
    return out


SOLID_CASE = dict(CASE, Tc=-0.25, Tm=0.0, solid=1, ks_kl=1.0)


def solid_leg(steps=200, twin_steps=400):
    """Heat conduction in a subcooled solid (Eq. 6's k_s term): the 256^3
    workload with the cold wall at Tc = -0.25 (Tm = 0, k_s = k_l), every node
    updated each step.  Liquid and all-node MLUPS, the stream-collide's
    roofline (208 B per liquid node, 56 B per solid node: its 7 energy
    populations read and written), the step's share outside it, and the
    error against the FP64 oracle on a 64^3 twin."""
    import torch
    import oracle
    from paper_1604_03478_gb300 import Cavity
    stream = torch.cuda.current_stream()
    peak, _ = hbm_peak()
    n = N_EDGE
    cav = Cavity(n, n, n, stream=stream.cuda_stream, **SOLID_CASE)
    cav.step(10)
    cav.sync()
    S0 = cav.get(T=False, u=False)[2]
    cav.set_timing(True)
    cav.kernel_time(reset=True)
    e0, e1 = _events()
    e0.record(stream)
    cav.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    k1, nk = cav.kernel_time(reset=True)
    T, _, S1, lf = cav.get(u=False)
    cav.close()
    js = lambda S: float(np.clip(np.ceil(S - 0.5), 0, n).sum())  # noqa: E731
    n_liq = 0.5 * (js(S0) + js(S1))
    n_sol = float(n ** 3) - n_liq
    alg = 208.0 * n_liq + 56.0 * n_sol
    gbs = alg / (k1 / nk * 1e-3) / 1e9
    # the 64^3 twin against the oracle
    m = 64
    case = dict(SOLID_CASE, s0=0.4 * m)
    o = oracle.Oracle(m, m, m, **case)
    g = Cavity(m, m, m, stream=stream.cuda_stream, **case)
    o.step(twin_steps)
    g.step(twin_steps)
    To, _, So, lfo = o.get()
    Tg, _, Sg, lfg = g.get()
    o.close()
    g.close()
    return {"steps": steps, "ms_per_step": ms / steps, "liquid_mlups": n_liq * steps / (ms * 1e-3) / 1e6,
            "all_node_mlups": n ** 3 * steps / (ms * 1e-3) / 1e6,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "kernel": "fused stream-collide with conduction in the solid (k_even_cond/k_odd_cond)",
                         "algorithmic_bytes_per_launch": alg, "avg_launch_ms": k1 / nk,
                         "bytes": "208 per liquid node, 56 per solid node"},
            "stream_collide_share_of_step": k1 / ms, "min_T": float(T.min()), "liquid_fraction": lf,
            "twin_error": {"steps": twin_steps, "max_abs_dT": float(np.abs(Tg - To).max()),
                           "max_abs_dS": float(np.abs(Sg - So).max()), "abs_d_liquid_fraction": abs(lfg - lfo)},
            "workload": "256^3 heated at y=0, Ra 1e6, Pr 0.02, Ste 0.05, Ma 0.1, cold wall Tc = -0.25 < Tm = 0, "
                        "k_s = k_l, front at 0.4 H, FP32; twin 64^3 over %d steps" % twin_steps}


def ensemble_leg(steps=10000, seq_steps=1000, n_cav=48, seed=2016):
    """48 seeded cavities of uneven sizes advanced by the persistent kernel
    for the configured 10000 steps (replayed from its captured graph), then
    the same cavities stepped one after another (each by its own step-by-step
    or graph-replayed launches) over seq_steps.  MLUPS count liquid
    node-updates (liquid counts averaged over each run); the roofline
    fraction is the ensemble's whole step (all three phases) against the
    stream-collide's 208 B per liquid node (28 B per active solid node), and
    the same bytes over the stream-collide phase alone (the kernel's own
    phase timers)."""
    import torch
    from paper_1604_03478_gb300 import Ensemble, autotune, inputs
    stream = torch.cuda.current_stream()
    peak, _ = hbm_peak()
    draws = inputs.ensemble(n_cav, seed)
    cases = [dict(nx=d["n"], ny=d["n"], nz=d["n"], face=d["face"], Ra=d["Ra"], Pr=0.02, Ste=d["Ste"], Ma=0.1,
                  s0=0.4 * d["n"], derive=True) for d in draws]
    ens = Ensemble(cases, stream=stream.cuda_stream)
    shape, _ = autotune.tune_ensemble(ens, steps=4)
    ens.step(4)
    ens.sync()
    members = [ens.member(k) for k in range(n_cav)]

    def counts():
        liq = sol = 0
        for m in members:
            S = m.get(T=False, u=False)[2]
            a, b = liquid_counts(S, m.H)
            liq += a
            sol += b
        return liq, sol

    c0 = counts()
    ens.phase_times(reset=True)
    e0, e1 = _events()
    e0.record(stream)
    ens.step(steps)
    e1.record(stream)
    ens.sync()
    torch.cuda.synchronize()
    ms_ens = e0.elapsed_time(e1)
    phases = ens.phase_times()
    c1 = counts()
    liq_ens = 0.5 * (c0[0] + c1[0])
    sol_ens = 0.5 * (c0[1] + c1[1])
    e0.record(stream)
    for m in members:
        m.step(seq_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1)
    c2 = counts()
    liq_seq = 0.5 * (c1[0] + c2[0])
    info = ens.info()
    ens.close()
    mlups = liq_ens * steps / (ms_ens * 1e-3) / 1e6
    seq_mlups = liq_seq * seq_steps / (ms_seq * 1e-3) / 1e6
    gbs = (208.0 * liq_ens + 28.0 * sol_ens) * steps / (ms_ens * 1e-3) / 1e9
    sc_gbs = (208.0 * liq_ens + 28.0 * sol_ens) / (phases["stream_collide_us"] * 1e-6) / 1e9
    return {"cavities": n_cav, "nodes": info["nodes"], "liquid_nodes": liq_ens, "steps": steps,
            "mlups": mlups, "sequential_mlups": seq_mlups, "sequential_steps": seq_steps,
            "speedup_vs_sequential": mlups / seq_mlups,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                         "timed": "whole ensemble step (stream-collide, front and flip phases with their barriers)"},
            "phases_us_per_step": phases,
            "stream_collide_phase_roofline": {
                "bound": "hbm", "achieved": sc_gbs, "peak": peak, "unit": "GB/s", "frac": sc_gbs / peak,
                "timed": "phase 1 alone (the fused stream-collide of every cavity, up to block 0 leaving its "
                         "closing grid barrier), on the GPU's global timer"},
            "launch": {"block": shape[0], "nodes_per_thread": shape[1]},
            "workload": "sizes uniform in {48,64,96,128,160}, Ra log-uniform [1e4,1e6], Ste U[0.05,0.2], "
                        "Pr 0.02, heated face y0 or z0, seed %d, front at 0.4 H, FP32" % seed}


def adjoint_leg(steps=4000, n=96):
    """Gradient of the final liquid fraction w.r.t. the heated-wall field and
    Ra on the 96^3 side-heated cube (Ra 1e5, Pr 0.02, Ste 0.1), sqrt(N)
    checkpoints; times of the plain forward run, the recorded forward and
    the backward."""
    import torch
    from paper_1604_03478_gb300 import Cavity, inputs
    stream = torch.cuda.current_stream()
    case = dict(face=0, Ra=1e5, Pr=0.02, Ste=0.1, Ma=0.1, s0=1.0, derive=True)
    wall = (1.0 + inputs.gaussian_field(n * n, 0.01, 5)).astype(np.float32)
    res = {}
    seed = np.full(n * n, 1.0 / (n * n * n))

    def gradient(cav, key):
        e0, e1 = _events()
        torch.cuda.synchronize()
        e0.record(stream)
        cav.tape_forward(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        res["tape" + key] = e0.elapsed_time(e1)
        t0 = time.perf_counter()
        dth, par = cav.tape_backward(seed)
        res["backward" + key] = (time.perf_counter() - t0) * 1e3
        return dth, par

    # the plain forward run
    cav = Cavity(n, n, n, stream=stream.cuda_stream, **case)
    cav.set_hot_wall(wall)
    e0, e1 = _events()
    torch.cuda.synchronize()
    e0.record(stream)
    cav.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    res["plain"] = e0.elapsed_time(e1)
    cav.close()
    # the gradient: first on a new handle (allocating the checkpoints and the
    # backward's buffers), then again from the same initial state on that
    # handle (buffers kept: the cost of each gradient of a loop)
    cav = Cavity(n, n, n, stream=stream.cuda_stream, **case)
    cav.set_hot_wall(wall)
    f0, g0, s0 = cav.get_state()
    dth, par = gradient(cav, "_first")
    res["dL_dRa"] = par["Ra"]
    res["grad_norm_wall"] = float(np.linalg.norm(dth))
    res["dL_dv1"] = float(dth.ravel() @ inputs.gaussian_field(n * n, 1.0, 7))
    res["dL_dv2"] = float(dth.ravel() @ inputs.gaussian_field(n * n, 1.0, 8))
    cav.set_state(f0, g0, s0)
    dth2, par2 = gradient(cav, "")
    res["repeat_rel_diff"] = float(abs(par2["Ra"] / par["Ra"] - 1.0))
    cav.close()
    out = {"cube": n, "steps": steps, "forward_ms": res["plain"], "recorded_forward_ms": res["tape"],
           "backward_ms": res["backward"], "adjoint_forward_ratio": res["backward"] / res["plain"],
           "total_over_forward": (res["tape"] + res["backward"]) / res["plain"],
           "first_gradient": {"recorded_forward_ms": res["tape_first"], "backward_ms": res["backward_first"],
                              "total_over_forward": (res["tape_first"] + res["backward_first"]) / res["plain"],
                              "note": "a new handle: includes allocating the checkpoints and the backward's buffers"},
           "repeat": "timed: a second gradient from the same initial state on the same handle (buffers kept); "
                     "its dL/dRa differs from the first by %.1e (the state round trip through get/set_state "
                     "rounds the shifted populations once)" % res["repeat_rel_diff"],
           "dL_dRa": res["dL_dRa"], "grad_norm_wall": res["grad_norm_wall"],
           "dL_dv1": res["dL_dv1"], "dL_dv2": res["dL_dv2"],
           "loss": "final liquid fraction", "checkpoints": "every ceil(sqrt(steps)) steps",
           "directions": "v1, v2 = N(0, 1) per wall column, seeds 7 and 8"}
    if steps == 4000 and n == 96:
        # the FP64 oracle's complex-step values for this workload
        golden = {}
        with open(os.path.join(ROOT, "tests", "golden", "adjoint_96cube_4000steps.txt")) as f:
            for ln in f:
                if ln.strip() and not ln.startswith("#"):
                    k, v = ln.split()
                    golden[k] = float(v)
        out["vs_oracle_tangent"] = {k: abs(out[a] / golden[b] - 1.0) for k, a, b in
                                    (("rel_err_dRa", "dL_dRa", "dlf_dRa"), ("rel_err_dv1", "dL_dv1", "dlf_dv1"),
                                     ("rel_err_dv2", "dL_dv2", "dlf_dv2"))}
    return out


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import torch
    rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1604_03478_gb300 import Cavity
    stream = torch.cuda.current_stream()
    n = args.edge
    cav = Cavity(n, n, n, stream=stream.cuda_stream, precision=args.precision, **dict(CASE, s0=0.4 * n))
    H = cav.H
    warm = max(3, args.warmup)
    cav.step(warm)
    cav.sync()
    S0 = cav.get(T=False, u=False)[2]
    n_liq0, n_sol0 = liquid_counts(S0, H)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
            torch.cuda.synchronize()

    gpu_id = torch.cuda.get_device_properties(local).uuid
    gpu_id = "GPU-" + str(gpu_id) if not str(gpu_id).startswith("GPU-") else str(gpu_id)
    cav.set_timing(True)
    cav.kernel_time(reset=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    with ClockSampler(gpu_id) as clk:
        ev0.record(stream)
        cav.step(args.steps)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    k1_ms, k1_n = cav.kernel_time(reset=True)
    cav.set_timing(False)
    S1 = cav.get(T=False, u=False)[2]
    n_liq1, n_sol1 = liquid_counts(S1, H)
    n_liq = 0.5 * (n_liq0 + n_liq1)
    n_sol = 0.5 * (n_sol0 + n_sol1)
    ms_max, units = reduce_across_ranks(ms, n_liq * args.steps, dist, "cuda")
    value = units / (ms_max * 1e-3) / 1e6

    # roofline of the dominant kernel (the fused stream-collide)
    k1_avg_ms = k1_ms / max(k1_n, 1)
    bl, bs = (208.0, 28.0) if args.precision == 0 else (104.0, 14.0)
    alg_bytes = bl * n_liq + bs * n_sol
    achieved = alg_bytes / (k1_avg_ms * 1e-3) / 1e9
    peak, peak_src = hbm_peak()

    # end to end through the C ABI with host buffers
    ncols = cav.ncols
    thw_host = torch.full((ncols,), 1.0, dtype=torch.float32).pin_memory()
    S_host = torch.empty((ncols,), dtype=torch.float64).pin_memory()
    lf_host = torch.empty((1,), dtype=torch.float64).pin_memory()
    from paper_1604_03478_gb300 import _abi
    import ctypes as C
    L = _abi.load()
    h = cav._h
    e2e_steps = args.e2e_steps
    # (a) pipelined: the step's front and liquid fraction are read back with
    # lbm_melt_get_async into alternating page-locked buffers, so the copies
    # of step t travel while step t + 1 runs; one sync at the end
    S2 = [torch.empty((ncols,), dtype=torch.float64).pin_memory() for _ in range(2)]
    lf2 = [torch.empty((1,), dtype=torch.float64).pin_memory() for _ in range(2)]
    barrier()
    t0 = time.perf_counter()
    for t in range(e2e_steps):
        st = L.lbm_melt_set_hot_wall(h, C.c_void_p(thw_host.data_ptr()), 0)
        st |= L.lbm_melt_step(h, 1)
        st |= L.lbm_melt_get_async(h, C.c_void_p(S2[t & 1].data_ptr()), C.c_void_p(lf2[t & 1].data_ptr()), 0)
        if st != 0:
            raise RuntimeError(L.lbm_melt_last_error(h).decode())
    if L.lbm_melt_sync(h) != 0:
        raise RuntimeError(L.lbm_melt_last_error(h).decode())
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_ms, e2e_units = reduce_across_ranks(e2e_s * 1e3, n_liq1 * e2e_steps, dist, "cuda")
    e2e_value = e2e_units / (e2e_ms * 1e-3) / 1e6
    # (b) synchronous: lbm_melt_get waits for every step's results
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st = L.lbm_melt_set_hot_wall(h, C.c_void_p(thw_host.data_ptr()), 0)
        st |= L.lbm_melt_step(h, 1)
        st |= L.lbm_melt_get(h, None, None, C.c_void_p(S_host.data_ptr()), C.c_void_p(lf_host.data_ptr()), 0)
        if st != 0:
            raise RuntimeError(L.lbm_melt_last_error(h).decode())
    barrier()
    e2e_sync_s = time.perf_counter() - t0
    e2e_sync_ms, _ = reduce_across_ranks(e2e_sync_s * 1e3, n_liq1 * e2e_steps, dist, "cuda")
    e2e_sync_value = e2e_units / (e2e_sync_ms * 1e-3) / 1e6

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, cores, (v1, dt1) = oracle_sample(2, n=n, single_steps=1)
        cpu = {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": "2 oracle steps of the full %d^3 workload from its initial state (%.1f s)" % (n, dt),
               "single_thread": {"value": v1, "unit": "MLUPS", "cores": 1,
                                 "sample": "1 more oracle step of the same run on one thread (%.1f s)" % dt1}}

    extra = {}
    if rank == 0 and world == 1 and not args.skip_extra and n == N_EDGE and args.precision == 0:
        extra["precision"] = precision_leg()
        extra["ensemble"] = ensemble_leg()
        extra["adjoint"] = adjoint_leg()
        extra["convection"] = convection_leg(dump_dir=args.dump_dir)
        extra["table1"] = table1_leg()
        extra["solid"] = solid_leg()

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if (n == N_EDGE and args.precision == 0) else
                   "%d^3 cavity, %s storage, otherwise as the 256^3 workload" % (n, "FP32" if args.precision == 0
                                                                                   else "shifted FP16"),
                   "nodes": n ** 3, "liquid_nodes": n_liq,
                   "liquid_fraction": float(np.mean(S1) / H), "parallelism": "replicas" if world > 1 else "single",
                   "l2": "state 1.7 GB > L2 (inputs larger than L2, no flush)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": recorded_traffic() if (n == N_EDGE and args.precision == 0) else None,
                     "traffic_source": TRAFFIC_RECORD, "kernel": "fused stream-collide (k_even/k_odd)",
                     "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": k1_avg_ms, "peak_source": peak_src},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": ncols * 4,
                "d2h_bytes_per_step": ncols * 8 + 8, "steps": e2e_steps,
                "read_back": "lbm_melt_get_async into alternating page-locked buffers, one sync at the end",
                "synchronous_value": e2e_sync_value},
        "gpu_launches": 3 * args.steps,
        "clocks": clk.summary(),
        "all_node_mlups": (units / n_liq) * (n ** 3) / (ms_max * 1e-3) / 1e6,
    }
    line.update(extra)
    cav.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_leg(args):
    import torch
    torch.cuda.set_device(0)
    legs = {"precision": precision_leg, "ensemble": ensemble_leg, "adjoint": adjoint_leg,
            "convection": convection_leg, "table1": table1_leg, "solid": solid_leg}
    kw = {"steps": args.leg_steps} if args.leg_steps > 0 and args.leg != "table1" else {}
    if args.leg == "convection":
        kw["dump_dir"] = args.dump_dir
    print(json.dumps({"leg": args.leg, **legs[args.leg](**kw)}))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.leg:
        return run_leg(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
