"""Project autotuner: picks launch shapes by timing them on the device and
caches the choice as JSON (one file per machine, next to the built library).

Two searches:
  * single cavity: the (bx, by) block shape of the stream-collide kernels,
    per (cavity edge lengths, precision);
  * ensemble: (threads per block, nodes per thread) of the persistent kernel,
    per (number of cavities, total nodes, precision).
Timing is by CUDA events on the handle's stream; the state advances while
tuning (tune before the run you care about, or on a scratch copy).
"""
from __future__ import annotations

import json
import os

from . import build as _build

CACHE = os.path.join(_build.BUILD, "autotune.json")
CAVITY_SHAPES = ((128, 1), (64, 2), (32, 4))
ENSEMBLE_SHAPES = ((64, 2), (128, 1), (128, 2), (128, 4), (128, 8), (256, 1), (256, 2), (256, 4))


def _device_key():
    import torch
    return torch.cuda.get_device_name()


def _load():
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _save(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp%d" % os.getpid()
    with open(tmp, "w") as fh:
        json.dump(d, fh, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time(step, sync, steps, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step(2)
    sync()
    e0.record(stream)
    step(steps)
    e1.record(stream)
    sync()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tune_cavity(cav, steps=20, shapes=CAVITY_SHAPES, use_cache=True):
    """Best (bx, by) for this cavity's size and precision; applied to cav."""
    import torch
    key = "cavity|%s|%s|p%d" % (_device_key(), "x".join(map(str, cav.shape)), cav.grid.precision)
    cache = _load()
    if use_cache and key in cache:
        bx, by = cache[key]["shape"]
        cav.set_launch(bx, by)
        return tuple(cache[key]["shape"]), cache[key]
    stream = torch.cuda.current_stream()
    res = {}
    for bx, by in shapes:
        cav.set_launch(bx, by)
        res["%dx%d" % (bx, by)] = _time(cav.step, cav.sync, steps, stream)
    best = min(res, key=res.get)
    shape = tuple(int(v) for v in best.split("x"))
    cav.set_launch(*shape)
    cache[key] = {"shape": shape, "ms_per_step": res}
    _save(cache)
    return shape, cache[key]


def tune_ensemble(ens, steps=8, shapes=ENSEMBLE_SHAPES, use_cache=True, graph_steps=8):
    """Best (block, nodes per thread) of the persistent kernel; applied."""
    import torch
    info = ens.info()
    prec = ens.member(0).grid.precision if hasattr(ens.member(0), "grid") else 0
    key = "ensemble|%s|n%d|%d|p%d" % (_device_key(), ens.n, info["nodes"], prec)
    cache = _load()
    if use_cache and key in cache:
        b, k = cache[key]["shape"]
        ens.set_launch(b, k, graph_steps)
        return tuple(cache[key]["shape"]), cache[key]
    stream = torch.cuda.current_stream()
    res = {}
    for b, k in shapes:
        ens.set_launch(b, k, graph_steps)
        res["%dx%d" % (b, k)] = _time(ens.step, ens.sync, steps, stream)
    best = min(res, key=res.get)
    shape = tuple(int(v) for v in best.split("x"))
    ens.set_launch(shape[0], shape[1], graph_steps)
    cache[key] = {"shape": shape, "ms_per_step": res}
    _save(cache)
    return shape, cache[key]
