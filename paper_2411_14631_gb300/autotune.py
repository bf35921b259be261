"""Autotuner of the launch shape of the Godunov update.

Candidates are the tile depths the library offers (1: 2x2x2 octs per CTA, 128 threads;
2: 4x4x4 octs, 512 threads).  A cell's arithmetic does not depend on the tile it is
updated in, so every candidate gives bitwise identical states (tested); only speed is
tuned.  Each candidate runs a few steps on the actual mesh, timed with CUDA events;
the winner is cached per (mesh, precision, Riemann solver, GPU name) in a JSON file
(default ``~/.cache/amrhydro/tune.json``, or ``$AMRHYDRO_TUNE_CACHE``)."""
import hashlib
import json
import os

import numpy as np
import torch

from . import abi
from . import hydro as H


def _cache_path():
    return os.environ.get("AMRHYDRO_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "amrhydro",
                                                               "tune.json"))


def mesh_key(tree, precision, riemann):
    h = hashlib.sha256()
    h.update(np.asarray(tree.lvl_off).tobytes())
    h.update(np.asarray(tree.t.bc[:]).tobytes())
    gpu = torch.cuda.get_device_name(tree.device)
    return "%s|p%d|r%d|%s" % (h.hexdigest()[:16], precision, riemann, gpu)


def tune(tree, gamma, w0, precision=abi.PREC_FP32, riemann=abi.RIEMANN_HLLC, steps=3, use_cache=True, **kw):
    """Return the fastest tile depth for this mesh (and the timings, ms per step)."""
    key = mesh_key(tree, precision, riemann)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]["tile"], cache[key]["ms"]
    cands = [1] if (precision == abi.PREC_FP64 or riemann == abi.RIEMANN_MLP) else [1, 2]
    times = {}
    for tile in cands:
        prm = H.Params(gamma, precision=precision, riemann=riemann, tile=tile, device=tree.device, **kw)
        sim = H.Simulation(tree, prm, w0=w0)
        sim.step()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            sim.step()
        e1.record()
        e1.synchronize()
        times[tile] = e0.elapsed_time(e1) / steps
        del sim
    best = min(times, key=times.get)
    if use_cache:
        cache[key] = {"tile": best, "ms": {str(k): v for k, v in times.items()}}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return best, {str(k): v for k, v in times.items()}
