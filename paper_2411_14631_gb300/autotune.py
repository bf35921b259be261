"""Autotuner of the launch shape of the Godunov update.

The candidates are launch shapes only; a cell's arithmetic does not depend on them, so
every candidate gives bitwise identical states and time steps (tested):
  - the z-column kernel of the deepest complete level: the column-per-thread kernel
    (16 x 16-cell footprints, FP32 path) or the slab kernel (8 x 8-cell footprints, two
    planes per step), each with the z segment a CTA marches (``col_kernel``, ``col_seg``);
  - the tile depth of the levels above it (1: 2x2x2 octs per CTA, 2: 4x4x4 octs).
The column candidates are timed first (tile depth at its default), then the tile depths
with the fastest column shape; a mesh with no tile levels skips the second round.  Each
candidate runs a few whole steps on the actual mesh, timed with CUDA events; the winner
is cached per (mesh, precision, Riemann solver, GPU name, kernel source version) in a
JSON file (default ``~/.cache/amrhydro/tune.json``, or ``$AMRHYDRO_TUNE_CACHE``)."""
import hashlib
import json
import os

import numpy as np
import torch

from . import abi
from . import build
from . import hydro as H

CACHE_VERSION = 3


def _cache_path():
    return os.environ.get("AMRHYDRO_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "amrhydro",
                                                               "tune.json"))


def mesh_key(tree, precision, riemann):
    h = hashlib.sha256()
    h.update(np.asarray(tree.lvl_off).tobytes())
    h.update(np.asarray(tree.t.bc[:]).tobytes())
    h.update(np.asarray([int(tree.t.n_inst), int(tree.t.grid_level), int(tree.t.col_work)]).tobytes())
    gpu = torch.cuda.get_device_name(tree.device)
    # a winner timed on other kernel code is timed again
    return "v%d|%s|p%d|r%d|%s|%s" % (CACHE_VERSION, h.hexdigest()[:16], precision, riemann, gpu,
                                     build.library_hash())


def _name(c):
    return "%s/z%d/t%d" % ({0: "auto", 1: "slab", 2: "pencil"}[c["col_kernel"]], c["col_seg"], c["tile"])


def column_candidates(tree, precision, riemann):
    """Launch shapes of the z-column kernel that apply to this mesh."""
    if riemann in (abi.RIEMANN_MLP, abi.RIEMANN_MLP_SEEDED):
        return [dict(col_kernel=0, col_seg=0)]       # the surrogate runs in the tile kernel only
    if tree.t.n_inst > 0:
        n = None                                      # box batches: the segment is fixed (16)
        has_col = int(tree.t.col_work) > 0
    else:
        gl = int(tree.t.grid_level)
        n = 1 << gl
        has_col = gl >= 3
    if not has_col:
        return [dict(col_kernel=0, col_seg=0)]
    cands = []
    if precision == abi.PREC_FP32 and (n is None or n % 16 == 0):
        segs = [0] if n is None else sorted({0} | {s for s in (16, 24, 32, 38, 44, 52, 64, 96, 128) if s <= n})
        cands += [dict(col_kernel=2, col_seg=s) for s in segs]
    segs = [0] if n is None else sorted({0} | {s for s in (16, 32, 64, 128) if s <= n and n % s == 0})
    cands += [dict(col_kernel=1, col_seg=s) for s in segs]
    return cands


def _time(tree, gamma, w0, precision, riemann, steps, cand, kw):
    prm = H.Params(gamma, precision=precision, riemann=riemann, device=tree.device, **cand, **kw)
    sim = H.Simulation(tree, prm, w0=w0)
    sim.step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        sim.step()
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    del sim
    return ms


def tune(tree, gamma, w0, precision=abi.PREC_FP32, riemann=abi.RIEMANN_HLLC, steps=3, use_cache=True, **kw):
    """Return the fastest launch shape for this mesh, as hydro_params fields
    {"col_kernel", "col_seg", "tile"}, and the timings (ms per step) of every candidate."""
    key = mesh_key(tree, precision, riemann)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return dict(cache[key]["best"]), cache[key]["ms"]
    times = {}
    tile0 = 1 if (precision == abi.PREC_FP64 or riemann in (abi.RIEMANN_MLP, abi.RIEMANN_MLP_SEEDED)) else 0
    best_col, best_ms = None, None
    for c in column_candidates(tree, precision, riemann):
        cand = dict(c, tile=tile0)
        ms = _time(tree, gamma, w0, precision, riemann, steps, cand, kw)
        times[_name(cand)] = ms
        if best_ms is None or ms < best_ms:
            best_col, best_ms = cand, ms
    best = best_col
    # tile depth of the levels above the complete one (none on a uniform mesh, and depth 2
    # only in the FP32 path without the surrogate)
    has_tiles = tree.t.n_inst > 0 and int(tree.t.col_work) == 0
    if tree.t.n_inst == 0:
        has_tiles = int(tree.t.grid_level) < tree.levelmax or int(tree.t.grid_level) < 3
    if has_tiles and tile0 == 0:
        for d in (1, 2):
            cand = dict(best_col, tile=d)
            ms = _time(tree, gamma, w0, precision, riemann, steps, cand, kw)
            times[_name(cand)] = ms
            if ms < best_ms:
                best, best_ms = cand, ms
    if use_cache:
        cache[key] = {"best": best, "ms": times}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, path)
    return dict(best), times
