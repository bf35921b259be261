"""Benchmark: hydro cell-updates/s on one GB300 (turbulent 256^3 periodic box).

One step = the whole hot path on the device: Godunov update of every level (gather,
primitives, MinMod slopes, MUSCL-Hancock predictor, HLLC at every face, FP64 update,
fused CFL candidate of the next step), then reflux + restriction from the finest level
up.  The timed path is the chosen form (FP32 reconstruction and Riemann solve, FP64
state accumulation); the plain FP64 path is timed beside it, the FP64 CPU oracle on the
host cores as a baseline.  Prints one JSON line (rank 0).

Multi-GPU: a single box has a halo exchange every step, so this workload runs as
independent replicas (one box per GPU, weak scaling, no data-path collective).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hydro cell-updates/s on 1 GB300, chosen vs plain FP64 at equal L1 err; HBM GB/s"
UNIT = "cell-updates/s"
LEVEL = 8                     # 256^3 cells
GAMMA = 5.0 / 3.0
CFL = 0.8
BYTES_PER_UPDATE = 80         # FP64 state read (5 x 8 B) + write (5 x 8 B) per cell update
WORKLOAD = "turbulent periodic box 256^3, single level (octree levels 1-8), gamma=5/3, HLLC, CFL 0.8"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload():
    import numpy as np
    from paper_2411_14631_gb300 import workloads as W
    lx = W.uniform_tree(LEVEL)
    rho, v = W.turbulent_fields(LEVEL)
    return lx, rho, v


def prims_for(lx_sorted_xyz, rho, v):
    from paper_2411_14631_gb300 import workloads as W
    return W.grid_prims(lx_sorted_xyz, LEVEL, rho, v)


def gpu_cell_centres(tree):
    """Cell centres in the device tree's cell order (from its coordinate tables)."""
    import numpy as np
    tab = tree.tables()
    l = tab["lvl"].cpu().numpy().astype(np.int64)
    xyz = np.stack([tab["ix"].cpu().numpy(), tab["iy"].cpu().numpy(), tab["iz"].cpu().numpy()], axis=1)
    c = np.arange(8)
    off = np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], axis=1)
    dx = np.ldexp(1.0, -l)
    return ((xyz[:, None, :] * 2.0 + off[None] + 0.5) * dx[:, None, None]).reshape(-1, 3)


def time_path(H, tree, prm, w0, steps, warmup, stream, label, kernel_events=True):
    """Run warmup + timed steps; returns (ms_per_step, godunov_ms_per_launch, sim)."""
    import torch
    sim = H.Simulation(tree, prm, w0=w0)
    nlev = tree.levelmax

    def one_step(ev=None):
        sim.dt_next.fill_(1.0e300)
        if ev is not None:
            ev[0].record(stream)
        H.hydro_godunov_level(tree, -1, prm, sim.u, sim.u_new, sim.reg, sim.dt, sim.dt_next, stream)
        if ev is not None:
            ev[1].record(stream)
        for l in range(nlev - 1, 0, -1):
            H.hydro_reflux_level(tree, l, prm, sim.reg, sim.u_new, sim.dt, sim.dt_next, stream)
        sim.u, sim.u_new = sim.u_new, sim.u
        sim.dt, sim.dt_next = sim.dt_next, sim.dt

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            one_step()
        stream.synchronize()
        kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        for k in range(steps):
            one_step(kev[k] if kernel_events else None)
        t1.record(stream)
        t1.synchronize()
    ms = t0.elapsed_time(t1) / steps
    gms = statistics.mean(a.elapsed_time(b) for a, b in kev) if kernel_events else None
    launches_per_step = 1 + (nlev - 1)
    return ms, gms, sim, launches_per_step


def time_e2e(H, tree, prm, w0, steps, stream):
    """Public-API end to end: per step, H2D of the state from pinned host memory,
    hydro_step, D2H of the new state to pinned host memory."""
    import torch
    sim = H.Simulation(tree, prm, w0=w0)
    host_in = torch.empty_like(sim.u, device="cpu").pin_memory()
    host_in.copy_(sim.u.cpu())
    host_out = torch.empty_like(host_in).pin_memory()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(steps):
            sim.u.copy_(host_in, non_blocking=True)
            H.hydro_step(tree, prm, sim.u, sim.u_new, sim.reg, sim.dt, sim.dt_next, stream)
            host_out.copy_(sim.u_new, non_blocking=True)
        t1.record(stream)
        t1.synchronize()
    ms = t0.elapsed_time(t1) / steps
    nbytes = sim.u.numel() * 8
    return ms, nbytes


def cpu_baseline(lx, rho, v, sample_steps=1):
    import numpy as np
    import oracle as O
    from paper_2411_14631_gb300 import workloads as W
    O.build()
    t = O.Tree(lx, LEVEL, (0,) * 6)
    xyz, _ = t.cell_centres()
    w = W.grid_prims(xyz, LEVEL, rho, v)
    prm = O.params(gamma=GAMMA, cfl=CFL)
    u = t.init_from_prim(w, prm)
    leaf = int((t.son < 0).sum())
    t0 = time.perf_counter()
    for _ in range(sample_steps):
        u, dt, st = t.step(u, prm)
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": leaf * sample_steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d full step(s) of the 256^3 box (%d leaf cells), FP64 C oracle, OpenMP static over octs"
                      % (sample_steps, leaf), "seconds": el}


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    lx, rho, v = make_workload()
    import oracle as O
    from paper_2411_14631_gb300 import workloads as W
    O.build()
    t = O.Tree(lx, LEVEL, (0,) * 6)
    xyz, _ = t.cell_centres()
    prm = O.params(gamma=GAMMA, cfl=CFL)
    u = t.init_from_prim(W.grid_prims(xyz, LEVEL, rho, v), prm)
    leaf = int((t.son < 0).sum())
    # each step is a bounded sample: the Godunov update of one eighth of the level-8 octs
    # (round robin), counted as the leaf-cell updates it performs
    o0, o1 = int(t.lvl_off[LEVEL]), int(t.lvl_off[LEVEL + 1])
    chunk = (o1 - o0 + 7) // 8
    import numpy as np
    u_new = np.empty_like(u)
    reg = np.zeros(t.noct * 30)
    dt = t.courant(u, prm)
    for k in range(args.warmup):
        a = o0 + (k % 8) * chunk
        O.lib().or_octs_update(t._h, O.C.byref(prm), a, min(o1, a + chunk), O._p(u), O._p(u_new), O._p(reg), dt)
    t0 = time.perf_counter()
    cells = 0
    for k in range(args.steps):
        a = o0 + (k % 8) * chunk
        b = min(o1, a + chunk)
        O.lib().or_octs_update(t._h, O.C.byref(prm), a, b, O._p(u), O._p(u_new), O._p(reg), dt)
        cells += 8 * (b - a)
    el = time.perf_counter() - t0
    val = cells / el
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "leaf_cells": leaf},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": "per step: Godunov update of 1/8 of the 256^3 box's octs (%d cells)" % (8 * chunk)},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import numpy as np
    import torch
    from paper_2411_14631_gb300 import build, abi
    build.build()
    from paper_2411_14631_gb300 import hydro as H
    torch.cuda.set_device(local)
    dev = "cuda:%d" % local
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(dev))
    stream = torch.cuda.Stream(device=dev)

    lx, rho, v = make_workload()
    tree = H.Octree(lx, LEVEL, (abi.BC_PERIODIC,) * 6, device=dev)
    xyz = gpu_cell_centres(tree)
    w0 = prims_for(xyz, rho, v)
    leaf = tree.leaf_cells()

    prm32 = H.Params(GAMMA, cfl=CFL, precision=abi.PREC_FP32, tile=args.tile, device=dev)
    clk = Clocks(local)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    barrier()
    clk.start()
    ms, gms, sim32, lps = time_path(H, tree, prm32, w0, args.steps, args.warmup, stream, "fp32")
    barrier()
    clocks = clk.stop()
    if ws > 1:
        tt = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        ms = float(tt.item())
    value = ws * leaf / (ms * 1e-3)
    status, counters = prm32.read_status()

    hbm, peak_kind = peaks()
    achieved = leaf * BYTES_PER_UPDATE / (gms * 1e-3) / 1e9
    traffic_path = os.path.join(ROOT, "profiles", "traffic.json")
    traffic = None
    if os.path.exists(traffic_path):
        tj = json.load(open(traffic_path))
        if tj.get("kernel_source_hash") == build.source_hash():
            traffic = tj.get("dram_bytes_per_launch")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "leaf_cells": leaf, "octs": tree.noct,
                      "precision": "FP32 reconstruction + Riemann, FP64 state accumulation",
                      "tile_depth": args.tile or 1, "parallelism": "replicas" if ws > 1 else "single GPU",
                      "l2": "inputs larger than L2 (two 671 MB FP64 state arrays)"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                        "kernel": "k_godunov (fp32, all levels)", "godunov_ms": gms,
                        "algorithmic_bytes_per_launch": leaf * BYTES_PER_UPDATE},
           "gpu_launches": args.steps * lps, "clocks": clocks, "device_status": status}

    if not args.skip_plain:
        prm64 = H.Params(GAMMA, cfl=CFL, precision=abi.PREC_FP64, device=dev)
        ms64, gms64, sim64, _ = time_path(H, tree, prm64, w0, args.steps, args.warmup, stream, "fp64")
        u32 = sim32.u
        u64 = sim64.u
        l1 = (torch.abs(u32[0] - u64[0]).sum() / torch.abs(u64[0]).sum()).item()
        out["fp64_plain"] = {"value": ws * leaf / (ms64 * 1e-3), "ms_per_step": ms64, "godunov_ms": gms64,
                             "speedup_chosen_vs_plain": ms64 / ms}
        out["l1_rho_chosen_vs_fp64"] = l1
        del sim64
    if not args.skip_e2e:
        ems, nbytes = time_e2e(H, tree, prm32, w0, args.steps, stream)
        out["e2e"] = {"value": ws * leaf / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": nbytes, "ms_per_step": ems}
    if rank == 0 and ws == 1 and not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(lx, rho, v)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
