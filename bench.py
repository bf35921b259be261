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


def job_ms(ms, ws, device):
    """Whole-job time of a step: the slowest rank's (every rank runs its own box)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, ws, ms):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return ws * units_per_rank / (ms * 1e-3)


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
    # the initial state and dt are made on the current stream; the steps below run on
    # `stream`, which does not wait for it by itself
    stream.wait_stream(torch.cuda.current_stream())
    def one_step(ev=None):
        sim.dt_next.fill_(1.0e300)
        if ev is not None:
            ev[0].record(stream)
        H.hydro_godunov_level(tree, -1, prm, sim.u, sim.u_new, sim.reg, sim.dt, sim.dt_next, stream)
        if ev is not None:
            ev[1].record(stream)
        # the rest of the step, per level (the same bits as hydro_step's launches)
        for l in range(tree.levelmax - 1, 0, -1):
            H.reflux_level(tree, l, prm, sim.reg, sim.u_new, sim.dt, sim.dt_next, stream)
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
    return ms, gms, sim, launches_per_step(tree)


def launches_per_step(tree):
    """Kernels one hydro_step launches on this mesh: the z-column kernel of the deepest
    complete level (when it is level 3 or deeper), one tile-kernel launch for the levels
    above it (plus one that interpolates the ghost fathers' children, when there are any),
    one reflux launch per level from levelmax-1 down to the one above the deepest complete
    level (none when the deepest complete level is the finest), and one restriction launch
    per three complete levels below that."""
    if tree.t.n_inst > 0:
        return 1
    gl, lmax = int(tree.t.grid_level), tree.levelmax
    n = 1 if gl >= 3 else 0
    if gl < lmax or gl < 3:
        n += 1 + (1 if int(tree.t.n_ghost) > 0 else 0)
    lstop = gl - 1 if gl >= 2 else 1
    lfirst = gl - 2 if (gl >= 2 and gl == lmax) else lmax - 1
    n += max(0, lfirst - lstop + 1)
    n += (max(0, lstop - 1) + 2) // 3
    return n


def time_graph(H, tree, prm, w0, steps, warmup, overlap=False):
    """Whole steps replayed from CUDA graphs (two graphs, alternating state buffers); with
    overlap, the restriction of the complete levels below runs on a second stream during
    the next step, and the timed region ends after the last of them."""
    import torch
    sim = H.Simulation(tree, prm, w0=w0, overlap=overlap).use_graph()
    for _ in range(warmup):
        sim.step()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record()
    for _ in range(steps):
        sim.step()
    sim.join()
    t1.record()
    t1.synchronize()
    return t0.elapsed_time(t1) / steps, sim


def time_e2e(H, tree, prm, w0, steps, stream):
    """Public-API end to end: every step copies its input state from pinned host memory to
    the device, runs hydro_step, and copies the new state back to pinned host memory.
    Steps are independent (each starts from the host input), so they are pipelined over
    three streams with two device slots: the copy-in of step k+1 and the copy-out of step
    k-1 overlap the update of step k (one copy engine each way)."""
    import torch
    sim = H.Simulation(tree, prm, w0=w0)
    host_in = torch.empty_like(sim.u, device="cpu").pin_memory()
    host_in.copy_(sim.u.cpu())
    host_out = [torch.empty_like(host_in).pin_memory() for _ in range(2)]
    u_in = [sim.u, sim.u_new]
    u_out = [torch.empty_like(sim.u) for _ in range(2)]
    reg = sim.reg
    dt = sim.dt
    dtn = [torch.empty_like(sim.dt) for _ in range(2)]
    s_in, s_cmp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    e_in = [torch.cuda.Event() for _ in range(2)]
    e_cmp = [torch.cuda.Event() for _ in range(2)]
    e_out = [torch.cuda.Event() for _ in range(2)]
    e_free_in = [torch.cuda.Event() for _ in range(2)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def run(nsteps):
        for k in range(nsteps):
            j = k % 2
            if k >= 2:
                s_in.wait_event(e_free_in[j])            # step k-2 finished reading u_in[j]
            with torch.cuda.stream(s_in):
                u_in[j].copy_(host_in, non_blocking=True)
                e_in[j].record(s_in)
            s_cmp.wait_event(e_in[j])
            if k >= 2:
                s_cmp.wait_event(e_out[j])               # step k-2's copy-out of u_out[j] done
            H.hydro_step(tree, prm, u_in[j], u_out[j], reg, dt, dtn[j], stream=s_cmp)
            e_cmp[j].record(s_cmp)
            e_free_in[j].record(s_cmp)
            s_out.wait_event(e_cmp[j])
            with torch.cuda.stream(s_out):
                host_out[j].copy_(u_out[j], non_blocking=True)
                e_out[j].record(s_out)

    run(2)                                               # warm-up
    torch.cuda.synchronize()
    t0.record(s_in)
    s_cmp.wait_event(t0)
    s_out.wait_event(t0)
    run(steps)
    s_out.wait_stream(s_cmp)
    s_out.wait_stream(s_in)
    t1.record(s_out)
    t1.synchronize()
    ms = t0.elapsed_time(t1) / steps
    nbytes = sim.u.numel() * 8
    # the copies alone, in and out concurrently on two streams: the floor this pipeline
    # approaches (the host link, not the kernel, bounds the end-to-end step)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    c0.record(s_in)
    s_out.wait_event(c0)
    for k in range(steps):
        with torch.cuda.stream(s_in):
            u_in[k % 2].copy_(host_in, non_blocking=True)
        with torch.cuda.stream(s_out):
            host_out[k % 2].copy_(u_out[k % 2], non_blocking=True)
    s_in.wait_stream(s_out)
    c1.record(s_in)
    c1.synchronize()
    copy_ms = c0.elapsed_time(c1) / steps
    return ms, nbytes, copy_ms


def cpu_baseline(lx, rho, v, min_seconds=10.0, max_steps=8):
    """The FP64 oracle on the host cores: whole steps of the same box, as many as take at
    least min_seconds (at most max_steps, at least one)."""
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
    sample_steps = 0
    while sample_steps < max_steps:
        u, dt, st = t.step(u, prm)
        sample_steps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
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


def l1_fields(u, ref):
    """Relative L1 of rho, |momentum| and E over the (equal-volume) leaf cells."""
    import torch
    mom = torch.sqrt(u[1] ** 2 + u[2] ** 2 + u[3] ** 2)
    momr = torch.sqrt(ref[1] ** 2 + ref[2] ** 2 + ref[3] ** 2)
    out = {}
    for name, a, b in (("rho", u[0], ref[0]), ("mom", mom, momr), ("E", u[4], ref[4])):
        out[name] = float((torch.abs(a - b).sum() / torch.abs(b).sum()).item())
    return out


def equal_l1(H, tree, w0, shape, steps=10):
    """The metric's "at equal L1 err": after `steps` steps at a common fixed dt (3/4 of the
    initial FP32 CFL step), L1 of rho, |momentum| and E of the chosen path (FP32
    reconstruction + HLLC, FP64 accumulation) and of the plain FP64 HLLC path against the
    FP64 exact-Riemann-solver path (equal to the oracle within 1e-12), and between them."""
    import torch
    from paper_2411_14631_gb300 import abi
    dt0 = torch.zeros(1, dtype=torch.float64, device=tree.device)
    H.hydro_courant(tree, H.Params(GAMMA, cfl=CFL, precision=abi.PREC_FP32, device=tree.device),
                    H.Simulation(tree, H.Params(GAMMA, cfl=CFL, device=tree.device), w0=w0).u, dt0)
    dt_fixed = float(dt0.item()) * 0.75
    dt = torch.full((1,), dt_fixed, dtype=torch.float64, device=tree.device)

    def run(prm):
        s_ = H.Simulation(tree, prm, w0=w0)
        for _ in range(steps):
            H.hydro_step(tree, prm, s_.u, s_.u_new, s_.reg, dt, None)
            s_.u, s_.u_new = s_.u_new, s_.u
        torch.cuda.synchronize()
        st, _ = prm.read_status()
        return s_.u, st

    ref, st_ref = run(H.Params(GAMMA, cfl=CFL, riemann=abi.RIEMANN_EXACT, device=tree.device))
    chosen, st_c = run(H.Params(GAMMA, cfl=CFL, precision=abi.PREC_FP32, device=tree.device, **shape))
    plain, st_p = run(H.Params(GAMMA, cfl=CFL, device=tree.device))
    out = {"reference": "FP64 exact-Riemann-solver path (equal to the oracle within 1e-12)", "steps": steps,
           "dt_fixed": dt_fixed, "chosen_fp32_vs_ref": l1_fields(chosen, ref),
           "plain_fp64_vs_ref": l1_fields(plain, ref), "chosen_vs_plain": l1_fields(chosen, plain),
           "status": [st_ref, st_c, st_p]}
    out["chosen_over_plain_rho"] = out["chosen_fp32_vs_ref"]["rho"] / out["plain_fp64_vs_ref"]["rho"]
    out["equal_within_5pct"] = bool(out["chosen_over_plain_rho"] <= 1.05)
    return out


def conservation_drift(H, tree, u0, u1):
    """Relative drift of the leaf totals (mass, momenta, energy) between two states,
    measured on the GPU (hydro_conservation, FP64, fixed summation order); each total's
    drift relative to the larger of its absolute sums."""
    t0 = H.hydro_conservation(tree, u0).cpu().numpy()[0]
    t1 = H.hydro_conservation(tree, u1).cpu().numpy()[0]
    scale = [max(a, b) for a, b in zip(t0[1], t1[1])]
    return [float(abs(b - a) / c) for a, b, c in zip(t0[0], t1[0], scale)]


def study_surrogate(args):
    """Learned Riemann surrogate study on the turbulent 256^3 box: harvest, label, train,
    then exact vs surrogate+fallback vs HLLC against the FP64 exact-solver reference."""
    import numpy as np
    import torch
    from paper_2411_14631_gb300 import build, abi
    build.build()
    from paper_2411_14631_gb300 import hydro as H
    from paper_2411_14631_gb300 import workloads as W
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    torch.cuda.set_device(0)
    out = {"study": "learned Riemann surrogate (BF16 tensor-core MLP + exact fallback)", "data": "synthetic"}
    lx, rho, v = make_workload()
    tree = H.Octree(lx, LEVEL, (abi.BC_PERIODIC,) * 6)
    w0 = prims_for(cell_centres_of(tree), rho, v)
    # ---- harvest from FP64 runs: the turbulent box (10 steps) and the Sod tube (20 steps)
    t0 = time.perf_counter()
    per_step = args.harvest // 10
    chunks = []
    prm64 = H.Params(GAMMA, cfl=CFL)
    sim = H.Simulation(tree, prm64, w0=w0)
    buf = torch.empty((per_step, 6), dtype=torch.float64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    stride = max(1, int(3.75 * leaf_count(tree) / per_step))
    for _ in range(10):
        cnt.zero_()
        H.hydro_harvest_faces(tree, prm64, sim.u, sim.dt, buf, stride, cnt)
        chunks.append(buf[:min(per_step, int(cnt.item()))].clone())
        sim.step()
    del sim
    sod_tree = H.Octree(W.uniform_tree(5), 5, (abi.BC_OUTFLOW,) * 6)
    prm_sod = H.Params(1.4, cfl=CFL)
    sim = H.Simulation(sod_tree, prm_sod, w0=W.sod_prims(cell_centres_of(sod_tree)))
    sod = []
    for _ in range(20):
        cnt.zero_()
        H.hydro_harvest_faces(sod_tree, prm_sod, sim.u, sim.dt, buf, 1, cnt)
        sod.append(buf[:min(per_step, int(cnt.item()))].clone())
        sim.step()
    turb = torch.unique(torch.cat(chunks), dim=0)
    sod = torch.unique(torch.cat(sod), dim=0)
    g = torch.Generator(device="cpu").manual_seed(4)
    sod = sod[torch.randperm(sod.shape[0], generator=g)[:max(1, turb.shape[0] // 99)].cuda()]
    states = torch.cat([turb, sod])
    perm = torch.randperm(states.shape[0], generator=g).cuda()
    states = states[perm].contiguous()
    # both workloads' gammas appear in the set: the turbulent faces at 5/3, the Sod faces at 1.4
    n = states.shape[0]
    n_turb = turb.shape[0]
    gam = torch.where(perm < n_turb, torch.tensor(GAMMA, device="cuda"), torch.tensor(1.4, device="cuda"))
    x = torch.empty((n, 8), dtype=torch.float32, device="cuda")
    y = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for gval in (GAMMA, 1.4):
        idx = torch.nonzero(gam == gval).flatten()
        xs = torch.empty((idx.numel(), 8), dtype=torch.float32, device="cuda")
        ys = torch.empty((idx.numel(), 2), dtype=torch.float32, device="cuda")
        H.mlp_make_dataset(states[idx].contiguous(), gval, xs, ys, status)
        x[idx] = xs
        y[idx] = ys
    out["harvest"] = {"faces": n, "turbulent": n_turb, "sod": int(sod.shape[0]), "stride": stride,
                      "status": int(status.item()), "seconds": time.perf_counter() - t0}
    ntr = int(0.9 * n)
    sur = H.Surrogate(seed=4)
    t1 = time.perf_counter()
    hist = sur.train(x[:ntr], y[:ntr], epochs=args.epochs, batch=4096, lr=3e-3, lr_final=1e-4, seed=4)
    torch.cuda.synchronize()
    ttrain = time.perf_counter() - t1
    yv = sur.forward(x[ntr:])
    val = float(((yv - y[ntr:]) ** 2).sum(dim=1).mean().item())
    out["training"] = {"samples": ntr, "epochs": args.epochs, "batch": 4096, "loss_first_epoch": hist[0],
                       "loss_last_epoch": hist[-1], "val_loss": val, "seconds": ttrain,
                       "samples_per_s": ntr * args.epochs / ttrain}
    # ---- 10 steps at a common fixed dt: the reference and the paths reach the same time
    dt0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    H.hydro_courant(tree, H.Params(GAMMA, cfl=CFL, precision=abi.PREC_FP32), H.Simulation(tree, prm64, w0=w0).u, dt0)
    dt_fixed = float(dt0.item()) * 0.75
    dt = torch.full((1,), dt_fixed, dtype=torch.float64, device="cuda")

    def run(prm, steps=10):
        s_ = H.Simulation(tree, prm, w0=w0)
        for _ in range(steps):
            H.hydro_step(tree, prm, s_.u, s_.u_new, s_.reg, dt, None)
            s_.u, s_.u_new = s_.u_new, s_.u
        torch.cuda.synchronize()
        return s_.u

    ref = run(H.Params(GAMMA, cfl=CFL, riemann=abi.RIEMANN_EXACT))
    paths = {}
    for name, riemann, prec, tonly in (("exact_fp32", abi.RIEMANN_EXACT, abi.PREC_FP32, False),
                                       ("exact_fp32_tiles", abi.RIEMANN_EXACT, abi.PREC_FP32, True),
                                       ("mlp_fallback_fp32", abi.RIEMANN_MLP, abi.PREC_FP32, False),
                                       ("mlp_seeded_newton_fp32", abi.RIEMANN_MLP_SEEDED, abi.PREC_FP32, False),
                                       ("hllc_fp32", abi.RIEMANN_HLLC, abi.PREC_FP32, False),
                                       ("hllc_fp64_plain", abi.RIEMANN_HLLC, abi.PREC_FP64, False)):
        prm = H.Params(GAMMA, cfl=CFL, riemann=riemann, precision=prec, tiles_only=tonly)
        prm.c.mlp_weights = sur.packed.data_ptr()
        prm.c.mlp_resid_tol = args.tol
        u = run(prm)
        st, cntr = prm.read_status()
        prm.clear_status()
        ms, _ = time_graph(H, tree, prm, w0, 5, 2)
        st2, cntr2 = prm.read_status()
        rec = {"l1_vs_fp64_exact": l1_fields(u, ref), "ms_per_step": ms,
               "cell_updates_per_s": leaf_count(tree) / (ms * 1e-3), "status": st}
        if riemann == abi.RIEMANN_MLP:
            tot = cntr[0] + cntr[1]
            rec["faces_accepted"] = cntr[0]
            rec["fallbacks"] = cntr[1]
            rec["fallback_rate"] = cntr[1] / max(1, tot)
            rec["tol"] = args.tol
        if riemann == abi.RIEMANN_MLP_SEEDED:
            rec["faces_seeded"] = cntr[0]
            rec["cold_starts"] = cntr[1]
        if cntr[3] > 0:
            rec["newton_iterations_per_solve"] = cntr[2] / cntr[3]
            rec["newton_solves"] = cntr[3]
        if tonly:
            rec["kernel"] = "tile kernel for every level (the Newton counters are kept there)"
        paths[name] = rec
    out["paths"] = paths
    out["reference"] = "FP64 exact-solver path on the GPU (equal to the oracle within 1e-12), 10 steps, fixed dt"
    out["dt_fixed"] = dt_fixed
    print(json.dumps(out))
    return 0


def study_mlp(args):
    """Throughput of the surrogate network's inference: the tcgen05 kernel (TMEM
    accumulators and activations) against the mma.sync kernel, on as many samples as the
    turbulent 256^3 box has faces per step (3 x 256^3), inputs resident in HBM.  The
    SiLU's tanh runs on the MUFU unit (measured here by mlp_tanh_rate: 16 results per clock
    per SM on GB300), 192 per sample: the ceiling the line reports beside the result."""
    import numpy as np
    import torch
    from paper_2411_14631_gb300 import build
    build.build()
    from paper_2411_14631_gb300 import hydro as H
    torch.cuda.set_device(0)
    n = args.mlp_n
    # seeded parameters, biases included (std 1/sqrt(fan in) for the weights, 0.3 for the biases)
    rng = np.random.default_rng(1)
    th = np.concatenate([rng.normal(0.0, 1.0 / np.sqrt(sh[1]) if len(sh) == 2 else 0.3, int(np.prod(sh)))
                         for sh in [(64, 7), (64,), (64, 64), (64,), (64, 64), (64,), (2, 64), (2,)]])
    sur = H.Surrogate(theta=th.astype(np.float32))
    g = torch.Generator(device="cuda").manual_seed(5)
    # face features of the shape the harvest produces: six normalised states and gamma
    x = torch.randn((n, 8), device="cuda", generator=g)
    x[:, 6] = 5.0 / 3.0
    y = torch.empty((n, 2), device="cuda")
    y_ref = torch.empty((n, 2), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    clocks = Clocks(0)
    clk = None
    reps = max(args.steps, 100)           # about half a second per path: the clock sampler sees it
    rec = {}
    for name, fn in (("tcgen05", lambda: H.mlp_forward_tc(sur.packed, x, y, status)),
                     ("mma_sync", lambda: H.mlp_forward(sur.packed, x, y_ref))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if name == "tcgen05":
            clocks.start()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        if name == "tcgen05":
            clk = clocks.stop()
        ms = e0.elapsed_time(e1) / reps
        rec[name] = {"ms": ms, "samples_per_s": n / (ms * 1e-3), "tflops": 2.0 * 8962 * n / (ms * 1e-3) / 1e12}
    diff = float((y - y_ref).abs().max().item()) / max(float(y_ref.abs().max().item()), 1e-30)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = clk.get("sm_mhz") or 2070
    tanh_per_clk = H.mlp_tanh_rate()          # measured MUFU tanh results per clock per SM
    ceiling = tanh_per_clk * mhz * 1e6 * nsm / 192.0
    out = {"study": "surrogate inference throughput (tcgen05 vs mma.sync)", "data": "synthetic",
           "samples": n, "repetitions": reps, "paths": rec, "status": int(status.item()), "max_rel_diff_tc_vs_mma_sync": diff,
           "tanh_results_per_clock_per_sm": tanh_per_clk, "tanh_ceiling_samples_per_s": ceiling,
           "tcgen05_frac_of_tanh_ceiling": rec["tcgen05"]["samples_per_s"] / ceiling, "clocks": clk}
    print(json.dumps(out))
    return 0


def study_sedov(args):
    """Batch of 48 independent Sedov-Taylor blasts on uneven boxes (32^3..192^3, sizes from
    default_rng(5)), one launch per step with a CFL step per box.  Throughput of the chosen
    FP32 path and the plain FP64 path (CUDA graphs); then each box runs until its exact
    shock radius reaches 0.3 (frozen afterwards by a zero time step) and its numerical
    radius (peak of the radially averaged density) is compared with R = xi0 (E t^2/rho)^(1/5),
    xi0 = 0.851^(-1/5) for gamma = 1.4 (Kamm & Timmes 2007)."""
    import numpy as np
    import torch
    from paper_2411_14631_gb300 import build, abi
    build.build()
    from paper_2411_14631_gb300 import hydro as H
    from paper_2411_14631_gb300 import workloads as W
    torch.cuda.set_device(0)
    sizes = W.sedov_batch_sizes(48, seed=5)
    tree = H.Octree.boxes(sizes, (abi.BC_OUTFLOW,) * 6)
    w0 = W.batch_prims(sizes, lambda N: W.sedov_box_prims_lex(N))
    cells = tree.ncell
    out = {"study": "Sedov-Taylor batch: 48 boxes, one launch per step, per-box CFL", "data": "synthetic",
           "sizes": [int(x) for x in sizes], "cells": cells}
    from paper_2411_14631_gb300 import autotune
    shape, tune_ms = autotune.tune(tree, 1.4, w0, precision=abi.PREC_FP32, cfl=CFL, use_cache=False)
    res = {}
    for name, prec, steps in (("fp32_chosen", abi.PREC_FP32, args.steps), ("fp64_plain", abi.PREC_FP64, 3)):
        prm = H.Params(1.4, cfl=CFL, precision=prec, **(shape if prec == abi.PREC_FP32 else dict(tile=1)))
        ms, _ = time_graph(H, tree, prm, w0, steps, 2)
        res[name] = {"ms_per_step": ms, "cell_updates_per_s": cells / (ms * 1e-3), "steps_timed": steps}
    res["speedup"] = res["fp64_plain"]["ms_per_step"] / res["fp32_chosen"]["ms_per_step"]
    out["throughput"] = res
    out["launch_shape"] = shape
    out["autotune_ms_per_step"] = tune_ms
    # accuracy run: FP32 chosen path, each box frozen at its own target radius
    xi0 = 0.851 ** -0.2
    prm = H.Params(1.4, cfl=CFL, precision=abi.PREC_FP32, **shape)
    sim = H.Simulation(tree, prm, w0=w0)
    tb = np.zeros(len(sizes))
    frozen = np.zeros(len(sizes), dtype=bool)
    nstep = 0
    while not frozen.all() and nstep < 5000:
        d = sim.dt.cpu().numpy()
        d[frozen] = 0.0
        # freeze a box when its next step would pass the target time
        t_target = (0.3 / xi0) ** 2.5
        over = (~frozen) & (tb + d > t_target)
        d[over] = np.maximum(t_target - tb[over], 0.0)
        sim.dt.copy_(torch.as_tensor(d))
        tb += d
        frozen |= over
        sim.step()
        nstep += 1
    rho = sim.u[0].cpu().numpy()
    radii = []
    for b, N in enumerate(sizes):
        N = int(N)
        i, j, k = W.box_cell_ijk(N)
        seg = rho[tree.cell_off[b]:tree.cell_off[b + 1]]
        c = (N // 2 + 0.5) / N
        r = np.sqrt(((i + 0.5) / N - c) ** 2 + ((j + 0.5) / N - c) ** 2 + ((k + 0.5) / N - c) ** 2)
        nb = int(0.5 * N)
        idx = np.minimum((r * N).astype(np.int64), nb)
        sums = np.bincount(idx, weights=seg, minlength=nb + 1)[:nb]
        cnts = np.bincount(idx, minlength=nb + 1)[:nb]
        prof = sums / np.maximum(cnts, 1)
        R_num = (np.argmax(prof) + 0.5) / N
        R_ex = xi0 * (tb[b] ** 2) ** 0.2
        radii.append({"N": N, "t": float(tb[b]), "R_exact": R_ex, "R_num": R_num,
                      "rel_err": abs(R_num - R_ex) / R_ex, "ok": bool(abs(R_num - R_ex) <= max(2.0 / N, 0.05 * R_ex))})
    out["accuracy"] = {"steps": nstep, "all_within_max(2 cells, 5%)": all(r["ok"] for r in radii),
                       "max_rel_err": max(r["rel_err"] for r in radii), "per_box": radii}
    st, _ = prm.read_status()
    out["device_status"] = st
    print(json.dumps(out))
    return 0


def study_amr(args):
    """Plummer-clump AMR mesh (base level 7 refined to level 12 by default, 64 clumps): throughput of
    the chosen FP32 path and the plain FP64 path (all levels in one update launch, then
    reflux + restriction per level, CUDA graphs), and conservation over 10 steps."""
    import numpy as np
    import torch
    from paper_2411_14631_gb300 import build, abi
    build.build()
    from paper_2411_14631_gb300 import hydro as H
    from paper_2411_14631_gb300 import workloads as W
    from paper_2411_14631_gb300.bench_util import cell_centres_of
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    base, lmax = args.amr_base, args.amr_lmax
    lx, centres = W.plummer_tree(base=base, lmax=lmax)
    tree = H.Octree(lx, base, (abi.BC_PERIODIC,) * 6)
    w0 = W.plummer_prims(cell_centres_of(tree), centres)
    tab = tree.tables()
    son = tab["son"].cpu().numpy()
    lvl = np.repeat(tab["lvl"].cpu().numpy(), 8)
    leaf = son < 0
    out = {"study": "Plummer-clump AMR mesh, levels %d-%d, all levels in one launch" % (base, lmax),
           "data": "synthetic", "octs": tree.noct, "leaf_cells": int(leaf.sum()),
           "leaf_cells_per_level": {int(l): int((leaf & (lvl == l)).sum()) for l in range(base, lmax + 1)},
           "setup_seconds": time.perf_counter() - t0}
    from paper_2411_14631_gb300 import autotune
    shape, tune_ms = autotune.tune(tree, 5.0 / 3.0, w0, precision=abi.PREC_FP32, cfl=CFL, use_cache=False)
    res = {}
    for name, prec, steps in (("fp32_chosen", abi.PREC_FP32, args.steps), ("fp64_plain", abi.PREC_FP64, 3)):
        prm = H.Params(5.0 / 3.0, cfl=CFL, precision=prec, **(shape if prec == abi.PREC_FP32 else dict(tile=1)))
        ms, sim = time_graph(H, tree, prm, w0, steps, 2, overlap=prec == abi.PREC_FP32 and not args.no_overlap)
        res[name] = {"ms_per_step": ms, "cell_updates_per_s": int(leaf.sum()) / (ms * 1e-3), "steps_timed": steps}
    res["speedup"] = res["fp64_plain"]["ms_per_step"] / res["fp32_chosen"]["ms_per_step"]
    out["throughput"] = res
    # sub-cycled levels (level l makes 2^(l-base) steps per coarse step): simulated time per
    # wall-clock second against one time step for all levels, FP32 path, CUDA graphs
    prm32 = H.Params(5.0 / 3.0, cfl=CFL, precision=abi.PREC_FP32, **shape)
    single = H.Simulation(tree, prm32, w0=w0)
    dt_single = float(single.dt.item())
    del single
    sc = H.SubcycledSimulation(tree, prm32, w0=w0).use_graph()
    for _ in range(2):
        sc.step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nsc = max(3, args.steps // 2)
    e0.record()
    for _ in range(nsc):
        sc.step()
    e1.record()
    torch.cuda.synchronize()
    ms_sc = e0.elapsed_time(e1) / nsc
    dt_sc = float(sc.dt.item())
    per_level = {int(l): int((leaf & (lvl == l)).sum()) for l in range(base, lmax + 1)}
    upd = sum(n * 2 ** (l - base) for l, n in per_level.items())
    out["subcycled"] = {"ms_per_coarse_step": ms_sc, "dt_coarse": dt_sc, "dt_single_level_step": dt_single,
                        "leaf_updates_per_coarse_step": upd, "leaf_updates_per_s": upd / (ms_sc * 1e-3),
                        "sim_time_per_wall_s": dt_sc / (ms_sc * 1e-3),
                        "sim_time_per_wall_s_single_dt": dt_single / (res["fp32_chosen"]["ms_per_step"] * 1e-3),
                        "steps_timed": nsc}
    out["subcycled"]["gain_in_sim_time_per_wall_s"] = (out["subcycled"]["sim_time_per_wall_s"] /
                                                       out["subcycled"]["sim_time_per_wall_s_single_dt"])
    del sc
    out["launch_shape"] = shape
    out["autotune_ms_per_step"] = tune_ms
    for name, prec in (("fp64", abi.PREC_FP64), ("fp32", abi.PREC_FP32)):
        sim = H.Simulation(tree, H.Params(5.0 / 3.0, cfl=CFL, precision=prec, **(shape if prec else dict(tile=1))),
                           w0=w0)
        u0 = sim.u.clone()
        for _ in range(10):
            sim.step()
        # drift of each leaf total relative to the larger of its start and end absolute sums
        # (momenta start at zero), from the GPU conservation diagnostics
        out["conservation_" + name] = {"steps": 10, "rel_drift": conservation_drift(H, tree, u0, sim.u),
                                       "how": "hydro_conservation (GPU FP64 leaf totals)"}
        del u0
        if prec == abi.PREC_FP32:
            # refine_fine on the evolved state: flags, 2:1 balance, device oct list, the new
            # tree (Hilbert keys, sort, tables) and the state remap
            thr = 2.0 ** (-3 * base)              # one background base cell of mass
            tree.refine(sim.u, thr, lmax)               # warm-up (allocations, first launches)
            torch.cuda.synchronize()
            t0r = time.perf_counter()
            reps = 5
            for _ in range(reps):
                new, u_new = tree.refine(sim.u, thr, lmax)
            torch.cuda.synchronize()
            dtr = (time.perf_counter() - t0r) / reps
            out["refine"] = {"ms": dtr * 1e3, "octs_before": tree.noct, "octs_after": new.noct,
                             "levelmax_after": new.levelmax, "mass_thr": thr,
                             "note": "wall time of Octree.refine (three synchronising C calls, buffers allocated "
                                     "by the caller each time), after 10 FP32 steps",
                             "step_ms_fp32": res["fp32_chosen"]["ms_per_step"]}
            del new, u_new
    print(json.dumps(out))
    return 0


def study_poisson(args):
    """Poisson solve of Sec. 2.3 on an N^3 Dirichlet box (Plummer-clump source): CG
    (pipelined, no preconditioner) against PPCG (incomplete-Poisson preconditioner).
    Per-iteration kernel time (events around a fixed number of fused iteration launches on
    the launching stream), iterations and time to eps = 1e-4 (Eq. 3), roofline of the
    iteration kernel against HBM and the FP64 pipe, and the oracle on the host cores."""
    import numpy as np
    import torch
    from paper_2411_14631_gb300 import build, abi
    build.build()
    from paper_2411_14631_gb300 import poisson as PS
    from paper_2411_14631_gb300 import workloads as W
    torch.cuda.set_device(0)
    N = args.poisson_n
    shape = (N, N, N)
    n = N ** 3
    b_h = W.poisson_rhs(N)
    b = torch.tensor(b_h, device="cuda:0")
    stream = torch.cuda.Stream()
    hbm, peak_kind = peaks()
    # FP64 pipe: 1.25 TFLOP/s nominal = 0.625e12 DFMA/s, i.e. 2 DP instructions per clock
    # per SM at 2.07 GHz on 152 SMs
    fp64_peak = 152 * 2 * 2.07e9
    # algorithmic DP instructions and HBM bytes per cell and iteration
    alg = {abi.PRECOND_IP: (23, 16 * 8), abi.PRECOND_NONE: (14, 12 * 8)}
    out = {"study": "Poisson solve on a %d^3 Dirichlet box, CG vs PPCG (Sec. 2.3, Fig. 4)" % N,
           "data": "synthetic: 64 Plummer clumps (core 0.005, contrast 1e4, truncated at r = 0.1), "
                   "b = -4 pi h^2 (rho - mean)", "cells": n, "tol": 1e-4,
           "l2": "inputs larger than L2 (8 FP64 vectors of %d MB)" % (n * 8 >> 20)}
    clk = Clocks(0)
    res = {}
    K = args.steps if args.steps > 10 else 50
    for name, pc in (("cg", abi.PRECOND_NONE), ("ppcg", abi.PRECOND_IP)):
        best = None
        sweep = {}
        for ty in ((8, 16) if args.poisson_tile_y == 0 else (args.poisson_tile_y,)):
            for seg in ((0, 14, 16, 22, 32, 43, 64) if args.poisson_seg < 0 else (args.poisson_seg,)):
                s = PS.PPCG(shape, precond=pc, tol=0.0, max_iter=K + 10, tile_y=ty, seg=seg)
                x = torch.zeros(n, dtype=torch.float64, device="cuda:0")
                with torch.cuda.stream(stream):
                    s.start(b, x, stream)
                    s.iterate(x, 5, stream)            # warm-up
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    s.iterate(x, K, stream)
                    e1.record(stream)
                stream.synchronize()
                ms = e0.elapsed_time(e1) / K
                sweep["%d/%d" % (ty, seg)] = round(ms, 4)
                if best is None or ms < best[0]:
                    best = (ms, ty, seg)
                del s, x
        ms, ty, seg = best
        # time to solution at the best launch shape, clocks sampled meanwhile
        s = PS.PPCG(shape, precond=pc, tol=1e-4, max_iter=5000, tile_y=ty, seg=seg)
        x = torch.zeros(n, dtype=torch.float64, device="cuda:0")
        s.solve(b, x.clone(), stream)             # warm-up solve
        torch.cuda.synchronize()
        clk.start()
        with torch.cuda.stream(stream):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, eps, info = s.solve(b, x, stream)
            e1.record(stream)
        stream.synchronize()
        clocks = clk.stop()
        clk = Clocks(0)
        solve_ms = e0.elapsed_time(e1)
        ops, nbytes = alg[pc]
        res[name] = {"iterations_to_tol": info.iters, "status": info.status, "eps_final": info.eps,
                     "solve_ms": solve_ms, "iteration_ms": ms, "tile_y": ty, "seg": seg,
                     "iteration_ms_by_tile_y_seg": sweep,
                     "cell_iterations_per_s": n / (ms * 1e-3),
                     "hbm": {"algorithmic_bytes_per_cell": nbytes, "achieved_gbs": n * nbytes / (ms * 1e-3) / 1e9,
                             "peak_gbs": hbm, "peak_kind": peak_kind,
                             "frac": n * nbytes / (ms * 1e-3) / 1e9 / hbm},
                     "fp64": {"algorithmic_dp_instr_per_cell": ops, "achieved_gops": n * ops / (ms * 1e-3) / 1e9,
                              "peak_gops": fp64_peak / 1e9, "peak_kind": "derived from the nominal 1.25 TFLOP/s",
                              "frac": n * ops / (ms * 1e-3) / fp64_peak},
                     "launches_per_iteration": 1, "clocks": clocks,
                     "eps_history_every_10": [float(e) for e in eps[::10]]}
        del s, x
    res["iteration_ratio_cg_over_ppcg"] = res["cg"]["iterations_to_tol"] / res["ppcg"]["iterations_to_tol"]
    res["time_ratio_cg_over_ppcg"] = res["cg"]["solve_ms"] / res["ppcg"]["solve_ms"]
    out.update(res)
    if not args.skip_cpu:
        import oracle as O
        O.build()
        t0 = time.perf_counter()
        it = 20
        O.ppcg(shape, b_h, precond=O.PRECOND_IP, tol=0.0, maxit=it)
        dt = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": n * it / dt, "unit": "cell-iterations/s", "cores": 1, "kind": "oracle",
                               "sample": "oracle PPCG, %d iterations of the %d^3 solve (incl. set-up)" % (it, N)}
    print(json.dumps(out))
    return 0


def leaf_count(tree):
    return tree.leaf_cells()


def main():
    global LEVEL, WORKLOAD
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-l1", action="store_true", help="skip the equal-L1 runs (FP64 exact-solver reference)")
    ap.add_argument("--study", default=None, choices=["surrogate", "sedov", "amr", "poisson", "mlp"])
    ap.add_argument("--mlp-n", type=int, default=3 * 256 ** 3, help="samples of --study mlp")
    ap.add_argument("--no-overlap", action="store_true",
                    help="run the complete levels' restriction inside each step instead of overlapping the next")
    ap.add_argument("--amr-base", type=int, default=7, help="complete base level of --study amr")
    ap.add_argument("--amr-lmax", type=int, default=12, help="finest level of --study amr")
    ap.add_argument("--level", type=int, default=8,
                    help="level of the turbulent box (2^level cells per axis); 8 is the benchmark's 256^3")
    ap.add_argument("--poisson-n", type=int, default=256)
    ap.add_argument("--poisson-tile-y", type=int, default=0, help="8 or 16; 0 tries both")
    ap.add_argument("--poisson-seg", type=int, default=-1, help="z planes per block; -1 tries several")
    ap.add_argument("--harvest", type=int, default=10_000_000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--tol", type=float, default=0.02)
    args = ap.parse_args()
    if args.level != LEVEL:
        n = 1 << args.level
        WORKLOAD = WORKLOAD.replace("256^3", "%d^3" % n).replace("levels 1-8", "levels 1-%d" % args.level)
        LEVEL = args.level
    ws, rank, local = dist_setup()
    if args.study == "surrogate":
        return study_surrogate(args)
    if args.study == "sedov":
        return study_sedov(args)
    if args.study == "amr":
        return study_amr(args)
    if args.study == "poisson":
        return study_poisson(args)
    if args.study == "mlp":
        return study_mlp(args)
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

    shape = dict(tile=args.tile, col_kernel=0, col_seg=0)
    tune_ms = None
    if args.tile == 0:
        from paper_2411_14631_gb300 import autotune
        shape, tune_ms = autotune.tune(tree, GAMMA, w0, precision=abi.PREC_FP32, cfl=CFL)
    prm32 = H.Params(GAMMA, cfl=CFL, precision=abi.PREC_FP32, device=dev, **shape)
    clk = Clocks(local)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    # per-kernel timing (eager launches, events around the update kernel)
    _, gms, sim32e, lps = time_path(H, tree, prm32, w0, args.steps, args.warmup, stream, "fp32")
    barrier()
    clk.start()
    ms, sim32 = time_graph(H, tree, prm32, w0, args.steps, args.warmup, overlap=not args.no_overlap)
    barrier()
    clocks = clk.stop()
    drift = conservation_drift(H, tree, H.Simulation(tree, prm32, w0=w0).u, sim32.u)
    ms = job_ms(ms, ws, dev)
    value = job_value(leaf, ws, ms)
    status, counters = prm32.read_status()

    hbm, peak_kind = peaks()
    achieved = leaf * BYTES_PER_UPDATE / (gms * 1e-3) / 1e9
    if shape.get("col_kernel", 0) != 1 and (1 << LEVEL) % 16 == 0:
        kernel_name = ("k_godunov_pen<HLLC> (column-per-thread z-column update of the complete level, "
                       "16x16-cell footprints, %s-cell segments)" % (shape.get("col_seg") or "default"))
    else:
        kernel_name = "k_godunov_col<float, HLLC> (slab z-column update of the complete level, 8x8-cell footprints)"
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
                      "launch_shape": shape, "autotune_ms_per_step": tune_ms, "cuda_graph": True,
                      "restriction_overlap": not args.no_overlap,
                      "parallelism": "replicas" if ws > 1 else "single GPU",
                      "l2": "inputs larger than L2 (two 671 MB FP64 state arrays)"},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                        "frac": achieved / hbm, "traffic": traffic, "peak_kind": peak_kind,
                        "kernel": kernel_name,
                        "godunov_ms": gms,
                        "algorithmic_bytes_per_launch": leaf * BYTES_PER_UPDATE},
           "gpu_launches": args.steps * lps, "launches_per_step": lps, "clocks": clocks, "device_status": status,
           "conservation": {"steps": sim32.nsteps, "rel_drift_mass_momx_momy_momz_energy": drift,
                            "how": "hydro_conservation (GPU FP64 leaf totals) before and after the timed run"}}

    if not args.skip_plain:
        prm64 = H.Params(GAMMA, cfl=CFL, precision=abi.PREC_FP64, device=dev)
        ms64, gms64, sim64, _ = time_path(H, tree, prm64, w0, args.steps, args.warmup, stream, "fp64")
        # the eager FP32 run made the same number of steps as the FP64 one (the graph run
        # makes one more, before its capture); each path takes its own CFL steps
        u32 = sim32e.u
        u64 = sim64.u
        l1 = (torch.abs(u32[0] - u64[0]).sum() / torch.abs(u64[0]).sum()).item()
        out["fp64_plain"] = {"value": ws * leaf / (ms64 * 1e-3), "ms_per_step": ms64, "godunov_ms": gms64,
                             "speedup_chosen_vs_plain": ms64 / ms}
        out["l1_rho_chosen_vs_fp64"] = l1
        out["l1_note"] = ("rho, sum|FP32 - FP64| / sum|FP64| over all cells after %d steps of each path"
                          % (args.steps + args.warmup))
        del sim64
    if not args.skip_l1:
        out["equal_l1"] = equal_l1(H, tree, w0, shape)
    if not args.skip_e2e:
        ems, nbytes, copy_ms = time_e2e(H, tree, prm32, w0, args.steps, stream)
        out["e2e"] = {"value": ws * leaf / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": nbytes, "ms_per_step": ems,
                      "copies_only_ms_per_step": copy_ms, "frac_of_copy_floor": copy_ms / ems,
                      "link_gbs_per_direction": nbytes / (copy_ms * 1e-3) / 1e9}
    if rank == 0 and ws == 1 and not args.skip_cpu:
        out["cpu_baseline"] = cpu_baseline(lx, rho, v)
    if rank == 0:
        print(json.dumps(out))
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
