"""Python front end of the C ABI: the same entry points, with PyTorch tensors for
device memory and streams (no arithmetic of the method happens here)."""
import ctypes as C

import numpy as np
import torch

from . import abi
from .abi import check, lib


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Octree:
    """amr_build_octree: the octree on the device, in caller-owned (torch) memory."""

    def __init__(self, lxyz, levelmin, bc=(abi.BC_PERIODIC,) * 6, device="cuda:0", stream=None):
        lxyz = np.ascontiguousarray(lxyz, dtype=np.int32).reshape(-1, 4)
        self.device = torch.device(device)
        g = abi.AmrGeom(levelmin, (C.c_int32 * 6)(*bc))
        tb, wb = C.c_size_t(), C.c_size_t()
        check("amr_build_octree_query",
              lib().amr_build_octree_query(C.byref(g), lxyz.ctypes.data_as(C.c_void_p), lxyz.shape[0],
                                           C.byref(tb), C.byref(wb)))
        self.mem = torch.empty(tb.value, dtype=torch.uint8, device=self.device)
        ws = torch.empty(wb.value, dtype=torch.uint8, device=self.device)
        self.t = abi.AmrTree()
        check("amr_build_octree",
              lib().amr_build_octree(C.byref(g), lxyz.ctypes.data_as(C.c_void_p), lxyz.shape[0], _ptr(self.mem),
                                     tb.value, _ptr(ws), wb.value, C.byref(self.t), _stream(stream)))
        del ws
        self.noct = int(self.t.noct)
        self.ncell = 8 * self.noct
        self.levelmin, self.levelmax = int(self.t.levelmin), int(self.t.levelmax)
        self.lvl_off = np.array(self.t.lvl_off[:], dtype=np.int64)

    @classmethod
    def boxes(cls, sizes, bc=(abi.BC_OUTFLOW,) * 6, device="cuda:0", stream=None):
        """Batch mode: independent uniform unit boxes of sizes[i]^3 cells (multiples of 4)."""
        self = cls.__new__(cls)
        sizes = np.ascontiguousarray(sizes, dtype=np.int32)
        self.device = torch.device(device)
        g = abi.AmrGeom(0, (C.c_int32 * 6)(*bc), sizes.size, sizes.ctypes.data_as(C.c_void_p))
        tb, wb = C.c_size_t(), C.c_size_t()
        check("amr_build_octree_query", lib().amr_build_octree_query(C.byref(g), None, 0, C.byref(tb), C.byref(wb)))
        self.mem = torch.empty(tb.value, dtype=torch.uint8, device=self.device)
        ws = torch.empty(wb.value, dtype=torch.uint8, device=self.device)
        self.t = abi.AmrTree()
        check("amr_build_octree", lib().amr_build_octree(C.byref(g), None, 0, _ptr(self.mem), tb.value, _ptr(ws),
                                                         wb.value, C.byref(self.t), _stream(stream)))
        self.noct = int(self.t.noct)
        self.ncell = 8 * self.noct
        self.levelmin = self.levelmax = 0
        self.lvl_off = np.array(self.t.lvl_off[:], dtype=np.int64)
        self.sizes = sizes
        self.cell_off = np.concatenate([[0], np.cumsum(sizes.astype(np.int64) ** 3)])
        return self

    @property
    def n_inst(self):
        return int(self.t.n_inst)

    def refine(self, u, mass_thr, levelmax, stream=None):
        """refine_fine: the refined tree and the state on it.  Cells with rho dx^3 >
        mass_thr are refined (levels levelmin .. levelmax-1), then 2:1-balanced; the new
        oct list stays on the device, the new tree is built from it and the state is
        copied or interpolated (amr_refine, amr_build_octree_device, amr_remap_state)."""
        L = lib()
        rp = abi.RefineParams(float(mass_thr), int(levelmax), 0)
        wb = L.amr_refine_work_bytes(C.byref(self.t))
        work = torch.empty(wb, dtype=torch.uint8, device=self.device)
        cap = self.ncell + 1
        lxyz = torch.empty((cap, 4), dtype=torch.int32, device=self.device)
        counts = (C.c_int64 * (abi.MAXLEV + 1))()
        n = C.c_int64()
        check("amr_refine", L.amr_refine(C.byref(self.t), C.byref(rp), _ptr(u), _ptr(work), wb, _ptr(lxyz), cap,
                                         counts, C.byref(n), _stream(stream)))
        del work
        new = Octree.__new__(Octree)
        new.device = self.device
        g = abi.AmrGeom(self.levelmin, (C.c_int32 * 6)(*self.t.bc))
        tb, wsb = C.c_size_t(), C.c_size_t()
        check("amr_build_octree_device_query",
              L.amr_build_octree_device_query(C.byref(g), counts, C.byref(tb), C.byref(wsb)))
        new.mem = torch.empty(tb.value, dtype=torch.uint8, device=self.device)
        ws = torch.empty(wsb.value, dtype=torch.uint8, device=self.device)
        new.t = abi.AmrTree()
        check("amr_build_octree_device",
              L.amr_build_octree_device(C.byref(g), _ptr(lxyz), counts, _ptr(new.mem), tb.value, _ptr(ws), wsb.value,
                                        C.byref(new.t), _stream(stream)))
        del ws, lxyz
        new.noct = int(new.t.noct)
        new.ncell = 8 * new.noct
        new.levelmin, new.levelmax = int(new.t.levelmin), int(new.t.levelmax)
        new.lvl_off = np.array(new.t.lvl_off[:], dtype=np.int64)
        u_new = torch.empty((5, new.ncell), dtype=torch.float64, device=self.device)
        status = torch.zeros(1, dtype=torch.int32, device=self.device)
        check("amr_remap_state", L.amr_remap_state(C.byref(self.t), _ptr(u), C.byref(new.t), _ptr(u_new),
                                                   _ptr(status), _stream(stream)))
        st = int(status.item())
        if st != abi.OK:
            raise abi.AmrError("amr_remap_state", st)
        return new, u_new

    def _view(self, ptr, n, dtype):
        off = ptr - self.mem.data_ptr()
        nbytes = n * torch.tensor([], dtype=dtype).element_size()
        return self.mem[off:off + nbytes].view(dtype)

    def tables(self):
        """Device tables as torch views (lvl, ix, iy, iz, key, son, father, nbor, nb27, refmask)."""
        n = self.noct
        t = self.t
        return {"lvl": self._view(t.lvl, n, torch.int32), "ix": self._view(t.ix, n, torch.int32),
                "iy": self._view(t.iy, n, torch.int32), "iz": self._view(t.iz, n, torch.int32),
                "key": self._view(t.key, n, torch.int64), "son": self._view(t.son, 8 * n, torch.int32),
                "father": self._view(t.father, n, torch.int32), "nbor": self._view(t.nbor, 6 * n, torch.int32),
                "nb27": self._view(t.nb27, 27 * n, torch.int32), "refmask": self._view(t.refmask, n, torch.uint8)}

    def ntiles(self, depth):
        return int(self.t.tile_off[depth - 1][abi.MAXLEV + 1])

    def leaf_cells(self):
        if self.t.n_inst > 0:
            return self.ncell
        return int((self.tables()["son"] < 0).sum())

    def flux_reg_bytes(self):
        return int(lib().hydro_flux_reg_bytes(C.byref(self.t)))


class Params:
    """hydro_params with device status word and counters."""

    def __init__(self, gamma, cfl=0.8, rho_floor=1e-10, p_floor=1e-20, riemann=abi.RIEMANN_HLLC,
                 precision=abi.PREC_FP64, tile=0, device="cuda:0", tiles_only=False, limiter=abi.LIMITER_MINMOD,
                 col_kernel=0, col_seg=0, defer_restriction=False):
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.counters = torch.zeros(abi.NCOUNTERS, dtype=torch.int64, device=device)
        self.c = abi.HydroParams(gamma, cfl, rho_floor, p_floor, riemann, precision, tile, int(tiles_only), None,
                                 0.0, limiter, self.status.data_ptr(), self.counters.data_ptr(), col_kernel, col_seg,
                                 int(defer_restriction), 0)

    def with_fields(self, **fields):
        """A copy of these parameters with some hydro_params fields replaced; it shares the
        device status word and counters."""
        known = {f[0] for f in abi.HydroParams._fields_}
        unknown = sorted(set(fields) - known)
        if unknown:
            raise TypeError("hydro_params has no field %s" % ", ".join(unknown))
        q = Params.__new__(Params)
        q.status, q.counters = self.status, self.counters
        q.c = abi.HydroParams.from_buffer_copy(self.c)
        for k, v in fields.items():
            setattr(q.c, k, v)
        return q

    def read_status(self):
        s = C.c_int32()
        cnt = (C.c_ulonglong * abi.NCOUNTERS)()
        check("amr_get_status", lib().amr_get_status(C.byref(self.c), C.byref(s), cnt))
        return s.value, list(cnt)

    def clear_status(self):
        self.status.zero_()
        self.counters.zero_()


def hydro_init_from_prim(tree, prm, w, u, stream=None):
    check("hydro_init_from_prim", lib().hydro_init_from_prim(C.byref(tree.t), C.byref(prm.c), _ptr(w), _ptr(u),
                                                             _stream(stream)))


def hydro_prim_of_state(tree, prm, u, w, stream=None):
    check("hydro_prim_of_state", lib().hydro_prim_of_state(C.byref(tree.t), C.byref(prm.c), _ptr(u), _ptr(w),
                                                           _stream(stream)))


def hydro_courant(tree, prm, u, dt, stream=None):
    check("hydro_courant", lib().hydro_courant(C.byref(tree.t), C.byref(prm.c), _ptr(u), _ptr(dt), _stream(stream)))


def hydro_godunov_level(tree, level, prm, u_old, u_new, reg, dt, dt_next=None, stream=None):
    check("hydro_godunov_level",
          lib().hydro_godunov_level(C.byref(tree.t), level, C.byref(prm.c), _ptr(u_old), _ptr(u_new), _ptr(reg),
                                    _ptr(dt), _ptr(dt_next), _stream(stream)))


def hydro_restrict_complete(tree, u, stream=None):
    check("hydro_restrict_complete", lib().hydro_restrict_complete(C.byref(tree.t), _ptr(u), _stream(stream)))


def hydro_reflux_level(tree, level, prm, reg, u_new, dt, dt_next=None, stream=None):
    check("hydro_reflux_level",
          lib().hydro_reflux_level(C.byref(tree.t), level, C.byref(prm.c), _ptr(reg), _ptr(u_new), _ptr(dt),
                                   _ptr(dt_next), _stream(stream)))


def reflux_level(tree, level, prm, reg, u_new, dt, dt_next=None, stream=None):
    """hydro_reflux_level under its shorter exported name."""
    check("reflux_level",
          lib().reflux_level(C.byref(tree.t), level, C.byref(prm.c), _ptr(reg), _ptr(u_new), _ptr(dt),
                             _ptr(dt_next), _stream(stream)))


def hydro_step(tree, prm, u_old, u_new, reg, dt, dt_next=None, stream=None):
    check("hydro_step", lib().hydro_step(C.byref(tree.t), C.byref(prm.c), _ptr(u_old), _ptr(u_new), _ptr(reg),
                                         _ptr(dt), _ptr(dt_next), _stream(stream)))


def hydro_step_static_scratch(tree, prm, u_old, u_new, dt, dt_next=None, stream=None):
    """hydro_step with the flux register inside the library (for callers that cannot
    allocate device memory when they step); see include/amrhydro.h."""
    check("hydro_step_static_scratch",
          lib().hydro_step_static_scratch(C.byref(tree.t), C.byref(prm.c), _ptr(u_old), _ptr(u_new), _ptr(dt),
                                          _ptr(dt_next), _stream(stream)))


def hydro_conservation(tree, u, totals=None, work=None, blocks=0, stream=None):
    """Leaf totals [nbox][2][5] on the device: sum U dV and sum |U| dV per box (see
    include/amrhydro.h); returns the device tensor."""
    nbox = max(1, tree.n_inst)
    if totals is None:
        totals = torch.empty((nbox, 2, 5), dtype=torch.float64, device=u.device)
    if work is None:
        work = torch.empty(int(lib().hydro_conservation_work_bytes(C.byref(tree.t))), dtype=torch.uint8,
                           device=u.device)
    check("hydro_conservation", lib().hydro_conservation(C.byref(tree.t), _ptr(u), _ptr(totals), _ptr(work),
                                                         work.numel(), blocks, _stream(stream)))
    return totals


def hydro_state_to_fp32(x, y, stream=None):
    """The FP32 path's FP64 -> FP32 conversion of state values (see include/amrhydro.h)."""
    check("hydro_state_to_fp32", lib().hydro_state_to_fp32(_ptr(x), _ptr(y), x.numel(), _stream(stream)))


def hydro_state_from_fp32(y, x, stream=None):
    """The FP32 path's FP32 -> FP64 conversion (exact)."""
    check("hydro_state_from_fp32", lib().hydro_state_from_fp32(_ptr(y), _ptr(x), y.numel(), _stream(stream)))


def hydro_harvest_faces(tree, prm, u, dt, states, stride, count, stream=None):
    """Sampled face-normal (L, R) states of one reconstruction of u (see include/amrhydro.h)."""
    check("hydro_harvest_faces",
          lib().hydro_harvest_faces(C.byref(tree.t), C.byref(prm.c), _ptr(u), _ptr(dt), _ptr(states),
                                    states.shape[0], stride, _ptr(count), _stream(stream)))


def mlp_pack(theta, packed, stream=None):
    check("mlp_pack", lib().mlp_pack(_ptr(theta), _ptr(packed), _stream(stream)))


def mlp_make_dataset(states, gamma, x, y, status=None, stream=None):
    check("mlp_make_dataset", lib().mlp_make_dataset(_ptr(states), states.shape[0], gamma, _ptr(x), _ptr(y),
                                                     _ptr(status), _stream(stream)))


def mlp_forward(packed, x, y, stream=None):
    check("mlp_forward", lib().mlp_forward(_ptr(packed), _ptr(x), _ptr(y), x.shape[0], _stream(stream)))


def mlp_forward_tc(packed, x, y, status=None, stream=None):
    """The network on the tcgen05 tensor cores (tiles of 128 samples)."""
    check("mlp_forward_tc", lib().mlp_forward_tc(_ptr(packed), _ptr(x), _ptr(y), x.shape[0], _ptr(status),
                                                 _stream(stream)))


def mlp_tanh_rate(stream=None):
    """Measured MUFU tanh results per SM clock per SM (mlp_forward_tc's bound)."""
    cycles = torch.zeros(1, dtype=torch.int64, device="cuda")
    results = C.c_int64(0)
    check("mlp_tanh_rate", lib().mlp_tanh_rate(_ptr(cycles), C.byref(results), _stream(stream)))
    torch.cuda.synchronize()
    nsm = torch.cuda.get_device_properties(cycles.device).multi_processor_count
    return results.value / (nsm * int(cycles.item()))


def mlp_grad(packed, x, dy, grad, scratch, stream=None):
    check("mlp_grad", lib().mlp_grad(_ptr(packed), _ptr(x), _ptr(dy), x.shape[0], _ptr(grad), _ptr(scratch),
                                     scratch.numel() * 4, _stream(stream)))


def mlp_train_step(theta, m, v, packed, x, y, lr, t, loss, scratch, stream=None):
    check("mlp_train_step", lib().mlp_train_step(_ptr(theta), _ptr(m), _ptr(v), _ptr(packed), _ptr(x), _ptr(y),
                                                 x.shape[0], lr, t, _ptr(loss), _ptr(scratch), scratch.numel() * 4,
                                                 _stream(stream)))


class Surrogate:
    """The learned Riemann surrogate's device state: FP32 master parameters, Adam
    moments and the packed BF16 block the kernels read.  Initial weights: seeded
    Gaussian, std 1/sqrt(fan_in), zero biases."""

    def __init__(self, seed=4, device="cuda:0", theta=None):
        n = int(lib().mlp_nparams())
        self.device = torch.device(device)
        if theta is None:
            rng = np.random.default_rng(seed)
            th = np.zeros(n, dtype=np.float32)
            shapes = [(64, 7), (64,), (64, 64), (64,), (64, 64), (64,), (2, 64), (2,)]
            o = 0
            for sh in shapes:
                size = int(np.prod(sh))
                if len(sh) == 2:
                    th[o:o + size] = rng.normal(0.0, 1.0 / np.sqrt(sh[1]), size)
                o += size
            theta = th
        self.theta = torch.as_tensor(np.asarray(theta, dtype=np.float32)).to(self.device)
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.packed = torch.empty(int(lib().mlp_packed_bytes()), dtype=torch.uint8, device=self.device)
        self.t = 0
        mlp_pack(self.theta, self.packed)

    def forward(self, x):
        y = torch.empty((x.shape[0], 2), dtype=torch.float32, device=self.device)
        mlp_forward(self.packed, x, y)
        return y

    def train(self, x, y, epochs=1, batch=4096, lr=1e-3, seed=0, lr_final=None):
        """Adam over shuffled minibatches; returns the mean loss of each epoch."""
        n = x.shape[0]
        scratch = torch.empty(int(lib().mlp_scratch_bytes(batch)) // 4 + 1, dtype=torch.float32, device=self.device)
        loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        gen = torch.Generator(device="cpu").manual_seed(seed)
        hist = []
        nb = max(1, n // batch)
        total = epochs * nb
        for ep in range(epochs):
            perm = torch.randperm(n, generator=gen).to(self.device)
            xs, ys = x[perm].contiguous(), y[perm].contiguous()
            acc = torch.zeros(1, dtype=torch.float32, device=self.device)
            for b in range(nb):
                self.t += 1
                rate = lr if lr_final is None else lr * (lr_final / lr) ** (min(self.t, total) / total)
                mlp_train_step(self.theta, self.m, self.v, self.packed, xs[b * batch:(b + 1) * batch],
                               ys[b * batch:(b + 1) * batch], rate, self.t, loss, scratch)
                acc += loss
            hist.append(float(acc.item()) / nb)
        return hist


def hydro_courant_levels(tree, prm, u, dt, stream=None):
    check("hydro_courant_levels", lib().hydro_courant_levels(C.byref(tree.t), C.byref(prm.c), _ptr(u), _ptr(dt),
                                                             _stream(stream)))


def hydro_step_subcycled(tree, prm, u, scratch, reg, dt, dt_levels, stream=None):
    check("hydro_step_subcycled",
          lib().hydro_step_subcycled(C.byref(tree.t), C.byref(prm.c), _ptr(u), _ptr(scratch), _ptr(reg), _ptr(dt),
                                     _ptr(dt_levels), _stream(stream)))


class SubcycledSimulation:
    """A run with sub-cycled levels: each ``step()`` advances the coarsest level by its
    step and every finer level by 2^(l - levelmin) steps of half the previous size
    (hydro_step_subcycled); ``dt`` holds the coarsest level's last step on the device."""

    def __init__(self, tree, prm, w0=None, u0=None):
        self.tree, self.prm = tree, prm
        dev = tree.device
        self.u = torch.empty((5, tree.ncell), dtype=torch.float64, device=dev)
        self.scratch = torch.empty_like(self.u)
        self.reg = torch.zeros(max(1, tree.flux_reg_bytes() // 8), dtype=torch.float64, device=dev)
        self.dt = torch.zeros(1, dtype=torch.float64, device=dev)
        self.dt_levels = torch.zeros(abi.MAXLEV + 2, dtype=torch.float64, device=dev)
        if u0 is not None:
            self.u.copy_(u0)
        else:
            w = torch.as_tensor(np.ascontiguousarray(w0), dtype=torch.float64).to(dev)
            hydro_init_from_prim(tree, prm, w, self.u)
        self.nsteps = 0
        self._graph = None

    def step(self, stream=None):
        if self._graph is not None:
            self._graph.replay()
        else:
            hydro_step_subcycled(self.tree, self.prm, self.u, self.scratch, self.reg, self.dt, self.dt_levels, stream)
        self.nsteps += 1

    def use_graph(self):
        """Capture one step in a CUDA graph (the buffers do not alternate)."""
        self.step()
        torch.cuda.synchronize()
        s = torch.cuda.Stream(device=self.tree.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            hydro_step_subcycled(self.tree, self.prm, self.u, self.scratch, self.reg, self.dt, self.dt_levels,
                                 stream=s)
        self._graph = g
        torch.cuda.synchronize()
        return self


class Simulation:
    """State buffers and the step sequence of one run (u_old -> u_new, dt on the device).

    Each ``step()`` is one pass of the hot path: Godunov update of every level (one
    launch), reflux + restriction from the finest level up, and the CFL step of the next
    step fused into both (dt never leaves the device).  With ``use_graph()`` the step is
    replayed from two CUDA graphs (state A -> B and B -> A), captured once.

    With ``overlap=True`` the restriction of the complete levels below the deepest
    complete level minus one (which no later step reads) runs on a second stream,
    concurrently with the next step: every step first waits for that restriction of the
    step before last, whose buffer it overwrites.  ``join()`` makes the current stream
    wait for the last one (the state is then complete on that stream)."""

    def __init__(self, tree, prm, w0=None, u0=None, overlap=False):
        self.tree, self.prm = tree, prm
        self.overlap = bool(overlap) and tree.t.n_inst == 0 and int(tree.t.grid_level) >= 3
        if self.overlap:
            # the same parameters (and device status words), with the restriction deferred
            self.prm_step = prm.with_fields(defer_restriction=1)
            self._aux = torch.cuda.Stream(device=tree.device)
            self._ev_fork = [torch.cuda.Event(), torch.cuda.Event()]
            self._ev_done = [torch.cuda.Event(), torch.cuda.Event()]
            self._last_done = None
        else:
            self.prm_step = prm
        dev = tree.device
        self.u = torch.empty((5, tree.ncell), dtype=torch.float64, device=dev)
        self.u_new = torch.empty_like(self.u)
        self.reg = torch.zeros(max(1, tree.flux_reg_bytes() // 8), dtype=torch.float64, device=dev)
        ndt = max(1, int(tree.t.n_inst))          # batch mode: one time step per box
        self.dt = torch.zeros(ndt, dtype=torch.float64, device=dev)
        self.dt_next = torch.zeros(ndt, dtype=torch.float64, device=dev)
        if u0 is not None:
            self.u.copy_(u0)
        else:
            w = torch.as_tensor(np.ascontiguousarray(w0), dtype=torch.float64).to(dev)
            hydro_init_from_prim(tree, prm, w, self.u)
        hydro_courant(tree, prm, self.u, self.dt)
        self.time = 0.0
        self.nsteps = 0

        self._graphs = None

    def step(self, stream=None):
        k = self.nsteps % 2
        main = stream if stream is not None else torch.cuda.current_stream(self.tree.device)
        if self.overlap:
            main.wait_event(self._ev_done[k])    # the restriction that read this step's output buffer
        if self._graphs is not None:
            with torch.cuda.stream(main):
                self._graphs[k].replay()
        else:
            hydro_step(self.tree, self.prm_step, self.u, self.u_new, self.reg, self.dt, self.dt_next, main)
        if self.overlap:
            self._ev_fork[k].record(main)
            self._aux.wait_event(self._ev_fork[k])
            hydro_restrict_complete(self.tree, self.u_new, self._aux)
            self._ev_done[k].record(self._aux)
            self._last_done = self._ev_done[k]
        self.u, self.u_new = self.u_new, self.u
        self.dt, self.dt_next = self.dt_next, self.dt
        self.nsteps += 1

    def join(self, stream=None):
        """Order `stream` (default: the current one) after every restriction issued so far."""
        if self.overlap and self._last_done is not None:
            (stream if stream is not None else torch.cuda.current_stream(self.tree.device)).wait_event(self._last_done)

    def use_graph(self):
        """Capture the two step graphs (after one eager step, which sets kernel attributes)."""
        self.step()
        torch.cuda.synchronize()
        graphs = []
        s = torch.cuda.Stream(device=self.tree.device)
        bufs = [(self.u, self.u_new, self.dt, self.dt_next), (self.u_new, self.u, self.dt_next, self.dt)]
        # graph k is used when nsteps % 2 == k; the buffers alternate with every step
        order = bufs if self.nsteps % 2 == 0 else bufs[::-1]
        for (a, b, d0, d1) in order:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=s):
                hydro_step(self.tree, self.prm_step, a, b, self.reg, d0, d1, stream=s)
            graphs.append(g)
        self._graphs = graphs
        torch.cuda.synchronize()
        return self

    def prims(self):
        w = torch.empty_like(self.u)
        hydro_prim_of_state(self.tree, self.prm, self.u, w)
        return w


# ---------------------------------------------------------------------------------------
# Checkpoint / resume: a snapshot of a run through the host, in one .npz file.

CHECKPOINT_VERSION = 1


def save_checkpoint(path, sim):
    """Write the octree's oct list (level, ix, iy, iz per oct; the box sizes in batch
    mode), its levelmin and boundary codes, the FP64 state, the time step(s) of the next
    step, the step count and the time.  The oct list rebuilds the same tree, so a run
    resumed from the file continues bit for bit."""
    tree = sim.tree
    torch.cuda.synchronize(tree.device)
    rec = {"version": np.int32(CHECKPOINT_VERSION), "bc": np.array(tree.t.bc[:], dtype=np.int32),
           "levelmin": np.int32(tree.levelmin), "u": sim.u.cpu().numpy(), "dt": sim.dt.cpu().numpy(),
           "nsteps": np.int64(sim.nsteps), "time": np.float64(sim.time)}
    if tree.n_inst > 0:
        rec["sizes"] = np.asarray(tree.sizes, dtype=np.int32)
    else:
        tab = tree.tables()
        rec["lxyz"] = torch.stack([tab["lvl"], tab["ix"], tab["iy"], tab["iz"]], dim=1).cpu().numpy()
    with open(path, "wb") as f:
        np.savez(f, **rec)


def load_checkpoint(path, prm, device="cuda:0"):
    """Rebuild the octree and the run of a checkpoint written by save_checkpoint;
    returns the Simulation (prm gives the scheme's parameters, which the file does not
    hold)."""
    with np.load(path) as z:
        if int(z["version"]) != CHECKPOINT_VERSION:
            raise ValueError("checkpoint version %d, expected %d" % (int(z["version"]), CHECKPOINT_VERSION))
        bc = tuple(int(b) for b in z["bc"])
        if "sizes" in z:
            tree = Octree.boxes(z["sizes"], bc=bc, device=device)
        else:
            tree = Octree(z["lxyz"], int(z["levelmin"]), bc, device=device)
        u = torch.as_tensor(z["u"]).to(tree.device)
        if tuple(u.shape) != (5, tree.ncell):
            raise ValueError("checkpoint state has shape %s, the rebuilt tree %d cells" % (tuple(u.shape), tree.ncell))
        sim = Simulation(tree, prm, u0=u)
        sim.dt.copy_(torch.as_tensor(z["dt"]))
        sim.nsteps = int(z["nsteps"])
        sim.time = float(z["time"])
    return sim
