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
        return int((self.tables()["son"] < 0).sum())

    def flux_reg_bytes(self):
        return int(lib().hydro_flux_reg_bytes(C.byref(self.t)))


class Params:
    """hydro_params with device status word and counters."""

    def __init__(self, gamma, cfl=0.8, rho_floor=1e-10, p_floor=1e-20, riemann=abi.RIEMANN_HLLC,
                 precision=abi.PREC_FP64, tile=0, device="cuda:0"):
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.counters = torch.zeros(abi.NCOUNTERS, dtype=torch.int64, device=device)
        self.c = abi.HydroParams(gamma, cfl, rho_floor, p_floor, riemann, precision, tile, 0, None, 0.0, 0.0,
                                 self.status.data_ptr(), self.counters.data_ptr())

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


def hydro_reflux_level(tree, level, prm, reg, u_new, dt, dt_next=None, stream=None):
    check("hydro_reflux_level",
          lib().hydro_reflux_level(C.byref(tree.t), level, C.byref(prm.c), _ptr(reg), _ptr(u_new), _ptr(dt),
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


class Simulation:
    """State buffers and the step sequence of one run (u_old -> u_new, dt on the device).

    Each ``step()`` is one pass of the hot path: Godunov update of every level (one
    launch), reflux + restriction from the finest level up, and the CFL step of the next
    step fused into both (dt never leaves the device)."""

    def __init__(self, tree, prm, w0=None, u0=None):
        self.tree, self.prm = tree, prm
        dev = tree.device
        self.u = torch.empty((5, tree.ncell), dtype=torch.float64, device=dev)
        self.u_new = torch.empty_like(self.u)
        self.reg = torch.zeros(max(1, tree.flux_reg_bytes() // 8), dtype=torch.float64, device=dev)
        self.dt = torch.zeros(1, dtype=torch.float64, device=dev)
        self.dt_next = torch.zeros(1, dtype=torch.float64, device=dev)
        if u0 is not None:
            self.u.copy_(u0)
        else:
            w = torch.as_tensor(np.ascontiguousarray(w0), dtype=torch.float64).to(dev)
            hydro_init_from_prim(tree, prm, w, self.u)
        hydro_courant(tree, prm, self.u, self.dt)
        self.time = 0.0
        self.nsteps = 0

    def step(self, stream=None):
        hydro_step(self.tree, self.prm, self.u, self.u_new, self.reg, self.dt, self.dt_next, stream)
        self.u, self.u_new = self.u_new, self.u
        self.dt, self.dt_next = self.dt_next, self.dt
        self.nsteps += 1

    def prims(self):
        w = torch.empty_like(self.u)
        hydro_prim_of_state(self.tree, self.prm, self.u, w)
        return w
