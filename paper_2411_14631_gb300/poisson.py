"""Python front end of the Poisson entry points (include/ppcg.h): the preconditioned
pipelined CG of Sec. 2.3 on a box of cells, with PyTorch tensors for device memory and
streams.  Argument marshalling only; every step runs in the library's kernels."""
import ctypes as C

import torch

from . import abi
from .abi import check, lib
from .hydro import _ptr, _stream


def apply(shape, op, x, stream=None):
    """A x (op = abi.OP_A) or M^-1 x (abi.OP_MINV) for an FP64 device vector of nx*ny*nz cells."""
    nx, ny, nz = shape
    y = torch.empty_like(x)
    check("poisson_apply", lib().poisson_apply(nx, ny, nz, op, _ptr(x), _ptr(y), _stream(stream)))
    return y


class PPCG:
    """A solver for A x = b on a box of shape (nx, ny, nz), vectors indexed i + nx (j + ny k)."""

    def __init__(self, shape, precond=abi.PRECOND_IP, tol=1e-4, max_iter=1000, check_every=16, tile_y=0, seg=0,
                 device="cuda:0"):
        nx, ny, nz = (int(s) for s in shape)
        self.shape = (nx, ny, nz)
        self.n = nx * ny * nz
        self.prm = abi.PpcgParams(nx, ny, nz, precond, tol, max_iter, check_every, tile_y, seg)
        self.device = torch.device(device)
        nb = lib().ppcg_workspace_bytes(nx, ny, nz)
        if nb == 0:
            raise ValueError("bad box size %r" % (shape,))
        self.work = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.nbytes = nb
        self.eps = torch.full((max_iter + 1,), float("nan"), dtype=torch.float64, device=self.device)

    def start(self, b, x, stream=None):
        check("ppcg_start", lib().ppcg_start(C.byref(self.prm), _ptr(b), _ptr(x), _ptr(self.work), self.nbytes,
                                             _ptr(self.eps), _stream(stream)))

    def iterate(self, x, count, stream=None):
        check("ppcg_iterate", lib().ppcg_iterate(C.byref(self.prm), _ptr(x), _ptr(self.work), self.nbytes,
                                                 _ptr(self.eps), count, _stream(stream)))

    def poll(self, stream=None):
        info = abi.PpcgInfo()
        check("ppcg_poll", lib().ppcg_poll(_ptr(self.work), C.byref(info), _stream(stream)))
        return info

    def solve(self, b, x=None, stream=None):
        """Solve in place of x (zeros if None); returns (x, eps history on the host, info).
        A solve that does not converge is returned with info.status = abi.ENOCONV."""
        if x is None:
            x = torch.zeros(self.n, dtype=torch.float64, device=self.device)
        info = abi.PpcgInfo()
        st = lib().ppcg_solve(C.byref(self.prm), _ptr(b), _ptr(x), _ptr(self.work), self.nbytes, _ptr(self.eps),
                              C.byref(info), _stream(stream))
        if st not in (abi.OK, abi.ENOCONV, abi.EBREAKDOWN):
            check("ppcg_solve", st)
        return x, self.eps[:info.iters + 1].cpu().numpy(), info
