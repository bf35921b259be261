"""Host-side helpers shared by bench.py and the tests (no arithmetic of the method)."""
import numpy as np


def cell_centres_of(tree):
    """Cell centres (ncell, 3) in the device tree's cell order, from its coordinate tables."""
    tab = tree.tables()
    l = tab["lvl"].cpu().numpy().astype(np.int64)
    xyz = np.stack([tab["ix"].cpu().numpy(), tab["iy"].cpu().numpy(), tab["iz"].cpu().numpy()], axis=1)
    c = np.arange(8)
    off = np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], axis=1)
    dx = np.ldexp(1.0, -l)
    return ((xyz[:, None, :] * 2.0 + off[None] + 0.5) * dx[:, None, None]).reshape(-1, 3)
