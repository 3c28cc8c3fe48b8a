"""Oracle for the topology markers of the zero sublevel set on 2-D value slices
(Appendix D, phase-transition markers of the murmuration study).

Test infrastructure only: the tests, the smoke check and the benchmark's CPU leg use it;
the product path never imports it.

Per slice: optional Gaussian smoothing (scipy.ndimage.gaussian_filter over the two slice
axes, truncate 4, mode "reflect"), the set {v <= 0} labelled with 4-connectivity and its
complement with 8-connectivity (scipy.ndimage.label), n_comp = number of set components,
beta_1 = number of complement components that touch no border cell, chi = n_comp - beta_1;
events against the previous slice: chi drop below -0.5 (vacuole nucleation), beta_1 from 0
to >= 1 (cordon formation), n_comp growth (fragmentation).
"""
from __future__ import annotations

import numpy as np

VACUOLE, CORDON, FRAGMENTATION = 1, 2, 4
_CROSS = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]])
_SQUARE = np.ones((3, 3), dtype=int)


def smooth(v, cells):
    """Gaussian smoothing of each slice of v [H, m, m] by `cells` grid cells."""
    from scipy import ndimage
    v = np.asarray(v, dtype=np.float64)
    if cells <= 0:
        return v.copy()
    return ndimage.gaussian_filter(v, sigma=(0.0, cells, cells), mode="reflect", truncate=4.0)


def markers(v, cells=1.5):
    """Returns (markers [H, 3] = (n_comp, beta_1, chi), events [H], smoothed field)."""
    from scipy import ndimage
    f = smooth(v, cells)
    H = f.shape[0]
    out = np.zeros((H, 3), dtype=np.int64)
    for h in range(H):
        fg = f[h] <= 0.0
        _, n = ndimage.label(fg, structure=_CROSS)
        bl, nb = ndimage.label(~fg, structure=_SQUARE)
        edge = np.unique(np.concatenate([bl[0], bl[-1], bl[:, 0], bl[:, -1]]))
        holes = nb - int(np.count_nonzero(edge))
        out[h] = (n, holes, n - holes)
    ev = np.zeros(H, dtype=np.int64)
    for h in range(1, H):
        a, b = out[h - 1], out[h]
        ev[h] = (VACUOLE if b[2] - a[2] < -0.5 else 0) | (CORDON if b[1] >= 1 and a[1] == 0 else 0) | \
            (FRAGMENTATION if b[0] > a[0] else 0)
    return out, ev, f
