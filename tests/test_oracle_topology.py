"""Pins for the oracle's topology markers (Appendix D): shapes whose topology is known,
a breadth-first flood fill written here on random grids, the smoothing weights on an
impulse (including the border reflection), and the event rules on a scripted sequence."""
import math
from collections import deque

import numpy as np
import pytest

pytest.importorskip("scipy")
from oracle import topology  # noqa: E402

m = 64
I, J = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")


def disc(ci, cj, r):
    return np.hypot(I - ci, J - cj) - r


def annulus(ci, cj, r0, r1):
    d = np.hypot(I - ci, J - cj)
    return np.maximum(r0 - d, d - r1)


@pytest.mark.parametrize("field,expect", [
    (disc(32, 32, 10), (1, 0, 1)),
    (annulus(32, 32, 8, 16), (1, 1, 0)),
    (np.minimum(disc(20, 20, 6), disc(44, 44, 6)), (2, 0, 2)),
    (np.minimum(annulus(32, 32, 12, 20), disc(32, 32, 5)), (2, 1, 1)),
    (annulus(0, 0, 10, 20), (1, 0, 1)),            # the "hole" reaches the border
    (np.ones((m, m)), (0, 0, 0)),
    (-np.ones((m, m)), (1, 0, 1)),
], ids=["disc", "annulus", "two-discs", "annulus-island", "border-annulus", "empty", "full"])
def test_known_shapes(field, expect):
    mk, ev, _ = topology.markers(field[None], cells=0.0)
    assert tuple(mk[0]) == expect


def flood(mask, nbrs):
    seen = np.zeros_like(mask, dtype=bool)
    comps = []
    for i in range(mask.shape[0]):
        for j in range(mask.shape[1]):
            if mask[i, j] and not seen[i, j]:
                q, cells = deque([(i, j)]), []
                seen[i, j] = True
                while q:
                    a, b = q.popleft()
                    cells.append((a, b))
                    for da, db in nbrs:
                        x, y = a + da, b + db
                        if 0 <= x < mask.shape[0] and 0 <= y < mask.shape[1] and mask[x, y] and not seen[x, y]:
                            seen[x, y] = True
                            q.append((x, y))
                comps.append(cells)
    return comps


def test_random_grids_against_flood_fill():
    four = [(1, 0), (-1, 0), (0, 1), (0, -1)]
    eight = four + [(1, 1), (1, -1), (-1, 1), (-1, -1)]
    rng = np.random.default_rng(3)
    v = rng.normal(size=(40, 12, 12)) + rng.uniform(-0.8, 0.8, size=(40, 1, 1))
    mk, _, _ = topology.markers(v, cells=0.0)
    for h in range(len(v)):
        fg = v[h] <= 0
        n = len(flood(fg, four))
        holes = sum(1 for c in flood(~fg, eight)
                    if not any(a in (0, 11) or b in (0, 11) for a, b in c))
        assert tuple(mk[h]) == (n, holes, n - holes), h


def test_smoothing_weights_on_impulses():
    s = 1.5
    r = int(4 * s + 0.5)
    w = np.exp(-0.5 * np.arange(-r, r + 1) ** 2 / s**2)
    w /= w.sum()
    v = np.zeros((1, 32, 32)); v[0, 16, 16] = 1.0
    f = topology.smooth(v, s)
    np.testing.assert_allclose(f[0, 16, 16 - r:16 + r + 1], w[r] * w, rtol=1e-12, atol=1e-18)
    np.testing.assert_allclose(f[0].sum(), 1.0, rtol=1e-12)
    e = np.zeros((1, 32, 32)); e[0, 0, 16] = 1.0      # the border cell reflects onto itself
    g = topology.smooth(e, s)
    col = np.zeros(32)
    for k in range(-r, r + 1):
        i = k if k >= 0 else -k - 1
        col[i] += w[k + r]
    np.testing.assert_allclose(g[0, :, 16], col * w[r], rtol=1e-12, atol=1e-18)


def test_event_rules_on_a_sequence():
    seq = np.stack([disc(32, 32, 10), annulus(32, 32, 6, 16), annulus(32, 32, 6, 16),
                    np.minimum(disc(16, 16, 5), disc(48, 48, 5)), disc(32, 32, 10)])
    mk, ev, _ = topology.markers(seq, cells=0.0)
    assert [tuple(x) for x in mk] == [(1, 0, 1), (1, 1, 0), (1, 1, 0), (2, 0, 2), (1, 0, 1)]
    V, C, F = topology.VACUOLE, topology.CORDON, topology.FRAGMENTATION
    assert list(ev) == [0, V | C, 0, F, V]
