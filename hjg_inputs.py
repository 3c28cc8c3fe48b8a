"""Seeded synthetic workloads shared by the tests, the benchmark and the smoke check.

This module only describes problems and draws evaluation states; it holds none of the
method's arithmetic (no estimator, no Hamiltonian, no sampler of the sweep), so both the
CUDA path and the CPU oracle can take their inputs from it.

Evaluation states carry no randomness of the method (Remark 2.3: they may be laid out on a
grid or scattered arbitrarily), so they are drawn here once, in FP64 from numpy's Philox
generator keyed by ``seed ^ 0x504F494E54``, and rounded to FP32; both sides receive the
same FP32 values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

POINT_KEY = 0x504F494E54


@dataclasses.dataclass
class Workload:
    name: str
    game: str
    n: int
    nu: float
    T: float
    M: int
    N: int
    K: int
    radius: float
    seed: int = 0
    speed: tuple = ()

    @property
    def delta(self) -> float:
        """Viscosity of the paper's (delta/2) Laplacian: delta = 2 nu."""
        return 2.0 * self.nu

    @property
    def sigma2(self) -> float:
        return self.delta * self.T

    @property
    def point_samples_per_sweep(self) -> int:
        return self.M * self.N


# The five workloads of the benchmark suite (sizes, viscosities and horizons as stated
# for each game; nu is the viscosity in y = x + sqrt(2 nu t) z).
DUBINS3 = Workload("dubins3_grid16", "dubins3", 3, 0.1, 1.0, 4096, 4096, 10, 0.5)
ROCKETS6 = Workload("rockets6_uniform", "rockets6", 6, 0.05, 2.0, 65536, 65536, 20, 0.3)
ROCKETS45 = Workload("rockets45_gauss", "rockets45", 45, 0.05, 2.0, 262144, 131072, 30, 0.3)
FLOCK = Workload("flock_murmuration", "flock4", 4, 0.02, 1.0, 100000, 16384, 15, 0.2)
# The two further games of the appendix: the relative two-rocket game on a 25^3 grid over
# (x, z) in [-100, 100]^2, theta in [-pi/2, pi/2] (a = 64, g = 32 ft/s^2, capture radius 1.5,
# delta = 0.08, N = 14,000, 12 sweeps), and the double integrator on a 64^2 grid over
# [-2, 2]^2 (target disc of radius 0.25 about the origin, delta = 0.08, N = 8,000, 15 sweeps,
# horizons 0.2, 0.5, 0.8).
ROCKETS_REL3 = Workload("rockets_rel3_grid25", "rockets_rel3", 3, 0.04, 1.0, 15625, 14000, 12, 1.5,
                        speed=(64.0, 32.0))
DOUBLE_INT2 = Workload("double_int2_grid64", "double_int2", 2, 0.04, 0.8, 4096, 8000, 15, 0.25)
DOUBLE_INT2_HORIZONS = (0.2, 0.5, 0.8)
WORKLOADS = {w.name: w for w in (DUBINS3, ROCKETS6, ROCKETS45, FLOCK, ROCKETS_REL3, DOUBLE_INT2)}

# The mixed batch that runs alongside the flock: (workload, states) per instance, all at
# nu = 0.02, T = 1, N = 16,384, 15 sweeps.
MIXED = [(DUBINS3, 1024), (DUBINS3, 65536), (ROCKETS6, 4096), (ROCKETS6, 131072),
         (ROCKETS45, 16384), (ROCKETS45, 262144)]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=(seed ^ POINT_KEY)))


def dubins_grid(m_side: int = 16) -> np.ndarray:
    """m_side^3 grid over [-2,2]^2 x [-pi,pi], endpoints included; index
    m = (i1*m_side + i2)*m_side + i3."""
    a = np.linspace(-2.0, 2.0, m_side)
    th = np.linspace(-math.pi, math.pi, m_side)
    g = np.stack(np.meshgrid(a, a, th, indexing="ij"), axis=-1).reshape(-1, 3)
    return g.astype(np.float32)


def rockets6_points(M: int, seed: int = 0) -> np.ndarray:
    """M states uniform in [-3,3]^4 x [-pi,pi]^2, order (xA, zA, xB, zB, thA, thB)."""
    r = _rng(seed)
    pos = r.uniform(-3.0, 3.0, size=(M, 4))
    ang = r.uniform(-math.pi, math.pi, size=(M, 2))
    return np.concatenate([pos, ang], axis=1).astype(np.float32)


def rockets45_points(M: int, seed: int = 0) -> np.ndarray:
    """M states of 15 planar agents (x_i, z_i, theta_i): positions ~ N(0, 2^2),
    headings uniform in [-pi, pi]."""
    r = _rng(seed)
    pos = r.normal(0.0, 2.0, size=(M, 15, 2))
    ang = r.uniform(-math.pi, math.pi, size=(M, 15, 1))
    return np.concatenate([pos, ang], axis=2).reshape(M, 45).astype(np.float32)


def rockets45_wide_points(M: int, seed: int = 0, half_width: float = 100.0) -> np.ndarray:
    """M states of the 15 planar agents spread as in the paper's 45-D evaluation: positions
    uniform in [-half_width, half_width] per coordinate, headings uniform in [-pi, pi]."""
    r = _rng(seed)
    pos = r.uniform(-half_width, half_width, size=(M, 15, 2))
    ang = r.uniform(-math.pi, math.pi, size=(M, 15, 1))
    return np.concatenate([pos, ang], axis=2).reshape(M, 45).astype(np.float32)


def flock_states(M: int, seed: int = 0, clusters: int = 6, ring: float = 40.0,
                 std: float = 2.4, heading_std: float = 0.3) -> np.ndarray:
    """M starlings (p_x, p_y, p_z, psi) in `clusters` Gaussian flocks spaced on a ring of
    radius `ring` in the horizontal plane; per-axis spread `std` (2.4 puts the median
    nearest-neighbour distance at about 0.2); each flock's mean heading is the ring's
    tangent there, each bird's heading that plus N(0, heading_std^2), wrapped to [-pi, pi)."""
    r = _rng(seed)
    k = np.arange(M) % clusters
    ang = 2.0 * math.pi * k / clusters
    centers = np.stack([ring * np.cos(ang), ring * np.sin(ang), np.zeros(M)], axis=1)
    pos = centers + r.normal(0.0, std, size=(M, 3))
    psi = ang + 0.5 * math.pi + r.normal(0.0, heading_std, size=M)
    psi = (psi + math.pi) % (2.0 * math.pi) - math.pi
    return np.concatenate([pos, psi[:, None]], axis=1).astype(np.float32)


def box_grid(lo, hi, m_side: int) -> np.ndarray:
    """m_side points per axis on the box [lo, hi] (numpy linspace, endpoints included),
    row-major over the axes (last axis fastest)."""
    axes = [np.linspace(a, b, m_side) for a, b in zip(lo, hi)]
    g = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, len(axes))
    return g.astype(np.float32)


def points(w: Workload, M: int | None = None, seed: int | None = None) -> np.ndarray:
    """Evaluation states of workload ``w``.  With M given: the first M states of a grid
    workload, or M states drawn by a scattered workload's recipe (a draw of its own, not a
    prefix of the full set: the recipe draws each coordinate block for all states at once)."""
    seed = w.seed if seed is None else seed
    if w.game == "dubins3":
        x = dubins_grid(16)
        return x if M is None else x[:M].copy()
    if w.game == "rockets_rel3":
        x = box_grid((-100.0, -100.0, -0.5 * math.pi), (100.0, 100.0, 0.5 * math.pi), 25)
        return x if M is None else x[:M].copy()
    if w.game == "double_int2":
        x = box_grid((-2.0, -2.0), (2.0, 2.0), 64)
        return x if M is None else x[:M].copy()
    M = w.M if M is None else M
    if w.game == "rockets6":
        return rockets6_points(M, seed)
    if w.game == "rockets45":
        return rockets45_points(M, seed)
    if w.game == "flock4":
        return flock_states(M, seed)
    raise KeyError(w.game)


def subset_indices(M: int, count: int, seed: int = 1) -> np.ndarray:
    """A seeded, sorted subset of point indices (used for sampled parity at full size)."""
    r = _rng(seed)
    return np.sort(r.choice(M, size=min(count, M), replace=False)).astype(np.int64)


def random_states(M: int, n: int, scale: float = 1.0, seed: int = 0) -> np.ndarray:
    """Generic Gaussian states for unit tests."""
    return (_rng(seed).normal(0.0, scale, size=(M, n))).astype(np.float32)


def spd_matrix(n: int, lo: float = 0.3, hi: float = 1.5, seed: int = 0) -> np.ndarray:
    """A seeded symmetric positive definite matrix with eigenvalues in [lo, hi]."""
    r = _rng(seed)
    q, _ = np.linalg.qr(r.normal(size=(n, n)))
    ev = r.uniform(lo, hi, size=n)
    return (q * ev) @ q.T
