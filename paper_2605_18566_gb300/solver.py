"""Python binding of the C ABI: a thin wrapper that marshals torch tensors (device memory,
streams) into libhjg.so calls.  No arithmetic of the method happens here."""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import HJGError


def _check(lib, ctx, st):
    if st != _lib.HJG_OK:
        msg = lib.hjg_last_error(ctx).decode() if ctx else ""
        raise HJGError(st, msg)


def _stream_handle(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Solver:
    """One game instance of the frozen-coefficient Picard sweep (Algorithm 1).

    game: 'dubins3' | 'rockets6' | 'rockets45' | 'flock4' | 'rockets_rel3' | 'double_int2'
    | 'quadratic' | 'zero_h' (the last two need n, A, x0, d: the closed-form test games);
    nu: viscosity with delta = 2 nu; T: horizon; N: samples per state and sweep;
    K: sweeps run by value_grad.  The keyword options map one to one onto hjg_options and
    hjg_target (tilt, tube, cv, obstacle=(cx, cy, r), precision 'fp32' | 'fp64', variant,
    point_offset, seed, instance, eps, eta, c_min, c_max).
    """

    def __init__(self, game: str, nu: float, T: float, N: int, K: int = 10, *,
                 n: Optional[int] = None, radius: float = 0.5,
                 speed: Optional[Sequence[float]] = None, h_sign: float = 1.0,
                 A=None, x0=None, d: float = 0.0, seed: int = 0, instance: int = 0,
                 tilt: bool = False, eps: float = 0.0, eta: float = -1.0,
                 c_min: float = 0.0, c_max: float = 0.0, block_threads: int = 0,
                 grid_blocks: int = 0, variant: int = -1, point_offset: int = 0,
                 tube: bool = False, cv: bool = False, obstacle: Optional[Sequence[float]] = None,
                 precision: str = "fp32", stream: Optional[torch.cuda.Stream] = None):
        self.lib = _lib.load()
        if n is None:
            n = _lib.GAME_DIMS[game]
        self.n = n
        self.game = game
        dyn = _lib.Dynamics()
        dyn.game = _lib.GAMES[game]
        dyn.n = n
        for i, s in enumerate(speed or []):
            dyn.speed[i] = s
        dyn.h_sign = h_sign
        tgt = _lib.Target()
        tgt.radius = radius
        if A is not None:
            for i, a in enumerate(np.asarray(A, dtype=np.float64).ravel()):
                tgt.A[i] = a
        if x0 is not None:
            for i, a in enumerate(np.asarray(x0, dtype=np.float64).ravel()):
                tgt.x0[i] = a
        tgt.d = d
        if obstacle is not None:   # reach-avoid avoid disc (cx, cy, r) in the plane of dims 0, 1
            cx, cy, r = (float(a) for a in obstacle)
            tgt.obstacle_center[0], tgt.obstacle_center[1] = cx, cy
            tgt.obstacle_radius = r
        opt = _lib.Options()
        opt.N = N; opt.K = K; opt.tilt = 1 if tilt else 0; opt.eps = eps; opt.eta = eta
        opt.c_min = c_min; opt.c_max = c_max; opt.seed = seed; opt.instance = instance
        opt.block_threads = block_threads; opt.grid_blocks = grid_blocks
        opt.variant = variant + 1 if variant >= 0 else 0
        opt.point_offset = point_offset
        opt.tube = 1 if tube else 0
        opt.cv = 1 if cv else 0
        if precision not in ("fp32", "fp64"):
            raise ValueError("precision must be 'fp32' or 'fp64'")
        opt.precision = 1 if precision == "fp64" else 0
        self.opt = opt
        ctx = C.c_void_p()
        torch.cuda.init()
        st = self.lib.hjg_create(C.byref(dyn), C.byref(tgt), nu, T, C.byref(opt), C.byref(ctx))
        if st != _lib.HJG_OK:
            raise HJGError(st, "hjg_create")
        self.ctx = ctx
        self.M = 0
        self.set_stream(stream)

    # ------------------------------------------------------------------ plumbing
    def set_stream(self, stream: Optional[torch.cuda.Stream]):
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _check(self.lib, self.ctx, self.lib.hjg_set_stream(self.ctx, _stream_handle(self.stream)))

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.hjg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ptr(self, t: Optional[torch.Tensor]):
        return C.c_void_p(t.data_ptr()) if t is not None else None

    # ------------------------------------------------------------------ API
    def set_horizons(self, times):
        """Solve at several horizons t_h at once; afterwards every per-state array has
        len(times) * M rows (horizon-major).  An empty list returns to the single T."""
        t = np.ascontiguousarray(np.asarray(times, dtype=np.float64).ravel())
        _check(self.lib, self.ctx, self.lib.hjg_set_horizons(
            self.ctx, t.ctypes.data_as(C.c_void_p) if t.size else None, int(t.size)))
        self.n_horizons = max(1, int(t.size))
        self.M = 0

    def set_points(self, x: torch.Tensor):
        """x: [M, ld] float32 (ld >= n), on the GPU or in host memory."""
        assert x.dtype == torch.float32 and x.dim() == 2 and x.stride(1) == 1
        on_dev = 1 if x.is_cuda else 0
        self.M = 0   # a refused load leaves no states to read back
        _check(self.lib, self.ctx, self.lib.hjg_set_points(
            self.ctx, self._ptr(x), x.shape[0], x.stride(0), on_dev, None))
        self.M = x.shape[0] * getattr(self, "n_horizons", 1)

    def picard_sweep(self, n_sweeps: int, residuals: bool = True):
        """Run n_sweeps sweeps; returns (relative L2 residual, sup-norm) per sweep as numpy,
        or None when residuals=False (asynchronous)."""
        if not residuals:
            _check(self.lib, self.ctx, self.lib.hjg_picard_sweep(self.ctx, n_sweeps, None, None))
            return None
        r = np.zeros(max(n_sweeps, 1)); s = np.zeros(max(n_sweeps, 1))
        st = self.lib.hjg_picard_sweep(self.ctx, n_sweeps, r.ctypes.data_as(C.c_void_p),
                                       s.ctypes.data_as(C.c_void_p))
        if st not in (_lib.HJG_OK, _lib.HJG_ENONFINITE):
            _check(self.lib, self.ctx, st)
        self.last_status = st
        return r[:n_sweeps], s[:n_sweeps]

    def residual_parts(self, n_sweeps: int) -> np.ndarray:
        """[n_sweeps, 3] (sum dv^2, sum v^2, max |dv|) of the last picard_sweep call."""
        out = np.zeros((max(n_sweeps, 1), 3))
        _check(self.lib, self.ctx, self.lib.hjg_get_residual_parts(self.ctx, out.ctypes.data_as(C.c_void_p)))
        return out[:n_sweeps]

    def certify(self, e0: float = 0.0, q: float = 0.0, delta_p: float = 0.05, ess_min: float = 0.0):
        """Conservative certificate of the current iterate (Cor. 2.9): returns (labels int8
        [M] with +1 SAFE / -1 UNSAFE / 0 UNDETERMINED, band half-widths [M], Monte-Carlo
        standard errors [M], counts (safe, unsafe, undetermined)), tensors on the GPU."""
        M = self.M
        lab = torch.empty(M, dtype=torch.int8, device="cuda")
        band = torch.empty(M, dtype=torch.float32, device="cuda")
        se = torch.empty(M, dtype=torch.float32, device="cuda")
        cnt = np.zeros(3, dtype=np.int64)
        _check(self.lib, self.ctx, self.lib.hjg_certify(
            self.ctx, e0, q, delta_p, ess_min, self._ptr(lab), self._ptr(band), self._ptr(se),
            cnt.ctypes.data_as(C.c_void_p), 1))
        return lab, band, se, tuple(int(x) for x in cnt)

    def get_state(self, device: bool = True):
        M, n = self.M, self.n
        kw = dict(device="cuda") if device else {}
        v = torch.empty(M, dtype=torch.float64, **kw)
        p = torch.empty(M, n, dtype=torch.float32, **kw)
        c = torch.empty(M, dtype=torch.float32, **kw)
        ess = torch.empty(M, dtype=torch.float32, **kw)
        _check(self.lib, self.ctx, self.lib.hjg_get_state(
            self.ctx, self._ptr(v), self._ptr(p), n, self._ptr(c), self._ptr(ess),
            1 if device else 0))
        return {"v": v, "p": p, "c": c, "ess": ess}

    def set_state(self, v=None, p=None, c=None, next_sweep: int = 0):
        ts = [t for t in (v, p, c) if t is not None]
        dev = ts[0].is_cuda if ts else True
        if p is not None:
            assert p.dtype == torch.float32 and p.stride(1) == 1
        _check(self.lib, self.ctx, self.lib.hjg_set_state(
            self.ctx, self._ptr(v), self._ptr(p), p.stride(0) if p is not None else self.n,
            self._ptr(c), next_sweep, 1 if dev else 0))

    def history(self, n_sweeps: int) -> torch.Tensor:
        out = torch.empty(n_sweeps + 1, self.M, dtype=torch.float64, device="cuda")
        _check(self.lib, self.ctx, self.lib.hjg_get_history(self.ctx, self._ptr(out), 1))
        return out

    def value_grad(self, x: torch.Tensor, v_out=None, grad_out=None):
        """Algorithm 1 end to end: set points, run K sweeps (or stop at eps), copy out.
        Host tensors in -> host tensors out (copies inside the call); device -> device."""
        assert x.dtype == torch.float32 and x.dim() == 2 and x.stride(1) == 1
        M = x.shape[0] * getattr(self, "n_horizons", 1)   # rows of the outputs
        dev = x.is_cuda
        kw = dict(device=x.device) if dev else dict(pin_memory=False)
        if v_out is None:
            v_out = torch.empty(M, dtype=torch.float64, **kw)
        if grad_out is None:
            grad_out = torch.empty(M, self.n, dtype=torch.float32, **kw)
        K = self.opt.K
        r = np.full(max(K, 1), np.nan)
        self.M = 0
        st = self.lib.hjg_value_grad(self.ctx, self._ptr(x), x.shape[0], x.stride(0), 1 if dev else 0,
                                     self._ptr(v_out), self._ptr(grad_out), grad_out.stride(0),
                                     r.ctypes.data_as(C.c_void_p), None)
        if st not in (_lib.HJG_OK, _lib.HJG_ENONFINITE):
            _check(self.lib, self.ctx, st)
        self.M = M
        self.last_status = st
        return v_out, grad_out, r[:K]

    def warm_start(self, p0: torch.Tensor, v0: Optional[torch.Tensor] = None):
        """Replace the initial iterate by (v0, p0) and set c = Gamma(p0) (hjg_warm_start)."""
        assert p0.dtype == torch.float32 and p0.stride(1) == 1 and p0.is_cuda
        if v0 is not None:
            assert v0.dtype == torch.float64 and v0.is_cuda
        _check(self.lib, self.ctx, self.lib.hjg_warm_start(
            self.ctx, self._ptr(v0), self._ptr(p0), p0.stride(0), 1))

    def warm_start_delta(self, d: torch.Tensor):
        """Initial iterate (l, Dl) plus a learned correction d [M, >= n + 1] (column 0 the
        value, 1..n the gradient), c = Gamma(Dv) (hjg_warm_start_delta)."""
        assert d.is_cuda and d.dtype == torch.float32 and d.stride(1) == 1 and d.shape[1] >= self.n + 1
        _check(self.lib, self.ctx, self.lib.hjg_warm_start_delta(self.ctx, self._ptr(d), d.stride(0)))

    def state_delta(self) -> torch.Tensor:
        """[M, n + 1] FP32: (v - l(x), Dv - Dl(x)) of the current iterate (hjg_get_state_delta)."""
        out = torch.empty(self.M, self.n + 1, dtype=torch.float32, device="cuda")
        _check(self.lib, self.ctx, self.lib.hjg_get_state_delta(self.ctx, self._ptr(out), out.stride(0)))
        return out

    def frame_features(self) -> torch.Tensor:
        """45-D game: [M, 56] invariant-frame inputs of the loaded states (hjg_frame_features)."""
        out = torch.empty(self.M, 56, dtype=torch.float32, device="cuda")
        _check(self.lib, self.ctx, self.lib.hjg_frame_features(self.ctx, self._ptr(out), out.stride(0)))
        return out

    def frame_targets(self) -> torch.Tensor:
        """45-D game: [M, 43] invariant-frame correction of the current iterate (hjg_frame_targets)."""
        out = torch.empty(self.M, 43, dtype=torch.float32, device="cuda")
        _check(self.lib, self.ctx, self.lib.hjg_frame_targets(self.ctx, self._ptr(out), out.stride(0)))
        return out

    def warm_start_frame(self, pred: torch.Tensor, positions_only: bool = True):
        """45-D game: warm start from an invariant-frame prediction [M, >= 43]
        (hjg_warm_start_frame); by default only the position rows of Dv take the correction."""
        assert pred.is_cuda and pred.dtype == torch.float32 and pred.stride(1) == 1 and pred.shape[1] >= 43
        _check(self.lib, self.ctx, self.lib.hjg_warm_start_frame(self.ctx, self._ptr(pred), pred.stride(0),
                                                                 1 if positions_only else 0))

    def autotune(self, max_states: int = 0) -> dict:
        """Pick the fastest sweep launch variant on the loaded states (see hjg_autotune)."""
        v = C.c_int32(); t = C.c_int32(); ms = C.c_double()
        _check(self.lib, self.ctx, self.lib.hjg_autotune(self.ctx, max_states, C.byref(v),
                                                         C.byref(t), C.byref(ms)))
        return {"variant": v.value, "threads": t.value, "ms": ms.value}

    def diagnostics(self) -> dict:
        d = _lib.Diag()
        _check(self.lib, self.ctx, self.lib.hjg_get_diagnostics(self.ctx, C.byref(d)))
        return {f: getattr(d, f) for f, _ in _lib.Diag._fields_}


class Surrogate:
    """The BF16 tensor-core MLP of hjg_mlp_*: n_in -> width x3 -> n_out, SiLU."""

    def __init__(self, n_in: int, n_out: int, width: int = 256, seed: int = 0,
                 stream: Optional[torch.cuda.Stream] = None):
        self.lib = _lib.load()
        self.n_in, self.n_out, self.width = n_in, n_out, width
        m = C.c_void_p()
        torch.cuda.init()
        st = self.lib.hjg_mlp_create(n_in, n_out, width, seed, C.byref(m))
        if st:
            raise HJGError(st, "hjg_mlp_create")
        self.m = m
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.lib.hjg_mlp_set_stream(self.m, _stream_handle(self.stream))
        self.n_params = int(self.lib.hjg_mlp_num_params(self.m))

    def close(self):
        if getattr(self, "m", None):
            self.lib.hjg_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        st = self.lib.hjg_mlp_get_params(self.m, out.ctypes.data_as(C.c_void_p), 0)
        if st:
            raise HJGError(st, "hjg_mlp_get_params")
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        st = self.lib.hjg_mlp_set_params(self.m, p.ctypes.data_as(C.c_void_p), 0)
        if st:
            raise HJGError(st, "hjg_mlp_set_params")

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        assert x.is_cuda and x.dtype == torch.float32 and x.stride(1) == 1
        out = torch.empty(x.shape[0], self.n_out, dtype=torch.float32, device=x.device)
        st = self.lib.hjg_mlp_forward(self.m, C.c_void_p(x.data_ptr()), x.stride(0), x.shape[0],
                                      C.c_void_p(out.data_ptr()), self.n_out)
        if st:
            raise HJGError(st, "hjg_mlp_forward")
        return out

    def input_grad(self, x: torch.Tensor, j: int = 0) -> torch.Tensor:
        """d output_j / d input at each row of x ([B, n_in])."""
        assert x.is_cuda and x.dtype == torch.float32 and x.stride(1) == 1
        gx = torch.empty(x.shape[0], self.n_in, dtype=torch.float32, device=x.device)
        st = self.lib.hjg_mlp_input_grad(self.m, C.c_void_p(x.data_ptr()), x.stride(0), x.shape[0], j,
                                         C.c_void_p(gx.data_ptr()), self.n_in)
        if st:
            raise HJGError(st, "hjg_mlp_input_grad")
        return gx

    def gradients(self, x: torch.Tensor, y: torch.Tensor):
        loss = C.c_double()
        g = np.zeros(self.n_params, dtype=np.float32)
        st = self.lib.hjg_mlp_gradients(self.m, C.c_void_p(x.data_ptr()), x.stride(0),
                                        C.c_void_p(y.data_ptr()), y.stride(0), x.shape[0],
                                        C.byref(loss), g.ctypes.data_as(C.c_void_p))
        if st:
            raise HJGError(st, "hjg_mlp_gradients")
        return loss.value, g

    def train_step(self, x: torch.Tensor, y: torch.Tensor, lr: float, want_loss: bool = True):
        loss = C.c_double()
        st = self.lib.hjg_mlp_train_step(self.m, C.c_void_p(x.data_ptr()), x.stride(0),
                                         C.c_void_p(y.data_ptr()), y.stride(0), x.shape[0],
                                         lr, C.byref(loss) if want_loss else None)
        if st:
            raise HJGError(st, "hjg_mlp_train_step")
        return loss.value if want_loss else None

    def fit_scaling(self, x: torch.Tensor, y: torch.Tensor):
        """Standardise inputs and targets by their per-feature mean and std (hjg_mlp_fit_scaling)."""
        st = self.lib.hjg_mlp_fit_scaling(self.m, C.c_void_p(x.data_ptr()), x.stride(0),
                                          C.c_void_p(y.data_ptr()), y.stride(0), x.shape[0])
        if st:
            raise HJGError(st, "hjg_mlp_fit_scaling")

    def scaling(self) -> np.ndarray:
        out = np.zeros(2 * (self.n_in + self.n_out), dtype=np.float32)
        st = self.lib.hjg_mlp_get_scaling(self.m, out.ctypes.data_as(C.c_void_p))
        if st:
            raise HJGError(st, "hjg_mlp_get_scaling")
        return out

    def save(self, path: str) -> None:
        """Write the network (FP32 master parameters, feature standardisation, shape) to an
        .npz file; the optimiser state is not saved (a loaded network predicts, and training
        it further starts Adam afresh)."""
        np.savez(path, params=self.params(), scaling=self.scaling(),
                 shape=np.array([self.n_in, self.n_out, self.width], dtype=np.int64))

    @classmethod
    def load(cls, path: str, stream: Optional[torch.cuda.Stream] = None) -> "Surrogate":
        """A network written by save(); its predictions equal the saved network's."""
        with np.load(path) as f:
            n_in, n_out, width = (int(v) for v in f["shape"])
            s = cls(n_in, n_out, width, stream=stream)
            s.set_params(f["params"])
            s.set_scaling(f["scaling"])
        return s

    def set_scaling(self, sc) -> None:
        sc = np.ascontiguousarray(np.asarray(sc, dtype=np.float32).ravel())
        st = self.lib.hjg_mlp_set_scaling(self.m, sc.ctypes.data_as(C.c_void_p))
        if st:
            raise HJGError(st, "hjg_mlp_set_scaling")

    def fit(self, x: torch.Tensor, y: torch.Tensor, epochs: int, batch: int = 4096,
            lr: float = 1e-3, lr_final: float = 1e-5, standardize: bool = True):
        """Adam over contiguous minibatches of (x, y) (shuffle the rows beforehand), with
        the learning rate decayed geometrically from lr to lr_final, after fitting the
        feature standardisation to (x, y) when `standardize` (hjg_mlp_fit: the loop runs in
        the library); returns the loss (on standardised targets) of each epoch's last
        minibatch."""
        hist = np.zeros(epochs, dtype=np.float64)
        st = self.lib.hjg_mlp_fit(self.m, C.c_void_p(x.data_ptr()), x.stride(0),
                                  C.c_void_p(y.data_ptr()), y.stride(0), x.shape[0], epochs, batch,
                                  lr, lr_final, 1 if standardize else 0, hist.ctypes.data_as(C.c_void_p))
        if st:
            raise HJGError(st, "hjg_mlp_fit")
        return [float(h) for h in hist]


class Batch:
    """Several Solver instances advanced by one CUDA-graph launch (hjg_batch_*)."""

    def __init__(self, solvers):
        self.lib = _lib.load()
        self.solvers = list(solvers)
        b = C.c_void_p()
        st = self.lib.hjg_batch_create(C.byref(b))
        if st:
            raise HJGError(st, "hjg_batch_create")
        self.b = b
        for s in self.solvers:
            st = self.lib.hjg_batch_add(self.b, s.ctx)
            if st:
                raise HJGError(st, "hjg_batch_add")

    def run(self, n_sweeps: int, stream: Optional[torch.cuda.Stream] = None):
        """Returns (residuals [instances, n_sweeps] numpy, device ms)."""
        r = np.zeros((len(self.solvers), n_sweeps))
        ms = C.c_double()
        st = self.lib.hjg_batch_run(self.b, n_sweeps, r.ctypes.data_as(C.c_void_p),
                                    _stream_handle(stream), C.byref(ms))
        if st not in (_lib.HJG_OK, _lib.HJG_ENONFINITE):
            raise HJGError(st, self.lib.hjg_batch_last_error(self.b).decode())
        return r, ms.value

    def close(self):
        if getattr(self, "b", None):
            self.lib.hjg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def flock_neighbours(states: torch.Tensor, k: int = 7):
    """7 nearest neighbours of each agent and their circular mean heading (device)."""
    lib = _lib.load()
    M = states.shape[0]
    idx = torch.empty(M, k, dtype=torch.int32, device=states.device)
    psibar = torch.empty(M, dtype=torch.float32, device=states.device)
    st = lib.hjg_flock_neighbours(C.c_void_p(states.data_ptr()), M, states.stride(0), k,
                                  C.c_void_p(idx.data_ptr()), C.c_void_p(psibar.data_ptr()),
                                  _stream_handle(None))
    if st:
        raise HJGError(st, "hjg_flock_neighbours")
    return idx, psibar


def topology(v: torch.Tensor, smooth_cells: float = 1.5):
    """Topology markers of {v <= 0} on slices v [H, m, m] (FP64, device): returns
    (markers int32 [H, 3] = (n_comp, beta_1, chi), events int32 [H] (HJG_EVENT_* bits),
    smoothed field [H, m, m], component labels [H, m, m]) -- hjg_topology."""
    lib = _lib.load()
    assert v.dtype == torch.float64 and v.dim() == 3 and v.shape[1] == v.shape[2] and v.is_cuda
    v = v.contiguous()
    H, m = v.shape[0], v.shape[1]
    markers = np.zeros((H, 3), dtype=np.int32)
    events = np.zeros(H, dtype=np.int32)
    sm = torch.empty_like(v)
    lab = torch.empty(H, m, m, dtype=torch.int32, device=v.device)
    st = lib.hjg_topology(C.c_void_p(v.data_ptr()), H, m, smooth_cells, C.c_void_p(sm.data_ptr()),
                          markers.ctypes.data_as(C.c_void_p), events.ctypes.data_as(C.c_void_p),
                          C.c_void_p(lab.data_ptr()), _stream_handle(None))
    if st:
        raise HJGError(st, "hjg_topology")
    return markers, events, sm, lab


def philox_blocks(ctr: torch.Tensor, key: torch.Tensor) -> torch.Tensor:
    """Device Philox4x32-10: ctr int32/uint32 [K,4], key [K,2] (CUDA tensors)."""
    lib = _lib.load()
    out = torch.empty_like(ctr)
    st = lib.hjg_philox_blocks(C.c_void_p(ctr.data_ptr()), C.c_void_p(key.data_ptr()),
                               C.c_void_p(out.data_ptr()), ctr.shape[0],
                               _stream_handle(None))
    if st:
        raise HJGError(st, "hjg_philox_blocks")
    return out


def sample_normals(n: int, seed: int, instance: int, point: int, sweep: int,
                   n_samples: int) -> torch.Tensor:
    lib = _lib.load()
    out = torch.empty(n_samples, n, dtype=torch.float32, device="cuda")
    st = lib.hjg_sample_normals(n, seed, instance, point, sweep, n_samples,
                                C.c_void_p(out.data_ptr()), _stream_handle(None))
    if st:
        raise HJGError(st, "hjg_sample_normals")
    return out


def microbench(op: str, iters: int = 4096):
    """Throughput of one instruction class (ops/s) and the launch time (ms)."""
    lib = _lib.load()
    r = C.c_double(); ms = C.c_double()
    st = lib.hjg_microbench(_lib.MICROBENCH[op], iters, C.byref(r), C.byref(ms))
    if st:
        raise HJGError(st, "hjg_microbench")
    return r.value, ms.value
