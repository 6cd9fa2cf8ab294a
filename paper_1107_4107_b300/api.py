"""Python face of libarnold: an ensemble of trajectories of Eqs. 1-2 on the GPU.

    ens = ArnoldEnsemble(n=2048 * 2048, precision="fp64")
    ens.init_grid(G=2048, E=400.0)      # 2-D slice of initial actions (Sec. IV)
    ens.iterate(10_000)                 # composite steps of the 6th-order map (Sec. III)
    chi = ens.indicator("chi")          # FTLE per trajectory (numpy, host)

Every step runs in the CUDA library; this module only marshals arguments.
Device buffers (torch CUDA tensors) are passed by pointer; host buffers are
numpy arrays.  torch is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import _lib
from ._lib import ArnoldError, check  # noqa: F401  (re-exported)
from .params import paper_h


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr_kind(a):
    """(pointer, ptr_kind) of a numpy array or a contiguous torch CUDA tensor."""
    if a is None:
        return None, _lib.HOST
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), (_lib.DEVICE if a.is_cuda else _lib.HOST)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data), _lib.HOST


def _dtype_name(a) -> str:
    return str(a.dtype).split(".")[-1]


def _buf(a, count: int, dtypes, what: str, device: int, kind=None):
    """(pointer, ptr_kind) of a caller buffer that the library reads or writes
    as `count` elements of one of `dtypes`, checked first: the C ABI takes bare
    pointers, so a short, mistyped or foreign-device buffer would be accessed
    out of bounds.  A torch CUDA tensor must live on the context's `device`;
    kind (_lib.HOST or _lib.DEVICE) is required where the call fixes it."""
    p, k = _ptr_kind(a)
    n = a.numel() if _is_torch(a) else a.size
    if n != count or _dtype_name(a) not in dtypes:
        raise ValueError(f"{what}: expected {count} elements of {'/'.join(dtypes)}, "
                         f"got {n} of {_dtype_name(a)}")
    if k == _lib.DEVICE and a.device.index != device:
        raise ValueError(f"{what}: tensor is on cuda:{a.device.index}, the context on cuda:{device}")
    if kind is not None and k != kind:
        raise ValueError(f"{what} must be {'device' if kind == _lib.DEVICE else 'host'} memory")
    return p, k


class ArnoldEnsemble:
    """n independent trajectories held on one GPU (library-owned device memory).

    precision: "fp64" (FP64 accuracy), "df64f" (double-float state, kicks and
    tangent with a ~3e-10 sincos on the FP32 pipes: the compensated mode for
    long runs), "df64" (the same with an accurate sincos) or "fp32c"
    (compensated state updates, FP32 forces and tangent: short horizons);
    scheme: "yoshida6a", "triplejump6" or "leapfrog2"."""

    def __init__(self, n: int, eps: float = 1.0, h: float | None = None, scheme: str = "yoshida6a",
                 precision: str = "fp64", tangent: bool = True, renorm_every: int = 100, window: int = 0,
                 kappa: float = 10.0, device: int = 0, stream=None, block_size: int = 0, launch_steps: int = 0,
                 megno: bool = False):
        L = _lib.lib()
        self.n = int(n)
        self.params = _lib.Params(eps, paper_h() if h is None else h, _lib.SCHEMES[scheme],
                                  _lib.PRECISIONS[precision], int(bool(tangent)), renorm_every, window, kappa,
                                  block_size, launch_steps, int(bool(megno)), 0)
        if stream is None:
            stream_ptr = None
            try:
                import torch
                if torch.cuda.is_available():
                    stream_ptr = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
            except ImportError:
                pass
        else:
            stream_ptr = ctypes.c_void_p(stream)
        self._stream = stream_ptr
        handle = ctypes.c_void_p()
        check(L.arnold_create(ctypes.byref(self.params), self.n, device, stream_ptr, ctypes.byref(handle)),
              "arnold_create")
        self._h = handle
        self.device = device

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().arnold_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state --
    def set_state(self, X, P, W=None):
        """X, P: [3][n] f64 (numpy host, or torch CUDA); W: [6][n] or None."""
        px, kx = _ptr_kind(X)
        pp, kp = _ptr_kind(P)
        pw, kw = _ptr_kind(W)
        if kx != kp or (W is not None and kw != kx):
            raise ValueError("X, P, W must all be host or all device")
        for a, rows in ((X, 3), (P, 3), (W, 6)):
            if a is not None and (tuple(a.shape) != (rows, self.n) or str(a.dtype).split(".")[-1] != "float64"):
                raise ValueError(f"expected float64 [{rows}][{self.n}]")
            if a is not None:
                _buf(a, rows * self.n, ("float64",), "set_state", self.device)
        check(_lib.lib().arnold_set_state(self._h, px, pp, pw, kx), "arnold_set_state")

    def init_grid(self, G: int, E: float, seed: int = 0, row0: int = 0, raw_out=None):
        """Grid-slice initial conditions generated on the device (Sec. IV);
        raw_out: None or a CUDA float64 tensor [6][n] for the generated X, P."""
        pr = None if raw_out is None else \
            _buf(raw_out, 6 * self.n, ("float64",), "raw_out", self.device, _lib.DEVICE)[0]
        check(_lib.lib().arnold_init_grid(self._h, G, row0, E, seed, pr), "arnold_init_grid")

    def set_state_shell(self, X, Pdir, mode: int, E: float):
        """Fixed-energy initial momenta (Sec. IV): mode 1 scales unit directions
        Pdir to the shell, mode 2 takes (p_x, p_y) and sets p_z from the energy."""
        px, kx = _buf(X, 3 * self.n, ("float64",), "X", self.device)
        pp, kp = _buf(Pdir, 3 * self.n, ("float64",), "P", self.device)
        if kx != kp:
            raise ValueError("X and P must both be host or both device")
        check(_lib.lib().arnold_set_state_shell(self._h, px, pp, int(mode), float(E), kx), "arnold_set_state_shell")

    def init_sphere(self, E: float, seed: int = 0, cos_range=(-1.0, 1.0), phi_range=(0.0, 2 * math.pi),
                    offset: int = 0):
        """Ensemble uniform over (a patch of) the momentum sphere S and over the
        torus (Sec. IV, Figs. 2-3), drawn on the device (arnold_init_sphere)."""
        check(_lib.lib().arnold_init_sphere(self._h, float(E), int(seed), int(offset), float(cos_range[0]),
                                            float(cos_range[1]), float(phi_range[0]), float(phi_range[1])),
              "arnold_init_sphere")

    def init_gaussian(self, E: float, center, sigma: float = 0.01, seed: int = 0, offset: int = 0) -> int:
        """Gaussian cloud in (p_x, p_y) about `center`, p_z from the energy (Fig. 4),
        drawn on the device; draws without a real p_z are skipped, so the ensemble
        holds the first n draws that have one.  Returns the number of draws
        examined."""
        drawn = _lib.i64()
        check(_lib.lib().arnold_init_gaussian(self._h, float(E), float(center[0]), float(center[1]), float(sigma),
                                              int(seed), int(offset), ctypes.byref(drawn)), "arnold_init_gaussian")
        return drawn.value

    def track_patch(self, cos_lo: float, cos_hi: float, phi_lo: float, phi_hi: float):
        check(_lib.lib().arnold_track_patch(self._h, cos_lo, cos_hi, phi_lo, phi_hi), "arnold_track_patch")

    def velocity_histogram(self, n_cos: int, n_phi: int, patch=(-1.0, 1.0, 0.0, 2 * math.pi), filtered: bool = False,
                           out=None, accumulate: bool = False):
        """Counts of the direction of V on the momentum sphere (F of Sec. IV)."""
        if out is None:
            out = np.zeros((n_cos, n_phi), dtype=np.uint64)
        po, ko = _buf(out, int(n_cos) * int(n_phi), ("uint64", "int64"), "histogram", self.device)
        check(_lib.lib().arnold_velocity_histogram(self._h, n_cos, n_phi, *[float(v) for v in patch], int(filtered), po,
                                                   ko, int(accumulate)), "arnold_velocity_histogram")
        return out

    def set_snapshots(self, v_snap=None):
        """Record V of window w into v_snap[w - 1] (a torch CUDA float64 tensor
        [k][3][n], kept alive by the caller) as the kernels close windows; None
        disables."""
        if v_snap is None:
            check(_lib.lib().arnold_set_snapshots(self._h, None, 0), "arnold_set_snapshots")
            self._snap = None
            return
        if not _is_torch(v_snap) or not v_snap.is_cuda or v_snap.dtype != __import__("torch").float64 \
                or v_snap.dim() != 3 or tuple(v_snap.shape[1:]) != (3, self.n) or not v_snap.is_contiguous():
            raise ValueError(f"v_snap must be a contiguous CUDA float64 tensor [k][3][{self.n}]")
        check(_lib.lib().arnold_set_snapshots(self._h, ctypes.c_void_p(v_snap.data_ptr()), int(v_snap.shape[0])),
              "arnold_set_snapshots")
        self._snap = v_snap

    def iterate(self, n_steps: int):
        check(_lib.lib().arnold_iterate(self._h, int(n_steps)), "arnold_iterate")

    @property
    def steps(self) -> int:
        return _lib.lib().arnold_steps_done(self._h)

    @property
    def launches(self) -> int:
        return _lib.lib().arnold_launch_count(self._h)

    @property
    def time(self) -> float:
        return self.steps * self.params.h

    def sync(self):
        check(_lib.lib().arnold_sync(self._h), "arnold_sync")

    # -- read-out --
    def indicator(self, kind: str, out=None):
        """Indicator `kind` (see _lib.IND) into `out` (numpy host array, torch CUDA
        tensor) or a new numpy array."""
        rows = _lib.IND_SHAPE[kind]
        dtype = np.uint8 if kind in ("class", "left") else np.float64
        if out is None:
            out = np.empty((rows, self.n) if rows > 1 else (self.n,), dtype=dtype)
        po, ko = _buf(out, rows * self.n, (np.dtype(dtype).name,), f"indicator({kind})", self.device)
        check(_lib.lib().arnold_indicator(self._h, _lib.IND[kind], po, ko), f"arnold_indicator({kind})")
        return out

    def stats(self) -> dict:
        s = _lib.Stats()
        check(_lib.lib().arnold_stats_compute(self._h, ctypes.byref(s)), "arnold_stats_compute")
        return stats_dict(s)

    def stats_arrays(self, chi, dE, P, t: float, kappa: float = 10.0) -> dict:
        """Statistics of caller device arrays (torch CUDA float64)."""
        s = _lib.Stats()
        n = int(chi.shape[0])
        pc, _ = _buf(chi, n, ("float64",), "chi", self.device, _lib.DEVICE)
        pd, _ = _buf(dE, n, ("float64",), "dE", self.device, _lib.DEVICE)
        pp, _ = _buf(P, 3 * n, ("float64",), "P", self.device, _lib.DEVICE)
        check(_lib.lib().arnold_stats_arrays(self._h, n, pc, pd, pp, t, kappa, ctypes.byref(s)),
              "arnold_stats_arrays")
        return stats_dict(s)

    # -- checkpoint / resume --
    def checkpoint(self) -> bytes:
        """Complete state as bytes (resume continues bit for bit)."""
        size = ctypes.c_size_t()
        check(_lib.lib().arnold_checkpoint_size(self._h, ctypes.byref(size)), "arnold_checkpoint_size")
        buf = ctypes.create_string_buffer(size.value)
        check(_lib.lib().arnold_checkpoint_save(self._h, buf, size.value), "arnold_checkpoint_save")
        return buf.raw

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        check(_lib.lib().arnold_checkpoint_load(self._h, buf, len(blob)), "arnold_checkpoint_load")

    def save(self, path: str):
        with open(path, "wb") as f:
            f.write(self.checkpoint())

    def load(self, path: str):
        with open(path, "rb") as f:
            self.restore(f.read())

    # -- differentiation --
    def forward_ckpt(self, n_steps: int, ckpt_every: int = 0):
        """Advance n_steps keeping sqrt(N) checkpoints for grad()."""
        check(_lib.lib().arnold_forward_ckpt(self._h, int(n_steps), int(ckpt_every)), "arnold_forward_ckpt")

    def grad(self, dL_dx=None, dL_dp=None, out_x=None, out_p=None):
        """Reverse sweep: returns (dL/dX0, dL/dP0, dL/dh, dL/deps).  Upstream and
        outputs are numpy (host) or torch CUDA tensors, [3][n] float64."""
        like = dL_dp if dL_dp is not None else dL_dx
        if like is None:
            raise ValueError("need dL_dx or dL_dp")
        if _is_torch(like) and like.is_cuda:
            import torch
            out_x = torch.empty((3, self.n), device=like.device, dtype=torch.float64) if out_x is None else out_x
            out_p = torch.empty((3, self.n), device=like.device, dtype=torch.float64) if out_p is None else out_p
            gpar = torch.empty(2, device=like.device, dtype=torch.float64)
        else:
            out_x = np.empty((3, self.n)) if out_x is None else out_x
            out_p = np.empty((3, self.n)) if out_p is None else out_p
            gpar = np.empty(2)
        c3 = 3 * self.n
        px, k = _buf(dL_dx, c3, ("float64",), "dL_dx", self.device) if dL_dx is not None else (None, None)
        pp, k2 = _buf(dL_dp, c3, ("float64",), "dL_dp", self.device) if dL_dp is not None else (None, None)
        kind = k if k is not None else k2
        if k is not None and k2 is not None and k != k2:
            raise ValueError("dL_dx and dL_dp must both be host or both device")
        ox, _ = _buf(out_x, c3, ("float64",), "out_x", self.device, kind)
        op, _ = _buf(out_p, c3, ("float64",), "out_p", self.device, kind)
        og, _ = _buf(gpar, 2, ("float64",), "gpar", self.device, kind)
        check(_lib.lib().arnold_grad(self._h, px, pp, ox, op, og, kind), "arnold_grad")
        return out_x, out_p, gpar[0], gpar[1]

    def debug_sincos(self, x, s, c, precision: str = "fp64"):
        px, _ = _ptr_kind(x)
        ps, _ = _ptr_kind(s)
        pc, _ = _ptr_kind(c)
        check(_lib.lib().arnold_debug_sincos(self._h, _lib.PRECISIONS[precision], int(x.shape[0]), px, ps, pc),
              "arnold_debug_sincos")


_MAP_FN = None


def _map_function():
    """The torch.autograd.Function of the N-step map, built on first use (importing
    this module does not import torch)."""
    global _MAP_FN
    if _MAP_FN is None:
        import torch

        class ArnoldMap(torch.autograd.Function):
            """(X0, P0, h, eps) -> (X_N unwrapped, P_N) on CUDA tensors [3][n]; the
            backward pass is the CUDA adjoint (arnold_grad) over the sqrt(N)
            checkpoints the forward pass stored.  h and eps may be floats or
            0-d tensors; a tensor gets its gradient as a 0-d tensor, a float
            none."""

            @staticmethod
            def forward(ctx, X0, P0, h, eps, n_steps, ckpt_every, precision, scheme):
                # autograd accepts a gradient only for tensor inputs
                ctx.h_is_tensor = torch.is_tensor(h)
                ctx.eps_is_tensor = torch.is_tensor(eps)
                n = X0.shape[1]
                ens = ArnoldEnsemble(n, eps=float(eps), h=float(h), scheme=scheme, precision=precision,
                                     tangent=False, device=X0.device.index or 0)
                ens.set_state(X0.detach().contiguous(), P0.detach().contiguous())
                ens.forward_ckpt(n_steps, ckpt_every)
                dX = torch.empty_like(X0)
                PN = torch.empty_like(P0)
                ens.indicator("dX", out=dX)
                ens.indicator("P", out=PN)
                ctx.ens = ens
                return X0.detach() + dX, PN

            @staticmethod
            def backward(ctx, gX, gP):
                ens = ctx.ens
                gx0, gp0, gh, ge = ens.grad(gX.contiguous(), gP.contiguous())
                ens.close()   # the checkpoints are spent: one backward per forward
                ctx.ens = None
                dev = gX.device
                gh = gh.to(dev).reshape(()) if ctx.h_is_tensor else None
                ge = ge.to(dev).reshape(()) if ctx.eps_is_tensor else None
                return gx0, gp0, gh, ge, None, None, None, None

        _MAP_FN = ArnoldMap
    return _MAP_FN


def __getattr__(name):
    if name == "ArnoldMap":
        return _map_function()
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")


def arnold_map(X0, P0, h, eps, n_steps: int, ckpt_every: int = 0, precision: str = "fp64", scheme: str = "yoshida6a"):
    """Differentiable N-step map (X0, P0, h, eps) -> (X_N unwrapped, P_N) on torch CUDA
    tensors (ArnoldMap.apply); backward runs the CUDA adjoint with sqrt(N)
    checkpointing (ckpt_every = 0: sqrt(N))."""
    return _map_function().apply(X0, P0, h, eps, int(n_steps), int(ckpt_every), precision, scheme)


class ArnoldBatch:
    """Many parameter sets advanced by one CUDA-graph launch.

    sets: list of dicts with eps, h, E, G, n_steps, seed (see arnold_batch_set).
    precision: "fp32c" (short horizons), "df64f" (the long-horizon compensated
    mode) or "df64".  tuning: dict with block_size, traj_per_thread,
    renorm_every, epoch_ms, or None for the library defaults
    (paper_1107_4107_b300.tune picks one)."""

    def __init__(self, sets, scheme: str = "yoshida6a", tangent: bool = True, tuning: dict | None = None,
                 device: int = 0, stream=None, precision: str = "fp32c"):
        L = _lib.lib()
        arr = (_lib.BatchSet * len(sets))()
        for k, q in enumerate(sets):
            arr[k] = _lib.BatchSet(float(q["eps"]), float(q["h"]), float(q["E"]), int(q["G"]), int(q["n_steps"]),
                                   int(q.get("seed", 0)))
        tu = _lib.BatchTuning()
        L.arnold_batch_tuning_default(ctypes.byref(tu))
        for k, v in (tuning or {}).items():
            setattr(tu, k, int(v))
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        check(L.arnold_batch_create(arr, len(sets), _lib.SCHEMES[scheme], _lib.PRECISIONS[precision],
                                    int(bool(tangent)), ctypes.byref(tu), device, ctypes.c_void_p(stream),
                                    ctypes.byref(h)), "arnold_batch_create")
        self._h = h
        self.device = device
        self.precision = precision
        self.sets = [dict(q) for q in sets]
        self.tuning = {f: getattr(tu, f) for f, _ in _lib.BatchTuning._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().arnold_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self):
        check(_lib.lib().arnold_batch_init(self._h), "arnold_batch_init")

    def run(self):
        check(_lib.lib().arnold_batch_run(self._h), "arnold_batch_run")

    def sync(self):
        check(_lib.lib().arnold_batch_sync(self._h), "arnold_batch_sync")

    @property
    def launches(self) -> int:
        return _lib.lib().arnold_batch_launch_count(self._h)

    def info(self) -> dict:
        e, i, m = _lib.i64(), _lib.i64(), _lib.i64()
        check(_lib.lib().arnold_batch_info(self._h, ctypes.byref(e), ctypes.byref(i), ctypes.byref(m)),
              "arnold_batch_info")
        return {"epochs": e.value, "items": i.value, "map_steps_per_run": m.value}

    def indicator(self, set_index: int, kind: str, out=None):
        q = self.sets[set_index]
        n = int(q["G"]) ** 2
        rows = _lib.IND_SHAPE[kind]
        dtype = np.uint8 if kind in ("class", "left") else np.float64
        if out is None:
            out = np.empty((rows, n) if rows > 1 else (n,), dtype=dtype)
        po, ko = _buf(out, rows * n, (np.dtype(dtype).name,), f"indicator({kind})", self.device)
        check(_lib.lib().arnold_batch_indicator(self._h, set_index, _lib.IND[kind], po, ko), "arnold_batch_indicator")
        return out

    def stats(self, set_index: int) -> dict:
        s = _lib.Stats()
        check(_lib.lib().arnold_batch_stats(self._h, set_index, ctypes.byref(s)), "arnold_batch_stats")
        return stats_dict(s)


def stats_dict(s) -> dict:
    return {"hist": np.array(list(s.hist), dtype=np.int64), "under": int(s.under), "over": int(s.over),
            "chaotic": int(s.chaotic), "n": int(s.n), "dE_max": float(s.dE_max),
            "p_mean": np.array(list(s.p_mean)), "p_var": np.array(list(s.p_var)), "t": float(s.t)}


def stats_arrays_noalloc(chi, dE, P, t: float, kappa: float = 10.0, device: int = 0, stream=None) -> dict:
    """Ensemble statistics of device arrays without any device allocation (for
    callers that cannot call cudaMalloc; see arnold_stats_arrays_noalloc in
    include/arnold.h).  The library's fixed scratch is shared by all calls on a
    device, so overlapping calls must be serialised by the caller."""
    n = int(chi.shape[0])
    if n > _lib.NOALLOC_MAX_N:
        raise ValueError(f"n = {n} exceeds the allocation-free limit {_lib.NOALLOC_MAX_N}")
    s = _lib.Stats()
    pc, _ = _ptr_kind(chi)
    pd, _ = _ptr_kind(dE)
    pp, _ = _ptr_kind(P)
    st = None if stream is None else ctypes.c_void_p(stream)
    check(_lib.lib().arnold_stats_arrays_noalloc(device, st, n, pc, pd, pp, t, kappa, ctypes.byref(s)),
          "arnold_stats_arrays_noalloc")
    return stats_dict(s)


def probe_peak(kind: str, device: int = 0) -> float:
    """Measured lane-operations/s of one pipe: 'dfma', 'ffma' or 'mufu'."""
    v = ctypes.c_double()
    check(_lib.lib().arnold_probe_peak(device, {"dfma": 0, "ffma": 1, "mufu": 2}[kind], ctypes.byref(v)),
          "arnold_probe_peak")
    return v.value


def chaos_threshold(t: float, kappa: float = 10.0) -> float:
    return kappa * math.log(max(abs(t), math.e)) / abs(t)
