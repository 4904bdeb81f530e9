"""Thin ctypes binding of the C ABI in include/jz.h (argument marshalling only).

Every step of the solver runs in the CUDA library ``_build/libjz.so``; this
module only converts Python/NumPy/torch arguments to pointers and status
codes to exceptions.  There is no CPU fallback: if the library is missing,
loading fails loudly.

Functions keep the C names (``jz_create_grid``, ``jz_rk_step``, ...); the
``Grid`` and ``Solver`` classes own the handles.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libjz.so")

JZ_OK, JZ_ERR_ARG, JZ_ERR_CUDA, JZ_ERR_OOM, JZ_ERR_NONFINITE, JZ_ERR_STATE = 0, -1, -2, -3, -4, -5
JZ_TOPO_PERIODIC, JZ_TOPO_JET = 1, 2
JZ_PREC_FP64, JZ_PREC_FP32FLUX, JZ_PREC_FP64PAIR = 0, 1, 2
N_MODES, N_FREQ = 8, 4

# Entry points declared in include/jz.h (checked by the tests).
EXPORTS = ("jz_last_error", "jz_version", "jz_create_grid", "jz_destroy_grid", "jz_compute_metrics",
           "jz_get_metrics", "jz_create", "jz_destroy", "jz_set_state", "jz_get_state", "jz_residual",
           "jz_rk_step", "jz_profile", "jz_profile_read", "jz_profile_name", "jz_residual_noalloc",
           "jz_adjoint_step", "jz_save_snapshot", "jz_load_snapshot", "jz_stats_begin", "jz_stats_sample",
           "jz_stats_read", "jz_stats_end", "jz_station_profile", "jz_potential_core", "jz_check_math",
           "jz_grid_compact", "jz_check_wait", "jz_check_pair")
JZ_NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024
JZ_NPROF = 10


class JzError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"jz error {code}: {msg}")
        self.code = code


class jz_params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "gamma", "Pr", "Pr_sgs", "Re", "mach_ref", "T_ref_K", "S1_K", "C_s", "kappa2", "kappa4",
        "sigma", "cfl", "dt_fixed", "jet_mach", "theta_mom")] + [
        ("forcing_amp", ctypes.c_double * (N_MODES * N_FREQ)),
        ("forcing_phi", ctypes.c_double * (N_MODES * N_FREQ)),
        ("forcing_psi", ctypes.c_double * (N_MODES * N_FREQ)),
        ("strouhal", ctypes.c_double * N_FREQ),
        ("precision", ctypes.c_int)]


class jz_step_stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("res_l2", ctypes.c_double),
                ("totals", ctypes.c_double * 5), ("min_rho", ctypes.c_double), ("min_p", ctypes.c_double),
                ("steps", ctypes.c_longlong)]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libjz.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing: build it with paper_2003_08746_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    sig = {
        "jz_last_error": ([], ctypes.c_char_p),
        "jz_version": ([], i),
        "jz_create_grid": ([i, i, i, vp, vp, i, ctypes.POINTER(vp)], i),
        "jz_destroy_grid": ([vp], i),
        "jz_compute_metrics": ([vp], i),
        "jz_get_metrics": ([vp, vp], i),
        "jz_create": ([vp, ctypes.POINTER(jz_params), vp, ctypes.POINTER(vp)], i),
        "jz_destroy": ([vp], i),
        "jz_set_state": ([vp, vp, d], i),
        "jz_get_state": ([vp, vp], i),
        "jz_residual": ([vp, vp, vp], i),
        "jz_rk_step": ([vp, i, ctypes.POINTER(jz_step_stats)], i),
        "jz_profile": ([vp, i], i),
        "jz_profile_read": ([vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)], i),
        "jz_profile_name": ([i], ctypes.c_char_p),
        "jz_residual_noalloc": ([vp, ctypes.POINTER(jz_params), vp, vp, vp], i),
        "jz_adjoint_step": ([vp, vp, i, i, d, ctypes.POINTER(ctypes.c_double), vp], i),
        "jz_save_snapshot": ([vp, ctypes.c_char_p], i),
        "jz_load_snapshot": ([vp, ctypes.c_char_p], i),
        "jz_grid_compact": ([vp], i),
        "jz_check_math": ([ctypes.POINTER(ctypes.c_double)] * 3, i),
        "jz_check_wait": ([ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)], i),
        "jz_check_pair": ([ctypes.POINTER(ctypes.c_double)], i),
        "jz_stats_begin": ([vp, i], i),
        "jz_stats_sample": ([vp], i),
        "jz_stats_read": ([vp, vp, vp, ctypes.POINTER(ctypes.c_longlong)], i),
        "jz_stats_end": ([vp], i),
        "jz_station_profile": ([vp, vp, i, i, d, vp], i),
        "jz_potential_core": ([vp, vp, i, d, d, ctypes.POINTER(ctypes.c_double)], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes, fn.restype = args, res
    _lib = lib
    return lib


def _check(code: int) -> None:
    if code != JZ_OK:
        raise JzError(code, load().jz_last_error().decode())


def _ptr(x):
    """Data pointer of a C-contiguous float64 NumPy array or torch tensor (CPU or CUDA)."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a C-contiguous float64 array")
        return ctypes.c_void_p(x.ctypes.data)
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("expected a contiguous float64 tensor")
        return ctypes.c_void_p(x.data_ptr())
    raise TypeError(f"unsupported array type {type(x)}")


# --- C names ---------------------------------------------------------------
def jz_version() -> int:
    return load().jz_version()


def jz_create_grid(ni, nj, nk, xyz, period, topology):
    h = ctypes.c_void_p()
    per = None if period is None else np.ascontiguousarray(period, dtype=np.float64).reshape(9)
    _check(load().jz_create_grid(ni, nj, nk, _ptr(xyz), None if per is None else _ptr(per), topology,
                                 ctypes.byref(h)))
    return h


def jz_destroy_grid(h):
    _check(load().jz_destroy_grid(h))


def jz_compute_metrics(h):
    _check(load().jz_compute_metrics(h))


def jz_get_metrics(h, out):
    _check(load().jz_get_metrics(h, _ptr(out)))


def make_params(prm, precision: int = JZ_PREC_FP64) -> jz_params:
    """jz_params from a workloads.FlowParams-like object (plain values)."""
    p = jz_params()
    for name in ("gamma", "Pr", "Pr_sgs", "Re", "mach_ref", "T_ref_K", "S1_K", "C_s", "kappa2", "kappa4",
                 "sigma", "cfl", "dt_fixed", "jet_mach", "theta_mom"):
        setattr(p, name, float(getattr(prm, name)))
    for name in ("forcing_amp", "forcing_phi", "forcing_psi"):
        v = getattr(prm, name, None)
        arr = np.zeros(N_MODES * N_FREQ) if v is None else np.asarray(v, dtype=np.float64).reshape(-1)
        getattr(p, name)[:] = list(arr)
    p.strouhal[:] = [float(s) for s in prm.strouhal]
    p.precision = int(precision)
    return p


def jz_create(grid_h, params: jz_params, stream=None):
    h = ctypes.c_void_p()
    st = ctypes.c_void_p(0 if stream is None else int(stream))
    _check(load().jz_create(grid_h, ctypes.byref(params), st, ctypes.byref(h)))
    return h


def jz_destroy(h):
    _check(load().jz_destroy(h))


def jz_set_state(h, q, t: float = 0.0):
    _check(load().jz_set_state(h, _ptr(q), float(t)))


def jz_get_state(h, q):
    _check(load().jz_get_state(h, _ptr(q)))


def jz_residual(h, q, rhs):
    _check(load().jz_residual(h, _ptr(q), _ptr(rhs)))


def _stream_handle(stream):
    """cudaStream_t of a torch.cuda.Stream (its .cuda_stream), a raw handle, or, for None,
    torch's current stream on the current device."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def jz_residual_noalloc(grid_h, params: jz_params, q, rhs, stream=None):
    """Residual with the library's fixed scratch array (no device allocation); device q and rhs.
    The work is queued on `stream` (default: torch's current stream), and the call returns
    without waiting for it."""
    st = ctypes.c_void_p(_stream_handle(stream))
    _check(load().jz_residual_noalloc(grid_h, ctypes.byref(params), _ptr(q), _ptr(rhs), st))


def jz_grid_compact(grid_h) -> None:
    _check(load().jz_grid_compact(grid_h))


def jz_check_math():
    """(max relative error of the library's FP64 reciprocal, cube roots, square root) on the
    device."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().jz_check_math(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def jz_check_pair():
    """Largest errors of the pair (double-float) operations against FP64 on the device:
    {add, mul, fma, rcp, sqrt, cbrt, roundtrip, sqrt_tiny, cbrt_tiny}."""
    out = (ctypes.c_double * 9)()
    _check(load().jz_check_pair(out))
    return dict(zip(("add", "mul", "fma", "rcp", "sqrt", "cbrt", "roundtrip", "sqrt_tiny", "cbrt_tiny"), list(out)))


def jz_check_wait():
    """(timed_out, milliseconds) of the stage kernel's bounded mbarrier wait run on a barrier
    that nothing arrives at (timed_out is 1 when the wait ran out and returned)."""
    t, ms = ctypes.c_int(), ctypes.c_double()
    _check(load().jz_check_wait(ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def jz_stats_begin(h, every: int) -> None:
    _check(load().jz_stats_begin(h, int(every)))


def jz_stats_sample(h) -> None:
    _check(load().jz_stats_sample(h))


def jz_stats_read(h, mean=None, rms=None) -> int:
    """Fill mean and rms ([nj][ni] float64, host or device; None to skip); returns the sample count."""
    n = ctypes.c_longlong()
    _check(load().jz_stats_read(h, None if mean is None else _ptr(mean), None if rms is None else _ptr(rms),
                                ctypes.byref(n)))
    return n.value


def jz_stats_end(h) -> None:
    _check(load().jz_stats_end(h))


def jz_station_profile(field, x, x0: float):
    """Profile of field [nj][ni] at axial position x0 (x [ni] increasing): array [nj]."""
    field = np.ascontiguousarray(field, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    nj, ni = field.shape
    if x.shape != (ni,):
        raise ValueError("x must have one entry per i line")
    out = np.empty(nj)
    _check(load().jz_station_profile(_ptr(field), _ptr(x), ni, nj, float(x0), _ptr(out)))
    return out


def jz_potential_core(axis, x, u_jet: float, frac: float = 0.95):
    """First x where axis [ni] falls below frac * u_jet (linear interpolation); None if never."""
    axis = np.ascontiguousarray(axis, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    if axis.shape != x.shape:
        raise ValueError("axis and x must have the same length")
    xc = ctypes.c_double()
    _check(load().jz_potential_core(_ptr(axis), _ptr(x), axis.size, float(u_jet), float(frac), ctypes.byref(xc)))
    return None if np.isnan(xc.value) else xc.value


def jz_save_snapshot(h, path) -> None:
    _check(load().jz_save_snapshot(h, os.fsencode(path)))


def jz_load_snapshot(h, path) -> None:
    _check(load().jz_load_snapshot(h, os.fsencode(path)))


SNAPSHOT_HEADER_BYTES = 256
_SNAP_FIELDS = np.dtype([("magic", "S8"), ("version", "<i4"), ("header_bytes", "<i4"), ("ni", "<i4"),
                         ("nj", "<i4"), ("nk", "<i4"), ("topology", "<i4"), ("precision", "<i4"),
                         ("flags", "<i4"), ("steps", "<i8"), ("t", "<f8"), ("dt", "<f8"), ("rate", "<f8"),
                         ("res_sum", "<f8"), ("params_hash", "<u8"), ("data_hash", "<u8")])


def read_snapshot(path):
    """Parse a snapshot file on the host (no GPU): (header dict, Q^n as [5][nk][nj][ni] float64).

    File layout (as written by jz_save_snapshot): a 256-byte little-endian header, then
    Q^n in the jz_get_state layout."""
    with open(path, "rb") as f:
        raw = f.read(SNAPSHOT_HEADER_BYTES)
        if len(raw) != SNAPSHOT_HEADER_BYTES:
            raise ValueError("short snapshot header")
        hd = np.frombuffer(raw[:_SNAP_FIELDS.itemsize], dtype=_SNAP_FIELDS)[0]
        head = {k: (hd[k].item() if k != "magic" else bytes(hd[k])) for k in _SNAP_FIELDS.names}
        if head["magic"] != b"JZSNAP01" or head["version"] != 1:
            raise ValueError("not a version-1 jz snapshot")
        n = 5 * head["ni"] * head["nj"] * head["nk"]
        q = np.fromfile(f, dtype="<f8", count=n)
    if q.size != n:
        raise ValueError("short snapshot data")
    return head, q.reshape(5, head["nk"], head["nj"], head["ni"])


def jz_rk_step(h, nsteps: int, want_stats: bool = True):
    st = jz_step_stats() if want_stats else None
    _check(load().jz_rk_step(h, int(nsteps), ctypes.byref(st) if st is not None else None))
    return st


def jz_adjoint_step(h, amps, nsteps: int, ckpt_every: int, r_obs: float):
    """(J, dJ/dA [8][4]) of the observer functional by the discrete adjoint (see include/jz.h)."""
    a = np.ascontiguousarray(np.asarray(amps, dtype=np.float64).reshape(N_MODES * N_FREQ))
    J = ctypes.c_double()
    g = np.empty(N_MODES * N_FREQ)
    _check(load().jz_adjoint_step(h, _ptr(a), int(nsteps), int(ckpt_every), float(r_obs), ctypes.byref(J), _ptr(g)))
    return J.value, g.reshape(N_MODES, N_FREQ)


def _jet_functional_class():
    import torch

    class JetFunctional(torch.autograd.Function):
        """J(A) of the observer functional as a differentiable function of the forcing
        amplitudes A [8][4]: forward and gradient both come from jz_adjoint_step."""

        @staticmethod
        def forward(ctx, amps, solver, nsteps, ckpt_every, r_obs):
            J, g = jz_adjoint_step(solver.h, amps.detach().cpu().numpy(), nsteps, ckpt_every, r_obs)
            ctx.save_for_backward(torch.as_tensor(g, dtype=amps.dtype, device=amps.device))
            return amps.new_tensor(J)

        @staticmethod
        def backward(ctx, gJ):
            (g,) = ctx.saved_tensors
            return gJ * g, None, None, None, None

    return JetFunctional


def jet_functional(amps, solver, nsteps: int, ckpt_every: int, r_obs: float):
    """Differentiable J(A) (torch.autograd.Function over jz_adjoint_step)."""
    return _jet_functional_class().apply(amps, solver, nsteps, ckpt_every, r_obs)


def jz_profile(h, enable: bool):
    _check(load().jz_profile(h, 1 if enable else 0))


def jz_profile_read(h):
    """{kind name: (device ms, launches)} since the last read."""
    ms = (ctypes.c_double * JZ_NPROF)()
    n = (ctypes.c_longlong * JZ_NPROF)()
    _check(load().jz_profile_read(h, ms, n))
    lib = load()
    return {lib.jz_profile_name(k).decode(): (ms[k], n[k]) for k in range(JZ_NPROF)}


# --- owners ----------------------------------------------------------------
class Grid:
    """Owner of a jz_grid handle; metrics are computed on construction."""

    def __init__(self, ni, nj, nk, xyz, topology, period=None, metrics=True):
        """metrics=False leaves jz_compute_metrics to the caller (e.g. after freeing xyz)."""
        self.ni, self.nj, self.nk, self.topology = int(ni), int(nj), int(nk), int(topology)
        self.h = jz_create_grid(self.ni, self.nj, self.nk, xyz, period, self.topology)
        if metrics:
            jz_compute_metrics(self.h)

    def compute_metrics(self):
        jz_compute_metrics(self.h)

    def compact(self):
        """Keep FP32 metrics only (FP32-flux solvers; frees 96 bytes per padded node)."""
        jz_grid_compact(self.h)

    @classmethod
    def from_workload(cls, g):
        return cls(g.ni, g.nj, g.nk, g.xyz, g.topology, g.period)

    @property
    def npts(self):
        return self.ni * self.nj * self.nk

    def metrics(self):
        out = np.empty((10, self.nk, self.nj, self.ni))
        jz_get_metrics(self.h, out)
        return out

    def close(self):
        if self.h:
            jz_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owner of a jz_solver handle on a Grid."""

    def __init__(self, grid: Grid, prm, precision: int = JZ_PREC_FP64, stream=None):
        self.grid = grid
        self.params = make_params(prm, precision)
        self.h = jz_create(grid.h, self.params, stream)

    def set_state(self, q, t: float = 0.0):
        jz_set_state(self.h, q, t)

    def get_state(self, out=None):
        if out is None:
            out = np.empty((5, self.grid.nk, self.grid.nj, self.grid.ni))
        jz_get_state(self.h, out)
        return out

    def residual(self, q, out=None):
        if out is None:
            out = np.empty((5, self.grid.nk, self.grid.nj, self.grid.ni))
        jz_residual(self.h, q, out)
        return out

    def step(self, nsteps: int = 1, stats: bool = True):
        return jz_rk_step(self.h, nsteps, stats)

    def save(self, path):
        jz_save_snapshot(self.h, path)

    def stats_begin(self, every: int = 1):
        jz_stats_begin(self.h, every)

    def stats_sample(self):
        jz_stats_sample(self.h)

    def stats_read(self):
        """(mean, rms, samples): azimuthally averaged axial-velocity statistics, [nj][ni] each."""
        mean = np.empty((self.grid.nj, self.grid.ni))
        rms = np.empty_like(mean)
        n = jz_stats_read(self.h, mean, rms)
        return mean, rms, n

    def stats_end(self):
        jz_stats_end(self.h)

    def load(self, path):
        jz_load_snapshot(self.h, path)

    def profile(self, enable: bool = True):
        jz_profile(self.h, enable)

    def profile_read(self):
        return jz_profile_read(self.h)

    def close(self):
        if self.h:
            jz_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
