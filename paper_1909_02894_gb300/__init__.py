"""Python binding of libdirac.so, the GB300 (sm_103a) implementation of the Scheme II
pseudospectral step for the 2D Dirac equation in static curved space (arXiv:1909.02894).

Argument marshalling only: every numerical step runs in the library's CUDA kernels.
The functions carry the names of the C ABI in ``include/dirac.h``. There is no CPU
fallback: if the compiled library is absent, :func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# DIRAC_LIB may name another build of the same library (e.g. one made with other
# DIRAC_NVCC_EXTRA flags); by default the in-tree libdirac.so.
LIB_PATH = os.environ.get("DIRAC_LIB") or os.path.join(HERE, "libdirac.so")

DIRAC_OK, DIRAC_EINVAL, DIRAC_ENOMEM, DIRAC_EUNSUPPORTED = 0, 1, 2, 3
DIRAC_ECUDA, DIRAC_ETIMEOUT, DIRAC_ENONFINITE, DIRAC_ESTATE = 4, 5, 6, 7
DIRAC_ENOCONV = 8
STATUS_NAMES = {0: "DIRAC_OK", 1: "DIRAC_EINVAL", 2: "DIRAC_ENOMEM", 3: "DIRAC_EUNSUPPORTED",
                4: "DIRAC_ECUDA", 5: "DIRAC_ETIMEOUT", 6: "DIRAC_ENONFINITE", 7: "DIRAC_ESTATE",
                8: "DIRAC_ENOCONV"}
DIRAC_C64, DIRAC_C128 = 0, 1
DIRAC_CONN_COVARIANT, DIRAC_CONN_PAPER_2D, DIRAC_CONN_NONE = 0, 1, 2
DIRAC_SCHEME_II, DIRAC_SCHEME_II_SYMMETRIC = 0, 1
DIRAC_SCHEME_POLY_TAYLOR, DIRAC_SCHEME_POLY_CHEBYSHEV = 2, 3
DIRAC_SCHEME_CRANK_NICOLSON = 4
# dirac_set_launch flag: the other radix schedule of the FFT passes (with 256 or 512)
DIRAC_LAUNCH_ALT_RADIX = 0x10000

# Every symbol the header declares; the CPU tests check that the library exports them.
ABI_SYMBOLS = (
    "dirac_create", "dirac_set_state", "dirac_get_state", "dirac_step",
    "dirac_observables", "dirac_synchronize", "dirac_last_error", "dirac_destroy",
    "dirac_set_launch", "dirac_launch_count", "dirac_norms_noalloc", "dirac_footprint_bytes",
    "dirac_autotune", "dirac_test_timeout_next_step", "dirac_set_scheme",
    "dirac_set_poly_degree", "dirac_set_krylov", "dirac_krylov_iterations",
    "dirac_set_potentials",
    "dirac_batch_create", "dirac_batch_submit", "dirac_batch_run", "dirac_batch_poll",
    "dirac_batch_release", "dirac_batch_synchronize", "dirac_batch_active",
    "dirac_batch_launch_count", "dirac_batch_last_error", "dirac_batch_destroy",
    "dirac_batch_autotune", "dirac_batch_launch_shape", "dirac_measure_alu_peak",
)


class DiracError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int)]


class _Domain(C.Structure):
    _fields_ = [("ax", C.c_double), ("ay", C.c_double)]


class _Metric(C.Structure):
    _fields_ = [("g00", C.c_void_p), ("g11", C.c_void_p), ("g22", C.c_void_p), ("conn", C.c_int)]


class _Absorber(C.Structure):
    _fields_ = [("width_x", C.c_int), ("width_y", C.c_int), ("type", C.c_int),
                ("sigma0", C.c_double), ("theta", C.c_double)]


class _Obs(C.Structure):
    _fields_ = [("norm", C.c_double), ("norm_gamma", C.c_double), ("energy", C.c_double),
                ("energy_imag", C.c_double)]


_lib = None


def build(force: bool = False) -> str:
    """Compile libdirac.so in place (nvcc, sm_103a)."""
    from . import _build

    return _build.build(force=force)


def lib():
    """The loaded CUDA library. Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(LIB_PATH)
        vp, dp, i, d, l = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double, C.c_long
        L.dirac_create.argtypes = [C.POINTER(_Grid), C.POINTER(_Domain), C.POINTER(_Metric), d, d,
                                   C.POINTER(_Absorber), i, vp, C.POINTER(vp)]
        L.dirac_set_state.argtypes = [vp, vp, i]
        L.dirac_get_state.argtypes = [vp, vp, i]
        L.dirac_step.argtypes = [vp, l, d]
        L.dirac_observables.argtypes = [vp, C.POINTER(_Obs), vp]
        L.dirac_synchronize.argtypes = [vp]
        L.dirac_last_error.argtypes = [vp]
        L.dirac_last_error.restype = C.c_char_p
        L.dirac_destroy.argtypes = [vp]
        L.dirac_destroy.restype = None
        L.dirac_set_launch.argtypes = [vp, i, i]
        L.dirac_set_scheme.argtypes = [vp, i]
        L.dirac_set_poly_degree.argtypes = [vp, i]
        L.dirac_set_krylov.argtypes = [vp, d, i, i]
        L.dirac_set_potentials.argtypes = [vp, vp, vp, vp]
        L.dirac_krylov_iterations.argtypes = [vp]
        L.dirac_krylov_iterations.restype = l
        L.dirac_launch_count.argtypes = [vp]
        L.dirac_launch_count.restype = l
        L.dirac_norms_noalloc.argtypes = [vp, vp, i, i, d, d, vp, vp]
        L.dirac_norms_noalloc.restype = C.c_int
        L.dirac_test_timeout_next_step.argtypes = [vp]
        L.dirac_test_timeout_next_step.restype = C.c_int
        L.dirac_autotune.argtypes = [vp, i, C.POINTER(i), C.POINTER(i)]
        L.dirac_autotune.restype = C.c_int
        L.dirac_measure_alu_peak.argtypes = [i, dp, vp]
        L.dirac_measure_alu_peak.restype = C.c_int
        L.dirac_footprint_bytes.argtypes = [C.POINTER(_Grid), i]
        L.dirac_footprint_bytes.restype = C.c_size_t
        L.dirac_batch_create.argtypes = [C.c_size_t, i, vp, i, C.POINTER(vp)]
        L.dirac_batch_submit.argtypes = [vp, vp, l, d, C.POINTER(i)]
        L.dirac_batch_run.argtypes = [vp, i]
        L.dirac_batch_poll.argtypes = [vp, i, C.POINTER(i)]
        L.dirac_batch_release.argtypes = [vp, i]
        L.dirac_batch_synchronize.argtypes = [vp]
        L.dirac_batch_autotune.argtypes = [vp, i]
        L.dirac_batch_launch_shape.argtypes = [vp, i, i, C.POINTER(i), C.POINTER(i)]
        for f in ("dirac_batch_create", "dirac_batch_submit", "dirac_batch_run",
                  "dirac_batch_poll", "dirac_batch_release", "dirac_batch_synchronize",
                  "dirac_batch_autotune", "dirac_batch_launch_shape"):
            getattr(L, f).restype = C.c_int
        L.dirac_batch_active.argtypes = [vp]
        L.dirac_batch_active.restype = C.c_int
        L.dirac_batch_launch_count.argtypes = [vp]
        L.dirac_batch_launch_count.restype = l
        L.dirac_batch_last_error.argtypes = [vp]
        L.dirac_batch_last_error.restype = C.c_char_p
        L.dirac_batch_destroy.argtypes = [vp]
        L.dirac_batch_destroy.restype = None
        for f in ("dirac_create", "dirac_set_state", "dirac_get_state", "dirac_step",
                  "dirac_observables", "dirac_synchronize", "dirac_set_launch"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def dirac_last_error(ctx=None) -> str:
    s = lib().dirac_last_error(ctx)
    return s.decode() if s else ""


def _check(status, ctx=None):
    if status != DIRAC_OK:
        raise DiracError(status, dirac_last_error(ctx))


def _f64_field(a, ny, nx):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (ny, nx):
        raise ValueError(f"metric field shape {a.shape} != {(ny, nx)}")
    return a


def dirac_create(nx: int, ny: int, ax: float, ay: float, *, g00=None, g11=None, g22=None,
                 conn: int = DIRAC_CONN_COVARIANT, mass: float = 0.0, c: float = 1.0,
                 pml_wx: int = 0, pml_wy: int = 0, pml_type: int = 1, sigma0: float = 1.0,
                 theta: float = 0.0, precision: int = DIRAC_C64, stream: Optional[int] = None):
    """dirac_create: returns the context handle (an int)."""
    g = [_f64_field(x, ny, nx) for x in (g00, g11, g22)]
    metric = _Metric(*[None if x is None else x.ctypes.data for x in g], conn)
    absorber = _Absorber(pml_wx, pml_wy, pml_type, sigma0, theta)
    out = C.c_void_p()
    st = lib().dirac_create(C.byref(_Grid(nx, ny)), C.byref(_Domain(ax, ay)), C.byref(metric),
                            mass, c, C.byref(absorber), precision, stream, C.byref(out))
    _check(st, None)
    return out.value


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def dirac_set_state(ctx, psi):
    """psi: numpy complex128 [2][ny][nx] (host) or a CUDA torch complex128 tensor."""
    if _is_torch(psi):
        assert psi.is_cuda and psi.is_contiguous() and str(psi.dtype) == "torch.complex128"
        _check(lib().dirac_set_state(ctx, psi.data_ptr(), 1), ctx)
        return
    a = np.ascontiguousarray(psi, dtype=np.complex128)
    _check(lib().dirac_set_state(ctx, a.ctypes.data, 0), ctx)


def dirac_get_state(ctx, out):
    """Fills out (numpy complex128 [2][ny][nx], or a CUDA torch complex128 tensor)."""
    if _is_torch(out):
        assert out.is_cuda and out.is_contiguous() and str(out.dtype) == "torch.complex128"
        _check(lib().dirac_get_state(ctx, out.data_ptr(), 1), ctx)
        return out
    assert out.dtype == np.complex128 and out.flags.c_contiguous
    _check(lib().dirac_get_state(ctx, out.ctypes.data, 0), ctx)
    return out


def dirac_step(ctx, n_steps: int, dt: float):
    _check(lib().dirac_step(ctx, int(n_steps), float(dt)), ctx)


def dirac_observables(ctx, density=None):
    """Returns {norm, norm_gamma, energy, energy_imag}; fills density (numpy [ny][nx])."""
    o = _Obs()
    dp = None
    if density is not None:
        assert density.dtype == np.float64 and density.flags.c_contiguous
        dp = density.ctypes.data
    st = lib().dirac_observables(ctx, C.byref(o), dp)
    res = {"norm": o.norm, "norm_gamma": o.norm_gamma, "energy": o.energy,
           "energy_imag": o.energy_imag}
    if st == DIRAC_ENONFINITE:
        raise DiracError(st, dirac_last_error(ctx))
    _check(st, ctx)
    return res


def dirac_synchronize(ctx):
    _check(lib().dirac_synchronize(ctx), ctx)


def dirac_set_launch(ctx, threads_x: int, threads_y: int):
    _check(lib().dirac_set_launch(ctx, int(threads_x), int(threads_y)), ctx)


def dirac_set_scheme(ctx, scheme: int):
    _check(lib().dirac_set_scheme(ctx, int(scheme)), ctx)


def dirac_set_poly_degree(ctx, degree: int):
    _check(lib().dirac_set_poly_degree(ctx, int(degree)), ctx)


def dirac_set_krylov(ctx, tol: float = 0.0, restart: int = 20, max_restarts: int = 100):
    _check(lib().dirac_set_krylov(ctx, float(tol), int(restart), int(max_restarts)), ctx)


def dirac_krylov_iterations(ctx) -> int:
    return int(lib().dirac_krylov_iterations(ctx))


def dirac_set_potentials(ctx, V=None, Ax=None, Ay=None, shape=None):
    """Static potentials as [ny][nx] arrays (None = 0); the library copies them."""
    arrs = [None if f is None else np.ascontiguousarray(f, dtype=np.float64) for f in (V, Ax, Ay)]
    if shape is not None:
        for a in arrs:
            if a is not None and a.shape != tuple(shape):
                raise ValueError(f"potential shape {a.shape} != {tuple(shape)}")
    ptrs = [None if a is None else a.ctypes.data for a in arrs]
    _check(lib().dirac_set_potentials(ctx, *ptrs), ctx)


def dirac_launch_count(ctx) -> int:
    return int(lib().dirac_launch_count(ctx))


def dirac_norms_noalloc(psi, weight, ax: float, ay: float, out, stream=None):
    """Norms of a CUDA complex128 [2][ny][nx] tensor without device allocation: writes
    {norm, weighted norm} into out (a CUDA float64 tensor of at least 2 elements).
    weight: CUDA float64 [ny][nx] tensor or None. All tensors must be contiguous and on
    one device; the call is enqueued on that device, on `stream` (a raw handle; None =
    the default stream). Raises ValueError before any launch if a tensor does not fit."""
    def need(cond, msg):
        if not cond:
            raise ValueError(f"dirac_norms_noalloc: {msg}")

    need(_is_torch(psi) and _is_torch(out), "psi and out must be torch tensors")
    need(psi.dim() == 3 and int(psi.shape[0]) == 2,
         f"psi must have shape (2, ny, nx), got {tuple(psi.shape)}")
    ny, nx = int(psi.shape[1]), int(psi.shape[2])
    need(str(psi.dtype) == "torch.complex128" and psi.is_contiguous(),
         "psi must be contiguous complex128")
    need(str(out.dtype) == "torch.float64" and out.is_contiguous() and out.numel() >= 2,
         "out must be a contiguous float64 tensor of at least 2 elements")
    if weight is not None:
        need(_is_torch(weight) and tuple(weight.shape) == (ny, nx),
             f"weight must have shape {(ny, nx)}, got {tuple(getattr(weight, 'shape', ()))}")
        need(str(weight.dtype) == "torch.float64" and weight.is_contiguous(),
             "weight must be contiguous float64")
    need(psi.is_cuda and out.is_cuda and (weight is None or weight.is_cuda),
         "psi, weight and out must be CUDA tensors")
    need(out.device == psi.device and (weight is None or weight.device == psi.device),
         "psi, weight and out must be on one device")
    import torch

    with torch.cuda.device(psi.device):
        _check(lib().dirac_norms_noalloc(psi.data_ptr(),
                                         None if weight is None else weight.data_ptr(), nx,
                                         ny, float(ax), float(ay), out.data_ptr(), stream),
               None)


ALU_FP64, ALU_FP32, ALU_FP32X2 = 0, 1, 2


def dirac_measure_alu_peak(kind: int, stream=None) -> float:
    """Measured FMA throughput in TFLOP/s (kind: ALU_FP64, ALU_FP32, ALU_FP32X2)."""
    t = C.c_double(0.0)
    _check(lib().dirac_measure_alu_peak(int(kind), C.byref(t), stream), None)
    return t.value


def dirac_test_timeout_next_step(ctx):
    _check(lib().dirac_test_timeout_next_step(ctx), ctx)


def dirac_autotune(ctx, reps: int = 20):
    """Times every CTA shape of both passes and keeps the fastest; returns (tx, ty)."""
    tx, ty = C.c_int(0), C.c_int(0)
    _check(lib().dirac_autotune(ctx, int(reps), C.byref(tx), C.byref(ty)), ctx)
    return tx.value, ty.value


def dirac_footprint_bytes(nx: int, ny: int, precision: int = DIRAC_C64) -> int:
    return int(lib().dirac_footprint_bytes(C.byref(_Grid(nx, ny)), precision))


def dirac_batch_last_error(batch) -> str:
    s = lib().dirac_batch_last_error(batch)
    return s.decode() if s else ""


def _bcheck(status, batch):
    if status != DIRAC_OK:
        raise DiracError(status, dirac_batch_last_error(batch))


def dirac_batch_autotune(batch, reps: int = 10):
    """Times every CTA shape of each class's passes over its stepping contexts and keeps
    the fastest (no state changes)."""
    _bcheck(lib().dirac_batch_autotune(batch, int(reps)), batch)


def dirac_batch_launch_shape(batch, nx: int, ny: int):
    """(threads_x, threads_y) in dirac_set_launch terms of the nx x ny class."""
    tx, ty = C.c_int(0), C.c_int(0)
    _bcheck(lib().dirac_batch_launch_shape(batch, int(nx), int(ny), C.byref(tx), C.byref(ty)),
            batch)
    return tx.value, ty.value


def dirac_batch_create(budget_bytes: int, precision: int = DIRAC_C64, steps_per_tick: int = 32,
                       stream: Optional[int] = None):
    out = C.c_void_p()
    st = lib().dirac_batch_create(int(budget_bytes), precision, stream, int(steps_per_tick),
                                  C.byref(out))
    if st != DIRAC_OK:
        raise DiracError(st, "dirac_batch_create failed")
    return out.value


def dirac_batch_submit(batch, ctx, n_steps: int, dt: float) -> int:
    slot = C.c_int(-1)
    _bcheck(lib().dirac_batch_submit(batch, ctx, int(n_steps), float(dt), C.byref(slot)), batch)
    return slot.value


def dirac_batch_run(batch, n_ticks: int = 1):
    _bcheck(lib().dirac_batch_run(batch, int(n_ticks)), batch)


def dirac_batch_poll(batch, slot: int) -> bool:
    done = C.c_int(0)
    _bcheck(lib().dirac_batch_poll(batch, int(slot), C.byref(done)), batch)
    return bool(done.value)


def dirac_batch_release(batch, slot: int):
    _bcheck(lib().dirac_batch_release(batch, int(slot)), batch)


def dirac_batch_synchronize(batch):
    _bcheck(lib().dirac_batch_synchronize(batch), batch)


def dirac_batch_active(batch) -> int:
    return int(lib().dirac_batch_active(batch))


def dirac_batch_launch_count(batch) -> int:
    return int(lib().dirac_batch_launch_count(batch))


def dirac_batch_destroy(batch):
    if batch:
        lib().dirac_batch_destroy(batch)


def dirac_destroy(ctx):
    if ctx:
        lib().dirac_destroy(ctx)


class Simulation:
    """Owns one context; marshalling only (same calls as the C ABI)."""

    def __init__(self, workload, precision=DIRAC_C64, stream=None, conn=None,
                 scheme=DIRAC_SCHEME_II, poly_degree=None):
        w = workload
        self.nx, self.ny = w.nx, w.ny
        self.ctx = dirac_create(
            w.nx, w.ny, w.ax, w.ay, g00=w.g00, g11=w.g11, g22=w.g22,
            conn=w.conn if conn is None else conn, mass=w.mass, c=w.c,
            pml_wx=w.pml_width_x, pml_wy=w.pml_width_y, pml_type=w.pml_type,
            sigma0=w.sigma0, theta=w.theta, precision=precision, stream=stream)
        if scheme != DIRAC_SCHEME_II:
            dirac_set_scheme(self.ctx, scheme)
        if poly_degree is not None:
            dirac_set_poly_degree(self.ctx, poly_degree)

    def set_state(self, psi):
        dirac_set_state(self.ctx, psi)

    def get_state(self):
        out = np.empty((2, self.ny, self.nx), dtype=np.complex128)
        return dirac_get_state(self.ctx, out)

    def step(self, n, dt):
        dirac_step(self.ctx, n, dt)

    def observables(self, with_density=False):
        dens = np.empty((self.ny, self.nx)) if with_density else None
        r = dirac_observables(self.ctx, dens)
        if with_density:
            r["density"] = dens
        return r

    def close(self):
        dirac_destroy(self.ctx)
        self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
