"""FP64 CPU oracle for Scheme II (arXiv:1909.02894), loaded through ctypes.

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg import this package. The product path (the CUDA library and its
binding) never does. The oracle shares no code with the CUDA path.

``build()`` compiles ``dirac_oracle.c`` with gcc (``-O3 -ffp-contract=off -fopenmp``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "dirac_oracle.c")

CONN_COVARIANT, CONN_PAPER_2D, CONN_NONE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (idempotent)."""
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(os.path.join(HERE, "dirac_oracle.h"))):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("ax", C.c_double), ("ay", C.c_double),
        ("mass", C.c_double), ("c", C.c_double),
        ("conn", C.c_int),
        ("pml_wx", C.c_int), ("pml_wy", C.c_int), ("pml_type", C.c_int),
        ("sigma0", C.c_double), ("theta", C.c_double),
        ("V", C.c_void_p), ("Ax", C.c_void_p), ("Ay", C.c_void_p),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        P = C.POINTER(_Params)
        dp = C.c_void_p
        L.oracle_fft.argtypes = [C.c_int, dp, C.c_int]
        L.oracle_deriv.argtypes = [P, C.c_int, dp, dp]
        L.oracle_coefficients.argtypes = [P, dp, dp, dp] + [dp] * 8
        L.oracle_half_step.argtypes = [P, dp, dp, dp, C.c_double, dp]
        L.oracle_run.argtypes = [P, dp, dp, dp, C.c_double, C.c_long, dp]
        L.oracle_observables.argtypes = [P, dp, dp, dp, dp, dp, dp]
        L.oracle_modes_evolve.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double,
                                          C.c_long, C.c_int, dp, dp, dp, C.c_int, dp, dp, dp]
        L.oracle_run_scheme.argtypes = [P, dp, dp, dp, C.c_double, C.c_long, C.c_int, dp]
        L.oracle_apply_A.argtypes = [P, dp, dp, dp, dp, dp]
        L.oracle_bessel_j.argtypes = [C.c_double, C.c_int, dp]
        L.oracle_run_poly.argtypes = [P, dp, dp, dp, C.c_double, C.c_long, C.c_int, C.c_int, dp]
        L.oracle_run_cn.argtypes = [P, dp, dp, dp, C.c_double, C.c_long, C.c_double, C.c_int,
                                    C.c_int, C.POINTER(C.c_long), dp]
        L.oracle_modes_evolve_scheme.argtypes = [P, C.c_double, C.c_double, C.c_double,
                                                 C.c_double, C.c_long, C.c_int, C.c_int, dp,
                                                 dp, dp, C.c_int, dp, dp, dp]
        L.oracle_threads.argtypes = []
        L.oracle_set_threads.argtypes = [C.c_int]
        for f in ("oracle_fft", "oracle_deriv", "oracle_coefficients", "oracle_half_step",
                  "oracle_run", "oracle_observables", "oracle_modes_evolve", "oracle_threads",
                  "oracle_run_scheme", "oracle_modes_evolve_scheme", "oracle_apply_A",
                  "oracle_bessel_j", "oracle_run_poly", "oracle_run_cn",
                  "oracle_set_threads"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == shape, (a.shape, shape)
    return a


@dataclass
class Problem:
    """The run parameters of one simulation, as the oracle reads them."""

    nx: int
    ny: int
    ax: float
    ay: float
    mass: float = 0.0
    c: float = 1.0
    conn: int = CONN_COVARIANT
    pml_wx: int = 0
    pml_wy: int = 0
    pml_type: int = 1
    sigma0: float = 1.0
    theta: float = 0.0
    g00: np.ndarray = None
    g11: np.ndarray = None
    g22: np.ndarray = None
    V: np.ndarray = None   # static potentials (None = 0), see oracle_params
    Ax: np.ndarray = None
    Ay: np.ndarray = None

    @classmethod
    def from_workload(cls, w, conn=None):
        return cls(nx=w.nx, ny=w.ny, ax=w.ax, ay=w.ay, mass=w.mass, c=w.c,
                   conn=w.conn if conn is None else conn, pml_wx=w.pml_width_x,
                   pml_wy=w.pml_width_y, pml_type=w.pml_type, sigma0=w.sigma0,
                   theta=w.theta, g00=w.g00, g11=w.g11, g22=w.g22,
                   V=getattr(w, "V", None), Ax=getattr(w, "Ax", None), Ay=getattr(w, "Ay", None))

    def _params(self):
        s = (self.ny, self.nx)
        # the arrays must outlive the call that receives the struct: keep them here
        self._pot = [None if f is None else np.ascontiguousarray(f, dtype=np.float64).reshape(s)
                     for f in (self.V, self.Ax, self.Ay)]
        ptrs = [None if f is None else f.ctypes.data for f in self._pot]
        return _Params(self.nx, self.ny, self.ax, self.ay, self.mass, self.c, self.conn,
                       self.pml_wx, self.pml_wy, self.pml_type, self.sigma0, self.theta, *ptrs)

    def _g(self):
        s = (self.ny, self.nx)
        return _f64(self.g00, s), _f64(self.g11, s), _f64(self.g22, s)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def fft(x, inverse=False):
    y = np.ascontiguousarray(x, dtype=np.complex128).copy()
    _check(lib().oracle_fft(y.size, _ptr(y), int(inverse)), "fft")
    return y


def deriv(prob: Problem, f, axis):
    f = np.ascontiguousarray(f, dtype=np.complex128)
    out = np.empty_like(f)
    p = prob._params()
    _check(lib().oracle_deriv(C.byref(p), axis, _ptr(f), _ptr(out)), "deriv")
    return out


def coefficients(prob: Problem):
    n = (prob.ny, prob.nx)
    out = {k: np.empty(n) for k in ("a1", "a2", "meff", "w", "omx", "omy")}
    out["b1"] = np.empty(n, dtype=np.complex128)
    out["b2"] = np.empty(n, dtype=np.complex128)
    g = prob._g()
    p = prob._params()
    _check(lib().oracle_coefficients(
        C.byref(p), *[_ptr(x) for x in g],
        *[_ptr(out[k]) for k in ("a1", "a2", "meff", "w", "omx", "omy", "b1", "b2")]),
        "coefficients")
    return out


def half_step(prob: Problem, dt):
    u = np.empty((prob.ny, prob.nx, 4), dtype=np.complex128)
    g = prob._g()
    p = prob._params()
    _check(lib().oracle_half_step(C.byref(p), *[_ptr(x) for x in g], dt, _ptr(u)), "half_step")
    return u.reshape(prob.ny, prob.nx, 2, 2)


SCHEME_II, SCHEME_II_SYMMETRIC = 0, 1


def run(prob: Problem, psi, dt, n_steps, scheme=SCHEME_II):
    """n_steps of Scheme II (Sec. 5.2) or of its symmetric sub-step order."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    assert psi.shape == (2, prob.ny, prob.nx)
    g = prob._g()
    p = prob._params()
    _check(lib().oracle_run_scheme(C.byref(p), *[_ptr(x) for x in g], dt, int(n_steps),
                                   int(scheme), _ptr(psi)), "run")
    return psi


POLY_TAYLOR, POLY_CHEBYSHEV = 0, 1


def apply_A(prob: Problem, psi):
    """A psi = - sum_j b^j sigma_j [[d_j]] psi (the unsplit middle-step operator)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    _check(lib().oracle_apply_A(C.byref(prob._params()), *[_ptr(x) for x in prob._g()],
                                _ptr(psi), _ptr(out)), "apply_A")
    return out


def bessel_j(x, n):
    out = np.empty(n + 1)
    _check(lib().oracle_bessel_j(float(x), int(n), _ptr(out)), "bessel_j")
    return out


def run_poly(prob: Problem, psi, dt, n_steps, family=POLY_CHEBYSHEV, order=8):
    """n_steps of the polynomial scheme (eq. poly) with a Taylor or Chebyshev middle step."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    _check(lib().oracle_run_poly(C.byref(prob._params()), *[_ptr(x) for x in prob._g()],
                                 float(dt), int(n_steps), int(family), int(order), _ptr(psi)),
           "run_poly")
    return psi


def run_cn(prob: Problem, psi, dt, n_steps, tol=1e-13, restart=30, max_restarts=100):
    """n_steps of Scheme I (Crank-Nicolson, GMRES); returns (psi, Arnoldi steps)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    it = C.c_long(0)
    rc = lib().oracle_run_cn(C.byref(prob._params()), *[_ptr(x) for x in prob._g()], float(dt),
                             int(n_steps), float(tol), int(restart), int(max_restarts),
                             C.byref(it), _ptr(psi))
    if rc == -2:
        raise RuntimeError("oracle GMRES did not converge")
    _check(rc, "run_cn")
    return psi, it.value


def observables(prob: Problem, psi, with_density=False):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    obs = np.empty(4)
    dens = np.empty((prob.ny, prob.nx)) if with_density else None
    g = prob._g()
    p = prob._params()
    _check(lib().oracle_observables(C.byref(p), *[_ptr(x) for x in g], _ptr(psi), _ptr(obs),
                                    _ptr(dens)), "observables")
    res = {"norm": obs[0], "norm_gamma": obs[1], "energy": obs[2], "energy_imag": obs[3]}
    if with_density:
        res["density"] = dens
    return res


def modes_evolve(prob: Problem, g00, g11, g22, dt, n_steps, modes, ix, iy, scheme=SCHEME_II):
    """modes = [(qx, qy, (A1, A2))]; returns [len(ix)][2] complex."""
    qx = np.array([m[0] for m in modes], dtype=np.int32)
    qy = np.array([m[1] for m in modes], dtype=np.int32)
    amps = np.array([m[2] for m in modes], dtype=np.complex128).reshape(-1)
    ix = np.ascontiguousarray(ix, dtype=np.int32)
    iy = np.ascontiguousarray(iy, dtype=np.int32)
    out = np.empty((ix.size, 2), dtype=np.complex128)
    p = prob._params()
    _check(lib().oracle_modes_evolve_scheme(C.byref(p), g00, g11, g22, dt, int(n_steps),
                                            int(scheme), len(modes), _ptr(qx), _ptr(qy),
                                            _ptr(amps), ix.size, _ptr(ix), _ptr(iy),
                                            _ptr(out)), "modes_evolve")
    return out


def threads() -> int:
    return lib().oracle_threads()


def set_threads(n: int) -> None:
    """Number of OpenMP threads for later oracle calls (for single-thread timing)."""
    _check(lib().oracle_set_threads(int(n)), "set_threads")
