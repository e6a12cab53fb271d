"""Parity of the polynomial scheme (eq. poly: U, unsplit middle step sum_q a_q P_q(dt A),
U) on the GPU with the FP64 CPU oracle, for the Taylor and the Chebyshev middle step.

Tolerances: rel-L2 1e-11 (complex128) and 1e-5 (complex64).
"""
import numpy as np
import pytest

import oracle
import paper_1909_02894_gb300 as D
from paper_1909_02894_gb300 import workloads as W
from parity_util import assert_parity

pytestmark = pytest.mark.gpu

TOL = {D.DIRAC_C128: 1e-11, D.DIRAC_C64: 1e-5}
PREC = [D.DIRAC_C128, D.DIRAC_C64]
PID = ["c128", "c64"]
FAM = {"taylor": (D.DIRAC_SCHEME_POLY_TAYLOR, oracle.POLY_TAYLOR),
       "chebyshev": (D.DIRAC_SCHEME_POLY_CHEBYSHEV, oracle.POLY_CHEBYSHEV)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    D.build()
    oracle.build()


def gpu_run(w, prec, steps, family, degree, dt=None, calls=(None,)):
    with D.Simulation(w, precision=prec, scheme=FAM[family][0], poly_degree=degree) as s:
        s.set_state(w.psi0)
        if calls == (None,):
            s.step(steps, w.dt if dt is None else dt)
        else:
            for n in calls:
                s.step(n, w.dt if dt is None else dt)
        return s.get_state()


def oracle_run(w, steps, family, degree, dt=None):
    return oracle.run_poly(oracle.Problem.from_workload(w), w.psi0, w.dt if dt is None else dt,
                           steps, FAM[family][1], degree)


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("family,degree", [("taylor", 4), ("taylor", 6), ("chebyshev", 6),
                                           ("chebyshev", 10)])
def test_plain_128_poly_matches_oracle(prec, family, degree):
    w = W.plain_128()
    steps = 200
    ref = oracle_run(w, steps, family, degree)
    assert_parity(gpu_run(w, prec, steps, family, degree), ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("family", ["taylor", "chebyshev"])
def test_poly_curved_metric_layer_mass_split_calls(prec, family):
    """Strained metric with a spin connection, mass and absorbing layer; U^2 merging
    across the steps of a call and half steps at the ends of each call."""
    w = W.graphene_strained(n=256, steps=60)
    w.mass = 0.3
    ref = oracle_run(w, 60, family, 8)
    got = gpu_run(w, prec, 60, family, 8, calls=(10, 20, 30))
    assert_parity(got, ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("nx,ny", [(16, 64), (256, 32), (64, 1024), (2048, 16)])
def test_poly_rectangular_grids(prec, nx, ny):
    ax, ay = 0.2 * nx, 0.2 * ny
    X, Y = W.mesh(nx, ny, ax, ay)
    g11 = 1.0 + 0.2 * np.exp(-(X ** 2 + Y ** 2) / (0.1 * ax * ay))
    g22 = 1.0 + 0.1 * np.exp(-((X - 0.1 * ax) ** 2 + Y ** 2) / (0.2 * ax * ay))
    psi0 = W.wave_packet(nx, ny, ax, ay, 0.1 * min(ax, ay) + 0.5, (0.8, 0.3))
    w = W.Workload("grid", nx, ny, ax, ay, np.ones_like(X), g11, g22, mass=0.2, c=1.0,
                   pml_width_x=max(1, nx // 16), pml_width_y=max(1, ny // 16), pml_type=1,
                   sigma0=0.5, theta=0.0, psi0=psi0, dt=0.02, steps=5)
    ref = oracle_run(w, 5, "chebyshev", 8)
    assert_parity(gpu_run(w, prec, 5, "chebyshev", 8), ref, w, TOL[prec])


def test_chebyshev_reaches_the_free_propagator_on_the_gpu():
    """Flat space, m = 0, complex128: enough Chebyshev terms reproduce exp(-i T H(xi))."""
    n, a, T = 64, 10.0, 1.0
    psi0 = W.wave_packet(n, n, a, a, 1.5, (1.0, -0.5))
    psi0[1] = 0.5j * psi0[0]
    ones = np.ones((n, n))
    w = W.Workload("flat", n, n, a, a, ones, ones, ones, mass=0.0, c=1.0, pml_width_x=0,
                   pml_width_y=0, pml_type=1, sigma0=1.0, theta=0.0, psi0=psi0, dt=0.1,
                   steps=10)
    xs = np.fft.fftfreq(n, d=2 * a / n) * 2 * np.pi
    KX, KY = np.meshgrid(xs, xs, indexing="xy")
    E = np.sqrt(KX ** 2 + KY ** 2) + 1e-300
    h0, h1 = np.fft.fft2(psi0[0]), np.fft.fft2(psi0[1])
    cs, sn = np.cos(T * E), np.sin(T * E) / E
    r0 = cs * h0 - 1j * sn * ((KX - 1j * KY) * h1)
    r1 = cs * h1 - 1j * sn * ((KX + 1j * KY) * h0)
    exact = np.stack([np.fft.ifft2(r0), np.fft.ifft2(r1)])
    got = gpu_run(w, D.DIRAC_C128, 10, "chebyshev", 24)
    assert_parity(got, exact, w, 1e-11)


def test_poly_degree_validation_and_batch_guard():
    w = W.plain_128()
    with D.Simulation(w, precision=D.DIRAC_C64, scheme=D.DIRAC_SCHEME_POLY_CHEBYSHEV) as s:
        for bad in (0, 257, -3):
            with pytest.raises(D.DiracError):
                D.dirac_set_poly_degree(s.ctx, bad)
        s.set_state(w.psi0)
        b = D.dirac_batch_create(1 << 30, D.DIRAC_C64, 8, None)
        try:
            with pytest.raises(D.DiracError) as e:
                D.dirac_batch_submit(b, s.ctx, 10, w.dt)
            assert e.value.status == D.DIRAC_EUNSUPPORTED
        finally:
            D.dirac_batch_destroy(b)
