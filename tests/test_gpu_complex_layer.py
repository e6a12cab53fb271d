"""Complex stretching of the absorbing layer (S = 1 + exp(i theta) Sigma~, Sec. 3),
complex128, against the FP64 CPU oracle in every time-step scheme (rel-L2 1e-11)."""
import numpy as np
import pytest

import oracle
import paper_1909_02894_gb300 as D
from paper_1909_02894_gb300 import workloads as W
from parity_util import assert_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    D.build()
    oracle.build()


def layer_workload(ptype, theta, n=128, steps=60):
    w = W.graphene_strained(n=n, steps=steps)
    w.pml_type = ptype
    w.theta = theta
    w.mass = 0.2
    return w


def gpu_run(w, steps, scheme=D.DIRAC_SCHEME_II):
    with D.Simulation(w, precision=D.DIRAC_C128, scheme=scheme) as s:
        s.set_state(w.psi0)
        s.step(steps, w.dt)
        return s.get_state()


@pytest.mark.parametrize("ptype", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("theta", [0.4, -0.9])
def test_scheme_ii_complex_layer(ptype, theta):
    w = layer_workload(ptype, theta)
    ref = oracle.run(oracle.Problem.from_workload(w), w.psi0, w.dt, 60)
    assert_parity(gpu_run(w, 60), ref, w, 1e-11)


def test_other_schemes_complex_layer():
    w = layer_workload(1, 0.5, steps=20)
    prob = oracle.Problem.from_workload(w)
    ref = oracle.run(prob, w.psi0, w.dt, 20, scheme=oracle.SCHEME_II_SYMMETRIC)
    assert_parity(gpu_run(w, 20, D.DIRAC_SCHEME_II_SYMMETRIC), ref, w, 1e-11)
    ref = oracle.run_poly(prob, w.psi0, w.dt, 20, oracle.POLY_CHEBYSHEV, 8)
    assert_parity(gpu_run(w, 20, D.DIRAC_SCHEME_POLY_CHEBYSHEV), ref, w, 1e-11)
    ref, _ = oracle.run_cn(prob, w.psi0, w.dt, 20, tol=1e-14)
    assert_parity(gpu_run(w, 20, D.DIRAC_SCHEME_CRANK_NICOLSON), ref, w, 1e-11)


def test_complex_layer_rectangular_and_long_lines():
    """4096-point lines in complex128 (non-persistent passes) with a complex layer."""
    nx, ny = 4096, 32
    ax, ay = 0.2 * nx, 0.2 * ny
    X, Y = W.mesh(nx, ny, ax, ay)
    g11 = 1.0 + 0.2 * np.exp(-(X ** 2 + Y ** 2) / (0.1 * ax * ay))
    psi0 = W.wave_packet(nx, ny, ax, ay, 0.05 * ay + 0.5, (0.8, 0.3))
    w = W.Workload("grid", nx, ny, ax, ay, np.ones_like(X), g11, np.ones_like(X), mass=0.2,
                   c=1.0, pml_width_x=nx // 16, pml_width_y=ny // 8, pml_type=2, sigma0=0.5,
                   theta=0.7, psi0=psi0, dt=0.05, steps=5)
    ref = oracle.run(oracle.Problem.from_workload(w), psi0, w.dt, 5)
    assert_parity(gpu_run(w, 5), ref, w, 1e-11)
