"""Parity of Scheme I (Crank-Nicolson middle step, restarted GMRES; eq. cn) on the GPU
with the FP64 CPU oracle's Scheme I.

Both solve the same linear system each step to a relative residual below their
tolerance (oracle 1e-14; GPU 1e-14 in complex128, 3e-7 in complex64), so they agree to
rel-L2 1e-11 (complex128) and 1e-5 (complex64).
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
CN = D.DIRAC_SCHEME_CRANK_NICOLSON


@pytest.fixture(scope="module", autouse=True)
def _built():
    D.build()
    oracle.build()


def gpu_run(w, prec, steps, dt=None, calls=None, restart=20):
    with D.Simulation(w, precision=prec, scheme=CN) as s:
        D.dirac_set_krylov(s.ctx, 0.0, restart, 100)
        s.set_state(w.psi0)
        for n in (calls or [steps]):
            s.step(n, w.dt if dt is None else dt)
        return s.get_state(), D.dirac_krylov_iterations(s.ctx)


def oracle_run(w, steps, dt=None):
    psi, _ = oracle.run_cn(oracle.Problem.from_workload(w), w.psi0, w.dt if dt is None else dt,
                           steps, tol=1e-14)
    return psi


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_plain_128_cn_matches_oracle(prec):
    w = W.plain_128()
    steps = 100 if prec == D.DIRAC_C128 else 40
    ref = oracle_run(w, steps)
    got, iters = gpu_run(w, prec, steps)
    assert_parity(got, ref, w, TOL[prec])
    assert iters >= steps


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_cn_curved_metric_layer_mass_split_calls(prec):
    w = W.graphene_strained(n=256, steps=30)
    w.mass = 0.3
    ref = oracle_run(w, 30)
    got, _ = gpu_run(w, prec, 30, calls=[5, 10, 15])
    assert_parity(got, ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("nx,ny", [(16, 64), (256, 32), (64, 512)])
def test_cn_rectangular_grids(prec, nx, ny):
    ax, ay = 0.2 * nx, 0.2 * ny
    X, Y = W.mesh(nx, ny, ax, ay)
    g11 = 1.0 + 0.2 * np.exp(-(X ** 2 + Y ** 2) / (0.1 * ax * ay))
    g22 = 1.0 + 0.1 * np.exp(-((X - 0.1 * ax) ** 2 + Y ** 2) / (0.2 * ax * ay))
    psi0 = W.wave_packet(nx, ny, ax, ay, 0.1 * min(ax, ay) + 0.5, (0.8, 0.3))
    w = W.Workload("grid", nx, ny, ax, ay, np.ones_like(X), g11, g22, mass=0.2, c=1.0,
                   pml_width_x=max(1, nx // 16), pml_width_y=max(1, ny // 16), pml_type=1,
                   sigma0=0.5, theta=0.0, psi0=psi0, dt=0.05, steps=5)
    ref = oracle_run(w, 5)
    got, _ = gpu_run(w, prec, 5)
    assert_parity(got, ref, w, TOL[prec])


def test_cn_conserves_the_norm_in_flat_space_with_a_short_restart():
    """Flat space, complex128: the Cayley step is unitary (Prop. 5.1); a Krylov dimension
    of 3 forces restarts."""
    n, a = 64, 10.0
    psi0 = W.wave_packet(n, n, a, a, 1.5, (1.0, -0.5))
    ones = np.ones((n, n))
    w = W.Workload("flat", n, n, a, a, ones, ones, ones, mass=0.5, c=1.0, pml_width_x=0,
                   pml_width_y=0, pml_type=1, sigma0=1.0, theta=0.0, psi0=psi0, dt=0.2,
                   steps=10)
    got, _ = gpu_run(w, D.DIRAC_C128, 10, restart=3)
    assert abs(np.linalg.norm(got) / np.linalg.norm(psi0) - 1.0) <= 1e-11
    ref = oracle_run(w, 10)
    assert_parity(got, ref, w, 1e-11)


def test_cn_reports_non_convergence():
    """No restarts and a one-vector basis cannot reach the tolerance: DIRAC_ENOCONV."""
    w = W.plain_128()
    with D.Simulation(w, precision=D.DIRAC_C128, scheme=CN) as s:
        D.dirac_set_krylov(s.ctx, 1e-14, 1, 0)
        s.set_state(w.psi0)
        with pytest.raises(D.DiracError) as e:
            s.step(1, w.dt)
        assert e.value.status == D.DIRAC_ENOCONV
    with pytest.raises(D.DiracError):
        with D.Simulation(w, precision=D.DIRAC_C64) as s:
            D.dirac_set_krylov(s.ctx, 1e-8, 0, 5)
