"""Static electromagnetic potentials (the F of the curved-space Hamiltonian, Sec. 2) on the
GPU against the FP64 CPU oracle, in every time-step scheme.

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


@pytest.fixture(scope="module", autouse=True)
def _built():
    D.build()
    oracle.build()


def fields(w):
    X, Y = W.mesh(w.nx, w.ny, w.ax, w.ay)
    V = 0.4 * np.exp(-(X ** 2 + Y ** 2) / (0.1 * w.ax * w.ay))
    Ax = 0.3 * np.cos(np.pi * Y / w.ay)
    Ay = -0.2 * X / w.ax
    return V, Ax, Ay


def gpu_run(w, prec, steps, scheme=D.DIRAC_SCHEME_II, calls=None, pot=None):
    with D.Simulation(w, precision=prec, scheme=scheme) as s:
        V, Ax, Ay = fields(w) if pot is None else pot
        D.dirac_set_potentials(s.ctx, V, Ax, Ay, shape=(w.ny, w.nx))
        s.set_state(w.psi0)
        for n in (calls or [steps]):
            s.step(n, w.dt)
        return s.get_state()


def oracle_problem(w, pot=None):
    prob = oracle.Problem.from_workload(w)
    prob.V, prob.Ax, prob.Ay = fields(w) if pot is None else pot
    return prob


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("calls", [[200], [50, 70, 80]], ids=["one-call", "three-calls"])
def test_scheme_ii_with_potentials(prec, calls):
    w = W.graphene_strained(n=128, steps=200)
    w.mass = 0.3
    ref = oracle.run(oracle_problem(w), w.psi0, w.dt, 200)
    assert_parity(gpu_run(w, prec, 200, calls=calls), ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_symmetric_order_with_potentials(prec):
    w = W.plain_128(steps=100)
    ref = oracle.run(oracle_problem(w), w.psi0, w.dt, 100, scheme=oracle.SCHEME_II_SYMMETRIC)
    got = gpu_run(w, prec, 100, scheme=D.DIRAC_SCHEME_II_SYMMETRIC)
    assert_parity(got, ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_polynomial_and_cn_with_potentials(prec):
    w = W.plain_128(steps=30)
    ref = oracle.run_poly(oracle_problem(w), w.psi0, w.dt, 30, oracle.POLY_CHEBYSHEV, 8)
    got = gpu_run(w, prec, 30, scheme=D.DIRAC_SCHEME_POLY_CHEBYSHEV)
    assert_parity(got, ref, w, TOL[prec])
    ref, _ = oracle.run_cn(oracle_problem(w), w.psi0, w.dt, 30, tol=1e-14)
    got = gpu_run(w, prec, 30, scheme=D.DIRAC_SCHEME_CRANK_NICOLSON)
    assert_parity(got, ref, w, TOL[prec])


def test_constant_scalar_potential_is_a_phase_on_the_gpu():
    """A constant V multiplies the V = 0 result by exp(-i V n dt) (4096^2 complex64,
    persistent passes, U outside the passes)."""
    w = W.large_4096(steps=20)
    with D.Simulation(w, precision=D.DIRAC_C64) as s:
        s.set_state(w.psi0)
        s.step(20, w.dt)
        ref = s.get_state()
        D.dirac_set_potentials(s.ctx, np.full((w.ny, w.nx), 0.7), None, None)
        s.set_state(w.psi0)
        s.step(20, w.dt)
        got = s.get_state()
    assert W.rel_l2(got, np.exp(-1j * 0.7 * 20 * w.dt) * ref) <= 1e-5


def test_potentials_can_be_removed_and_batches_refuse_them():
    w = W.plain_128(steps=10)
    ref = oracle.run(oracle.Problem.from_workload(w), w.psi0, w.dt, 10)
    with D.Simulation(w, precision=D.DIRAC_C128) as s:
        D.dirac_set_potentials(s.ctx, *fields(w))
        s.set_state(w.psi0)
        b = D.dirac_batch_create(1 << 30, D.DIRAC_C128, 8, None)
        try:
            with pytest.raises(D.DiracError) as e:
                D.dirac_batch_submit(b, s.ctx, 10, w.dt)
            assert e.value.status == D.DIRAC_EUNSUPPORTED
        finally:
            D.dirac_batch_destroy(b)
        D.dirac_set_potentials(s.ctx, None, None, None)
        s.set_state(w.psi0)
        s.step(10, w.dt)
        assert_parity(s.get_state(), ref, w, 1e-11)
        with pytest.raises(D.DiracError):
            D.dirac_set_potentials(s.ctx, np.full((w.ny, w.nx), np.nan), None, None)


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_energy_with_potentials_matches_oracle(prec):
    w = W.graphene_strained(n=128, steps=10)
    w.mass = 0.3
    psi = w.psi0 + 0.05 * W.random_state(w.nx, w.ny, 8)
    ref = oracle.observables(oracle_problem(w), psi)
    with D.Simulation(w, precision=prec) as s:
        D.dirac_set_potentials(s.ctx, *fields(w))
        s.set_state(psi)
        got = s.observables()
    tol = 1e-11 if prec == D.DIRAC_C128 else 1e-5
    for k in ("norm", "norm_gamma", "energy"):
        assert abs(got[k] - ref[k]) <= tol * abs(ref[k]), (k, got[k], ref[k])
