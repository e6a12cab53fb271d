"""Parity of the symmetric sub-step order (U, x over dt/2, y over dt, x over dt/2, U) of
Scheme II on the GPU with the FP64 CPU oracle's implementation of the same order.

Tolerances as for the printed order: rel-L2 1e-11 (complex128) and 1e-5 (complex64)
after up to 1000 steps; full-size grids on a few steps against the whole oracle grid and
over 1000 steps through the exact per-mode solution of a constant metric.
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
SYM = D.DIRAC_SCHEME_II_SYMMETRIC


@pytest.fixture(scope="module", autouse=True)
def _built():
    D.build()
    oracle.build()


def gpu_run(w, prec, steps, dt=None, psi0=None, calls=1):
    with D.Simulation(w, precision=prec, scheme=SYM) as s:
        s.set_state(w.psi0 if psi0 is None else psi0)
        per = steps // calls
        for k in range(calls):
            s.step(per if k + 1 < calls else steps - per * (calls - 1), w.dt if dt is None else dt)
        return s.get_state()


def oracle_run(w, steps, psi0=None):
    return oracle.run(oracle.Problem.from_workload(w), w.psi0 if psi0 is None else psi0, w.dt,
                      steps, scheme=oracle.SCHEME_II_SYMMETRIC)


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("steps", [1, 2, 1000])
def test_plain_128_symmetric_matches_oracle(prec, steps):
    w = W.plain_128()
    ref = oracle_run(w, steps)
    assert_parity(gpu_run(w, prec, steps), ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_symmetric_split_into_several_calls(prec):
    """U is merged across steps inside a call and applied as a half step at each end of a
    call: 3 calls of 20, 30 and 50 steps give the 100-step result."""
    w = W.graphene_strained(n=128, steps=100)
    w.mass = 0.3
    ref = oracle_run(w, 100)
    with D.Simulation(w, precision=prec, scheme=SYM) as s:
        s.set_state(w.psi0)
        for n in (20, 30, 50):
            s.step(n, w.dt)
        got = s.get_state()
    assert_parity(got, ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("nx,ny", [(16, 16), (64, 32), (256, 16), (16, 512), (128, 1024),
                                   (2048, 32), (4096, 16), (32, 4096)])
def test_symmetric_every_line_length_and_aspect(prec, nx, ny):
    """Both store layouts of every line length (the last x pass writes rows back in the
    input layout), curved metric, mass, absorbing layer, covariant connection."""
    rng = np.random.default_rng(nx * 5 + ny)
    ax, ay = 0.15 * nx, 0.15 * ny
    X, Y = W.mesh(nx, ny, ax, ay)
    g11 = 1.0 + 0.2 * np.exp(-((X - 0.1 * ax) ** 2 + Y ** 2) / (0.2 * ax * ay))
    g22 = 1.0 + 0.1 * np.exp(-(X ** 2 + (Y + 0.1 * ay) ** 2) / (0.3 * ax * ay))
    g00 = 1.0 + 0.05 * np.exp(-(X ** 2 + Y ** 2) / (0.4 * ax * ay))
    psi0 = W.wave_packet(nx, ny, ax, ay, 0.1 * min(ax, ay) + 0.5, (1.0, -0.7))
    psi0 += 0.01 * W.random_state(nx, ny, int(rng.integers(1 << 30)))
    w = W.Workload("grid", nx, ny, ax, ay, g00, g11, g22, mass=0.4, c=1.0,
                   pml_width_x=max(1, nx // 16), pml_width_y=max(1, ny // 16), pml_type=1,
                   sigma0=0.5, theta=0.0, psi0=psi0, dt=0.05, steps=5)
    ref = oracle_run(w, 5)
    assert_parity(gpu_run(w, prec, 5), ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_symmetric_strained_graphene_1024(prec):
    w = W.graphene_strained(n=1024, steps=6)
    ref = oracle_run(w, 6)
    assert_parity(gpu_run(w, prec, 6), ref, w, TOL[prec])


def test_symmetric_large_4096_c64_vs_oracle():
    """The 4096^2 complex64 benchmark grid (persistent passes, both store layouts)."""
    w = W.large_4096(steps=2)
    ref = oracle_run(w, 2)
    assert_parity(gpu_run(w, D.DIRAC_C64, 2), ref, w, TOL[D.DIRAC_C64])


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("n", [256, 4096])
def test_symmetric_constant_metric_1000_steps_exact_modes(prec, n):
    a = 0.1 * n
    modes = [(3, 1, (0.7, 0.2j)), (n - 5, 7, (0.1 - 0.3j, 0.4)), (n // 2, n - 2, (0.05, 0.02)),
             (11, n // 2, (0.0, 0.3))]
    psi0 = W.plane_waves(n, n, a, a, modes)
    g = (1.1, 0.9, 1.2)
    w = W.Workload("const", n, n, a, a, np.full((n, n), g[0]), np.full((n, n), g[1]),
                   np.full((n, n), g[2]), mass=0.6, c=1.0, pml_width_x=0, pml_width_y=0,
                   pml_type=1, sigma0=1.0, theta=0.0, psi0=psi0, dt=0.02, steps=1000)
    got = gpu_run(w, prec, 1000)
    rng = np.random.default_rng(n + 1)
    ix = rng.integers(0, n, 4096)
    iy = rng.integers(0, n, 4096)
    prob = oracle.Problem.from_workload(w)
    ref = oracle.modes_evolve(prob, *g, w.dt, 1000, modes, ix, iy,
                              scheme=oracle.SCHEME_II_SYMMETRIC)
    sampled = np.stack([got[0][iy, ix], got[1][iy, ix]], axis=1)
    err = np.linalg.norm(sampled - ref) / np.linalg.norm(ref)
    assert err <= TOL[prec]


def test_scheme_switch_and_batch_guard():
    """Switching the order back gives the printed order's result; a batch refuses a
    context in the symmetric order; three launches per symmetric step."""
    w = W.plain_128()
    ref = oracle.run(oracle.Problem.from_workload(w), w.psi0, w.dt, 10)
    with D.Simulation(w, precision=D.DIRAC_C128, scheme=SYM) as s:
        s.set_state(w.psi0)
        n0 = D.dirac_launch_count(s.ctx)
        s.step(4, w.dt)
        assert D.dirac_launch_count(s.ctx) - n0 >= 12
        D.dirac_set_scheme(s.ctx, D.DIRAC_SCHEME_II)
        s.set_state(w.psi0)
        s.step(10, w.dt)
        assert_parity(s.get_state(), ref, w, 1e-11)
        D.dirac_set_scheme(s.ctx, SYM)
        b = D.dirac_batch_create(1 << 30, D.DIRAC_C128, 8, None)
        try:
            with pytest.raises(D.DiracError) as e:
                D.dirac_batch_submit(b, s.ctx, 10, w.dt)
            assert e.value.status == D.DIRAC_EUNSUPPORTED
        finally:
            D.dirac_batch_destroy(b)
    with pytest.raises(D.DiracError):
        with D.Simulation(w, precision=D.DIRAC_C64) as s:
            D.dirac_set_scheme(s.ctx, 7)


def test_symmetric_is_second_order_on_the_gpu():
    """Flat space, complex128: against the exact free propagator exp(-i T H(xi)) the
    symmetric order's error falls as dt^2 (the printed order's as dt)."""
    n, a, mass, T = 64, 10.0, 0.5, 1.0
    psi0 = W.wave_packet(n, n, a, a, 1.5, (1.0, -0.5))
    psi0[1] = 0.5j * psi0[0]
    ones = np.ones((n, n))
    w = W.Workload("flat", n, n, a, a, ones, ones, ones, mass=mass, c=1.0, pml_width_x=0,
                   pml_width_y=0, pml_type=1, sigma0=1.0, theta=0.0, psi0=psi0, dt=0.04,
                   steps=25)
    xs = np.fft.fftfreq(n, d=2 * a / n) * 2 * np.pi
    KX, KY = np.meshgrid(xs, xs, indexing="xy")
    E = np.sqrt(KX ** 2 + KY ** 2 + mass ** 2)
    h0, h1 = np.fft.fft2(psi0[0]), np.fft.fft2(psi0[1])
    cs, sn = np.cos(T * E), np.sin(T * E) / E
    r0 = cs * h0 - 1j * sn * (mass * h0 + (KX - 1j * KY) * h1)
    r1 = cs * h1 - 1j * sn * ((KX + 1j * KY) * h0 - mass * h1)
    exact = np.stack([np.fft.ifft2(r0), np.fft.ifft2(r1)])
    errs = [W.rel_l2(gpu_run(w, D.DIRAC_C128, int(round(T / dt)), dt=dt), exact)
            for dt in (0.04, 0.02, 0.01)]
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o - 2.0) <= 0.15 for o in orders), (errs, orders)
