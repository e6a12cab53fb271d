"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (rel-L2 over both components and all points): 1e-11 for complex128 and
1e-5 for complex64, after up to 1000 steps. Full-size configurations are checked on
a few steps against the whole oracle grid, and over 1000 steps through the exact
per-mode solution of a constant metric.
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


def gpu_run(w, prec, steps, dt=None, psi0=None, conn=None):
    with D.Simulation(w, precision=prec, conn=conn) as s:
        s.set_state(w.psi0 if psi0 is None else psi0)
        s.step(steps, w.dt if dt is None else dt)
        return s.get_state()


def oracle_run(w, steps, dt=None, psi0=None, conn=None):
    return oracle.run(oracle.Problem.from_workload(w, conn=conn),
                      w.psi0 if psi0 is None else psi0, w.dt if dt is None else dt, steps)


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("steps", [1, 200, 1000])
def test_plain_128_matches_oracle(prec, steps):
    w = W.plain_128()
    ref = oracle_run(w, steps)
    got = gpu_run(w, prec, steps)
    assert_parity(got, ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_plain_128_flat_twin_matches_oracle(prec):
    w = W.plain_128(flat=True)
    ref = oracle_run(w, 200)
    assert_parity(gpu_run(w, prec, 200), ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 16), (16, 64), (64, 32), (256, 16),
                                   (16, 512), (128, 1024), (2048, 32), (4096, 16)])
def test_every_line_length_and_aspect(prec, nx, ny):
    """Each FFT length 16..4096 in both passes, square and rectangular grids, curved
    metric, mass, absorbing layer and the covariant connection."""
    rng = np.random.default_rng(nx * 7 + ny)
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
@pytest.mark.parametrize("conn", [D.DIRAC_CONN_COVARIANT, D.DIRAC_CONN_PAPER_2D, D.DIRAC_CONN_NONE])
@pytest.mark.parametrize("ptype", [1, 2, 3, 4, 5, 6])
def test_connection_modes_and_layer_profiles(prec, conn, ptype):
    w = W.graphene_strained(n=128, steps=50)
    w.pml_type = ptype
    w.g00 = 1.0 + 0.1 * (w.g22 - 1.0)
    w.mass = 0.3
    ref = oracle_run(w, 50, conn=conn)
    assert_parity(gpu_run(w, prec, 50, conn=conn), ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_strained_graphene_full_size_vs_oracle(prec):
    """1024^2 strained graphene (layer 64, non-constant vielbein and connection)."""
    w = W.graphene_strained(n=1024, steps=10)
    ref = oracle_run(w, 10)
    assert_parity(gpu_run(w, prec, 10), ref, w, TOL[prec])


_C2_1000 = {}


def _graphene_1024_oracle_1000():
    """The full-size strained-graphene oracle run over 1000 steps, computed once."""
    if not _C2_1000:
        w = W.graphene_strained(n=1024, steps=1000)
        _C2_1000["w"] = w
        _C2_1000["ref"] = oracle_run(w, 1000)
    return _C2_1000["w"], _C2_1000["ref"]


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_strained_graphene_full_size_1000_steps_vs_oracle(prec):
    """1024^2 strained graphene over 1000 of its 5000 steps against the whole oracle grid
    (Prop. 5.2's convergence regime; the layer keeps the packet's norm over this span)."""
    w, ref = _graphene_1024_oracle_1000()
    assert_parity(gpu_run(w, prec, 1000), ref, w, TOL[prec])


def test_large_4096_c64_full_size_50_steps_vs_oracle():
    """The benchmark's 4096^2 complex64 grid over 50 steps, whole grid, in the benchmark's
    launch configuration."""
    w = W.large_4096(steps=50)
    ref = oracle_run(w, 50)
    assert_parity(gpu_run(w, D.DIRAC_C64, 50), ref, w, TOL[D.DIRAC_C64])


def test_large_4096_c64_full_size_vs_oracle():
    """The benchmark's 4096^2 complex64 grid, in the benchmark's launch configuration."""
    w = W.large_4096(steps=3)
    ref = oracle_run(w, 3)
    assert_parity(gpu_run(w, D.DIRAC_C64, 3), ref, w, TOL[D.DIRAC_C64])


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("n", [256, 4096])
def test_constant_metric_1000_steps_exact_modes(prec, n):
    """Constant metric: plane waves evolve by a per-mode 2x2 matrix power; compare
    sampled points after 1000 steps at any size (the oracle evaluates them one by one)."""
    a = 0.1 * n
    modes = [(3, 1, (0.7, 0.2j)), (n - 5, 7, (0.1 - 0.3j, 0.4)), (n // 2, n - 2, (0.05, 0.02)),
             (11, n // 2, (0.0, 0.3))]
    psi0 = W.plane_waves(n, n, a, a, modes)
    g = (1.1, 0.9, 1.2)
    w = W.Workload("const", n, n, a, a, np.full((n, n), g[0]), np.full((n, n), g[1]),
                   np.full((n, n), g[2]), mass=0.6, c=1.0, pml_width_x=0, pml_width_y=0,
                   pml_type=1, sigma0=1.0, theta=0.0, psi0=psi0, dt=0.02, steps=1000)
    got = gpu_run(w, prec, 1000)
    rng = np.random.default_rng(n)
    ix = rng.integers(0, n, 4096)
    iy = rng.integers(0, n, 4096)
    prob = oracle.Problem.from_workload(w)
    ref = oracle.modes_evolve(prob, *g, w.dt, 1000, modes, ix, iy)
    sub = np.stack([got[0, iy, ix], got[1, iy, ix]], axis=1)
    assert np.linalg.norm(sub - ref) / np.linalg.norm(ref) <= TOL[prec]


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_observables_match_oracle(prec):
    w = W.graphene_strained(n=256, steps=30)
    w.mass = 0.5
    with D.Simulation(w, precision=prec) as s:
        s.set_state(w.psi0)
        s.step(30, w.dt)
        psi = s.get_state()
        got = s.observables(with_density=True)
    ref = oracle.observables(oracle.Problem.from_workload(w), psi, with_density=True)
    tol = 1e-12 if prec == D.DIRAC_C128 else 1e-6
    for k in ("norm", "norm_gamma", "energy"):
        assert abs(got[k] - ref[k]) <= tol * max(1.0, abs(ref[k])), k
    assert abs(got["energy_imag"] - ref["energy_imag"]) <= tol * max(1.0, abs(ref["energy"]))
    assert np.abs(got["density"] - ref["density"]).max() <= tol * ref["density"].max()


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_checkpoint_resume(prec):
    """run(n) equals run(k); get_state; set_state; run(n - k)."""
    w = W.plain_128(n=128)
    full = gpu_run(w, prec, 60)
    with D.Simulation(w, precision=prec) as s:
        s.set_state(w.psi0)
        s.step(25, w.dt)
        mid = s.get_state()
    with D.Simulation(w, precision=prec) as s:
        s.set_state(mid)
        s.step(35, w.dt)
        resumed = s.get_state()
    assert W.rel_l2(resumed, full) <= (1e-13 if prec == D.DIRAC_C128 else 1e-6)


def test_set_get_roundtrip_and_device_pointers():
    torch = pytest.importorskip("torch")
    w = W.plain_128(n=64)
    for prec in PREC:
        with D.Simulation(w, precision=prec) as s:
            dev = torch.from_numpy(w.psi0.copy()).cuda()
            s.set_state(dev)
            out = torch.empty_like(dev)
            D.dirac_get_state(s.ctx, out)
            torch.cuda.synchronize()
            host = s.get_state()
            exp = w.psi0 if prec == D.DIRAC_C128 else w.psi0.astype(np.complex64).astype(np.complex128)
            assert np.array_equal(host, exp)
            assert np.array_equal(out.cpu().numpy(), exp)


def test_step_before_state_and_nonfinite_state():
    w = W.plain_128(n=32)
    with D.Simulation(w, precision=D.DIRAC_C128) as s:
        with pytest.raises(D.DiracError) as e:
            s.step(1, 0.01)
        assert e.value.status == D.DIRAC_ESTATE
        bad = w.psi0.copy()
        bad[0, 3, 4] = np.nan
        s.set_state(bad)
        with pytest.raises(D.DiracError) as e:
            s.observables()
        assert e.value.status == D.DIRAC_ENONFINITE


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_zero_steps_and_invalid_step_arguments(prec):
    """n_steps = 0 leaves the state bit for bit; negative n_steps and dt <= 0, NaN or inf
    are refused with DIRAC_EINVAL before any device work, and the context keeps working."""
    w = W.plain_128(n=64)
    with D.Simulation(w, precision=prec) as s:
        s.set_state(w.psi0)
        before = s.get_state()
        s.step(0, w.dt)
        assert np.array_equal(s.get_state(), before)
        for n, dt in ((-1, w.dt), (1, 0.0), (1, -w.dt), (1, float("nan")), (1, float("inf"))):
            with pytest.raises(D.DiracError) as e:
                s.step(n, dt)
            assert e.value.status == D.DIRAC_EINVAL
        assert np.array_equal(s.get_state(), before)
        s.step(5, w.dt)
        got = s.get_state()
    assert W.rel_l2(got, oracle_run(w, 5)) <= TOL[prec]


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("scheme", [D.DIRAC_SCHEME_II, D.DIRAC_SCHEME_II_SYMMETRIC],
                         ids=["printed", "symmetric"])
def test_dt_change_between_calls(prec, scheme):
    """A call with another dt rebuilds the half steps and k-space tables: 7 steps of dt
    then 5 of dt / 2 give the oracle's 7 + 5 steps (the U of the first call's last half
    step and the second call's first are those of their own dt)."""
    w = W.graphene_strained(n=128, steps=12)
    w.mass = 0.3
    prob = oracle.Problem.from_workload(w)
    osch = oracle.SCHEME_II if scheme == D.DIRAC_SCHEME_II else oracle.SCHEME_II_SYMMETRIC
    ref = oracle.run(prob, w.psi0, w.dt, 7, scheme=osch)
    ref = oracle.run(prob, ref, 0.5 * w.dt, 5, scheme=osch)
    with D.Simulation(w, precision=prec, scheme=scheme) as s:
        s.set_state(w.psi0)
        s.step(7, w.dt)
        s.step(5, 0.5 * w.dt)
        got = s.get_state()
    assert_parity(got, ref, w, TOL[prec])


def test_norm_conserved_in_flat_space_on_gpu():
    w = W.plain_128(flat=True)
    w.mass = 0.5
    with D.Simulation(w, precision=D.DIRAC_C128) as s:
        s.set_state(w.psi0)
        n0 = s.observables()["norm"]
        s.step(500, w.dt)
        n1 = s.observables()["norm"]
    assert abs(n1 / n0 - 1.0) <= 1e-12


ALT = D.DIRAC_LAUNCH_ALT_RADIX
SHAPES = [256, 512, 1024, 256 | ALT, 512 | ALT]


@pytest.mark.parametrize("prec", PREC, ids=PID)
@pytest.mark.parametrize("threads", SHAPES, ids=["256", "512", "1024", "256alt", "512alt"])
@pytest.mark.parametrize("nx,ny", [(512, 256), (1024, 2048), (4096, 256), (256, 4096),
                                   (128, 64), (64, 128)])
def test_every_cta_shape_matches_oracle(prec, threads, nx, ny):
    """All launch shapes, including the persistent prefetching pass (1024; complex64,
    lines of 256..4096 points) and the alternative radix schedules (radix-16 passes for
    complex64, radix-8 for complex128), give the oracle's result."""
    ax, ay = 0.1 * nx, 0.1 * ny
    X, Y = W.mesh(nx, ny, ax, ay)
    g = 1.0 + 0.15 * np.exp(-((X - 0.2 * ax) ** 2 + Y ** 2) / (0.1 * ax * ay))
    psi0 = W.wave_packet(nx, ny, ax, ay, 0.05 * min(ax, ay) + 1.0, (1.2, 0.4))
    w = W.Workload("shape", nx, ny, ax, ay, np.ones((ny, nx)), g, 1.0 + 0.5 * (g - 1.0),
                   mass=0.3, c=1.0, pml_width_x=nx // 32, pml_width_y=ny // 32, pml_type=1,
                   sigma0=1.0, theta=0.0, psi0=psi0, dt=0.05, steps=4)
    ref = oracle_run(w, 4)
    with D.Simulation(w, precision=prec) as s:
        D.dirac_set_launch(s.ctx, threads, threads)
        s.set_state(w.psi0)
        s.step(4, w.dt)
        got = s.get_state()
    assert_parity(got, ref, w, TOL[prec])


@pytest.mark.parametrize("prec", PREC, ids=PID)
def test_autotune_keeps_state_and_picks_a_valid_shape(prec, tmp_path):
    from paper_1909_02894_gb300 import autotune

    w = W.graphene_strained(n=512, steps=6)
    ref = oracle_run(w, 6)
    with D.Simulation(w, precision=prec) as s:
        s.set_state(w.psi0)
        tx, ty = autotune.tune(s, prec, cache_path=str(tmp_path / "cache.json"), reps=5)
        assert tx in SHAPES and ty in SHAPES
        s.step(6, w.dt)
        assert_parity(s.get_state(), ref, w, TOL[prec])
        assert autotune.tune(s, prec, cache_path=str(tmp_path / "cache.json")) == (tx, ty)


def test_bounded_wait_timeout_in_the_clustered_4096_pass():
    """The same on the 4096^2 complex64 grid: the persistent 4096-point pass runs as
    clusters whose CTAs keep taking part in the cluster barriers after a wait has run out,
    so every CTA returns; the context works again afterwards."""
    w = W.large_4096(steps=1)
    with D.Simulation(w, precision=D.DIRAC_C64) as s:
        s.set_state(w.psi0)
        D.dirac_test_timeout_next_step(s.ctx)
        s.step(1, w.dt)
        with pytest.raises(D.DiracError) as e:
            D.dirac_synchronize(s.ctx)
        assert e.value.status == D.DIRAC_ETIMEOUT
        s.set_state(w.psi0)
        s.step(1, w.dt)
        got = s.get_state()
    ref = oracle_run(w, 1)
    assert_parity(got, ref, w, TOL[D.DIRAC_C64])


def test_bounded_wait_timeout_is_reported_and_context_recovers():
    """Failure detection without a GPU fault: a bulk-copy wait that nothing completes
    runs out after its bound; the kernel returns, dirac_synchronize reports
    DIRAC_ETIMEOUT, and the context works again after the state is set anew."""
    w = W.graphene_strained(n=1024, steps=2)
    with D.Simulation(w, precision=D.DIRAC_C64) as s:
        D.dirac_set_launch(s.ctx, 1024, 1024)
        s.set_state(w.psi0)
        D.dirac_test_timeout_next_step(s.ctx)
        s.step(1, w.dt)
        with pytest.raises(D.DiracError) as e:
            D.dirac_synchronize(s.ctx)
        assert e.value.status == D.DIRAC_ETIMEOUT
        s.set_state(w.psi0)
        s.step(2, w.dt)
        got = s.get_state()
    ref = oracle_run(w, 2)
    assert_parity(got, ref, w, TOL[D.DIRAC_C64])
