"""Batched stepping: every context gives the same result alone and in a mix of uneven
sizes and step counts, admission respects the device-memory budget, and slots are
released and reused."""
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


def mix(seed, sizes, steps):
    rng = np.random.default_rng(seed)
    return [(W.batched_instance(n, rng, steps=s)) for n, s in zip(sizes, steps)]


def alone(w, prec):
    with D.Simulation(w, precision=prec) as s:
        # same CTA shapes as the batch: persistent for complex64 lines >= 256, else 512
        t = 1024 if (prec == D.DIRAC_C64 and w.nx >= 256) else 512
        D.dirac_set_launch(s.ctx, t, t)
        s.set_state(w.psi0)
        s.step(w.steps, w.dt)
        return s.get_state()


@pytest.mark.parametrize("tick", ["0", "1"], ids=["per-step", "tick-launch"])
@pytest.mark.parametrize("prec", [D.DIRAC_C64, D.DIRAC_C128], ids=["c64", "c128"])
def test_alone_equals_in_mix(prec, tick, monkeypatch):
    """Per-step launches and (DIRAC_BATCH_TICK=1) one persistent launch per tick for the
    complex64 classes of 256..1024 points: every result equals its alone run bit for bit."""
    monkeypatch.setenv("DIRAC_BATCH_TICK", tick)
    sizes = [128, 256, 128, 512, 256, 128, 1024, 256, 128, 512]
    steps = [37, 64, 5, 50, 16, 33, 20, 47, 64, 1]
    ws = mix(7, sizes, steps)
    ref = [alone(w, prec) for w in ws]
    batch = D.dirac_batch_create(64 << 30, prec, steps_per_tick=16)
    sims, slots = [], []
    try:
        for w in ws:
            s = D.Simulation(w, precision=prec)
            s.set_state(w.psi0)
            sims.append(s)
            slots.append(D.dirac_batch_submit(batch, s.ctx, w.steps, w.dt))
        for _ in range(10):
            D.dirac_batch_run(batch, 1)
            if D.dirac_batch_active(batch) == 0:
                break
        D.dirac_batch_synchronize(batch)
        assert D.dirac_batch_active(batch) == 0
        for sl in slots:
            assert D.dirac_batch_poll(batch, sl)
        for w, s, sl, r in zip(ws, sims, slots, ref):
            D.dirac_batch_release(batch, sl)
            got = s.get_state()
            assert np.array_equal(got, r), (w.name, W.rel_l2(got, r))
    finally:
        D.dirac_batch_destroy(batch)
        for s in sims:
            s.close()


@pytest.mark.parametrize("prec", [D.DIRAC_C64, D.DIRAC_C128], ids=["c64", "c128"])
def test_autotuned_batch_equals_alone_runs_with_its_shapes(prec):
    """The batch autotuner times each class's CTA shapes on its contexts without changing
    any state: after it, every context's result equals, bit for bit, the context stepped
    alone with the shapes the autotuner chose for its class."""
    sizes = [128, 256, 512, 1024, 256, 128]
    steps = [20, 33, 17, 12, 40, 9]
    ws = mix(11, sizes, steps)
    batch = D.dirac_batch_create(64 << 30, prec, steps_per_tick=8)
    sims, slots = [], []
    try:
        for w in ws:
            s = D.Simulation(w, precision=prec)
            s.set_state(w.psi0)
            sims.append(s)
            slots.append(D.dirac_batch_submit(batch, s.ctx, w.steps, w.dt))
        with pytest.raises(D.DiracError) as e:
            D.dirac_batch_autotune(batch, 0)
        assert e.value.status == D.DIRAC_EINVAL
        D.dirac_batch_autotune(batch, 3)
        shapes = {n: D.dirac_batch_launch_shape(batch, n, n) for n in set(sizes)}
        for n, (tx, ty) in shapes.items():
            shapes_ok = (256, 512, 1024, 256 | D.DIRAC_LAUNCH_ALT_RADIX,
                         512 | D.DIRAC_LAUNCH_ALT_RADIX)
            assert tx in shapes_ok and ty in shapes_ok, (n, tx, ty)
            if prec == D.DIRAC_C128:
                assert tx != 1024 and ty != 1024
        with pytest.raises(D.DiracError):
            D.dirac_batch_launch_shape(batch, 64, 64)
        while D.dirac_batch_active(batch):
            D.dirac_batch_run(batch, 1)
        D.dirac_batch_synchronize(batch)
        for w, s, sl in zip(ws, sims, slots):
            D.dirac_batch_release(batch, sl)
            got = s.get_state()
            with D.Simulation(w, precision=prec) as a:
                D.dirac_set_launch(a.ctx, *shapes[w.nx])
                a.set_state(w.psi0)
                a.step(w.steps, w.dt)
                ref = a.get_state()
            assert np.array_equal(got, ref), (w.name, shapes[w.nx], W.rel_l2(got, ref))
    finally:
        D.dirac_batch_destroy(batch)
        for s in sims:
            s.close()


def test_batch_matches_oracle_and_admits_late_arrivals():
    """A context submitted while others run is stepped from its own start and matches
    the oracle; the budget refuses an instance that does not fit."""
    rng = np.random.default_rng(3)
    w1 = W.batched_instance(256, rng, steps=40)
    w2 = W.batched_instance(128, rng, steps=25)
    need = D.dirac_footprint_bytes(256, 256) + D.dirac_footprint_bytes(128, 128)
    batch = D.dirac_batch_create(need, D.DIRAC_C64, steps_per_tick=8)
    s1 = D.Simulation(w1, precision=D.DIRAC_C64)
    s2 = D.Simulation(w2, precision=D.DIRAC_C64)
    s3 = D.Simulation(w2, precision=D.DIRAC_C64)
    try:
        s1.set_state(w1.psi0)
        s2.set_state(w2.psi0)
        s3.set_state(w2.psi0)
        a = D.dirac_batch_submit(batch, s1.ctx, w1.steps, w1.dt)
        D.dirac_batch_run(batch, 2)
        b = D.dirac_batch_submit(batch, s2.ctx, w2.steps, w2.dt)   # arrives mid-run
        with pytest.raises(D.DiracError) as e:
            D.dirac_batch_submit(batch, s3.ctx, 10, w2.dt)        # over budget
        assert e.value.status == D.DIRAC_ENOMEM
        while D.dirac_batch_active(batch):
            D.dirac_batch_run(batch, 1)
        D.dirac_batch_synchronize(batch)
        D.dirac_batch_release(batch, a)
        D.dirac_batch_release(batch, b)
        for w, s in ((w1, s1), (w2, s2)):
            ref = oracle.run(oracle.Problem.from_workload(w), w.psi0, w.dt, w.steps)
            assert_parity(s.get_state(), ref, w, 1e-5)
        # the freed budget admits the third one in a reused slot
        c = D.dirac_batch_submit(batch, s3.ctx, 3, w2.dt)
        assert c in (a, b)
        D.dirac_batch_run(batch, 1)
        D.dirac_batch_synchronize(batch)
        assert D.dirac_batch_poll(batch, c)
        D.dirac_batch_release(batch, c)
    finally:
        D.dirac_batch_destroy(batch)
        for s in (s1, s2, s3):
            s.close()


def test_batched_4096_point_lines_equal_the_alone_run():
    """A 4096^2 instance in a batch (clusters of two CTAs gather the output through
    distributed shared memory and store it from registers) gives, bit for bit, the result
    of the same instance stepped alone (each CTA's line written by tensor stores), beside a
    small instance of another class."""
    rng = np.random.default_rng(17)
    ws = [W.batched_instance(4096, rng, steps=6), W.batched_instance(256, rng, steps=9)]
    ref = [alone(w, D.DIRAC_C64) for w in ws]
    batch = D.dirac_batch_create(64 << 30, D.DIRAC_C64, steps_per_tick=4)
    sims, slots = [], []
    try:
        for w in ws:
            s = D.Simulation(w, precision=D.DIRAC_C64)
            s.set_state(w.psi0)
            sims.append(s)
            slots.append(D.dirac_batch_submit(batch, s.ctx, w.steps, w.dt))
        while D.dirac_batch_active(batch):
            D.dirac_batch_run(batch, 1)
        D.dirac_batch_synchronize(batch)
        for w, s, sl, r in zip(ws, sims, slots, ref):
            D.dirac_batch_release(batch, sl)
            got = s.get_state()
            assert np.array_equal(got, r), (w.name, W.rel_l2(got, r))
    finally:
        D.dirac_batch_destroy(batch)
        for s in sims:
            s.close()
