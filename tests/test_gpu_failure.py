"""Failure detection without a GPU fault: an injected host-side allocation failure, and a
bounded device wait that runs out inside a batched tick.

Neither test faults, traps or hangs the GPU: the allocation failure is made on the host
(DIRAC_FAULT=alloc:N makes the N-th device allocation of a new context report
cudaErrorMemoryAllocation without allocating), and the batched wait expects bytes that
no copy delivers, so it gives up after its bound and the kernel returns.
"""
import os

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


def _free_bytes():
    import torch

    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_injected_allocation_failure_gives_enomem_and_leaks_nothing(monkeypatch):
    pytest.importorskip("torch")
    w = W.graphene_strained(n=1024, steps=3)
    base = _free_bytes()
    failed = 0
    for k in range(1, 65):
        monkeypatch.setenv("DIRAC_FAULT", f"alloc:{k}")
        try:
            s = D.Simulation(w, precision=D.DIRAC_C64)
        except D.DiracError as e:
            assert e.status == D.DIRAC_ENOMEM, e
            failed += 1
            # everything the failed creation allocated has been freed (the smallest
            # persistent buffer of a 1024^2 context is 4 MiB)
            assert base - _free_bytes() < (2 << 20), k
            continue
        s.close()  # k is past the creation's last allocation: nothing was injected
        break
    else:
        pytest.fail("creation never succeeded")
    assert failed >= 10  # every allocation of the creation was made to fail once
    monkeypatch.delenv("DIRAC_FAULT")
    with D.Simulation(w, precision=D.DIRAC_C64) as s:
        s.set_state(w.psi0)
        s.step(3, w.dt)
        got = s.get_state()
    assert_parity(got, oracle.run(oracle.Problem.from_workload(w), w.psi0, w.dt, 3), w, 1e-5)


def test_malformed_fault_variable_is_ignored(monkeypatch):
    w = W.plain_128(n=64, steps=2)
    for v in ("alloc:", "alloc:0", "alloc:-3", "alloc:2x", "oom", ""):
        monkeypatch.setenv("DIRAC_FAULT", v)
        with D.Simulation(w, precision=D.DIRAC_C64) as s:
            s.set_state(w.psi0)
            s.step(2, w.dt)


def _alone(w, steps):
    with D.Simulation(w, precision=D.DIRAC_C64) as s:
        s.set_state(w.psi0)
        s.step(steps, w.dt)
        return s.get_state()


@pytest.mark.parametrize("tick", ["0", "1"], ids=["per-step", "tick-launch"])
def test_batched_wait_timeout_is_reported_and_the_batch_recovers(tick, monkeypatch):
    """A context whose first batched x pass waits for bytes that never arrive: the wait
    runs out, dirac_batch_poll reports DIRAC_ETIMEOUT for every context then in the batch,
    and after release, new states and resubmission the batch gives the alone results bit
    for bit -- with per-step launches and with one persistent launch per tick."""
    monkeypatch.setenv("DIRAC_BATCH_TICK", tick)
    rng = np.random.default_rng(5)
    ws = [W.batched_instance(n, rng, steps=6) for n in (512, 256, 1024, 512)]
    sims = [D.Simulation(w, precision=D.DIRAC_C64) for w in ws]
    batch = D.dirac_batch_create(1 << 34, D.DIRAC_C64, steps_per_tick=4)
    try:
        for s, w in zip(sims, ws):
            s.set_state(w.psi0)
        D.dirac_test_timeout_next_step(sims[0].ctx)
        slots = [D.dirac_batch_submit(batch, s.ctx, 6, w.dt) for s, w in zip(sims, ws)]
        while D.dirac_batch_active(batch):
            D.dirac_batch_run(batch, 1)
        with pytest.raises(D.DiracError) as e:
            D.dirac_batch_synchronize(batch)
        assert e.value.status == D.DIRAC_ETIMEOUT
        for sl in slots:
            with pytest.raises(D.DiracError) as e:
                D.dirac_batch_poll(batch, sl)
            assert e.value.status == D.DIRAC_ETIMEOUT
            D.dirac_batch_release(batch, sl)
        # recovery: the same contexts, states set again
        for s, w in zip(sims, ws):
            s.set_state(w.psi0)
        slots = [D.dirac_batch_submit(batch, s.ctx, 6, w.dt) for s, w in zip(sims, ws)]
        while D.dirac_batch_active(batch):
            D.dirac_batch_run(batch, 1)
        D.dirac_batch_synchronize(batch)
        for sl in slots:
            assert D.dirac_batch_poll(batch, sl)
            D.dirac_batch_release(batch, sl)
        for s, w in zip(sims, ws):
            assert np.array_equal(s.get_state(), _alone(w, 6)), w.name
    finally:
        D.dirac_batch_destroy(batch)
        for s in sims:
            s.close()
