"""Continuous batching: requests arriving while others run are admitted as memory
frees up, and each result equals the same simulation stepped alone."""
import numpy as np
import pytest

import paper_1909_02894_gb300 as D
from paper_1909_02894_gb300 import serve as S
from paper_1909_02894_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def alone(w, steps):
    with D.Simulation(w, precision=D.DIRAC_C64) as s:
        t = 1024 if w.nx >= 256 else 512
        D.dirac_set_launch(s.ctx, t, t)
        s.set_state(w.psi0)
        s.step(steps, w.dt)
        return s.get_state()


def test_served_results_equal_alone_runs():
    D.build()
    reqs = S.graphene_requests(rate=400.0, duration=0.05, seed=5, sizes=(64, 128, 256),
                               steps_range=(20, 120), check_fraction=0.0)
    assert len(reqs) >= 8
    # room for about three 256^2 requests at a time: later arrivals must wait for memory
    budget = 3 * D.dirac_footprint_bytes(256, 256) + D.dirac_footprint_bytes(128, 128)
    srv = S.Server(budget, steps_per_tick=8, keep_states=True)
    try:
        for r in reqs:
            srv.submit(r)
        results = srv.run(deadline=300.0)
    finally:
        srv.close()
    assert len(results) == len(reqs)
    assert srv.max_active > 1 and srv.admitted_while_busy > 0
    by_id = {r.rid: r for r in reqs}
    for res in results:
        req = by_id[res.rid]
        ref = alone(req.make(), req.steps)
        assert np.array_equal(res.state, ref), (res.rid, W.rel_l2(res.state, ref))
        assert res.latency > 0
    summ = S.latency_summary(results)
    assert summ["p99_ms"] >= summ["p50_ms"] > 0


def test_fp64_check_of_served_requests():
    D.build()
    reqs = S.graphene_requests(rate=200.0, duration=0.03, seed=9, sizes=(128,),
                               steps_range=(200, 300), check_fraction=1.0)
    srv = S.Server(1 << 34, steps_per_tick=16)
    try:
        for r in reqs:
            srv.submit(r)
        results = srv.run(deadline=300.0)
    finally:
        srv.close()
    checks = S.fp64_check(results)
    assert len(checks) == len(reqs) > 0
    assert all(c["rel_l2"] <= 1e-5 for c in checks), checks
    assert all(c["short_rel_l2"] <= 1e-5 and c["short_reference"] == "c128" for c in checks)


def test_served_large_grids_equal_alone_runs():
    """The serving sizes above 256^2 (persistent passes: 512-, 1024- and 2048-point lines)
    running together in one batch give the alone results bit for bit."""
    D.build()
    reqs = S.graphene_requests(rate=300.0, duration=0.04, seed=21, sizes=(512, 1024, 2048),
                               steps_range=(30, 70), check_fraction=0.0)
    assert len(reqs) >= 6
    srv = S.Server(1 << 36, steps_per_tick=16, keep_states=True)
    try:
        for r in reqs:
            srv.submit(r)
        results = srv.run(deadline=300.0)
    finally:
        srv.close()
    assert len(results) == len(reqs) and srv.max_active > 1
    by_id = {r.rid: r for r in reqs}
    for res in results:
        req = by_id[res.rid]
        assert np.array_equal(res.state, alone(req.make(), req.steps)), res.rid


def test_shortest_job_first_admission_keeps_results_and_orders_by_work():
    """The sjf policy admits the arrived request with the least work first and keeps the
    active points under the cap; every result still equals the alone run bit for bit."""
    D.build()
    reqs = S.graphene_requests(rate=400.0, duration=0.05, seed=33, sizes=(64, 128, 256),
                               steps_range=(20, 120), check_fraction=0.0)
    assert len(reqs) >= 8
    for r in reqs:  # everything has arrived at the start
        r.arrival = 0.0
    cap = 256 * 256 + 128 * 128
    srv = S.Server(1 << 34, steps_per_tick=8, keep_states=True, policy="sjf",
                   max_active_points=cap)
    started = []
    orig = srv._start

    def spy(req, need):
        started.append((req.nx * req.ny * req.steps, req.rid, srv.active_points))
        orig(req, need)

    srv._start = spy
    try:
        for r in reqs:
            srv.submit(r)
        results = srv.run(deadline=300.0)
    finally:
        srv.close()
    assert len(results) == len(reqs)
    # the first admissions come in order of work, and the cap is respected whenever
    # something else was running
    first = [w for w, _, _ in started[:3]]
    assert first == sorted(first)
    by_id = {r.rid: r for r in reqs}
    for w, rid, before in started:
        if before:
            assert before + by_id[rid].nx * by_id[rid].ny <= cap
    for res in results:
        req = by_id[res.rid]
        assert np.array_equal(res.state, alone(req.make(), req.steps)), res.rid
    with pytest.raises(ValueError):
        S.Server(1 << 30, policy="lifo")
