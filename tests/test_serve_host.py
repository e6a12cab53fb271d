"""The serving loop's admission logic on the CPU: the batch ABI is replaced by a fake
that steps every active request by steps_per_tick per tick, so only the host-side
scheduling is under test (FIFO order, shortest-job-first order, the active-points cap,
the memory budget, and a request that can never fit)."""
import pytest

from paper_1909_02894_gb300 import serve as S


class FakeSim:
    def __init__(self, w, precision=None, stream=None):
        self.ctx = w

    def set_state(self, psi):
        pass

    def get_state(self):
        return None

    def close(self):
        pass


class FakeBatch:
    def __init__(self, tick):
        self.tick = tick
        self.left = {}
        self.next_slot = 0


@pytest.fixture
def fake(monkeypatch):
    state = {}

    def create(budget, precision, steps_per_tick, stream):
        state["b"] = FakeBatch(steps_per_tick)
        return state["b"]

    def submit(b, ctx, steps, dt):
        slot = b.next_slot
        b.next_slot += 1
        b.left[slot] = steps
        return slot

    def run(b, ticks):
        for s in b.left:
            b.left[s] = max(0, b.left[s] - b.tick * ticks)

    monkeypatch.setattr(S, "Simulation", FakeSim)
    monkeypatch.setattr(S, "dirac_batch_create", create)
    monkeypatch.setattr(S, "dirac_batch_submit", submit)
    monkeypatch.setattr(S, "dirac_batch_run", run)
    monkeypatch.setattr(S, "dirac_batch_poll", lambda b, s: b.left[s] == 0)
    monkeypatch.setattr(S, "dirac_batch_release", lambda b, s: b.left.pop(s))
    monkeypatch.setattr(S, "dirac_batch_synchronize", lambda b: None)
    monkeypatch.setattr(S, "dirac_batch_destroy", lambda b: None)
    monkeypatch.setattr(S, "dirac_footprint_bytes", lambda nx, ny, p=None: nx * ny)
    return state


class W:
    psi0 = None
    dt = 0.05


def reqs(spec):
    """(n, steps) per request, all arrived at time 0, rid in list order."""
    return [S.Request(0.0, rid, lambda: W(), n, n, steps) for rid, (n, steps) in enumerate(spec)]


def run(server, rs):
    order = []
    orig = server._start

    def spy(req, need):
        order.append((req.rid, server.active_points, server.used))
        orig(req, need)

    server._start = spy
    for r in rs:
        server.submit(r)
    res = server.run(deadline=60.0)
    server.close()
    return order, res


SPEC = [(64, 400), (16, 50), (32, 100), (16, 300), (64, 20), (32, 30)]


def test_fifo_admits_in_arrival_order(fake):
    srv = S.Server(10 ** 9, steps_per_tick=10, policy="fifo")
    order, res = run(srv, reqs(SPEC))
    assert [o[0] for o in order] == list(range(len(SPEC)))
    assert len(res) == len(SPEC)


def test_sjf_admits_least_work_first_under_the_cap(fake):
    cap = 64 * 64 + 32 * 32
    srv = S.Server(10 ** 9, steps_per_tick=10, policy="sjf", max_active_points=cap)
    order, res = run(srv, reqs(SPEC))
    work = {rid: n * n * steps for rid, (n, steps) in enumerate(SPEC)}
    # the first admission is the cheapest request, and the first round goes in order of work
    assert order[0][0] == min(work, key=work.get)
    first_round = [rid for rid, _, _ in order[:2]]
    assert [work[r] for r in first_round] == sorted(work[r] for r in first_round)
    for rid, active_before, _ in order:
        n = SPEC[rid][0]
        assert active_before == 0 or active_before + n * n <= cap
    assert sorted(r.rid for r in res) == list(range(len(SPEC)))
    # every result's latency is positive and finishing is consistent with admission
    assert all(r.finished >= r.admitted >= r.arrival for r in res)


def test_sjf_runs_everything_when_uncapped_and_respects_the_budget(fake):
    budget = 2 * 64 * 64
    srv = S.Server(budget, steps_per_tick=10, policy="sjf")
    order, res = run(srv, reqs(SPEC))
    assert len(res) == len(SPEC)
    for rid, _, used_before in order:
        n = SPEC[rid][0]
        assert used_before + n * n <= budget


def test_a_request_larger_than_the_budget_is_refused(fake):
    srv = S.Server(32 * 32, steps_per_tick=10, policy="sjf")
    with pytest.raises(ValueError):
        run(srv, reqs([(16, 10), (64, 10)]))


def test_unknown_policy_is_refused(fake):
    with pytest.raises(ValueError):
        S.Server(10 ** 6, policy="lifo")
