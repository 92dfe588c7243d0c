"""Host logic of the serving loop (no GPU): admission by memory budget in arrival order,
exact step counts under chunked ticks, class grouping, completion metrics."""
import itertools

import pytest

from paper_2405_11489_gb300.serve import Server, percentile


class FakeCase:
    def __init__(self, nx, ny):
        self.nx, self.ny = nx, ny


class FakeReq:
    def __init__(self, rid, arrival, nx, ny, steps, precision="fp32", order=3):
        self.rid, self.arrival, self.steps = rid, arrival, steps
        self.case = FakeCase(nx, ny)
        self.precision, self.interp_order = precision, order


class FakeBackend:
    """Counts steps per simulation; memory = 100 bytes per node."""

    def __init__(self):
        self.steps = {}
        self.calls = []
        self.live = 0
        self.max_live = 0

    def workspace_bytes(self, req):
        return 100 * req.case.nx * req.case.ny

    def class_key(self, req):
        return (req.precision, req.interp_order, req.case.ny == 1)

    def create(self, req):
        self.steps[req.rid] = 0
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return req.rid

    def advance(self, key, sims, n):
        self.calls.append((key, tuple(sims), n))
        for s in sims:
            self.steps[s] += n
        return len(self.calls)

    def ready(self, token):
        return True

    def wait_for(self, token):
        pass

    def finish(self, sim):
        self.live -= 1
        return ("fields", sim, self.steps[sim]), "ok"


def _clock():
    c = itertools.count()
    return lambda: next(c) * 1e-3


def test_every_request_runs_exactly_its_steps():
    be = FakeBackend()
    reqs = [FakeReq(i, 0.0, 10 + i, 1 if i % 2 else 5, steps=7 + 3 * i) for i in range(9)]
    srv = Server(be, budget_bytes=10 ** 9, chunk=4, keep_fields=True, clock=_clock())
    m = srv.run(reqs, realtime=False)
    assert m["served"] == 9 and m["rejected"] == 0
    for c in srv.done:
        assert c.fields[2] == c.steps == 7 + 3 * c.rid
    # every advance call moves a class by at most the chunk
    assert all(n <= 4 for _, _, n in be.calls)
    # members of one call share the class key
    for key, sims, n in be.calls:
        assert len({be_key for be_key in [key]}) == 1


def test_admission_waits_for_memory_in_arrival_order():
    be = FakeBackend()
    # each request needs 1000 bytes; budget fits two at a time
    reqs = [FakeReq(i, 0.0, 10, 1, steps=5 + i) for i in range(6)]
    srv = Server(be, budget_bytes=2000, chunk=3, clock=_clock())
    m = srv.run(reqs, realtime=False)
    assert m["served"] == 6 and be.max_live == 2
    assert m["peak_workspace_bytes"] <= 2000
    admitted = sorted(srv.done, key=lambda c: c.admitted)
    assert [c.rid for c in admitted] == sorted(c.rid for c in srv.done)


def test_oversized_request_is_rejected_not_blocking():
    be = FakeBackend()
    reqs = [FakeReq(0, 0.0, 100, 100, steps=3), FakeReq(1, 0.0, 10, 1, steps=3)]
    srv = Server(be, budget_bytes=5000, chunk=8, clock=_clock())
    m = srv.run(reqs, realtime=False)
    assert m["rejected"] == 1 and m["served"] == 1


def test_new_arrivals_join_running_classes():
    be = FakeBackend()
    clock = _clock()
    reqs = [FakeReq(0, 0.0, 10, 1, steps=40), FakeReq(1, 0.005, 10, 1, steps=8)]
    srv = Server(be, budget_bytes=10 ** 6, chunk=2, clock=clock)
    srv.run(reqs, realtime=True)
    # some tick advanced both requests together (continuous batching, not a queue)
    assert any(set(sims) == {0, 1} for _, sims, _ in be.calls)
    done = {c.rid: c for c in srv.done}
    assert done[1].done < done[0].done


def test_percentile():
    assert percentile([1, 2, 3, 4, 5], 50) == 3
    assert abs(percentile(list(range(101)), 99) - 99) < 1e-12
    assert percentile([], 50) is None
