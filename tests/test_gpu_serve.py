"""Serving loop on the GPU: requests of different types, sizes, splits and precisions arrive
while others run, share batched launches and streams, and each result equals the result of
the same request run alone (the stated tolerance is 1e-12 relative; in practice the fields
are bit-identical, since a batched launch does the same per-node arithmetic)."""
import numpy as np
import pytest

from paper_2405_11489_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pond():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_11489_gb300 import build, pond as P
    build.build()
    P.load_library()
    return P


def _mix():
    reqs = W.serving_requests(count=14, rate=60.0, seed=11, step_scale=0.08, max_side=160)
    # shorter tubes keep the test quick
    for r in reqs:
        if r.case.ny == 1:
            r.steps = min(r.steps, 60)
    return reqs


def test_each_result_is_the_same_alone_and_in_the_mix(pond):
    from paper_2405_11489_gb300.serve import PondBackend, Server
    reqs = _mix()
    be = PondBackend("cuda:0")
    srv = Server(be, budget_bytes=2 ** 30, chunk=8, keep_fields=True)
    m = srv.run(reqs, realtime=True)
    assert m["served"] == len(reqs) and m["rejected"] == 0
    assert m["p50_time_to_result_s"] is not None and m["p99_time_to_result_s"] >= m["p50_time_to_result_s"]
    # continuous batching: some class advanced several requests in one launch sequence
    assert m["ticks"] > 0
    done = {c.rid: c for c in srv.done}
    for r in reqs:
        alone = be.create(r)
        alone.step(r.steps)
        ref, _ = be.finish(alone)
        got = done[r.rid].fields
        for a, b in zip(got, ref):
            scale = max(np.max(np.abs(b)), 1.0)
            assert np.max(np.abs(a - b)) <= 1e-12 * scale, r.rid


def test_admission_respects_the_memory_budget(pond):
    from paper_2405_11489_gb300.serve import PondBackend, Server
    reqs = _mix()[:8]
    be = PondBackend("cuda:0")
    biggest = max(be.workspace_bytes(r) for r in reqs)
    srv = Server(be, budget_bytes=int(1.5 * biggest), chunk=8)
    m = srv.run(reqs, realtime=False)
    assert m["served"] == len(reqs) and m["peak_workspace_bytes"] <= int(1.5 * biggest)
