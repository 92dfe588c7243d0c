"""Batched stepping (pond_batch): uneven cases advanced by one launch per time step give
the same state, bit for bit, as stepping each case on its own (same arithmetic per node),
with plain launches and with a captured CUDA graph."""
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


def _tube_sims(pond, cases, precision="fp32", split="total", order=3):
    sims = []
    for c in cases:
        s = pond.Simulation(pond.Config(nx=c.nx, ny=c.ny, precision=precision, split=split,
                                        gamma=c.gamma, mu=c.mu, bc_x=c.bc_x, bc_y=c.bc_y,
                                        interp_order=order))
        s.set_state(c.rho, c.ux, c.uy, c.T)
        sims.append(s)
    return sims


def _grid_cases():
    return [W.shear_wave(n=40, ny=23, ma=0.5, mu=0.05), W.thermal_pulse(n=35, amp=1e-2, width=4.0),
            W.shear_wave(n=70, ny=9, ma=1.5, mu=0.02)]


@pytest.mark.parametrize("graph", [0, 4])
def test_batch_of_uneven_tubes_matches_single_steps(pond, graph):
    import torch
    cases = W.tube_batch(count=12, seed=1, nmin=200, nmax=900)
    ref = _tube_sims(pond, cases, order=2)
    for s in ref:
        s.step(7)
    sims = _tube_sims(pond, cases, order=2)
    stream = torch.cuda.Stream()
    batch = pond.Batch(sims, stream=stream)
    if graph:
        batch.use_graph(graph)
    batch.step(7)
    stream.synchronize()
    for a, b in zip(sims, ref):
        for x, y in zip(a.moments(), b.moments()):
            assert np.array_equal(x, y)
        rc, st = a.stats()
        assert st.steps == 7
    batch.close()


@pytest.mark.parametrize("split", ["total", "internal"])
def test_batch_of_2d_grids_matches_single_steps(pond, split):
    cases = _grid_cases()
    ref = _tube_sims(pond, cases, split=split)
    for s in ref:
        s.step(5)
    sims = _tube_sims(pond, cases, split=split)
    batch = pond.Batch(sims)
    batch.step(5)
    for a, b in zip(sims, ref):
        for x, y in zip(a.moments(), b.moments()):
            assert np.array_equal(x, y)
    batch.close()


def test_batch_rejects_mismatched_members(pond):
    a = pond.Simulation(pond.Config(nx=32, ny=8, precision="fp32"))
    b = pond.Simulation(pond.Config(nx=32, ny=8, precision="fp64"))
    with pytest.raises(pond.PondError):
        pond.Batch([a, b])
    c = pond.Simulation(pond.Config(nx=32, ny=1, precision="fp32"))
    with pytest.raises(pond.PondError):
        pond.Batch([a, c])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_set_state_and_moments_equal_the_per_member_calls(pond, precision):
    """pond_batch_set_state / pond_batch_get_moments (one synchronisation for all members)
    give the same states and fields, bit for bit, as pond_set_state / pond_get_moments per
    member, with host and with device input, before and after batched steps."""
    import torch
    cases = _grid_cases()
    ref = _tube_sims(pond, cases, precision=precision)
    for s in ref:
        s.step(3)
    sims = _tube_sims(pond, cases, precision=precision)     # states to be replaced
    for s in sims:
        s.step(2)
    batch = pond.Batch(sims)
    batch.set_state([(c.rho, c.ux, c.uy, c.T) for c in cases])
    for got, s in zip(batch.moments(), _tube_sims(pond, cases, precision=precision)):
        for x, y in zip(got, s.moments()):
            assert np.array_equal(x, y)
    batch.step(3)
    for got, s in zip(batch.moments(), ref):
        for x, y in zip(got, s.moments()):
            assert np.array_equal(x, y)
        assert s.stats()[1].steps == 3
    for s in sims:
        assert s.stats()[1].steps == 3
    # device input
    dev = [tuple(torch.as_tensor(a, device="cuda") for a in (c.rho, c.ux, c.uy, c.T)) for c in cases]
    batch.set_state(dev)
    batch.step(3)
    for got, s in zip(batch.moments(), ref):
        for x, y in zip(got, s.moments()):
            assert np.array_equal(x, y)
    batch.close()


def test_batch_set_state_rejects_bad_host_input_and_changes_no_member(pond):
    cases = _grid_cases()
    sims = _tube_sims(pond, cases)
    batch = pond.Batch(sims)
    batch.step(2)
    before = [s.export_state() for s in sims]
    fields = [(c.rho.copy(), c.ux.copy(), c.uy.copy(), c.T.copy()) for c in cases]
    fields[1][3][2, 5] = -1.0                                # one negative temperature
    with pytest.raises(pond.PondError):
        batch.set_state(fields)
    for s, (mac, neq) in zip(sims, before):
        m2, n2 = s.export_state()
        assert np.array_equal(mac.cpu().numpy(), m2.cpu().numpy())
        assert np.array_equal(neq.cpu().numpy(), n2.cpu().numpy())
        assert s.stats()[0] == pond.POND_OK
    batch.close()


def test_page_locked_host_buffers_are_used_in_place(pond):
    """Page-locked host buffers: the moments are written by the kernel in place (no staging
    copy); set_state / moments give the same results, bit for bit, as with pageable memory,
    single and batched, and a bad page-locked input is rejected without changing the state."""
    import torch
    cases = _grid_cases()
    pinned = [tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (c.rho, c.ux, c.uy, c.T))
              for c in cases]
    a = _tube_sims(pond, cases)                       # pageable numpy input
    b = []
    for c, f in zip(cases, pinned):
        s = pond.Simulation(pond.Config(nx=c.nx, ny=c.ny, precision="fp32", gamma=c.gamma, mu=c.mu,
                                        bc_x=c.bc_x, bc_y=c.bc_y))
        rc = pond.pond_set_state(s.handle, *[t.data_ptr() for t in f], 0)
        assert rc == 0
        b.append(s)
    for x, y in zip(a, b):
        x.step(3)
        y.step(3)
        outs = [torch.empty(x.cfg.ny, x.cfg.nx, dtype=torch.float64).pin_memory() for _ in range(4)]
        assert pond.pond_get_moments(y.handle, *[o.data_ptr() for o in outs], 0) == 0
        for u, v in zip(x.moments(), outs):
            assert np.array_equal(u, v.numpy())
    # batched, page-locked in and out
    batch = pond.Batch(b)
    cols = [[f[k].data_ptr() for f in pinned] for k in range(4)]
    assert pond.pond_batch_set_state(batch.handle, *cols, 0) == 0
    batch.step(3)
    outs = [[torch.empty(s.cfg.ny, s.cfg.nx, dtype=torch.float64).pin_memory() for _ in range(4)] for s in b]
    assert pond.pond_batch_get_moments(batch.handle, *[[o[k].data_ptr() for o in outs] for k in range(4)], 0) == 0
    for x, o in zip(a, outs):
        for u, v in zip(x.moments(), o):
            assert np.array_equal(u, v.numpy())
    # a bad page-locked input is rejected and changes nothing
    before = b[0].export_state()
    bad = [t.clone().pin_memory() for t in pinned[0]]
    bad[3][1, 2] = float("nan")
    assert pond.pond_set_state(b[0].handle, *[t.data_ptr() for t in bad], 0) == pond.POND_EINVAL
    after = b[0].export_state()
    assert torch.equal(before[0], after[0]) and torch.equal(before[1], after[1])
    batch.close()


@pytest.mark.parametrize("split", ["total", "internal"])
def test_batch_state_calls_over_several_launch_chunks(pond, split):
    """More members than one batched auxiliary launch takes (64): uneven tubes, host
    (pageable and page-locked) and device fields, against the per-member calls bit for bit;
    a bad value in a member of a later chunk is rejected and changes no member."""
    import torch
    cases = W.tube_batch(count=150, seed=5, nmin=40, nmax=700)
    ref = _tube_sims(pond, cases, split=split)
    for s in ref:
        s.step(2)
    sims = _tube_sims(pond, cases, split=split)
    for s in sims:
        s.step(1)                                          # states to be replaced
    batch = pond.Batch(sims)
    batch.set_state([(c.rho, c.ux, c.uy, c.T) for c in cases])
    batch.step(2)
    for got, s in zip(batch.moments(), ref):
        for x, y in zip(got, s.moments()):
            assert np.array_equal(x, y)
    # page-locked in and out
    pinned = [tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (c.rho, c.ux, c.uy, c.T))
              for c in cases]
    assert pond.pond_batch_set_state(batch.handle, *[[f[k].data_ptr() for f in pinned] for k in range(4)], 0) == 0
    batch.step(2)
    outs = [[torch.empty(c.ny, c.nx, dtype=torch.float64).pin_memory() for _ in range(4)] for c in cases]
    rc = pond.pond_batch_get_moments(batch.handle, *[[o[k].data_ptr() for o in outs] for k in range(4)], 0)
    assert rc in (pond.POND_OK, pond.POND_ENOCONV)
    for o, s in zip(outs, ref):
        for u, v in zip(s.moments(), o):
            assert np.array_equal(u, v.numpy())
    # device in and out
    dev = [tuple(torch.as_tensor(a, device="cuda") for a in (c.rho, c.ux, c.uy, c.T)) for c in cases]
    batch.set_state(dev)
    batch.step(2)
    douts = [[torch.empty(c.ny, c.nx, dtype=torch.float64, device="cuda") for _ in range(4)] for c in cases]
    rc = pond.pond_batch_get_moments(batch.handle, *[[o[k].data_ptr() for o in douts] for k in range(4)], 1)
    assert rc in (pond.POND_OK, pond.POND_ENOCONV)
    for o, s in zip(douts, ref):
        for u, v in zip(s.moments(), o):
            assert np.array_equal(u, v.cpu().numpy())
    # a bad value in member 130 (third chunk)
    before = [s.export_state() for s in sims]
    fields = [(c.rho.copy(), c.ux.copy(), c.uy.copy(), c.T.copy()) for c in cases]
    fields[130][0][0, 3] = float("inf")
    with pytest.raises(pond.PondError):
        batch.set_state(fields)
    # and the same through page-locked input (read in place by the staging kernel)
    bad = [tuple(t.clone().pin_memory() for t in f) for f in pinned]
    bad[130][3][0, 7] = -2.0
    rc = pond.pond_batch_set_state(batch.handle, *[[f[k].data_ptr() for f in bad] for k in range(4)], 0)
    assert rc == pond.POND_EINVAL
    for s, (mac, neq) in zip(sims, before):
        m2, n2 = s.export_state()
        assert torch.equal(mac, m2) and torch.equal(neq, n2)
        assert s.stats()[0] == pond.POND_OK
    batch.close()


@pytest.mark.parametrize("where", ["device", "page-locked"])
def test_batched_moments_skip_absent_outputs(pond, where):
    """pond_batch_get_moments with whole fields absent (NULL arrays) and single members'
    buffers absent (NULL entries): the given buffers get the per-member values, bit for bit,
    and the absent ones are skipped."""
    import torch
    cases = W.tube_batch(count=70, seed=8, nmin=40, nmax=300)     # two launch chunks
    ref = _tube_sims(pond, cases)
    sims = _tube_sims(pond, cases)
    for s in ref:
        s.step(2)
    batch = pond.Batch(sims)
    batch.step(2)
    dev = where == "device"

    def buf(c):
        if dev:
            return torch.full((c.ny, c.nx), -7.0, dtype=torch.float64, device="cuda")
        return torch.full((c.ny, c.nx), -7.0, dtype=torch.float64).pin_memory()

    T_out = [buf(c) for c in cases]
    ux_out = [buf(c) if i % 3 else None for i, c in enumerate(cases)]   # every third member absent
    rc = pond.pond_batch_get_moments(batch.handle, None, [o.data_ptr() if o is not None else 0 for o in ux_out],
                                     None, [o.data_ptr() for o in T_out], 1 if dev else 0)
    assert rc in (pond.POND_OK, pond.POND_ENOCONV)
    for i, s in enumerate(ref):
        rho, ux, uy, T = s.moments()
        assert np.array_equal(T_out[i].cpu().numpy(), T)
        if ux_out[i] is not None:
            assert np.array_equal(ux_out[i].cpu().numpy(), ux)
    batch.close()
