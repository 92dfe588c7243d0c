"""pond_step_static: stepping without any device allocation.

Callers that cannot allocate device memory (an application whose own pool owns all GPU
memory, a real-time loop that cannot pay for cudaMalloc's latency and implicit
synchronisation, a foreign-language host holding only its state buffers) cannot give
pond_create a workspace.  pond_step_static advances a raw state kept in the caller's own
device buffers in place, with the second state copy in the library's 16 MiB static device
array.  These tests call it through the C ABI and check, on two calls in a row, that it
gives the same state as pond_step on a regular simulation, within the tolerances the
parity tests use.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_11489_gb300 import build, pond
    build.build()
    pond.load_library()
    return pond


def _fields(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx]
    T = 1.0 + 1e-3 * np.exp(-((x - nx / 2) ** 2 + (y - ny / 2) ** 2) / (2 * 6.0 ** 2))
    rho = 1.0 / T
    ux = np.full((ny, nx), 0.8)
    uy = 0.05 * np.sin(2 * np.pi * x / nx)
    return rho, ux, uy, T


def _views(torch, mac, neq, precision, nx, ny, planes=19):
    dt = {"fp64": torch.float64, "fp32": torch.float32, "fp16": torch.float16,
          "bf16": torch.bfloat16}[precision]
    N = nx * ny
    return (mac[: 4 * N * 8].view(torch.float64).cpu().numpy().reshape(4, N),
            neq[: planes * N * torch.tensor([], dtype=dt).element_size()].view(dt).float()
            .cpu().numpy().astype(np.float64).reshape(planes, N))


@pytest.mark.parametrize("precision,split,tol,lattice", [("fp64", "total", 1e-12, 16), ("fp32", "total", 1e-6, 16),
                                                         ("fp64", "internal", 1e-12, 16),
                                                         ("fp32", "nt", 1e-6, 25)])
def test_static_step_matches_pond_step_on_two_calls(P, precision, split, tol, lattice):
    import torch
    nx, ny = 70, 45
    planes = 19 if lattice == 16 else 29
    cfg = P.Config(nx=nx, ny=ny, precision=precision, split=split, mu=0.05, lattice=lattice)
    sim = P.Simulation(cfg)
    sim.set_state(*_fields(nx, ny))
    mac, neq = sim.export_state(on_device=True)      # the caller's own device buffers
    c = cfg.to_c()
    stream = torch.cuda.current_stream().cuda_stream
    for call, nsteps in enumerate((3, 2)):             # an odd and an even step count
        rc, st = P.pond_step_static(c, mac.data_ptr(), neq.data_ptr(), nsteps, stream)
        assert rc in (P.POND_OK, P.POND_ENOCONV), P.strerror(rc)
        assert st.node_updates == nsteps * nx * ny and st.pc_iters_total >= st.node_updates
        sim.step(nsteps)
        ref_mac, ref_neq = sim.export_state(on_device=True)
        a_mac, a_neq = _views(torch, mac, neq, precision, nx, ny, planes)
        r_mac, r_neq = _views(torch, ref_mac, ref_neq, precision, nx, ny, planes)
        for k in range(4):
            scale = max(np.max(np.abs(r_mac[k])), 1.0 if k in (1, 2) else 0.0)
            assert np.max(np.abs(a_mac[k] - r_mac[k])) <= tol * scale, (call, k)
        assert np.max(np.abs(a_neq - r_neq)) <= tol * max(np.max(np.abs(r_neq)), 1e-300), call
    sim.close()


def test_static_step_rejects_grids_beyond_the_array(P):
    """A grid larger than the array is refused before any launch; the caller's (real) buffers
    are left as they were."""
    import torch
    cfg = P.Config(nx=512, ny=512, precision="fp32")             # 262 144 nodes > 155 341
    c = cfg.to_c()
    mb, nb = P.pond_state_bytes(c)
    mac = torch.full((mb // 8,), 1.25, dtype=torch.float64, device="cuda")
    neq = torch.full((nb // 4,), -0.5, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc, _ = P.pond_step_static(c, mac.data_ptr(), neq.data_ptr(), 1, stream)
    assert rc == P.POND_ENOMEM
    torch.cuda.synchronize()
    assert bool((mac == 1.25).all()) and bool((neq == -0.5).all())
    lib = P.load_library()
    assert lib.pond_step_static(ctypes.byref(c), None, None, 1, None, None) == P.POND_EINVAL
