"""Benchmark of the PonD DDF-BGK step on GB300.

Workload (one "step"): one PonD time step of the periodic 256 x 256 decay configuration —
a shear wave u_y = 0.05 sin(2 pi x / 256) on rho = 1, T = 1 plus a Gaussian isobaric
thermal pulse (dT/T = 1e-3, width 16 cells), with background flow u_x = Ma sqrt(gamma)
for the four Mach numbers 0.5, 1, 1.5, 2 (four independent 256^2 grids), D2Q16, total
energy split, mixed precision (FP32 arithmetic, FP64 frames).  The four grids advance as one
batch (pond_batch: one kernel launch per time step).  Synthetic, seeded inputs.

Metric: MLUPS = node updates per second / 1e6 over the whole job (all ranks).  The line
also carries the plain-FP64 GPU step on the same workload, the L1 error of the mixed path
against the FP64 path, the ALU roofline (FP32 and FP64 pipes) of the step kernel, the end-to-end rate
through the C-ABI with host buffers, and the FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU (torchrun): each rank advances its own copy of the workload (independent
problems, no collective on the data path); value = all ranks' node updates / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2405_11489_gb300 import workloads as W  # noqa: E402

NX = NY = 256
MACHS = (0.5, 1.0, 1.5, 2.0)
GAMMA = 1.4
MU = 0.05
METRIC = "PonD-DDF MLUPS, mixed-prec vs plain FP64 at stated L1 err; serving p50/p99 latency"
WORKLOAD = ("periodic 256x256 shear wave (u_y = 0.05 sin 2pi x/L) + Gaussian thermal pulse "
            "(dT/T = 1e-3, width 16), background Ma 0.5/1/1.5/2 (4 grids), D2Q16 total split")
# Unit counts of the CUDA-core pipes, flop per SM per clock: FP32 128 lanes x FMA (2 flop);
# FP64 2 FMA.  The peaks are these times the SM count read from the device and the SM clock
# sampled (nvidia-smi) while the timed kernels run.
FP32_FLOP_PER_SM_CLK = 128 * 2
FP64_FLOP_PER_SM_CLK = 2 * 2
FALLBACK_SM_MHZ = 2070.0        # the part's maximum SM clock, used only if sampling fails
# Algorithmic work of one node update, K = measured mean predictor-corrector iterations,
# for Q populations and P-point Lagrange stencils:
#  FP32: per iteration and population, the interpolation of the 20 order-<=3 Hermite
#        coefficients (f and g) over the stencil's taps (2 flop x 20 x P^2 in 2-D, x P along
#        the single row of a quasi-1-D grid, whose y taps all read that row) plus ~160 flop
#        for the frame move, the reconstruction and the moment sums; plus ~1000 flop per
#        update for staging and collision.  Cubic 2-D D2Q16: 800 Q K + 1000.
#  FP64: the conserved-moment sums (~130) and the frame update (~20) per iteration, plus ~50
#        per update (temperature recovery, final frame): 150 K + 50.
# The mixed-precision kernels execute all of it on the FP32 pipe (their moment sums and frame
# updates are FP32 deviations from FP64 reference values), so the roofline time of a node
# update is (F32 + F64) / P32, and the fraction of the roofline is that over the measured
# time.  The plain FP64 step executes all of it on the FP64 pipe: (F32 + F64) / P64.
FLOP_PER_POP_ITER_OVERHEAD = 160.0
FLOP_PER_UPDATE = 1000.0
F64_PER_ITER = 150.0
F64_PER_UPDATE = 50.0


def pipe_peaks(sms, sm_mhz):
    """FP32 and FP64 CUDA-core peaks (TFLOP/s) from the unit counts at sm_mhz."""
    hz = sm_mhz * 1e6
    return sms * FP32_FLOP_PER_SM_CLK * hz / 1e12, sms * FP64_FLOP_PER_SM_CLK * hz / 1e12


def algorithmic_flops(nodes, K, q=16, taps=4, one_d=False):
    """FP32 and FP64 algorithmic flop of `nodes` updates at mean iterations K."""
    n_taps = taps if one_d else taps * taps
    per_pop_iter = 2.0 * 20 * n_taps + FLOP_PER_POP_ITER_OVERHEAD
    f32 = nodes * (per_pop_iter * q * K + FLOP_PER_UPDATE)
    f64 = nodes * (F64_PER_ITER * K + F64_PER_UPDATE)
    return f32, f64


def roofline_fraction(f32, f64, seconds, peak_tflops):
    """Roofline time of the work on one pipe, (F32 + F64) / peak, over the measured time."""
    return (f32 + f64) / (peak_tflops * 1e12) / seconds


def case_fields(ma):
    shear = W.shear_wave(n=NX, ma=ma, amp=0.05, gamma=GAMMA, mu=MU)
    pulse = W.thermal_pulse(n=NX, amp=1e-3, width=16.0, gamma=GAMMA, mu=MU, ma=ma)
    return pulse.rho, shear.ux, shear.uy, pulse.T


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(step_ms, world, device=None):
    """The slowest rank's time per step (every rank gets it); a barrier follows.  device:
    where the reduction tensor lives (the rank's GPU under NCCL, the CPU under gloo)."""
    if world <= 1:
        return step_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([step_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def whole_job_mlups(world, nodes_per_step, step_ms):
    """Replicas (weak scaling): every rank advances its own copy of the workload, so the
    job's throughput is the node updates of all ranks over the slowest rank's time."""
    return world * nodes_per_step / (step_ms * 1e-3) / 1e6


class ClockSampler:
    """nvidia-smi samples (clocks and throttle reasons) taken while the timed kernels run.

    Sampling is live before the region starts (the first sample is awaited), every sample is
    stamped on arrival, and the summary keeps the samples between the region's start and end
    plus the first one after the end, which reports the state at the region's close (a region
    of a few milliseconds holds no sample of its own)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 50

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.stamped = []             # (monotonic seconds at arrival, csv line)
        self.t0 = self.t1 = None

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.stamped.append((time.monotonic(), line))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.INTERVAL_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        if self.proc is not None:
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            deadline = time.monotonic() + 5.0
            while not self.stamped and time.monotonic() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        self.t0 = time.monotonic()
        return self

    def __exit__(self, *exc):
        self.t1 = time.monotonic()
        if self.proc is None:
            return
        deadline = self.t1 + 4.0 * self.INTERVAL_MS * 1e-3
        while time.monotonic() < deadline and not any(t > self.t1 for t, _ in self.stamped):
            time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.reader.join(timeout=5)

    def region_lines(self):
        inside = [l for t, l in self.stamped if self.t0 <= t <= self.t1]
        after = [l for t, l in self.stamped if t > self.t1][:1]
        return inside + after

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.region_lines() if self.t0 is not None and self.t1 is not None else []
        for l in lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": self.INTERVAL_MS,
                "region_ms": round(1e3 * (self.t1 - self.t0), 1)}


def l2_flusher(torch, device):
    buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)  # > 129 MB L2
    def flush():
        buf.zero_()
    return flush


def make_sims(pond, precision, device, stream, tune=False):
    """The four decay grids as one batch; with tune, the launch shape is picked by the
    library's autotuner on the first grid and used for all four (same class)."""
    sims = []
    for ma in MACHS:
        cfg = pond.Config(nx=NX, ny=NY, precision=precision, gamma=GAMMA, mu=MU)
        s = pond.Simulation(cfg, device=device, stream=stream)
        s.set_state(*case_fields(ma))
        sims.append(s)
    tuning = None
    if tune:
        tuning = sims[0].autotune(steps=8, apply=True)
        for s in sims[1:]:
            s.set_launch(tuning["tile_x"], tuning["tile_y"], tuning["halo"])
    batch = pond.Batch(sims, stream=stream)
    return (sims, batch, tuning) if tune else (sims, batch)


def time_steps(torch, batch, stream, steps, warmup, flush, clock=None):
    """CUDA-event time of every batched step (one launch over all grids), L2 flushed before
    each timed step; a clock sampler's region starts after the warm-up steps."""
    for _ in range(warmup):
        batch.step(1)
    torch.cuda.nvtx.range_push("warm_up")            # the first range call loads the NVTX library
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if clock is not None:
        clock.t0 = time.monotonic()
    starts, ends = [], []
    torch.cuda.nvtx.range_push("timed_steps")       # lets a profiler select the timed launches
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.step(1)
        e1.record(stream)
        starts.append(e0)
        ends.append(e1)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in zip(starts, ends)]


def tube_batch_rates(torch, pond, device, steps=20):
    """The 256 uneven quasi-1-D shock tubes (N ~ logU[200, 4000], seed 1), D2Q16 FP32:
    MLUPS of a per-case launch loop, of one batched launch per step, and of the batched
    steps replayed from a captured CUDA graph."""
    cases = W.tube_batch(count=256, seed=1)
    stream = torch.cuda.Stream(device)
    sims = []
    for c in cases:
        s = pond.Simulation(pond.Config(nx=c.nx, ny=c.ny, precision="fp32", gamma=c.gamma, mu=c.mu,
                                        bc_x=c.bc_x, bc_y=c.bc_y, interp_order=2),
                            device=device, stream=stream)
        s.set_state(c.rho, c.ux, c.uy, c.T)
        sims.append(s)
    nodes = sum(c.nx * c.ny for c in cases)
    out = {"cases": len(cases), "nodes": nodes}
    # launch shape: autotuned on the longest tube, used by every member (one class)
    big = max(range(len(cases)), key=lambda i: cases[i].nx)
    out["autotune"] = sims[big].autotune(steps=3, apply=True)
    for s in sims:
        s.set_launch(0, 0, out["autotune"]["halo"])

    def timed(fn):
        fn(2)
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        e1.synchronize()
        return nodes * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6

    def loop(n):
        for _ in range(n):
            for s in sims:
                s.step(1)
    out["per_case_loop_mlups"] = timed(loop)
    batch = pond.Batch(sims, stream=stream)
    out["batched_launch_mlups"] = timed(batch.step)
    batch.use_graph(steps)
    out["batched_graph_mlups"] = timed(batch.step)
    out["launches_per_step"] = {"per_case_loop": len(cases), "batched": 1}
    batch.close()
    out["statuses"] = sorted({pond.strerror(s.stats()[0]) for s in sims})
    out["pc_iters_mean"] = mean_iters(sims)
    out["interp_order"] = 2
    for s in sims:
        s.close()
    return out


def config_rates(torch, pond, device, steps=6):
    """MLUPS of the other configurations, and the two relative costs the paper reports
    (internal vs total energy split, D2Q25 vs D2Q16), each measured on one GPU."""
    def rate(case, steps, **kw):
        stream = torch.cuda.current_stream(device)
        walls = case.meta.get("walls")
        cfg = pond.Config(nx=case.nx, ny=case.ny, gamma=case.gamma, mu=case.mu, bc_x=case.bc_x,
                          bc_y=case.bc_y, walls=tuple(walls) if walls else None, **kw)
        s = pond.Simulation(cfg, device=device, stream=stream)
        if case.meta.get("profile") is not None:
            s.set_boundary_profile("x_low", case.meta["profile"])
        s.set_state(case.rho, case.ux, case.uy, case.T)
        tuning = s.autotune(steps=2, apply=True)
        s.step(2)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step(steps)
        e1.record(stream)
        e1.synchronize()
        rc, st = s.stats()
        s.close()
        return {"mlups": case.nx * case.ny * steps / (e0.elapsed_time(e1) * 1e-3) / 1e6,
                "pc_iters_mean": st.pc_iters_total / max(st.node_updates, 1),
                "status": pond.strerror(rc),
                "launch_shape": "%dx%d halo %d" % (tuning["tile_x"], tuning["tile_y"], tuning["halo"])}
    out = {}
    rie = W.riemann2d(n=1024, seed=0)
    out["riemann_1024_total_fp32"] = rate(rie, steps, interp_order=2)
    out["riemann_1024_internal_fp32"] = rate(rie, steps, split="internal", interp_order=2)
    out["internal_over_total_time"] = (out["riemann_1024_total_fp32"]["mlups"]
                                       / out["riemann_1024_internal_fp32"]["mlups"])
    dec = W.shear_wave(n=NX, ma=1.0, amp=0.05, gamma=GAMMA, mu=MU)
    out["decay_256_d2q16_fp32"] = rate(dec, 4 * steps)
    out["decay_256_d2q16_fp16_storage"] = rate(dec, 4 * steps, precision="fp16")
    out["decay_256_d2q16_bf16_storage"] = rate(dec, 4 * steps, precision="bf16")
    out["decay_256_d2q25_fp32"] = rate(dec, 4 * steps, lattice=25)
    out["d2q25_over_d2q16_time"] = (out["decay_256_d2q16_fp32"]["mlups"]
                                    / out["decay_256_d2q25_fp32"]["mlups"])
    # the non-translational split on its lattice (D2Q25, Grad order 4) and on D2Q16
    out["decay_256_d2q25_nt_fp32"] = rate(dec, 4 * steps, lattice=25, split="nt")
    out["decay_256_d2q16_nt_fp32"] = rate(dec, 4 * steps, split="nt")
    out["nt_over_total_time_d2q25"] = (out["decay_256_d2q25_fp32"]["mlups"]
                                       / out["decay_256_d2q25_nt_fp32"]["mlups"])
    # the jet of Sec. III.C at its resolution (2000 x 1000, D = 100, the paper's jet and
    # ambient states) through a profiled inflow side, at Mach 1.5 (the paper's Mach 80 turns
    # non-physical within a few steps, also in the FP64 oracle)
    out["jet_2000x1000_ma1.5_fp32"] = rate(W.jet(ma=1.5), steps)
    sod = W.sod(nx=400, ny=4)
    out["sod_400x4_fp64"] = rate(sod, 50, precision="fp64")
    out["grad_order"] = {"d2q16": 3, "d2q25": 4}
    out["paper_reports"] = {"internal_over_total_time": 1.15, "d2q25_over_d2q16_time": 1.6,
                            "hardware": "not stated (CSCS allocation acknowledged)"}
    return out


def mean_iters(sims):
    tot = it = 0
    for s in sims:
        rc, st = s.stats()
        tot += st.node_updates
        it += st.pc_iters_total
    return it / max(tot, 1)


def l1_error(pond, device, stream, nsteps=200):
    """Per-field relative L1 error of the mixed paths (FP32 storage, and FP16 / BF16 storage
    with FP32 arithmetic) against the FP64 path (which matches the oracle to 1e-12 in the
    parity tests) on the Ma = 1 grid after nsteps."""
    res = {}
    for prec in ("fp32", "fp16", "bf16", "fp64"):
        s = pond.Simulation(pond.Config(nx=NX, ny=NY, precision=prec, gamma=GAMMA, mu=MU),
                            device=device, stream=stream)
        s.set_state(*case_fields(1.0))
        s.step(nsteps)
        res[prec] = s.moments()
        s.close()
    names = ("rho", "ux", "uy", "T")

    def errors(prec):
        out = {}
        for n, a, b in zip(names, res[prec], res["fp64"]):
            out[n] = float(np.mean(np.abs(a - b)) / np.mean(np.abs(b)))
        # the perturbations themselves: error relative to the signal (deviation from the mean)
        for n, a, b in zip(names, res[prec], res["fp64"]):
            dev = np.mean(np.abs(b - b.mean()))
            out[n + "_vs_signal"] = float(np.mean(np.abs(a - b)) / dev) if dev > 0 else None
        return out
    return {"steps": nsteps, "rel_l1": errors("fp32"), "rel_l1_fp16_storage": errors("fp16"),
            "rel_l1_bf16_storage": errors("bf16")}


def decay_physics(torch, pond, device, steps=2000):
    """The 256^2 decay configuration over `steps` steps in mixed FP32 and in FP64: decay of the
    shear wave's Fourier mode against exp(-nu k^2 t), nu = mu / rho (Sec. III.B), of the
    thermal pulse's peak against 2-D diffusion sigma0^2 / (sigma0^2 + 2 alpha t) with
    alpha = nu (Pr = 1) (in the combined grids and, without the shear wave, in pulse-only
    grids on the same backgrounds), the drift of total mass, momentum and energy, and the per-field
    relative L1 difference of the FP32 result from the FP64 one."""
    k = 2 * math.pi / NX
    shear_expected = math.exp(-MU * k * k * steps)
    sigma0 = 16.0
    pulse_expected = sigma0 ** 2 / (sigma0 ** 2 + 2 * MU * steps)
    cv = 1.0 / (GAMMA - 1.0)

    def totals(f):
        rho, ux, uy, T = f
        E = rho * (cv * T + 0.5 * (ux * ux + uy * uy))
        return np.array([rho.sum(), (rho * ux).sum(), (rho * uy).sum(), E.sum()])

    def pulse(T):
        # the pulse over the local background: the shear wave's viscous heating varies along x
        # only, and the pulse covers a small part of each column, so the column median is the
        # background
        return (T - np.median(T, axis=0, keepdims=True)).max()

    def measure(fields0, fields):
        uy0, uy1 = fields0[2], fields[2]
        a0 = abs(np.fft.fft(uy0.mean(axis=0))[1])
        a1 = abs(np.fft.fft(uy1.mean(axis=0))[1])
        t0, t1 = totals(fields0), totals(fields)
        rho, ux, uy, T = fields0
        mom = (rho * (np.sqrt(ux * ux + uy * uy) + np.sqrt(T))).sum()   # momentum scale
        scale = np.array([t0[0], mom, mom, t0[3]])
        # (the pulse-only grids carry no shear wave: no amplitude ratio there)
        shear = a1 / a0 if a0 > 0 else float("nan")
        return shear, pulse(fields[3]) / pulse(fields0[3]), np.abs(t1 - t0) / scale

    out = {"steps": steps, "shear_expected": shear_expected, "pulse_expected": pulse_expected}
    finals = {}
    for prec in ("fp32", "fp64"):
        stream = torch.cuda.current_stream(device)
        sims, _ = make_sims(pond, prec, device, stream)
        # the pulse alone on the same backgrounds: its decay without the shear wave's heating
        solo = []
        for ma in MACHS:
            c = W.thermal_pulse(n=NX, amp=1e-3, width=sigma0, gamma=GAMMA, mu=MU, ma=ma)
            s = pond.Simulation(pond.Config(nx=NX, ny=NY, precision=prec, gamma=GAMMA, mu=MU),
                                device=device, stream=stream)
            s.set_state(c.rho, c.ux, c.uy, c.T)
            solo.append(s)
        batch = pond.Batch(sims + solo, stream=stream)
        f0 = [s.moments() for s in sims + solo]
        batch.step(steps)
        stream.synchronize()
        f1 = [s.moments() for s in sims + solo]
        n = len(sims)
        res = [measure(a, b) for a, b in zip(f0[:n], f1[:n])]
        res_solo = [measure(a, b) for a, b in zip(f0[n:], f1[n:])]
        out[prec] = {"shear_ratio_over_expected": [r[0] / shear_expected for r in res],
                     "pulse_ratio_over_expected": [r[1] / pulse_expected for r in res],
                     "pulse_only_ratio_over_expected": [r[1] / pulse_expected for r in res_solo],
                     "max_rel_drift_mass_momx_momy_energy": np.max([r[2] for r in res], axis=0).tolist(),
                     "statuses": sorted({pond.strerror(s.stats()[0]) for s in sims + solo})}
        finals[prec] = f1[:n]
        batch.close()
        for s in sims + solo:
            s.close()
    l1 = {}
    for name, idx in (("rho", 0), ("ux", 1), ("uy", 2), ("T", 3)):
        num = sum(np.abs(a[idx] - b[idx]).sum() for a, b in zip(finals["fp32"], finals["fp64"]))
        den = sum(np.abs(b[idx]).sum() for b in finals["fp64"])
        l1[name] = num / den
    out["l1_fp32_vs_fp64"] = l1
    out["machs"] = list(MACHS)
    return out


def alu_peak(torch, pond, device, sms, seconds=0.3, launches=3):
    """The FP32 and FP64 FMA rates of the device's CUDA-core pipes (pond_alu_peak: independent
    FMA chains, 4 blocks of 256 threads per SM), each over `launches` launches of about
    `seconds` each, with the SM clock sampled meanwhile; beside each, the unit-count peak at
    the sampled clock and the measured fraction of it."""
    out = {}
    stream = torch.cuda.current_stream(device).cuda_stream
    for name, fp64 in (("fp32", False), ("fp64", True)):
        flop, ms = pond.pond_alu_peak(fp64, 64, stream)                  # warm-up, sizing
        iters = max(64, int(64 * seconds * 1e3 / max(ms, 1e-3)))
        rates = []
        with ClockSampler(device.index or 0) as clk:
            for _ in range(launches):
                flop, ms = pond.pond_alu_peak(fp64, iters, stream)
                rates.append(flop / (ms * 1e-3) / 1e12)
        c = clk.summary()
        mhz = c["sm_mhz"] or FALLBACK_SM_MHZ
        unit = pipe_peaks(sms, mhz)[1 if fp64 else 0]
        best = max(rates)
        out[name] = {"tflops": best, "sm_mhz": c["sm_mhz"], "clock_reasons": c["reasons"],
                     "unit_count_tflops_at_that_clock": unit, "fraction_of_unit_count": best / unit,
                     "launch_ms": ms, "launches": launches}
    return out


def e2e_rate(torch, pond, device, steps, warmup, tuning=None):
    """MLUPS of the benchmark's workload (the four grids, one batched launch per time step)
    through the public C-ABI with host buffers: every step uploads the four grids' input
    fields from pinned host memory (pond_batch_set_state: copies, input check, one
    synchronisation), advances the batch one time step (pond_batch_step) and reads every
    grid's resulting fields back (pond_batch_get_moments: one synchronisation), all inside
    the timed region.  tuning: the launch shape the device-timed steps use (as a user who
    tuned once would set it), else the default shape."""
    stream = torch.cuda.Stream(device)
    sims = [pond.Simulation(pond.Config(nx=NX, ny=NY, precision="fp32", gamma=GAMMA, mu=MU),
                            device=device, stream=stream) for _ in MACHS]
    if tuning is not None:
        for s in sims:
            s.set_launch(tuning["tile_x"], tuning["tile_y"], tuning["halo"])
    host_in = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in case_fields(ma)]
               for ma in MACHS]
    outs = [[torch.empty((NY, NX), dtype=torch.float64).pin_memory() for _ in range(4)]
            for _ in MACHS]
    batch = pond.Batch(sims, stream=stream)
    cols_in = [[fin[k].data_ptr() for fin in host_in] for k in range(4)]
    cols_out = [[fout[k].data_ptr() for fout in outs] for k in range(4)]

    def one():
        assert pond.pond_batch_set_state(batch.handle, *cols_in, 0) == 0
        assert pond.pond_batch_step(batch.handle, 1) == 0
        assert pond.pond_batch_get_moments(batch.handle, *cols_out, 0) in (0, pond.POND_ENOCONV)
        return outs[0][0][0, 0].item()

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    t = time.perf_counter() - t0
    batch.close()
    for s in sims:
        s.close()
    nbytes = len(MACHS) * 4 * NX * NY * 8          # four FP64 fields per grid, each direction
    return {"value": len(MACHS) * NX * NY * steps / t / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "note": "per step: pond_batch_set_state(host, 4 grids) + pond_batch_step(1) + "
                    "pond_batch_get_moments(host, 4 grids); host wall clock"}


def cpu_baseline(target_seconds=10.0, single_seconds=6.0):
    """The FP64 oracle, as it stands, on the host cores: the Ma = 1 grid of the workload,
    whole 256^2 field, as many time steps as fit in ~target_seconds (at least one) with
    OpenMP over every core; then the same on one thread (at least one step)."""
    import oracle
    oracle.build()
    cores = oracle.set_threads(os.cpu_count() or 1)
    cfg = oracle.make_config(NX, NY, gamma=GAMMA, mu=MU, pc_tol=1e-12)

    def rate(seconds):
        st = oracle.init_state(cfg, *case_fields(1.0))
        t0 = time.perf_counter()
        n = 0
        while True:
            st = oracle.step(cfg, st).state
            n += 1
            if time.perf_counter() - t0 > seconds:
                break
        return NX * NY * n / (time.perf_counter() - t0) / 1e6, n

    v, n = rate(target_seconds)
    oracle.set_threads(1)
    v1, n1 = rate(single_seconds)
    oracle.set_threads(cores)
    return {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": "FP64 oracle, %d time step(s) of the Ma = 1 256x256 grid (OpenMP, %d threads)"
                      % (n, cores),
            "single_thread": {"value": v1, "unit": "MLUPS", "steps": n1}}


def run_reference(args, world, rank):
    """The oracle as the reference arm: each step is one full time step of one of the four
    grids (rotating through the Mach numbers), so the run stays within a few minutes."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    cfgs, states = [], []
    for ma in MACHS:
        cfg = oracle.make_config(NX, NY, gamma=GAMMA, mu=MU, pc_tol=1e-12)
        cfgs.append(cfg)
        states.append(oracle.init_state(cfg, *case_fields(ma)))
    counter = [0]
    def one():
        k = counter[0] % len(states)
        states[k] = oracle.step(cfgs[k], states[k]).state
        counter[0] += 1
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    t = time.perf_counter() - t0
    v = NX * NY * args.steps / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "grids": len(MACHS)},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": "%d full time steps of single 256x256 grids (Ma cycling "
                                       "0.5/1/1.5/2), FP64 oracle, OpenMP" % args.steps},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def profile_case(torch, pond, device, stream, flush, args):
    """Batched steps of another configuration for a profiler: the four 256^2 decay grids on
    D2Q25 (mixed FP32) or in plain FP64, the 256 uneven tubes (3-point stencil, mixed FP32),
    or the 1024^2 four-quadrant Riemann problem (total split, 3-point stencil, mixed FP32),
    each with the launch shape the autotuner picks; prints one JSON line."""
    if args.profile_case == "riemann":
        c = W.riemann2d(n=1024, seed=0)
        s = pond.Simulation(pond.Config(nx=c.nx, ny=c.ny, precision="fp32", gamma=c.gamma, mu=c.mu,
                                        bc_x=c.bc_x, bc_y=c.bc_y, interp_order=2),
                            device=device, stream=stream)
        s.set_state(c.rho, c.ux, c.uy, c.T)
        tuning = s.autotune(steps=2, apply=True)
        sims = [s]
        nodes = c.nx * c.ny
    elif args.profile_case == "tubes":
        cases = W.tube_batch(count=256, seed=1)
        sims = []
        for c in cases:
            s = pond.Simulation(pond.Config(nx=c.nx, ny=c.ny, precision="fp32", gamma=c.gamma,
                                            mu=c.mu, bc_x=c.bc_x, bc_y=c.bc_y, interp_order=2),
                                device=device, stream=stream)
            s.set_state(c.rho, c.ux, c.uy, c.T)
            sims.append(s)
        big = max(range(len(cases)), key=lambda i: cases[i].nx)
        tuning = sims[big].autotune(steps=3, apply=True)
        for s in sims:
            s.set_launch(0, 0, tuning["halo"])
        nodes = sum(c.nx * c.ny for c in cases)
    else:
        prec, lattice = ("fp32", 25) if args.profile_case == "d2q25" else ("fp64", 16)
        sims = []
        for ma in MACHS:
            s = pond.Simulation(pond.Config(nx=NX, ny=NY, precision=prec, lattice=lattice, gamma=GAMMA,
                                            mu=MU), device=device, stream=stream)
            s.set_state(*case_fields(ma))
            sims.append(s)
        tuning = sims[0].autotune(steps=3, apply=True)
        for s in sims[1:]:
            s.set_launch(tuning["tile_x"], tuning["tile_y"], tuning["halo"])
        nodes = len(MACHS) * NX * NY
    batch = pond.Batch(sims, stream=stream)
    per = time_steps(torch, batch, stream, args.steps, args.warmup, flush)
    ms = sum(per) / len(per)
    print(json.dumps({"case": args.profile_case, "mlups": nodes / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                      "pc_iters_mean": mean_iters(sims), "launch_shape": tuning}))
    batch.close()
    for s in sims:
        s.close()
    return 0


def other_rooflines(tubes, others, p32, sm_mhz):
    """ALU roofline fractions of the larger workloads: the 1024^2 Riemann problem (total split,
    3-point stencils, 2-D) and the 256 tubes in one batched launch per step (3-point stencils,
    quasi-1-D), each from its measured MLUPS and mean iterations, against the FP32 peak at the
    headline's sampled SM clock."""
    out = {}
    rie = others["riemann_1024_total_fp32"]
    cases = (("riemann_1024_total_fp32", rie["mlups"], rie["pc_iters_mean"], False),
             ("tube_batch_256_batched", tubes["batched_launch_mlups"], tubes["pc_iters_mean"], True))
    for name, mlups, K, one_d in cases:
        f32, f64 = algorithmic_flops(1, K, taps=3, one_d=one_d)
        t = 1.0 / (mlups * 1e6)                      # seconds per node update
        out[name] = {"bound": "alu", "achieved": (f32 + f64) / t / 1e12, "peak": p32,
                     "unit": "TFLOP/s", "frac": roofline_fraction(f32, f64, t, p32),
                     "flop_per_update": f32 + f64, "pc_iters_mean": K, "mlups": mlups,
                     "stencil": "3-point, %s" % ("quasi-1-D (x taps only)" if one_d else "2-D (3 x 3 taps)"),
                     "sm_mhz": sm_mhz}
    return out


def profiled_traffic(key):
    """DRAM bytes (read + write) per launch of the timed kernel from the committed ncu record,
    or None when the record is missing or the kernel sources have changed since the capture."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(prof))[key]
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
    except (OSError, ValueError, KeyError):
        return None
    return rec["bytes_per_launch"] if h.hexdigest() == rec["sources_sha256"] else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pond", choices=["pond", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10000,
                    help="requests of the Poisson serving run (default: the configured stream of "
                         "10 000 requests at 50 per second, about 200 s)")
    ap.add_argument("--profile-case", choices=["d2q25", "fp64", "tubes", "riemann"], default=None,
                    help="time one other configuration's batched steps (inside the NVTX range "
                         "timed_steps, for profiler runs) and print its rate")
    ap.add_argument("--quick", action="store_true",
                    help="timed mixed-precision steps only (for profiler runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_init()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    from paper_2405_11489_gb300 import build as B
    B.build()
    from paper_2405_11489_gb300 import pond
    pond.load_library()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    stream = torch.cuda.current_stream(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)

    flush = l2_flusher(torch, device)
    if args.profile_case:
        return profile_case(torch, pond, device, stream, flush, args)
    sims, batch, tuning = make_sims(pond, "fp32", device, stream, tune=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        per_launch = time_steps(torch, batch, stream, args.steps, args.warmup, flush, clock=clk)
    step_ms = max_over_ranks(sum(per_launch) / args.steps, world, device)
    K = mean_iters(sims)
    batch.close()
    for s in sims:
        s.close()
    nodes_per_step = len(MACHS) * NX * NY
    value = whole_job_mlups(world, nodes_per_step, step_ms)
    launch_ms = sum(per_launch) / len(per_launch)
    clocks = clk.summary()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    sm_mhz = clocks["sm_mhz"] or FALLBACK_SM_MHZ
    p32, p64 = pipe_peaks(sms, sm_mhz)
    f32_launch, f64_launch = algorithmic_flops(nodes_per_step, K)
    flops_per_launch = f32_launch + f64_launch
    achieved = flops_per_launch / (launch_ms * 1e-3) / 1e12
    frac = roofline_fraction(f32_launch, f64_launch, launch_ms * 1e-3, p32)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    if args.quick:
        print(json.dumps({"metric": METRIC, "value": value, "unit": "MLUPS", "quick": True,
                          "ms_per_step": step_ms, "pc_iters_mean": K, "launch_ms": launch_ms,
                          "achieved_tflops": achieved, "roofline_frac": frac, "clocks": clocks}))
        return 0
    # plain FP64 GPU step on the same workload (fewer steps: it is ~two orders slower)
    sims64, batch64, tune64 = make_sims(pond, "fp64", device, stream, tune=True)
    per64 = time_steps(torch, batch64, stream, max(2, args.steps // 10), 1, flush)
    K64 = mean_iters(sims64)
    batch64.close()
    for s in sims64:
        s.close()
    fp64_ms = sum(per64) / max(2, args.steps // 10)
    err = l1_error(pond, device, stream)
    decay = decay_physics(torch, pond, device)
    e2e = e2e_rate(torch, pond, device, steps=max(5, args.steps), warmup=3, tuning=tuning)
    tubes = tube_batch_rates(torch, pond, device)
    others = config_rates(torch, pond, device)
    from paper_2405_11489_gb300.serve import serve_benchmark
    serving = serve_benchmark(args.serve_requests, rate=50.0, seed=2, load=0.7, chunk=32,
                              device=device)
    alu = alu_peak(torch, pond, device, sms)
    others_roofline = other_rooflines(tubes, others, p32, sm_mhz)
    cpu = None if args.no_cpu_baseline else cpu_baseline()
    traffic = profiled_traffic("step_kernel_fp32_batched_4x256x256")
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "grids": len(MACHS),
                   "precision": "mixed: FP32 arithmetic and non-equilibrium state, FP64 rho/u/T, "
                                "compensated moment sums",
                   "l2": "flushed (256 MB write) before every timed step",
                   "launch_shape": "tile %dx%d, halo %d (autotuned)" % (tuning["tile_x"], tuning["tile_y"],
                                                                      tuning["halo"]),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "pc_iters_mean": K,
        "autotune": tuning,
        "fp64": {"value": nodes_per_step / (fp64_ms * 1e-3) / 1e6, "unit": "MLUPS",
                 "ms_per_step": fp64_ms, "speedup_mixed_over_fp64": fp64_ms / step_ms,
                 "pc_iters_mean": K64,
                 # every flop on the FP64 pipe: (F32 + F64) / P64 over the measured time
                 "roofline_frac": roofline_fraction(*algorithmic_flops(nodes_per_step, K64),
                                                    fp64_ms * 1e-3, p64),
                 "launch_shape": "tile %dx%d, halo %d (autotuned)" % (tune64["tile_x"], tune64["tile_y"],
                                                                    tune64["halo"])},
        "l1_err_mixed_vs_fp64": err,
        "decay_2000": decay,
        "tube_batch": tubes,
        "other_configs": others,
        "serving": serving,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": p32, "unit": "TFLOP/s",
                     "frac": frac, "traffic": traffic,
                     "flop_basis": "algorithmic FP32 + FP64 flop per launch, all executed on the "
                                   "FP32 pipe (the mixed kernel forms its moment sums and frame "
                                   "updates as FP32 deviations); frac = (F32 + F64) / P32 / t",
                     "f32_flop_per_launch": f32_launch, "f64_flop_per_launch": f64_launch,
                     "kernel": "step_kernel<float,float,4,4,false,256> (batched over the 4 grids)",
                     "peak_basis": "unit counts: %d SMs (device) x 128 FP32 lanes x 2 flop x %.0f MHz "
                                   "(median SM clock sampled during the timed launches)" % (sms, sm_mhz),
                     "sms": sms, "sm_mhz": sm_mhz,
                     "measured_fma_tflops": alu["fp32"]["tflops"],
                     "frac_of_measured_fma": achieved / alu["fp32"]["tflops"],
                     "launch_ms": launch_ms},
        "rooflines_other": others_roofline,
        "alu_peak": alu,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": len(per_launch),
        "clocks": clocks,
    }
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
