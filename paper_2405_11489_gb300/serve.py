"""Continuous-batching serving loop for PonD simulations (a host scheduler over libpond).

Requests (an initial state, a configuration and a number of time steps) arrive over time.
The server admits them in arrival order while their device workspace fits the memory budget
(free HBM at start-up, or a given cap), keeps their state resident on the GPU, and advances
every admitted request in ticks.  In a tick the active requests are grouped into
compatibility classes (precision, lattice, interpolation order, 1-D/2-D) and each class
advances as one pond_batch -- one kernel launch per time step for all its members -- on its
own CUDA stream, so classes overlap on the device and requests that arrived while others were
running join at the next tick.  A tick advances a class by min(chunk, smallest remaining step
count of its members) steps, so every request stops exactly at its step count; finished
requests return their fields (rho, u_x, u_y, T) and free their workspace for waiting ones.

Each result is the same as running the request alone: the per-node arithmetic of a batched
launch does not depend on the other members.

The GPU work goes through a backend object (``PondBackend`` here); the scheduling logic is
backend-agnostic so that it can be exercised without a GPU.
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Active:
    req: object
    sim: object
    bytes: int
    remaining: int
    admitted_at: float


@dataclass
class Completion:
    rid: int
    arrival: float
    admitted: float
    done: float
    steps: int
    nodes: int
    status: str
    fields: tuple = field(default=None, repr=False)
    what: str = ""              # request type, grid, split and precision


def percentile(values, q):
    if not values:
        return None
    v = sorted(values)
    k = (len(v) - 1) * q / 100.0
    lo, hi = math.floor(k), math.ceil(k)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


class Server:
    """Admission, resident state and ticked continuous batching over a backend."""

    def __init__(self, backend, budget_bytes, chunk=16, keep_fields=False, clock=time.perf_counter):
        self.be = backend
        self.budget = int(budget_bytes)
        self.chunk = int(chunk)
        self.keep_fields = keep_fields
        self.clock = clock
        self.used = 0
        self.waiting = deque()
        self.active = []
        self.done = []
        self.peak_used = 0
        self.ticks = 0
        self.node_updates = 0

    # -- admission -----------------------------------------------------------------------
    def _admit(self, now):
        while self.waiting:
            req = self.waiting[0]
            need = self.be.workspace_bytes(req)
            if need > self.budget:
                self.waiting.popleft()
                self.done.append(Completion(req.rid, req.arrival, now, now, 0, 0,
                                            "rejected: needs %d bytes, budget %d" % (need, self.budget)))
                continue
            if self.used + need > self.budget:
                break                                   # FIFO: wait for memory to free up
            self.waiting.popleft()
            sim = self.be.create(req)
            self.used += need
            self.peak_used = max(self.peak_used, self.used)
            self.active.append(Active(req, sim, need, req.steps, now))

    # -- ticks: each class advances on its own cadence -------------------------------------
    def _issue(self):
        """Start the next chunk of every class that has no work in flight."""
        classes = {}
        for a in self.active:
            key = self.be.class_key(a.req)
            if key not in self.inflight:
                classes.setdefault(key, []).append(a)
        for key, members in classes.items():
            n = min(self.chunk, min(a.remaining for a in members))
            token = self.be.advance(key, [a.sim for a in members], n)
            self.inflight[key] = (members, n, token)
            self.ticks += 1

    def _collect(self, block):
        """Retire finished chunks (waiting for the oldest one if block and none is ready)."""
        ready = [k for k, (_, _, tok) in self.inflight.items() if self.be.ready(tok)]
        if not ready and block and self.inflight:
            k0 = next(iter(self.inflight))
            self.be.wait_for(self.inflight[k0][2])
            ready = [k0]
        now = self.clock()
        for key in ready:
            members, n, _ = self.inflight.pop(key)
            for a in members:
                a.remaining -= n
                nodes = a.req.case.nx * a.req.case.ny
                self.node_updates += nodes * n
                if a.remaining <= 0:
                    fields, status = self.be.finish(a.sim)
                    self.used -= a.bytes
                    self.active.remove(a)
                    r = a.req
                    what = "%s %dx%d %s %s" % (getattr(r.case, "name", "case"), r.case.nx, r.case.ny,
                                               getattr(r, "split", ""), getattr(r, "precision", ""))
                    self.done.append(Completion(r.rid, r.arrival, a.admitted_at, now, r.steps, nodes,
                                                status, fields if self.keep_fields else None, what))
        return bool(ready)

    # -- the loop --------------------------------------------------------------------------
    def run(self, requests, realtime=True):
        """Serve the requests (sorted by arrival, seconds from the start); returns metrics."""
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        self.inflight = {}
        t0 = self.clock()
        offset = t0                      # arrival times are shifted to the server clock
        while pending or self.waiting or self.active:
            now = self.clock()
            while pending and (pending[0].arrival + offset <= now or not realtime):
                r = pending.popleft()
                r.arrival = r.arrival + offset if realtime else now
                self.waiting.append(r)
            self._admit(now)
            self._issue()
            next_arrival = pending[0].arrival + offset if (pending and realtime) else None
            # block on the GPU only when no arrival is due before the work could finish
            block = next_arrival is None or next_arrival - self.clock() > 0.002
            if not self._collect(block=block and bool(self.inflight)) and not self.inflight:
                if next_arrival is not None:
                    time.sleep(max(0.0, min(0.002, next_arrival - self.clock())))
        t1 = self.clock()
        return self.metrics(t1 - t0)

    def metrics(self, wall):
        served = [c for c in self.done if c.status != "" and not c.status.startswith("rejected")]
        ttr = [c.done - c.arrival for c in served]
        queue = [c.admitted - c.arrival for c in served]
        return {"requests": len(self.done), "served": len(served),
                "rejected": len(self.done) - len(served),
                "p50_time_to_result_s": percentile(ttr, 50), "p99_time_to_result_s": percentile(ttr, 99),
                "p50_queue_s": percentile(queue, 50), "p99_queue_s": percentile(queue, 99),
                "aggregate_mlups": self.node_updates / wall / 1e6 if wall > 0 else None,
                "wall_s": wall, "ticks": self.ticks, "peak_workspace_bytes": self.peak_used,
                "budget_bytes": self.budget,
                "statuses": sorted({c.status for c in served}),
                "status_counts": {st: sum(1 for c in served if c.status == st)
                                  for st in sorted({c.status for c in served})},
                "nonphysical_count": sum(1 for c in served if c.status.startswith("non-physical")),
                # requests whose state turned non-physical (first 20): id, type, grid, split, precision
                "nonphysical": [(c.rid, c.what) for c in served if c.status.startswith("non-physical")][:20]}


class PondBackend:
    """libpond on one GPU: a Simulation per request, one pond_batch per class per tick, one
    CUDA stream per class."""

    def __init__(self, device="cuda:0"):
        import torch
        from paper_2405_11489_gb300 import pond
        self.torch = torch
        self.pond = pond
        self.device = torch.device(device)
        self.streams = {}
        self.batches = {}

    def config(self, req):
        c = req.case
        return self.pond.Config(nx=c.nx, ny=c.ny, precision=req.precision, split=req.split,
                                interp_order=req.interp_order, gamma=c.gamma, mu=c.mu, bc_x=c.bc_x,
                                bc_y=c.bc_y)

    def workspace_bytes(self, req):
        return self.pond.pond_workspace_bytes(self.config(req).to_c()) + 256

    def class_key(self, req):
        return (req.precision, req.interp_order, req.case.ny == 1)

    def _stream(self, key):
        if key not in self.streams:
            self.streams[key] = self.torch.cuda.Stream(self.device)
        return self.streams[key]

    def create(self, req):
        key = self.class_key(req)
        stream = self._stream(key)
        sim = self.pond.Simulation(self.config(req), device=self.device, stream=stream)
        c = req.case
        # the fields go to the device on the class's stream and pond_set_state takes device
        # input, which does not synchronise: admitting a request never waits for the class's
        # chunk in flight (host input would be checked first, and the check waits for the
        # stream).  The generator's fields are physical; a bad value would show in the
        # request's status after its first step.
        torch = self.torch
        with torch.cuda.stream(stream):
            fields = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.device, non_blocking=True)
                      for a in (c.rho, c.ux, c.uy, c.T)]
            sim.set_state(*fields)
        return sim

    def advance(self, key, sims, n):
        """n time steps of the class on its stream, returning an event that completes with
        them; the class's pond_batch is rebuilt only when its membership has changed."""
        ids = tuple(id(x) for x in sims)
        cached = self.batches.get(key)
        if cached is None or cached[0] != ids:
            if cached is not None:
                cached[1].close()
            self.batches[key] = (ids, self.pond.Batch(sims, stream=self._stream(key)))
        self.batches[key][1].step(n)
        ev = self.torch.cuda.Event()
        ev.record(self._stream(key))
        return ev

    def ready(self, token):
        return token.query()

    def wait_for(self, token):
        token.synchronize()

    def finish(self, sim):
        rho, ux, uy, T = sim.moments(allow=(self.pond.POND_ENOCONV, self.pond.POND_ENONPHYSICAL))
        status = self.pond.strerror(sim.last_status)
        sim.close()
        return (rho, ux, uy, T), status


def calibrate(backend, requests, budget, chunk=16):
    """Node updates per second of the mix at saturation: every request admitted at once (as
    memory allows) and advanced to completion; used to scale step counts to a target load."""
    srv = Server(backend, budget_bytes=budget, chunk=chunk)
    t0 = time.perf_counter()
    srv.run(requests, realtime=False)
    return srv.node_updates / max(time.perf_counter() - t0, 1e-9)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--load", type=float, default=0.7, help="target offered load / capacity")
    ap.add_argument("--chunk", type=int, default=32)
    ap.add_argument("--budget-gb", type=float, default=0.0, help="0: 80 percent of free HBM")
    args = ap.parse_args(argv)
    result = serve_benchmark(args.requests, args.rate, args.seed, args.load, args.chunk,
                             args.budget_gb)
    print(json.dumps(result))
    return 0


def serve_benchmark(n_requests, rate=50.0, seed=2, load=0.7, chunk=32, budget_gb=0.0,
                    device="cuda:0"):
    """Poisson serving run: calibrate the capacity on a sample of the mix, scale the step
    counts so that the offered work is `load` x capacity at the given rate, serve."""
    import torch
    from paper_2405_11489_gb300 import workloads as W
    be = PondBackend(device)
    free, total = torch.cuda.mem_get_info(be.device)
    budget = int(budget_gb * 2 ** 30) if budget_gb > 0 else int(0.8 * free)
    sample = W.serving_requests(count=min(48, n_requests), rate=rate, seed=seed + 1000)
    capacity = calibrate(be, sample, budget, chunk)        # node updates per second
    work = sum(r.case.nx * r.case.ny * r.steps for r in sample) / len(sample)
    scale = load * capacity / (rate * work)
    reqs = W.serving_requests(count=n_requests, rate=rate, seed=seed, step_scale=scale)
    srv = Server(be, budget_bytes=budget, chunk=chunk)
    m = srv.run(reqs, realtime=True)
    offered = rate * sum(r.case.nx * r.case.ny * r.steps for r in reqs) / len(reqs)
    m.update({"rate_per_s": rate, "capacity_mlups": capacity / 1e6, "offered_mlups": offered / 1e6,
              "offered_load": offered / capacity, "step_scale": scale, "chunk_steps": chunk})
    return m


if __name__ == "__main__":
    sys.exit(main())
