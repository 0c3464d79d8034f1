"""Serving loop for several simulated scanners: continuous batching of scan solves.

A model of the paper's multi-scanner hospital scenario (Sec. VI.D, where a discrete
event simulation feeds scans to a reconstruction cluster, earlier scans first), run
on one GPU with real reconstructions:

* scans arrive from several scanners (Poisson arrivals, seeded) and queue in arrival
  order (FCFS: the earlier scan goes first);
* a scan is admitted when its device footprint (plan workspace + its k-space and maps
  + the result) fits in the memory budget; its k-space and FISTA state then stay on the
  device until it finishes;
* admitted scans advance together in ticks of a few FISTA iterations, each on its own
  CUDA stream so that their kernels overlap; scans that arrive meanwhile join at the
  next tick boundary and finished scans leave (continuous batching);
* a virtual clock advances by the measured time of every tick, of every admission
  (the plan: maps, Psi, step; and A^H y) and of every completion (the result copy and
  the plan's release), and jumps over idle gaps, so arrival rates of minutes per scan
  need no waiting.  Latency = completion time - arrival time on that clock;
* a scan can be withdrawn (cancel): a queued one leaves the queue, a resident one has
  its plan closed and its memory returned at the next tick boundary.

Every step of a reconstruction runs in libt2sh (t2sh_solve_begin / _iterate / _end);
this module only schedules.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class ScanRequest:
    scan_id: int
    scanner: int
    arrival_s: float
    shape_index: int
    dims: object                 # t2sh.Dims
    phi: object                  # device tensors
    mask: object
    maps: object
    kspace: object
    kform: int
    footprint: int = 0
    # filled in by the server
    admitted_s: float = -1.0
    done_s: float = -1.0
    cancelled_s: float = -1.0
    result: object = None
    plan: object = field(default=None, repr=False)
    stream: object = field(default=None, repr=False)


def footprint_bytes(t2sh, dims, kform) -> int:
    """Device bytes one admitted scan holds: plan workspace, k-space, maps and result."""
    N = dims.ny * dims.nz
    kdim = dims.nechoes if kform == t2sh.KSPACE_TE else dims.nbasis
    k = dims.nslices * dims.ncoils * kdim * N * 8
    maps = dims.nslices * dims.ncoils * dims.nmaps * N * 8
    out = dims.nslices * dims.nmaps * dims.nbasis * N * 8
    return t2sh.workspace_bytes(dims) + k + maps + out


def poisson_arrivals(n_scans: int, n_scanners: int, mean_gap_s: float, seed: int):
    """(arrival time, scanner) of n_scans scans from n_scanners independent Poisson
    streams, each with mean inter-arrival mean_gap_s, merged in time order."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 7])))
    heap = [(rng.exponential(mean_gap_s), s) for s in range(n_scanners)]
    heapq.heapify(heap)
    out = []
    while len(out) < n_scans:
        t, s = heapq.heappop(heap)
        out.append((t, s))
        heapq.heappush(heap, (t + rng.exponential(mean_gap_s), s))
    return out


class Server:
    def __init__(self, t2sh, memory_budget: int, iters_per_tick: int = 10):
        import torch
        self.t2sh = t2sh
        self.torch = torch
        self.budget = int(memory_budget)
        self.iters_per_tick = int(iters_per_tick)
        self.queue: list[ScanRequest] = []
        self.active: list[ScanRequest] = []
        self.done: list[ScanRequest] = []
        self.cancelled: list[ScanRequest] = []
        self.cancel_requests: list[tuple[float, int]] = []
        self.now = 0.0
        self.used = 0
        self.busy_s = 0.0
        self.admit_s = 0.0  # part of busy_s spent admitting scans (plan + A^H y)
        self.ticks = 0
        self.max_active = 0

    def submit(self, req: ScanRequest):
        req.footprint = footprint_bytes(self.t2sh, req.dims, req.kform)
        if req.footprint > self.budget:
            raise ValueError(f"scan {req.scan_id} needs {req.footprint} bytes, budget {self.budget}")
        self.queue.append(req)
        self.queue.sort(key=lambda r: (r.arrival_s, r.scan_id))

    def cancel(self, scan_id: int, at_s: float = 0.0):
        """Withdraw scan `scan_id` at virtual time at_s (applied at the first tick boundary
        at or after it).  A scan that has already finished by then is left alone."""
        self.cancel_requests.append((float(at_s), int(scan_id)))
        self.cancel_requests.sort()

    def _apply_cancellations(self):
        while self.cancel_requests and self.cancel_requests[0][0] <= self.now:
            _, sid = self.cancel_requests.pop(0)
            for i, r in enumerate(self.queue):
                if r.scan_id == sid:
                    self.queue.pop(i)
                    r.cancelled_s = self.now
                    self.cancelled.append(r)
                    break
            else:
                for r in self.active:
                    if r.scan_id == sid:
                        r.stream.synchronize()
                        r.plan.close()
                        r.plan = None
                        r.cancelled_s = self.now
                        self.used -= r.footprint
                        self.active.remove(r)
                        self.cancelled.append(r)
                        break

    def _admit(self):
        # FCFS: the head of the queue goes first; a later scan never overtakes it
        while self.queue and self.queue[0].arrival_s <= self.now and self.used + self.queue[0].footprint <= self.budget:
            r = self.queue.pop(0)
            r.admitted_s = self.now
            # admission work (plan: maps, Psi, step; A^H y) runs on the GPU before the scan's
            # first tick, so its time is charged to the clock like a tick's
            t0 = time.perf_counter()
            r.stream = self.torch.cuda.Stream()
            with self.torch.cuda.stream(r.stream):
                r.plan = self.t2sh.Plan(r.dims, r.phi, r.mask, r.maps, stream=r.stream)
                r.plan.solve_begin(r.kspace, r.kform)
            r.stream.synchronize()
            dt = time.perf_counter() - t0
            self.now += dt
            self.busy_s += dt
            self.admit_s += dt
            self.used += r.footprint
            self.active.append(r)
        self.max_active = max(self.max_active, len(self.active))

    def _tick(self):
        torch = self.torch
        t0 = time.perf_counter()
        finished = []
        for r in self.active:
            with torch.cuda.stream(r.stream):
                if r.plan.solve_iterate(self.iters_per_tick) >= r.dims.iters:
                    finished.append(r)
        for r in self.active:
            r.stream.synchronize()
        dt = time.perf_counter() - t0
        self.now += dt
        self.busy_s += dt
        self.ticks += 1
        for r in finished:
            t1 = time.perf_counter()
            with torch.cuda.stream(r.stream):
                r.result = r.plan.solve_end()
            r.stream.synchronize()
            r.plan.close()
            r.plan = None
            dt = time.perf_counter() - t1  # the result copy and the plan's release
            self.now += dt
            self.busy_s += dt
            r.done_s = self.now
            self.used -= r.footprint
            self.active.remove(r)
            self.done.append(r)

    def run(self):
        while self.queue or self.active:
            self._apply_cancellations()
            if not (self.queue or self.active):
                break
            self._admit()
            if not self.active:
                self.now = max(self.now, self.queue[0].arrival_s)  # idle: jump to the next arrival
                continue
            self._tick()
        return self.report()

    def report(self) -> dict:
        lat = np.array([r.done_s - r.arrival_s for r in self.done])
        wait = np.array([r.admitted_s - r.arrival_s for r in self.done])
        slices = sum(r.dims.nslices for r in self.done)
        span = max(r.done_s for r in self.done) - min(r.arrival_s for r in self.done) if self.done else 0.0
        return {"scans": len(self.done), "cancelled": len(self.cancelled), "slices": int(slices),
                "latency_p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "latency_p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "latency_max_s": float(lat.max()) if len(lat) else None,
                "wait_p50_s": float(np.percentile(wait, 50)) if len(wait) else None,
                "busy_s": self.busy_s, "admission_s": self.admit_s, "span_s": span,
                "slices_per_busy_s": slices / self.busy_s if self.busy_s else None,
                "utilisation": self.busy_s / span if span else None,
                "ticks": self.ticks, "max_concurrent_scans": self.max_active}


def main(argv=None):
    """200 scans from 4 scanners, each scan one of the three batch shapes (320 x 256x160 C=12,
    288 x 240x128 C=8, 256 x 192x192 C=16; T=80, K=4, 100 iterations), at the real
    arrival rate (one scan per scanner every `gap` s on average) and time-compressed to an
    offered load of `load` x the measured capacity.  Prints one JSON line per run."""
    import argparse
    import json

    import torch

    import t2sh_synth as synth

    from . import build as B
    from .workload import make_scan

    ap = argparse.ArgumentParser()
    ap.add_argument("--scans", type=int, default=200)
    ap.add_argument("--scanners", type=int, default=4)
    ap.add_argument("--gap", type=float, default=300.0, help="mean seconds between scans of one scanner")
    ap.add_argument("--load", type=float, default=0.7, help="offered load of the time-compressed run")
    ap.add_argument("--iters-per-tick", type=int, default=10)
    ap.add_argument("--budget-gb", type=float, default=80.0)
    ap.add_argument("--seed", type=int, default=1814)
    a = ap.parse_args(argv)
    B.build()
    from . import t2sh
    dev = torch.device("cuda", 0)
    shapes = synth.BATCH_SCANS
    tmpl = [make_scan(sh, sh.nslices, dev) for sh in shapes]

    def request(i, scanner, t, k):
        sh = shapes[k]
        phi, mask, maps, ytil = tmpl[k]
        dims = t2sh.make_dims(sh.ny, sh.nz, sh.ncoils, sh.nechoes, sh.nbasis, nslices=sh.nslices, block=sh.block,
                              lam=sh.lam, iters=sh.iters, seed=sh.seed + i)
        return ScanRequest(i, scanner, t, k, dims, phi, mask, maps, ytil, t2sh.KSPACE_PROJ)

    # measured capacity: one solo reconstruction per shape (plan, solve, release)
    service = []
    for k in range(3):
        r = request(-1, 0, 0.0, k)
        for rep_ in range(2):  # the first one warms up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with t2sh.Plan(r.dims, r.phi, r.mask, r.maps) as p:
                p.solve(r.kspace, r.kform)
                torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        service.append(dt)
    mean_service = float(np.mean(service))
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([a.seed, 11])))
    kinds = rng.integers(0, 3, a.scans)
    runs = {"real_rate": a.gap, "time_compressed": a.scanners * mean_service / a.load}
    for name, gap in runs.items():
        srv = Server(t2sh, int(a.budget_gb * 1e9), a.iters_per_tick)
        for i, (t, s) in enumerate(poisson_arrivals(a.scans, a.scanners, gap, a.seed)):
            srv.submit(request(i, s, t, int(kinds[i])))
        rep = srv.run()
        rep.update({"run": name, "scanners": a.scanners, "mean_gap_per_scanner_s": gap,
                    "solo_service_s": dict(zip(["320x256x160 C12", "288x240x128 C8", "256x192x192 C16"], service)),
                    "offered_load": mean_service * a.scanners / gap, "iters_per_scan": shapes[0].iters})
        print(json.dumps(rep), flush=True)


if __name__ == "__main__":
    main()
