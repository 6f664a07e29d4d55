"""Continuous-batching request loop over liblbm contexts (argument marshalling + scheduling).

Requests (independent solves of different grid sizes, PML widths and boundary conditions)
arrive over time. The loop admits queued requests whenever their estimated device footprint
(lbm_estimate_bytes) fits in the HBM budget, keeps their populations resident, and advances
every resident instance together through an lbm_batch (one combined CUDA-graph launch per
step). Admission and retirement happen between chunks of steps, so requests that arrive while
others are on the GPU join the running batch as memory frees up. An instance that flags an
unphysical state is retired with status "unstable" without affecting the others.
"""
from __future__ import annotations

import ctypes as C
import time
from dataclasses import dataclass, field

import numpy as np

from . import _lib as L
from .solver import _BC, _PREC, Solver, _check


def estimate_bytes(case, precision="fp32dev", q=37):
    """Device bytes lbm_create would allocate for a workloads.Case (lbm_estimate_bytes_bc: no
    allocation; counts the link gradient's wider accumulator)."""
    from .solver import estimate_bytes as est
    return int(est(case.nx, case.ny, case.W, q=q, bc=case.bc, precision=precision,
                   pml_grad=getattr(case, "pml_grad", "central")))


class Batch:
    """A resident set of contexts advanced together (lbm_batch_*)."""

    def __init__(self, stream=None):
        import torch
        st = stream if stream is not None else torch.cuda.current_stream()
        out = C.c_void_p()
        _check(L.lib().lbm_batch_create(C.c_void_p(st.cuda_stream), C.byref(out)))
        self.h = out

    def set(self, solvers):
        arr = (C.c_void_p * max(1, len(solvers)))(*[s.ctx.value for s in solvers])
        _check(L.lib().lbm_batch_set(self.h, arr, len(solvers)))

    def tile(self, tx=0, by=0):
        """Interior block shape of the batched launch (0, 0: tuned or default)."""
        _check(L.lib().lbm_batch_tile(self.h, int(tx), int(by)))

    def autotune(self, steps=5):
        """Time the candidate interior block shapes on this batch (advances every member by
        8 (steps + 1) steps) and keep the fastest; returns (tx, by)."""
        tx, by = C.c_int(), C.c_int()
        _check(L.lib().lbm_batch_autotune(self.h, int(steps), C.byref(tx), C.byref(by)))
        return tx.value, by.value

    def step(self, n):
        """Returns True, or False if a member flagged an unphysical state (nobody stepped)."""
        st = L.lib().lbm_batch_step(self.h, int(n))
        if st == L.LBM_EUNSTABLE:
            return False
        _check(st)
        return True

    def close(self):
        if getattr(self, "h", None):
            L.lib().lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    case: object            # workloads.Case
    steps: int
    status: str = "queued"  # queued | running | done | unstable
    admitted: float = None
    finished: float = None
    remaining: int = 0
    result: tuple = None
    nbytes: int = 0
    solver: object = field(default=None, repr=False)

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class Scheduler:
    """HBM-budget admission: FIFO order with backfill (a request that does not fit lets later,
    smaller ones in, within a bounded look-ahead so large requests are not starved forever)."""

    def __init__(self, budget_bytes, lookahead=16):
        self.budget = int(budget_bytes)
        self.used = 0
        self.lookahead = lookahead

    def pick(self, queue):
        chosen = []
        for r in queue[:self.lookahead]:
            if r.nbytes > self.budget:
                continue                       # can never fit: left for the caller to reject
            if self.used + r.nbytes <= self.budget:
                self.used += r.nbytes
                chosen.append(r)
        return chosen

    def release(self, r):
        self.used -= r.nbytes


class Engine:
    """Continuous batching. Between chunks of steps the loop retires finished and unstable
    instances and admits queued requests by HBM budget; the initial fields of the requests
    admitted next are generated on the host and uploaded (on a side stream) while the GPU runs
    the current chunk, so admission does not leave the GPU idle."""

    def __init__(self, budget_bytes, precision="fp32dev", chunk=100, keep_fields=True,
                 autotune=False, keep_ids=None, lookahead=16):
        import torch
        self.precision = precision
        self.chunk = chunk
        self.keep_fields = keep_fields
        self.keep_ids = keep_ids          # request ids whose fields are kept (None: all)
        self.autotune = autotune
        self.tuned = None
        self.sched = Scheduler(budget_bytes, lookahead)
        # the batch steps on its own stream and new instances are initialized on another, so
        # that admission overlaps the running chunk
        self.stream = torch.cuda.Stream()
        self.batch = Batch(self.stream)
        self.side = torch.cuda.Stream()
        self.steps_done = 0
        self.sites_steps = 0
        self.step_seconds = 0.0   # wall time of the batched stepping (launch to sync)

    def _start(self, r, now):
        c = r.case
        s = Solver(c.nx, c.ny, c.W, c.tau, c.sigma_max, c.sigma_power, c.bc, 37, c.nrbc_edges,
                   c.beta, c.mean, precision=self.precision, stream=self.side,
                   pml_grad=getattr(c, "pml_grad", "central"))
        s.init(*c.fields())
        r.solver, r.status, r.admitted, r.remaining = s, "running", now, r.steps

    def _finish(self, r, now, status="done"):
        if status == "done":
            try:
                r.solver.sync()
                if self.keep_fields and (self.keep_ids is None or r.rid in self.keep_ids):
                    r.result = r.solver.moments(region="bulk")
            except L.LBMError:
                status = "unstable"
        r.solver.close()
        r.solver = None
        r.status, r.finished = status, now
        self.sched.release(r)

    def _retire_unstable(self, running, now):
        for r in list(running):
            try:
                r.solver.sync()
            except L.LBMError:
                running.remove(r)
                self._finish(r, now, status="unstable")

    def run(self, requests, clock=time.perf_counter):
        """Serve requests (with arrival times) to completion; returns the requests."""
        main = self.stream
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in pending:
            r.nbytes = estimate_bytes(r.case, self.precision)
        queue, running = [], []
        t0 = clock()
        inflight = None          # (n, launch time) of the chunk the GPU is running
        while pending or queue or running or inflight:
            now = clock() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.pop(0))
            for r in [r for r in queue if r.nbytes > self.sched.budget]:
                queue.remove(r)
                r.status, r.finished = "rejected", now
            # admission: host fields + upload on the side stream, overlapping the chunk
            admitted = self.sched.pick(queue)
            for r in admitted:
                queue.remove(r)
                self._start(r, now)
            if inflight is not None:
                n, t_launch = inflight
                main.synchronize()
                self.step_seconds += clock() - t_launch
                inflight = None
                if not self._ok:
                    self._retire_unstable(running, clock() - t0)
                else:
                    for r in running:
                        r.remaining -= n
                        self.sites_steps += r.solver.Lx * r.solver.Ly * n
                    for r in [r for r in running if r.remaining == 0]:
                        running.remove(r)
                        self._finish(r, clock() - t0)
            self.side.synchronize()
            running += admitted
            if not running:
                if pending and not queue:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival - (clock() - t0))))
                continue
            self.batch.set([r.solver for r in running])
            if self.autotune and self.tuned is None:
                k = min(r.remaining for r in running)
                if k > 8 * 3:
                    t_launch = clock()
                    try:
                        self.tuned = self.batch.autotune(steps=2)
                        for r in running:
                            r.remaining -= 8 * 3
                            self.sites_steps += r.solver.Lx * r.solver.Ly * 8 * 3
                    except L.LBMError:
                        self.tuned = ("failed",)
                        self._retire_unstable(running, clock() - t0)
                    main.synchronize()
                    self.step_seconds += clock() - t_launch
                    continue
            n = min(self.chunk, min(r.remaining for r in running))
            inflight = (n, clock())
            self._ok = self.batch.step(n)
        self.batch.set([])
        self.wall = clock() - t0
        return requests

    def close(self):
        self.batch.close()


def summarize(requests, wall, sites_steps, step_seconds=None):
    lat = np.array([r.latency for r in requests if r.status == "done"])
    out = {"requests": len(requests), "done": int(np.sum([r.status == "done" for r in requests])),
           "unstable": int(np.sum([r.status == "unstable" for r in requests])),
           "rejected": int(np.sum([r.status == "rejected" for r in requests])),
           "wall_s": wall, "aggregate_mlups": sites_steps / wall / 1e6 if wall > 0 else 0.0}
    if step_seconds:
        out["stepping_s"] = step_seconds
        out["stepping_mlups"] = sites_steps / step_seconds / 1e6
    if lat.size:
        out["latency_p50_s"] = float(np.percentile(lat, 50))
        out["latency_p99_s"] = float(np.percentile(lat, 99))
    return out


def main():
    """Serve a seeded Poisson request stream and print one JSON summary line."""
    import argparse
    import json
    import os
    import sys
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as wl
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--nmax", type=int, default=1024)
    ap.add_argument("--smin", type=int, default=100)
    ap.add_argument("--smax", type=int, default=300)
    ap.add_argument("--budget-gb", type=float, default=40.0)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--precision", default="fp32dev")
    a = ap.parse_args()
    torch.cuda.init()
    stream = wl.request_stream(a.requests, a.rate, seed=0, nmax=a.nmax, smin=a.smin, smax=a.smax)
    reqs = [Request(k, t, c, c.steps) for k, (t, c) in enumerate(stream)]
    eng = Engine(a.budget_gb * 1e9, a.precision, a.chunk, keep_fields=False)
    eng.run(reqs)
    out = summarize(reqs, eng.wall, eng.sites_steps, eng.step_seconds)
    out.update({"rate_per_s": a.rate, "steps": [a.smin, a.smax], "nmax": a.nmax,
                "precision": a.precision, "budget_gb": a.budget_gb})
    print(json.dumps(out))
    eng.close()


if __name__ == "__main__":
    main()
