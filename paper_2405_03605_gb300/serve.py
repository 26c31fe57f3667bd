"""Continuous-batching service for GA runs.

Requests (a run shape plus a generation count) arrive over time.  The server admits a request
as soon as its device workspace fits in the HBM budget, adds it to the running batch (one
shared set of launches per generation for every active run), advances the batch in chunks of
generations, and retires each run when it has done its generations; populations stay on the
device for the whole life of a run.  Scheduling is host logic; every generation of every run
is computed by the library's kernels (ga_batch_step).  A run's result does not depend on what
else was in the batch (draws are keyed by seed, run_id, generation, island and slot).

`serve_one_at_a_time` is the comparison: the same requests, first come first served, each run
alone on the GPU (ga_step), one after the other.
"""
import time
from dataclasses import dataclass, field

from . import ga


@dataclass
class Request:
    rid: int
    arrival: float            # seconds after the trace starts
    shape: object             # workloads.RunShape; shape.generations = generations to run
    admitted: float = None
    finished: float = None
    result: object = None     # host snapshot (optional) or None

    @property
    def work(self):
        return self.shape.n_agents * self.shape.generations


@dataclass
class ServeReport:
    requests: list
    makespan: float
    agent_gens: float
    launches: int = 0
    peak_bytes: int = 0
    notes: dict = field(default_factory=dict)

    @property
    def throughput(self):
        return self.agent_gens / self.makespan if self.makespan > 0 else 0.0

    def latencies(self):
        return sorted(r.finished - r.arrival for r in self.requests)

    def percentile(self, q):
        lat = self.latencies()
        if not lat:
            return 0.0
        k = min(len(lat) - 1, max(0, int(round(q / 100.0 * (len(lat) - 1)))))
        return lat[k]


def _now(t0):
    return time.perf_counter() - t0


def serve_continuous(trace, hbm_budget_bytes, chunk_gens=64, keep_results=False,
                     autotune=False):
    """Serve `trace` (list of (arrival_seconds, RunShape)) with continuous batching."""
    import torch
    stream = torch.cuda.Stream()
    batch = ga.Batch(stream=stream)
    reqs = [Request(i, t, s) for i, (t, s) in enumerate(trace)]
    pending = list(reqs)          # in arrival order
    active = {}                   # rid -> (request, run, remaining generations)
    used = 0
    peak = 0
    t0 = time.perf_counter()
    while pending or active:
        now = _now(t0)
        # admission: arrived requests, first come first served, while they fit
        while pending and pending[0].arrival <= now:
            need = ga.workspace_bytes(pending[0].shape)
            if need > hbm_budget_bytes:
                raise ValueError(f"request {pending[0].rid} alone exceeds the HBM budget")
            if used + need > hbm_budget_bytes:
                break
            req = pending.pop(0)
            run = ga.Run(req.shape, stream=stream)
            batch.add(run)
            req.admitted = _now(t0)
            active[req.rid] = [req, run, req.shape.generations]
            used += need
            peak = max(peak, used)
        if not active:
            if pending:
                time.sleep(max(0.0, min(pending[0].arrival - _now(t0), 0.01)))
            continue
        if autotune:
            batch.autotune(trial_gens=4)
            autotune = False
        step = min(chunk_gens, min(a[2] for a in active.values()))
        batch.step(step)
        batch.sync()
        done = []
        for rid, a in active.items():
            a[2] -= step
            if a[2] == 0:
                done.append(rid)
        for rid in done:
            req, run, _ = active.pop(rid)
            batch.remove(run)
            req.finished = _now(t0)
            if keep_results:
                req.result = run.snapshot()
            used -= ga.workspace_bytes(req.shape)
            run.close()
    makespan = _now(t0)
    launches = batch.launches
    batch.close()
    return ServeReport(reqs, makespan, float(sum(r.work for r in reqs)), launches, peak)


def serve_one_at_a_time(trace, keep_results=False):
    """The same trace, first come first served, one run alone on the GPU at a time."""
    import torch
    reqs = [Request(i, t, s) for i, (t, s) in enumerate(trace)]
    t0 = time.perf_counter()
    launches = 0
    for req in reqs:
        wait = req.arrival - _now(t0)
        if wait > 0:
            time.sleep(wait)
        req.admitted = _now(t0)
        run = ga.Run(req.shape)
        run.step(req.shape.generations)
        run.sync()
        req.finished = _now(t0)
        if keep_results:
            req.result = run.snapshot()
        launches += run.launches
        run.close()
    torch.cuda.synchronize()
    makespan = _now(t0)
    return ServeReport(reqs, makespan, float(sum(r.work for r in reqs)), launches)
