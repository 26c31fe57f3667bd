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
                     autotune=False, run_streams=8, max_active_agents=1 << 24):
    """Serve `trace` (list of (arrival_seconds, RunShape)) with continuous batching.

    The batch advances in chunks of at most `chunk_gens` generations, cut so that runs finish
    at chunk ends.  Two chunks are kept queued on the batch's stream: while the GPU works on
    them the host admits arrivals (each new run is created on one of `run_streams` streams;
    ga_batch_add orders the batch after its founder initialisation without blocking the host)
    and retires runs whose last chunk has completed, which it learns from a CUDA event.

    Admission is first come first served and stops at the first request that does not fit:
    in the HBM budget, and in `max_active_agents` agents in flight (about what fills the GPU;
    a request larger than that is admitted when nothing else runs).  Small requests thus
    share the GPU while a large one is not slowed by everything admitted beside it."""
    import collections
    import torch
    stream = torch.cuda.Stream()
    streams = [torch.cuda.Stream() for _ in range(max(1, run_streams))]
    batch = ga.Batch(stream=stream)
    reqs = [Request(i, t, s) for i, (t, s) in enumerate(trace)]
    pending = collections.deque(reqs)   # in arrival order
    active = {}                         # rid -> [request, run, remaining generations]
    inflight = collections.deque()      # (event, [(request, run)] finishing with that chunk)
    used = 0
    peak = 0
    agents = 0  # agents of the admitted, unfinished runs
    created = 0
    tuned = not autotune
    t0 = time.perf_counter()

    def retire_oldest():
        nonlocal used, agents
        ev, finishing = inflight.popleft()
        ev.synchronize()
        now = _now(t0)
        for req, run in finishing:
            req.finished = now
            if keep_results:
                req.result = run.snapshot()
            used -= ga.workspace_bytes(req.shape)
            agents -= req.shape.n_agents
            run.close()

    while pending or active or inflight:
        now = _now(t0)
        # admission: arrived requests, first come first served, while they fit
        while pending and pending[0].arrival <= now:
            need = ga.workspace_bytes(pending[0].shape)
            if need > hbm_budget_bytes:
                raise ValueError(f"request {pending[0].rid} alone exceeds the HBM budget")
            if used + need > hbm_budget_bytes:
                break
            if agents > 0 and agents + pending[0].shape.n_agents > max_active_agents:
                break
            req = pending.popleft()
            run = ga.Run(req.shape, stream=streams[created % len(streams)])
            created += 1
            batch.add(run)
            req.admitted = _now(t0)
            active[req.rid] = [req, run, req.shape.generations]
            used += need
            agents += req.shape.n_agents
            peak = max(peak, used)
        if active:
            if not tuned:
                batch.autotune(trial_gens=4)
                tuned = True
            step = min(chunk_gens, min(a[2] for a in active.values()))
            batch.step(step)
            ev = torch.cuda.Event()
            ev.record(stream)
            finishing = []
            for rid in list(active):
                a = active[rid]
                a[2] -= step
                if a[2] == 0:
                    finishing.append((a[0], a[1]))
                    batch.remove(a[1])
                    del active[rid]
            inflight.append((ev, finishing))
        # keep at most two chunks queued (with nothing left to launch, wait for the oldest),
        # and retire every run whose last chunk has completed
        while inflight and (len(inflight) > 2 or not active):
            retire_oldest()
        while inflight and inflight[0][0].query():
            retire_oldest()
        if not active and not inflight and pending:
            time.sleep(max(0.0, min(pending[0].arrival - _now(t0), 0.01)))
    makespan = _now(t0)
    batch.sync()
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
