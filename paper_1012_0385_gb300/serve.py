"""Serving: continuous batching of ensemble jobs on one GPU.

A job is one ensemble request (model, L, rates, disorder seed, samples,
n_mcs, sample times).  :func:`serve_batched` and :func:`serve_plain` replay
an arrival trace against the GPU:

``batched``  (continuous batching) -- the server keeps every admitted job's
    packed lattices and Philox clock on the device.  Jobs are admitted as
    they arrive while the device-memory budget and the shared-memory budget
    allow; both footprints come from the library's own launch plan
    (``asep_plan``, before anything is allocated).  Every step advances all
    active jobs by a quantum of sweeps in ONE persistent launch
    (``asep_batch_sweep``: the CTAs of all jobs share one work queue, so jobs
    of very different size overlap on the device); jobs whose lattices stream
    from HBM run their own launches beside it on their own streams.  The host
    never waits for a step: it keeps up to two steps in flight, admits arrivals
    and reads back finished jobs (each job has its own stream, so reading one
    waits for nothing else) while the GPU runs.
``plain``    -- one launch per job, first come first served: each job is
    created, swept to n_mcs in one ``asep_sweep`` call, read back and
    destroyed before the next one starts.

Every sample's randomness depends only on its own counters, so a job's
result is bit-identical in both modes and whatever else runs beside it.
Latency = time from a job's arrival to its W(t) table on the host.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import asep as A
from .sampling import log_times

SMEM_PER_SM = 228 * 1024  # bytes of shared memory per SM (GB300)
STREAMED = 32  # asep_info.cluster of a context whose lattice streams from HBM
KINDS = ("tasep", "asep", "bimodal", "two_lane")


@dataclass
class Job:
    """One ensemble request.  ``kind`` follows the four workload families of
    the paper: plain TASEP growth (p = 1), ASEP growth (p = 0.75, q = 0.25),
    quenched bimodal disorder (Eq. bimodal; Q = 0.1, slow rate 0.3) and the
    two-lane model with turning sites (density 0.05, omega = 0.1)."""

    id: int
    kind: str
    L: int
    samples: int
    n_mcs: int
    seed: int
    arrival: float = 0.0
    D: int = 256
    # filled by serve()
    admitted: float = math.nan
    finished: float = math.nan
    result: dict = field(default_factory=dict)
    _plan: dict | None = field(default=None, repr=False)

    @property
    def planes(self) -> int:
        return 2 if self.kind == "two_lane" else 1

    @property
    def realizations(self) -> int:
        return max(1, self.samples // 4) if self.kind == "bimodal" else 1

    @property
    def S(self) -> int:
        """Samples the context holds (bimodal jobs: whole realizations of 4)."""
        r = self.realizations
        return r * max(1, self.samples // r)

    @property
    def attempts(self) -> int:
        return self.L * self.planes * self.S * self.n_mcs

    def params(self):
        th = A.asep_threshold
        kw = dict(L=self.L, domain_sites=self.D, seed=self.seed, samples_per_real=self.samples)
        if self.kind == "tasep":
            kw.update(p_thr=A.ASEP_ALWAYS, q_thr=0)
        elif self.kind == "asep":
            kw.update(p_thr=th(0.75), q_thr=th(0.25))
        elif self.kind == "bimodal":
            r = self.realizations
            kw.update(n_realizations=r, samples_per_real=max(1, self.samples // r), p_thr=A.ASEP_ALWAYS, q_thr=0,
                      dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=self.seed + 1)
        elif self.kind == "two_lane":
            kw.update(model=A.ASEP_MODEL_TWO_LANE, p_thr=A.ASEP_ALWAYS, q_thr=A.ASEP_ALWAYS,
                      init_kind=A.ASEP_INIT_BERNOULLI_HALF, init_seed=self.seed + 2, dis_kind=A.ASEP_DIS_TURNING,
                      dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=self.seed + 1)
        else:
            raise ValueError(self.kind)
        return A.make_params(**kw)

    def times(self):
        return log_times(self.n_mcs) + ([self.n_mcs] if log_times(self.n_mcs)[-1] != self.n_mcs else [])

    def plan(self) -> dict:
        """The library's plan of the job's context (asep_plan): launch shape,
        device bytes, shared memory per CTA; nothing is allocated."""
        if self._plan is None:
            self._plan = A.asep_plan(self.params(), sample_times=self.times())
        return self._plan

    def device_bytes(self) -> int:
        return int(self.plan()["device_bytes"])

    def smem_demand(self) -> int:
        """Shared memory the job's work items occupy when all are resident:
        CTAs (a cluster-tier sample holds `cluster` CTAs) x bytes per CTA."""
        pl = self.plan()
        per_item = pl["cluster"] if 1 < pl["cluster"] < STREAMED else 1
        return int(pl["groups"]) * per_item * int(pl["smem_bytes"])


def make_trace(n_jobs: int, seed: int = 0, rate_hz: float = 50.0, L_range=(1 << 10, 1 << 19),
               samples_range=(1, 256), n_mcs_range=(10, 10_000), kinds=KINDS, D: int = 256,
               load: float | None = None, capacity: float | None = None) -> list[Job]:
    """Seeded Poisson arrivals; L, samples and n_mcs log-uniform in their
    ranges (L rounded to a multiple of 2D), the kind uniform over `kinds`.
    With `load` and `capacity` (attempts/s), the arrival rate is set so the
    trace offers load x capacity: rate = load * capacity / mean job attempts."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for i in range(n_jobs):
        t += rng.exponential(1.0 / rate_hz)
        L = int(round(math.exp(rng.uniform(math.log(L_range[0]), math.log(L_range[1])))))
        L = max(2 * D, (L // (2 * D)) * 2 * D)
        S = int(round(math.exp(rng.uniform(math.log(samples_range[0]), math.log(samples_range[1])))))
        n = int(round(math.exp(rng.uniform(math.log(n_mcs_range[0]), math.log(n_mcs_range[1])))))
        kind = kinds[int(rng.integers(len(kinds)))]
        jobs.append(Job(id=i, kind=kind, L=L, samples=max(1, S), n_mcs=max(1, n), seed=1000 + 7 * i, arrival=t, D=D))
    if load is not None and capacity is not None:
        mean_attempts = sum(j.attempts for j in jobs) / len(jobs)
        scale = rate_hz * mean_attempts / (load * capacity)  # new gaps = old gaps x scale
        for j in jobs:
            j.arrival *= scale
    return jobs


def _finish(job: Job, ctx, t0: float):
    sh, sh2, w2 = A.asep_width(ctx)
    job.result = {"w2": w2, "sum_h": sh, "sum_h2": sh2, "counters": A.asep_counters(ctx)}
    job.finished = time.perf_counter() - t0


def _summary(jobs: list[Job], makespan: float, mode: str) -> dict:
    lat = np.array([j.finished - j.arrival for j in jobs])
    att = sum(j.attempts for j in jobs)
    return {"mode": mode, "jobs": len(jobs), "attempts": att, "makespan_s": makespan,
            "throughput_attempts_per_s": att / makespan, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean())}


def serve_plain(trace: list[Job]) -> dict:
    """One launch per job, first come first served."""
    jobs = sorted(trace, key=lambda j: j.arrival)
    t0 = time.perf_counter()
    for job in jobs:
        now = time.perf_counter() - t0
        if now < job.arrival:
            time.sleep(job.arrival - now)
        job.admitted = time.perf_counter() - t0
        with A.asep_create(job.params(), sample_times=job.times()) as ctx:
            A.asep_sweep(ctx, job.n_mcs)
            _finish(job, ctx, t0)
    return _summary(jobs, time.perf_counter() - t0, "plain")


@dataclass
class _Active:
    job: Job
    ctx: object
    stream: object
    left: int
    streamed: bool
    mem: int
    smem: int
    item_attempts: int  # attempts per sweep of one work item (a CTA's samples, or a cluster's sample)
    item_sms: int       # SMs one work item occupies


@dataclass
class _Step:
    events: list
    finishing: list
    attempts: int


def serve_batched(trace: list[Job], quantum_s: float = 0.02, mem_budget: int | None = None, waves: float = 8.0,
                  max_active: int = 10_000, rate_guess: float = 4e11, depth: int = 2,
                  age_s: float | None = 0.5, max_weight: float = 32.0) -> dict:
    """Continuous batching (see the module docstring).

    Admission, first come first served: a job enters when its device bytes
    fit `mem_budget` (default 60 % of the free device memory) and its
    shared-memory demand fits `waves` times the device's shared memory
    beside the active jobs (a job larger than half of that counts as half, so
    that it still enters when the load dips); at most `max_active` jobs.
    Quantum: each job advances by the sweeps one of its work items runs in
    about `quantum_s` at the measured per-SM rate (less for a job whose
    demand exceeds half the allowance), so a step lasts about `waves` quanta
    at most.  With `age_s`, a job's quantum is weighted by 1 + (time since
    its arrival) / age_s (at most `max_weight`): jobs that have waited or run
    long get a larger share of each step, so the largest jobs, which make the
    latency tail, are not stretched by the stream of small ones."""
    import torch

    dev = torch.cuda.current_device()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if mem_budget is None:
        mem_budget = int(0.6 * torch.cuda.mem_get_info(dev)[0])
    allowance = int(waves * sms * SMEM_PER_SM)
    main = torch.cuda.current_stream(dev)
    pending = deque(sorted(trace, key=lambda j: j.arrival))
    active: list[_Active] = []
    in_flight: deque[_Step] = deque()
    free_streams: list = []
    used_mem = used_smem = 0
    peak_active = 0
    rate = rate_guess
    last_retire = None
    t0 = time.perf_counter()
    batch = A.asep_batch_create(max_jobs=min(max_active, 16384), max_items=1 << 20, stream=main.cuda_stream)
    try:
        while pending or active or in_flight:
            now = time.perf_counter() - t0
            progressed = False
            # admit arrived jobs while both budgets allow
            while pending and pending[0].arrival <= now and len(active) < max_active:
                job = pending[0]
                mem, dem = job.device_bytes(), int(min(job.smem_demand(), allowance // 2))
                if (active or in_flight) and (used_mem + mem > mem_budget or used_smem + dem > allowance):
                    break
                pending.popleft()
                st = free_streams.pop() if free_streams else torch.cuda.Stream(dev)
                job.admitted = now
                ctx = A.asep_create(job.params(), sample_times=job.times(), stream=st.cuda_stream)
                info = A.asep_get_info(ctx)
                per_item = info["cluster"] if 1 < info["cluster"] < STREAMED else 1
                active.append(_Active(job, ctx, st, job.n_mcs, info["cluster"] == STREAMED, mem, dem,
                                      info["attempts_per_sweep"] * info["samples_per_group"], per_item))
                used_mem += mem
                used_smem += dem
                progressed = True
            peak_active = max(peak_active, len(active) + sum(len(s.finishing) for s in in_flight))
            # enqueue a step for every active job
            if active and len(in_flight) < depth:
                per_sm = rate / sms
                ctxs, qs, events, finishing, still, attempts = [], [], [], [], [], 0
                t_now = time.perf_counter() - t0
                for a in active:
                    target = quantum_s * min(1.0, (allowance / 2) / max(1, a.job.smem_demand()))
                    if age_s:
                        target *= min(max_weight, 1.0 + (t_now - a.job.arrival) / age_s)
                    q = max(1, min(a.left, int(per_sm * a.item_sms * target // max(1, a.item_attempts))))
                    attempts += q * a.job.L * a.job.planes * a.job.S
                    if a.streamed:  # its own launches, on its own stream, beside the batch
                        A.asep_sweep(a.ctx, q)
                        ev = torch.cuda.Event()
                        ev.record(a.stream)
                        events.append(ev)
                    else:
                        ctxs.append(a.ctx)
                        qs.append(q)
                    a.left -= q
                    (finishing if a.left == 0 else still).append(a)
                if ctxs:
                    A.asep_batch_sweep(batch, ctxs, qs)
                ev = torch.cuda.Event()
                ev.record(main)
                events.append(ev)
                in_flight.append(_Step(events, finishing, attempts))
                active = still
                progressed = True
            # retire the oldest step once the GPU has finished it
            if in_flight and all(ev.query() for ev in in_flight[0].events):
                step = in_flight.popleft()
                t_now = time.perf_counter()
                if last_retire is not None and t_now > last_retire:
                    rate = 0.5 * rate + 0.5 * step.attempts / (t_now - last_retire)
                last_retire = t_now
                for a in step.finishing:
                    _finish(a.job, a.ctx, t0)
                    a.ctx.close()
                    used_mem -= a.mem
                    used_smem -= a.smem
                    free_streams.append(a.stream)
                if not in_flight:
                    last_retire = None  # the GPU idles until the next step: restart the rate clock
                progressed = True
            if not progressed:
                wait = pending[0].arrival - (time.perf_counter() - t0) if pending and not active and not in_flight \
                    else 2e-4
                time.sleep(min(max(wait, 0.0), 0.05))
    finally:
        for s in in_flight:
            for a in s.finishing:
                a.ctx.close()
        for a in active:
            a.ctx.close()
        batch.close()
    out = _summary(sorted(trace, key=lambda j: j.arrival), time.perf_counter() - t0, "batched")
    out["peak_active_jobs"] = peak_active
    return out
