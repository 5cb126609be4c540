"""Serving: continuous batching of ensemble jobs on one GPU.

A job is one ensemble request (model, L, rates, disorder seed, samples,
n_mcs, sample times).  :func:`serve` replays an arrival trace against the
GPU in one of two modes:

``batched``  (continuous batching) -- the server keeps every admitted job's
    packed lattices and Philox clock on the device.  Each step it admits the
    jobs that have arrived, as far as the device-memory budget allows, and
    advances every active job by a quantum of sweeps in ONE persistent launch
    (``asep_batch_sweep``: the CTAs of all jobs share one work queue, so jobs
    of very different size overlap on the device); jobs that have finished
    are read back and their memory is released before the next step.
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
from dataclasses import dataclass, field

import numpy as np

from . import asep as A
from .sampling import log_times

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

    def footprint(self) -> int:
        """Device bytes the job's context holds (lattices, disorder, tables)."""
        S = self.S
        W = self.L // 32
        nt = len(self.times())
        return S * self.planes * W * 4 + S * W * 4 + nt * S * self.planes * 24 + S * 32 + 4096


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


def _group_work(ctx) -> tuple[int, int]:
    """(attempts per sweep of one work item, SMs one item occupies): a
    resident group is samples_per_group samples on one CTA, a cluster-tier
    item one sample on `cluster` CTAs."""
    info = A.asep_get_info(ctx)
    return info["attempts_per_sweep"] * info["samples_per_group"], info["cluster"]


def serve_batched(trace: list[Job], quantum_s: float = 0.02, mem_budget: int = 16 << 30, max_active: int = 256,
                  rate_guess: float = 4e11, sms: int = 152) -> dict:
    """Continuous batching: admit at step boundaries by footprint, one
    persistent launch per step over all active jobs, retire finished jobs.
    Each job's quantum of sweeps is chosen so that one of its work items (a
    CTA's sample group, or a cluster's sample) takes about `quantum_s` at the
    per-SM rate, so the items of a step have similar lengths."""
    pending = sorted(trace, key=lambda j: j.arrival)
    active: list[tuple[Job, object, int]] = []  # (job, ctx, sweeps left)
    shape: dict[int, tuple[int, int]] = {}
    used = 0
    t0 = time.perf_counter()
    batch = A.asep_batch_create(max_jobs=max_active, max_items=1 << 20)
    rate = rate_guess
    try:
        while pending or active:
            now = time.perf_counter() - t0
            # admit every arrived job the memory budget allows (first come first served)
            while pending and pending[0].arrival <= now and len(active) < max_active:
                fp = pending[0].footprint()
                if used + fp > mem_budget and active:
                    break
                job = pending.pop(0)
                job.admitted = now
                ctx = A.asep_create(job.params(), sample_times=job.times())
                shape[job.id] = _group_work(ctx)
                active.append((job, ctx, job.n_mcs))
                used += fp
            if not active:
                time.sleep(max(0.0, pending[0].arrival - now))
                continue
            # one quantum: every work item runs about quantum_s at the per-SM rate
            per_sm = rate / sms
            q = [max(1, min(left, int(per_sm * shape[job.id][1] * quantum_s // shape[job.id][0])))
                 for job, _, left in active]
            t_step = time.perf_counter()
            A.asep_batch_sweep(batch, [c for _, c, _ in active], q)
            A.asep_sync(active[0][1])
            dt = time.perf_counter() - t_step
            done = sum(k * job.L * job.planes * job.S for k, (job, _, _) in zip(q, active))
            if dt > 0:
                rate = 0.5 * rate + 0.5 * done / dt
            still = []
            for k, (job, ctx, left) in zip(q, active):
                if left - k == 0:
                    _finish(job, ctx, t0)
                    ctx.close()
                    used -= job.footprint()
                else:
                    still.append((job, ctx, left - k))
            active = still
    finally:
        for _, ctx, _ in active:
            ctx.close()
        batch.close()
    return _summary(sorted(trace, key=lambda j: j.arrival), time.perf_counter() - t0, "batched")
