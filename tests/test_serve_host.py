"""Host logic of the serving layer (no GPU): traces are seeded and shaped as
asked, jobs map onto valid parameters of the four workload families."""
import math

import numpy as np
import pytest

from paper_1012_0385_gb300 import serve


def test_trace_is_seeded_and_in_range():
    a = serve.make_trace(200, seed=7, rate_hz=100.0, L_range=(1 << 10, 1 << 19), samples_range=(1, 256),
                         n_mcs_range=(10, 10_000))
    b = serve.make_trace(200, seed=7, rate_hz=100.0, L_range=(1 << 10, 1 << 19), samples_range=(1, 256),
                         n_mcs_range=(10, 10_000))
    assert [(j.kind, j.L, j.samples, j.n_mcs, j.arrival) for j in a] == \
           [(j.kind, j.L, j.samples, j.n_mcs, j.arrival) for j in b]
    arr = np.array([j.arrival for j in a])
    assert np.all(np.diff(arr) > 0)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert 0.5 / 100 < gaps.mean() < 2.0 / 100  # Poisson arrivals at 100 Hz
    for j in a:
        assert j.L % 512 == 0 and 512 <= j.L <= 1 << 19
        assert 1 <= j.samples <= 256 and 10 <= j.n_mcs <= 10_000
        assert j.kind in serve.KINDS
    assert {j.kind for j in a} == set(serve.KINDS)
    # log-uniform L: about as many jobs below the geometric middle as above
    mid = math.sqrt((1 << 10) * (1 << 19))
    below = sum(j.L < mid for j in a)
    assert 60 < below < 140


@pytest.mark.parametrize("kind", serve.KINDS)
def test_job_parameters_are_consistent(kind):
    A = pytest.importorskip("paper_1012_0385_gb300.asep")
    j = serve.Job(id=0, kind=kind, L=4096, samples=10, n_mcs=100, seed=5)
    p = j.params()
    assert p.L == 4096 and p.domain_sites == 256
    assert p.n_realizations * p.samples_per_real == j.S
    assert j.attempts == 4096 * j.planes * j.S * 100
    t = j.times()
    assert t[0] == 0 and t[-1] == 100 and all(x < y for x, y in zip(t, t[1:]))
    # admission footprints come from the library's plan (no device needed for one-CTA plans)
    pl = j.plan()
    assert pl["S"] == j.S and pl["planes"] == j.planes and pl["cluster"] == 1
    assert j.device_bytes() > j.S * j.planes * 4096 // 8
    assert j.smem_demand() == pl["groups"] * pl["smem_bytes"] > 0
    if kind == "two_lane":
        assert p.model == A.ASEP_MODEL_TWO_LANE and p.dis_kind == A.ASEP_DIS_TURNING
    if kind == "bimodal":
        assert p.dis_kind == A.ASEP_DIS_BIMODAL and p.n_realizations == 2
