"""Serving with continuous batching: each job's result is bit-identical to
running it alone (one launch per job), whatever else runs beside it, and the
server reports latency percentiles."""
import numpy as np
import pytest

from paper_1012_0385_gb300 import serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_0385_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def test_batched_serving_equals_one_launch_per_job():
    trace = serve.make_trace(24, seed=3, rate_hz=400.0, L_range=(1 << 10, 1 << 16), samples_range=(1, 32),
                             n_mcs_range=(5, 400))
    plain = [serve.Job(**{k: getattr(j, k) for k in ("id", "kind", "L", "samples", "n_mcs", "seed", "arrival")})
             for j in trace]
    s_batched = serve.serve_batched(trace, quantum_s=0.002)
    s_plain = serve.serve_plain(plain)
    assert s_batched["jobs"] == s_plain["jobs"] == 24
    assert s_batched["attempts"] == s_plain["attempts"]
    for a, b in zip(sorted(trace, key=lambda j: j.id), sorted(plain, key=lambda j: j.id)):
        for key in ("sum_h", "sum_h2", "counters"):
            assert np.array_equal(a.result[key], b.result[key]), (a.id, a.kind, key)
        assert a.finished >= a.arrival and b.finished >= b.arrival
    for s in (s_batched, s_plain):
        assert 0 < s["p50_latency_s"] <= s["p99_latency_s"]
        assert s["throughput_attempts_per_s"] > 0


def test_jobs_join_while_others_run():
    """A late job is admitted while an early long job is on the GPU."""
    early = serve.Job(id=0, kind="asep", L=1 << 16, samples=64, n_mcs=2000, seed=11, arrival=0.0)
    late = serve.Job(id=1, kind="tasep", L=4096, samples=8, n_mcs=50, seed=12, arrival=0.05)
    serve.serve_batched([early, late], quantum_s=0.005)
    assert late.admitted < early.finished  # admitted before the early job finished
    assert late.finished < early.finished
