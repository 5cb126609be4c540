"""Serving with continuous batching: each job's result is bit-identical to
running it alone (one launch per job), whatever else runs beside it, and to
the oracle for one job of each workload family; a job whose lattice streams
from HBM is served beside the batch; more than 256 jobs are in flight at
once; the admission footprints (asep_plan) equal what the contexts then hold;
the server reports latency percentiles."""
import numpy as np
import pytest

import oracle
from paper_1012_0385_gb300 import asep as A
from paper_1012_0385_gb300 import serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_0385_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def copy_jobs(trace):
    return [serve.Job(**{k: getattr(j, k) for k in ("id", "kind", "L", "samples", "n_mcs", "seed", "arrival", "D")})
            for j in trace]


def assert_same_results(a_jobs, b_jobs):
    for a, b in zip(sorted(a_jobs, key=lambda j: j.id), sorted(b_jobs, key=lambda j: j.id)):
        for key in ("sum_h", "sum_h2", "counters"):
            assert np.array_equal(a.result[key], b.result[key]), (a.id, a.kind, key)
        assert a.finished >= a.arrival and b.finished >= b.arrival


def test_batched_serving_equals_one_launch_per_job():
    trace = serve.make_trace(24, seed=3, rate_hz=400.0, L_range=(1 << 10, 1 << 16), samples_range=(1, 32),
                             n_mcs_range=(5, 400))
    plain = copy_jobs(trace)
    s_batched = serve.serve_batched(trace, quantum_s=0.002)
    s_plain = serve.serve_plain(plain)
    assert s_batched["jobs"] == s_plain["jobs"] == 24
    assert s_batched["attempts"] == s_plain["attempts"]
    assert_same_results(trace, plain)
    for s in (s_batched, s_plain):
        assert 0 < s["p50_latency_s"] <= s["p99_latency_s"]
        assert s["throughput_attempts_per_s"] > 0


def test_served_jobs_match_the_oracle():
    """One served job of each family (plain TASEP, ASEP, bimodal disorder,
    two lanes with turning sites), served together, against the oracle's
    replay of the same job: every record of the height sums and the hop
    counters, bit for bit."""
    jobs = [serve.Job(id=i, kind=k, L=4096, samples=4, n_mcs=40 + 7 * i, seed=300 + 11 * i, arrival=0.001 * i)
            for i, k in enumerate(serve.KINDS)]
    serve.serve_batched(jobs, quantum_s=0.001)
    for job in jobs:
        p = job.params()
        P = oracle.Params(model=p.model, schedule=p.schedule, L=p.L, D=p.domain_sites,
                          n_realizations=p.n_realizations, samples_per_real=p.samples_per_real, p_thr=p.p_thr,
                          q_thr=p.q_thr, dis_kind=p.dis_kind, dis_a_thr=p.dis_a_thr, dis_b_thr=p.dis_b_thr,
                          dis_c_thr=p.dis_c_thr, init_kind=p.init_kind, seed=p.seed, dis_seed=p.dis_seed,
                          init_seed=p.init_seed)
        ref = oracle.run(P, job.n_mcs, job.times())
        assert np.array_equal(job.result["counters"], ref.counters), job.kind
        sh, sh2 = job.result["sum_h"], job.result["sum_h2"]
        for ti in range(len(job.times())):
            for s in range(P.S):
                for pl in range(P.planes):
                    assert int(sh[ti, s, pl]) == ref.sum_h[ti, s, pl], (job.kind, ti, s, pl)
                    assert ((int(sh2[ti, s, pl, 1]) << 64) | int(sh2[ti, s, pl, 0])) == ref.sum_h2[ti, s, pl]


def test_streamed_job_is_served_beside_the_batch():
    """A ring of 2^24 sites (beyond a 16-CTA cluster: its lattice streams
    from HBM) in a mix of resident jobs: the same results as alone."""
    trace = serve.make_trace(10, seed=5, rate_hz=300.0, L_range=(1 << 10, 1 << 14), samples_range=(1, 16),
                             n_mcs_range=(5, 60))
    trace.append(serve.Job(id=99, kind="asep", L=1 << 24, samples=1, n_mcs=6, seed=77, arrival=0.002))
    assert trace[-1].plan()["cluster"] == serve.STREAMED
    plain = copy_jobs(trace)
    serve.serve_batched(trace, quantum_s=0.002)
    serve.serve_plain(plain)
    assert_same_results(trace, plain)


def test_more_than_256_jobs_in_flight():
    """600 small jobs arriving together: all admitted at once (the slot cap
    is beyond 256), advanced in shared steps, results equal to alone for a
    sample of them."""
    trace = serve.make_trace(600, seed=9, rate_hz=1e6, L_range=(1 << 10, 1 << 12), samples_range=(1, 4),
                             n_mcs_range=(20, 200))
    s = serve.serve_batched(trace, quantum_s=0.002)
    assert s["jobs"] == 600 and s["peak_active_jobs"] > 256
    some = [j for j in trace if j.id % 50 == 0]
    alone = copy_jobs(some)
    serve.serve_plain(alone)
    assert_same_results(some, alone)


def test_admission_footprint_equals_the_context():
    """asep_plan's device bytes and launch plan (what the server admits by)
    equal what the created context reports, for every family, the cluster
    tier, the streamed tier and the observable buffers."""
    th = A.asep_threshold
    cases = [j.params() for j in (serve.Job(id=0, kind=k, L=1 << 14, samples=8, n_mcs=100, seed=1)
                                  for k in serve.KINDS)]
    cases += [A.make_params(L=1 << 21, domain_sites=256, samples_per_real=2, p_thr=th(0.75), q_thr=th(0.25)),
              A.make_params(L=1 << 24, domain_sites=256, samples_per_real=1),
              A.make_params(L=1 << 18, schedule=A.ASEP_SCHED_SCA, samples_per_real=3),
              A.make_params(L=4096, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=5),
              A.make_params(model=A.ASEP_MODEL_TWO_LANE, L=1 << 16, domain_sites=128, samples_per_real=4,
                            flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=10, init_kind=1)]
    for prm in cases:
        times = [0, 10, 50]
        pl = A.asep_plan(prm, sample_times=times)
        with A.asep_create(prm, sample_times=times) as ctx:
            info = A.asep_get_info(ctx)
        for k in ("device_bytes", "cluster", "samples_per_group", "groups", "threads", "smem_bytes", "S", "planes"):
            assert pl[k] == info[k], (k, pl[k], info[k], prm.L, prm.schedule)


def test_jobs_join_while_others_run():
    """A late job is admitted while an early long job is on the GPU."""
    early = serve.Job(id=0, kind="asep", L=1 << 16, samples=64, n_mcs=2000, seed=11, arrival=0.0)
    late = serve.Job(id=1, kind="tasep", L=4096, samples=8, n_mcs=50, seed=12, arrival=0.05)
    serve.serve_batched([early, late], quantum_s=0.005)
    assert late.admitted < early.finished  # admitted before the early job finished
    assert late.finished < early.finished
