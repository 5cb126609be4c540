"""Batched execution: many contexts of uneven size in one persistent launch
(and in replayed CUDA graphs) give bit-identical results to each context
alone, whatever the launch shape."""
import numpy as np
import pytest

import oracle
from paper_1012_0385_gb300 import asep as A

pytestmark = pytest.mark.gpu

th = oracle.threshold


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_0385_gb300 import build

    build.build()
    torch.cuda.set_device(0)


MIX = [
    (dict(L=1 << 15, domain_sites=256, samples_per_real=5, p_thr=th(0.75), q_thr=th(0.25), seed=3,
          flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=7), [0, 7, 20, 33]),
    (dict(L=4096, domain_sites=128, samples_per_real=40, p_thr=th(0.6), seed=5), [0, 30]),
    (dict(L=1 << 16, domain_sites=256, n_realizations=2, samples_per_real=2, dis_kind=A.ASEP_DIS_BIMODAL,
          dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=21, seed=4), [0, 12, 40]),
    (dict(model=A.ASEP_MODEL_TWO_LANE, L=8192, domain_sites=64, samples_per_real=3, init_kind=1, init_seed=8,
          dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=9, q_thr=A.ASEP_ALWAYS,
          seed=10, flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=5), [5, 25]),
    (dict(L=1 << 17, domain_sites=256, samples_per_real=3, p_thr=th(0.75), q_thr=th(0.25), seed=1,
          flags=A.ASEP_FLAG_NO_HOP_COUNTS), [0, 16]),
    (dict(L=128, domain_sites=32, samples_per_real=300, p_thr=th(0.7), q_thr=th(0.2), seed=2), [0, 50]),
]
N_MCS = [33, 30, 40, 25, 16, 50]


def snapshot(ctx):
    words, sweep = A.asep_state(ctx)
    sh, sh2, _ = A.asep_width(ctx)
    out = dict(words=words, sweep=sweep, sh=sh, sh2=sh2, cnt=A.asep_counters(ctx), cur=A.asep_currents(ctx))
    try:
        out["prof"], out["ac"] = A.asep_profile(ctx), A.asep_autocorr(ctx)
    except A.AsepError:  # context made without the observable flags
        out["prof"] = out["ac"] = np.zeros(0)
    return out


def same(a, b):
    for k in ("words", "sh", "sh2", "cnt", "cur", "prof", "ac"):
        assert np.array_equal(a[k], b[k]), k
    assert a["sweep"] == b["sweep"]


def alone():
    out = []
    for (kw, times), n in zip(MIX, N_MCS):
        with A.asep_create(A.make_params(**kw), sample_times=times) as ctx:
            A.asep_sweep(ctx, n)
            out.append(snapshot(ctx))
    return out


@pytest.fixture(scope="module")
def reference():
    return alone()


def test_batch_equals_alone(reference):
    ctxs = [A.asep_create(A.make_params(**kw), sample_times=t) for kw, t in MIX]
    with A.asep_batch_create(max_jobs=16, max_items=4096) as b:
        A.asep_batch_sweep(b, ctxs, N_MCS)
        for c, ref in zip(ctxs, reference):
            same(snapshot(c), ref)
    for c in ctxs:
        c.close()


def test_batch_in_uneven_steps_equals_alone(reference):
    """Continuous-batching pattern: contexts join late and leave early."""
    ctxs = [A.asep_create(A.make_params(**kw), sample_times=t) for kw, t in MIX]
    left = list(N_MCS)
    with A.asep_batch_create(max_jobs=16, max_items=4096) as b:
        step = 0
        while any(left):
            active = [i for i in range(len(ctxs)) if left[i] and i <= step]  # context i joins at step i
            q = [min(left[i], 7 + 3 * (i % 3)) for i in active]
            A.asep_batch_sweep(b, [ctxs[i] for i in active], q)
            for i, k in zip(active, q):
                left[i] -= k
            step += 1
        for c, ref in zip(ctxs, reference):
            same(snapshot(c), ref)
    for c in ctxs:
        c.close()


def test_batch_graph_replays_equal_alone(reference):
    ctxs = [A.asep_create(A.make_params(**kw), sample_times=t) for kw, t in MIX]
    # per-context step n // 5: replay the captured step 3 + 2 times, then finish the rest
    step = [n // 5 for n in N_MCS]
    with A.asep_batch_create(max_jobs=16, max_items=4096) as b:
        A.asep_batch_graph(b, ctxs, step, replays=3)
        A.asep_batch_graph(b, ctxs, step, replays=2)  # cached graph
        A.asep_batch_sweep(b, ctxs, [n - 5 * k for n, k in zip(N_MCS, step)])
        for c, ref in zip(ctxs, reference):
            same(snapshot(c), ref)
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("threads,ctas", [(0, 0), (512, 1), (1024, 2), (0, 1)])
def test_launch_shape_does_not_change_results(reference, threads, ctas):
    ctxs = [A.asep_create(A.make_params(**kw), sample_times=t) for kw, t in MIX]
    with A.asep_batch_create(max_jobs=16, max_items=4096) as b:
        A.asep_batch_set_launch(b, threads, ctas)
        A.asep_batch_sweep(b, ctxs, N_MCS)
        for c, ref in zip(ctxs, reference):
            same(snapshot(c), ref)
    for c in ctxs:
        c.close()


def test_batch_with_a_cluster_tier_context_equals_alone():
    big = (dict(L=1 << 19, domain_sites=256, n_realizations=1, samples_per_real=2, dis_kind=A.ASEP_DIS_BIMODAL,
                dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=3, seed=77), [0, 3, 6])
    mix = [big] + MIX[:2]
    n = [6, 9, 7]
    ref = []
    for (kw, t), k in zip(mix, n):
        with A.asep_create(A.make_params(**kw), sample_times=t) as c:
            A.asep_sweep(c, k)
            ref.append(snapshot(c))
    ctxs = [A.asep_create(A.make_params(**kw), sample_times=t) for kw, t in mix]
    with A.asep_batch_create(max_jobs=8, max_items=4096) as b:
        A.asep_batch_sweep(b, ctxs, [2, 4, 3])
        A.asep_batch_graph(b, ctxs, [2, 5, 4], replays=1)
        A.asep_batch_sweep(b, ctxs, [2, 0, 0])
        for c, r in zip(ctxs, ref):
            same(snapshot(c), r)
    with pytest.raises(A.AsepError):
        A.asep_batch_sweep_static(ctxs[:1], [1])  # the static batch takes resident contexts only
    for c in ctxs:
        c.close()


def test_batch_rejects_bad_input():
    with A.asep_create(A.make_params(L=1024, schedule=A.ASEP_SCHED_SERIAL), sample_times=[]) as c, \
            A.asep_batch_create(max_jobs=2, max_items=64) as b:
        with pytest.raises(A.AsepError):
            A.asep_batch_sweep(b, [c], [3])
        with A.asep_create(A.make_params(L=1024, domain_sites=32), sample_times=[]) as d:
            with pytest.raises(A.AsepError):
                A.asep_batch_sweep(b, [d, d], [3, 3])
            with pytest.raises(A.AsepError):
                A.asep_batch_sweep(b, [d, d, d], [1, 1, 1])  # more than max_jobs
