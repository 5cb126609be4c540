"""The allocation-free batch sweep (asep_batch_sweep_static).

It is for callers that may not allocate device memory when they run work;
its work queue lives in a static device array of the library.  The tests run
the same contexts through it and through the batch object's sweep
(asep_batch_sweep, which owns allocated workspace) and require bit-identical
lattices, height tables, counters and sweep indices after each of two calls
in a row -- once with one launch step per call and once with several (a cap
on the sweeps per launch), so the step loop that reuses the static
descriptors and items runs too.  They check that, after the start-up call and
one call, a further call leaves the device's free memory and PyTorch's
allocated bytes unchanged, and that requests beyond the array's limits are
rejected.  The file is collected last so that a run stopping at the first
failure has run every other test first.
"""
import numpy as np
import pytest

import oracle
from paper_1012_0385_gb300 import asep as A

pytestmark = pytest.mark.gpu

th = oracle.threshold

MIX = [
    (dict(L=1 << 15, domain_sites=256, samples_per_real=5, p_thr=th(0.75), q_thr=th(0.25), seed=3), [0, 7, 20, 33]),
    (dict(L=4096, domain_sites=128, samples_per_real=40, p_thr=th(0.6), seed=5), [0, 30]),
    (dict(L=1 << 16, domain_sites=256, n_realizations=2, samples_per_real=2, dis_kind=A.ASEP_DIS_BIMODAL,
          dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=21, seed=4), [0, 12, 40]),
    (dict(model=A.ASEP_MODEL_TWO_LANE, L=8192, domain_sites=64, samples_per_real=3, init_kind=1, init_seed=8,
          dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=9, q_thr=A.ASEP_ALWAYS,
          seed=10), [5, 25]),
    (dict(L=128, domain_sites=32, samples_per_real=300, p_thr=th(0.7), q_thr=th(0.2), seed=2), [0, 50]),
]
CALLS = [[13, 9, 20, 11, 30], [20, 21, 20, 14, 20]]


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_0385_gb300 import build

    build.build()
    torch.cuda.set_device(0)
    A.asep_batch_sweep_static([], [])  # the start-up call: set-up of this device only


def snapshot(ctx):
    words, sweep = A.asep_state(ctx)
    sh, sh2, _ = A.asep_width(ctx)
    return dict(words=words, sweep=sweep, sh=sh, sh2=sh2, cnt=A.asep_counters(ctx))


def compare_on_two_calls(launch_sweeps):
    ref = [A.asep_create(A.make_params(**kw), sample_times=t) for kw, t in MIX]
    got = [A.asep_create(A.make_params(**kw), sample_times=t) for kw, t in MIX]
    for c in ref + got:
        A.asep_set_launch_sweeps(c, launch_sweeps)
    with A.asep_batch_create(max_jobs=16, max_items=4096) as b:
        for k, n_mcs in enumerate(CALLS):
            A.asep_batch_sweep(b, ref, n_mcs)
            A.asep_batch_sweep_static(got, n_mcs)
            for i, (r, g) in enumerate(zip(ref, got)):
                a, c = snapshot(r), snapshot(g)
                for key in ("words", "sh", "sh2", "cnt"):
                    assert np.array_equal(a[key], c[key]), (k, i, key)
                assert a["sweep"] == c["sweep"] == sum(call[i] for call in CALLS[: k + 1])
    for c in ref + got:
        c.close()


def test_static_batch_matches_batch_sweep_on_two_calls():
    compare_on_two_calls(0)  # automatic bound: one launch step per call


def test_static_batch_matches_batch_sweep_with_several_steps_per_call():
    compare_on_two_calls(7)  # at most 7 sweeps per step: 2 to 5 steps per call


def test_static_batch_allocates_nothing():
    import torch

    ctxs = [A.asep_create(A.make_params(**kw), sample_times=t) for kw, t in MIX]
    A.asep_batch_sweep_static(ctxs, CALLS[0])
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    A.asep_batch_sweep_static(ctxs, CALLS[1])
    torch.cuda.synchronize()
    free1, alloc1 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert (free1, alloc1) == (free0, alloc0), (free0 - free1, alloc1 - alloc0)
    assert A.asep_get_info(ctxs[0])["sweep"] == sum(call[0] for call in CALLS)
    for c in ctxs:
        c.close()


def test_static_batch_rejects_requests_beyond_its_limits():
    ctxs = [A.asep_create(A.make_params(L=64, domain_sites=32), sample_times=[]) for _ in range(65)]
    with pytest.raises(A.AsepError) as ei:
        A.asep_batch_sweep_static(ctxs, [1] * 65)  # more than 64 contexts
    assert ei.value.code == A.ASEP_ERR_INVALID and "64" in str(ei.value)
    for c in ctxs:
        c.close()
    big = A.asep_create(A.make_params(L=64, domain_sites=32, samples_per_real=128 * 16385), sample_times=[])
    with pytest.raises(A.AsepError) as ei:
        A.asep_batch_sweep_static([big], [1])  # more sample groups than the static item list holds
    assert ei.value.code == A.ASEP_ERR_INVALID and "16384" in str(ei.value)
    big.close()
