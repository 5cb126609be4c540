"""Launch plans and the autotuner: every plan gives bit-identical results,
impossible plans are rejected without changing the context, and the tuner
applies the fastest valid plan."""
import numpy as np
import pytest

import oracle
from paper_1012_0385_gb300 import asep as A
from paper_1012_0385_gb300 import autotune

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


def run(ctx, n):
    A.asep_reset(ctx, seed=77)
    A.asep_sweep(ctx, n)
    words, _ = A.asep_state(ctx)
    sh, sh2, _ = A.asep_width(ctx)
    return words, sh, sh2, A.asep_counters(ctx)


@pytest.mark.parametrize("kw", [
    dict(L=1 << 17, domain_sites=256, samples_per_real=6, p_thr=th(0.75), q_thr=th(0.25)),
    dict(L=1 << 15, domain_sites=128, n_realizations=2, samples_per_real=3, dis_kind=A.ASEP_DIS_BIMODAL,
         dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=4),
    dict(model=A.ASEP_MODEL_TWO_LANE, L=1 << 16, domain_sites=128, samples_per_real=3, init_kind=1, init_seed=2,
         dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=3),
])
def test_every_plan_gives_the_same_result(kw):
    with A.asep_create(A.make_params(**kw), sample_times=[0, 3, 9]) as ctx:
        cands = autotune.candidates(ctx)
        assert any(c > 1 for c, _ in cands) and (0, 0) in cands
        ref = run(ctx, 9)
        tried = 0
        for cluster, spc in cands:
            try:
                A.asep_set_plan(ctx, cluster, spc)
            except A.AsepError:
                continue
            tried += 1
            got = run(ctx, 9)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b), (cluster, spc)
        assert tried >= 3


def test_impossible_plans_are_rejected_and_the_plan_kept():
    with A.asep_create(A.make_params(L=4096, domain_sites=256, samples_per_real=2), sample_times=[]) as ctx:
        before = A.asep_get_info(ctx)
        # 8 columns cannot fill 16 CTAs; 3 and 32 are not cluster sizes; samples per CTA needs the
        # one-CTA plan; a CTA cannot hold more samples than exist
        for cluster, spc in [(16, 0), (3, 0), (32, 0), (2, 4), (1, 3)]:
            with pytest.raises(A.AsepError):
                A.asep_set_plan(ctx, cluster, spc)
            after = A.asep_get_info(ctx)
            assert (after["cluster"], after["samples_per_group"], after["groups"]) == \
                   (before["cluster"], before["samples_per_group"], before["groups"])


def test_autotune_applies_the_fastest_valid_plan(tmp_path):
    kw = dict(L=1 << 16, domain_sites=256, samples_per_real=40, p_thr=th(0.75), q_thr=th(0.25))
    with A.asep_create(A.make_params(**kw), sample_times=[]) as ctx:
        choice, table = autotune.autotune(ctx, probe_sweeps=16)
        assert len(table) >= 3
        assert choice.ms_per_sweep == min(r["ms_per_sweep"] for r in table if r["knob"] == "plan")
        info = A.asep_get_info(ctx)
        assert info["cluster"] == choice.cluster
        cache = autotune.PlanCache(str(tmp_path / "plans.json"))
        cache.put(ctx.params, choice)
        assert autotune.PlanCache(str(tmp_path / "plans.json")).get(ctx.params)["cluster"] == choice.cluster


@pytest.mark.parametrize("schedule", [A.ASEP_SCHED_DOMAIN, A.ASEP_SCHED_SCA, A.ASEP_SCHED_SERIAL])
def test_sweeps_per_launch_never_change_results(schedule):
    """The launch-sweeps knob splits a run into more launches; lattices,
    every record and the counters stay bit-identical."""
    kw = dict(L=1 << 14, schedule=schedule, samples_per_real=5, p_thr=th(0.75), q_thr=th(0.25))
    if schedule == A.ASEP_SCHED_DOMAIN:
        kw["domain_sites"] = 128
    with A.asep_create(A.make_params(**kw), sample_times=[0, 2, 7, 19, 20]) as ctx:
        ref = run(ctx, 20)
        for cap in (1, 3, 7, 0):
            A.asep_set_launch_sweeps(ctx, cap)
            launches0 = A.asep_get_info(ctx)["kernel_launches"]
            got = run(ctx, 20)
            for a, b in zip(ref, got):
                assert np.array_equal(a, b), cap
            if cap:
                assert A.asep_get_info(ctx)["kernel_launches"] - launches0 >= 20 // cap


def test_autotune_times_the_launch_sweeps_and_batch_mode():
    kw = dict(L=1 << 15, domain_sites=256, samples_per_real=20, p_thr=th(0.75), q_thr=th(0.25))
    with A.asep_create(A.make_params(**kw), sample_times=[]) as ctx:
        choice, table = autotune.autotune(ctx, probe_sweeps=16)
        caps = [r["launch_sweeps"] for r in table if r["knob"] == "launch_sweeps"]
        probe = table[0]["probe_sweeps"]
        assert caps == ["auto", probe // 2, probe // 4, probe // 8]
        assert choice.launch_sweeps in (0, probe // 2, probe // 4, probe // 8)
    shapes = [dict(L=2048, domain_sites=128, samples_per_real=3, p_thr=th(0.6), seed=5 + i) for i in range(6)]

    def make():
        return [A.asep_create(A.make_params(**k), sample_times=[]) for k in shapes]

    mode, rows = autotune.tune_batch_mode(make, [4] * len(shapes), steps=5)
    assert mode in ("eager", "graph") and [r["mode"] for r in rows] == ["eager", "graph"]
    assert all(r["ms_per_step"] > 0 for r in rows)
