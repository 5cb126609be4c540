"""Host logic of the launch-plan autotuner without a GPU: the plan cache keys
plans by everything that decides which plans are valid, and round-trips them
through its JSON file."""
import json

from paper_1012_0385_gb300 import asep as A
from paper_1012_0385_gb300 import autotune


def test_plan_cache_keys_and_round_trip(tmp_path):
    path = str(tmp_path / "plans.json")
    cache = autotune.PlanCache(path)
    dom = A.make_params(L=1 << 17, samples_per_real=256)
    sca = A.make_params(L=1 << 17, samples_per_real=256, schedule=A.ASEP_SCHED_SCA)
    small = A.make_params(L=1 << 16, samples_per_real=256)
    keys = {autotune.PlanCache.key(p) for p in (dom, sca, small)}
    assert len(keys) == 3  # schedule and L each give their own entry
    cache.put(dom, autotune.Choice(1, 2, 0.07))
    cache.put(sca, autotune.Choice(32, 0, 0.01))
    assert cache.get(small) is None
    again = autotune.PlanCache(path)
    assert again.get(dom)["cluster"] == 1 and again.get(dom)["samples_per_group"] == 2
    assert again.get(sca)["cluster"] == 32
    with open(path) as f:
        assert len(json.load(f)) == 2


def test_plan_candidates_include_streamed_tile_widths(monkeypatch):
    """Candidate plans from the context's sizes: one-CTA plans while a sample
    fits 1024 columns, cluster splits leaving >= 32 columns per CTA, and the
    streamed tier at tile widths leaving >= 2 tiles per sample."""
    def fake(L, D, S, cluster):
        return lambda ctx: {"L": L, "D": D, "S": S, "cluster": cluster}

    monkeypatch.setattr(A, "asep_get_info", fake(1 << 17, 256, 256, 1))  # 256 columns per sample
    c = autotune.candidates(None, sms=152)
    assert (0, 0) in c and (1, 1) in c and (1, 4) in c and (1, 8) not in c
    assert [x for x in c if x[0] in (2, 4, 8, 16)] == [(2, 0), (4, 0), (8, 0)]
    assert not [x for x in c if x[0] == 32]  # 256 samples fill 152 SMs: no streamed plans
    monkeypatch.setattr(A, "asep_get_info", fake(1 << 17, 256, 128, 1))  # 128 samples on 152 SMs
    assert [x for x in autotune.candidates(None, sms=152) if x[0] == 32] == [(32, 64), (32, 128)]
    monkeypatch.setattr(A, "asep_get_info", fake(1 << 24, 256, 16, 32))  # 32768 columns: streamed only
    c = autotune.candidates(None)
    assert [x for x in c if x[0] == 32] == [(32, w) for w in autotune.STREAM_TILE_COLUMNS]
    assert not [x for x in c if x[0] == 1]
    monkeypatch.setattr(A, "asep_get_info", fake(48 * 64, 32, 4, 1))  # 48 columns: no two tiles of 32
    assert not [x for x in autotune.candidates(None, sms=152) if x[0] == 32]
    monkeypatch.setattr(A, "asep_get_info", fake(65 * 64, 32, 4, 1))  # 130 words per plane: bulk copies need 4k
    assert not [x for x in autotune.candidates(None, sms=152) if x[0] == 32]
