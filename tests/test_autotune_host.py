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
