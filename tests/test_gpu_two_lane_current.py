"""The paper's two-lane result (sec. 3), on the GPU under its SCA sequence:
in the steady state the total current density c = J/L (J = hops along lane
A minus hops along lane B) has zero mean and a fluctuation <c^2> that grows
linearly in time (tests/golden/paper_values.json, "two_lane").  Here the
paper's unmarked crossing case: in-lane rate 0.5, lane changes at every site
with probability 0.8, random half filling."""
import json
import os

import numpy as np
import pytest

from paper_1012_0385_gb300 import asep as A
from paper_1012_0385_gb300.sampling import log_times

pytestmark = pytest.mark.gpu

th = A.asep_threshold


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_0385_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def current_fluctuation(L: int, n_mcs: int, samples: int, marked: bool = False):
    times = log_times(n_mcs)
    if marked:  # the paper's model: u_i, v_i = 0.8, or 0.2 at marked sites (half of them, u and v apart)
        dis = dict(dis_kind=A.ASEP_DIS_CROSSING, dis_a_thr=th(0.5), dis_b_thr=th(0.8), dis_c_thr=th(0.2))
        prm = A.make_params(model=A.ASEP_MODEL_TWO_LANE, L=L, schedule=A.ASEP_SCHED_SCA, n_realizations=samples,
                            samples_per_real=1, init_kind=A.ASEP_INIT_BERNOULLI_HALF, init_seed=7, p_thr=th(0.5),
                            q_thr=th(0.5), dis_seed=3, seed=5, **dis)
    else:
        prm = A.make_params(model=A.ASEP_MODEL_TWO_LANE, L=L, schedule=A.ASEP_SCHED_SCA, samples_per_real=samples,
                            init_kind=A.ASEP_INIT_BERNOULLI_HALF, init_seed=7, p_thr=th(0.5), q_thr=th(0.5),
                            dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=A.ASEP_ALWAYS, dis_b_thr=th(0.8), dis_seed=3,
                            seed=5)
    with A.asep_create(prm, sample_times=times) as ctx:
        A.asep_sweep(ctx, n_mcs)
        cur = A.asep_currents(ctx).reshape(len(times), samples, 4).astype(np.float64)
    c = (cur[:, :, 0] - cur[:, :, 1]) / L
    return np.array(times, dtype=np.float64), c


def test_two_lane_current_fluctuation_grows_linearly():
    """<c> stays within 4 standard errors of 0; log <c^2> against log t has
    slope 1 within 0.1 over t = 300 .. 2*10^4; <c^2> L / t is the same for
    L = 256 and 512 within 15 % (the current is a sum of L diffusive parts)."""
    marked = False
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
        assert "linear" in json.load(f)["two_lane"]["c2_growth"]
    level = {}
    for L in (256, 512):
        t, c = current_fluctuation(L, 20_000, 512, marked)
        sel = t >= 300
        m, se = c[sel].mean(axis=1), c[sel].std(axis=1) / np.sqrt(c.shape[1])
        assert np.all(np.abs(m) < 4 * se + 1e-12), L
        c2 = (c[sel] ** 2).mean(axis=1)
        slope = np.polyfit(np.log(t[sel]), np.log(c2), 1)[0]
        assert abs(slope - 1.0) < 0.1, (L, slope)
        level[L] = np.mean(c2 * L / t[sel])
    assert abs(level[512] / level[256] - 1.0) < 0.15, level


def test_two_lane_quenched_crossing_current():
    """The paper's quenched crossing probabilities (u_i, v_i = 0.8, or 0.2 at
    marked sites, u and v marked independently), one realization per sample:
    <c> is 0 within 4 standard errors (left/right symmetric in distribution),
    while <c^2> grows faster than linearly -- each realization's u_i != v_i
    give it a drift, so the realization average mixes diffusive and ballistic
    growth (slope 1.2 at L = 256 over t = 300 .. 2*10^4, rising later)."""
    t, c = current_fluctuation(256, 20_000, 512, True)
    sel = t >= 300
    m, se = c[sel].mean(axis=1), c[sel].std(axis=1) / np.sqrt(c.shape[1])
    assert np.all(np.abs(m) < 4 * se + 1e-12)
    slope = np.polyfit(np.log(t[sel]), np.log((c[sel] ** 2).mean(axis=1)), 1)[0]
    assert 1.05 < slope < 1.6, slope
