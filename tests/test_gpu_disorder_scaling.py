"""Quenched-disorder scaling of the paper's sec. 2.3, on the GPU under the
paper's own SCA schedule (p = 0.8, its default), checked against the values
it prints (tests/golden/paper_values.json).

Q-SSEP: forward and backward hops both present, each site slow for right hops
with probability Q = 0.5 and, independently, slow for left hops with the same
probability (the paper's separate tag bits), slow rate r p with r = 0.2.  The
paper finds activated growth W ~ (ln t)^beta~ with beta~ = 2.85(30) and a
saturated width scaling with alpha = 1.  Q-TASEP (q = 0, Q = 0.5; the paper
does not print its r, 0.2 here): saturated width with alpha = 1.
Statistical tests: 128-256 disorder realizations, a few seconds each on a
GB300."""
import json
import os

import numpy as np
import pytest

from paper_1012_0385_gb300 import asep as A
from paper_1012_0385_gb300.sampling import log_times

pytestmark = pytest.mark.gpu

th = A.asep_threshold

with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
    GOLDEN = json.load(f)


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_0385_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def qssep_width2(L: int, n_mcs: int, realizations: int, dis_kind: int = A.ASEP_DIS_BIMODAL_PQ):
    """Mean W^2 over the realizations at the log-spaced sample times."""
    times = log_times(n_mcs)
    prm = A.make_params(L=L, schedule=A.ASEP_SCHED_SCA, n_realizations=realizations, samples_per_real=1,
                        p_thr=th(0.8), q_thr=th(0.8), dis_kind=dis_kind, dis_a_thr=th(0.5), dis_b_thr=th(0.16),
                        dis_c_thr=th(0.16), dis_seed=3, seed=5, flags=A.ASEP_FLAG_NO_HOP_COUNTS)
    with A.asep_create(prm, sample_times=times) as ctx:
        A.asep_sweep(ctx, n_mcs)
        w2 = A.asep_width(ctx)[2][:, :, 0]
    return np.array(times, dtype=np.float64), w2.mean(axis=1)


def test_qssep_activated_growth_exponent():
    """L = 4096 before saturation: a fit of ln W against ln ln t gives the
    paper's beta~ within twice its error, and the power-law exponent
    d ln W / d ln t keeps falling (logarithmic, not power-law, growth)."""
    g = GOLDEN["qssep_activated"]
    t, w2 = qssep_width2(4096, 800_000, 128)
    sel = t >= 1400
    lw, llt = 0.5 * np.log(w2[sel]), np.log(np.log(t[sel]))
    beta_tilde = np.polyfit(llt, lw, 1)[0]
    assert abs(beta_tilde - g["beta_tilde"]) < 2 * g["beta_tilde_err"], beta_tilde
    lt = np.log(t[sel])
    half = len(lt) // 2
    early = np.polyfit(lt[:half], lw[:half], 1)[0]
    late = np.polyfit(lt[half:], lw[half:], 1)[0]
    assert early - late > 0.06, (early, late)


def test_qssep_saturated_width_scales_with_alpha_one():
    """Saturated W^2 at L = 256 and 512: the ratio 2^(2 alpha) gives alpha
    within 0.2 of the paper's alpha = 1 -- where the one-class reading (q_i
    slow exactly where p_i is) saturates with alpha = 1/2."""
    g = GOLDEN["qssep_activated"]
    _, a = qssep_width2(256, 1_000_000, 256)
    _, b = qssep_width2(512, 4_000_000, 256)
    alpha = 0.5 * np.log2(b[-6:].mean() / a[-6:].mean())
    assert abs(alpha - g["alpha"]) < 0.2, alpha
    _, a1 = qssep_width2(256, 400_000, 256, dis_kind=A.ASEP_DIS_BIMODAL)
    _, b1 = qssep_width2(512, 400_000, 256, dis_kind=A.ASEP_DIS_BIMODAL)
    alpha1 = 0.5 * np.log2(b1[-6:].mean() / a1[-6:].mean())
    assert abs(alpha1 - 0.5) < 0.15, alpha1


def test_qtasep_saturated_width_scales_with_alpha_one():
    """Q-TASEP (columnar-disorder KPZ) at L = 256 and 512, saturated: alpha
    within 0.15 of the paper's alpha = 1 (clean KPZ has 1/2)."""
    g = GOLDEN["qtasep_exponents"]
    w = []
    for L in (256, 512):
        times = log_times(400_000)
        prm = A.make_params(L=L, schedule=A.ASEP_SCHED_SCA, n_realizations=256, samples_per_real=1, p_thr=th(0.8),
                            q_thr=0, dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.5), dis_b_thr=th(0.16),
                            dis_seed=3, seed=5, flags=A.ASEP_FLAG_NO_HOP_COUNTS)
        with A.asep_create(prm, sample_times=times) as ctx:
            A.asep_sweep(ctx, 400_000)
            w.append(A.asep_width(ctx)[2][-10:, :, 0].mean())
    alpha = 0.5 * np.log2(w[1] / w[0])
    assert abs(alpha - g["alpha"]) < 0.15, alpha
