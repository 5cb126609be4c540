"""Spot checks deep into long runs (the replay oracle's protocol for runs too
long to replay whole): the GPU state is pulled at sweep s of a long run, the
oracle replays sweeps s .. s + k from that state with the same schedule and
random stream, and the GPU's state at s + k -- and every record of the height
sums in between -- must equal the replay bit for bit.  (state, sweep index,
parameters) is a complete description of a run, because nothing of the
generator is stored.  Runs: configuration 2's shape (bimodal disorder,
L = 2^16) and configuration 3's (two lanes with turning sites, D = 128) to
10^5 sweeps, and configuration 1 in full (L = 2^17, 256 samples, 2^14 sweeps)
as a balanced launch, checked over its last 16 sweeps."""
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
    oracle.build()
    torch.cuda.set_device(0)


def oracle_params(kw):
    return oracle.Params(model=kw.get("model", 0), L=kw["L"], D=kw["domain_sites"],
                         n_realizations=kw.get("n_realizations", 1), samples_per_real=kw["samples_per_real"],
                         p_thr=kw.get("p_thr", A.ASEP_ALWAYS), q_thr=kw.get("q_thr", 0), dis_kind=kw.get("dis_kind", 0),
                         dis_a_thr=kw.get("dis_a_thr", 0), dis_b_thr=kw.get("dis_b_thr", 0),
                         dis_c_thr=kw.get("dis_c_thr", 0), init_kind=kw.get("init_kind", 0), seed=kw["seed"],
                         dis_seed=kw.get("dis_seed", 0), init_seed=kw.get("init_seed", 0))


def deep_spot_check(kw, s, k, picks, balance=0):
    records = [s + 1, s + k // 2, s + k]
    with A.asep_create(A.make_params(**kw), sample_times=records) as ctx:
        A.asep_set_balance(ctx, balance)
        A.asep_sweep(ctx, s)
        at_s, sweep = A.asep_state(ctx)
        assert sweep == s
        A.asep_sweep(ctx, k)
        at_sk, _ = A.asep_state(ctx)
        sh, sh2, _ = A.asep_width(ctx)
        A.asep_sync(ctx)
    P = oracle_params(kw)
    mask = oracle.disorder(P)
    st = at_s.copy()
    done = s
    for ti, t in enumerate(records):
        oracle.replay(P, st, done, t - done, mask=mask, samples=picks)
        done = t
        for n in picks:
            for pl in range(P.planes):
                a, b = oracle.heights(st[n, pl], P.L)
                assert int(sh[ti, n, pl]) == a, (n, t, pl)
                assert ((int(sh2[ti, n, pl, 1]) << 64) | int(sh2[ti, n, pl, 0])) == b, (n, t, pl)
    for n in picks:
        assert np.array_equal(at_sk[n], st[n]), n
        # particle number per lane (ring) or in total (two lanes) is conserved
        assert np.unpackbits(at_sk[n].view(np.uint8)).sum() == np.unpackbits(at_s[n].view(np.uint8)).sum()


def test_bimodal_run_checked_at_sweep_100000():
    kw = dict(L=1 << 16, domain_sites=256, n_realizations=4, samples_per_real=2, p_thr=A.ASEP_ALWAYS, q_thr=0,
              dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=2, seed=11)
    deep_spot_check(kw, 100_000, 20, picks=[0, 3, 7])


def test_two_lane_run_checked_at_sweep_100000():
    kw = dict(model=A.ASEP_MODEL_TWO_LANE, L=1 << 16, domain_sites=128, samples_per_real=4, p_thr=A.ASEP_ALWAYS,
              q_thr=A.ASEP_ALWAYS, dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=3,
              init_kind=A.ASEP_INIT_BERNOULLI_HALF, init_seed=4, seed=12)
    deep_spot_check(kw, 100_000, 20, picks=[0, 3])


def test_growth_workload_balanced_checked_over_its_last_sweeps():
    kw = dict(L=1 << 17, domain_sites=256, samples_per_real=256, p_thr=th(0.75), q_thr=th(0.25), seed=13)
    deep_spot_check(kw, (1 << 14) - 16, 16, picks=[0, 101, 255], balance=16)
