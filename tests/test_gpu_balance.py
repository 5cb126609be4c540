"""Balanced launches (asep_set_balance): persistent CTAs take (sample group,
chunk of sweeps) items, so groups move between SMs between chunks.  Results
must be those of the one-launch kernel bit for bit -- lattices, every record
of the height sums, hop counters, profiles and overlaps -- and of the oracle;
the bounded wait for a previous chunk reports ASEP_ERR_TIMEOUT when it runs
out (fault injection), and the context recovers."""
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


def outputs(kw, times, chunks, balance):
    with A.asep_create(A.make_params(**kw), sample_times=times) as ctx:
        A.asep_set_balance(ctx, balance)
        for n in chunks:
            A.asep_sweep(ctx, n)
        words, sweep = A.asep_state(ctx)
        sh, sh2, _ = A.asep_width(ctx)
        out = dict(words=words, sh=sh, sh2=sh2, cnt=A.asep_counters(ctx), cur=A.asep_currents(ctx))
        if kw.get("flags", 0) & A.ASEP_FLAG_PROFILE:
            out["prof"] = A.asep_profile(ctx)
        if kw.get("flags", 0) & A.ASEP_FLAG_AUTOCORR:
            out["ac"] = A.asep_autocorr(ctx)
        assert sweep == sum(chunks)
    return out


CASES = {
    # the benchmarked shape, more groups than resident slots' worth of work, ragged last chunk
    "ring_cfg1_shape": (dict(L=1 << 17, domain_sites=256, samples_per_real=40, p_thr=th(0.75), q_thr=th(0.25),
                             seed=3, flags=A.ASEP_FLAG_NO_HOP_COUNTS), [0, 4, 9, 23, 30], [30], 7),
    # several samples per CTA (16 columns each), hop counts, profile and autocorrelation
    "ring_packed_observables": (dict(L=4096, domain_sites=128, samples_per_real=300, p_thr=th(0.7), q_thr=th(0.2),
                                     seed=4, flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=5),
                                [0, 5, 6, 17, 25], [12, 13], 4),
    "bimodal_pq": (dict(L=1 << 14, domain_sites=128, n_realizations=6, samples_per_real=5, p_thr=th(0.5),
                        q_thr=th(0.5), dis_kind=A.ASEP_DIS_BIMODAL_PQ, dis_a_thr=th(0.5), dis_b_thr=th(0.1),
                        dis_c_thr=th(0.1), dis_seed=5, seed=6), [0, 11, 20], [20], 3),
    "two_lane_crossing": (dict(model=A.ASEP_MODEL_TWO_LANE, L=1 << 14, domain_sites=64, samples_per_real=50,
                               init_kind=1, init_seed=7, p_thr=th(0.5), q_thr=th(0.5), dis_kind=A.ASEP_DIS_CROSSING,
                               dis_a_thr=th(0.5), dis_b_thr=th(0.8), dis_c_thr=th(0.2), dis_seed=8, seed=9,
                               flags=A.ASEP_FLAG_PROFILE), [0, 8, 16], [16], 5),
    "two_lane_turning": (dict(model=A.ASEP_MODEL_TWO_LANE, L=1 << 15, domain_sites=128, samples_per_real=24,
                              init_kind=1, init_seed=10, q_thr=A.ASEP_ALWAYS, dis_kind=A.ASEP_DIS_TURNING,
                              dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=11, seed=12), [0, 10], [10], 2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_balanced_equals_one_launch_and_oracle(name):
    kw, times, chunks, balance = CASES[name]
    ref = outputs(kw, times, chunks, 0)
    got = outputs(kw, times, chunks, balance)
    for key in ref:
        assert np.array_equal(ref[key], got[key]), key
    P = oracle.Params(model=kw.get("model", 0), L=kw["L"], D=kw["domain_sites"],
                      n_realizations=kw.get("n_realizations", 1), samples_per_real=kw["samples_per_real"],
                      p_thr=kw.get("p_thr", A.ASEP_ALWAYS), q_thr=kw.get("q_thr", 0), dis_kind=kw.get("dis_kind", 0),
                      dis_a_thr=kw.get("dis_a_thr", 0), dis_b_thr=kw.get("dis_b_thr", 0),
                      dis_c_thr=kw.get("dis_c_thr", 0), init_kind=kw.get("init_kind", 0), seed=kw["seed"],
                      dis_seed=kw.get("dis_seed", 0), init_seed=kw.get("init_seed", 0))
    picks = [0, P.S // 2, P.S - 1]
    o = oracle.run(P, sum(chunks), times, samples=picks)
    for s in picks:
        assert np.array_equal(got["words"][s], o.state[s]), s
        for ti in range(len(times)):
            for pl in range(P.planes):
                assert int(got["sh"][ti, s, pl]) == o.sum_h[ti, s, pl], (s, ti, pl)


def test_balanced_wait_runs_out_and_the_context_recovers():
    """Group 0 never announces its first chunk: the wait for it runs out
    after its bound, the launch reports ASEP_ERR_TIMEOUT, the GPU still
    answers, and after a reset the balanced run is bit-exact again."""
    import torch

    kw = dict(L=1 << 14, domain_sites=128, samples_per_real=8, p_thr=th(0.75), q_thr=th(0.25), seed=13)
    ref = outputs(kw, [0, 12], [12], 0)
    with A.asep_create(A.make_params(**kw), sample_times=[0, 12]) as ctx:
        A.asep_set_balance(ctx, 4)
        A.asep_inject_fault(ctx, A.ASEP_FAULT_BALANCE_STALL)
        A.asep_sweep(ctx, 12)
        with pytest.raises(A.AsepError) as ei:
            A.asep_sync(ctx)
        assert ei.value.code == A.ASEP_ERR_TIMEOUT
        assert torch.ones(4, device="cuda").sum().item() == 4.0  # the device answers
        A.asep_inject_fault(ctx, A.ASEP_FAULT_NONE)
        A.asep_reset(ctx, seed=13)
        A.asep_sweep(ctx, 12)
        words, _ = A.asep_state(ctx)
        assert np.array_equal(words, ref["words"])
