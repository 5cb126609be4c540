"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer work, so the bar is bit-exact: lattice words after the run, every
recorded (sum h, sum h^2), and the hop counters.  Cases span several CTAs and
ragged last CTAs, domain sizes 32..2048, disorder, two lanes, the serial
schedule, launch splitting and checkpoint/resume.  At the full sizes of the
configurations the oracle checks sampled samples, replayed from their own
initial state, and properties that hold at any size check the rest.  The statistical tests compare W(t) of the domain schedule on
the GPU with the independent serial RSU reference within 3 sigma.
"""
import numpy as np
import pytest

import oracle
from paper_1012_0385_gb300 import asep as A
from paper_1012_0385_gb300.sampling import every, log_times

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


ORACLE_KEYS = {"flags": None, "autocorr_t0": None, "plan": None, "model": "model", "schedule": "schedule", "L": "L", "domain_sites": "D",
               "n_realizations": "n_realizations", "samples_per_real": "samples_per_real",
               "first_sample": "first_sample", "p_thr": "p_thr", "q_thr": "q_thr", "dis_kind": "dis_kind",
               "dis_a_thr": "dis_a_thr", "dis_b_thr": "dis_b_thr", "dis_c_thr": "dis_c_thr",
               "init_kind": "init_kind", "seed": "seed", "dis_seed": "dis_seed", "init_seed": "init_seed"}


def oracle_params(kw):
    P = oracle.Params()
    for k, v in kw.items():
        if ORACLE_KEYS[k]:
            setattr(P, ORACLE_KEYS[k], v)
    if kw.get("schedule", 0) == A.ASEP_SCHED_DOMAIN and not kw.get("domain_sites"):
        P.D = 256
    return P


def run_gpu(kw, chunks, times):
    prm = A.make_params(**{k: v for k, v in kw.items() if k != "plan"})
    with A.asep_create(prm, sample_times=times) as ctx:
        if "plan" in kw:
            A.asep_set_plan(ctx, *kw["plan"])
        for c in chunks:
            A.asep_sweep(ctx, c)
        words, sweep = A.asep_state(ctx)
        sh, sh2, w2 = A.asep_width(ctx)
        cnt = A.asep_counters(ctx)
        dis = A.asep_disorder(ctx)
        cur = A.asep_currents(ctx)
        ring_counts = kw.get("model", 0) == 0 and not kw.get("flags", 0) & A.ASEP_FLAG_NO_HOP_COUNTS
        hoff = A.asep_height_offset(ctx) if ring_counts else None
        prof = A.asep_profile(ctx) if kw.get("flags", 0) & A.ASEP_FLAG_PROFILE else None
        ac = A.asep_autocorr(ctx) if kw.get("flags", 0) & A.ASEP_FLAG_AUTOCORR else None
    assert sweep == sum(chunks)
    return dict(words=words, sh=sh, sh2=sh2, w2=w2, cnt=cnt, dis=dis, cur=cur, prof=prof, ac=ac, hoff=hoff)


def assert_same(g, ref, P, times):
    assert np.array_equal(g["cur"], ref.extra["counters_at"]), "hop counters at the sample times"
    if g["hoff"] is not None:
        assert np.array_equal(g["hoff"], ref.extra["height_offset"]), "height of the seam column"
    if g["prof"] is not None:
        assert np.array_equal(g["prof"].astype(np.int64), ref.extra["profile"]), "occupancy profile"
    if g["ac"] is not None:
        assert np.array_equal(g["ac"], ref.extra["overlap"]), "autocorrelation overlap"
    assert g["words"].shape == ref.state.shape
    bad = np.argwhere(g["words"] != ref.state)
    assert bad.size == 0, f"{len(bad)} words differ, first at {bad[:3].tolist()}"
    assert np.array_equal(g["cnt"], ref.counters), (g["cnt"][:3], ref.counters[:3])
    nt = len([t for t in times if t <= max(times)])
    assert g["sh"].shape[0] == nt
    for ti in range(nt):
        for s in range(P.S):
            for pl in range(P.planes):
                assert int(g["sh"][ti, s, pl]) == ref.sum_h[ti, s, pl], (ti, s, pl)
                s2 = (int(g["sh2"][ti, s, pl, 1]) << 64) | int(g["sh2"][ti, s, pl, 0])
                assert s2 == ref.sum_h2[ti, s, pl], (ti, s, pl)
                assert g["w2"][ti, s, pl] == pytest.approx(ref.w2[ti, s, pl], rel=1e-15, abs=0)


RING = A.ASEP_MODEL_RING
TWO = A.ASEP_MODEL_TWO_LANE
SCA = A.ASEP_SCHED_SCA
PQ = A.ASEP_DIS_BIMODAL_PQ
XING = A.ASEP_DIS_CROSSING
CASES = {
    # several CTAs (16 samples each) with a ragged last CTA
    "ring_asep_ragged": (dict(L=4096, domain_sites=256, samples_per_real=20, p_thr=th(0.75), q_thr=th(0.25),
                              seed=3), 40, [0, 1, 2, 7, 40]),
    "ring_tasep_d32": (dict(L=2048, domain_sites=32, samples_per_real=6, seed=5), 30, [0, 30]),
    "ring_d64": (dict(L=8192, domain_sites=64, samples_per_real=3, p_thr=th(0.6), q_thr=th(0.1), seed=9), 20,
                 [3, 20]),
    "ring_d2048": (dict(L=8192, domain_sites=2048, samples_per_real=3, p_thr=th(0.75), q_thr=th(0.25), seed=11),
                   10, [0, 5, 10]),
    "ring_multi_tile": (dict(L=1 << 15, domain_sites=256, samples_per_real=5, p_thr=th(0.8), seed=13), 25,
                        [0, 25]),
    "ring_cfg1_columns": (dict(L=1 << 17, domain_sites=256, samples_per_real=3, p_thr=th(0.75), q_thr=th(0.25),
                               seed=1), 6, [0, 3, 6]),
    # 64 columns per sample, several samples per CTA: warps sort their domains by Poisson count (hop counts on)
    "ring_sorted_packed": (dict(L=1 << 14, domain_sites=128, samples_per_real=20, p_thr=th(0.75), q_thr=th(0.25),
                                seed=31, flags=A.ASEP_FLAG_PROFILE), 25, [0, 9, 25]),
    "ring_min_L": (dict(L=64, domain_sites=32, samples_per_real=40, p_thr=th(0.7), q_thr=th(0.3), seed=2), 50,
                   [0, 50]),
    "ring_first_sample": (dict(L=4096, domain_sites=128, samples_per_real=4, first_sample=8, p_thr=th(0.75),
                               q_thr=th(0.25), seed=3), 12, [12]),
    "ring_bernoulli": (dict(L=4096, domain_sites=128, samples_per_real=4, init_kind=1, init_seed=77,
                            p_thr=th(0.75), q_thr=th(0.25), seed=3), 12, [0, 12]),
    "ring_frozen": (dict(L=4096, domain_sites=128, samples_per_real=2, p_thr=0, q_thr=0, seed=3), 5, [0, 5]),
    "bimodal_cfg2_shape": (dict(L=1 << 16, domain_sites=256, n_realizations=3, samples_per_real=2,
                                dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_c_thr=0,
                                dis_seed=21, seed=4), 20, [0, 10, 20]),
    "bimodal_qssep": (dict(L=8192, domain_sites=128, n_realizations=2, samples_per_real=2, p_thr=th(0.5),
                           q_thr=th(0.5), dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.5), dis_b_thr=th(0.1),
                           dis_c_thr=th(0.1), dis_seed=5, seed=6), 15, [15]),
    "two_lane_cfg3_shape": (dict(model=TWO, L=1 << 16, domain_sites=256, samples_per_real=3, init_kind=1,
                                 init_seed=8, dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1),
                                 dis_seed=9, q_thr=A.ASEP_ALWAYS, flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR,
                                 autocorr_t0=4), 10, [0, 2, 4, 7, 10]),
    "two_lane_autocorr_from_start": (dict(model=TWO, L=4096, domain_sites=128, samples_per_real=2, init_kind=1,
                                          init_seed=3, dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05),
                                          dis_b_thr=th(0.1), dis_seed=4, q_thr=A.ASEP_ALWAYS, seed=5,
                                          flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=0),
                                     6, [0, 3, 6]),
    "two_lane_plain": (dict(model=TWO, L=4096, domain_sites=64, samples_per_real=4, init_kind=1, init_seed=1,
                            p_thr=th(0.5), q_thr=th(0.7), seed=7), 15, [15]),
    "serial_cfg0_shape": (dict(L=4096, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=8, seed=1), 200,
                          every(100, 200)),
    "serial_asep": (dict(L=1024, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=5, p_thr=th(0.75),
                         q_thr=th(0.25), seed=12), 30, [0, 10, 30]),
    # 2^21 sites (256 KB per sample): too large to stage in shared memory, the lattice stays in global memory
    "serial_global_lattice": (dict(L=1 << 21, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=2, p_thr=th(0.75),
                                   q_thr=th(0.25), seed=21), 2, [0, 2]),
    "serial_two_lane": (dict(model=TWO, L=1024, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=3, init_kind=1,
                             init_seed=4, dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1),
                             dis_seed=2, q_thr=A.ASEP_ALWAYS, seed=3,
                             flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=5), 20, [0, 5, 20]),
    "serial_bimodal": (dict(L=2048, schedule=A.ASEP_SCHED_SERIAL, n_realizations=2, samples_per_real=2,
                            dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=3, seed=4),
                       20, [20]),
    # the serial schedule's two plans: one CTA per sample running a sweep in dependency rounds (the automatic
    # plan while the lattice and the sweep's draws fit shared memory: the cases above), and one warp per
    # sample taking committed prefixes of 32 attempts (plan 2; the automatic plan beyond)
    "serial_rounds_largest_ring": (dict(L=1 << 14, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=2,
                                        p_thr=th(0.75), q_thr=th(0.25), seed=31, plan=(1, 0)), 6, [0, 3, 6]),
    "serial_rounds_largest_two_lane": (dict(model=TWO, L=1 << 13, schedule=A.ASEP_SCHED_SERIAL, n_realizations=2,
                                            samples_per_real=1, init_kind=1, init_seed=32, q_thr=A.ASEP_ALWAYS,
                                            dis_kind=XING, dis_a_thr=th(0.5), dis_b_thr=th(0.8),
                                            dis_c_thr=th(0.2), dis_seed=33, seed=34, plan=(1, 0)), 4, [0, 2, 4]),
    "serial_rounds_smallest_two_lane": (dict(model=TWO, L=64, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=5,
                                             init_kind=1, init_seed=42, q_thr=A.ASEP_ALWAYS,
                                             dis_kind=A.ASEP_DIS_CROSSING, dis_a_thr=th(0.5), dis_b_thr=th(0.8),
                                             dis_c_thr=th(0.2), dis_seed=43, seed=44), 30, [0, 7, 30]),
    "serial_rounds_smallest": (dict(L=64, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=33, p_thr=th(0.6),
                                    q_thr=th(0.3), seed=35, flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR,
                                    autocorr_t0=10), 40, [0, 10, 25, 40]),
    "serial_warp_cfg0_shape": (dict(L=4096, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=8, seed=1,
                                    plan=(2, 0)), 50, [0, 50]),
    "serial_warp_two_lane": (dict(model=TWO, L=1024, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=3,
                                  init_kind=1, init_seed=4, dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05),
                                  dis_b_thr=th(0.1), dis_seed=2, q_thr=A.ASEP_ALWAYS, seed=3, plan=(2, 0),
                                  flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=5), 20,
                             [0, 5, 20]),
    "serial_warp_bimodal_pq": (dict(L=2048, schedule=A.ASEP_SCHED_SERIAL, n_realizations=2, samples_per_real=2,
                                    p_thr=th(0.5), q_thr=th(0.5), dis_kind=A.ASEP_DIS_BIMODAL_PQ,
                                    dis_a_thr=th(0.5), dis_b_thr=th(0.1), dis_c_thr=th(0.1), dis_seed=52,
                                    seed=53, plan=(2, 0)), 12, [0, 12]),
    # cluster tier: one sample spread over 2..16 CTAs of a thread-block cluster
    # the paper's two-sub-lattice SCA schedule (bit-sliced, one CTA per ring)
    "sca_asep": (dict(L=1 << 15, schedule=SCA, samples_per_real=6, p_thr=th(0.75), q_thr=th(0.25), seed=5,
                      flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=3), 40, [0, 3, 17, 40]),
    "sca_tasep_deterministic": (dict(L=4096, schedule=SCA, samples_per_real=3, seed=2), 25, [0, 1, 25]),
    "sca_twenty_bit_rates": (dict(L=2048, schedule=SCA, samples_per_real=9, p_thr=th(0.6), q_thr=th(0.3), seed=8),
                             30, [0, 7, 30]),
    "sca_bimodal": (dict(L=1 << 14, schedule=SCA, n_realizations=2, samples_per_real=2, p_thr=th(0.9),
                         q_thr=th(0.2), dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3),
                         dis_c_thr=th(0.05), dis_seed=12, seed=14), 30, [0, 30]),
    "sca_one_unit": (dict(L=256, schedule=SCA, samples_per_real=20, p_thr=th(0.7), q_thr=th(0.2), seed=6), 40,
                     [0, 40]),
    "sca_growth_regime_shape": (dict(L=1 << 17, schedule=SCA, samples_per_real=4, p_thr=th(0.75), q_thr=th(0.25),
                                     seed=1, flags=A.ASEP_FLAG_NO_HOP_COUNTS), 20, [0, 10, 20]),
    "sca_max_L": (dict(L=1 << 20, schedule=SCA, samples_per_real=1, p_thr=th(0.75), q_thr=th(0.25), seed=3), 3,
                  [0, 3]),
    "sca_bimodal_max_L": (dict(L=1 << 19, schedule=SCA, samples_per_real=1, p_thr=A.ASEP_ALWAYS, q_thr=0,
                               dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=4,
                               seed=7), 3, [0, 3]),
    # the two-lane SCA (paper sec. 3): even bonds, A -> B, odd bonds, B -> A
    "sca_two_lane_turning": (dict(model=TWO, L=4096, schedule=SCA, samples_per_real=3, init_kind=1, init_seed=9,
                                  p_thr=th(0.5), q_thr=th(0.5), dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.1),
                                  dis_b_thr=th(0.3), dis_seed=10, seed=11,
                                  flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=5), 20, [0, 5, 20]),
    "sca_two_lane_rate1": (dict(model=TWO, L=1 << 16, schedule=SCA, samples_per_real=2, init_kind=1, init_seed=4,
                                p_thr=A.ASEP_ALWAYS, q_thr=A.ASEP_ALWAYS, dis_kind=A.ASEP_DIS_TURNING,
                                dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=5, seed=6), 10, [0, 10]),
    "sca_two_lane_plain": (dict(model=TWO, L=2048, schedule=SCA, samples_per_real=5, init_kind=1, init_seed=2,
                                p_thr=th(0.7), q_thr=th(0.4), seed=12), 25, [0, 12, 25]),
    "sca_two_lane_max_L": (dict(model=TWO, L=1 << 18, schedule=SCA, samples_per_real=1, init_kind=1, init_seed=3,
                                p_thr=th(0.5), q_thr=th(0.5), dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05),
                                dis_b_thr=th(0.1), dis_seed=6, seed=7), 3, [0, 3]),
    # streamed SCA (plan 32): the ring in global memory, one launch per phase, a thread per unit of 8 words;
    # ragged unit counts leave most of the last block idle, one unit wraps onto its own first word
    "sca_stream_asep": (dict(L=1 << 15, schedule=SCA, samples_per_real=3, p_thr=th(0.75), q_thr=th(0.25), seed=5,
                             plan=(32, 0), flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=3), 25,
                        [0, 3, 17, 25]),
    "sca_stream_twenty_bit_ragged": (dict(L=256 * 9, schedule=SCA, samples_per_real=7, p_thr=th(0.6),
                                          q_thr=th(0.3), seed=8, plan=(32, 0)), 30, [0, 7, 30]),
    "sca_stream_tasep_deterministic": (dict(L=4096, schedule=SCA, samples_per_real=3, seed=2, plan=(32, 0)), 25,
                                       [0, 1, 25]),
    "sca_stream_bimodal_ragged": (dict(L=(1 << 14) + 768, schedule=SCA, n_realizations=2, samples_per_real=2,
                                       p_thr=th(0.9), q_thr=th(0.2), dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1),
                                       dis_b_thr=th(0.3), dis_c_thr=th(0.05), dis_seed=12, seed=14, plan=(32, 0)),
                                  30, [0, 30]),
    "sca_stream_one_unit": (dict(L=256, schedule=SCA, samples_per_real=20, p_thr=th(0.7), q_thr=th(0.2), seed=6,
                                 plan=(32, 0)), 40, [0, 40]),
    "sca_stream_two_lane_turning": (dict(model=TWO, L=4096 + 256, schedule=SCA, samples_per_real=3, init_kind=1,
                                         init_seed=9, p_thr=th(0.5), q_thr=th(0.5), dis_kind=A.ASEP_DIS_TURNING,
                                         dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=10, seed=11, plan=(32, 0),
                                         flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=5), 20,
                                    [0, 5, 20]),
    "sca_stream_two_lane_dense_turning": (dict(model=TWO, L=2048, schedule=SCA, samples_per_real=4, init_kind=1,
                                               init_seed=19, p_thr=A.ASEP_ALWAYS, q_thr=th(0.8),
                                               dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.9), dis_b_thr=th(0.6),
                                               dis_seed=20, seed=21, plan=(32, 0)), 15, [0, 15]),
    "sca_stream_two_lane_one_unit": (dict(model=TWO, L=256, schedule=SCA, samples_per_real=6, init_kind=1,
                                          init_seed=3, p_thr=th(0.5), q_thr=th(0.5), dis_kind=A.ASEP_DIS_TURNING,
                                          dis_a_thr=th(0.5), dis_b_thr=th(0.5), dis_seed=4, seed=5, plan=(32, 0)),
                                     30, [0, 30]),
    "sca_stream_two_lane_plain": (dict(model=TWO, L=2048, schedule=SCA, samples_per_real=5, init_kind=1,
                                       init_seed=2, p_thr=th(0.7), q_thr=th(0.4), seed=12, plan=(32, 0)), 25,
                                  [0, 12, 25]),
    # independent p and q classes (the paper's separate tag bits; Q-SSEP): resident and streamed SCA, serial
    "sca_bimodal_pq": (dict(L=1 << 14, schedule=SCA, n_realizations=2, samples_per_real=2, p_thr=th(0.5),
                            q_thr=th(0.5), dis_kind=PQ, dis_a_thr=th(0.5), dis_b_thr=th(0.1), dis_c_thr=th(0.1),
                            dis_seed=44, seed=45, flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=6),
                       30, [0, 6, 30]),
    "sca_bimodal_pq_twenty_bit": (dict(L=4096, schedule=SCA, n_realizations=3, samples_per_real=1, p_thr=th(0.6),
                                       q_thr=th(0.3), dis_kind=PQ, dis_a_thr=th(0.3), dis_b_thr=th(0.15),
                                       dis_c_thr=A.ASEP_ALWAYS, dis_seed=46, seed=47), 25, [0, 25]),
    "sca_stream_bimodal_pq": (dict(L=256 * 2085, schedule=SCA, n_realizations=2, samples_per_real=1,
                                   p_thr=th(0.5), q_thr=th(0.5), dis_kind=PQ, dis_a_thr=th(0.5),
                                   dis_b_thr=th(0.1), dis_c_thr=th(0.1), dis_seed=48, seed=49, plan=(32, 0)), 6,
                              [0, 3, 6]),
    # two quenched planes do not fit one CTA's shared memory at 2^20 sites: streamed by itself
    "sca_bimodal_pq_beyond_smem": (dict(L=1 << 20, schedule=SCA, samples_per_real=1, p_thr=th(0.5),
                                        q_thr=th(0.5), dis_kind=PQ, dis_a_thr=th(0.5), dis_b_thr=th(0.1),
                                        dis_c_thr=th(0.1), dis_seed=50, seed=51), 3, [0, 3]),
    "serial_bimodal_pq": (dict(L=2048, schedule=A.ASEP_SCHED_SERIAL, n_realizations=2, samples_per_real=2,
                               p_thr=th(0.5), q_thr=th(0.5), dis_kind=PQ, dis_a_thr=th(0.5), dis_b_thr=th(0.1),
                               dis_c_thr=th(0.1), dis_seed=52, seed=53), 12, [0, 12]),
    # the paper's two-lane crossing probabilities: every site, u_i / v_i 0.8 or 0.2 at marked sites
    "sca_two_lane_crossing": (dict(model=TWO, L=4096, schedule=SCA, n_realizations=2, samples_per_real=2,
                                   init_kind=1, init_seed=12, p_thr=th(0.5), q_thr=th(0.5), dis_kind=XING,
                                   dis_a_thr=th(0.5), dis_b_thr=th(0.8), dis_c_thr=th(0.2), dis_seed=13, seed=14,
                                   flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=4), 15, [0, 4, 15]),
    "sca_stream_two_lane_crossing": (dict(model=TWO, L=256 * 2085, schedule=SCA, n_realizations=2,
                                          samples_per_real=1, init_kind=1, init_seed=15, p_thr=th(0.5),
                                          q_thr=th(0.5), dis_kind=XING, dis_a_thr=th(0.5), dis_b_thr=th(0.8),
                                          dis_c_thr=th(0.2), dis_seed=16, seed=17, plan=(32, 0)), 4, [0, 4]),
    # two lanes and two class planes do not fit one CTA's shared memory at 2^19 sites: streamed by itself
    "sca_two_lane_crossing_beyond_smem": (dict(model=TWO, L=1 << 19, schedule=SCA, samples_per_real=1,
                                               init_kind=1, init_seed=18, p_thr=th(0.5), q_thr=th(0.5),
                                               dis_kind=XING, dis_a_thr=th(0.5), dis_b_thr=th(0.8),
                                               dis_c_thr=th(0.2), dis_seed=19, seed=20), 2, [0, 2]),
    "serial_two_lane_crossing": (dict(model=TWO, L=1024, schedule=A.ASEP_SCHED_SERIAL, n_realizations=2,
                                      samples_per_real=2, init_kind=1, init_seed=21, q_thr=A.ASEP_ALWAYS,
                                      dis_kind=XING, dis_a_thr=th(0.5), dis_b_thr=th(0.8), dis_c_thr=th(0.2),
                                      dis_seed=22, seed=23), 10, [0, 10]),
    # many blocks of unit threads, the last one ragged (2085 units, 1025 units), so carries and lane-change
    # sites cross block boundaries; 16680 words per lattice: records in two chunks (16384 + 296 words)
    "sca_stream_ring_nine_blocks": (dict(L=256 * 2085, schedule=SCA, n_realizations=2, samples_per_real=1,
                                         p_thr=th(0.8), q_thr=th(0.35), dis_kind=A.ASEP_DIS_BIMODAL,
                                         dis_a_thr=th(0.2), dis_b_thr=th(0.4), dis_c_thr=th(0.1), dis_seed=31,
                                         seed=32, plan=(32, 0), flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR,
                                         autocorr_t0=1), 7, [0, 1, 4, 7]),
    "sca_stream_ring_five_blocks_fast": (dict(L=256 * 1025, schedule=SCA, samples_per_real=3, p_thr=th(0.75),
                                              q_thr=th(0.25), seed=33, plan=(32, 0)), 6, [0, 3, 6]),
    "sca_stream_two_lane_nine_blocks": (dict(model=TWO, L=256 * 2085, schedule=SCA, samples_per_real=1,
                                             init_kind=1, init_seed=40, p_thr=th(0.6), q_thr=th(0.45),
                                             dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.3), dis_b_thr=th(0.5),
                                             dis_seed=41, seed=42, plan=(32, 0)), 5, [0, 5]),
    # beyond one CTA's shared memory the SCA streams by itself
    "sca_stream_beyond_smem": (dict(L=1 << 21, schedule=SCA, samples_per_real=2, p_thr=th(0.75), q_thr=th(0.25),
                                    seed=13), 3, [0, 3]),
    "sca_stream_two_lane_beyond_smem": (dict(model=TWO, L=1 << 20, schedule=SCA, samples_per_real=1, init_kind=1,
                                             init_seed=3, p_thr=th(0.5), q_thr=th(0.5), dis_kind=A.ASEP_DIS_TURNING,
                                             dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=6, seed=7), 2, [0, 2]),
    # streamed tier (plan 32): lattice in global memory, tiles of columns through shared memory
    "stream_ring": (dict(L=1 << 16, domain_sites=256, samples_per_real=3, p_thr=th(0.75), q_thr=th(0.25), seed=61,
                         plan=(32, 0), flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=5), 13,
                    [0, 5, 13]),
    "stream_ring_four_tiles": (dict(L=1 << 18, domain_sites=32, samples_per_real=2, p_thr=th(0.6), q_thr=th(0.3),
                                    seed=62, plan=(32, 1024)), 6, [0, 6]),
    "stream_bimodal": (dict(L=1 << 16, domain_sites=128, n_realizations=2, samples_per_real=2, p_thr=A.ASEP_ALWAYS,
                            dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_c_thr=th(0.05),
                            q_thr=th(0.1), dis_seed=63, seed=64, plan=(32, 0)), 9, [0, 9]),
    "stream_two_lane": (dict(model=TWO, L=1 << 16, domain_sites=128, samples_per_real=2, init_kind=1, init_seed=65,
                             dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=66,
                             q_thr=A.ASEP_ALWAYS, seed=67, plan=(32, 0),
                             flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=4), 8, [0, 4, 8]),
    # 2^24 sites = 32768 columns: more than 16 CTAs of 1024 columns, so the streamed tier is chosen
    "stream_beyond_cluster": (dict(L=1 << 24, domain_sites=256, samples_per_real=1, p_thr=th(0.75), q_thr=th(0.25),
                                   seed=68), 2, [0, 2]),
    "cluster_ring_2x": (dict(L=1 << 20, domain_sites=256, samples_per_real=2, p_thr=th(0.75), q_thr=th(0.25),
                             seed=51), 5, [0, 2, 5]),
    "cluster_ring_d64": (dict(L=1 << 18, domain_sites=64, samples_per_real=2, p_thr=th(0.6), seed=52), 6, [0, 6]),
    "cluster_uneven_slices": (dict(L=1025 * 512, domain_sites=256, samples_per_real=1, p_thr=th(0.75),
                                   q_thr=th(0.25), seed=53), 4, [0, 4]),
    "cluster_bimodal": (dict(L=1 << 19, domain_sites=256, n_realizations=2, samples_per_real=1,
                             dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=7, seed=54),
                        4, [0, 4]),
    "cluster_two_lane": (dict(model=TWO, L=1 << 19, domain_sites=256, samples_per_real=1, init_kind=1, init_seed=5,
                              dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=8,
                              q_thr=A.ASEP_ALWAYS, seed=55, flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR,
                              autocorr_t0=1), 3, [0, 1, 3]),
    # the paper's independent p and q classes (sec. 2.3) and crossing marks (sec. 3) under the domain schedule:
    # resident (with several samples per CTA and the lane sort), streamed and cluster tiers
    "domain_bimodal_pq": (dict(L=8192, domain_sites=128, n_realizations=2, samples_per_real=2, p_thr=th(0.5),
                               q_thr=th(0.5), dis_kind=PQ, dis_a_thr=th(0.5), dis_b_thr=th(0.1), dis_c_thr=th(0.1),
                               dis_seed=70, seed=71, flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=5),
                          20, [0, 5, 20]),
    "domain_bimodal_pq_packed": (dict(L=1 << 14, domain_sites=128, n_realizations=4, samples_per_real=3,
                                      p_thr=th(0.8), q_thr=th(0.8), dis_kind=PQ, dis_a_thr=th(0.3),
                                      dis_b_thr=th(0.2), dis_c_thr=A.ASEP_ALWAYS, dis_seed=72, seed=73), 15, [0, 15]),
    "domain_bimodal_pq_cfg1_columns": (dict(L=1 << 17, domain_sites=256, n_realizations=2, samples_per_real=1,
                                            p_thr=th(0.75), q_thr=th(0.25), dis_kind=PQ, dis_a_thr=th(0.1),
                                            dis_b_thr=th(0.3), dis_c_thr=th(0.05), dis_seed=74, seed=75), 5, [0, 5]),
    "stream_bimodal_pq": (dict(L=1 << 16, domain_sites=128, n_realizations=2, samples_per_real=1, p_thr=th(0.5),
                               q_thr=th(0.5), dis_kind=PQ, dis_a_thr=th(0.5), dis_b_thr=th(0.1), dis_c_thr=th(0.1),
                               dis_seed=76, seed=77, plan=(32, 0)), 7, [0, 7]),
    "cluster_bimodal_pq": (dict(L=1 << 19, domain_sites=256, n_realizations=2, samples_per_real=1, p_thr=th(0.5),
                                q_thr=th(0.5), dis_kind=PQ, dis_a_thr=th(0.5), dis_b_thr=th(0.1),
                                dis_c_thr=th(0.1), dis_seed=78, seed=79), 3, [0, 3]),
    "domain_two_lane_crossing": (dict(model=TWO, L=4096, domain_sites=64, n_realizations=2, samples_per_real=2,
                                      init_kind=1, init_seed=80, p_thr=th(0.5), q_thr=th(0.5), dis_kind=XING,
                                      dis_a_thr=th(0.5), dis_b_thr=th(0.8), dis_c_thr=th(0.2), dis_seed=81, seed=82,
                                      flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=4),
                                 12, [0, 4, 12]),
    "domain_two_lane_crossing_cfg3_shape": (dict(model=TWO, L=1 << 16, domain_sites=128, samples_per_real=3,
                                                 init_kind=1, init_seed=83, p_thr=A.ASEP_ALWAYS,
                                                 q_thr=A.ASEP_ALWAYS, dis_kind=XING, dis_a_thr=th(0.5),
                                                 dis_b_thr=th(0.8), dis_c_thr=th(0.2), dis_seed=84, seed=85),
                                            6, [0, 6]),
    "stream_two_lane_crossing": (dict(model=TWO, L=1 << 16, domain_sites=128, n_realizations=2, samples_per_real=1,
                                      init_kind=1, init_seed=86, p_thr=th(0.5), q_thr=th(0.5), dis_kind=XING,
                                      dis_a_thr=th(0.5), dis_b_thr=th(0.8), dis_c_thr=th(0.2), dis_seed=87, seed=88,
                                      plan=(32, 0)), 5, [0, 5]),
    "cluster_two_lane_crossing": (dict(model=TWO, L=1 << 18, domain_sites=256, samples_per_real=1, init_kind=1,
                                       init_seed=89, p_thr=A.ASEP_ALWAYS, q_thr=A.ASEP_ALWAYS, dis_kind=XING,
                                       dis_a_thr=th(0.5), dis_b_thr=th(0.8), dis_c_thr=th(0.2), dis_seed=90,
                                       seed=91), 3, [0, 3]),
    "cluster_ring_max_L": (dict(L=1 << 22, domain_sites=256, samples_per_real=1, p_thr=th(0.75), q_thr=th(0.25),
                                seed=56), 2, [0, 2]),
    "cluster_two_lane_max_L": (dict(model=TWO, L=1 << 22, domain_sites=256, samples_per_real=1, init_kind=1,
                                    init_seed=6, dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05),
                                    dis_b_thr=th(0.1), dis_seed=9, q_thr=A.ASEP_ALWAYS, seed=57), 1, [0, 1]),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_bit_exact_against_oracle(name):
    kw, n, times = CASES[name]
    g = run_gpu(kw, [n], times)
    P = oracle_params(kw)
    ref = oracle.run(P, n, times, autocorr_t0=kw.get("autocorr_t0") if kw.get("flags", 0) & A.ASEP_FLAG_AUTOCORR
                     else None)
    if P.dis_kind != 0:
        assert np.array_equal(g["dis"], oracle.disorder(P))
    if kw.get("flags", 0) & A.ASEP_FLAG_NO_HOP_COUNTS:  # the ring's hop counters stay off
        ref.counters[:] = 0
        ref.extra["counters_at"][:] = 0
    assert_same(g, ref, P, times)


def test_launch_splitting_is_invisible():
    kw = dict(L=8192, domain_sites=128, samples_per_real=5, p_thr=th(0.75), q_thr=th(0.25), seed=31)
    times = [0, 4, 7, 20, 25]
    a = run_gpu(kw, [25], times)
    b = run_gpu(kw, [7, 13, 5], times)
    c = run_gpu(kw, [1] * 25, times)
    for x in (b, c):
        assert np.array_equal(a["words"], x["words"])
        assert np.array_equal(a["sh"], x["sh"]) and np.array_equal(a["sh2"], x["sh2"])
        assert np.array_equal(a["cnt"], x["cnt"])


def test_hop_count_flag_changes_nothing_else():
    kw = dict(L=1 << 15, domain_sites=256, samples_per_real=3, p_thr=th(0.75), q_thr=th(0.25), seed=43)
    a = run_gpu(kw, [20], [0, 20])
    b = run_gpu(dict(kw, flags=A.ASEP_FLAG_NO_HOP_COUNTS), [20], [0, 20])
    assert np.array_equal(a["words"], b["words"]) and np.array_equal(a["sh"], b["sh"])
    assert a["cnt"][:, :2].sum() > 0 and not b["cnt"].any()


def test_checkpoint_resume_is_bit_exact():
    kw = dict(model=TWO, L=4096, domain_sites=128, samples_per_real=3, init_kind=1, init_seed=6,
              dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=5, seed=8)
    full = run_gpu(kw, [30], [30])
    with A.asep_create(A.make_params(**kw), sample_times=[30]) as c1:
        A.asep_sweep(c1, 11)
        words, s = A.asep_state(c1)
    with A.asep_create(A.make_params(**kw), sample_times=[30]) as c2:
        A.asep_load_state(c2, words, s)
        A.asep_sweep(c2, 19)
        w2, s2 = A.asep_state(c2)
        sh, sh2, _ = A.asep_width(c2)
    assert s2 == 30 and np.array_equal(w2, full["words"])
    assert np.array_equal(sh[-1], full["sh"][-1]) and np.array_equal(sh2[-1], full["sh2"][-1])


def test_reset_reproduces_a_fresh_context():
    kw = dict(L=8192, domain_sites=256, samples_per_real=4, p_thr=th(0.75), q_thr=th(0.25), seed=41)
    fresh = run_gpu(kw, [9], [0, 9])
    with A.asep_create(A.make_params(**dict(kw, seed=5)), sample_times=[0, 9]) as ctx:
        A.asep_sweep(ctx, 17)
        A.asep_reset(ctx, seed=41)
        A.asep_sweep(ctx, 9)
        words, _ = A.asep_state(ctx)
        sh, _, _ = A.asep_width(ctx)
        cnt = A.asep_counters(ctx)
        hoff = A.asep_height_offset(ctx)
    assert np.array_equal(words, fresh["words"]) and np.array_equal(sh, fresh["sh"])
    assert np.array_equal(cnt, fresh["cnt"]) and np.array_equal(hoff, fresh["hoff"])


def test_height_offset_restarts_at_a_loaded_state():
    """After asep_load_state the column height is measured from the loaded
    lattice: resumed H(30) = H(30) - H(11) of the uninterrupted run."""
    kw = dict(L=8192, domain_sites=128, samples_per_real=5, p_thr=th(0.75), q_thr=th(0.25), seed=13)
    with A.asep_create(A.make_params(**kw), sample_times=[11, 30]) as c1:
        A.asep_sweep(c1, 11)
        words, s = A.asep_state(c1)
        A.asep_sweep(c1, 19)
        full = A.asep_height_offset(c1)
    with A.asep_create(A.make_params(**kw), sample_times=[11, 30]) as c2:
        A.asep_load_state(c2, words, s)
        A.asep_sweep(c2, 19)
        resumed = A.asep_height_offset(c2)
    assert np.any(full[1] != full[0])
    assert np.array_equal(resumed[1], full[1] - full[0])
    with A.asep_create(A.make_params(model=TWO, L=4096, domain_sites=128), sample_times=[]) as c3:
        with pytest.raises(A.AsepError):
            A.asep_height_offset(c3)


def test_cfg0_full_run_snapshots_every_100_mcs():
    """Plain serial RSU, L = 4096, 8 samples, p = 1, q = 0, 10^4 MCS: the
    lattice every 100 MCS and W(t) bit-exact against the oracle."""
    kw = dict(L=4096, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=8, seed=1)
    times = every(100, 10**4)
    P = oracle_params(kw)
    ref_state = oracle.init_state(P)
    ref_sums = [[oracle.heights(ref_state[s, 0], P.L) for s in range(P.S)]]
    with A.asep_create(A.make_params(**kw), sample_times=times) as ctx:
        for k in range(100):
            A.asep_sweep(ctx, 100)
            words, _ = A.asep_state(ctx)
            oracle.replay(P, ref_state, 100 * k, 100)
            assert np.array_equal(words, ref_state), f"lattice differs after {100 * (k + 1)} MCS"
            ref_sums.append([oracle.heights(ref_state[s, 0], P.L) for s in range(P.S)])
        sh, sh2, w2 = A.asep_width(ctx)
    assert sh.shape[0] == len(times) == len(ref_sums)
    for ti in range(len(times)):
        for s in range(P.S):
            a, b = ref_sums[ti][s]
            assert int(sh[ti, s, 0]) == a and ((int(sh2[ti, s, 0, 1]) << 64) | int(sh2[ti, s, 0, 0])) == b
    assert np.all(w2[0] == 0.25)


def _np_sums(row: np.ndarray, L: int) -> tuple[int, int]:
    """(sum h, sum h^2) of one packed lattice row by plain numpy, h_i = sum_{j<=i} (2 n_j - 1);
    |h| <= L = 2^17 keeps sum h^2 below 2^51."""
    bits = np.unpackbits(row.view(np.uint8), bitorder="little")[:L].astype(np.int64)
    h = np.cumsum(2 * bits - 1)
    return int(h.sum()), int((h * h).sum())


def test_cfg1_full_size_spot_checks():
    """The benchmarked launch configuration (L = 2^17, 256 samples, D = 256,
    log times): sampled samples bit-exact against the oracle, which replays
    them from their own initial state, over the first 1000 sweeps (lattices
    and every record up to there); then the rest of the 2^14 sweeps, checked
    by properties that hold at any size: particle number, the final record
    equals the sums of the final lattice, W^2(0) = 1/4."""
    n_mcs, k1 = 1 << 14, 1000
    times = log_times(n_mcs) + [n_mcs]  # the log times end below 2^14; record the last sweep too
    kw = dict(L=1 << 17, domain_sites=256, samples_per_real=256, p_thr=th(0.75), q_thr=th(0.25), seed=1)
    P = oracle_params(kw)
    picks = [0, 97, 255]
    with A.asep_create(A.make_params(**kw), sample_times=times) as ctx:
        A.asep_sweep(ctx, k1)
        at_k1, _ = A.asep_state(ctx)
        A.asep_sweep(ctx, n_mcs - k1)
        final, s_final = A.asep_state(ctx)
        sh, sh2, w2 = A.asep_width(ctx)
    early = [t for t in times if t <= k1]
    ref = oracle.run(P, k1, early, samples=picks)
    for s in picks:
        assert np.array_equal(at_k1[s], ref.state[s]), s
        for ti in range(len(early)):
            assert int(sh[ti, s, 0]) == int(ref.sum_h[ti, s, 0]), (s, early[ti])
            assert ((int(sh2[ti, s, 0, 1]) << 64) | int(sh2[ti, s, 0, 0])) == int(ref.sum_h2[ti, s, 0]), (s, early[ti])
    assert s_final == n_mcs
    # every sample keeps half filling; the last record is the final lattice's sums; W^2(0) = 1/4 exactly
    pop = np.unpackbits(final.view(np.uint8), axis=-1).sum(axis=-1)
    assert np.all(pop == P.L // 2)
    for s in range(P.S):
        a, b = _np_sums(final[s, 0], P.L)
        assert int(sh[-1, s, 0]) == a and ((int(sh2[-1, s, 0, 1]) << 64) | int(sh2[-1, s, 0, 0])) == b, s
    assert np.all(w2[0] == 0.25)


# ---------------------------------------------------------------------------
# Statistics: W(t) of the GPU domain schedule vs the serial RSU reference
# ---------------------------------------------------------------------------

def _serial_w2(P, times, mask=None):
    st = oracle.init_state(P)
    out = np.zeros((len(times), P.S, P.planes))
    done = 0
    for i, t in enumerate(times):
        if t > done:
            oracle.serial_reference(P, st, t - done, rng_seeds=np.arange(P.S) * 104729 + t, mask=mask)
            done = t
        for s in range(P.S):
            for pl in range(P.planes):
                out[i, s, pl] = oracle.width2(P.L, *oracle.heights(st[s, pl], P.L))
    return out


@pytest.mark.parametrize("case", ["asep", "tasep", "bimodal", "two_lane", "two_lane_d128"])
def test_width_within_3_sigma_of_serial_reference(case):
    times = [4, 16, 64]
    if case == "asep":
        kw = dict(L=1 << 14, domain_sites=256, samples_per_real=96, p_thr=th(0.75), q_thr=th(0.25), seed=17)
    elif case == "tasep":
        kw = dict(L=1 << 14, domain_sites=256, samples_per_real=96, seed=19)
    elif case == "bimodal":
        kw = dict(L=1 << 14, domain_sites=256, n_realizations=1, samples_per_real=96, dis_kind=A.ASEP_DIS_BIMODAL,
                  dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=23, seed=29)
    else:  # two lanes; D = 128 gives a domain 256 bonds, as the ring's D = 256
        kw = dict(model=TWO, L=1 << 14, domain_sites=128 if case == "two_lane_d128" else 256, samples_per_real=96,
                  init_kind=1, init_seed=3, dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1),
                  dis_seed=31, q_thr=A.ASEP_ALWAYS, seed=37)
    g = run_gpu(kw, [times[-1]], times)
    P = oracle_params(kw)
    mask = oracle.disorder(P)
    ser = _serial_w2(P, times, mask=mask)
    for ti in range(len(times)):
        for pl in range(P.planes):
            a, b = g["w2"][ti, :, pl], ser[ti, :, pl]
            sig = np.sqrt(a.var(ddof=1) / a.size + b.var(ddof=1) / b.size)
            assert abs(a.mean() - b.mean()) < 3 * sig, (case, times[ti], pl, a.mean(), b.mean(), sig)


# ---------------------------------------------------------------------------
# Degenerate inputs
# ---------------------------------------------------------------------------

def test_zero_sweeps_and_no_sample_times():
    """asep_sweep(0) changes nothing; a context without sample times runs and
    reports an empty height table; the lattice still matches the oracle."""
    kw = dict(L=4096, domain_sites=128, samples_per_real=3, p_thr=th(0.75), q_thr=th(0.25), seed=4)
    with A.asep_create(A.make_params(**kw), sample_times=[]) as ctx:
        before, s0 = A.asep_state(ctx)
        A.asep_sweep(ctx, 0)
        after, s1 = A.asep_state(ctx)
        assert s0 == s1 == 0 and np.array_equal(before, after)
        A.asep_sweep(ctx, 9)
        words, s = A.asep_state(ctx)
        sh, sh2, w2 = A.asep_width(ctx)
        assert s == 9 and sh.shape[0] == 0 and A.asep_get_info(ctx)["n_recorded"] == 0
    ref = oracle.run(oracle_params(kw), 9, [])
    assert np.array_equal(words, ref.state)


@pytest.mark.parametrize("schedule", [A.ASEP_SCHED_DOMAIN, A.ASEP_SCHED_SCA])
def test_many_tiny_samples(schedule):
    """Thousands of minimal rings (many samples per CTA, many CTAs), bit-exact
    on sampled samples, counters and heights for all."""
    L = 64 if schedule == A.ASEP_SCHED_DOMAIN else 256
    kw = dict(L=L, schedule=schedule, samples_per_real=5000, p_thr=th(0.7), q_thr=th(0.2), seed=8)
    if schedule == A.ASEP_SCHED_DOMAIN:
        kw["domain_sites"] = 32
    g = run_gpu(kw, [13], [0, 13])
    P = oracle_params(kw)
    ref = oracle.run(P, 13, [0, 13], samples=[0, 1, 2499, 4998, 4999])
    for s in (0, 1, 2499, 4998, 4999):
        assert np.array_equal(g["words"][s], ref.state[s]), s
        assert np.array_equal(g["cnt"][s], ref.counters[s]), s
        assert int(g["sh"][-1, s, 0]) == int(ref.sum_h[-1, s, 0]), s
    # every ring keeps its particle number
    pop = np.unpackbits(g["words"].view(np.uint8), axis=-1).sum(axis=-1)
    assert np.all(pop == L // 2)


def test_sca_growth_exponent_is_kpz():
    """The paper's SCA schedule stays in the KPZ class (sec. 2.2: the SCA
    results were compared with RSU): W^2 - 1/4 grows as t^(2 beta) with
    beta = alpha / z = 1/3 in the growth regime (t << L^(3/2) = 5.9e6).  The
    local slope approaches 2/3 from below (0.56 at t = 16, 0.65 at t = 4096
    for both schedules), so the fit window is t = 256 .. 4096.  (p = 1 from
    the flat state is no test: the deterministic SCA returns to flat.)"""
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
        g = json.load(f)["kpz_exponents"]
    beta = g["alpha"] / g["z"]
    times = [256, 512, 1024, 2048, 4096]
    kw = dict(L=1 << 15, schedule=SCA, samples_per_real=128, seed=17, p_thr=th(0.75), q_thr=th(0.25))
    w2 = run_gpu(kw, [times[-1]], times)["w2"][:, :, 0].mean(axis=1)
    slope = np.polyfit(np.log(times), np.log(w2 - 0.25), 1)[0]
    assert abs(slope - 2 * beta) < 0.07, slope


@pytest.mark.parametrize("model", [0, 1])
def test_sca_plans_switch_mid_run_without_changing_results(model):
    """The SCA's resident and streamed plans, switched between sweeps and
    with launches split differently, give the same lattices, records and
    counters; a ring one CTA cannot hold is streamed and refuses the
    resident plan."""
    if model == 1:
        kw = dict(model=TWO, L=8192, schedule=SCA, samples_per_real=3, init_kind=1, init_seed=4, p_thr=th(0.6),
                  q_thr=th(0.45), dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.2), dis_b_thr=th(0.4), dis_seed=8,
                  seed=9)
    else:
        kw = dict(L=8192, schedule=SCA, samples_per_real=3, p_thr=th(0.6), q_thr=th(0.45), seed=9)
    times = [0, 3, 9, 16]
    ref = run_gpu(kw, [16], times)
    with A.asep_create(A.make_params(**kw), sample_times=times) as ctx:
        assert A.asep_get_info(ctx)["cluster"] == 1
        for k, plan in enumerate([32, 1, 32, 0, 32]):
            A.asep_set_plan(ctx, plan, 0)
            A.asep_sweep(ctx, [2, 5, 1, 4, 4][k])
        words, sweep = A.asep_state(ctx)
        sh, sh2, _ = A.asep_width(ctx)
        assert sweep == 16
        assert np.array_equal(words, ref["words"]) and np.array_equal(sh, ref["sh"]) and np.array_equal(sh2, ref["sh2"])
        assert np.array_equal(A.asep_counters(ctx), ref["cnt"])
        assert np.array_equal(A.asep_currents(ctx), ref["cur"])
    with A.asep_create(A.make_params(L=1 << 21, schedule=SCA), sample_times=[]) as ctx:
        assert A.asep_get_info(ctx)["cluster"] == 32
        with pytest.raises(A.AsepError):
            A.asep_set_plan(ctx, 1, 0)
        assert A.asep_get_info(ctx)["cluster"] == 32  # the previous plan stays
        with pytest.raises(A.AsepError):
            A.asep_set_plan(ctx, 4, 0)



def test_streamed_sca_units_per_thread_do_not_change_results():
    """Streamed SCA rings of 2^23 sites: 192 samples run with four units per
    thread, 96 with two, one with one (the count follows the launch size);
    sample 0 is the same in all three and equals the oracle's."""
    kw = dict(L=1 << 23, schedule=SCA, p_thr=th(0.75), q_thr=th(0.25), seed=71)
    runs = {S: run_gpu(dict(kw, samples_per_real=S), [3], [0, 3]) for S in (192, 96, 1)}
    P = oracle_params(dict(kw, samples_per_real=1))
    assert_same(runs[1], oracle.run(P, 3, [0, 3]), P, [0, 3])
    for S in (192, 96):
        assert np.array_equal(runs[S]["words"].reshape(S, -1)[0], runs[1]["words"].reshape(-1)), S
        assert np.array_equal(runs[S]["cnt"][0], runs[1]["cnt"][0]), S
        assert np.array_equal(runs[S]["sh"][:, 0], runs[1]["sh"][:, 0]), S


def test_streamed_copy_wait_runs_out_and_the_context_recovers():
    """Fault injection on the streamed tier: each tile's copies announce 16
    bytes more than they carry, so the kernels' wait for them runs out after
    its one-second bound; the host reports ASEP_ERR_TIMEOUT (and keeps
    reporting it), the GPU stays usable, and loading a state clears it --
    the sweeps after that are bit-exact again."""
    import time

    kw = dict(L=1 << 16, domain_sites=256, samples_per_real=1, p_thr=th(0.75), q_thr=th(0.25), seed=81)
    ref = run_gpu(dict(kw, plan=(32, 0)), [3], [0, 3])
    with A.asep_create(A.make_params(**kw), sample_times=[0, 3]) as ctx:
        A.asep_set_plan(ctx, 32, 0)
        start, _ = A.asep_state(ctx)
        A.asep_inject_fault(ctx, A.ASEP_FAULT_COPY_STALL)
        t0 = time.time()
        A.asep_sweep(ctx, 1)
        with pytest.raises(A.AsepError) as ei:
            A.asep_sync(ctx)
        assert ei.value.code == A.ASEP_ERR_TIMEOUT
        assert time.time() - t0 < 30  # two launches, each bounded by the one-second wait (twice)
        with pytest.raises(A.AsepError) as ei:
            A.asep_counters(ctx)
        assert ei.value.code == A.ASEP_ERR_TIMEOUT
        A.asep_inject_fault(ctx, A.ASEP_FAULT_NONE)
        A.asep_load_state(ctx, start, 0)
        A.asep_sweep(ctx, 3)
        words, sweep = A.asep_state(ctx)
        assert sweep == 3 and np.array_equal(words, ref["words"])
        with pytest.raises(A.AsepError):
            A.asep_inject_fault(ctx, 7)
    x = torch_probe_ok()
    assert x


def torch_probe_ok() -> bool:
    """A plain device computation after the timeout test: the GPU answers."""
    import torch

    y = torch.arange(1024, device="cuda", dtype=torch.int64).sum().item()
    return y == 1023 * 1024 // 2


@pytest.mark.parametrize("model", [0, TWO, "pq", "crossing"])
def test_streamed_tile_width_does_not_change_results(model):
    """The streamed tier's tile width (columns per CTA, an autotuner knob):
    widths of 32, 96 (a ragged last tile), 128 and 1024 columns give the
    same lattices, heights and counters, and they equal the oracle's -- on
    a ring, two lanes with turning sites, independent p and q classes, and
    two lanes with crossing marks (two quenched planes each)."""
    m = TWO if model in (TWO, "crossing") else 0
    kw = dict(model=m, L=1 << 18, domain_sites=32 if m == 0 else 64, samples_per_real=2, p_thr=th(0.6),
              q_thr=th(0.3), seed=81, init_kind=1, init_seed=82)
    if model == TWO:
        kw.update(dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=83)
    elif model == "pq":
        kw.update(dis_kind=PQ, dis_a_thr=th(0.5), dis_b_thr=th(0.1), dis_c_thr=th(0.2), dis_seed=84)
    elif model == "crossing":
        kw.update(dis_kind=XING, dis_a_thr=th(0.5), dis_b_thr=th(0.8), dis_c_thr=th(0.2), dis_seed=85)
    times = [0, 3, 7]
    runs = {}
    for cols in (32, 96, 128, 1024):
        runs[cols] = run_gpu(dict(kw, plan=(32, cols)), [3, 4], times)
    P = oracle_params(kw)
    assert_same(runs[128], oracle.run(P, 7, times), P, times)
    for cols in (32, 96, 1024):
        for key in ("words", "sh", "sh2", "cnt", "cur"):
            assert np.array_equal(runs[cols][key], runs[128][key]), (cols, key)


def test_streamed_tile_width_is_a_plan_knob():
    with A.asep_create(A.make_params(L=1 << 24, domain_sites=256, samples_per_real=1), sample_times=[]) as ctx:
        info = A.asep_get_info(ctx)
        assert info["cluster"] == 32 and info["tile_columns"] == 128  # the automatic width
        A.asep_set_plan(ctx, 32, 512)
        info = A.asep_get_info(ctx)
        assert info["tile_columns"] == 512 and info["threads"] == 512 and info["groups"] == (1 << 24) // 512 // 512
        for bad in (48, 2048):
            with pytest.raises(A.AsepError):
                A.asep_set_plan(ctx, 32, bad)
            assert A.asep_get_info(ctx)["tile_columns"] == 512  # the previous plan stays
    with A.asep_create(A.make_params(L=1 << 16, domain_sites=256, samples_per_real=1), sample_times=[]) as ctx:
        with pytest.raises(A.AsepError):
            A.asep_set_plan(ctx, 32, 128)  # 128 columns: one tile would hold the whole ring
        A.asep_set_plan(ctx, 32, 0)
        assert A.asep_get_info(ctx)["tile_columns"] == 64


def test_serial_plans():
    """The serial schedule's plan: one CTA per sample (dependency rounds)
    while it fits, one warp per sample beyond; both give the same lattices."""
    kw = dict(L=4096, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=3, p_thr=th(0.7), q_thr=th(0.2), seed=41)
    with A.asep_create(A.make_params(**kw), sample_times=[0, 9]) as ctx:
        info = A.asep_get_info(ctx)
        assert (info["cluster"], info["threads"], info["groups"]) == (1, 1024, 3)
        A.asep_sweep(ctx, 9)
        rounds, _ = A.asep_state(ctx)
        A.asep_reset(ctx, seed=41)
        A.asep_set_plan(ctx, 2, 0)
        assert A.asep_get_info(ctx)["cluster"] == 2
        A.asep_sweep(ctx, 9)
        warp, _ = A.asep_state(ctx)
        assert np.array_equal(rounds, warp)
        with pytest.raises(A.AsepError):
            A.asep_set_plan(ctx, 1, 4)  # samples_per_group is not a serial knob
        with pytest.raises(A.AsepError):
            A.asep_set_plan(ctx, 3, 0)
    with A.asep_create(A.make_params(L=1 << 21, schedule=A.ASEP_SCHED_SERIAL), sample_times=[]) as ctx:
        assert A.asep_get_info(ctx)["cluster"] == 2  # 2^21 attempts per sweep: one warp per sample
        with pytest.raises(A.AsepError):
            A.asep_set_plan(ctx, 1, 0)
        assert A.asep_get_info(ctx)["cluster"] == 2


def test_streamed_tier_is_chosen_beyond_a_cluster():
    with A.asep_create(A.make_params(L=1 << 24, domain_sites=256, samples_per_real=1), sample_times=[]) as ctx:
        info = A.asep_get_info(ctx)
        assert info["cluster"] == 32 and info["groups"] >= 2
    with A.asep_create(A.make_params(L=1 << 16, domain_sites=256, samples_per_real=2), sample_times=[]) as ctx:
        with A.asep_batch_create(max_jobs=2, max_items=64) as b:
            A.asep_set_plan(ctx, 32, 0)
            with pytest.raises(A.AsepError):
                A.asep_batch_sweep(b, [ctx], [1])  # streamed contexts are swept with asep_sweep
