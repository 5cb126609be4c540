"""Randomised parity: configurations drawn from a fixed seed across every
schedule, model, disorder kind, size, rate class (0, "always", two-plane,
twenty-bit), initial state, observable flag and sample-time pattern, each
bit-exact against the oracle (lattices, every record of the height sums, the
hop counters at every record, profiles, overlaps and the seam height)."""
import numpy as np
import pytest

import oracle
from paper_1012_0385_gb300 import asep as A

pytestmark = pytest.mark.gpu

th = oracle.threshold
N_CASES = 144
RATES = [0, A.ASEP_ALWAYS, th(0.75), th(0.25), th(0.5), th(0.6), th(0.3), th(0.9)]


def draw(k: int):
    rng = np.random.default_rng(1000 + k)
    schedule = int(rng.choice([A.ASEP_SCHED_DOMAIN, A.ASEP_SCHED_DOMAIN, A.ASEP_SCHED_SCA, A.ASEP_SCHED_SERIAL]))
    model = int(rng.integers(2))
    if model == 1:  # none, turning sites, or the paper's crossing probabilities at every site
        dis = int(rng.choice([0, 2, 4]))
    else:  # none, one slow class, or independent p and q classes
        dis = int(rng.choice([0, 1, 3]))
    if schedule == A.ASEP_SCHED_SERIAL:
        L = int(2 ** rng.integers(6, 12))
        kw = dict(schedule=schedule)
    elif schedule == A.ASEP_SCHED_SCA:
        L = 256 * int(rng.integers(1, 24))
        kw = dict(schedule=schedule)
    else:
        D = int(2 ** rng.integers(5, 9))
        L = 2 * D * int(rng.integers(1, 40))
        kw = dict(domain_sites=D)
    n_real = int(rng.integers(1, 3)) if dis else 1
    spr = int(rng.integers(1, 6))
    p, q = (int(rng.choice(RATES)) for _ in range(2))
    if model == 1 and schedule == A.ASEP_SCHED_DOMAIN and rng.random() < 0.5:
        p = q = A.ASEP_ALWAYS  # the two-lane configuration's rate 1
    kw.update(model=model, L=L, n_realizations=n_real, samples_per_real=spr, p_thr=p, q_thr=q,
              seed=int(rng.integers(1, 2**40)), init_kind=int(rng.integers(2)), init_seed=int(rng.integers(1, 1000)))
    if dis in (1, 3):
        kw.update(dis_kind=dis, dis_a_thr=th(float(rng.choice([0.1, 0.5]))), dis_b_thr=int(rng.choice(RATES)),
                  dis_c_thr=int(rng.choice(RATES)), dis_seed=int(rng.integers(1, 1000)))
    elif dis in (2, 4):
        kw.update(dis_kind=dis, dis_a_thr=th(float(rng.choice([0.05, 0.3]))), dis_b_thr=th(float(rng.choice([0.1, 0.7]))),
                  dis_seed=int(rng.integers(1, 1000)), dis_c_thr=th(0.2))
    n = int(rng.integers(1, 25))
    times = sorted(set([0] * int(rng.integers(2)) + [int(x) for x in rng.integers(1, n + 1, size=int(rng.integers(1, 4)))]))
    flags = 0
    if model == 0 and rng.random() < 0.3:
        flags |= A.ASEP_FLAG_NO_HOP_COUNTS
    if rng.random() < 0.5:
        flags |= A.ASEP_FLAG_PROFILE
    if rng.random() < 0.5:
        flags |= A.ASEP_FLAG_AUTOCORR
        kw["autocorr_t0"] = int(rng.choice(times))
    kw["flags"] = flags
    chunks = [n] if rng.random() < 0.5 else [n // 2, n - n // 2]
    return kw, [c for c in chunks if c > 0], times


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_0385_gb300 import build

    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("k", range(N_CASES))
def test_random_configuration_bit_exact(k):
    from test_gpu_parity import assert_same, oracle_params, run_gpu

    kw, chunks, times = draw(k)
    g = run_gpu(kw, chunks, times)
    P = oracle_params(kw)
    t0 = kw.get("autocorr_t0") if kw["flags"] & A.ASEP_FLAG_AUTOCORR else None
    ref = oracle.run(P, sum(chunks), times, autocorr_t0=t0)
    if kw["flags"] & A.ASEP_FLAG_NO_HOP_COUNTS:
        ref.counters[:] = 0
        ref.extra["counters_at"][:] = 0
    if P.dis_kind != 0:
        assert np.array_equal(g["dis"], oracle.disorder(P))
    assert_same(g, ref, P, times)


def test_random_contexts_in_one_batch_bit_exact():
    """The domain-schedule draws, all in one persistent batch, advanced in
    uneven steps (contexts join late and finish early), each bit-exact
    against the oracle."""
    from test_gpu_parity import assert_same, oracle_params

    cases = [draw(k) for k in range(N_CASES)]
    cases = [c for c in cases if c[0].get("schedule", A.ASEP_SCHED_DOMAIN) == A.ASEP_SCHED_DOMAIN][:16]
    assert len(cases) >= 8
    ctxs = [A.asep_create(A.make_params(**kw), sample_times=times) for kw, _, times in cases]
    try:
        left = [sum(chunks) for _, chunks, _ in cases]
        rng = np.random.default_rng(7)
        with A.asep_batch_create(max_jobs=len(ctxs), max_items=1 << 16) as b:
            step = 0
            while any(left):
                active = [i for i in range(len(ctxs)) if left[i] and i <= 2 * step]
                q = [min(left[i], int(rng.integers(1, 9))) for i in active]
                A.asep_batch_sweep(b, [ctxs[i] for i in active], q)
                for i, k in zip(active, q):
                    left[i] -= k
                step += 1
        for (kw, chunks, times), c in zip(cases, ctxs):
            words, sweep = A.asep_state(c)
            sh, sh2, w2 = A.asep_width(c)
            g = dict(words=words, sh=sh, sh2=sh2, w2=w2, cnt=A.asep_counters(c), dis=A.asep_disorder(c),
                     cur=A.asep_currents(c), hoff=None,
                     prof=A.asep_profile(c) if kw["flags"] & A.ASEP_FLAG_PROFILE else None,
                     ac=A.asep_autocorr(c) if kw["flags"] & A.ASEP_FLAG_AUTOCORR else None)
            assert sweep == sum(chunks)
            P = oracle_params(kw)
            t0 = kw.get("autocorr_t0") if kw["flags"] & A.ASEP_FLAG_AUTOCORR else None
            ref = oracle.run(P, sum(chunks), times, autocorr_t0=t0)
            if kw["flags"] & A.ASEP_FLAG_NO_HOP_COUNTS:
                ref.counters[:] = 0
                ref.extra["counters_at"][:] = 0
            assert_same(g, ref, P, times)
    finally:
        for c in ctxs:
            c.close()


def draw_streamed(k: int):
    """A draw of the domain schedule on a lattice wide enough for the streamed
    tier (64 .. 300 columns, L a multiple of 128), other parameters as draw()."""
    kw, chunks, times = draw(k)
    rng = np.random.default_rng(5000 + k)
    D = int(rng.choice([32, 64, 128]))
    G = 2 * int(rng.integers(32, 151))
    kw = {x: v for x, v in kw.items() if x != "schedule"}
    if kw.get("dis_kind") == A.ASEP_DIS_BIMODAL_PQ:  # the domain schedule takes one class plane
        kw["dis_kind"] = A.ASEP_DIS_BIMODAL
    if kw.get("dis_kind") == A.ASEP_DIS_CROSSING:  # ... and turning sites, not crossing at every site
        kw["dis_kind"] = A.ASEP_DIS_TURNING
    kw.update(L=2 * D * G, domain_sites=D, samples_per_real=min(kw["samples_per_real"], 2))
    return kw, chunks, times


N_STREAMED = 24


@pytest.mark.parametrize("k", range(N_STREAMED))
def test_random_configuration_streamed_tier_bit_exact(k):
    """Draws forced onto the streamed tier (tiles through shared memory,
    boundary words merged atomically), bit-exact against the oracle."""
    from test_gpu_parity import assert_same, oracle_params, run_gpu

    kw, chunks, times = draw_streamed(k)
    kw = dict(kw, plan=(32, 0))
    g = run_gpu(kw, chunks, times)
    P = oracle_params(kw)
    t0 = kw.get("autocorr_t0") if kw["flags"] & A.ASEP_FLAG_AUTOCORR else None
    ref = oracle.run(P, sum(chunks), times, autocorr_t0=t0)
    if kw["flags"] & A.ASEP_FLAG_NO_HOP_COUNTS:
        ref.counters[:] = 0
        ref.extra["counters_at"][:] = 0
    assert_same(g, ref, P, times)


def draw_sca_streamed(k: int):
    """A draw moved onto the streamed SCA (L = 256 .. 256 * 40 in units of
    256, so the last block of threads is mostly idle), other parameters as
    draw()."""
    kw, chunks, times = draw(k)
    rng = np.random.default_rng(9000 + k)
    kw = dict(kw, schedule=A.ASEP_SCHED_SCA, L=256 * int(rng.integers(1, 41)), plan=(32, 0))
    kw.pop("domain_sites", None)
    return kw, chunks, times


N_SCA_STREAMED = 24


@pytest.mark.parametrize("k", range(N_SCA_STREAMED))
def test_random_configuration_streamed_sca_bit_exact(k):
    """Draws on the streamed SCA (lattice in global memory, a thread per
    unit, boundary words merged atomically), bit-exact against the oracle."""
    from test_gpu_parity import assert_same, oracle_params, run_gpu

    kw, chunks, times = draw_sca_streamed(k)
    g = run_gpu(kw, chunks, times)
    P = oracle_params(kw)
    t0 = kw.get("autocorr_t0") if kw["flags"] & A.ASEP_FLAG_AUTOCORR else None
    ref = oracle.run(P, sum(chunks), times, autocorr_t0=t0)
    if kw["flags"] & A.ASEP_FLAG_NO_HOP_COUNTS:
        ref.counters[:] = 0
        ref.extra["counters_at"][:] = 0
    assert_same(g, ref, P, times)
