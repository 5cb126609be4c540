"""Pins of the oracle's dynamics against exact enumeration and closed forms.

* Distributional: the replayed schedules (serial RSU on the Philox stream,
  the two-phase Poisson-domain schedule, the two-lane model) and the
  independent serial reference are compared state by state, by a chi-square
  test, with the exact master-equation evolution of :mod:`oracle.exact`.
  Each test also checks that the same samples REJECT a plausible mistake
  (wrong rate placement, wrong direction, fixed attempt counts ...), so the
  pin has power.
* Closed forms: uniform stationary measure of RSU, <W^2> = (L+1)/12 on the
  half-filled ring, current (p-q) N (L-N) / (L (L-1)) per bond and sweep.
* Conservation of particle number, and the paper's growth exponent
  beta = alpha / z = 1/3 (sec. 2.2).
"""
import json
import os

import numpy as np
import pytest
from scipy import stats
from scipy.linalg import expm

from oracle import exact as ex

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def chi2_pvalue(counts: np.ndarray, probs: np.ndarray, min_expected: float = 5.0) -> float:
    expected = probs * counts.sum()
    order = np.argsort(expected)
    obs_b, exp_b = [], []
    acc_o = acc_e = 0.0
    for k in order:
        acc_o += counts[k]
        acc_e += expected[k]
        if acc_e >= min_expected:
            obs_b.append(acc_o)
            exp_b.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0:
        obs_b[-1] += acc_o
        exp_b[-1] += acc_e
    obs_b, exp_b = np.array(obs_b), np.array(exp_b)
    stat = float(((obs_b - exp_b) ** 2 / exp_b).sum())
    return float(stats.chi2.sf(stat, len(obs_b) - 1))


def histogram(space: ex.Space, state: np.ndarray) -> np.ndarray:
    L = space.L
    mask = (1 << L) - 1
    counts = np.zeros(space.n)
    for s in range(state.shape[0]):
        x = int(state[s, 0, 0]) & mask
        if space.lanes == 2:
            x |= (int(state[s, 1, 0]) & mask) << L
        counts[space.index[x]] += 1
    return counts


S_DIST = 20000


def _replay_hist(oracle_mod, P, t, mask=None):
    st = oracle_mod.init_state(P)
    m = oracle_mod.disorder(P) if mask is None else mask
    oracle_mod.replay(P, st, 0, t, mask=m)
    return st


# ---------------------------------------------------------------------------
# Closed forms via the enumerator
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", [4, 6, 8, 10])
def test_rsu_stationary_uniform_width_and_current(L):
    p, q = 0.75, 0.25
    N = L // 2
    m = ex.RingModel(L, N, p, q)
    pi = ex.stationary(m.rsu_sweep())
    assert np.max(np.abs(pi - 1.0 / m.sp.n)) < 1e-12
    # uniform half-filled ring: E[W^2] = (L+1)/12 (random-walk bridge)
    assert abs(pi @ m.sp.w2() - (L + 1) / 12) < 1e-12
    # current per bond per sweep: L attempts x (1/L) x (p-q) P(10 at a bond)
    j = pi @ m.current_per_attempt_vector(p, q) / L
    assert abs(j - (p - q) * N * (L - N) / (L * (L - 1))) < 1e-12


# ---------------------------------------------------------------------------
# Ring: serial replay, domain replay and serial reference vs exact evolution
# ---------------------------------------------------------------------------

def test_serial_replay_matches_exact_rsu(oracle_mod):
    L, p, q = 8, 0.75, 0.25
    P = oracle_mod.Params(L=L, schedule=oracle_mod.SCHED_SERIAL, samples_per_real=S_DIST, seed=11,
                          p_thr=oracle_mod.threshold(p), q_thr=oracle_mod.threshold(q))
    m = ex.RingModel(L, L // 2, p, q)
    for t in (1, 3):
        st = _replay_hist(oracle_mod, P, t)
        counts = histogram(m.sp, st)
        exact = m.sp.flat_alt() @ np.linalg.matrix_power(m.rsu_sweep(), t)
        assert chi2_pvalue(counts, exact) > 1e-4, t
        wrong = m.sp.flat_alt() @ np.linalg.matrix_power(ex.RingModel(L, L // 2, q, p).rsu_sweep(), t)
        assert chi2_pvalue(counts, wrong) < 1e-6


@pytest.mark.parametrize("D", [1, 2, 4])
def test_domain_replay_matches_exact_domain_schedule(oracle_mod, D):
    L, p, q = 8, 0.75, 0.25
    P = oracle_mod.Params(L=L, D=D, samples_per_real=S_DIST, seed=3 + D, p_thr=oracle_mod.threshold(p),
                          q_thr=oracle_mod.threshold(q))
    m = ex.RingModel(L, L // 2, p, q)
    A = m.domain_sweep(D)
    for t in (1, 2):
        counts = histogram(m.sp, _replay_hist(oracle_mod, P, t))
        exact = m.sp.flat_alt() @ np.linalg.matrix_power(A, t)
        assert chi2_pvalue(counts, exact) > 1e-4, (D, t)
    # power: the same samples reject D fixed attempts per domain (no Poisson count)
    if D >= 2:
        I = np.eye(m.sp.n)
        fixed = np.zeros_like(I)
        for o in range(2 * D):
            B = I
            for phase in (0, 1):
                for g in range(L // (2 * D)):
                    base = o + 2 * D * g + phase * D
                    M = sum(m.K[(base + j) % L] for j in range(D)) / D
                    B = B @ np.linalg.matrix_power(M, D)
            fixed += B
        fixed /= 2 * D
        wrong = m.sp.flat_alt() @ np.linalg.matrix_power(fixed, 2)
        assert chi2_pvalue(counts, wrong) < 1e-6


def test_domain_replay_disorder_rate_placement(oracle_mod):
    """Right hops across (i, i+1) use p_i, left hops use q_{i+1} (paper
    sec. 2.1); the slow class of Eq. (bimodal) replaces both at a site."""
    L, D = 8, 2
    pf, ps, qf, qs = 0.9, 0.3, 0.4, 0.1
    th = oracle_mod.threshold
    P = oracle_mod.Params(L=L, D=D, samples_per_real=S_DIST, seed=21, p_thr=th(pf), q_thr=th(qf),
                          dis_kind=oracle_mod.DIS_BIMODAL, dis_a_thr=th(0.5), dis_b_thr=th(ps), dis_c_thr=th(qs),
                          dis_seed=5)
    mask = oracle_mod.disorder(P)
    slow = [(int(mask[0, 0]) >> i) & 1 for i in range(L)]
    assert 0 < sum(slow) < L
    pvec = [ps if c else pf for c in slow]
    qvec = [qs if c else qf for c in slow]
    m = ex.RingModel(L, L // 2, pvec, qvec)
    counts = histogram(m.sp, _replay_hist(oracle_mod, P, 2, mask=mask))
    exact = m.sp.flat_alt() @ np.linalg.matrix_power(m.domain_sweep(D), 2)
    assert chi2_pvalue(counts, exact) > 1e-4
    # plausible mistake: left hop out of site i+1 using q_i instead of q_{i+1}
    q_shift = [qvec[(i - 1) % L] for i in range(L)]
    wrong_m = ex.RingModel(L, L // 2, pvec, q_shift)
    wrong = m.sp.flat_alt() @ np.linalg.matrix_power(wrong_m.domain_sweep(D), 2)
    assert chi2_pvalue(counts, wrong) < 1e-6


def test_serial_reference_matches_exact_rsu(oracle_mod):
    L, p, q = 8, 0.6, 0.1
    P = oracle_mod.Params(L=L, schedule=oracle_mod.SCHED_SERIAL, samples_per_real=S_DIST,
                          p_thr=oracle_mod.threshold(p), q_thr=oracle_mod.threshold(q))
    m = ex.RingModel(L, L // 2, p, q)
    st = oracle_mod.init_state(P)
    oracle_mod.serial_reference(P, st, 2, rng_seeds=np.arange(S_DIST) + 1000)
    counts = histogram(m.sp, st)
    exact = m.sp.flat_alt() @ np.linalg.matrix_power(m.rsu_sweep(), 2)
    assert chi2_pvalue(counts, exact) > 1e-4
    wrong = m.sp.flat_alt() @ expm(2 * 0.5 * m.generator())  # half the time
    assert chi2_pvalue(counts, wrong) < 1e-10


# ---------------------------------------------------------------------------
# Two lanes
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("schedule", ["domain", "serial"])
def test_two_lane_replay_matches_exact(oracle_mod, schedule):
    L, D, omega = 4, 1, 0.5
    th = oracle_mod.threshold
    P = oracle_mod.Params(model=oracle_mod.MODEL_TWO_LANE, L=L, D=D, samples_per_real=S_DIST, seed=31,
                          schedule=oracle_mod.SCHED_DOMAIN if schedule == "domain" else oracle_mod.SCHED_SERIAL,
                          p_thr=oracle_mod.ALWAYS, q_thr=oracle_mod.ALWAYS, dis_kind=oracle_mod.DIS_TURNING,
                          dis_a_thr=th(0.5), dis_b_thr=th(omega), dis_seed=2)
    mask = oracle_mod.disorder(P)
    turning = [i for i in range(L) if (int(mask[0, 0]) >> i) & 1]
    assert 0 < len(turning) < L
    m = ex.TwoLaneModel(L, L, 1.0, 1.0, turning, omega)
    A = m.domain_sweep(D) if schedule == "domain" else m.rsu_sweep()
    st = _replay_hist(oracle_mod, P, 2, mask=mask)
    counts = histogram(m.sp, st)
    exact = m.sp.flat_alt() @ np.linalg.matrix_power(A, 2)
    assert chi2_pvalue(counts, exact) > 1e-4
    # plausible mistake: lane B moving right like lane A
    wrong_m = ex.TwoLaneModel(L, L, 1.0, 1.0, turning, omega)
    wrong_m.KB = [m.sp.bond_kernel(1, b, 1.0, 0.0) for b in range(L)]
    W = wrong_m.domain_sweep(D) if schedule == "domain" else wrong_m.rsu_sweep()
    assert chi2_pvalue(counts, m.sp.flat_alt() @ np.linalg.matrix_power(W, 2)) < 1e-6


# ---------------------------------------------------------------------------
# Conservation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("model,schedule,dis", [
    (0, 0, 0), (0, 1, 0), (0, 0, 1), (1, 0, 2), (1, 1, 2), (0, 2, 0), (0, 2, 1), (1, 2, 2), (1, 2, 0), (1, 2, 4),
    (1, 1, 4), (0, 0, 3), (1, 0, 4)])
def test_particle_number_conserved(oracle_mod, model, schedule, dis):
    th = oracle_mod.threshold
    P = oracle_mod.Params(model=model, schedule=schedule, L=1024, D=64, samples_per_real=3, seed=9,
                          init_kind=oracle_mod.INIT_BERNOULLI_HALF, init_seed=4,
                          p_thr=th(0.7) if model == 0 else oracle_mod.ALWAYS,
                          q_thr=th(0.2) if model == 0 else oracle_mod.ALWAYS,
                          dis_kind=dis, dis_a_thr=th(0.1 if dis == 1 else 0.05), dis_b_thr=th(0.3 if dis == 1 else 0.1),
                          dis_c_thr=th(0.05), dis_seed=8)
    st = oracle_mod.init_state(P)
    n0 = [[int(np.unpackbits(st[s, pl].view(np.uint8)).sum()) for pl in range(P.planes)] for s in range(P.S)]
    cnt = oracle_mod.replay(P, st, 0, 20, mask=oracle_mod.disorder(P))
    n1 = [[int(np.unpackbits(st[s, pl].view(np.uint8)).sum()) for pl in range(P.planes)] for s in range(P.S)]
    for s in range(P.S):
        if model == 0:
            assert n0[s] == n1[s]
            assert cnt[s, 0] + cnt[s, 1] > 0
        else:
            assert sum(n0[s]) == sum(n1[s])
            # lane A loses A->B turns and gains B->A turns
            assert n1[s][0] - n0[s][0] == int(cnt[s, 3]) - int(cnt[s, 2])


# ---------------------------------------------------------------------------
# Long runs: stationary width, current, growth exponent
# ---------------------------------------------------------------------------

def test_serial_reference_stationary_width_and_current(oracle_mod):
    L, p, q, S = 64, 0.75, 0.25, 64
    P = oracle_mod.Params(L=L, samples_per_real=S, p_thr=oracle_mod.threshold(p), q_thr=oracle_mod.threshold(q))
    st = oracle_mod.init_state(P)
    oracle_mod.serial_reference(P, st, 3000, rng_seeds=np.arange(S) + 77)  # burn-in past saturation
    w2 = np.zeros(S)
    n_meas, gap = 40, 50
    cnt_tot = np.zeros((S, 4), dtype=np.uint64)
    for k in range(n_meas):
        cnt_tot += oracle_mod.serial_reference(P, st, gap, rng_seeds=np.arange(S) * 1000 + k + 5)
        for s in range(S):
            w2[s] += oracle_mod.width2(L, *oracle_mod.heights(st[s, 0], L)) / n_meas
    sem = w2.std(ddof=1) / np.sqrt(S)
    assert abs(w2.mean() - (L + 1) / 12) < 4 * sem
    j = (cnt_tot[:, 0].astype(float) - cnt_tot[:, 1].astype(float)) / (L * n_meas * gap)
    jexp = (p - q) * (L // 2) * (L // 2) / (L * (L - 1))
    assert abs(j.mean() - jexp) < 4 * j.std(ddof=1) / np.sqrt(S)


def _growth_slope(times, w2):
    x = np.log(np.array(times, dtype=float))
    y = np.log(np.array(w2) - 0.25)  # paper sec. 2.2 subtracts W^2(0) = 0.25
    return float(np.polyfit(x, y, 1)[0])


def _w2_at(oracle_mod, P, times, serial_ref: bool):
    if not serial_ref:
        r = oracle_mod.run(P, times[-1], times)
        return r.w2[:, :, 0].mean(axis=1), r.w2[:, :, 0]
    st = oracle_mod.init_state(P)
    out = np.zeros((len(times), P.S))
    done = 0
    for i, t in enumerate(times):
        oracle_mod.serial_reference(P, st, t - done, rng_seeds=np.arange(P.S) * 7919 + t)
        done = t
        for s in range(P.S):
            out[i, s] = oracle_mod.width2(P.L, *oracle_mod.heights(st[s, 0], P.L))
    return out.mean(axis=1), out


def test_growth_exponent_beta_one_third(oracle_mod):
    with open(GOLDEN) as f:
        g = json.load(f)["kpz_exponents"]
    beta = g["alpha"] / g["z"]
    times = [16, 32, 64, 128, 256]
    P = oracle_mod.Params(L=4096, D=256, samples_per_real=24, seed=99)
    for serial_ref in (True, False):
        mean, _ = _w2_at(oracle_mod, P, times, serial_ref)
        slope = _growth_slope(times, mean)
        assert abs(slope - 2 * beta) < 0.07, (serial_ref, slope)


def test_domain_schedule_width_within_3sigma_of_serial_reference(oracle_mod):
    """W(t) of the D = 256 domain schedule vs the independent serial RSU."""
    times = [8, 32, 128]
    for p, q in [(1.0, 0.0), (0.75, 0.25)]:
        P = oracle_mod.Params(L=4096, D=256, samples_per_real=48, seed=123,
                              p_thr=oracle_mod.threshold(p), q_thr=oracle_mod.threshold(q))
        m_dom, all_dom = _w2_at(oracle_mod, P, times, False)
        m_ser, all_ser = _w2_at(oracle_mod, P, times, True)
        for i in range(len(times)):
            sig = np.sqrt(all_dom[i].var(ddof=1) / P.S + all_ser[i].var(ddof=1) / P.S)
            assert abs(m_dom[i] - m_ser[i]) < 3 * sig, (p, times[i], m_dom[i], m_ser[i], sig)


# ---------------------------------------------------------------------------
# Absolute height: hops across the seam bond (L-1, 0)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("schedule", [0, 1])
def test_seam_counter_closes_the_height_balance(oracle_mod, schedule):
    """A right hop across bond (i, i+1) lowers h_i by 2 and leaves every other
    h_k of the open prefix sum unchanged, except across the seam (L-1, 0),
    where it raises h_0 ... h_{L-2} by 2.  Hence, exactly,
    sum h(t) - sum h(0) = -2 (R - Lh) + 2 L (R_seam - Lh_seam): the seam
    counter is pinned by the recorded heights and total hop counters."""
    th = oracle_mod.threshold
    P = oracle_mod.Params(L=256, D=32, schedule=schedule, samples_per_real=6, p_thr=th(0.7), q_thr=th(0.4), seed=5)
    times = [0, 3, 10, 40]
    r = oracle_mod.run(P, 40, times)
    seam_moves = 0
    for ti in range(len(times)):
        for s in range(P.S):
            dsum = int(r.sum_h[ti, s, 0]) - int(r.sum_h[0, s, 0])
            R, Lh = r.extra["counters_at"][ti, s, :2]
            h_off = int(r.extra["height_offset"][ti, s])
            assert dsum == -2 * int(R - Lh) - P.L * h_off, (ti, s)
            seam_moves += abs(h_off)
    assert seam_moves > 0  # the seam was crossed in both directions over the run


def test_seam_current_equals_exact_rsu_current(oracle_mod):
    """Stationary net hops across the seam per sweep (serial RSU replay) equal
    the exact ring current (p - q) N (L - N) / (L (L - 1)) of the uniform
    measure; the column height there falls at twice that rate."""
    L, p, q, S = 64, 0.75, 0.25, 64
    th = oracle_mod.threshold
    P = oracle_mod.Params(L=L, schedule=1, samples_per_real=S, p_thr=th(p), q_thr=th(q), seed=11)
    st = oracle_mod.init_state(P)
    oracle_mod.replay(P, st, 0, 1500)  # burn-in past saturation (L^(3/2) = 512 sweeps)
    seam = np.zeros((S, 2), dtype=np.uint64)
    T = 3000
    oracle_mod.replay(P, st, 1500, T, seam=seam)
    j = (seam[:, 0].astype(float) - seam[:, 1].astype(float)) / T
    jexp = (p - q) * (L // 2) * (L // 2) / (L * (L - 1))
    assert abs(j.mean() - jexp) < 4 * j.std(ddof=1) / np.sqrt(S)
    # a seam counted at the wrong bond (0, 1) still sees the same mean current,
    # but the balance test above fails for it; here check the sign convention
    assert j.mean() > 0.5 * jexp


# ---------------------------------------------------------------------------
# The paper's two-sub-lattice SCA schedule (sec. 2.1)
# ---------------------------------------------------------------------------

def test_sca_replay_matches_exact_sca(oracle_mod):
    L, p, q = 8, 0.75, 0.25
    P = oracle_mod.Params(L=L, schedule=oracle_mod.SCHED_SCA, samples_per_real=S_DIST, seed=41,
                          p_thr=oracle_mod.threshold(p), q_thr=oracle_mod.threshold(q))
    m = ex.RingModel(L, L // 2, p, q)
    A = m.sca_sweep()
    E, O = m.I, m.I
    for b in range(0, L, 2):
        E = E @ m.K[b]
    for b in range(1, L, 2):
        O = O @ m.K[b]
    assert np.allclose(E @ O, A)
    for t in (1, 2, 3):
        counts = histogram(m.sp, _replay_hist(oracle_mod, P, t))
        exact = m.sp.flat_alt() @ np.linalg.matrix_power(A, t)
        assert chi2_pvalue(counts, exact) > 1e-4, t
        # plausible mistakes: odd bonds first; random-sequential instead of SCA; swapped rates
        for wrong_op in (O @ E, m.rsu_sweep(), ex.RingModel(L, L // 2, q, p).sca_sweep()):
            wrong = m.sp.flat_alt() @ np.linalg.matrix_power(wrong_op, t)
            assert chi2_pvalue(counts, wrong) < 1e-6, t


def test_sca_disorder_rate_placement(oracle_mod):
    """SCA with bimodal site classes: right hops across (i, i+1) use p_i, left
    hops q_{i+1} (paper sec. 2.1), exactly as in the other schedules."""
    L = 8
    pf, ps, qf, qs = 0.9, 0.3, 0.4, 0.1
    th = oracle_mod.threshold
    P = oracle_mod.Params(L=L, schedule=oracle_mod.SCHED_SCA, samples_per_real=S_DIST, seed=23, p_thr=th(pf),
                          q_thr=th(qf), dis_kind=oracle_mod.DIS_BIMODAL, dis_a_thr=th(0.5), dis_b_thr=th(ps),
                          dis_c_thr=th(qs), dis_seed=5)
    mask = oracle_mod.disorder(P)
    slow = [(int(mask[0, 0]) >> i) & 1 for i in range(L)]
    assert 0 < sum(slow) < L
    pvec = [ps if c else pf for c in slow]
    qvec = [qs if c else qf for c in slow]
    m = ex.RingModel(L, L // 2, pvec, qvec)
    counts = histogram(m.sp, _replay_hist(oracle_mod, P, 2, mask=mask))
    assert chi2_pvalue(counts, m.sp.flat_alt() @ np.linalg.matrix_power(m.sca_sweep(), 2)) > 1e-4
    q_shift = [qvec[(i - 1) % L] for i in range(L)]
    wrong = ex.RingModel(L, L // 2, pvec, q_shift).sca_sweep()
    assert chi2_pvalue(counts, m.sp.flat_alt() @ np.linalg.matrix_power(wrong, 2)) < 1e-6


def test_independent_pq_class_draws(oracle_mod):
    """Independent p and q classes (the paper tags reduced forward and
    backward rates with separate bits, both with the distribution of Eq.
    bimodal): plane 0 is the one-class draw itself, plane 1 has the same
    frequency Q and is uncorrelated with plane 0."""
    th = oracle_mod.threshold
    L, Q = 1 << 16, 0.3
    kw = dict(L=L, schedule=oracle_mod.SCHED_SCA, n_realizations=2, samples_per_real=1, dis_a_thr=th(Q),
              dis_b_thr=th(0.1), dis_c_thr=th(0.2), dis_seed=17)
    one = oracle_mod.disorder(oracle_mod.Params(dis_kind=oracle_mod.DIS_BIMODAL, **kw))
    two = oracle_mod.disorder(oracle_mod.Params(dis_kind=oracle_mod.DIS_BIMODAL_PQ, **kw))
    W = L // 32
    assert two.shape == (2, 2 * W)
    assert np.array_equal(two[:, :W], one)
    bits = np.unpackbits(two.view(np.uint8), bitorder="little").reshape(2, 2, L).astype(np.float64)
    n = 2 * L
    for pl in range(2):
        f = bits[:, pl].mean()
        assert abs(f - Q) < 5 * np.sqrt(Q * (1 - Q) / n), (pl, f)
    both = (bits[:, 0] * bits[:, 1]).mean()
    assert abs(both - Q * Q) < 5 * np.sqrt(Q * Q * (1 - Q * Q) / n), both
    assert not np.array_equal(two[:, :W], two[:, W:])


@pytest.mark.parametrize("schedule", ["sca", "serial", "domain"])
def test_independent_pq_classes_rate_placement(oracle_mod, schedule):
    """Independent classes: right hops across (i, i+1) use p_i from the p
    plane, left hops q_{i+1} from the q plane.  Chi-square against the exact
    operator; rejected: the one-class reading (q classes from the p plane)
    and left hops keyed by the departure site's predecessor."""
    L = 8
    pf, ps, qf, qs = 0.9, 0.2, 0.7, 0.1
    th = oracle_mod.threshold
    sched = {"sca": oracle_mod.SCHED_SCA, "serial": oracle_mod.SCHED_SERIAL, "domain": oracle_mod.SCHED_DOMAIN}[schedule]
    P = oracle_mod.Params(L=L, D=2, schedule=sched, samples_per_real=S_DIST, seed=29, p_thr=th(pf), q_thr=th(qf),
                          dis_kind=oracle_mod.DIS_BIMODAL_PQ, dis_a_thr=th(0.5), dis_b_thr=th(ps),
                          dis_c_thr=th(qs), dis_seed=11)
    mask = oracle_mod.disorder(P)
    pslow = [(int(mask[0, 0]) >> i) & 1 for i in range(L)]
    qslow = [(int(mask[0, 1]) >> i) & 1 for i in range(L)]
    assert pslow != qslow and 0 < sum(pslow) < L and 0 < sum(qslow) < L
    pvec = [ps if c else pf for c in pslow]
    qvec = [qs if c else qf for c in qslow]

    def op(pv, qv):
        m = ex.RingModel(L, L // 2, pv, qv)
        return {"sca": m.sca_sweep, "serial": m.rsu_sweep, "domain": lambda: m.domain_sweep(2)}[schedule]()

    sp = ex.RingModel(L, L // 2, pf, qf).sp
    counts = histogram(sp, _replay_hist(oracle_mod, P, 2, mask=mask))
    assert chi2_pvalue(counts, sp.flat_alt() @ np.linalg.matrix_power(op(pvec, qvec), 2)) > 1e-4
    one_class = [qs if c else qf for c in pslow]
    q_shift = [qvec[(i - 1) % L] for i in range(L)]
    for wrong_q in (one_class, q_shift):
        wrong = sp.flat_alt() @ np.linalg.matrix_power(op(pvec, wrong_q), 2)
        assert chi2_pvalue(counts, wrong) < 1e-6


def test_sca_deterministic_tasep_moves_every_particle_twice(oracle_mod):
    """p = 1, q = 0 from the flat 1010... state (site 0 occupied): the even
    bonds all carry 10 and hop, giving 0101...; the odd bonds, the closing
    bond (L-1, 0) among them, then all carry 10 and hop back.  So after every
    sweep the lattice is flat again, L hops happened, one of them across the
    seam, and the seam column sank by 2 -- for any L, random words and seed."""
    for L, seed in [(64, 1), (1000, 7), (4096, 123)]:
        P = oracle_mod.Params(L=L, schedule=oracle_mod.SCHED_SCA, samples_per_real=2, seed=seed,
                              p_thr=oracle_mod.ALWAYS, q_thr=0)
        r = oracle_mod.run(P, 5, [0, 1, 5])
        flat = oracle_mod.init_state(P)
        assert np.array_equal(r.state, flat)
        assert np.all(r.extra["counters_at"][:, :, 0] == np.array([0, L, 5 * L])[:, None])
        assert np.all(r.extra["counters_at"][:, :, 1] == 0)
        assert np.all(r.extra["height_offset"] == np.array([0, -2, -10])[:, None])


def test_sca_stationary_current_and_width(oracle_mod):
    """Exact enumeration: the SCA's stationary current per bond per sweep and
    width, compared with the replay over a long run (L = 10)."""
    L, p, q, S = 10, 0.75, 0.25, 400
    m = ex.RingModel(L, L // 2, p, q)
    pi = ex.stationary(m.sca_sweep())
    w2_exact = pi @ m.sp.w2()
    th = oracle_mod.threshold
    P = oracle_mod.Params(L=L, schedule=oracle_mod.SCHED_SCA, samples_per_real=S, seed=5, p_thr=th(p), q_thr=th(q))
    st = oracle_mod.init_state(P)
    oracle_mod.replay(P, st, 0, 200)
    w2 = np.zeros(S)
    cnt = np.zeros((S, 4), dtype=np.uint64)
    n_meas = 50
    for k in range(n_meas):
        cnt += oracle_mod.replay(P, st, 200 + 10 * k, 10)
        w2 += np.array([oracle_mod.width2(L, *oracle_mod.heights(st[s, 0], L)) for s in range(S)]) / n_meas
    assert abs(w2.mean() - w2_exact) < 4 * w2.std(ddof=1) / np.sqrt(S)
    # current per bond per sweep from the exact measure: each bond is attempted once per sweep,
    # so J = sum over states of pi(x) * (net hops in one sweep from x) / L
    n_st = m.sp.n
    A = m.sca_sweep()
    # expected net right hops of one sweep: even phase from x, odd phase from the even phase's result
    E = m.I
    for b in range(0, L, 2):
        E = E @ m.K[b]
    cur = m.current_per_attempt_vector(p, q)  # per state: sum over all bonds of p [10] - q [01]
    even_bonds = np.zeros(n_st)
    odd_bonds = np.zeros(n_st)
    for k, x in enumerate(m.sp.states):
        for b in range(L):
            a, c = m.sp.bit(x, 0, b), m.sp.bit(x, 0, b + 1)
            v = p if (a, c) == (1, 0) else (-q if (a, c) == (0, 1) else 0.0)
            (even_bonds if b % 2 == 0 else odd_bonds)[k] += v
    assert np.allclose(even_bonds + odd_bonds, cur)
    j_exact = (pi @ even_bonds + (pi @ E) @ odd_bonds) / L
    j = (cnt[:, 0].astype(float) - cnt[:, 1].astype(float)) / (L * 10 * n_meas)
    assert abs(j.mean() - j_exact) < 4 * j.std(ddof=1) / np.sqrt(S)
    assert abs(A.sum(axis=1) - 1).max() < 1e-12


def test_two_lane_sca_replay_matches_exact(oracle_mod):
    """The paper's two-lane SCA (sec. 3): even bonds of both lanes, A -> B
    lane changes, odd bonds, B -> A lane changes; in-lane rates 0.5 as in the
    paper's SCA runs, lane changes at turning sites."""
    L, omega, p = 4, 0.5, 0.5
    th = oracle_mod.threshold
    P = oracle_mod.Params(model=oracle_mod.MODEL_TWO_LANE, L=L, schedule=oracle_mod.SCHED_SCA,
                          samples_per_real=S_DIST, seed=37, p_thr=th(p), q_thr=th(p),
                          dis_kind=oracle_mod.DIS_TURNING, dis_a_thr=th(0.5), dis_b_thr=th(omega), dis_seed=2)
    mask = oracle_mod.disorder(P)
    turning = [i for i in range(L) if (int(mask[0, 0]) >> i) & 1]
    assert 0 < len(turning) < L
    m = ex.TwoLaneModel(L, L, p, p, turning, omega)
    A = m.sca_sweep()
    for t in (1, 2):
        counts = histogram(m.sp, _replay_hist(oracle_mod, P, t, mask=mask))
        assert chi2_pvalue(counts, m.sp.flat_alt() @ np.linalg.matrix_power(A, t)) > 1e-4, t
    # plausible mistakes: lane changes in both directions once per sweep (the RSU pass), B -> A first,
    # lane B moving right
    E, O = m.I, m.I
    for b in range(0, L, 2):
        E = E @ m.KA[b] @ m.KB[b]
    for b in range(1, L, 2):
        O = O @ m.KA[b] @ m.KB[b]
    KBr = [m.sp.bond_kernel(1, b, p, 0.0) for b in range(L)]
    Er, Or = m.I, m.I
    for b in range(0, L, 2):
        Er = Er @ m.KA[b] @ KBr[b]
    for b in range(1, L, 2):
        Or = Or @ m.KA[b] @ KBr[b]
    for wrong in (E @ O @ m.T, E @ m.TBA @ O @ m.TAB, Er @ m.TAB @ Or @ m.TBA):
        assert chi2_pvalue(counts, m.sp.flat_alt() @ np.linalg.matrix_power(wrong, 2)) < 1e-6


@pytest.mark.parametrize("schedule", ["sca", "serial", "domain"])
def test_two_lane_crossing_classes_match_exact(oracle_mod, schedule):
    """The paper's two-lane crossing (sec. 3): every site may cross, A -> B
    with u_i and B -> A with v_i, each 0.8 unless the site is marked (0.2) in
    its own class plane.  Chi-square against the exact operator; rejected:
    u and v swapped, and the u plane used for both directions."""
    L, p = 4, 0.5
    th = oracle_mod.threshold
    uf, us = 0.8, 0.2
    sched = {"sca": oracle_mod.SCHED_SCA, "serial": oracle_mod.SCHED_SERIAL, "domain": oracle_mod.SCHED_DOMAIN}[schedule]
    P = oracle_mod.Params(model=oracle_mod.MODEL_TWO_LANE, L=L, D=1, schedule=sched, samples_per_real=S_DIST, seed=41,
                          p_thr=th(p), q_thr=th(p), dis_kind=oracle_mod.DIS_CROSSING, dis_a_thr=th(0.5),
                          dis_b_thr=th(uf), dis_c_thr=th(us), dis_seed=5)
    mask = oracle_mod.disorder(P)
    assert mask.shape == (1, 2)
    mu = [(int(mask[0, 0]) >> i) & 1 for i in range(L)]
    mv = [(int(mask[0, 1]) >> i) & 1 for i in range(L)]
    assert mu != mv
    u = {i: us if mu[i] else uf for i in range(L)}
    v = {i: us if mv[i] else uf for i in range(L)}

    def op(uu, vv):
        m = ex.TwoLaneModel(L, L, p, p, range(L), uu, vv)
        return {"sca": m.sca_sweep, "serial": m.rsu_sweep, "domain": lambda: m.domain_sweep(1)}[schedule](), m.sp

    A, sp = op(u, v)
    counts = histogram(sp, _replay_hist(oracle_mod, P, 2, mask=mask))
    assert chi2_pvalue(counts, sp.flat_alt() @ np.linalg.matrix_power(A, 2)) > 1e-4
    for uu, vv in ((v, u), (u, u)):
        wrong, _ = op(uu, vv)
        assert chi2_pvalue(counts, sp.flat_alt() @ np.linalg.matrix_power(wrong, 2)) < 1e-6


def test_two_lane_sca_deterministic_counts(oracle_mod):
    """Rate 1 in both lanes, no lane changes, flat 1010... start.  Lane A
    (right hops) is flat again after every sweep, L hops each.  Lane B (left
    hops, 01 -> 10): its even bonds carry 10 at first, so only the odd bonds
    hop in sweep 1 (L/2 hops, leaving 0101...); from then on every bond of
    every phase carries 01 and hops (L per sweep), and after an odd number of
    sweeps lane B sits on the odd sites."""
    L = 256
    P = oracle_mod.Params(model=oracle_mod.MODEL_TWO_LANE, L=L, schedule=oracle_mod.SCHED_SCA, samples_per_real=2,
                          seed=3, p_thr=oracle_mod.ALWAYS, q_thr=oracle_mod.ALWAYS)
    r = oracle_mod.run(P, 3, [0, 1, 3])
    flat = oracle_mod.init_state(P)
    assert np.array_equal(r.state[:, 0], flat[:, 0])
    assert np.all(r.state[:, 1] == 0xAAAAAAAA)
    cur = r.extra["counters_at"]
    assert np.all(cur[:, :, 0] == np.array([0, L, 3 * L])[:, None])
    assert np.all(cur[:, :, 1] == np.array([0, L // 2, L // 2 + 2 * L])[:, None])
    assert np.all(cur[:, :, 2:] == 0)
