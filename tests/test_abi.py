"""The C ABI without a GPU: the library builds, loads, exports every symbol
include/asep.h declares, and its host-only functions agree with the oracle
and with the paper's sampling schedule."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def A():
    from paper_1012_0385_gb300 import build

    if not build.up_to_date():
        build.build()
    from paper_1012_0385_gb300 import asep

    return asep


def _declared():
    src = open(os.path.join(ROOT, "include", "asep.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|uint32_t|const char\*)\s+(asep_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(A):
    import subprocess

    declared = _declared()
    assert len(declared) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", A._build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (asep_\w+)", out))
    assert set(declared) <= exported, set(declared) - exported
    assert set(declared) == set(A.EXPORTED)
    lib = A.lib()
    for name in declared:
        assert getattr(lib, name) is not None


def test_version_and_thresholds(A, oracle_mod):
    assert "sm_103a" in A.asep_version()
    for p in [0.0, -1.0, 1.0, 2.0, 0.75, 0.25, 0.1, 0.3, 0.05, 0.999999, 1e-7]:
        assert A.asep_threshold(p) == oracle_mod.threshold(p), p


@pytest.mark.parametrize("m", [1, 2, 3, 32, 64, 100, 256, 512, 1000, 1024, 2048, 4096])
def test_poisson_table_identical_to_exact_oracle(A, oracle_mod, m):
    k_lo, tab = A.asep_poisson_table(m)
    ok, ot = oracle_mod.poisson_table(m)
    assert k_lo == ok and np.array_equal(tab, np.array(ot, dtype=np.uint32))


def test_sampling_times_match_paper_and_oracle(oracle_mod):
    from paper_1012_0385_gb300.sampling import every, log_times

    assert log_times(10**7) == oracle_mod.log_times(10**7)
    assert len(log_times(10**7, include_zero=False)) == 261  # t_0 plus the paper's 260 events
    assert every(100, 10**4)[:3] == [0, 100, 200] and every(100, 10**4)[-1] == 10**4


def test_create_rejects_bad_params_without_device(A):
    """Validation happens before any CUDA call."""
    bad = [dict(L=100), dict(L=1 << 29), dict(L=4096, domain_sites=48), dict(L=4096, p_thr=123),
           dict(L=4096, n_realizations=0), dict(L=4096, dis_kind=2), dict(L=4096, model=1, dis_kind=1),
           dict(L=4096 + 64, schedule=1), dict(L=4096, samples_per_real=3, first_sample=1),
           # SCA schedule: L a multiple of 256 (beyond shared memory it streams, up to 2^28)
           dict(L=4096 + 64, schedule=2), dict(L=(1 << 21) + 128, schedule=2), dict(L=1 << 29, schedule=2),
           dict(L=4096, schedule=3),
           # independent p and q classes: the ring model only; no kind 5
           dict(L=4096, schedule=2, model=1, dis_kind=3, dis_a_thr=4096), dict(L=4096, model=1, dis_kind=3),
           dict(L=4096, schedule=2, dis_kind=5),
           # crossing probabilities: the two-lane model only
           dict(L=4096, schedule=2, dis_kind=4, dis_a_thr=4096), dict(L=4096, dis_kind=4, dis_a_thr=4096)]
    for kw in bad:
        prm = A.make_params(**kw)
        with pytest.raises(A.AsepError) as ei:
            A.asep_create(prm, torch_alloc=False, stream=0)
        assert ei.value.code == A.ASEP_ERR_INVALID, kw
        assert A.asep_last_error(None)
    # observable flags: unknown bits; an autocorrelation reference time that is not a sample time
    for kw, times in [(dict(L=4096, flags=8), [0, 5]),
                      (dict(L=4096, flags=A.ASEP_FLAG_AUTOCORR, autocorr_t0=3), [0, 5]),
                      (dict(L=4096, flags=A.ASEP_FLAG_AUTOCORR), [])]:
        with pytest.raises(A.AsepError) as ei:
            A.asep_create(A.make_params(**kw), sample_times=times, torch_alloc=False, stream=0)
        assert ei.value.code == A.ASEP_ERR_INVALID, kw
        assert "autocorr" in A.asep_last_error(None) or "flags" in A.asep_last_error(None), kw


@pytest.mark.parametrize("flags,dis", [(0, 0), (6, 0), (0, 1)])
def test_allocation_failure_frees_everything_without_device(A, flags, dis):
    """An allocator hook that fails one request makes asep_create return
    ASEP_ERR_NOMEM and hand every other allocation back through free_fn
    exactly once.  A serial-schedule context allocates before its first CUDA
    call, so the hook's fake addresses are never dereferenced."""
    th = A.asep_threshold
    extra = dict(n_realizations=2, samples_per_real=2, dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1),
                 dis_b_thr=th(0.3)) if dis else {}
    times = [0, 5]

    def attempt(fail_at):
        calls, live, freed = [0], {}, []

        def alloc(nbytes, user):
            k = calls[0]
            calls[0] += 1
            if k == fail_at:
                return None
            ptr = 0x10000 * (k + 1)
            live[ptr] = nbytes
            return ptr

        def free(ptr, nbytes, user):
            freed.append((ptr, nbytes))

        prm = A.make_params(L=1024, schedule=A.ASEP_SCHED_SERIAL, flags=flags, autocorr_t0=5, **extra)
        prm.alloc, prm.free_fn = A.ALLOC_FN(alloc), A.FREE_FN(free)
        with pytest.raises(A.AsepError) as ei:
            A.asep_create(prm, sample_times=times, torch_alloc=False, stream=0)
        return ei.value, calls[0], live, freed

    # every request is made before the context is checked and released, so a
    # run that fails the first one counts them; no run gets as far as a copy
    _, n_calls, _, _ = attempt(fail_at=0)
    assert n_calls >= 7
    for k in range(n_calls):
        err, calls, live, freed = attempt(fail_at=k)
        assert err.code == A.ASEP_ERR_NOMEM and "allocation failed" in str(err), k
        assert calls == n_calls  # every request is made, then the context is released as a whole
        assert sorted(freed) == sorted(live.items()), k


def test_misaligned_allocation_is_refused_without_device(A):
    """A block that does not start on a 256-byte boundary is handed straight
    back through free_fn and counts as a failed allocation: asep_create
    returns ASEP_ERR_NOMEM and every block is freed exactly once."""
    for bad in range(3):
        live, freed, calls = {}, [], [0]

        def alloc(nbytes, user):
            k = calls[0]
            calls[0] += 1
            ptr = 0x10000 * (k + 1) + (16 if k == bad else 0)
            live[ptr] = nbytes
            return ptr

        def free(ptr, nbytes, user):
            freed.append((ptr, nbytes))

        prm = A.make_params(L=1024, schedule=A.ASEP_SCHED_SERIAL)
        prm.alloc, prm.free_fn = A.ALLOC_FN(alloc), A.FREE_FN(free)
        with pytest.raises(A.AsepError) as ei:
            A.asep_create(prm, sample_times=[0, 5], torch_alloc=False, stream=0)
        assert ei.value.code == A.ASEP_ERR_NOMEM and "allocation failed" in str(ei.value)
        assert sorted(freed) == sorted(live.items()), bad


def test_microbenchmarks_reject_bad_arguments_without_device(A):
    """The microbenchmarks refuse a missing sink, a launch shape that is not
    whole warps, and (the attempt stream) an "always" threshold, before any
    CUDA call."""
    cases = [lambda: A.asep_philox_bench(1, 32, 1, 0),
             lambda: A.asep_philox_bench(1, 33, 1, 0x10000),
             lambda: A.asep_attempt_bench(1, 32, 1, 0, 0, 0),
             lambda: A.asep_attempt_bench(0, 32, 1, 0, 0, 0x10000),
             lambda: A.asep_attempt_bench(1, 32, 1, A.ASEP_ALWAYS, 0, 0x10000),
             lambda: A.asep_attempt_bench(1, 32, 1, 0, A.ASEP_ALWAYS, 0x10000)]
    for case in cases:
        with pytest.raises(A.AsepError) as ei:
            case()
        assert ei.value.code == A.ASEP_ERR_INVALID
