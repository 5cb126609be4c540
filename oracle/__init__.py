"""CPU oracle for the bit-packed ASEP / 1+1-d KPZ Monte Carlo.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product package never imports
it, and it never imports the product package.

The arithmetic lives in ``asep_oracle.c`` (plain C, one site at a time); this
module compiles it with gcc, wraps it with ctypes and adds the pieces that are
clearer in Python:

* :func:`poisson_table` -- the Poisson(m) CDF in u32 fixed point, computed
  exactly with 150-digit decimals (the attempt count of a domain);
* :func:`threshold` -- the u32 rate encoding (20 significant bits);
* :func:`log_times` -- the sampling times of Eq. (sampling), paper sec. 2.2;
* :func:`width2` -- W^2 of Eq. (W), paper sec. 2.1, from exact integer sums;
* :func:`run` -- init + quenched disorder + sweeps + W^2 at sampling times,
  i.e. the whole hot path for a batch of samples.

Parity: every function here is pinned by ``tests/test_oracle_*.py`` against
the paper's printed values, closed forms, exact enumeration
(:mod:`oracle.exact`) or an independent Philox implementation.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from decimal import ROUND_FLOOR, Decimal, localcontext
from fractions import Fraction
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asep_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

MODEL_RING, MODEL_TWO_LANE = 0, 1
SCHED_DOMAIN, SCHED_SERIAL, SCHED_SCA = 0, 1, 2
DIS_NONE, DIS_BIMODAL, DIS_TURNING, DIS_BIMODAL_PQ, DIS_CROSSING = 0, 1, 2, 3, 4
INIT_FLAT_ALT, INIT_BERNOULLI_HALF = 0, 1
ALWAYS = 0xFFFFFFFF

_lib = None
_lib_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``asep_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CParams(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_uint32),
        ("schedule", ctypes.c_uint32),
        ("L", ctypes.c_uint64),
        ("D", ctypes.c_uint32),
        ("n_realizations", ctypes.c_uint32),
        ("samples_per_real", ctypes.c_uint32),
        ("first_sample", ctypes.c_uint32),
        ("p_thr", ctypes.c_uint32),
        ("q_thr", ctypes.c_uint32),
        ("dis_kind", ctypes.c_uint32),
        ("dis_a_thr", ctypes.c_uint32),
        ("dis_b_thr", ctypes.c_uint32),
        ("dis_c_thr", ctypes.c_uint32),
        ("init_kind", ctypes.c_uint32),
        ("seed", ctypes.c_uint64),
        ("dis_seed", ctypes.c_uint64),
        ("init_seed", ctypes.c_uint64),
    ]


def lib():
    global _lib
    with _lib_lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            pp = ctypes.POINTER(_CParams)
            L.orc_philox.argtypes = [u32p, u32p, u32p]
            L.orc_philox.restype = None
            L.orc_sweeps.argtypes = [pp, u32p, ctypes.c_uint32, ctypes.c_uint32, u32p, u32p, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_uint64, u64p]
            L.orc_sweeps.restype = ctypes.c_int
            L.orc_init.argtypes = [pp, u32p, ctypes.c_uint32]
            L.orc_init.restype = ctypes.c_int
            L.orc_disorder.argtypes = [pp, u32p, ctypes.c_uint32]
            L.orc_disorder.restype = ctypes.c_int
            L.orc_heights.argtypes = [u32p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64), u64p, u64p]
            L.orc_heights.restype = None
            L.orc_serial_reference.argtypes = [pp, u32p, u32p, ctypes.c_uint64, ctypes.c_uint64, u64p]
            L.orc_serial_reference.restype = ctypes.c_int
            _lib = L
    return _lib


def _u32p(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _u64p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


# ---------------------------------------------------------------------------
# Encodings
# ---------------------------------------------------------------------------

def threshold(p: float) -> int:
    """u32 threshold of a probability: 0 = never, 0xffffffff = always, else a
    multiple of 4096 (20 significant bits); a draw r is accepted iff
    ``(r & 0xfffff000) < t``, so the probability is exactly t / 2^32."""
    if p >= 1.0:
        return ALWAYS
    if p <= 0.0:
        return 0
    q = int(math.floor(p * (1 << 20) + 0.5))
    if q >= (1 << 20):
        return ALWAYS
    return q << 12


def probability(t: int) -> Fraction:
    """Exact acceptance probability of threshold t."""
    if t == ALWAYS:
        return Fraction(1)
    return Fraction(t, 1 << 32)


@lru_cache(maxsize=None)
def poisson_table(m: int) -> tuple[int, tuple[int, ...]]:
    """Attempt-count table of a domain with m bonds.

    T_k = floor(2^32 * P(Poisson(m) <= k)), evaluated with 150-digit decimal
    arithmetic.  Returns (k_lo, entries) where k_lo counts the leading zero
    entries and ``entries`` = T_{k_lo} .. T_{k_cap-1}, k_cap being the first k
    with T_k = 2^32 - 1.  A draw w maps to K = k_lo + #{j : entries[j] <= w}.
    """
    two32 = 1 << 32
    with localcontext() as ctx:
        ctx.prec = 150
        term = (-Decimal(m)).exp()  # P(K = 0)
        cdf = Decimal(0)
        scale = Decimal(two32)
        k = 0
        k_lo = 0
        entries = []
        while True:
            cdf += term
            t = int((cdf * scale).to_integral_value(rounding=ROUND_FLOOR))
            if t >= two32 - 1:
                break
            if t == 0:
                k_lo += 1
            else:
                entries.append(t)
            k += 1
            term = term * Decimal(m) / Decimal(k)
    return k_lo, tuple(entries)


def poisson_count(m: int, w: int) -> int:
    k_lo, tab = poisson_table(m)
    return k_lo + sum(1 for t in tab if t <= w)


def log_times(t_max: int, t0: int = 30, ratio: float = 1.05, include_zero: bool = True) -> list[int]:
    """Sampling sweeps of Eq. (sampling), paper sec. 2.2: t_0 = 30,
    t_{i+1} = 1.05 t_i (double recurrence), recorded at floor(t_i) <= t_max,
    duplicates dropped; t = 0 (the flat start) optionally first."""
    out = [0] if include_zero else []
    t = float(t0)
    while math.floor(t) <= t_max:
        v = int(math.floor(t))
        if not out or out[-1] != v:
            out.append(v)
        t = t * ratio
    return out


def width2(L: int, sum_h: int, sum_h2: int) -> float:
    """W^2 = (1/L) sum h^2 - ((1/L) sum h)^2, Eq. (W), evaluated exactly."""
    return float(Fraction(L * sum_h2 - sum_h * sum_h, L * L))


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------

@dataclass
class Params:
    model: int = MODEL_RING
    schedule: int = SCHED_DOMAIN
    L: int = 4096
    D: int = 256
    n_realizations: int = 1
    samples_per_real: int = 1
    first_sample: int = 0
    p_thr: int = ALWAYS
    q_thr: int = 0
    dis_kind: int = DIS_NONE
    dis_a_thr: int = 0
    dis_b_thr: int = 0
    dis_c_thr: int = 0
    init_kind: int = INIT_FLAT_ALT
    seed: int = 1
    dis_seed: int = 0
    init_seed: int = 0

    @property
    def S(self) -> int:
        return self.n_realizations * self.samples_per_real

    @property
    def planes(self) -> int:
        return 2 if self.model == MODEL_TWO_LANE else 1

    @property
    def W(self) -> int:
        return (self.L + 31) // 32

    @property
    def bonds_per_domain(self) -> int:
        return 2 * self.D if self.model == MODEL_TWO_LANE else self.D

    def c(self) -> _CParams:
        return _CParams(**{f: getattr(self, f) for f, _ in _CParams._fields_})


# ---------------------------------------------------------------------------
# Primitives
# ---------------------------------------------------------------------------

def philox(ctr, key) -> tuple[int, int, int, int]:
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_u32p(c), _u32p(k), _u32p(out))
    return tuple(int(x) for x in out)


def heights(words: np.ndarray, L: int) -> tuple[int, int]:
    """(sum_i h_i, sum_i h_i^2) with h_i = sum_{j<=i} (2 n_j - 1)."""
    w = np.ascontiguousarray(words, dtype=np.uint32)
    s1 = ctypes.c_int64()
    lo = ctypes.c_uint64()
    hi = ctypes.c_uint64()
    lib().orc_heights(_u32p(w), L, ctypes.byref(s1), ctypes.byref(lo), ctypes.byref(hi))
    return int(s1.value), (int(hi.value) << 64) | int(lo.value)


def init_state(P: Params) -> np.ndarray:
    """Initial lattices, shape [S, planes, L/32] (uint32, bit k of word w = site 32w+k)."""
    st = np.zeros((P.S, P.planes, P.W), dtype=np.uint32)
    cp = P.c()
    for s in range(P.S):
        row = np.ascontiguousarray(st[s])
        if lib().orc_init(ctypes.byref(cp), _u32p(row), P.first_sample + s) != 0:
            raise ValueError("orc_init rejected the parameters")
        st[s] = row
    return st


def disorder(P: Params) -> np.ndarray | None:
    """Quenched planes, shape [R, planes * L/32] (planes = 2 for independent
    p and q classes and for the two lanes' u and v crossing classes, else 1: a
    realization's planes one after the other), or None when there is no
    disorder."""
    if P.dis_kind == DIS_NONE:
        return None
    n = P.W * (2 if P.dis_kind in (DIS_BIMODAL_PQ, DIS_CROSSING) else 1)
    m = np.zeros((P.n_realizations, n), dtype=np.uint32)
    cp = P.c()
    first_real = P.first_sample // P.samples_per_real
    for r in range(P.n_realizations):
        row = np.zeros(n, dtype=np.uint32)
        lib().orc_disorder(ctypes.byref(cp), _u32p(row), first_real + r)
        m[r] = row
    return m


def _threads(n: int | None) -> int:
    return max(1, n if n is not None else (os.cpu_count() or 1))


def replay(P: Params, state: np.ndarray, s0: int, n_sweeps: int, mask: np.ndarray | None = None,
           samples=None, threads: int | None = None, seam: np.ndarray | None = None) -> np.ndarray:
    """Advance ``state`` ([S, planes, W]) in place by n_sweeps sweeps starting
    at sweep index s0, with the exact schedule of P.  Returns per-sample hop
    counters [S, 4] (ring: right, left; two lanes: A, B, A->B, B->A).  With
    ``seam`` ([S, 2]) the ring's right and left hops across the bond
    (L-1, 0) are added to it."""
    if P.schedule == SCHED_DOMAIN:
        k_lo, tab = poisson_table(P.bonds_per_domain)
    else:
        k_lo, tab = 0, (0,)
    tab_np = np.array(tab, dtype=np.uint32)
    cnt = np.zeros((P.S, 4), dtype=np.uint64)
    idx = list(range(P.S)) if samples is None else list(samples)
    cp = P.c()

    def one(s):
        row = np.ascontiguousarray(state[s])
        m = None
        if mask is not None:
            m = np.ascontiguousarray(mask[s // P.samples_per_real])
        c = np.zeros(6, dtype=np.uint64)
        rc = lib().orc_sweeps(ctypes.byref(cp), _u32p(tab_np), k_lo, len(tab), _u32p(row),
                              _u32p(m) if m is not None else None, P.first_sample + s, s0, n_sweeps, _u64p(c))
        if rc != 0:
            raise ValueError("orc_sweeps rejected the parameters")
        state[s] = row
        cnt[s] = c[:4]
        if seam is not None:
            seam[s] += c[4:6]

    with ThreadPoolExecutor(max_workers=_threads(threads)) as ex:
        list(ex.map(one, idx))
    return cnt


def serial_reference(P: Params, state: np.ndarray, n_sweeps: int, rng_seeds, mask: np.ndarray | None = None,
                     threads: int | None = None) -> np.ndarray:
    """Independent plain RSU (own xoshiro256** generator) on every sample."""
    cnt = np.zeros((P.S, 4), dtype=np.uint64)
    cp = P.c()

    def one(s):
        row = np.ascontiguousarray(state[s])
        m = np.ascontiguousarray(mask[s // P.samples_per_real]) if mask is not None else None
        c = np.zeros(6, dtype=np.uint64)
        rc = lib().orc_serial_reference(ctypes.byref(cp), _u32p(row), _u32p(m) if m is not None else None,
                                        int(rng_seeds[s]), n_sweeps, _u64p(c))
        if rc != 0:
            raise ValueError("orc_serial_reference rejected the parameters")
        state[s] = row
        cnt[s] = c[:4]

    with ThreadPoolExecutor(max_workers=_threads(threads)) as ex:
        list(ex.map(one, range(P.S)))
    return cnt


@dataclass
class RunResult:
    times: list
    sum_h: np.ndarray      # [n_times, S, planes] int64 (object for safety)
    sum_h2: np.ndarray     # [n_times, S, planes] python ints
    w2: np.ndarray         # [n_times, S, planes] float64
    state: np.ndarray      # final [S, planes, W]
    counters: np.ndarray   # [S, 4]
    extra: dict = field(default_factory=dict)


def run(P: Params, n_mcs: int, sample_times=(), threads: int | None = None, samples=None,
        autocorr_t0: int | None = None) -> RunResult:
    """The whole hot path on the CPU: initial state, quenched disorder, n_mcs
    sweeps, and at every time in ``sample_times`` (sweep counts after which
    to record; 0 = the initial state) the heights and W^2, the cumulative hop
    counters, the occupancy profile (occupied sites per 32-site word, summed
    over the sample times), the ring's height offset H(t) of the column
    between sites L-1 and 0 relative to the start (counted directly from the
    hops across that bond: -2 per right hop, +2 per left hop) and, with
    ``autocorr_t0``, the overlap sum_i n_i(t0) n_i(t) for t >= t0 (0 before)."""
    times = sorted(set(int(t) for t in sample_times if 0 <= t <= n_mcs))
    state = init_state(P)
    mask = disorder(P)
    idx = list(range(P.S)) if samples is None else list(samples)
    nt = len(times)
    sh = np.zeros((nt, P.S, P.planes), dtype=object)
    sh2 = np.zeros((nt, P.S, P.planes), dtype=object)
    w2 = np.zeros((nt, P.S, P.planes), dtype=np.float64)
    cnt = np.zeros((P.S, 4), dtype=np.uint64)
    cnt_at = np.zeros((nt, P.S, 4), dtype=np.int64)
    seam = np.zeros((P.S, 2), dtype=np.uint64)
    h_off = np.zeros((nt, P.S), dtype=np.int64)
    profile = np.zeros((P.S, P.planes, P.W), dtype=np.int64)
    overlap = np.zeros((nt, P.S, P.planes), dtype=np.int64)
    snap = None

    def popcounts(words):
        return np.array([bin(int(x)).count("1") for x in words.ravel()], dtype=np.int64).reshape(words.shape)

    def record(ti):
        nonlocal snap
        t = times[ti]
        if autocorr_t0 is not None and t == autocorr_t0:
            snap = state.copy()
        for s in idx:
            cnt_at[ti, s] = cnt[s].astype(np.int64)
            # height of the column between sites L-1 and 0 relative to the start:
            # a right hop across a bond lowers that bond's column by 2, a left hop raises it
            h_off[ti, s] = -2 * (int(seam[s, 0]) - int(seam[s, 1]))
            for pl in range(P.planes):
                a, b = heights(state[s, pl], P.L)
                sh[ti, s, pl] = a
                sh2[ti, s, pl] = b
                w2[ti, s, pl] = width2(P.L, a, b)
                profile[s, pl] += popcounts(state[s, pl])
                if snap is not None:
                    overlap[ti, s, pl] = int(popcounts(state[s, pl] & snap[s, pl]).sum())

    done = 0
    ti = 0
    while ti < nt and times[ti] == 0:
        record(ti)
        ti += 1
    for target in times[ti:] + ([n_mcs] if not times or times[-1] != n_mcs else []):
        if target > done:
            cnt += replay(P, state, done, target - done, mask=mask, samples=idx, threads=threads, seam=seam)
            done = target
        if ti < nt and times[ti] == done:
            record(ti)
            ti += 1
    return RunResult(times=times, sum_h=sh, sum_h2=sh2, w2=w2, state=state, counters=cnt,
                     extra={"counters_at": cnt_at, "profile": profile, "overlap": overlap, "height_offset": h_off,
                            "seam": seam})
