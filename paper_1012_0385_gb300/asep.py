"""Python binding of ``libasep.so`` (argument marshalling only).

Every function has the name of the C entry point it calls (see
``include/asep.h``); all lattice arithmetic runs in the library's CUDA
kernels.  Importing this module does not need a GPU; creating a context does.
The library is the in-tree build ``paper_1012_0385_gb300/_build/libasep.so``;
if it is missing, :func:`lib` raises instead of falling back to anything.

Device memory is taken from PyTorch's caching allocator and work goes to
PyTorch's current CUDA stream unless the caller passes ``stream=`` /
``torch_alloc=False``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ASEP_OK = 0
ASEP_ERR_INVALID = -1
ASEP_ERR_NOMEM = -2
ASEP_ERR_CUDA = -3
ASEP_ERR_TIMEOUT = -4
ASEP_ERR_STATE = -5

ASEP_MODEL_RING, ASEP_MODEL_TWO_LANE = 0, 1
ASEP_SCHED_DOMAIN, ASEP_SCHED_SERIAL, ASEP_SCHED_SCA = 0, 1, 2
ASEP_DIS_NONE, ASEP_DIS_BIMODAL, ASEP_DIS_TURNING, ASEP_DIS_BIMODAL_PQ, ASEP_DIS_CROSSING = 0, 1, 2, 3, 4
ASEP_INIT_FLAT_ALT, ASEP_INIT_BERNOULLI_HALF = 0, 1
ASEP_ALWAYS = 0xFFFFFFFF
ASEP_FAULT_NONE, ASEP_FAULT_COPY_STALL, ASEP_FAULT_BALANCE_STALL = 0, 1, 2
ASEP_FLAG_NO_HOP_COUNTS = 1
ASEP_FLAG_PROFILE = 2
ASEP_FLAG_AUTOCORR = 4

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class asep_params(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_uint32),
        ("schedule", ctypes.c_uint32),
        ("L", ctypes.c_uint64),
        ("domain_sites", ctypes.c_uint32),
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
        ("sample_times", ctypes.POINTER(ctypes.c_uint64)),
        ("n_sample_times", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN),
        ("free_fn", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
        ("autocorr_t0", ctypes.c_uint64),
    ]


class asep_info(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_uint64),
        ("D", ctypes.c_uint32),
        ("planes", ctypes.c_uint32),
        ("S", ctypes.c_uint32),
        ("n_recorded", ctypes.c_uint32),
        ("sweep", ctypes.c_uint64),
        ("attempts_per_sweep", ctypes.c_uint64),
        ("device_bytes", ctypes.c_uint64),
        ("kernel_launches", ctypes.c_uint64),
        ("cluster", ctypes.c_uint32),
        ("samples_per_group", ctypes.c_uint32),
        ("groups", ctypes.c_uint32),
        ("threads", ctypes.c_uint32),
        ("smem_bytes", ctypes.c_uint32),
        ("tile_columns", ctypes.c_uint32),
    ]


# Every symbol include/asep.h declares (tests check that the library exports them).
EXPORTED = ("asep_create", "asep_plan", "asep_sweep", "asep_width", "asep_state", "asep_load_state", "asep_reset", "asep_counters",
            "asep_disorder", "asep_get_info", "asep_sync", "asep_destroy", "asep_last_error", "asep_threshold",
            "asep_poisson_table", "asep_philox_bench", "asep_attempt_bench", "asep_version", "asep_batch_create", "asep_batch_sweep",
            "asep_batch_graph", "asep_batch_set_launch", "asep_batch_destroy", "asep_batch_last_error",
            "asep_batch_sweep_static", "asep_set_plan", "asep_set_launch_sweeps", "asep_set_balance", "asep_currents", "asep_profile", "asep_autocorr",
            "asep_height_offset", "asep_inject_fault")


class AsepError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"asep error {code}: {msg}")
        self.code = code


_lib = None
_lib_lock = threading.Lock()


def lib():
    """The loaded libasep.so.  Raises if the in-tree build is missing."""
    global _lib
    with _lib_lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() (nvcc, sm_103a)")
            L = ctypes.CDLL(path)
            P = ctypes.POINTER
            vp = ctypes.c_void_p
            L.asep_create.argtypes = [P(asep_params), P(vp)]
            L.asep_sweep.argtypes = [vp, ctypes.c_uint64]
            L.asep_width.argtypes = [vp, P(ctypes.c_int64), P(ctypes.c_uint64), P(ctypes.c_double), ctypes.c_size_t]
            L.asep_state.argtypes = [vp, P(ctypes.c_uint32), ctypes.c_size_t, P(ctypes.c_uint64)]
            L.asep_load_state.argtypes = [vp, P(ctypes.c_uint32), ctypes.c_size_t, ctypes.c_uint64]
            L.asep_reset.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64]
            L.asep_counters.argtypes = [vp, P(ctypes.c_uint64), ctypes.c_size_t]
            L.asep_disorder.argtypes = [vp, P(ctypes.c_uint32), ctypes.c_size_t]
            L.asep_get_info.argtypes = [vp, P(asep_info)]
            L.asep_plan.argtypes = [P(asep_params), P(asep_info)]
            L.asep_sync.argtypes = [vp]
            L.asep_inject_fault.argtypes = [vp, ctypes.c_uint32]
            L.asep_destroy.argtypes = [vp]
            L.asep_last_error.argtypes = [vp]
            L.asep_last_error.restype = ctypes.c_char_p
            L.asep_threshold.argtypes = [ctypes.c_double]
            L.asep_threshold.restype = ctypes.c_uint32
            L.asep_poisson_table.argtypes = [ctypes.c_uint32, P(ctypes.c_uint32), P(ctypes.c_uint32), ctypes.c_uint32,
                                             P(ctypes.c_uint32)]
            L.asep_philox_bench.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, vp,
                                            P(ctypes.c_float)]
            L.asep_attempt_bench.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                             ctypes.c_uint32, vp, P(ctypes.c_float)]
            L.asep_version.restype = ctypes.c_char_p
            L.asep_batch_create.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32, P(vp)]
            L.asep_batch_sweep.argtypes = [vp, P(vp), P(ctypes.c_uint64), ctypes.c_uint32]
            L.asep_batch_graph.argtypes = [vp, P(vp), P(ctypes.c_uint64), ctypes.c_uint32, ctypes.c_uint32]
            L.asep_batch_set_launch.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32]
            L.asep_batch_destroy.argtypes = [vp]
            L.asep_batch_last_error.argtypes = [vp]
            L.asep_batch_last_error.restype = ctypes.c_char_p
            L.asep_batch_sweep_static.argtypes = [P(vp), P(ctypes.c_uint64), ctypes.c_uint32, vp]
            L.asep_set_plan.argtypes = [vp, ctypes.c_uint32, ctypes.c_uint32]
            L.asep_set_launch_sweeps.argtypes = [vp, ctypes.c_uint32]
            L.asep_set_balance.argtypes = [vp, ctypes.c_uint32]
            L.asep_currents.argtypes = [vp, P(ctypes.c_int64), ctypes.c_size_t]
            L.asep_profile.argtypes = [vp, P(ctypes.c_uint32), ctypes.c_size_t]
            L.asep_autocorr.argtypes = [vp, P(ctypes.c_int64), ctypes.c_size_t]
            L.asep_height_offset.argtypes = [vp, P(ctypes.c_int64), ctypes.c_size_t]
            for name in EXPORTED:
                if name not in ("asep_last_error", "asep_threshold", "asep_version", "asep_batch_last_error"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(rc: int, ctx=None):
    if rc != ASEP_OK:
        raise AsepError(rc, asep_last_error(ctx))


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# ---------------------------------------------------------------------------
# Host-only helpers
# ---------------------------------------------------------------------------

def asep_version() -> str:
    return lib().asep_version().decode()


def asep_threshold(p: float) -> int:
    return int(lib().asep_threshold(float(p)))


def asep_poisson_table(m: int) -> tuple[int, np.ndarray]:
    k_lo = ctypes.c_uint32()
    n = ctypes.c_uint32()
    _check(lib().asep_poisson_table(m, ctypes.byref(k_lo), None, 0, ctypes.byref(n)))
    tab = np.zeros(n.value, dtype=np.uint32)
    _check(lib().asep_poisson_table(m, ctypes.byref(k_lo), _ptr(tab, ctypes.c_uint32), n.value, ctypes.byref(n)))
    return int(k_lo.value), tab


def asep_last_error(ctx=None) -> str:
    msg = lib().asep_last_error(ctx)
    return msg.decode() if msg else ""


# ---------------------------------------------------------------------------
# Torch plumbing: allocator hook and current stream
# ---------------------------------------------------------------------------

class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch

        self._torch = torch
        self.device = device
        self.stream = stream
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
        except Exception:  # out of memory -> the library reports ASEP_ERR_NOMEM
            return None

    def _free(self, ptr, nbytes, user):
        self._torch.cuda.caching_allocator_delete(ptr)


def make_params(**kw) -> asep_params:
    """asep_params with defaults (ring, domain schedule, flat start, TASEP)."""
    p = asep_params()
    p.model = kw.pop("model", ASEP_MODEL_RING)
    p.schedule = kw.pop("schedule", ASEP_SCHED_DOMAIN)
    p.L = kw.pop("L")
    p.domain_sites = kw.pop("domain_sites", 0)
    p.n_realizations = kw.pop("n_realizations", 1)
    p.samples_per_real = kw.pop("samples_per_real", 1)
    p.first_sample = kw.pop("first_sample", 0)
    p.p_thr = kw.pop("p_thr", ASEP_ALWAYS)
    p.q_thr = kw.pop("q_thr", 0)
    p.dis_kind = kw.pop("dis_kind", ASEP_DIS_NONE)
    p.dis_a_thr = kw.pop("dis_a_thr", 0)
    p.dis_b_thr = kw.pop("dis_b_thr", 0)
    p.dis_c_thr = kw.pop("dis_c_thr", 0)
    p.init_kind = kw.pop("init_kind", ASEP_INIT_FLAT_ALT)
    p.seed = kw.pop("seed", 1)
    p.dis_seed = kw.pop("dis_seed", 0)
    p.init_seed = kw.pop("init_seed", 0)
    p.flags = kw.pop("flags", 0)
    p.autocorr_t0 = kw.pop("autocorr_t0", 0)
    if kw:
        raise TypeError(f"unknown parameters {sorted(kw)}")
    return p


class Context:
    """An owning handle around ``asep_ctx*`` (keeps the allocator callbacks
    and the sample-time array alive)."""

    def __init__(self, handle, params: asep_params, keep):
        self.handle = handle
        self.params = params
        self._keep = keep

    def close(self):
        if self.handle:
            asep_destroy(self)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _h(ctx):
    return ctx.handle if isinstance(ctx, Context) else ctx


# ---------------------------------------------------------------------------
# The C ABI
# ---------------------------------------------------------------------------

def asep_create(params: asep_params, sample_times=(), stream=None, torch_alloc: bool = True) -> Context:
    """Create a context.  ``stream`` is a cudaStream_t as int (default: torch's
    current stream); device memory comes from torch unless torch_alloc=False."""
    times = np.ascontiguousarray(np.asarray(sorted(set(int(t) for t in sample_times)), dtype=np.uint64))
    keep = [times]
    params.sample_times = _ptr(times, ctypes.c_uint64) if times.size else None
    params.n_sample_times = int(times.size)
    dev = 0
    try:
        import torch

        if torch.cuda.is_available():
            dev = torch.cuda.current_device()
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
            if torch_alloc:
                al = _TorchAllocator(dev, int(stream or 0))
                keep.append(al)
                params.alloc = al.alloc
                params.free_fn = al.free
    except ImportError:
        pass
    params.stream = stream or None
    h = ctypes.c_void_p()
    rc = lib().asep_create(ctypes.byref(params), ctypes.byref(h))
    if rc != ASEP_OK:
        raise AsepError(rc, asep_last_error(None))
    return Context(h, params, keep)


def asep_plan(params: asep_params, sample_times=()) -> dict:
    """The context asep_create would make (sizes, launch plan, device bytes,
    shared memory per CTA), without allocating or launching anything."""
    times = np.ascontiguousarray(np.asarray(sorted(set(int(t) for t in sample_times)), dtype=np.uint64))
    params.sample_times = _ptr(times, ctypes.c_uint64) if times.size else None
    params.n_sample_times = int(times.size)
    info = asep_info()
    rc = lib().asep_plan(ctypes.byref(params), ctypes.byref(info))
    if rc != ASEP_OK:
        raise AsepError(rc, asep_last_error(None))
    return {f: getattr(info, f) for f, _ in asep_info._fields_}


def asep_sweep(ctx, n_mcs: int) -> None:
    _check(lib().asep_sweep(_h(ctx), int(n_mcs)), _h(ctx))


def asep_get_info(ctx) -> dict:
    info = asep_info()
    _check(lib().asep_get_info(_h(ctx), ctypes.byref(info)), _h(ctx))
    return {f: getattr(info, f) for f, _ in asep_info._fields_}


def asep_inject_fault(ctx, fault: int) -> None:
    """Fault injection for tests of the timeout path (ASEP_FAULT_*)."""
    _check(lib().asep_inject_fault(_h(ctx), int(fault)), _h(ctx))


def asep_set_plan(ctx, cluster: int = 0, samples_per_group: int = 0) -> None:
    _check(lib().asep_set_plan(_h(ctx), int(cluster), int(samples_per_group)), _h(ctx))


def asep_set_launch_sweeps(ctx, max_sweeps: int = 0) -> None:
    _check(lib().asep_set_launch_sweeps(_h(ctx), int(max_sweeps)), _h(ctx))


def asep_set_balance(ctx, chunk_sweeps: int = 0) -> None:
    _check(lib().asep_set_balance(_h(ctx), int(chunk_sweeps)), _h(ctx))


def asep_width(ctx):
    """(sum_h [T,S,planes] int64, sum_h2 [T,S,planes,2] uint64 (lo, hi), w2 [T,S,planes] float64)."""
    info = asep_get_info(ctx)
    shape = (info["n_recorded"], info["S"], info["planes"])
    n = int(np.prod(shape))
    sh = np.zeros(max(n, 1), dtype=np.int64)
    sh2 = np.zeros(2 * max(n, 1), dtype=np.uint64)
    w2 = np.zeros(max(n, 1), dtype=np.float64)
    _check(lib().asep_width(_h(ctx), _ptr(sh, ctypes.c_int64), _ptr(sh2, ctypes.c_uint64), _ptr(w2, ctypes.c_double),
                            max(n, 1)), _h(ctx))
    return sh[:n].reshape(shape), sh2[: 2 * n].reshape(shape + (2,)), w2[:n].reshape(shape)


def asep_state(ctx):
    """(words [S, planes, L/32] uint32, sweep)."""
    info = asep_get_info(ctx)
    shape = (info["S"], info["planes"], info["L"] // 32)
    words = np.zeros(shape, dtype=np.uint32)
    sweep = ctypes.c_uint64()
    _check(lib().asep_state(_h(ctx), _ptr(words, ctypes.c_uint32), words.size, ctypes.byref(sweep)), _h(ctx))
    return words, int(sweep.value)


def asep_load_state(ctx, words: np.ndarray, sweep: int) -> None:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    _check(lib().asep_load_state(_h(ctx), _ptr(w, ctypes.c_uint32), w.size, int(sweep)), _h(ctx))


def asep_reset(ctx, seed: int, init_seed: int = 0) -> None:
    _check(lib().asep_reset(_h(ctx), int(seed), int(init_seed)), _h(ctx))
    if isinstance(ctx, Context):
        ctx.params.seed = int(seed)
        ctx.params.init_seed = int(init_seed)


def asep_counters(ctx) -> np.ndarray:
    info = asep_get_info(ctx)
    c = np.zeros((info["S"], 4), dtype=np.uint64)
    _check(lib().asep_counters(_h(ctx), _ptr(c, ctypes.c_uint64), c.size), _h(ctx))
    return c


def asep_currents(ctx) -> np.ndarray:
    """Hop counters at every recorded sample time, [n_recorded, S, 4] int64."""
    info = asep_get_info(ctx)
    out = np.zeros((max(info["n_recorded"], 1), info["S"], 4), dtype=np.int64)
    _check(lib().asep_currents(_h(ctx), _ptr(out, ctypes.c_int64), out.size), _h(ctx))
    return out[: info["n_recorded"]]


def asep_profile(ctx) -> np.ndarray:
    """Occupied sites per 32-site word summed over the sample times, [S, planes, L/32]."""
    info = asep_get_info(ctx)
    out = np.zeros((info["S"], info["planes"], info["L"] // 32), dtype=np.uint32)
    _check(lib().asep_profile(_h(ctx), _ptr(out, ctypes.c_uint32), out.size), _h(ctx))
    return out


def asep_autocorr(ctx) -> np.ndarray:
    """Overlap sum_i n_i(t0) n_i(t) at every recorded sample time, [n_recorded, S, planes]."""
    info = asep_get_info(ctx)
    out = np.zeros((max(info["n_recorded"], 1), info["S"], info["planes"]), dtype=np.int64)
    _check(lib().asep_autocorr(_h(ctx), _ptr(out, ctypes.c_int64), out.size), _h(ctx))
    return out[: info["n_recorded"]]


def asep_height_offset(ctx) -> np.ndarray:
    """Height of the column between sites L-1 and 0 at every recorded sample
    time, relative to the last create/reset/load, [n_recorded, S] int64."""
    info = asep_get_info(ctx)
    out = np.zeros((max(info["n_recorded"], 1), info["S"]), dtype=np.int64)
    _check(lib().asep_height_offset(_h(ctx), _ptr(out, ctypes.c_int64), out.size), _h(ctx))
    return out[: info["n_recorded"]]


def asep_disorder(ctx) -> np.ndarray:
    """Quenched planes, [R, planes * L/32] (independent p and q classes: the
    p-class plane, then the q-class plane; crossing kind: u marks, v marks)."""
    p = ctx.params
    R = p.n_realizations if p.dis_kind != ASEP_DIS_NONE else 0
    planes = 2 if p.dis_kind in (ASEP_DIS_BIMODAL_PQ, ASEP_DIS_CROSSING) else 1
    m = np.zeros((max(R, 1), planes * (p.L // 32)), dtype=np.uint32)
    _check(lib().asep_disorder(_h(ctx), _ptr(m, ctypes.c_uint32), m.size), _h(ctx))
    return m[:R]


def asep_sync(ctx) -> None:
    _check(lib().asep_sync(_h(ctx)), _h(ctx))


def asep_destroy(ctx) -> None:
    h = _h(ctx)
    if h:
        _check(lib().asep_destroy(h))
    if isinstance(ctx, Context):
        ctx.handle = None


def asep_philox_bench(blocks: int, threads: int, calls: int, sink_ptr: int, stream=None) -> float:
    """Milliseconds for blocks*threads threads x `calls` Philox4x32-10 calls
    (sink_ptr: device buffer of blocks*threads uint32)."""
    ms = ctypes.c_float()
    _check(lib().asep_philox_bench(stream, blocks, threads, calls, ctypes.c_void_p(sink_ptr), ctypes.byref(ms)))
    return float(ms.value)


def asep_attempt_bench(blocks: int, threads: int, calls: int, p_thr: int, q_thr: int, sink_ptr: int,
                       stream=None) -> float:
    """Milliseconds for blocks*threads threads x `calls` Philox4x32-10 calls,
    each feeding four plain-ring attempts on a register-held word pair
    (sink_ptr: device buffer of 2*blocks*threads uint32, final pairs)."""
    ms = ctypes.c_float()
    _check(lib().asep_attempt_bench(stream, blocks, threads, calls, p_thr, q_thr, ctypes.c_void_p(sink_ptr),
                                    ctypes.byref(ms)))
    return float(ms.value)


# ---------------------------------------------------------------------------
# Batches
# ---------------------------------------------------------------------------

class Batch:
    """Owning handle around ``asep_batch*``."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            asep_batch_destroy(self)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bh(b):
    return b.handle if isinstance(b, Batch) else b


def asep_batch_last_error(b=None) -> str:
    msg = lib().asep_batch_last_error(_bh(b) if b is not None else None)
    return msg.decode() if msg else ""


def _bcheck(rc: int, b):
    if rc != ASEP_OK:
        raise AsepError(rc, asep_batch_last_error(b))


def asep_batch_create(max_jobs: int = 256, max_items: int = 1 << 16, stream=None) -> Batch:
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
    h = ctypes.c_void_p()
    rc = lib().asep_batch_create(stream or None, int(max_jobs), int(max_items), ctypes.byref(h))
    if rc != ASEP_OK:
        raise AsepError(rc, asep_batch_last_error(None))
    return Batch(h)


def _ctx_array(ctxs):
    arr = (ctypes.c_void_p * len(ctxs))(*[_h(c).value if isinstance(_h(c), ctypes.c_void_p) else _h(c)
                                          for c in ctxs])
    return arr


def asep_batch_sweep(b, ctxs, n_mcs) -> None:
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(n_mcs, dtype=np.uint64), (len(ctxs),)))
    _bcheck(lib().asep_batch_sweep(_bh(b), _ctx_array(ctxs), _ptr(n, ctypes.c_uint64), len(ctxs)), b)


def asep_batch_graph(b, ctxs, n_mcs, replays: int) -> None:
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(n_mcs, dtype=np.uint64), (len(ctxs),)))
    _bcheck(lib().asep_batch_graph(_bh(b), _ctx_array(ctxs), _ptr(n, ctypes.c_uint64), len(ctxs), int(replays)), b)


def asep_batch_set_launch(b, threads: int = 0, ctas_per_sm: int = 0) -> None:
    _bcheck(lib().asep_batch_set_launch(_bh(b), int(threads), int(ctas_per_sm)), b)


def asep_batch_destroy(b) -> None:
    h = _bh(b)
    if h:
        lib().asep_batch_destroy(h)
    if isinstance(b, Batch):
        b.handle = None


def asep_batch_sweep_static(ctxs, n_mcs, stream=None) -> None:
    """The batch sweep without any allocation (static device workspace): for
    callers that may not allocate device memory when they run work.  Every
    context must use `stream` (default: torch's current stream).  With no
    contexts it only sets up the current device (the start-up call)."""
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
    n = np.ascontiguousarray(np.broadcast_to(np.asarray(n_mcs, dtype=np.uint64), (len(ctxs),)))
    _check(lib().asep_batch_sweep_static(_ctx_array(ctxs), _ptr(n, ctypes.c_uint64), len(ctxs), stream or None))

