"""Replica sharding on the CPU: two gloo ranks, each on its own sample range,
reproduce one run over both ranges bit for bit, and the timing reduction
takes the slowest rank.  The per-rank compute is the oracle (the GPU path is
covered by the parity tests); what is tested here is the host logic of
``paper_1012_0385_gb300.replicas`` that ``bench.py --gpus N`` uses."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1012_0385_gb300 import replicas

WORLD = 2
S_RANK = 3
N_MCS = 12
TIMES = [0, 5, 12]


def _params(first: int, count: int) -> "oracle.Params":
    th = oracle.threshold
    return oracle.Params(L=2048, D=64, samples_per_real=count, first_sample=first, p_thr=th(0.75), q_thr=th(0.25),
                         seed=77)


def _words128(x: np.ndarray) -> np.ndarray:
    """Exact (object) 128-bit sums as (low, high) uint64 words, the layout asep_width returns."""
    flat = [int(v) for v in x.ravel()]
    out = np.array([[v & (2**64 - 1), (v >> 64) & (2**64 - 1)] for v in flat], dtype=np.uint64)
    return out.reshape(x.shape + (2,))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, port: int, out_dir: str):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        first, count = replicas.sample_range(rank, WORLD, S_RANK)
        res = oracle.run(_params(first, count), N_MCS, TIMES, threads=1)
        sh = replicas.gather_samples(res.sum_h.astype(np.int64), dist)
        sh2 = replicas.gather_samples(_words128(res.sum_h2), dist)
        words = replicas.gather_samples(res.state.astype(np.int64), dist, axis=0)
        slowest = replicas.max_over_ranks([10.0 * (rank + 1), 5.0 - rank], dist)
        if rank == 0:
            np.savez(os.path.join(out_dir, "gathered.npz"), sh=sh, sh2=sh2, words=words, slowest=np.array(slowest))
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def gathered(tmp_path_factory):
    import torch.multiprocessing as mp

    oracle.build()
    out = tmp_path_factory.mktemp("replicas")
    mp.start_processes(_worker, args=(_free_port(), str(out)), nprocs=WORLD, start_method="spawn", join=True)
    return np.load(out / "gathered.npz")


def test_sample_ranges_are_disjoint_and_cover():
    seen = []
    for r in range(4):
        first, count = replicas.sample_range(r, 4, 5)
        seen.extend(range(first, first + count))
    assert seen == list(range(20))
    for bad in [(2, 2, 5), (-1, 2, 5), (0, 0, 5), (0, 2, 0)]:
        with pytest.raises(ValueError):
            replicas.sample_range(*bad)


def test_two_replicas_equal_one_run_over_both_ranges(gathered):
    ref = oracle.run(_params(0, WORLD * S_RANK), N_MCS, TIMES, threads=1)
    assert np.array_equal(gathered["sh"], ref.sum_h.astype(np.int64))
    assert np.array_equal(gathered["sh2"], _words128(ref.sum_h2))
    assert np.array_equal(gathered["words"], ref.state.astype(np.int64))


def test_timing_reduction_takes_the_slowest_rank(gathered):
    assert list(gathered["slowest"]) == [20.0, 5.0]


def test_throughput_counts_all_ranks():
    assert replicas.throughput(1e9, 4, 2, 2000.0) == pytest.approx(4e9)
    with pytest.raises(ValueError):
        replicas.throughput(1.0, 1, 1, 0.0)
    # one process: helpers pass values through
    assert replicas.max_over_ranks([1.0, 2.0]) == [1.0, 2.0]
    t = np.arange(6, dtype=np.uint64).reshape(1, 3, 2)
    assert replicas.gather_samples(t) is t
