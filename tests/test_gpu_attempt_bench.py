"""The attempt-stream microbenchmark (the domain kernel's random stream and
bit operations on a register-held word pair), checked bit-exactly against a
plain restatement: the oracle's Philox4x32-10 in the attempt counter layout
and the sec. 2.1 bond rule applied to bits j, j + 1 of the 64-bit pair."""
import numpy as np
import pytest

import oracle
from paper_1012_0385_gb300 import asep as A

pytestmark = pytest.mark.gpu

SEED = 0x243F6A8885A308D3
TAG_DOM = 4
M32 = 0xFFFFFFFF


@pytest.fixture(scope="module", autouse=True)
def _device():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1012_0385_gb300 import build

    build.build()
    torch.cuda.set_device(0)


def expected_pairs(n_threads: int, calls: int, p: int, q: int) -> np.ndarray:
    key = (SEED & M32, SEED >> 32)
    out = np.zeros(2 * n_threads, dtype=np.uint32)
    for t in range(n_threads):
        pair = ((0xAAAAAAAA ^ ((t * 0x9E3779B9) & M32)) << 32) | (0x55555555 ^ t)
        for c in range(calls):
            ctr = ((c >> 4) & M32, ((c >> 36) & 0xFF) | (TAG_DOM << 8) | ((c & 15) << 12), t, t >> 5)
            for r in oracle.philox(ctr, key):
                j = r & 31
                site_i, site_next = (pair >> j) & 1, (pair >> (j + 1)) & 1
                if (site_i == 1 and site_next == 0 and r < p) or (site_i == 0 and site_next == 1 and r < q):
                    pair ^= 3 << j
        out[2 * t], out[2 * t + 1] = pair & M32, pair >> 32
    return out


@pytest.mark.parametrize("p,q", [(0.75, 0.25), (1 - 2**-20, 0.0), (0.5, 0.5)])
def test_attempt_bench_matches_restatement(p, q):
    import torch

    blocks, threads, calls = 3, 64, 37
    pt, qt = A.asep_threshold(p), A.asep_threshold(q)
    sink = torch.zeros(2 * blocks * threads, dtype=torch.int32, device="cuda")
    ms = A.asep_attempt_bench(blocks, threads, calls, pt, qt, sink.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert ms > 0
    got = sink.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, expected_pairs(blocks * threads, calls, pt, qt))


def test_attempt_bench_rejects_always():
    import torch

    sink = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(A.AsepError):
        A.asep_attempt_bench(1, 32, 1, A.ASEP_ALWAYS, 0, sink.data_ptr())
