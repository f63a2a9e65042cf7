"""The sampler's Philox4x32-10 on the device against the oracle's independent
implementation (itself pinned to the published known-answer vectors): 10^6
blocks bit for bit, over the counter layout the planner uses ({problem,
iteration, block, 0}), random counters and extreme words, for several keys."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2503_06757_gb300 import prrtc as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2503_06757_gb300 import build
    build.build()


def test_device_philox_matches_oracle_on_a_million_blocks():
    rng = np.random.default_rng(2503)
    n_rand = 600_000
    rand = rng.integers(0, 2 ** 32, size=(n_rand, 4), dtype=np.uint64).astype(np.uint32)
    # the planner's counters: {problem, iteration, block 0..9, 0}
    p, it, b = np.meshgrid(np.arange(200), np.arange(200), np.arange(10), indexing="ij")
    planner = np.stack([p.ravel(), it.ravel(), b.ravel(), np.zeros(p.size)], 1).astype(np.uint32)
    edge = np.array([[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0xFFFFFFFF, 0, 0xFFFFFFFF, 0], [1, 2, 3, 4]], np.uint32)
    ctr = np.concatenate([planner, rand, edge])
    assert len(ctr) >= 1_000_000
    for key in (1, 0, 2 ** 64 - 1, 0x243F6A8885A308D3):
        dev = P.prrtc_philox(ctr, key)
        ref = O.philox_blocks(ctr, key)
        bad = np.nonzero(np.any(dev != ref, axis=1))[0]
        assert len(bad) == 0, (key, bad[:5])


def test_device_philox_known_answers():
    import os
    golden = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    for line in open(golden):
        if not line.strip() or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        out = P.prrtc_philox(np.array([v[0:4]], np.uint32), v[4] | (v[5] << 32))[0]
        assert [int(x) for x in out] == v[6:10]


def test_device_philox_rejects_bad_arguments():
    assert P.prrtc_philox(np.zeros((0, 4), np.uint32), 1).shape == (0, 4)
