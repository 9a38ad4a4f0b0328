"""Pins of the oracle's Philox4x64-10 against independent implementations of the same
published definition (Salmon et al. 2011)."""
import numpy as np
import pytest

from oracle import philox as ph


def test_known_answer_counter0_key0():
    # the published known-answer vector of Philox4x64-10 for counter 0, key 0
    want = [0x16554D9ECA36314C, 0xDB20FE9D672D0FDC, 0xD7E772CEE186176B, 0x7E68B68AEC7BA23B]
    assert ph.philox4x64_scalar([0, 0, 0, 0], [0, 0]) == want
    assert [int(v) for v in ph.philox4x64(0, 0, 0, 0, 0, 0)] == want


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 + 7])
def test_matches_numpy_philox(seed):
    """numpy's Philox bit generator increments its 256-bit counter before each block, so its
    first block is counter + 1."""
    g = np.random.default_rng(seed)
    for _ in range(20):
        c = [int(x) for x in g.integers(0, 2**63, 4, dtype=np.uint64)]
        k = [int(x) for x in g.integers(0, 2**63, 2, dtype=np.uint64)]
        bg = np.random.Philox(key=k, counter=c)
        want = [int(v) for v in bg.random_raw(4)]
        got = ph.philox4x64(c[0] + 1, c[1], c[2], c[3], k[0], k[1])
        assert [int(v) for v in got] == want
        assert ph.philox4x64_scalar([c[0] + 1, c[1], c[2], c[3]], k) == want


def test_vectorised_equals_scalar():
    g = np.random.default_rng(9)
    c = g.integers(0, 2**63, (64, 4), dtype=np.uint64)
    out = ph.philox4x64(c[:, 0], c[:, 1], c[:, 2], c[:, 3], 77, 2**64 - 1)
    for i in range(64):
        assert [int(v) for v in out[i]] == ph.philox4x64_scalar([int(x) for x in c[i]], [77, 2**64 - 1])


def test_draw_conventions():
    x = np.array([0, 2**64 - 1, 2**63, 2**11], dtype=np.uint64)
    assert list(ph.u01(x)) == [0.0, 1.0 - 2.0**-53, 0.5, 2.0**-53]
    assert list(ph.uniform_int(x, 10)) == [0, 9, 5, 0]
    assert list(ph.bit(x)) == [0, 1, 1, 0]
