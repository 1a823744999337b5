"""Seeded generator and limb layout (no GPU)."""
import os

import numpy as np
import pytest

from synth import SplitMix64, from_limbs, pack, to_limbs, unpack

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_vectors():
    for line in open(os.path.join(GOLD, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        seed, *outs = line.split()
        r = SplitMix64(int(seed))
        assert [r.next64() for _ in outs] == [int(o, 16) for o in outs]


def test_below_is_in_range_and_covers():
    r = SplitMix64(7)
    seen = set()
    for _ in range(2000):
        v = r.below(37)
        assert 0 <= v < 37
        seen.add(v)
    assert seen == set(range(37))
    big = (1 << 1023) + 12345
    for _ in range(50):
        assert 0 <= r.below(big) < big


def test_fork_independent_and_deterministic():
    a = SplitMix64(5).fork(3)
    b = SplitMix64(5).fork(3)
    c = SplitMix64(5).fork(4)
    va = [a.next64() for _ in range(4)]
    assert va == [b.next64() for _ in range(4)]
    assert va != [c.next64() for _ in range(4)]


@pytest.mark.parametrize("bits", [1, 31, 32, 33, 1024, 2047])
def test_limbs_roundtrip(bits):
    r = SplitMix64(bits)
    n = (bits + 31) // 32
    for _ in range(20):
        x = r.randbits(bits)
        l = to_limbs(x, n)
        assert l.dtype == np.uint32 and l.shape == (n,)
        assert from_limbs(l) == x
        # little-endian: limb 0 is the low word
        assert int(l[0]) == x & 0xFFFFFFFF
    xs = [r.randbits(bits) for _ in range(5)]
    assert unpack(pack(xs, n)) == xs


def test_limbs_overflow_rejected():
    with pytest.raises(ValueError):
        to_limbs(1 << 64, 2)
