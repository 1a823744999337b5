"""Pins for the RNS model (oracle.rns): base choice, CRT round trip, MM congruence
and bound, exhaustive tiny cases and agreement with the plain definitions."""
import random

import pytest

from oracle import plain, primality, rns
from synth import SplitMix64, load_keys

CLASSES = [(512, 18), (1024, 36), (1536, 54), (2048, 72), (3072, 108), (4096, 145)]


@pytest.mark.parametrize("L,k", CLASSES)
def test_class_base_choice(L, k):
    c = rns.make_class(L)
    assert c.k == k
    pr = c.B + c.Bp
    assert len(set(pr)) == 2 * k and pr == sorted(pr, reverse=True)
    # channel bound: k products of residues always sum below 2^64
    assert c.bound <= 1 << 31 and k * (c.bound - 1) ** 2 < 1 << 64
    assert all(p < c.bound for p in pr)
    for p in pr[:8] + pr[-8:]:
        assert primality.is_prime_by_trial(p)
    # the base bounds hold for k ...
    assert c.M >= 4 * (k + 1) ** 2 << L and c.Mp >= 2 * (k + 1) << L
    # ... and fail for k-1 with the bound of k-1 channels
    pk = rns.primes_below(rns.prime_bound(k - 1), 2 * (k - 1))
    M1 = 1
    for p in pk[: k - 1]:
        M1 *= p
    Mp1 = 1
    for p in pk[k - 1:]:
        Mp1 *= p
    assert not (M1 >= 4 * k ** 2 << L and Mp1 >= 2 * k << L)


def test_fixed_point_factor_exact_near_limits():
    # floor(sum xi/m) recovered exactly when the value is below 3/4 of the product
    c = rns.make_class(1024)
    r = random.Random(9)
    for X in [0, 1, c.M // 2, (3 * c.M) // 4 - 1] + [r.randrange((3 * c.M) // 4) for _ in range(200)]:
        xi = [(X % m) * c.t["M_mi_inv"][i] % m for i, m in enumerate(c.B)]
        total = sum(xi[i] * (c.M // m) for i, m in enumerate(c.B))
        assert (total - X) % c.M == 0
        assert rns.fixed_point_factor(xi, c.B) == total // c.M


def test_primes_below_matches_brute_force():
    assert list(rns.primes_below(256, 6)) == [251, 241, 239, 233, 229, 227]
    assert all(primality.is_prime_by_trial(p) for p in rns.primes_below(1 << 31, 20))
    # no prime skipped between consecutive entries
    ps = rns.primes_below(1 << 31, 5)
    for a, b in zip(ps, ps[1:]):
        assert not any(primality.is_prime_by_trial(n) for n in range(b + 1, a))


@pytest.mark.parametrize("L", [512, 1024, 2048])
def test_crt_roundtrip(L):
    c = rns.make_class(L)
    r = random.Random(L)
    # the fixed-point CRT factor is exact below 3M/4; MM outputs stay far below that
    lim = (3 * c.M) // 4
    for X in [0, 1, lim - 1, c.M // 3] + [r.randrange(lim) for _ in range(30)]:
        assert rns.crt_value(c, rns.to_rns(c, X)) == X


def _mm_check(key, x, y):
    c = key.cls
    out = rns.mm(key, rns.to_rns(c, x), rns.to_rns(c, y))
    R = rns.crt_value(c, out)
    assert 0 <= R < (c.k + 1) * key.N
    assert (R * c.M - x * y) % key.N == 0
    assert rns.to_rns(c, R) == out          # every channel consistent with the integer


@pytest.mark.parametrize("L", [512, 1024])
def test_mm_congruence_and_bound(L):
    c = rns.make_class(L)
    r = random.Random(L + 1)
    for _ in range(4):
        N = r.getrandbits(L) | 1 | (1 << (L - 1))
        key = rns.make_key(c, N)
        hi = (c.k + 1) * N
        for x, y in [(0, 0), (1, 1), (N - 1, N - 1), (hi - 1, hi - 1), (hi - 1, 2 * hi - 1)] + \
                    [(r.randrange(hi), r.randrange(hi)) for _ in range(6)]:
            _mm_check(key, x, y)


def test_mm_exhaustive_tiny_bases():
    # 8-bit channel primes, 12-bit class: every x, y below N for several moduli
    c = rns.make_class(12, fixed_bound=256)
    assert c.k == 3
    for N in (3, 5, 7, 9, 15, 17, 33, 35, 63, 101):
        key = rns.make_key(c, N)
        for x in range(N):
            for y in range(N):
                _mm_check(key, x, y)


def test_mm_random_tiny_bases_extended_range():
    c = rns.make_class(12, fixed_bound=256)
    r = random.Random(4)
    for N in (4093, 4091, 2049, 3001, 255):
        key = rns.make_key(c, N)
        hi = (c.k + 1) * N
        for _ in range(3000):
            _mm_check(key, r.randrange(2 * hi), r.randrange(2 * hi))


def test_modexp_exhaustive_tiny():
    c = rns.make_class(12, fixed_bound=256)
    for N in (3, 25, 77, 255, 4091):
        key = rns.make_key(c, N)
        xs = range(N) if N < 100 else [0, 1, 2, N - 1, N // 2, 1234 % N]
        for x in xs:
            for e in range(0, 40):
                for w in (1, 3):
                    assert rns.modexp(key, x, e, w) == pow(x, e, N), (N, x, e, w)


@pytest.mark.parametrize("L", [512, 1024])
def test_modexp_matches_plain(L):
    c = rns.make_class(L)
    r = SplitMix64(L)
    for _ in range(3):
        N = r.randbits(L) | 1 | (1 << (L - 1))
        key = rns.make_key(c, N)
        for x, e in [(0, 5), (1, 7), (N - 1, 3), (r.below(N), 0), (r.below(N), 1),
                     (r.below(N), 65537), (r.below(N), r.randbits(L))]:
            assert rns.modexp(key, x, e) == plain.modexp(x, e, N)


def test_two_chunk_entry_and_crt_decrypt():
    for k in load_keys("test_small")[:4] + load_keys("rsa2048_x16")[:1]:
        half = k["bits"] // 2
        c = rns.make_class(((half + 31) // 32) * 32)
        kp, kq = rns.make_key(c, k["p"]), rns.make_key(c, k["q"])
        r = SplitMix64(k["N"] & 0xFFFFFFFF)
        for ct in (0, 1, k["N"] - 1, r.below(k["N"])):
            assert rns.rsa_decrypt_crt(kp, kq, ct, k["dp"], k["dq"], k["qinv"]) == pow(ct, k["d"], k["N"])


def test_rejects_bad_moduli():
    c = rns.make_class(512)
    with pytest.raises(ValueError):
        rns.make_key(c, 1 << 100)            # even
    with pytest.raises(ValueError):
        rns.make_key(c, (1 << 600) + 1)      # too long for the class
    with pytest.raises(ValueError):
        rns.make_key(c, c.B[0] * 3)          # shares a channel prime


def test_pins_catch_planted_mistakes(monkeypatch):
    """Dropping the q*N term's constant or the B'->B correction must fail the pins."""
    c = rns.make_class(512)
    key = rns.make_key(c, (1 << 511) + 187)
    good = key.t["NMinv_Bp"][3]
    key.t["NMinv_Bp"][3] = (good + 1) % c.Bp[3]
    with pytest.raises((AssertionError, ArithmeticError)):
        _mm_check(key, 12345678901234567, 98765432109876543)
    key.t["NMinv_Bp"][3] = good
    saved = c.t["Mp_B"][0]
    c.t["Mp_B"][0] = 0
    try:
        with pytest.raises((AssertionError, ArithmeticError)):
            for s in range(20):
                _mm_check(key, 3 ** 300 + s, 5 ** 200 + s)
    finally:
        c.t["Mp_B"][0] = saved
