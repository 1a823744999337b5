"""Pins for oracle.primality against published facts and brute force."""
import os
import random

import pytest

from oracle import keygen, primality
from oracle.plain import gcd
from synth import SplitMix64, load_keys

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_first_primes_published():
    for line in open(os.path.join(GOLD, "primes.txt")):
        f = line.split()
        if f and f[0] == "nth":
            assert primality.first_primes(int(f[1]))[-1] == int(f[2])
    ps = primality.first_primes(10000)
    assert len(ps) == 10000 and ps[:5] == (2, 3, 5, 7, 11)


def test_trial_division_matches_brute_force():
    for n in range(0, 5000):
        assert primality.trial_division_passes(n) == primality.is_prime_by_trial(n) or n < 2


def _smallest_factor(n):
    f = 2
    while f * f <= n:
        if n % f == 0:
            return f
        f += 1
    return n


def test_trial_division_short_lists_brute_force():
    """With the first `count` primes only, n passes exactly when n >= 2 and its smallest prime
    factor is n itself or exceeds the count-th prime (smallest factors found by brute force)."""
    for count, last in ((1, 2), (10, 29), (100, 541)):
        assert primality.first_primes(count)[-1] == last
        for n in range(0, 3000):
            want = n >= 2 and (_smallest_factor(n) == n or _smallest_factor(n) > last)
            assert primality.trial_division_passes(n, count) == want, (count, n)


def test_prime_test_verdict_cases():
    """Verdict 0 for small factors, 1 for composites without listed factors that a round
    catches, 2 for primes; primes above the list pass trial division."""
    w = [2, 3, 5, 7, 11, 13]
    assert [primality.prime_test_verdict(n, w) for n in (0, 1, 2, 17, 4, 9, 104729)] == [0, 0, 2, 2, 0, 0, 2]
    p10001 = 104743  # the 10,001st prime: not in the list
    assert primality.prime_test_verdict(p10001, w) == 2
    assert primality.prime_test_verdict(p10001 * p10001, w) == 1        # no listed factor
    assert primality.prime_test_verdict(p10001 * 104759, w) == 1
    assert primality.prime_test_verdict(104729 * p10001, w) == 0        # a listed factor
    assert primality.prime_test_verdict(p10001 * p10001, w, count=1) == 1
    assert primality.prime_test_verdict(3 * p10001, w, count=1) == 1    # 3 is not listed with count 1
    assert primality.prime_test_verdict(3 * p10001, w, count=2) == 0
    # 3215031751 = 151 * 751 * 28351 is a strong pseudoprime to bases 2, 3, 5, 7 (published):
    # Miller-Rabin alone passes it, the trial division (151 is listed) does not
    assert all(primality.miller_rabin(3215031751, [2, 3, 5, 7]))
    assert primality.prime_test_verdict(3215031751, [2, 3, 5, 7]) == 0


def test_key_from_pools_selection_and_identities():
    """Pool selection: composites, a prime with e | p-1 and a repeat of p are skipped; the key's
    parts satisfy the RSA identities (e d = 1 mod (p-1)(q-1), dp/dq, q qinv = 1 mod p, and
    decryption inverts encryption)."""
    ws = lambda pool: [[2, 3, 5, 7] for _ in pool]
    e = 3
    # 7: 3 | 7-1 (skipped for e = 3); 9, 15: composite; 11: first usable p; q pool: 11 repeats p, 13: 3 | 12
    key = keygen.rsa_key_from_pools([9, 7, 15, 11, 23], ws(range(5)), [11, 13, 17, 29], ws(range(4)), e)
    assert (key["p"], key["q"]) == (11, 17)
    assert keygen.rsa_key_from_pools([9, 15, 21], ws(range(3)), [17], ws(range(1)), e) is None
    r = SplitMix64(0x6B65)
    pool_p = [r.randbits(256) | (3 << 254) | 1 for _ in range(400)]
    pool_q = [r.randbits(256) | (3 << 254) | 1 for _ in range(400)]
    wp = [[r.between(2, n - 2) for _ in range(8)] for n in pool_p]
    wq = [[r.between(2, n - 2) for _ in range(8)] for n in pool_q]
    k = keygen.rsa_key_from_pools(pool_p, wp, pool_q, wq, 65537)
    assert k is not None
    p, q, d = k["p"], k["q"], k["d"]
    assert primality.is_prime_by_trial(p) if p < 1 << 40 else pow(2, p - 1, p) == 1
    assert k["N"] == p * q and (k["e"] * d) % ((p - 1) * (q - 1)) == 1
    assert k["dp"] == d % (p - 1) and k["dq"] == d % (q - 1) and (k["qinv"] * q) % p == 1
    m = r.below(k["N"])
    assert pow(pow(m, 65537, k["N"]), d, k["N"]) == m


def test_miller_rabin_exhaustive_below_2_16():
    # Bases {2,3,5,7} decide primality exactly below 3,215,031,751 (published bound).
    # (n > 7 so that no base is a multiple of n)
    for n in range(9, 1 << 16, 2):
        mr = all(primality.miller_rabin(n, [2, 3, 5, 7]))
        assert mr == primality.is_prime_by_trial(n), n


def test_miller_rabin_all_witnesses_small():
    # A prime passes every witness; an odd composite n > 9 has at most phi(n)/4
    # strong liars (Monier-Rabin bound).
    for n in range(5, 400, 2):
        passed = sum(primality.miller_rabin_round(n, a) for a in range(2, n - 1))
        if primality.is_prime_by_trial(n):
            assert passed == n - 3
        elif n > 9:
            phi = sum(1 for a in range(1, n) if gcd(a, n) == 1)
            assert passed + 2 <= phi / 4  # liars in [1, n-1]: the range plus 1 and n-1


def test_strong_pseudoprimes_published():
    for line in open(os.path.join(GOLD, "strong_pseudoprimes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        n, passed, failed = line.split()
        n = int(n)
        if passed != "-":
            for a in map(int, passed.split(",")):
                assert primality.miller_rabin_round(n, a), (n, a)
        assert not primality.miller_rabin_round(n, int(failed)), (n, failed)


def test_mersenne_primes_pass_every_witness():
    r = random.Random(5)
    for line in open(os.path.join(GOLD, "primes.txt")):
        f = line.split()
        if f and f[0] == "mersenne" and int(f[1]) <= 607:
            p = (1 << int(f[1])) - 1
            assert all(primality.miller_rabin(p, [r.randrange(2, p - 1) for _ in range(4)]))


def test_products_of_generated_primes_fail():
    for k in load_keys("test_small") + load_keys("rsa1024_x64")[:4]:
        N = k["N"]
        r = random.Random(N & 0xFFFF)
        assert not all(primality.miller_rabin(N, [r.randrange(2, N - 1) for _ in range(3)]))
        assert all(primality.miller_rabin(k["p"], [2, 3, 5]))


def test_witness_edge_values():
    p = 1000003
    assert primality.miller_rabin_round(p, 1) and primality.miller_rabin_round(p, p - 1)
    assert not primality.miller_rabin_round(p, 0) and not primality.miller_rabin_round(p, p)
    assert primality.miller_rabin_round(2, 5) and not primality.miller_rabin_round(9, 2)


def test_keygen_deterministic_and_well_formed():
    a = keygen.gen_rsa_key(SplitMix64(1).fork(0), 256)
    b = keygen.gen_rsa_key(SplitMix64(1).fork(0), 256)
    assert a == b
    assert a["N"].bit_length() == 256
    assert a["p"].bit_length() == 128 and a["q"].bit_length() == 128
    for prime in (a["p"], a["q"]):
        assert primality.is_prime_by_trial(prime) if prime < 1 << 40 else pow(3, prime - 1, prime) == 1
