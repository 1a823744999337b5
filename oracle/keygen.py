"""Seeded RSA key generation for the synthetic workloads (test infrastructure only).

Sec. 3.2 / 3.3 / 4.3: a random candidate is sieved by trial division with the
first 10,000 primes, then tested by Miller-Rabin with a chosen number of rounds;
N = pq, d = e^-1 mod (p-1)(q-1).  The paper's random bits come from its hardware
generator; here they come from the seeded SplitMix64 stream in ``synth`` so that
keys are reproducible.

Candidate recipe: draw bits/2 random bits, set the two top bits (so that pq has
exactly ``bits`` bits) and bit 0; sieve; then 40 Miller-Rabin rounds with
witnesses uniform in [2, n-2] from the same stream.  A prime p is kept only when
gcd(e, p-1) = 1; q is redrawn until q != p.
"""
from __future__ import annotations

from synth import SplitMix64

from .plain import gcd, rsa_private_parts
from .primality import miller_rabin_round, trial_division_passes


def gen_prime(rng: SplitMix64, bits: int, rounds: int = 40, e: int | None = None) -> int:
    if bits < 4:
        raise ValueError("bits too small")
    while True:
        n = rng.randbits(bits) | (3 << (bits - 2)) | 1
        if not trial_division_passes(n):
            continue
        if e is not None and gcd(e, n - 1) != 1:
            continue
        ok = True
        for _ in range(rounds):
            a = rng.between(2, n - 2)
            if not miller_rabin_round(n, a):
                ok = False
                break
        if ok:
            return n


def first_usable_prime(pool, witnesses, e: int, count: int = 10000, exclude: int | None = None):
    """The first candidate of ``pool`` that passes trial division by the first ``count`` primes
    and every Miller-Rabin round with its witnesses (Sec. 4.3, Sec. 3.2), has gcd(e, n-1) = 1
    and differs from ``exclude``; None when there is none."""
    from .primality import prime_test_verdict
    for n, ws in zip(pool, witnesses):
        if n == exclude or gcd(e, n - 1) != 1:
            continue
        if prime_test_verdict(n, ws, count) == 2:
            return n
    return None


def rsa_key_from_pools(p_pool, p_witnesses, q_pool, q_witnesses, e: int = 65537, count: int = 10000):
    """RSA key from given candidate pools (Sec. 3.3): p is the first usable prime of the p pool, q
    the first of the q pool other than p; N = pq and the private parts by Arazi's inversion
    (rsa_private_parts).  None when a pool holds no usable prime."""
    p = first_usable_prime(p_pool, p_witnesses, e, count)
    if p is None:
        return None
    q = first_usable_prime(q_pool, q_witnesses, e, count, exclude=p)
    if q is None:
        return None
    key = {"N": p * q, "e": e, "p": p, "q": q}
    key.update(rsa_private_parts(p, q, e))
    return key


def gen_rsa_key(rng: SplitMix64, bits: int, e: int = 65537, rounds: int = 40) -> dict:
    """A seeded RSA key of exactly ``bits`` bits with primes of bits/2 bits each."""
    half = bits // 2
    p = gen_prime(rng, half, rounds, e)
    while True:
        q = gen_prime(rng, bits - half, rounds, e)
        if q != p:
            break
    N = p * q
    assert N.bit_length() == bits
    key = {"bits": bits, "N": N, "e": e, "p": p, "q": q}
    key.update(rsa_private_parts(p, q, e))
    return key
