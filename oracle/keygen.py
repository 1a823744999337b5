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
