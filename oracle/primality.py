"""Primality tests of the key-generation tier (test infrastructure only).

Sec. 3.2: random candidates are tested with a Miller-Rabin test whose number of
iterations is a parameter.  Sec. 4.3: candidates are first sieved by trial
division with the first 10,000 primes.
"""
from __future__ import annotations

from functools import lru_cache
from typing import List, Sequence

from .plain import modexp


@lru_cache(maxsize=None)
def first_primes(count: int = 10000) -> tuple:
    """The first ``count`` primes, by a sieve of Eratosthenes (the 10,000th prime is 104729)."""
    limit = 16
    while True:
        sieve = bytearray([1]) * (limit + 1)
        sieve[0] = sieve[1] = 0
        i = 2
        while i * i <= limit:
            if sieve[i]:
                sieve[i * i:: i] = bytearray(len(sieve[i * i:: i]))
            i += 1
        primes = [i for i in range(limit + 1) if sieve[i]]
        if len(primes) >= count:
            return tuple(primes[:count])
        limit *= 2


def trial_division_passes(n: int, count: int = 10000) -> bool:
    """True when no prime among the first ``count`` divides n (or n is one of them)."""
    for p in first_primes(count):
        if p * p > n:
            return n > 1
        if n % p == 0:
            return n == p
    return True


def is_prime_by_trial(n: int) -> bool:
    """Brute-force primality by trial division up to sqrt(n): the textbook definition."""
    if n < 2:
        return False
    if n % 2 == 0:
        return n == 2
    f = 3
    while f * f <= n:
        if n % f == 0:
            return False
        f += 2
    return True


def decompose(n_minus_1: int):
    """n - 1 = 2^s * d with d odd."""
    s = 0
    d = n_minus_1
    while d % 2 == 0:
        d //= 2
        s += 1
    return s, d


def miller_rabin_round(n: int, a: int) -> bool:
    """One Miller-Rabin round with witness a: True = "probable prime" for this witness.

    For odd n >= 3 write n - 1 = 2^s d (d odd) and y = (a mod n)^d mod n; n passes
    for a when y is 1 or n - 1, or when y^(2^r) = n - 1 for some 0 < r < s.
    Witnesses are meant to lie in [2, n-2]; other values go through the same steps
    (a = 0 mod n gives "composite", a = +-1 mod n gives "probable prime").
    n = 2 is prime; even n and n < 2 are composite by definition.
    """
    if n == 2:
        return True
    if n < 2 or n % 2 == 0:
        return False
    s, d = decompose(n - 1)
    y = modexp(a % n, d, n)
    if y == 1 or y == n - 1:
        return True
    for _ in range(s - 1):
        y = (y * y) % n
        if y == n - 1:
            return True
    return False


def miller_rabin(n: int, witnesses: Sequence[int]) -> List[bool]:
    """Per-witness verdicts; n is a probable prime when all are True."""
    return [miller_rabin_round(n, a) for a in witnesses]


def prime_test_verdict(n: int, witnesses: Sequence[int], count: int = 10000) -> int:
    """The key-generation primality test: trial division by the first ``count`` primes
    (Sec. 4.3), then the Miller-Rabin rounds (Sec. 3.2) for candidates that pass it.

    0 = fails trial division, 1 = passes it and some round fails, 2 = passes every round.
    """
    if not trial_division_passes(n, count):
        return 0
    return 2 if all(miller_rabin(n, witnesses)) else 1
