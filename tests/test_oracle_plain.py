"""Pins for oracle.plain: each check is independent of the function it tests.

Pins used: CPython's pow() (a library routine), the definition of a power as a
repeated product (brute force on tiny inputs), Fermat's and Euler's theorems,
exponent laws, the RSA round trip, CRT consistency and Arazi's defining identity.
"""
import random

import pytest

from oracle import plain
from synth import SplitMix64, load_keys


def _rand_cases(seed, bits, n):
    r = random.Random(seed)
    out = []
    for _ in range(n):
        N = r.getrandbits(bits) | 1 | (1 << (bits - 1))
        out.append((r.getrandbits(bits) % N, r.getrandbits(bits), N))
    return out


@pytest.mark.parametrize("bits", [8, 64, 512, 1024])
def test_modexp_matches_library_pow(bits):
    for x, e, N in _rand_cases(bits, bits, 40 if bits <= 512 else 8):
        assert plain.modexp(x, e, N) == pow(x, e, N)


def test_modexp_brute_force_tiny():
    # power as repeated product, reduced at the end: the definition itself
    for N in range(1, 40):
        for x in range(0, N + 3):
            prod = 1
            for e in range(0, 12):
                assert plain.modexp(x, e, N) == prod % N, (x, e, N)
                prod *= x


def test_modexp_edge_cases():
    N = (1 << 127) - 1
    assert plain.modexp(0, 0, N) == 1
    assert plain.modexp(0, 5, N) == 0
    assert plain.modexp(1, 12345, N) == 1
    assert plain.modexp(5, 1, N) == 5
    assert plain.modexp(N - 1, 3, N) == N - 1        # (-1)^odd
    assert plain.modexp(N - 1, 10, N) == 1           # (-1)^even
    assert plain.modexp(7, 0, 1) == 0                # everything is 0 mod 1
    with pytest.raises(ValueError):
        plain.modexp(2, -1, 5)


def test_fermat_on_mersenne_primes():
    for p_exp in (127, 521, 607):
        p = (1 << p_exp) - 1
        r = random.Random(p_exp)
        for _ in range(3):
            a = r.randrange(2, p - 1)
            assert plain.modexp(a, p - 1, p) == 1


def test_exponent_law_and_euler():
    keys = load_keys("test_small")
    r = random.Random(11)
    for k in keys:
        N, p, q = k["N"], k["p"], k["q"]
        phi = (p - 1) * (q - 1)
        for _ in range(3):
            x = r.randrange(2, N - 1)
            a, b = r.getrandbits(300), r.getrandbits(200)
            assert plain.modexp(x, a + b, N) == (plain.modexp(x, a, N) * plain.modexp(x, b, N)) % N
            if plain.gcd(x, N) == 1:
                assert plain.modexp(x, phi, N) == 1


def test_inverse_and_arazi():
    r = random.Random(3)
    for e in (3, 5, 17, 257, 65537):
        for _ in range(30):
            f = r.getrandbits(r.choice([16, 64, 512, 2048])) | 2
            if plain.gcd(e, f) != 1:
                continue
            d = plain.arazi_inverse(e, f)
            assert 0 < d < f
            assert (d * e) % f == 1
            assert d == pow(e, -1, f)
            assert plain.inverse(e, f) == pow(e, -1, f)
    with pytest.raises(ValueError):
        plain.arazi_inverse(3, 9)
    with pytest.raises(ValueError):
        plain.inverse(6, 9)


def test_stored_keys_are_consistent():
    for name in ("test_small", "rsa1024_x64", "rsa2048_x16"):
        for k in load_keys(name):
            N, e, p, q, d = k["N"], k["e"], k["p"], k["q"], k["d"]
            assert N == p * q and N.bit_length() == k["bits"] and p != q
            phi = (p - 1) * (q - 1)
            assert (d * e) % phi == 1
            assert k["dp"] == d % (p - 1) and k["dq"] == d % (q - 1)
            assert (k["qinv"] * q) % p == 1
            # probable primality by the library routine (Fermat, several bases)
            for a in (2, 3, 5, 7):
                assert pow(a, p - 1, p) == 1 and pow(a, q - 1, q) == 1


def test_rsa_roundtrip_and_crt():
    r = SplitMix64(99)
    for k in load_keys("test_small") + load_keys("rsa1024_x64")[:4] + load_keys("rsa2048_x16")[:2]:
        N = k["N"]
        for m in (0, 1, N - 1, r.below(N), r.below(N)):
            c = plain.rsa_encrypt(m, k["e"], N)
            assert c == pow(m, k["e"], N)
            m1 = plain.rsa_decrypt(c, k["d"], N)
            m2 = plain.rsa_decrypt_crt(c, k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
            assert m1 == m == m2
            assert m2 % k["p"] == pow(c, k["dp"], k["p"])     # CRT consistency
        # a ciphertext sharing a factor with N still decrypts (N squarefree)
        c = k["p"] * 5 % N
        assert plain.rsa_decrypt_crt(c, k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) == pow(c, k["d"], N)


def test_pins_catch_planted_mistakes(monkeypatch):
    """A plausible slip in modexp (multiply before squaring) must fail a pin."""
    def wrong(x, e, N):
        x %= N
        r = 1 % N
        for bit in range(e.bit_length() - 1, -1, -1):
            if (e >> bit) & 1:
                r = (r * x) % N
            r = (r * r) % N
        return r
    monkeypatch.setattr(plain, "modexp", wrong)
    with pytest.raises(AssertionError):
        test_modexp_matches_library_pow(64)


def test_message_blocks_round_trip_and_bounds():
    """Blocks are below N, cover the message in order, the last one shorter; the byte string comes
    back from the blocks; RSA on the blocks round-trips; the empty message has no blocks."""
    from synth import SplitMix64
    r = SplitMix64(0x6D7367)
    for bits in (17, 64, 1024, 2051):
        N = r.randbits(bits) | 1 | (1 << (bits - 1))
        B = plain.message_block_bytes(N)
        assert 256 ** B <= N < 256 ** (B + 2)
        for length in (0, 1, B - 1, B, B + 1, 5 * B + 3):
            msg = bytes(r.below(256) for _ in range(length))
            blocks = plain.message_blocks(msg, N)
            assert len(blocks) == -(-length // B)
            assert all(0 <= v < N for v in blocks)
            assert plain.message_from_blocks(blocks, N, length) == msg
    assert plain.message_blocks(b"\x01\x02\x03", (1 << 17) + 1) == [0x0201, 0x03]
