"""Plain definitions of what the GPU path computes (test infrastructure only).

Everything is exact arithmetic on Python integers.  No residue number system,
no Montgomery form, nothing shared with the CUDA library.
"""
from __future__ import annotations


def modexp(x: int, e: int, N: int) -> int:
    """x^e mod N, in [0, N), by left-to-right binary square-and-multiply.

    Sec. 3.1 names "traditional square-and-multiply" for exponentiation; this is
    that algorithm on ordinary integers (scan e from its top bit: square, then
    multiply when the bit is set).  0^0 is taken as 1, and N = 1 gives 0.
    """
    if N <= 0:
        raise ValueError("modulus must be positive")
    if e < 0:
        raise ValueError("exponent must be non-negative")
    x %= N
    r = 1 % N
    for bit in range(e.bit_length() - 1, -1, -1):
        r = (r * r) % N
        if (e >> bit) & 1:
            r = (r * x) % N
    return r


def egcd(a: int, b: int):
    """Extended Euclid: (g, s, t) with s*a + t*b = g = gcd(a, b) >= 0."""
    s0, s1, t0, t1 = 1, 0, 0, 1
    while b:
        q, r = divmod(a, b)
        a, b = b, r
        s0, s1 = s1, s0 - q * s1
        t0, t1 = t1, t0 - q * t1
    if a < 0:
        a, s0, t0 = -a, -s0, -t0
    return a, s0, t0


def gcd(a: int, b: int) -> int:
    return egcd(a, b)[0]


def inverse(a: int, m: int) -> int:
    """a^-1 mod m by extended Euclid; ValueError when gcd(a, m) != 1."""
    if m <= 0:
        raise ValueError("modulus must be positive")
    g, s, _ = egcd(a % m, m)
    if g != 1:
        raise ValueError("not invertible")
    return s % m


def arazi_inverse(e: int, f: int) -> int:
    """d = e^-1 mod f for coprime e, f by Arazi's formula (Sec. 3.1).

    d = (1 + f * (-f^-1 mod e)) / e.  The only inverse taken is of f modulo the
    small number e; the division by e is exact because 1 + f*(-f^-1) is
    divisible by e by construction.  The result lies in [1, f) for e < f.
    """
    if e <= 0 or f <= 0:
        raise ValueError("arguments must be positive")
    if e == 1:
        return 1 % f
    t = (-inverse(f % e, e)) % e
    num = 1 + f * t
    d, rem = divmod(num, e)
    if rem:
        raise ValueError("e and f are not coprime")
    return d % f


def rsa_encrypt(m: int, e: int, N: int) -> int:
    """c = m^e mod N (Sec. 3.3: encryption applies modular exponentiation to each block)."""
    return modexp(m, e, N)


def rsa_decrypt(c: int, d: int, N: int) -> int:
    """m = c^d mod N, the plain definition of RSA decryption (Sec. 3.3)."""
    return modexp(c, d, N)


def rsa_decrypt_crt(c: int, p: int, q: int, dp: int, dq: int, qinv: int) -> int:
    """RSA decryption through the Chinese remainder theorem (Garner's recombination).

    m_p = c^dp mod p, m_q = c^dq mod q, h = qinv*(m_p - m_q) mod p, m = m_q + h*q,
    with dp = d mod (p-1), dq = d mod (q-1), qinv = q^-1 mod p.  The result equals
    c^d mod pq because pq is squarefree (the CRT, Sec. 3.1); tests pin that.
    """
    mp = modexp(c % p, dp, p)
    mq = modexp(c % q, dq, q)
    h = (qinv * (mp - mq)) % p
    return mq + h * q


def message_block_bytes(N: int) -> int:
    """Bytes per message block for modulus N: the largest whole number of bytes whose values all
    lie below N, (bits(N) - 1) // 8 (Sec. 3.3 splits messages into blocks of the key's length;
    the paper does not say how a block is kept below N: this is our reading)."""
    return (N.bit_length() - 1) // 8


def message_blocks(msg: bytes, N: int) -> list:
    """A byte string as integers below N: consecutive blocks of message_block_bytes(N) bytes (the
    last one shorter), each read little-endian (the library's limb order)."""
    B = message_block_bytes(N)
    if B < 1:
        raise ValueError("modulus too small")
    return [int.from_bytes(msg[i:i + B], "little") for i in range(0, len(msg), B)]


def message_from_blocks(blocks, N: int, length: int) -> bytes:
    """Inverse of message_blocks for a message of `length` bytes."""
    B = message_block_bytes(N)
    out = b"".join(int(v).to_bytes(B, "little") for v in blocks)
    return out[:length]


def rsa_private_parts(p: int, q: int, e: int) -> dict:
    """d = e^-1 mod (p-1)(q-1) (Sec. 3.3), by Arazi's formula (Sec. 3.1), and the CRT parts."""
    phi = (p - 1) * (q - 1)
    d = arazi_inverse(e, phi)
    return {"d": d, "dp": d % (p - 1), "dq": d % (q - 1), "qinv": inverse(q, p)}
