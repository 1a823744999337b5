"""Slow step-by-step model of RNS Montgomery multiplication (test infrastructure only).

Sec. 3.1 of the paper: a bignum X is held as its residues x_i = X mod m_i over
pairwise coprime moduli (unique for X < M = prod m_i by the CRT); products are
taken channel by channel; the Montgomery multiplication with R = M computes
X*Y*M^-1 mod N channel-wise (Bajard et al. 2001) using a second base B' and a
base extension whose constants depend only on the bases; exponentiation chains
these multiplications inside the Montgomery domain.  This module writes those
steps out on Python integers, in the order the method takes them, with no
blocking or fusion.  It fixes the base choice and every precomputed constant so
that the CUDA library's own tables can be checked against it value by value.

Readings where the paper is silent (each also recorded in the design notes):

* Bases.  For a size class of L bits and k channels per base, every channel
  prime lies below b_k = min(2^31, isqrt((2^64-1) // k)), so that a sum of k
  products of two residues never reaches 2^64.  B = the k largest primes below
  b_k, B' = the next k primes.  k is the smallest integer with
  M >= 4 (k+1)^2 2^L and M' >= 2 (k+1) 2^L.
* Extension B -> B' is the fast one without correction (the extended value is
  q + a*M with 0 <= a < k).  Extension B' -> B is exact: its correction factor
  a' = floor(sum_j xi'_j / m'_j) is computed in fixed point (Kawamura et al.,
  CHES 2000): a' = (sum_j floor(xi'_j floor(2^(32+Q)/m'_j) / 2^32) + 2^(Q-2)) >> Q
  with Q = 22, which equals the exact value whenever the extended number is
  below 3/4 M' (guaranteed by the M' bound above); the model also computes the
  exact factor from its definition and checks that the two agree.
* RNS -> binary uses the same fixed-point factor over B (the value is below M/4).
* Every multiplication output lies in [0, (k+1) N); only the final result is
  reduced to [0, N).
* Inputs longer than the class are split into L-bit chunks x = x_lo + 2^L x_hi
  and entered as MM(x_lo, M^2 mod N) + MM(x_hi, 2^L M^2 mod N) (at most 2 chunks).
* Exponentiation: fixed 2^w-ary windows from the top, w squarings then one
  multiplication by the table entry (entry 0 is the Montgomery form of 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from functools import lru_cache
from math import isqrt
from typing import Dict, List, Optional, Sequence

from .plain import inverse
from .primality import first_primes

PRIME_CAP = 1 << 31
KAW_Q = 22          # fixed-point bits of the correction-factor estimate


def prime_bound(k: int) -> int:
    """Channel primes stay below this, so that k products of residues sum below 2^64."""
    return min(PRIME_CAP, isqrt(((1 << 64) - 1) // k))


@lru_cache(maxsize=None)
def primes_below(bound: int, count: int) -> tuple:
    """The ``count`` largest primes strictly below ``bound``, in descending order.

    Sieve of Eratosthenes over windows [lo, hi) just below the bound, striking the
    multiples of every prime up to isqrt(bound); windows move down until enough
    primes are found."""
    small = [p for p in first_primes(5000) if p * p < bound]  # up to 48611, enough below 2^31
    out = []
    hi = bound
    span = max(1024, 64 * count)
    while len(out) < count:
        lo = max(2, hi - span)
        if hi <= 2:
            raise ValueError("not enough primes below bound")
        alive = [True] * (hi - lo)
        for p in small:
            start = max(p * p, ((lo + p - 1) // p) * p)
            for mult in range(start, hi, p):
                alive[mult - lo] = False
        for n in range(hi - 1, lo - 1, -1):
            if alive[n - lo]:
                out.append(n)
                if len(out) == count:
                    break
        hi = lo
    return tuple(out)


def _prod(xs: Sequence[int]) -> int:
    r = 1
    for x in xs:
        r *= x
    return r


@dataclass
class RNSClass:
    """Bases and class-wide constants for moduli of at most L bits."""
    L: int
    k: int
    B: List[int]
    Bp: List[int]
    M: int
    Mp: int
    bound: int
    t: Dict[str, object] = field(default_factory=dict)


def class_k(L: int, fixed_bound: Optional[int] = None) -> int:
    """Smallest k meeting M >= 4 (k+1)^2 2^L and M' >= 2 (k+1) 2^L.

    Every channel prime is below 2^31, so M < 2^(31k) and M >= 2^L needs k > L/31:
    the search starts there."""
    k = max(1, L // 31)
    while True:
        b = fixed_bound if fixed_bound is not None else prime_bound(k)
        pr = primes_below(b, 2 * k)
        M = _prod(pr[:k])
        Mp = _prod(pr[k:2 * k])
        if M >= 4 * (k + 1) ** 2 * (1 << L) and Mp >= 2 * (k + 1) * (1 << L):
            return k
        k += 1


def fixed_point_factor(xi: Sequence[int], mods: Sequence[int]) -> int:
    """floor(sum xi_j / m_j) estimated in Q-bit fixed point with a 1/4 offset (Kawamura)."""
    acc = 0
    for x, m in zip(xi, mods):
        u = (1 << (32 + KAW_Q)) // m
        acc += (x * u) >> 32
    return (acc + (1 << (KAW_Q - 2))) >> KAW_Q


@lru_cache(maxsize=None)
def make_class(L: int, fixed_bound: Optional[int] = None) -> RNSClass:
    """Base choice and the constants that stay fixed for every modulus of the class (Sec. 3.1).

    ``fixed_bound`` replaces the per-k prime bound (tests use tiny 8-bit bases).
    """
    k = class_k(L, fixed_bound)
    b = fixed_bound if fixed_bound is not None else prime_bound(k)
    pr = primes_below(b, 2 * k)
    B, Bp = list(pr[:k]), list(pr[k:2 * k])
    M, Mp = _prod(B), _prod(Bp)
    c = RNSClass(L=L, k=k, B=B, Bp=Bp, M=M, Mp=Mp, bound=b)
    t = c.t
    # B -> B' extension: |M/m_i|_{m'_j}, |(M/m_i)^-1|_{m_i}
    t["M_mi_inv"] = [inverse(M // m, m) for m in B]
    t["M_mi_Bp"] = [[(M // m) % mp for mp in Bp] for m in B]
    # Montgomery division by M in B'
    t["Minv_Bp"] = [inverse(M % mp, mp) for mp in Bp]
    # B' -> B extension: |(M'/m'_j)^-1|_{m'_j}, |M'/m'_j|_{m_i}, |M'|_{m_i}
    t["Mp_mj_inv"] = [inverse(Mp // mp, mp) for mp in Bp]
    t["Mp_mj_B"] = [[(Mp // mp) % m for m in B] for mp in Bp]
    t["Mp_B"] = [Mp % m for m in B]
    return c


@dataclass
class RNSValue:
    b: List[int]
    bp: List[int]


def to_rns(c: RNSClass, X: int) -> RNSValue:
    """Residues of a non-negative integer in B and B' (the definition, Sec. 3.1)."""
    return RNSValue([X % m for m in c.B], [X % m for m in c.Bp])


def crt_value(c: RNSClass, v: RNSValue) -> int:
    """RNS -> binary with the CRT (Sec. 3.1).

    X = sum_i xi_i (M/m_i) - a M with xi_i = |x_i (M/m_i)^-1|_{m_i} and
    a = floor(sum xi_i/m_i).  a is taken from the fixed-point estimate, which is
    exact for X < 3M/4; the exact value is checked against it.
    """
    t = c.t
    xi = [(v.b[i] * t["M_mi_inv"][i]) % c.B[i] for i in range(c.k)]
    total = sum(xi[i] * (c.M // c.B[i]) for i in range(c.k))
    a_exact = total // c.M
    a = fixed_point_factor(xi, c.B)
    if a != a_exact:
        raise ArithmeticError("fixed-point CRT factor differs from the exact one (value not below 3M/4)")
    return total - a * c.M


@dataclass
class RNSKey:
    cls: RNSClass
    N: int
    t: Dict[str, object] = field(default_factory=dict)


def make_key(c: RNSClass, N: int) -> RNSKey:
    """Per-modulus constants (Sec. 3.1): everything that depends on N."""
    if N < 3 or N % 2 == 0:
        raise ValueError("modulus must be odd and >= 3")
    if N.bit_length() > c.L:
        raise ValueError("modulus larger than the class")
    for m in c.B + c.Bp:
        if N % m == 0:
            raise ValueError("modulus shares a factor with a channel")
    key = RNSKey(cls=c, N=N)
    t = key.t
    M = c.M
    # xi_i = s_i * |-N^-1 (M/m_i)^-1|_{m_i}
    t["kxi"] = [(-inverse(N % m, m) * c.t["M_mi_inv"][i]) % m for i, m in enumerate(c.B)]
    # r_j = s_j |M^-1| + qhat_j |N M^-1|
    t["NMinv_Bp"] = [(N * c.t["Minv_Bp"][j]) % mp for j, mp in enumerate(c.Bp)]
    # Montgomery-domain constants
    t["one"] = to_rns(c, M % N)                      # 1 in the Montgomery domain
    t["r2"] = to_rns(c, (M * M) % N)                 # entry: MM(x, M^2 mod N) = xM mod N
    t["r2h"] = to_rns(c, ((M * M) << c.L) % N)       # entry of the high chunk of a 2L-bit input
    return key


def mm(key: RNSKey, x: RNSValue, y: RNSValue) -> RNSValue:
    """RNS Montgomery multiplication: r = (xy + qhat N)/M, r == x y M^-1 (mod N).

    Steps in order:
      1. s = x*y in every channel of B and B';
      2. xi_i = s_i |-N^-1 (M/m_i)^-1|_{m_i} in B  (so q = sum xi_i M/m_i == -s N^-1 mod M);
      3. extension B -> B': qhat_j = sum_i xi_i |M/m_i|_{m'_j}  (qhat = q + a M, 0 <= a < k);
      4. r_j = s_j |M^-1|_{m'_j} + qhat_j |N M^-1|_{m'_j} in B'  (r = (s + qhat N)/M);
      5. xi'_j = r_j |(M'/m'_j)^-1|_{m'_j};
      6. extension B' -> B (exact): t_i = sum_j xi'_j |M'/m'_j|_{m_i},
         a' = floor(sum_j xi'_j / m'_j) in fixed point, r_i = t_i - a' |M'|_{m_i}.
    """
    c, t, kt = key.cls, key.cls.t, key.t
    k = c.k
    s_b = [(x.b[i] * y.b[i]) % c.B[i] for i in range(k)]
    s_bp = [(x.bp[j] * y.bp[j]) % c.Bp[j] for j in range(k)]
    xi = [(s_b[i] * kt["kxi"][i]) % c.B[i] for i in range(k)]
    qhat_bp = [sum(xi[i] * t["M_mi_Bp"][i][j] for i in range(k)) % c.Bp[j] for j in range(k)]
    r_bp = [(s_bp[j] * t["Minv_Bp"][j] + qhat_bp[j] * kt["NMinv_Bp"][j]) % c.Bp[j] for j in range(k)]
    xip = [(r_bp[j] * t["Mp_mj_inv"][j]) % c.Bp[j] for j in range(k)]
    t_b = [sum(xip[j] * t["Mp_mj_B"][j][i] for j in range(k)) % c.B[i] for i in range(k)]
    a = fixed_point_factor(xip, c.Bp)
    a_exact = sum(xip[j] * (c.Mp // c.Bp[j]) for j in range(k)) // c.Mp
    if a != a_exact:
        raise ArithmeticError("B'->B correction estimate differs from the exact factor (operand bound violated)")
    r_b = [(t_b[i] - a * t["Mp_B"][i]) % c.B[i] for i in range(k)]
    return RNSValue(r_b, r_bp)


def add(key: RNSKey, x: RNSValue, y: RNSValue) -> RNSValue:
    c = key.cls
    return RNSValue([(x.b[i] + y.b[i]) % c.B[i] for i in range(c.k)],
                    [(x.bp[j] + y.bp[j]) % c.Bp[j] for j in range(c.k)])


def enter(key: RNSKey, x: int) -> RNSValue:
    """Montgomery form of x (up to a multiple of N): x < 2^(2L) is split into two L-bit chunks."""
    c = key.cls
    if x < 0 or x.bit_length() > 2 * c.L:
        raise ValueError("input longer than two class chunks")
    lo, hi = x & ((1 << c.L) - 1), x >> c.L
    v = mm(key, to_rns(c, lo), key.t["r2"])
    if hi:
        v = add(key, v, mm(key, to_rns(c, hi), key.t["r2h"]))
    return v


def leave(key: RNSKey, v: RNSValue) -> int:
    """Back from the Montgomery domain and to binary: MM(v, 1), CRT, reduce into [0, N)."""
    c = key.cls
    r = mm(key, v, to_rns(c, 1))
    X = crt_value(c, r)
    if X >= (c.k + 1) * key.N:
        raise ArithmeticError("output bound violated")
    return X % key.N


def window_digits(e: int, w: int, nbits: Optional[int] = None) -> List[int]:
    """w-bit digits of e from the most significant window down (fixed windows)."""
    nb = e.bit_length() if nbits is None else nbits
    nwin = (nb + w - 1) // w
    return [(e >> (w * i)) & ((1 << w) - 1) for i in range(nwin - 1, -1, -1)]


def modexp(key: RNSKey, x: int, e: int, w: int = 5) -> int:
    """x^e mod N by fixed-window exponentiation on RNS Montgomery multiplications."""
    xt = enter(key, x)
    table = [key.t["one"], xt]
    for j in range(2, 1 << w):
        table.append(mm(key, table[j - 1], xt))
    digits = window_digits(e, w)
    acc = table[digits[0]] if digits else key.t["one"]
    for dgt in digits[1:]:
        for _ in range(w):
            acc = mm(key, acc, acc)
        acc = mm(key, acc, table[dgt])
    return leave(key, acc)


def rsa_decrypt_crt(c_p: RNSKey, c_q: RNSKey, c: int, dp: int, dq: int, qinv: int, w: int = 5) -> int:
    """CRT decryption on the RNS path: two half-size modexps, Garner's recombination."""
    p, q = c_p.N, c_q.N
    mp = modexp(c_p, c, dp, w)
    mq = modexp(c_q, c, dq, w)
    h = (qinv * (mp - mq)) % p
    return mq + h * q
