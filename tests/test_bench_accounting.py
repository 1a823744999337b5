"""The multiplication counts bench.py uses for its roofline: the fixed-window formula and the
sliding-window count equal the multiplications an instrumented square-and-multiply performs
(which also has to produce x^e mod N), for random and edge exponents."""
import bench
from synth import SplitMix64


def _fixed(x, e, N, w, chunks):
    """Fixed w-bit windows as the lane-group kernel runs them for one number alone (zero digits
    skipped only when every number of the warp has one: never skipped here)."""
    mms = chunks + (2 ** w - 2) + 1  # entry products, table x^2..x^(2^w-1), exit
    nwin = max(1, -(-e.bit_length() // w))
    tab = [pow(x, j, N) for j in range(2 ** w)]
    acc = tab[(e >> ((nwin - 1) * w)) & (2 ** w - 1)]
    for i in range(nwin - 2, -1, -1):
        for _ in range(w):
            acc = acc * acc % N
            mms += 1
        acc = acc * tab[(e >> (i * w)) & (2 ** w - 1)] % N
        mms += 1
    return acc, mms


def _sliding(x, e, N, w, chunks):
    """Left-to-right sliding windows of up to w + 1 bits over the odd powers."""
    ws = w + 1
    mms = chunks + 2 ** w + 1  # entry, x^2 and the odd powers x^3..x^(2^(w+1)-1), exit
    tab = [pow(x, 2 * i + 1, N) for i in range(2 ** w)]
    top = e.bit_length() - 1
    lo = max(top - ws + 1, 0)
    while not (e >> lo) & 1:
        lo += 1
    acc = tab[((e >> lo) & ((1 << (top - lo + 1)) - 1)) >> 1]
    i = lo - 1
    while i >= 0:
        if not (e >> i) & 1:
            acc = acc * acc % N
            mms += 1
            i -= 1
            continue
        lo = max(i - ws + 1, 0)
        while not (e >> lo) & 1:
            lo += 1
        for _ in range(i - lo + 1):
            acc = acc * acc % N
            mms += 1
        acc = acc * tab[((e >> lo) & ((1 << (i - lo + 1)) - 1)) >> 1] % N
        mms += 1
        i = lo - 1
    return acc, mms


def test_multiplication_counts():
    r = SplitMix64(0x62656E)
    N = r.randbits(256) | 1
    k, W, WX = 36, 32, 34
    per_mm = 2 * k * k + 7 * k
    for w in (4, 5, 6):
        exps = [r.randbits(1024) | (1 << 1023), 1 << 700, (1 << 513) - 1, (r.randbits(300) << 200) | 1, 65537,
                r.randbits(1021) | (1 << 1020)]
        for e in exps:
            x = r.below(N)
            got, mms = _sliding(x, e, N, w, 2)
            assert got == pow(x, e, N)
            assert bench.mms_sliding(e, w, 2) == mms, (w, e.bit_length())
            assert bench.algorithmic_products_sliding(k, W, WX, e, w, 2) == mms * per_mm + 2 * W * 2 * k + k * WX
            got, mms = _fixed(x, e, N, w, 2)
            assert got == pow(x, e, N)
            assert bench.algorithmic_products_per_modexp(k, W, WX, e.bit_length(), w, 2) == \
                mms * per_mm + 2 * W * 2 * k + k * WX


def _primes_below_2_31(count):
    """The `count` largest primes below 2^31, by trial division (exact for 31-bit numbers)."""
    out, x = [], (1 << 31) - 1
    while len(out) < count:
        if x % 2:
            d, p = 3, True
            while d * d <= x:
                if x % d == 0:
                    p = False
                    break
                d += 2
            if p:
                out.append(x)
        x -= 1
    return out


def test_k31_is_the_closure_bound():
    """K31[L] is the smallest k with M >= (k+1)^2 2^L and M' >= (k+1) 2^L over the largest primes
    below 2^31 (B the first k, B' the next k)."""
    import math
    primes = _primes_below_2_31(2 * 530 + 2)
    for L, k in bench.K31.items():
        def ok(kk):
            M, Mp = math.prod(primes[:kk]), math.prod(primes[kk:2 * kk])
            return M >= (kk + 1) ** 2 * 2 ** L and Mp >= (kk + 1) * 2 ** L
        assert ok(k) and not ok(k - 1), L


def test_31bit_count_values():
    """One RSA-2048 CRT half (1024-bit, |e| = 1024, w = 5): 1263 multiplications of 5304 operations
    plus 13,320 operations of conversions; one 16384-bit exponentiation with |e| = 16128, w = 8:
    18,402 multiplications of 1,134,200 operations."""
    assert bench.ops_31bit_count(1024, 1024, 5) == 1263 * 5304 + 13320
    assert bench.ops_31bit_count(16384, 16128, 8) == 18402 * 1134200 + 2 * (2 * 512 * 1061 + 2 * 530 * 513)
    assert bench.tensor_ops_31bit_count(16384, 256, 16128, 8) == 18402 * 2 * 16 * 2 * 256 * 530 * 531
