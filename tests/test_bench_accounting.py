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
