"""GPU Miller-Rabin (mr_miller_rabin_batch) against the oracle, verdict by verdict."""
import os

import numpy as np
import pytest

from oracle import primality
from synth import SplitMix64, load_keys

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_3699_gb300 import mr as m
    return m


@pytest.fixture(scope="module")
def ctx(mr):
    c = mr.Context(0)
    yield c
    c.close()


def run_mr(mr, ctx, cands, witnesses, n_limbs):
    rounds = len(witnesses[0])
    c = mr.to_tensor(cands, n_limbs)
    w = mr.to_tensor([a for ws in witnesses for a in ws], n_limbs)
    flag = torch.full((len(cands),), 7, dtype=torch.uint8, device="cuda")
    mask = torch.zeros(len(cands), dtype=torch.int32, device="cuda")
    ctx.mr_miller_rabin_batch(c, w, rounds, flag, mask)
    torch.cuda.synchronize()
    return flag.cpu().tolist(), [int(v) & 0xFFFFFFFF for v in mask.cpu().numpy().astype(np.int64)]


def expect(n, ws):
    verdicts = primality.miller_rabin(n, ws)
    return int(all(verdicts)), sum(1 << r for r, v in enumerate(verdicts) if v)


def check(mr, ctx, cands, witnesses, n_limbs, skip_mask_for=()):
    flags, masks = run_mr(mr, ctx, cands, witnesses, n_limbs)
    for i, n in enumerate(cands):
        f, m = expect(n, witnesses[i])
        assert flags[i] == f, (n, witnesses[i])
        if n not in skip_mask_for:
            assert masks[i] == m, (n, witnesses[i], hex(masks[i]), hex(m))


def test_small_candidates_exhaustive_witnesses(mr, ctx):
    r = SplitMix64(1)
    cands = list(range(0, 200)) + [r.below(1 << 31) | 1 for _ in range(300)] + [2147483647, 2147483629]
    ws = [[2, 3, 5, 7, r.below(1 << 40)] for _ in cands]
    check(mr, ctx, cands, ws, 2)


def test_strong_pseudoprimes(mr, ctx):
    cands, ws = [], []
    for line in open(os.path.join(GOLD, "strong_pseudoprimes.txt")):
        if line.startswith("#") or not line.strip():
            continue
        n, passed, failed = line.split()
        bases = ([int(b) for b in passed.split(",")] if passed != "-" else []) + [int(failed)]
        bases = (bases + [2] * 6)[:6]
        cands.append(int(n))
        ws.append(bases)
    check(mr, ctx, cands, ws, 2)


@pytest.mark.parametrize("n_limbs", [16, 32, 48, 64])
def test_large_primes_and_composites(mr, ctx, n_limbs):
    bits = 32 * n_limbs
    r = SplitMix64(n_limbs)
    keys = load_keys("rsa2048_x16") + load_keys("rsa1024_x64")[:8] + load_keys("mix_x256")
    primes = sorted({k[x] for k in keys for x in ("p", "q") if bits - 32 < k[x].bit_length() <= bits})[:12]
    comps = [r.randbits(bits) | 1 for _ in range(12)]
    products = [k["N"] for k in keys if bits - 32 < k["N"].bit_length() <= bits][:6]
    cands = primes + comps + products
    ws = [[r.between(2, n - 2) for _ in range(3)] for n in cands]
    check(mr, ctx, cands, ws, n_limbs)


def test_mersenne_primes_and_witness_edges(mr, ctx):
    cands, ws = [], []
    for e in (521, 607, 1279):
        p = (1 << e) - 1
        cands += [p, p]
        ws += [[2, 3, 0, p - 1], [1, p, p + 1, 5]]
    check(mr, ctx, cands, ws, 64)


def test_candidate_with_channel_prime_factor(mr, ctx):
    B = mr.mr_debug_class_table(1024, "B")  # 17-limb candidates fall in the 1024-bit class
    big_prime = load_keys("rsa1024_x64")[0]["p"]  # 512 bits
    n = B[5] * big_prime  # odd composite above 2^31 sharing a channel prime
    assert n.bit_length() <= 17 * 32
    flags, masks = run_mr(mr, ctx, [n], [[2, 3]], 17)
    assert flags == [0] and masks == [0]
    assert not all(primality.miller_rabin(n, [2, 3]))


def test_device_derived_constants_match_host_setup(mr, ctx):
    """The Miller-Rabin kernel derives each candidate's constants on the device;
    they must equal the host setup's (which the CPU tests tie to the oracle model)."""
    from oracle import rns
    r = SplitMix64(77)
    for n_limbs in (2, 16, 32, 64):
        bits = 32 * n_limbs
        cands = [3215031751] if n_limbs == 2 else [r.randbits(bits) | 1 | (1 << (bits - 1)) for _ in range(3)]
        L, k = mr.mr_class_for_bits(bits)
        W = L // 32
        words = 4 + 2 * W + 5 * k
        out = torch.zeros((len(cands), words), dtype=torch.int32, device="cuda")
        ctx.mr_debug_mr_setup(mr.to_tensor(cands, n_limbs), out)
        got = out.cpu().numpy().view(np.uint32)
        c = rns.make_class(L)
        for i, N in enumerate(cands):
            row = [int(v) for v in got[i]]
            key = rns.make_key(c, N)
            s = (N - 1 & -(N - 1)).bit_length() - 1
            assert row[0] == 0 and row[1] == s and row[2] == N.bit_length(), row[:4]
            assert row[3] == (c.M % N) & 0xFFFFFFFF, (row[3], (c.M % N) & 0xFFFFFFFF, row[4])
            one = int.from_bytes(b"".join(v.to_bytes(4, "little") for v in row[4:4 + W]), "little")
            r2 = int.from_bytes(b"".join(v.to_bytes(4, "little") for v in row[4 + W:4 + 2 * W]), "little")
            assert one == c.M % N and r2 == c.M * c.M % N
            base = 4 + 2 * W
            assert row[base:base + k] == key.t["kxi"]
            assert row[base + k:base + 2 * k] == key.t["NMinv_Bp"]
            assert row[base + 3 * k:base + 4 * k] == [pow(N % m, -1, m) for m in c.B]
            assert row[base + 4 * k:base + 5 * k] == [pow(N % m, -1, m) for m in c.Bp]
            assert row[base + 2 * k:base + 3 * k] == [v * c.t["Mp_mj_inv"][j] % c.Bp[j]
                                                      for j, v in enumerate(key.t["NMinv_Bp"])]


def _oracle_rounds(cands, witnesses):
    """Per-round oracle verdicts of large candidates on a spawned process pool (a forked child of a
    CUDA process may hang); the oracle's square-and-multiply takes seconds per 16384-bit round."""
    import multiprocessing as mp

    pairs = [(n, a) for n, ws in zip(cands, witnesses) for a in ws]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        flat = pool.starmap(primality.miller_rabin_round, pairs, chunksize=1)
    out, i = [], 0
    for ws in witnesses:
        out.append(flat[i:i + len(ws)])
        i += len(ws)
    return out


def _check_large(mr, ctx, cands, witnesses, n_limbs, channel_factor=()):
    flags, masks = run_mr(mr, ctx, cands, witnesses, n_limbs)
    verdicts = _oracle_rounds(cands, witnesses)
    for i, n in enumerate(cands):
        v = verdicts[i]
        if n in channel_factor:  # reported composite without evaluating the rounds
            assert flags[i] == 0 and masks[i] == 0 and not all(v), i
            continue
        assert flags[i] == int(all(v)), (i, n.bit_length(), v)
        assert masks[i] == sum(1 << r for r, ok in enumerate(v) if ok), (i, n.bit_length(), v, hex(masks[i]))


def _prime_with_large_two_power(r, bits, s):
    """A seeded prime c * 2^s + 1 (c odd) of `bits` bits: n - 1 has s factors of two, so a round of
    the test may pass at any of s squaring steps.  Found by trial division and a base-2 Fermat check
    with CPython's pow; the test's expected verdicts still come from the oracle."""
    small = primality.first_primes(2000)[1:]
    while True:
        c = r.randbits(bits - s) | 1 | (1 << (bits - s - 1))
        n = (c << s) + 1
        if any(n % p == 0 for p in small):
            continue
        if pow(2, n - 1, n) == 1:
            return n


def test_large_class_candidates_8192(mr, ctx):
    """256-limb rows (the 8192-bit class): 8192-bit primes and composites through the large-class
    exponentiation, a 4423-bit Mersenne prime and a prime with 2^64 | n - 1 (many squaring steps),
    4096-bit primes and small values through the repacked lane-group path, witness edge values, and
    a candidate divisible by a channel prime of the class."""
    r = SplitMix64(0x8192)
    big = load_keys("mod16384_x4")
    mid = load_keys("rsa8192_x2")
    primes8k = [k[x] for k in big for x in ("p", "q")][:6]
    comps = [k["N"] for k in mid] + [r.randbits(8192) | 1 | (1 << 8191) for _ in range(3)]
    m4423 = (1 << 4423) - 1
    proth = _prime_with_large_two_power(r, 4200, 64)
    p4k = [mid[0]["p"], mid[1]["q"]]
    B = mr.mr_debug_class_table(8192, "B")
    chan = B[7] * mid[0]["q"]  # above 4096 bits: the large-class path finds the shared channel prime
    assert 4096 < chan.bit_length() <= 8192
    smalls = [0, 1, 2, 3, 9, 15, 2147483647]
    cands = primes8k + comps + [m4423, m4423, proth] + p4k + [chan] + smalls
    ws = []
    for n in cands:
        if n == m4423 and not any(c == m4423 for c in cands[:len(ws)]):
            ws.append([0, n - 1, n + 1])
        elif n == m4423:
            ws.append([1, n, 2])
        elif n < 5:
            ws.append([2, 3, 7])
        else:
            ws.append([r.between(2, n - 2) for _ in range(3)])
    _check_large(mr, ctx, cands, ws, 256, channel_factor=(chan,))


def test_large_class_candidates_16384(mr, ctx):
    """512-limb rows (the 16384-bit class): 16384-bit RSA moduli (composite), the 9689-bit Mersenne
    prime, and an 8192-bit prime, two rounds each."""
    r = SplitMix64(0x16384)
    big = load_keys("mod16384_x4")
    m9689 = (1 << 9689) - 1
    cands = [big[0]["N"], big[1]["N"], m9689, big[2]["p"]]
    ws = [[r.between(2, n - 2) for _ in range(2)] for n in cands]
    _check_large(mr, ctx, cands, ws, 512)
