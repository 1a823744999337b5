"""GPU RSA key generation from candidate pools (mr_rsa_keygen_batch) against the oracle's
rsa_key_from_pools: the same pools and witnesses give the same key, part by part."""
import pytest

from oracle import keygen, plain
from synth import SplitMix64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


def _pools(r, n_keys, pool, bits, rounds):
    pools = [[r.randbits(bits) | (3 << (bits - 2)) | 1 for _ in range(pool)] for _ in range(2 * n_keys)]
    wits = [[[r.between(2, c - 2) for _ in range(rounds)] for c in pl] for pl in pools]
    return pools, wits


def _run(mr, ctx, pools, wits, n_keys, pool, H, rounds, e):
    cand = mr.to_tensor([c for pl in pools for c in pl], H)
    wit = mr.to_tensor([w for wl in wits for ws in wl for w in ws], H)
    out = torch.full((n_keys, 9 * H), -1, dtype=torch.int32, device="cuda")
    st = torch.full((n_keys,), 255, dtype=torch.uint8, device="cuda")
    ctx.mr_rsa_keygen_batch(cand, wit, rounds, n_keys, pool, out, e=e, status=st)
    torch.cuda.synchronize()
    rows = out.cpu().numpy().astype("int64") & 0xFFFFFFFF
    keys = []
    for k in range(n_keys):
        row = [int(v) for v in rows[k]]
        part = lambda a, b: sum(v << (32 * i) for i, v in enumerate(row[a * H:b * H]))
        keys.append({"N": part(0, 2), "d": part(2, 4), "p": part(4, 5), "q": part(5, 6), "dp": part(6, 7),
                     "dq": part(7, 8), "qinv": part(8, 9)})
    return keys, st.cpu().tolist()


def _check(mr, ctx, n_keys, pool, bits, rounds, e, seed, empty=()):
    r = SplitMix64(seed)
    H = bits // 32
    pools, wits = _pools(r, n_keys, pool, bits, rounds)
    for k in empty:  # key k's p pool: odd multiples of 3 only
        pools[2 * k] = [3 * (r.randbits(bits - 2) | 1 | (1 << (bits - 3))) for _ in range(pool)]
    got, st = _run(mr, ctx, pools, wits, n_keys, pool, H, rounds, e)
    for k in range(n_keys):
        want = keygen.rsa_key_from_pools(pools[2 * k], wits[2 * k], pools[2 * k + 1], wits[2 * k + 1], e)
        if want is None:
            assert st[k] == 5 and all(v == 0 for v in got[k].values()), k
            continue
        assert st[k] == 0, k
        for part in ("N", "d", "p", "q", "dp", "dq", "qinv"):
            assert got[k][part] == want[part], (k, part)
    return got, st


def test_keygen_1024_bit_keys(mr, ctx):
    got, st = _check(mr, ctx, n_keys=3, pool=1024, bits=512, rounds=8, e=65537, seed=0x4B47)
    # the keys work end to end on the GPU: set up, encrypt, CRT-decrypt
    r = SplitMix64(0x4B48)
    for k, key in enumerate(got):
        if st[k]:
            continue
        h = ctx.mr_rsa_key_setup(key["N"], 65537, key["p"], key["q"], key["dp"], key["dq"], key["qinv"])
        m = r.below(key["N"])
        mt = mr.to_tensor([m], 32)
        ct = torch.zeros_like(mt)
        back = torch.zeros_like(mt)
        ctx.mr_rsa_encrypt([h], mt, ct)
        ctx.mr_rsa_decrypt_crt([h], ct, back)
        torch.cuda.synchronize()
        assert mr.from_tensor(ct) == [plain.rsa_encrypt(m, 65537, key["N"])]
        assert mr.from_tensor(back) == [m]


def test_keygen_small_primes_exponent_3_and_empty_pool(mr, ctx):
    """64-bit primes, e = 3 (primes with 3 | p - 1 are skipped), one key whose p pool holds only
    multiples of 3 (status MR_ERR_RANGE, zero row)."""
    got, st = _check(mr, ctx, n_keys=5, pool=64, bits=64, rounds=6, e=3, seed=0x4B49, empty=(2,))
    assert st[2] == 5 and st.count(0) >= 3


def test_keygen_degenerate_prime_two(mr, ctx):
    """A pool whose first candidate is 2: it passes the prime test and gcd(e, 1) = 1, so p = 2;
    dp = e^-1 mod 1 = 0 and qinv = 1, as the oracle has them."""
    q_pool = [(1 << 61) - 1, 18446744073709551557]  # primes (2^61 - 1; the largest 64-bit prime)
    p_pool = [2, 9]
    wits = [[1, 1], [2, 3]], [[2, 3], [2, 3]]
    got, st = _run(mr, ctx, [p_pool, q_pool], list(wits), 1, 2, 2, 2, 3)
    want = keygen.rsa_key_from_pools(p_pool, wits[0], q_pool, wits[1], 3)
    assert st == [0] and want["p"] == 2 and want["dp"] == 0
    for part in ("N", "d", "p", "q", "dp", "dq", "qinv"):
        assert got[0][part] == want[part], part


def test_keygen_2048_bit_primes(mr, ctx):
    """The largest size: 2048-bit primes (4096-bit N), one key."""
    _check(mr, ctx, n_keys=1, pool=1536, bits=2048, rounds=3, e=65537, seed=0x4B4A)


def test_keygen_argument_errors(mr, ctx):
    c = mr.to_tensor([7, 9], 1)
    out = torch.zeros((1, 9), dtype=torch.int32, device="cuda")
    with pytest.raises(mr.MRError) as e:
        ctx.mr_rsa_keygen_batch(c, c, 1, 1, 1, out)  # one-limb candidates
    assert e.value.code == 4
    c = mr.to_tensor([7, 9], 2)
    out = torch.zeros((1, 18), dtype=torch.int32, device="cuda")
    with pytest.raises(mr.MRError) as e:
        ctx.mr_rsa_keygen_batch(c, c, 1, 1, 1, out, e=4)
    assert e.value.code == 1


def test_keygen_8192_bit_keys_from_known_primes(mr, ctx):
    """RSA-8192 keys (4096-bit primes; the warp-wide inversion with four limbs per lane): each pool
    hides one of the seeded 4096-bit primes behind random odd candidates, and the key the GPU
    assembles equals the oracle's rsa_key_from_pools part by part, and encrypts and decrypts."""
    from synth import load_keys
    known = load_keys("rsa8192_x2")
    r = SplitMix64(0x4B4C)
    bits, pool, rounds, n_keys = 4096, 6, 4, 2
    H = bits // 32
    pools, wits = [], []
    for k in range(n_keys):
        for prime in (known[k]["p"], known[k]["q"]):
            pl = [r.randbits(bits) | (3 << (bits - 2)) | 1 for _ in range(pool - 1)] + [prime]
            pools.append(pl)
            wits.append([[r.between(2, c - 2) for _ in range(rounds)] for c in pl])
    got, st = _run(mr, ctx, pools, wits, n_keys, pool, H, rounds, 65537)
    for k in range(n_keys):
        want = keygen.rsa_key_from_pools(pools[2 * k], wits[2 * k], pools[2 * k + 1], wits[2 * k + 1], 65537)
        assert want is not None and st[k] == 0, k
        for part in ("N", "d", "p", "q", "dp", "dq", "qinv"):
            assert got[k][part] == want[part], (k, part)
        key = got[k]
        h = ctx.mr_rsa_key_setup(key["N"], 65537, key["p"], key["q"], key["dp"], key["dq"], key["qinv"])
        m = r.below(key["N"])
        mt = mr.to_tensor([m], 2 * H)
        ct = torch.zeros_like(mt)
        back = torch.zeros_like(mt)
        ctx.mr_rsa_encrypt([h], mt, ct)
        ctx.mr_rsa_decrypt_crt([h], ct, back)
        torch.cuda.synchronize()
        assert mr.from_tensor(ct) == [pow(m, 65537, key["N"])]
        assert mr.from_tensor(back) == [m]
