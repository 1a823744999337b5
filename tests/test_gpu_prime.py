"""GPU primality test of key generation (mr_prime_test_batch: trial division by the first
primes, then Miller-Rabin rounds on the survivors) against the oracle, verdict by verdict."""
import pytest

from oracle import primality
from synth import SplitMix64, load_keys

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


def run(mr, ctx, cands, witnesses, n_limbs, n_primes=10000):
    rounds = len(witnesses[0])
    c = mr.to_tensor(cands, n_limbs)
    w = mr.to_tensor([a for ws in witnesses for a in ws], n_limbs)
    verdict = torch.full((len(cands),), 7, dtype=torch.uint8, device="cuda")
    surv = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    ctx.mr_prime_test_batch(c, w, rounds, verdict, n_primes=n_primes, survivors=surv)
    torch.cuda.synchronize()
    return verdict.cpu().tolist(), int(surv.item())


def check(mr, ctx, cands, witnesses, n_limbs, n_primes=10000):
    got, surv = run(mr, ctx, cands, witnesses, n_limbs, n_primes)
    want = [primality.prime_test_verdict(n, ws, n_primes) for n, ws in zip(cands, witnesses)]
    for i, n in enumerate(cands):
        assert got[i] == want[i], (n, witnesses[i], got[i], want[i])
    assert surv == sum(1 for v in want if v > 0)
    return want


P10001 = 104743  # the 10,001st prime (just past the list)


@pytest.mark.parametrize("n_primes", [10000, 100, 1])
def test_small_candidates_and_list_edges(mr, ctx, n_primes):
    r = SplitMix64(0x5052 + n_primes)
    cands = list(range(0, 1500)) + [104723, 104729, P10001, P10001 * P10001, 104729 * P10001, P10001 * 104759,
                                    3215031751, (1 << 61) - 1, 541 * 547, 547 * 557]
    cands += [r.below(1 << 62) | 1 for _ in range(200)]
    ws = [[2, 3, 5, 7, r.between(2, 1 << 40)] for _ in cands]
    want = check(mr, ctx, cands, ws, 2, n_primes)
    assert set(want) == {0, 1, 2}


@pytest.mark.parametrize("n_limbs", [16, 17, 32, 64, 128])
def test_random_candidates_of_each_class(mr, ctx, n_limbs):
    """Random odd candidates (about nine in ten have a listed factor) and known primes of the
    size, 6 rounds with random witnesses in [2, n-2]."""
    bits = 32 * n_limbs
    r = SplitMix64(0x5053 + n_limbs)
    n = {16: 1024, 17: 512, 32: 512, 64: 256, 128: 96}[n_limbs]
    keys = load_keys("rsa2048_x16") + load_keys("rsa1024_x64")[:8] + load_keys("mix_x256") + load_keys("rsa8192_x2")
    primes = sorted({k[x] for k in keys for x in ("p", "q") if bits - 32 < k[x].bit_length() <= bits})[:8]
    cands = primes + [r.randbits(bits) | 1 | (1 << (bits - 1)) for _ in range(n - len(primes))]
    ws = [[r.between(2, c - 2) for _ in range(6)] for c in cands]
    want = check(mr, ctx, cands, ws, n_limbs)
    assert all(want[i] == 2 for i in range(len(primes)))
    assert 0 < sum(1 for v in want if v > 0) < len(cands)


def test_all_fail_trial_division(mr, ctx):
    """Every candidate has a listed factor: the Miller-Rabin launch has no items."""
    r = SplitMix64(0x5054)
    cands = [3 * (r.randbits(1000) | 1) for _ in range(64)]
    ws = [[2, 3] for _ in cands]
    got, surv = run(mr, ctx, cands, ws, 32)
    assert got == [0] * 64 and surv == 0


def test_argument_errors(mr, ctx):
    c = mr.to_tensor([7, 9], 2)
    w = mr.to_tensor([2, 2], 2)
    v = torch.zeros(2, dtype=torch.uint8, device="cuda")
    with pytest.raises(mr.MRError) as e:
        ctx.mr_prime_test_batch(c, w, 1, v, n_primes=0)
    assert e.value.code == 1
    with pytest.raises(mr.MRError) as e:
        ctx.mr_prime_test_batch(c, w, 1, v, n_primes=10001)
    assert e.value.code == 1
    big = mr.to_tensor([(1 << 4100) + 1], 129)
    with pytest.raises(mr.MRError) as e:
        ctx.mr_prime_test_batch(big, big, 1, v[:1])
    assert e.value.code == 4


def test_empty_inputs_of_the_key_generation_calls(mr, ctx):
    """Zero candidates, zero keys and an empty message are no-ops (the survivor count reads 0)."""
    none = torch.zeros((0, 32), dtype=torch.int32, device="cuda")
    v = torch.zeros(0, dtype=torch.uint8, device="cuda")
    surv = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    ctx.mr_prime_test_batch(none, none, 4, v, survivors=surv)
    out = torch.zeros((0, 9 * 32), dtype=torch.int32, device="cuda")
    ctx.mr_rsa_keygen_batch(none, none, 4, 0, 16, out)
    k = load_keys("rsa1024_x64")[0]
    h = ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
    empty = torch.zeros(0, dtype=torch.uint8, device="cuda")
    ctx.mr_rsa_encrypt_message(h, empty, none)
    ctx.mr_rsa_decrypt_message(h, none, empty)
    torch.cuda.synchronize()
    assert int(surv.item()) == 0
