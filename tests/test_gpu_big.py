"""GPU parity of the large size classes (8192 and 16384 bits: groups of 32 numbers
spread over several thread blocks, one cooperative launch).  Every output equals
the oracle's plain exponentiation bit for bit.  Most exponents are short so the
oracle and the device finish quickly; a few are full length."""
import pytest

from oracle import plain
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


def _run(mr, ctx, handles, Ns, xs, es, W, e_limbs):
    n = len(xs)
    x = mr.to_tensor(xs, W)
    e = mr.to_tensor(es, e_limbs)
    out = torch.full((n, W), -1, dtype=torch.int32, device="cuda")
    st = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    ctx.mr_modexp_batch(handles, x, e, out, st)
    torch.cuda.synchronize()
    return mr.from_tensor(out), st.cpu().tolist()


def test_modexp_16384_ragged_groups_and_edges(mr, ctx):
    keys = load_keys("mod16384_x4")
    handles_all = [ctx.mr_rns_setup(k["N"]) for k in keys]
    r = SplitMix64(0x4D520003)
    n = 40  # two groups of 32, the second one partial
    idx = [i % len(keys) for i in range(n)]
    Ns = [keys[i]["N"] for i in idx]
    xs = [r.below(N) for N in Ns]
    es = [r.randbits(64 + 61 * (j % 7)) for j in range(n)]
    xs[0], es[0] = 0, 5
    xs[1], es[1] = 1, r.randbits(300)
    xs[2], es[2] = Ns[2] - 1, 3
    xs[3], es[3] = r.below(Ns[3]), 0
    xs[4], es[4] = r.below(Ns[4]), 1
    es[5] = r.randbits(16128) | (1 << 16127)  # one full-length exponent (sets the group's window count)
    got, st = _run(mr, ctx, [handles_all[i] for i in idx], Ns, xs, es, 512, 504)
    for j in range(n):
        assert got[j] == plain.modexp(xs[j], es[j], Ns[j]), j
    assert st == [0] * n


@pytest.mark.parametrize("variant", [0, 1], ids=["integer", "tensor"])
def test_modexp_16384_both_forms_of_the_extension(mr, variant):
    """The same batch with the base extensions on the integer pipe (variant 0) and on the tensor
    cores (variant 1, fp16 slices, Sec. 3.1's constant-matrix products): every output equals the
    oracle's.  Three groups of 32, the last partial, edge values, one full-length exponent."""
    keys = load_keys("mod16384_x4")
    c = mr.Context(0)
    try:
        c.mr_set_variant(16384, variant)
        handles = [c.mr_rns_setup(k["N"]) for k in keys]
        r = SplitMix64(0x7C16384 + variant)
        n = 70
        idx = [(3 * i) % len(keys) for i in range(n)]
        Ns = [keys[i]["N"] for i in idx]
        xs = [r.below(N) for N in Ns]
        es = [r.randbits(40 + 37 * (j % 5)) for j in range(n)]
        xs[0], es[0] = 0, 9
        xs[1], es[1] = 1, r.randbits(200)
        xs[2], es[2] = Ns[2] - 1, 5
        xs[3], es[3] = r.below(Ns[3]), 0
        xs[33], es[33] = Ns[33] - 1, 2
        es[40] = r.randbits(16128) | (1 << 16127)
        got, st = _run(mr, c, [handles[i] for i in idx], Ns, xs, es, 512, 504)
        for j in range(n):
            assert got[j] == plain.modexp(xs[j], es[j], Ns[j]), j
        assert st == [0] * n
    finally:
        c.close()


def test_modexp_16384_range_status(mr, ctx):
    keys = load_keys("mod16384_x4")
    h = ctx.mr_rns_setup(keys[0]["N"])
    N = keys[0]["N"]
    xs = [N, N + 1, 7]
    got, st = _run(mr, ctx, [h] * 3, [N] * 3, xs, [65537] * 3, 512, 1)
    assert st == [5, 5, 0]
    assert got[:2] == [0, 0]
    assert got[2] == pow(7, 65537, N)


def test_encrypt_16384_rsa_keys(mr, ctx):
    keys = load_keys("mod16384_x4")
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"]) for k in keys]
    r = SplitMix64(0x4D520013)
    msgs = [r.below(k["N"]) for k in keys]
    m = mr.to_tensor(msgs, 512)
    c = torch.zeros_like(m)
    ctx.mr_rsa_encrypt(hk, m, c)
    torch.cuda.synchronize()
    got = mr.from_tensor(c)
    for i, k in enumerate(keys):
        assert got[i] == plain.rsa_encrypt(msgs[i], k["e"], k["N"]), i


def test_modexp_8192_random_moduli(mr, ctx):
    r = SplitMix64(0x4D520023)
    Ns = []
    while len(Ns) < 3:
        N = r.randbits(8192) | 1 | (1 << 8191)
        Ns.append(N)
    hs = [ctx.mr_rns_setup(N) for N in Ns]
    n = 33
    idx = [j % 3 for j in range(n)]
    xs = [r.below(Ns[i]) for i in idx]
    es = [r.randbits(40 + 97 * (j % 5)) for j in range(n)]
    es[7] = r.randbits(8192)
    got, st = _run(mr, ctx, [hs[i] for i in idx], [Ns[i] for i in idx], xs, es, 256, 256)
    for j in range(n):
        assert got[j] == plain.modexp(xs[j], es[j], Ns[idx[j]]), j
    assert st == [0] * n


def test_modexp_8192_every_slice_width(mr):
    """Every compiled slice width of the 8192-bit class (selected explicitly on a fresh context)
    gives the oracle's results: 40 items (a full group and a partial one), edge bases, and one
    16384-bit CRT decryption whose halves run in this class."""
    r = SplitMix64(0x4D520063)
    N = r.randbits(8192) | 1 | (1 << 8191)
    keys = load_keys("mod16384_x4")
    for v in range(len(mr.mr_class_variants(8192))):
        c = mr.Context(0)
        try:
            c.mr_set_variant(8192, v)
            h = c.mr_rns_setup(N)
            xs = [r.below(N) for _ in range(40)]
            es = [r.randbits(30 + 53 * (j % 5)) for j in range(40)]
            xs[0], xs[1], xs[2] = 0, 1, N - 1
            es[3] = r.randbits(8192)
            got, st = _run(mr, c, [h] * 40, [N] * 40, xs, es, 256, 256)
            assert st == [0] * 40
            for j in range(40):
                assert got[j] == plain.modexp(xs[j], es[j], N), (v, j)
            k = keys[v % len(keys)]
            hk = c.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
            msg = r.below(k["N"])
            ct = pow(msg, k["e"], k["N"])
            cin = mr.to_tensor([ct], 512)
            out = torch.zeros_like(cin)
            c.mr_rsa_decrypt_crt([hk], cin, out)
            torch.cuda.synchronize()
            assert mr.from_tensor(out) == [msg], v
        finally:
            c.close()


def test_large_class_mixed_call_and_plan_refusal(mr, ctx):
    """A mixed call takes 16384-bit keys (encryption in the 16384-bit class, decryption through the
    8192-bit CRT halves); a plan refuses them with MR_ERR_SIZE (plans hold lane-group classes only)."""
    k = load_keys("mod16384_x4")[0]
    h = ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
    r = SplitMix64(0x3177)
    xs = [5, r.below(k["N"])]
    c = mr.to_tensor(xs, 512)
    m = torch.zeros_like(c)
    ctx.mr_rsa_mixed([h, h], [0, 1], c, m)  # MR_OP_ENCRYPT, MR_OP_DECRYPT
    torch.cuda.synchronize()
    got = mr.from_tensor(m)
    assert got[0] == plain.modexp(5, k["e"], k["N"])
    assert got[1] == plain.rsa_decrypt_crt(xs[1], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
    with pytest.raises(mr.MRError) as e:
        ctx.mr_plan_create([h], [0], c[:1], m[:1])
    assert e.value.code == 4


def test_rsa16384_crt_decrypt(mr, ctx):
    """16384-bit keys: the two 8192-bit halves run in the large-class kernel, then the binary
    Garner recombination.  decrypt(encrypt(m)) = m for 36 messages over 4 keys (72 halves: three
    item groups, the last partial); decryption is a bijection, so each equality pins that output.
    Edge inputs 0, 1 and N-1 (odd d: (-1)^d = -1), an input N (status RANGE, output 0), and one
    output against the oracle's CRT decryption of a random ciphertext."""
    keys = load_keys("mod16384_x4")
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
    r = SplitMix64(0x4D520053)
    idx = [j % len(keys) for j in range(36)]
    msgs = [r.below(keys[i]["N"]) for i in idx]
    m = mr.to_tensor(msgs, 512)
    c = torch.zeros_like(m)
    ctx.mr_rsa_encrypt([hk[i] for i in idx], m, c)
    back = torch.full_like(m, -1)
    st = torch.full((len(msgs),), 255, dtype=torch.uint8, device="cuda")
    ctx.mr_rsa_decrypt_crt([hk[i] for i in idx], c, back, st)
    torch.cuda.synchronize()
    cs = mr.from_tensor(c)
    assert st.cpu().tolist() == [0] * len(msgs)
    assert mr.from_tensor(back) == msgs
    for j in (0, 5):
        k = keys[idx[j]]
        assert cs[j] == plain.rsa_encrypt(msgs[j], k["e"], k["N"]), j

    k0, k1 = keys[0], keys[1]
    ct = [0, 1, k0["N"] - 1, k0["N"], r.below(k1["N"])]
    kidx = [0, 0, 0, 0, 1]
    cin = mr.to_tensor(ct, 512)
    out = torch.full_like(cin, -1)
    st = torch.full((len(ct),), 255, dtype=torch.uint8, device="cuda")
    ctx.mr_rsa_decrypt_crt([hk[i] for i in kidx], cin, out, st)
    torch.cuda.synchronize()
    got = mr.from_tensor(out)
    assert st.cpu().tolist() == [0, 0, 0, 5, 0]
    assert got[:4] == [0, 1, k0["N"] - 1, 0]
    assert got[4] == plain.rsa_decrypt_crt(ct[4], k1["p"], k1["q"], k1["dp"], k1["dq"], k1["qinv"])


def test_bounded_wait_times_out_and_context_recovers(mr, ctx):
    """One channel slice never arrives at the inter-block waits (test hook): the other blocks
    give up after a short poll limit, every item reports MR_ERR_TIMEOUT, and the next call on
    the same context computes correct results."""
    r = SplitMix64(0x4D520033)
    N = r.randbits(8192) | 1 | (1 << 8191)
    h = ctx.mr_rns_setup(N)
    xs = [r.below(N) for _ in range(32)]
    es = [r.randbits(64) for _ in range(32)]
    ctx.mr_debug_big_wait(spin_limit=1 << 14, absent_slice=3)
    try:
        _, st = _run(mr, ctx, [h] * 32, [N] * 32, xs, es, 256, 2)
    finally:
        ctx.mr_debug_big_wait(0, -1)
    assert st == [8] * 32  # MR_ERR_TIMEOUT
    got, st = _run(mr, ctx, [h] * 32, [N] * 32, xs, es, 256, 2)
    assert st == [0] * 32
    for j in range(32):
        assert got[j] == plain.modexp(xs[j], es[j], N), j


def test_rsa8192_encrypt_decrypt_round_trip(mr, ctx):
    """8192-bit RSA keys: encryption in the 8192-bit class (multi-block groups), CRT decryption on
    4096-bit halves (lane-group class), both equal to the oracle, and decrypt(encrypt(m)) = m."""
    keys = load_keys("rsa8192_x2")
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
    r = SplitMix64(0x4D520043)
    idx = [j % 2 for j in range(10)]
    msgs = [r.below(keys[i]["N"]) for i in idx]
    msgs[0], msgs[1] = 0, keys[1]["N"] - 1
    m = mr.to_tensor(msgs, 256)
    c = torch.zeros_like(m)
    ctx.mr_rsa_encrypt([hk[i] for i in idx], m, c)
    m2 = torch.zeros_like(m)
    st = torch.full((len(msgs),), 255, dtype=torch.uint8, device="cuda")
    ctx.mr_rsa_decrypt_crt([hk[i] for i in idx], c, m2, st)
    torch.cuda.synchronize()
    cs, back = mr.from_tensor(c), mr.from_tensor(m2)
    assert st.cpu().tolist() == [0] * len(msgs)
    for j, i in enumerate(idx):
        k = keys[i]
        assert cs[j] == plain.rsa_encrypt(msgs[j], k["e"], k["N"]), j
        assert back[j] == msgs[j], j
    j = 3
    k = keys[idx[j]]
    assert back[j] == plain.rsa_decrypt_crt(cs[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
