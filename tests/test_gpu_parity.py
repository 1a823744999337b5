"""GPU parity: every output of the CUDA path equals the CPU oracle bit for bit.

All calls go through the C ABI (ctypes binding).  Inputs are seeded synthetic
numbers; expected values come only from ``oracle``.
"""
import numpy as np
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


def _status(n):
    return torch.full((n,), 255, dtype=torch.uint8, device="cuda")


def test_rsa1024_encrypt_all_keys(mr, ctx):
    keys = load_keys("rsa1024_x64")
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"]) for k in keys]
    r = SplitMix64(0x4D520001)
    msgs = []
    for i, k in enumerate(keys):
        N = k["N"]
        msgs.append([0, 1, N - 1, 2][i] if i < 4 else r.below(N))
    m = mr.to_tensor(msgs, 32)
    c = torch.zeros_like(m)
    st = _status(len(keys))
    ctx.mr_rsa_encrypt(hk, m, c, st)
    torch.cuda.synchronize()
    got = mr.from_tensor(c)
    for i, k in enumerate(keys):
        assert got[i] == plain.rsa_encrypt(msgs[i], k["e"], k["N"]), i
    assert st.cpu().tolist() == [0] * len(keys)


def _crt_case(mr, ctx, keys, n, seed, stride=64):
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
    r = SplitMix64(seed)
    idx = [i % len(keys) for i in range(n)]
    cts = []
    for j, i in enumerate(idx):
        N = keys[i]["N"]
        cts.append([0, 1, N - 1][j] if j < 3 else r.below(N))
    c = mr.to_tensor(cts, stride)
    m = torch.zeros_like(c)
    st = _status(n)
    ctx.mr_rsa_decrypt_crt([hk[i] for i in idx], c, m, st)
    torch.cuda.synchronize()
    return idx, cts, mr.from_tensor(m), st.cpu().tolist()


def test_rsa2048_crt_decrypt_ragged(mr, ctx):
    keys = load_keys("rsa2048_x16")
    n = 16 * 16 + 5  # several blocks plus a ragged tail
    idx, cts, got, st = _crt_case(mr, ctx, keys, n, 0x4D520002)
    assert st == [0] * n
    for j, i in enumerate(idx):
        k = keys[i]
        assert got[j] == plain.rsa_decrypt_crt(cts[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]), j


def test_crt_decrypt_equals_plain_definition(mr, ctx):
    keys = load_keys("test_small") + load_keys("rsa1024_x64")[:3]
    idx, cts, got, st = _crt_case(mr, ctx, keys, 40, 77, stride=32)
    for j, i in enumerate(idx):
        assert got[j] == pow(cts[j], keys[i]["d"], keys[i]["N"]), j


def _modexp_case(mr, ctx, bits_list, ebits_list, seed, stride=None, estride=None):
    r = SplitMix64(seed)
    mods = [r.randbits(b) | 1 | (1 << (b - 1)) for b in bits_list]
    hk = [ctx.mr_rns_setup(N) for N in mods]
    xs = [r.below(N) for N in mods]
    es = [r.randbits(eb) for eb in ebits_list]
    ls = stride or max((N.bit_length() + 31) // 32 for N in mods)
    el = estride or max(1, max((eb + 31) // 32 for eb in ebits_list))
    x = mr.to_tensor(xs, ls)
    e = mr.to_tensor(es, el)
    out = torch.zeros_like(x)
    st = _status(len(mods))
    ctx.mr_modexp_batch(hk, x, e, out, st)
    torch.cuda.synchronize()
    got = mr.from_tensor(out)
    for i, N in enumerate(mods):
        assert got[i] == plain.modexp(xs[i], es[i], N), (i, N.bit_length())
    assert st.cpu().tolist() == [0] * len(mods)
    for h in hk:
        h.free()


@pytest.mark.parametrize("bits", [64, 300, 512, 700, 1024, 1500, 2048, 3072, 4096])
def test_modexp_each_class(mr, ctx, bits):
    n = 37  # more than one warp, ragged
    _modexp_case(mr, ctx, [bits] * n, [min(bits, 256)] * n, bits)


def test_modexp_full_length_exponents(mr, ctx):
    _modexp_case(mr, ctx, [1024] * 9, [1024] * 9, 5)
    _modexp_case(mr, ctx, [2048] * 3, [2048] * 3, 6)


@pytest.mark.parametrize("bits", [512, 1024, 2048, 4096])
def test_modexp_shared_exponent_sliding_windows(mr, ctx, bits):
    """Warps whose numbers share one exponent run the sliding-window schedule: every item of a
    block of 40 (several warps, a ragged tail) has the same exponent, moduli and bases differ.
    Exponents: random, single bit, all ones, long zero runs inside and at the bottom, a last
    window ending on bit 0, one set bit in each of the top and bottom positions."""
    r = SplitMix64(0x51 + bits)
    eb = min(bits, 1024)
    exps = [r.randbits(eb) | (1 << (eb - 1)), 1 << (eb - 1), (1 << eb) - 1,
            (r.randbits(eb // 2) << (eb // 2)) | 1, (r.randbits(64) | (1 << 63)) << (eb - 64),
            (1 << (eb - 1)) | 1, (1 << (eb - 1)) | (0b1011 << 200) | 0b110001]
    el = (eb + 31) // 32
    for j, e in enumerate(exps):
        n = 40
        mods = [r.randbits(bits) | 1 | (1 << (bits - 1)) for _ in range(3)]
        hk = [ctx.mr_rns_setup(N) for N in mods]
        idx = [i % 3 for i in range(n)]
        xs = [r.below(mods[i]) for i in idx]
        xs[0], xs[1] = 1, mods[idx[1]] - 1
        x = mr.to_tensor(xs, bits // 32)
        et = mr.to_tensor([e] * n, el)
        out = torch.zeros_like(x)
        st = _status(n)
        ctx.mr_modexp_batch([hk[i] for i in idx], x, et, out, st)
        torch.cuda.synchronize()
        got = mr.from_tensor(out)
        for i in range(n):
            assert got[i] == plain.modexp(xs[i], e, mods[idx[i]]), (bits, j, i)
        assert st.cpu().tolist() == [0] * n
        for h in hk:
            h.free()


def test_modexp_mixed_sizes_one_call(mr, ctx):
    bits = [512, 1024, 2048, 3072, 4096, 1024, 768, 1536] * 5
    _modexp_case(mr, ctx, bits, [96] * len(bits), 9)


def test_modexp_edge_values(mr, ctx):
    r = SplitMix64(3)
    N = r.randbits(1024) | 1 | (1 << 1023)
    h = ctx.mr_rns_setup(N)
    cases = [(0, 0), (0, 5), (1, 12345), (N - 1, 3), (N - 1, 4), (r.below(N), 0), (r.below(N), 1),
             (r.below(N), (1 << 1024) - 1), (2, 1 << 200), (N - 2, 65537)]
    x = mr.to_tensor([c[0] for c in cases], 32)
    e = mr.to_tensor([c[1] for c in cases], 33)
    out = torch.zeros_like(x)
    ctx.mr_modexp_batch([h] * len(cases), x, e, out)
    torch.cuda.synchronize()
    for (xv, ev), g in zip(cases, mr.from_tensor(out)):
        assert g == plain.modexp(xv, ev, N), (xv, ev)


def test_range_errors_reported_per_item(mr, ctx):
    r = SplitMix64(4)
    N = r.randbits(512) | 1 | (1 << 511)
    h = ctx.mr_rns_setup(N)
    xs = [5, N, N + 1, N - 1, (1 << 512) - 1, 7]
    x = mr.to_tensor(xs, 16)
    e = mr.to_tensor([3] * len(xs), 1)
    out = torch.zeros_like(x)
    st = _status(len(xs))
    ctx.mr_modexp_batch([h] * len(xs), x, e, out, st)
    torch.cuda.synchronize()
    assert st.cpu().tolist() == [0, 5, 5, 0, 5, 0]
    got = mr.from_tensor(out)
    assert got[0] == pow(5, 3, N) and got[3] == pow(N - 1, 3, N) and got[5] == pow(7, 3, N)


def test_setup_errors(mr, ctx):
    with pytest.raises(mr.MRError) as e:
        ctx.mr_rns_setup(1 << 300)
    assert e.value.code == 2
    with pytest.raises(mr.MRError) as e:
        ctx.mr_rns_setup((1 << 16384) + 1)
    assert e.value.code == 4
    k = load_keys("test_small")[0]
    with pytest.raises(mr.MRError):
        ctx.mr_rsa_key_setup(k["N"], 65537, k["p"] + 2, k["q"], k["dp"], k["dq"], k["qinv"])
    pub = ctx.mr_rsa_key_setup(k["N"], 65537)
    c = mr.to_tensor([5], 16)
    with pytest.raises(mr.MRError) as e:
        ctx.mr_rsa_decrypt_crt([pub], c, torch.zeros_like(c))
    assert e.value.code == 10


def test_empty_batch_and_streams(mr, ctx):
    keys = load_keys("rsa1024_x64")[:8]
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"]) for k in keys]
    x = torch.zeros((0, 32), dtype=torch.int32, device="cuda")
    ctx.mr_rsa_encrypt([], x, x)
    s = torch.cuda.Stream()
    msgs = [k["N"] // 3 for k in keys]
    m = mr.to_tensor(msgs, 32)
    c = torch.zeros_like(m)
    with torch.cuda.stream(s):
        ctx.mr_rsa_encrypt(hk, m, c, stream=s)
    s.synchronize()
    assert mr.from_tensor(c) == [pow(mv, k["e"], k["N"]) for mv, k in zip(msgs, keys)]


def test_rsa2048_full_workload_sampled(mr, ctx):
    """The benchmark's configuration (4096 ciphertexts over 16 keys, one call):
    a seeded sample checked against the oracle, every output checked by the
    round-trip property m^e mod N == c."""
    keys = load_keys("rsa2048_x16")
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
    n = 4096
    r = SplitMix64(0x4D520002)
    idx = [i // 256 for i in range(n)]
    cts = [r.below(keys[i]["N"]) for i in idx]
    c = mr.to_tensor(cts, 64)
    m = torch.zeros_like(c)
    st = _status(n)
    ctx.mr_rsa_decrypt_crt([hk[i] for i in idx], c, m, st)
    torch.cuda.synchronize()
    assert int((st != 0).sum()) == 0
    got = mr.from_tensor(m)
    rs = SplitMix64(99)
    for _ in range(24):
        j = rs.below(n)
        k = keys[idx[j]]
        assert got[j] == plain.rsa_decrypt_crt(cts[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]), j
    for j in range(n):
        assert pow(got[j], 65537, keys[idx[j]]["N"]) == cts[j], j


@pytest.mark.parametrize("bits", [512, 1024, 1536, 2048, 3072, 4096])
def test_modexp_every_lane_mapping(mr, bits):
    """Every compiled lane mapping of every class gives the oracle's results (the default mapping is
    covered above; this selects each one explicitly on a fresh context)."""
    lanes = mr.mr_class_variants(bits)
    if bits == 512:
        pool = load_keys("rsa1024_x64")
    elif bits == 4096:
        pool = load_keys("rsa8192_x2")
    else:
        pool = [k for k in load_keys("mix_x256") if k["bits"] == 2 * bits]
    for v in range(len(lanes)):
        c = mr.Context(0)
        try:
            c.mr_set_variant(bits, v)
            _modexp_case(mr, c, [bits] * 41, [min(bits, 384)] * 41, 1000 + 10 * v + bits % 7)
            if pool:  # CRT decryption: both halves and the recombination run in this class
                keys = pool[:3]
                nk = len(keys)
                hk = [c.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
                r = SplitMix64(2000 + v + bits)
                cts = [r.below(keys[j % nk]["N"]) for j in range(9)]
                ct = mr.to_tensor(cts, 2 * bits // 32)
                m = torch.zeros_like(ct)
                c.mr_rsa_decrypt_crt([hk[j % nk] for j in range(9)], ct, m)
                torch.cuda.synchronize()
                got = mr.from_tensor(m)
                for j in range(9):
                    k = keys[j % nk]
                    assert got[j] == plain.rsa_decrypt_crt(cts[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]), (v, j)
        finally:
            c.close()
