"""Constant-time schedule (mr_set_constant_time): regular fixed windows over every exponent limb, a
multiplication for every window and masked table reads give exactly the results of the default
schedule.  Checked against the oracle's square-and-multiply on RSA-2048 CRT decryptions (halves whose
warps share an exponent, where the default runs sliding windows), on exponents with runs of zero
digits, zero limbs and the edge values, and on a mixed plan of encryptions and decryptions."""
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


def test_constant_time_crt_decryption_matches_oracle(mr):
    keys = load_keys("rsa2048_x16")
    r = SplitMix64(0xC7C7)
    with mr.Context(0) as ctx:
        hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
        idx = [i // 8 for i in range(128)]  # 8 ciphertexts per key: warps share an exponent
        cts = [r.below(keys[i]["N"]) for i in idx]
        c = mr.to_tensor(cts, 64)
        outs = []
        for ct in (False, True):
            ctx.mr_set_constant_time(ct)
            m = torch.zeros_like(c)
            st = torch.full((len(cts),), 255, dtype=torch.uint8, device="cuda")
            ctx.mr_rsa_decrypt_crt([hk[i] for i in idx], c, m, st)
            torch.cuda.synchronize()
            assert st.cpu().tolist() == [0] * len(cts)
            outs.append(m.clone())
        assert torch.equal(outs[0], outs[1])
        got = mr.from_tensor(outs[1])
        for j in range(0, len(cts), 7):
            k = keys[idx[j]]
            assert got[j] == plain.rsa_decrypt_crt(cts[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]), j


@pytest.mark.parametrize("bits", [512, 1024, 2048, 4096])
def test_constant_time_modexp_edge_exponents(mr, bits):
    r = SplitMix64(bits)
    N = r.randbits(bits) | 1 | (1 << (bits - 1))
    nl = bits // 32
    es = [0, 1, 2, 3, (1 << (bits - 1)), (1 << 64) - 1, r.randbits(bits), r.randbits(bits) & ~((1 << 300) - 1),
          r.randbits(40), (r.randbits(bits) >> 7) << 7]
    xs = [r.below(N) for _ in es]
    xs[1], xs[2] = 0, N - 1
    with mr.Context(0) as ctx:
        key = ctx.mr_rns_setup(N)
        ctx.mr_set_constant_time(True)
        x = mr.to_tensor(xs, nl)
        e = mr.to_tensor(es, nl)
        out = torch.full_like(x, -1)
        st = torch.full((len(es),), 255, dtype=torch.uint8, device="cuda")
        ctx.mr_modexp_batch([key] * len(es), x, e, out, st)
        torch.cuda.synchronize()
        got = mr.from_tensor(out)
    assert st.cpu().tolist() == [0] * len(es)
    for j, (xv, ev) in enumerate(zip(xs, es)):
        assert got[j] == plain.modexp(xv, ev, N), j


def test_constant_time_mixed_plan(mr):
    keys = load_keys("mix_x256")
    r = SplitMix64(0x4D4958)
    with mr.Context(0) as ctx:
        pick = [r.below(len(keys)) for _ in range(96)]
        ops = [r.below(2) for _ in pick]
        hk = {i: ctx.mr_rsa_key_setup(keys[i]["N"], keys[i]["e"], keys[i]["p"], keys[i]["q"], keys[i]["dp"],
                                      keys[i]["dq"], keys[i]["qinv"]) for i in set(pick)}
        xs = [r.below(keys[i]["N"]) for i in pick]
        inp = mr.to_tensor(xs, 128)
        out = torch.zeros_like(inp)
        ctx.mr_set_constant_time(True)
        plan = ctx.mr_plan_create(mr.KeyList([hk[i] for i in pick]), ops, inp, out,
                                  flags=mr.MR_PLAN_GRAPH | mr.MR_PLAN_CONCURRENT)
        ctx.mr_set_constant_time(False)  # the plan keeps the setting it was created with
        plan.launch()
        torch.cuda.synchronize()
        plan.free()
        got = mr.from_tensor(out)
    for j, (i, o) in enumerate(zip(pick, ops)):
        k = keys[i]
        want = plain.rsa_encrypt(xs[j], k["e"], k["N"]) if o == 0 else \
            plain.rsa_decrypt_crt(xs[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
        assert got[j] == want, j
