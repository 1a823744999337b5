"""Mixed-size batches (mr_rsa_mixed, plans): results are the same in every launch
mode, the same as the single-operation calls, and equal to the oracle."""
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
def setup(mr):
    ctx = mr.Context(0)
    keys = load_keys("mix_x256")
    by_bits = {}
    for k in keys:
        by_bits.setdefault(k["bits"], []).append(k)
    chosen = [k for b in (1024, 2048, 3072, 4096) for k in by_bits[b][:3]]
    handles = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in chosen]
    r = SplitMix64(0x4D520004)
    n = 150
    idx = [r.below(len(chosen)) for _ in range(n)]
    ops = [r.below(2) for _ in range(n)]
    xs = [r.below(chosen[i]["N"]) for i in idx]
    xs[0] = 0
    xs[1] = chosen[idx[1]]["N"] - 1
    yield ctx, chosen, handles, idx, ops, xs
    ctx.close()


def expected(chosen, idx, ops, xs, j):
    k = chosen[idx[j]]
    if ops[j] == 0:
        return plain.rsa_encrypt(xs[j], k["e"], k["N"])
    return plain.rsa_decrypt_crt(xs[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])


def test_mixed_all_modes_agree_with_single_calls_and_oracle(mr, setup):
    ctx, chosen, handles, idx, ops, xs = setup
    n = len(idx)
    keys = [handles[i] for i in idx]
    inp = mr.to_tensor(xs, 128)
    # single-operation calls
    ref = torch.zeros_like(inp)
    enc = [j for j in range(n) if ops[j] == 0]
    dec = [j for j in range(n) if ops[j] == 1]
    for sel, call in ((enc, ctx.mr_rsa_encrypt), (dec, ctx.mr_rsa_decrypt_crt)):
        sub_in = inp[sel].contiguous()
        sub_out = torch.zeros_like(sub_in)
        call([keys[j] for j in sel], sub_in, sub_out)
        ref[sel] = sub_out
    torch.cuda.synchronize()
    refv = mr.from_tensor(ref)
    r = SplitMix64(5)
    for _ in range(30):
        j = r.below(n)
        assert refv[j] == expected(chosen, idx, ops, xs, j), j
    for j in (0, 1):
        assert refv[j] == expected(chosen, idx, ops, xs, j)
    for flags in (0, mr.MR_PLAN_CONCURRENT, mr.MR_PLAN_PERSISTENT, mr.MR_PLAN_CONCURRENT | mr.MR_PLAN_PERSISTENT):
        out = torch.full_like(inp, -1)
        st = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        ctx.mr_rsa_mixed(keys, ops, inp, out, st, flags=flags)
        torch.cuda.synchronize()
        assert torch.equal(out, ref), flags
        assert int(st.sum()) == 0


def test_plans_replay_with_new_inputs(mr, setup):
    ctx, chosen, handles, idx, ops, xs = setup
    n = len(idx)
    keys = [handles[i] for i in idx]
    inp = mr.to_tensor(xs, 128)
    ref = torch.zeros_like(inp)
    ctx.mr_rsa_mixed(keys, ops, inp, ref)
    r = SplitMix64(6)
    xs2 = [r.below(chosen[i]["N"]) for i in idx]
    inp2 = mr.to_tensor(xs2, 128)
    ref2 = torch.zeros_like(inp2)
    ctx.mr_rsa_mixed(keys, ops, inp2, ref2)
    torch.cuda.synchronize()
    for flags in (0, mr.MR_PLAN_GRAPH, mr.MR_PLAN_CONCURRENT | mr.MR_PLAN_PERSISTENT | mr.MR_PLAN_GRAPH,
                  mr.MR_PLAN_PERSISTENT):
        buf_in = inp.clone()
        buf_out = torch.zeros_like(inp)
        plan = ctx.mr_plan_create(keys, ops, buf_in, buf_out, flags=flags)
        info = plan.info()
        assert info["groups"] >= 4 and info["kernels"] >= info["groups"]
        plan.launch()
        torch.cuda.synchronize()
        assert torch.equal(buf_out, ref), flags
        buf_in.copy_(inp2)
        plan.launch()
        torch.cuda.synchronize()
        assert torch.equal(buf_out, ref2), flags
        plan.free()
    j = 3
    assert mr.from_tensor(ref2[j:j + 1])[0] == expected(chosen, idx, ops, xs2, j)


def test_mixed_range_errors(mr, setup):
    ctx, chosen, handles, idx, ops, xs = setup
    keys = [handles[i] for i in idx[:8]]
    bad = [chosen[idx[j]]["N"] + (j % 2) for j in range(8)]  # N and N+1: both out of range
    inp = mr.to_tensor(bad, 128)
    out = torch.zeros_like(inp)
    st = torch.zeros(8, dtype=torch.uint8, device="cuda")
    ctx.mr_rsa_mixed(keys, [0, 1] * 4, inp, out, st, flags=mr.MR_PLAN_PERSISTENT)
    torch.cuda.synchronize()
    assert st.cpu().tolist() == [5] * 8


def test_mixed_batch_with_large_requests(mr):
    """One mr_rsa_mixed call over 2048-, 8192- and 16384-bit keys: 8192-bit encryptions and 16384-bit
    encryptions and decryptions run in the large classes (16384-bit decryptions as 8192-bit CRT halves
    plus the binary recombination), 8192-bit decryptions as 4096-bit halves with the lane-group
    requests; every result equals the oracle's, and a plan refuses the large requests."""
    keys = load_keys("rsa2048_x16")[:3] + load_keys("rsa8192_x2") + load_keys("mod16384_x4")[:2]
    r = SplitMix64(0x4C41524745)
    with mr.Context(0) as ctx:
        hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
        # key index, operation: small and large requests interleaved; 16384-bit decryptions kept few
        # (the oracle takes seconds for each)
        reqs = [(0, 0), (5, 0), (3, 1), (1, 1), (6, 0), (4, 0), (5, 1), (2, 0), (3, 0), (0, 1), (6, 0), (4, 1)]
        xs = [r.below(keys[i]["N"]) for i, _ in reqs]
        inp = mr.to_tensor(xs, 512)
        out = torch.full_like(inp, -1)
        st = torch.full((len(reqs),), 255, dtype=torch.uint8, device="cuda")
        ctx.mr_rsa_mixed([hk[i] for i, _ in reqs], [o for _, o in reqs], inp, out, st,
                         flags=mr.MR_PLAN_CONCURRENT)
        torch.cuda.synchronize()
        got = mr.from_tensor(out)
        assert st.cpu().tolist() == [0] * len(reqs)
        for j, (i, o) in enumerate(reqs):
            k = keys[i]
            want = plain.rsa_encrypt(xs[j], k["e"], k["N"]) if o == 0 else \
                plain.rsa_decrypt_crt(xs[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
            assert got[j] == want, (j, k["N"].bit_length(), o)
        with pytest.raises(mr.MRError) as exc:
            ctx.mr_plan_create([hk[5]], [0], inp[:1], out[:1])
        assert exc.value.code == 4
