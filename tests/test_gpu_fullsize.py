"""Parity at the benchmark's full sizes, in the launch configuration bench.py times, on
sampled outputs that the oracle computes one by one (every output of the smaller
configurations is checked in test_gpu_parity.py).

  RSA-2048 CRT decryption: 4096 ciphertexts over 16 keys in one call (8192 exponentiations)
  long exponent: 256 x 16384-bit moduli, 16128-bit exponents, one cooperative launch
  ragged mix: 65,536 requests over 256 keys through the persistent graph-captured plan
"""
import pytest

import bench
from oracle import plain
from synth import SplitMix64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mr():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_3699_gb300 import mr as m
    return m


def _samples(n, count, seed):
    r = SplitMix64(seed)
    picks = {0, n - 1}
    while len(picks) < count:
        picks.add(r.below(n))
    return sorted(picks)


def test_rsa2048_crt_full_batch(mr):
    keys, idx, cts = bench.workload(0)
    ctx = mr.Context(0)
    try:
        hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
        c = mr.to_tensor(cts, 64)
        m = torch.zeros_like(c)
        st = torch.full((len(cts),), 255, dtype=torch.uint8, device="cuda")
        ctx.mr_rsa_decrypt_crt(mr.KeyList([hk[i] for i in idx]), c, m, st)
        torch.cuda.synchronize()
        assert int(st.sum()) == 0
        for j in _samples(len(cts), 64, 11):
            k = keys[idx[j]]
            got = mr.from_tensor(m[j:j + 1])[0]
            assert got == plain.rsa_decrypt_crt(cts[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]), j
    finally:
        ctx.close()


def test_long_exponent_full_batch(mr):
    keys, idx, xs, es = bench.big_workload(0)
    ctx = mr.Context(0)
    try:
        hk = [ctx.mr_rns_setup(k["N"]) for k in keys]
        x = mr.to_tensor(xs, 512)
        e = mr.to_tensor(es, bench.BIG_EBITS // 32)
        out = torch.zeros_like(x)
        st = torch.full((len(xs),), 255, dtype=torch.uint8, device="cuda")
        ctx.mr_modexp_batch(mr.KeyList([hk[i] for i in idx]), x, e, out, st)
        torch.cuda.synchronize()
        assert int(st.sum()) == 0
        for j in _samples(len(xs), 4, 12):  # the oracle takes ~2-4 s per 16384-bit exponentiation
            got = mr.from_tensor(out[j:j + 1])[0]
            assert got == plain.modexp(xs[j], es[j], keys[idx[j]]["N"]), j
    finally:
        ctx.close()


def test_ragged_mix_full_plan(mr):
    keys, idx, ops, xs = bench.ragged_workload(0)
    ctx = mr.Context(0)
    try:
        hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
        kl = mr.KeyList([hk[i] for i in idx])
        inp = mr.to_tensor(xs, 128)
        out = torch.zeros_like(inp)
        st = torch.full((len(xs),), 255, dtype=torch.uint8, device="cuda")
        flags = mr.MR_PLAN_CONCURRENT | mr.MR_PLAN_PERSISTENT | mr.MR_PLAN_GRAPH
        plan = ctx.mr_plan_create(kl, ops, inp, out, st, flags=flags)
        plan.launch()
        torch.cuda.synchronize()
        plan.free()
        assert int(st.sum()) == 0
        for j in _samples(len(xs), 96, 13):
            k = keys[idx[j]]
            got = mr.from_tensor(out[j:j + 1])[0]
            if ops[j] == 0:
                want = plain.rsa_encrypt(xs[j], k["e"], k["N"])
            else:
                want = plain.rsa_decrypt_crt(xs[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
            assert got == want, j
    finally:
        ctx.close()
