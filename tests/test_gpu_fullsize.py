"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.  Sampled
outputs are compared with the oracle one by one, and every output is checked where a cheap
complete check exists: decryptions by re-encryption with e = 65537, the long-exponent results by
CPython's pow through the CRT over the moduli's known factors (a spawned process pool).

  RSA-2048 CRT decryption: 4096 ciphertexts over 16 keys in one call (8192 exponentiations)
  long exponent: 256 x 16384-bit moduli, 16128-bit exponents, one cooperative launch, on the
                 tensor-core and the integer form of the base extensions
  ragged mix: 65,536 requests over 256 keys through the persistent graph-captured plan
"""
import multiprocessing as mp
import os

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
        allm = mr.from_tensor(m)
        bad = [j for j, (mv, i) in enumerate(zip(allm, idx)) if pow(mv, keys[i]["e"], keys[i]["N"]) != cts[j]]
        assert not bad, bad[:8]
    finally:
        ctx.close()


@pytest.fixture(scope="module")
def long_exponent_expected():
    """Every expected output of the long-exponent workload, by CPython's pow through the CRT on a
    spawned pool (spawned: a forked child of a CUDA process may hang)."""
    from crt_pow import crt_modexp
    keys, idx, xs, es = bench.big_workload(0)
    jobs = [(x, e, keys[i]["p"], keys[i]["q"]) for x, e, i in zip(xs, es, idx)]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4)) as pool:
        want = pool.map(crt_modexp, jobs, chunksize=4)
    return keys, idx, xs, es, want


@pytest.mark.parametrize("variant", [None, 0, 1], ids=["default", "integer", "tensor"])
def test_long_exponent_full_batch(mr, long_exponent_expected, variant):
    """All 256 outputs, with the class's default variant and with each form of the base
    extensions pinned; a sample also against the oracle's own square-and-multiply."""
    keys, idx, xs, es, want = long_exponent_expected
    ctx = mr.Context(0)
    try:
        if variant is not None:
            ctx.mr_set_variant(16384, variant)
        hk = [ctx.mr_rns_setup(k["N"]) for k in keys]
        x = mr.to_tensor(xs, 512)
        e = mr.to_tensor(es, bench.BIG_EBITS // 32)
        out = torch.zeros_like(x)
        st = torch.full((len(xs),), 255, dtype=torch.uint8, device="cuda")
        ctx.mr_modexp_batch(mr.KeyList([hk[i] for i in idx]), x, e, out, st)
        torch.cuda.synchronize()
        assert int(st.sum()) == 0
        got = mr.from_tensor(out)
        bad = [j for j in range(len(xs)) if got[j] != want[j]]
        assert not bad, bad[:8]
        if variant is None:
            for j in _samples(len(xs), 2, 12):  # the oracle takes ~2-4 s per 16384-bit exponentiation
                assert got[j] == plain.modexp(xs[j], es[j], keys[idx[j]]["N"]), j
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
        # every decryption re-encrypts to its ciphertext; 1024 more encryptions against pow
        allo = mr.from_tensor(out)
        bad = [j for j in range(len(xs)) if ops[j] == 1 and pow(allo[j], keys[idx[j]]["e"], keys[idx[j]]["N"]) != xs[j]]
        assert not bad, bad[:8]
        enc = [j for j in range(len(xs)) if ops[j] == 0]
        r = SplitMix64(0x454E43)
        for j in sorted({enc[r.below(len(enc))] for _ in range(1024)}):
            k = keys[idx[j]]
            assert allo[j] == pow(xs[j], k["e"], k["N"]), j
    finally:
        ctx.close()
