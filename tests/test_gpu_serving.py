"""The serving loop: every request's result is the same whether it is served in the
continuous-batching loop (mixed with whatever arrived around it), in one mixed call over
all requests, or alone, and equals the oracle."""
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


def test_served_results_alone_and_in_the_mix(mr):
    from paper_1305_3699_gb300 import serve
    ctx = mr.Context(0)
    try:
        keys = load_keys("mix_x256")
        chosen = [keys[i] for i in (0, 3, 110, 190, 240, 255)]
        hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in chosen]
        r = SplitMix64(0x4D520015)
        n = 3000
        idx = np.array([r.below(len(chosen)) for _ in range(n)])
        ops = np.array([r.below(2) for _ in range(n)])
        xs = [r.below(chosen[i]["N"]) for i in idx]
        rows = np.zeros((n, 128), dtype=np.uint32)
        for i, x in enumerate(xs):
            rows[i] = np.frombuffer(x.to_bytes(512, "little"), dtype="<u4")
        rows = rows.view(np.int32)
        arrivals = serve.poisson_arrivals(100_000.0, n, 0x4D520016)
        srv = serve.Server(ctx, hk, capacity=512, slots=3)
        out, status, lat, stats = srv.run(arrivals, idx, ops, rows, max_queue_s=30.0)
        assert stats["completed"] == n and stats["rejected"] == 0 and stats["batches"] > 1
        assert (status == 0).all()
        # one mixed call over all requests
        inp = torch.from_numpy(rows.copy()).cuda()
        mixed = torch.zeros_like(inp)
        ctx.mr_rsa_mixed([hk[i] for i in idx], [int(o) for o in ops], inp, mixed)
        torch.cuda.synchronize()
        assert np.array_equal(mixed.cpu().numpy(), out)
        # alone: single-request calls on a sample, and the oracle
        for j in list(range(0, n, 97))[:30]:
            one = torch.zeros((1, 128), dtype=torch.int32, device="cuda")
            ctx.mr_rsa_mixed([hk[idx[j]]], [int(ops[j])], inp[j:j + 1].contiguous(), one)
            torch.cuda.synchronize()
            assert np.array_equal(one.cpu().numpy()[0], out[j]), j
            k = chosen[idx[j]]
            got = int.from_bytes(out[j].view(np.uint32).astype("<u4").tobytes(), "little")
            want = (plain.rsa_encrypt(xs[j], k["e"], k["N"]) if ops[j] == 0 else
                    plain.rsa_decrypt_crt(xs[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]))
            assert got == want, j
    finally:
        ctx.close()


def test_admission_budget_rejects_and_limits(mr):
    from paper_1305_3699_gb300 import serve
    ctx = mr.Context(0)
    try:
        k = load_keys("rsa1024_x64")[0]
        h = ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
        n = 64
        r = SplitMix64(0x4D520017)
        xs = [r.below(k["N"]) for _ in range(n)]
        rows = np.zeros((n, 128), dtype=np.uint32)
        for i, x in enumerate(xs):
            rows[i, :32] = np.frombuffer(x.to_bytes(128, "little"), dtype="<u4")
        rows = rows.view(np.int32)
        foot = serve.request_footprint_bytes(1024, 1, 128)
        # a budget of two requests: every batch holds at most two, all complete
        srv = serve.Server(ctx, [h], capacity=64, slots=2, hbm_budget=2 * foot)
        arrivals = np.zeros(n)
        out, status, lat, stats = srv.run(arrivals, np.zeros(n, dtype=np.int64), np.ones(n, dtype=np.int64), rows,
                                          max_queue_s=60.0)
        assert stats["completed"] == n and stats["batches"] >= n // 2
        for j in (0, n - 1):
            got = int.from_bytes(out[j].view(np.uint32).astype("<u4").tobytes(), "little")
            assert got == plain.rsa_decrypt_crt(xs[j], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
    finally:
        ctx.close()
