"""The autotuner picks a lane mapping and a window cap per size class by timing; results
of later calls stay equal to the oracle whatever it picks."""
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


def test_autotune_then_exact(mr):
    ctx = mr.Context(0)
    try:
        lanes = mr.mr_class_variants(1024)
        res = ctx.mr_autotune(1024, 512, 1024)
        assert 0 <= res["variant"] < len(lanes)
        assert res["lanes_per_number"] == lanes[res["variant"]]
        assert 1 <= res["window"] <= 6
        assert res["configs"] >= 3 and res["ms"] > 0 and res["ms_default"] > 0
        assert res["ms"] <= res["ms_default"] * 1.0001
        keys = load_keys("rsa2048_x16")[:4]
        hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
        r = SplitMix64(77)
        cts = [r.below(keys[i % 4]["N"]) for i in range(40)]
        c = mr.to_tensor(cts, 64)
        m = torch.zeros_like(c)
        ctx.mr_rsa_decrypt_crt([hk[i % 4] for i in range(40)], c, m)
        torch.cuda.synchronize()
        got = mr.from_tensor(m)
        for i in range(40):
            k = keys[i % 4]
            assert got[i] == plain.rsa_decrypt_crt(cts[i], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]), i
    finally:
        ctx.close()


def test_plan_autotune_flag_same_results(mr):
    ctx = mr.Context(0)
    try:
        keys = load_keys("mix_x256")
        chosen = [keys[i] for i in (0, 1, 120, 200, 250)]
        hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in chosen]
        r = SplitMix64(78)
        n = 60
        idx = [r.below(len(chosen)) for _ in range(n)]
        ops = [r.below(2) for _ in range(n)]
        xs = [r.below(chosen[i]["N"]) for i in idx]
        inp = mr.to_tensor(xs, 128)
        ref = torch.zeros_like(inp)
        ctx.mr_rsa_mixed([hk[i] for i in idx], ops, inp, ref)
        out = torch.zeros_like(inp)
        plan = ctx.mr_plan_create([hk[i] for i in idx], ops, inp, out,
                                  flags=mr.MR_PLAN_AUTOTUNE | mr.MR_PLAN_CONCURRENT | mr.MR_PLAN_PERSISTENT | mr.MR_PLAN_GRAPH)
        plan.launch()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        plan.free()
        got = mr.from_tensor(ref[:6])
        for j in range(6):
            k = chosen[idx[j]]
            want = pow(xs[j], k["e"] if ops[j] == 0 else k["d"], k["N"])
            assert got[j] == want
    finally:
        ctx.close()


def test_autotune_large_class_then_exact(mr):
    """The tuner on a large class (its channel-slice widths; window widths up to 8) and exact results
    after."""
    ctx = mr.Context(0)
    try:
        lanes = mr.mr_class_variants(8192)
        res = ctx.mr_autotune(8192, 40, 96)
        assert 0 <= res["variant"] < len(lanes) and res["lanes_per_number"] == lanes[res["variant"]]
        assert res["configs"] >= len(lanes)
        assert 1 <= res["window"] <= 8 and res["ms"] > 0
        r = SplitMix64(79)
        N = r.randbits(8192) | 1 | (1 << 8191)
        h = ctx.mr_rns_setup(N)
        xs = [r.below(N) for _ in range(33)]
        es = [r.randbits(96) for _ in range(33)]
        x = mr.to_tensor(xs, 256)
        e = mr.to_tensor(es, 3)
        out = torch.zeros_like(x)
        ctx.mr_modexp_batch([h] * 33, x, e, out)
        torch.cuda.synchronize()
        got = mr.from_tensor(out)
        for j in range(33):
            assert got[j] == plain.modexp(xs[j], es[j], N), j
    finally:
        ctx.close()


def test_tuning_saved_and_loaded(mr, tmp_path):
    """An autotune result written to JSON and installed on a new context: the same lane mapping and
    window cap, the class counts as tuned, and results stay exact."""
    c1 = mr.Context(0)
    try:
        res = c1.mr_autotune(2048, 256, 1024)
        state = c1.save_tuning(str(tmp_path / "tune.json"))
        assert state["2048"] == {"variant": res["variant"], "window_cap": res["window"]}
    finally:
        c1.close()
    c2 = mr.Context(0)
    try:
        assert not c2.mr_get_tuning(2048)["tuned"]
        c2.load_tuning(str(tmp_path / "tune.json"))
        t = c2.mr_get_tuning(2048)
        assert t == {"variant": res["variant"], "window_cap": res["window"], "tuned": True}
        with pytest.raises(mr.MRError):
            c2.mr_set_tuning(2048, 99, 0)
        keys = load_keys("mix_x256")
        ks = [k for k in keys if k["bits"] == 2048][:3]
        hk = [c2.mr_rsa_key_setup(k["N"], k["e"]) for k in ks]
        r = SplitMix64(81)
        msgs = [r.below(k["N"]) for k in ks]
        m = mr.to_tensor(msgs, 64)
        c = torch.zeros_like(m)
        c2.mr_rsa_encrypt(hk, m, c)
        torch.cuda.synchronize()
        got = mr.from_tensor(c)
        for i, k in enumerate(ks):
            assert got[i] == plain.rsa_encrypt(msgs[i], k["e"], k["N"])
    finally:
        c2.close()
