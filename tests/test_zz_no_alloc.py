"""The allocation-free entry point gives exactly what the regular one gives.

mr_modexp_batch_noalloc serves callers that cannot allocate device memory at
call time (an engine that owns all GPU memory through its own pool, or a
latency-bound loop that must stay out of the CUDA allocator).  Its scratch is a
static device array shared by every call, so these tests make calls in a row
with different inputs -- each finds the previous call's tables in the array --
and compare every output against mr_modexp_batch bit for bit and a seeded
sample against the oracle's square-and-multiply (integer results: tolerance
zero).  The file is collected last and depends on no other test having run.
"""
import pytest

from oracle import plain
from synth import SplitMix64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# largest batch of a 1024-bit modulus with 32-limb exponent rows: window width 5, 4 warps per block
# of 32 numbers, 32 entries x 18 words x 32 lanes x 4 bytes per warp -> 56 blocks in 16 MiB
MAX_1024_E32 = (16 << 20) // (4 * 32 * 18 * 32 * 4) * 32


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _check(ctx, mr, key, N, xs, es, nl, el, stream=None, sample=16):
    n = len(xs)
    x = mr.to_tensor(xs, nl)
    e = mr.to_tensor(es, el)
    ref = torch.zeros_like(x)
    got = torch.full_like(x, -1)
    st = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
    ctx.mr_modexp_batch([key] * n, x, e, ref)
    ctx.mr_modexp_batch_noalloc(key, x, e, got, st, stream=stream)
    torch.cuda.synchronize()
    assert torch.equal(got, ref), "outputs differ from mr_modexp_batch"
    vals = mr.from_tensor(got)
    r = SplitMix64(n)
    for j in sorted({r.below(n) for _ in range(sample)}):
        assert vals[j] == plain.modexp(xs[j], es[j], N), j
    return vals, st.cpu().tolist()


def test_noalloc_matches_regular_entry_point_on_two_calls():
    _need_gpu()
    from paper_1305_3699_gb300 import mr

    r = SplitMix64(0x5A5A)
    with mr.Context(0) as ctx:
        for call, bits in enumerate((1024, 2048)):
            N = r.randbits(bits) | 1 | (1 << (bits - 1))
            key = ctx.mr_rns_setup(N)
            n = 300 + 37 * call
            nl = bits // 32
            xs = [r.below(N) for _ in range(n)]
            es = [r.randbits(bits) for _ in range(n)]
            _, st = _check(ctx, mr, key, N, xs, es, nl, nl)
            assert st == [0] * n
        # a batch larger than the static array is refused, not truncated
        big = 1 << 16
        xb = torch.zeros((big, 32), dtype=torch.int32, device="cuda")
        eb = torch.zeros((big, 32), dtype=torch.int32, device="cuda")
        N = r.randbits(1024) | 1 | (1 << 1023)
        key = ctx.mr_rns_setup(N)
        with pytest.raises(mr.MRError) as exc:
            ctx.mr_modexp_batch_noalloc(key, xb, eb, torch.zeros_like(xb))
        assert exc.value.code == 4


def test_noalloc_edge_values_and_status():
    """x = 0, 1, N-1, e = 0, 1, and rows with x >= N (status MR_ERR_RANGE = 5, output zero) mixed
    with ordinary rows, on a stream of the caller's."""
    _need_gpu()
    from paper_1305_3699_gb300 import mr

    r = SplitMix64(0xED6E)
    with mr.Context(0) as ctx:
        for bits in (512, 1024, 1536, 2048):
            N = r.randbits(bits) | 1 | (1 << (bits - 1))
            key = ctx.mr_rns_setup(N)
            nl = bits // 32
            xs = [0, 1, N - 1, N - 1, r.below(N), 0, N, N + 5, (1 << bits) - 1, r.below(N)]
            es = [r.randbits(bits), r.randbits(bits), 3, 2, 0, 0, 7, 7, 9, 1]
            bad = [x >= N for x in xs]
            x = mr.to_tensor(xs, nl)
            e = mr.to_tensor(es, nl)
            got = torch.full_like(x, -1)
            st = torch.full((len(xs),), 255, dtype=torch.uint8, device="cuda")
            s = torch.cuda.Stream()
            ctx.mr_modexp_batch_noalloc(key, x, e, got, st, stream=s)
            s.synchronize()
            vals = mr.from_tensor(got)
            stl = st.cpu().tolist()
            for j, (xv, ev) in enumerate(zip(xs, es)):
                if bad[j]:
                    assert stl[j] == 5 and vals[j] == 0, (bits, j)
                else:
                    assert stl[j] == 0 and vals[j] == plain.modexp(xv, ev, N), (bits, j)


def test_noalloc_largest_accepted_batch():
    """The largest batch the size check accepts runs, with the last warp's table at the end of the
    static array; one item more is refused, and the message names the limit."""
    _need_gpu()
    from paper_1305_3699_gb300 import mr

    r = SplitMix64(0x1A26E)
    with mr.Context(0) as ctx:
        N = r.randbits(1024) | 1 | (1 << 1023)
        key = ctx.mr_rns_setup(N)
        n = MAX_1024_E32
        xs = [r.below(N) for _ in range(n)]
        es = [r.randbits(1024) for _ in range(n)]
        _, st = _check(ctx, mr, key, N, xs, es, 32, 32, sample=24)
        assert st == [0] * n
        x = torch.zeros((n + 1, 32), dtype=torch.int32, device="cuda")
        with pytest.raises(mr.MRError) as exc:
            ctx.mr_modexp_batch_noalloc(key, x, x.clone(), torch.zeros_like(x))
        assert exc.value.code == 4 and str(MAX_1024_E32) in str(exc.value)
        # short exponents in one-limb rows: a smaller window, so more items fit than with 32-limb rows
        n2 = MAX_1024_E32 + 256
        xs2 = [r.below(N) for _ in range(n2)]
        es2 = [65537] * n2
        _, st2 = _check(ctx, mr, key, N, xs2, es2, 32, 1)
        assert st2 == [0] * n2
