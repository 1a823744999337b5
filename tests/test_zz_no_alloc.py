"""The allocation-free entry point gives exactly what the regular one gives.

mr_modexp_batch_noalloc serves callers that cannot allocate device memory at
call time (an engine that owns all GPU memory through its own pool, or a
latency-bound loop that must stay out of the CUDA allocator).  Its scratch is a
static device array shared by every call, so this test makes two calls in a row
with different inputs -- the second finds the first call's tables in the array
-- and compares each against mr_modexp_batch bit for bit (integer results:
tolerance zero).  It is collected last (file name) and does not depend on any
other test having run.
"""
import pytest

from synth import SplitMix64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_noalloc_matches_regular_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_3699_gb300 import mr

    r = SplitMix64(0x5A5A)
    with mr.Context(0) as ctx:
        for call, bits in enumerate((1024, 2048)):
            N = r.randbits(bits) | 1 | (1 << (bits - 1))
            key = ctx.mr_rns_setup(N)
            n = 300 + 37 * call
            nl = bits // 32
            x = mr.to_tensor([r.below(N) for _ in range(n)], nl)
            e = mr.to_tensor([r.randbits(bits) for _ in range(n)], nl)
            ref = torch.zeros_like(x)
            got = torch.full_like(x, -1)
            st = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
            ctx.mr_modexp_batch([key] * n, x, e, ref)
            ctx.mr_modexp_batch_noalloc(key, x, e, got, st)
            torch.cuda.synchronize()
            assert torch.equal(got, ref), f"call {call}: outputs differ"
            assert st.cpu().tolist() == [0] * n
        # a batch larger than the static array is refused, not truncated
        big = 1 << 16
        xb = torch.zeros((big, 32), dtype=torch.int32, device="cuda")
        eb = torch.zeros((big, 32), dtype=torch.int32, device="cuda")
        N = r.randbits(1024) | 1 | (1 << 1023)
        key = ctx.mr_rns_setup(N)
        with pytest.raises(mr.MRError) as exc:
            ctx.mr_modexp_batch_noalloc(key, xb, eb, torch.zeros_like(xb))
        assert exc.value.code == 4
