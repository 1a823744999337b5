"""Tensor-core building blocks of the base extension (Sec. 3.1: the extensions are products with
constant matrices): the tcgen05 operand layout gives exact products of small integers, and the
throughput probes report plausible rates."""
import numpy as np
import pytest

from synth import SplitMix64

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _ints(r, rows, cols, hi):
    return np.array([[r.below(hi) for _ in range(cols)] for _ in range(rows)], dtype=np.float64)


@pytest.mark.parametrize("a_in_tmem", [0, 1])
@pytest.mark.parametrize("n,kdim", [(128, 64), (16, 16), (64, 32), (128, 16)])
def test_tc_mma_exact_small_integers(n, kdim, a_in_tmem):
    """7-bit integers (the slice width of the extension): every partial sum stays below 2^24, so
    fp32 accumulation is exact and D must equal the integer product A B^T exactly; with A in
    shared memory and with A in tensor memory (the resident-matrix layout)."""
    _need_gpu()
    from paper_1305_3699_gb300 import mr

    r = SplitMix64(n * 1000 + kdim)
    a = _ints(r, 128, kdim, 128)
    b = _ints(r, n, kdim, 128)
    with mr.Context(0) as ctx:
        d = ctx.mr_debug_tc_mma(a, b, swap_strides=2 if a_in_tmem else 0)
    want = a @ b.T
    assert np.array_equal(d.astype(np.float64), want), np.argwhere(d != want)[:8]


@pytest.mark.parametrize("n,kdim,off_col", [(96, 32, 3), (160, 64, 5), (224, 64, 7)])
def test_tc_mma_lane_group_extension_shape(n, kdim, off_col):
    """The lane-group extension's product: 8-bit integer slices in fp16, N = 32 x (channels per lane)
    columns, and one K column of 2048 x 4096 that adds 2^23 to every accumulator.  Every sum lies in
    [2^23, 2^24) and must come back exact (the integer is then the fp32 value's mantissa)."""
    _need_gpu()
    from paper_1305_3699_gb300 import mr

    r = np.random.default_rng(n)
    a = r.integers(0, 256, size=(128, kdim)).astype(np.float64)
    b = r.integers(0, 256, size=(n, kdim)).astype(np.float64)
    a[:, off_col] = 2048.0
    b[:, off_col] = 4096.0
    a[:3, :] = 255.0  # the largest sums
    b[:3, :] = 255.0
    a[:3, off_col] = 2048.0
    b[:3, off_col] = 4096.0
    want = a @ b.T
    assert want.min() >= 2 ** 23 and want.max() < 2 ** 24
    with mr.Context(0) as ctx:
        d = ctx.mr_debug_tc_mma(a, b)
    assert np.array_equal(d.astype(np.float64), want), np.argwhere(d != want)[:8]
    bits = d.view(np.uint32)
    assert np.array_equal((bits & 0x7FFFFF).astype(np.float64), want - 2 ** 23)


def test_tc_ld_16x256b_layout():
    """The 16x256b tensor-memory load returns, to thread i of a warp, lane i / 4 and lane i / 4 + 8 of
    each 16-lane half at columns 2 (i % 4) and + 1 of each 8-column group: D[r][c] = 256 r + c read back
    through that layout (swap_strides 3) lands at every (r, c)."""
    _need_gpu()
    from paper_1305_3699_gb300 import mr

    for n in (16, 144):
        a = np.zeros((128, 16))
        b = np.zeros((n, 16))
        a[:, 0] = np.arange(128)
        b[:, 0] = 256.0
        a[:, 1] = 1.0
        b[:, 1] = np.arange(n)
        with mr.Context(0) as ctx:
            d = ctx.mr_debug_tc_mma(a, b, swap_strides=3)
        want = a @ b.T
        assert np.array_equal(d.astype(np.float64), want), d[:2, :16]


def test_tc_mma_distinguishes_rows_and_columns():
    """A one-hot pattern: row i of A and row j of B share exactly one non-zero column, so each
    output names the pair it came from (a transposed or shifted operand would move the values)."""
    _need_gpu()
    from paper_1305_3699_gb300 import mr

    kdim, n = 64, 128
    a = np.zeros((128, kdim))
    b = np.zeros((n, kdim))
    for i in range(128):
        a[i, i % kdim] = 1 + i // kdim
    for j in range(n):
        b[j, (3 * j) % kdim] = 1 + j % 7
    with mr.Context(0) as ctx:
        d = ctx.mr_debug_tc_mma(a, b)
        d2 = ctx.mr_debug_tc_mma(a, b, swap_strides=2)
    assert np.array_equal(d.astype(np.float64), a @ b.T)
    assert np.array_equal(d2.astype(np.float64), a @ b.T)


def test_tensor_peaks_plausible():
    """Every probe completes and reports a rate between 1 TOP/s and 10 POP/s."""
    _need_gpu()
    from paper_1305_3699_gb300 import mr

    with mr.Context(0) as ctx:
        for kind in (0, 1, 2):
            v = ctx.mr_tensor_peak(kind)
            assert 1e12 < v < 1e16, (kind, v)
        for kind in (0, 1, 2, 3):
            v = ctx.mr_imad_peak(kind)
            assert 1e11 < v < 1e14, (kind, v)


def test_lane_tc_bounded_wait_times_out_and_context_recovers():
    """The 1024-bit class's tensor-core kernel with no product issued (test hook): every block's
    completion wait runs out after its limit (about a second), the call completes, every item reports
    MR_ERR_TIMEOUT (8), and the next call on the same context gives the oracle's results."""
    _need_gpu()
    from oracle import plain
    from paper_1305_3699_gb300 import mr

    assert mr.mr_lane_variant_info(1024, 0)["tensor"]
    r = SplitMix64(4242)
    n = 40  # two blocks, the second one ragged
    N = r.randbits(1024) | 1 | (1 << 1023)
    xs = [r.below(N) for _ in range(n)]
    es = [r.randbits(1024) for _ in range(n)]
    with mr.Context(0) as ctx:
        h = ctx.mr_rns_setup(N)
        x, e = mr.to_tensor(xs, 32), mr.to_tensor(es, 32)
        out = torch.zeros_like(x)
        st = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        ctx.mr_debug_lane_tc_wait(True)
        try:
            ctx.mr_modexp_batch([h] * n, x, e, out, st)
            torch.cuda.synchronize()
        finally:
            ctx.mr_debug_lane_tc_wait(False)
        assert st.cpu().tolist() == [8] * n
        st.fill_(255)
        ctx.mr_modexp_batch([h] * n, x, e, out, st)
        torch.cuda.synchronize()
        assert st.cpu().tolist() == [0] * n
        got = mr.from_tensor(out)
    assert got == [plain.modexp(a, b, N) for a, b in zip(xs, es)]
