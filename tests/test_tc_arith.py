"""The arithmetic the lane-group classes' tensor-core form relies on (Sec. 3.1: the base extensions
are products with constant matrices), checked on the CPU with each class's own channel primes and
extension matrices: byte slices of the CRT coefficients and matrix entries, every slice sum below
2^23 (so an fp32 accumulator offset by 2^23 holds it exactly in its mantissa), and the digit-sum
recombination giving back the exact 64-bit dot product.  The kernel's agreement with this
arithmetic is what the -m gpu parity tests check on every output."""
import numpy as np
import pytest

from synth import SplitMix64

mr = pytest.importorskip("paper_1305_3699_gb300.mr")

OFF = 0x4B000000  # bit pattern of the fp32 value 2^23


def _class(L):
    k = mr.mr_class_for_bits(L)[1]
    B = mr.mr_debug_class_table(L, "B")
    Bp = mr.mr_debug_class_table(L, "Bp")
    M_mi_Bp = mr.mr_debug_class_table(L, "M_mi_Bp")
    Mp_mj_B = mr.mr_debug_class_table(L, "Mp_mj_B")
    # the device matrices carry the factor 2^64 of the one reduction that follows the dot product
    T1 = [[M_mi_Bp[i * k + j] * (1 << 64) % Bp[j] for j in range(k)] for i in range(k)]
    T2 = [[Mp_mj_B[j * k + i] * (1 << 64) % B[i] for i in range(k)] for j in range(k)]
    return k, B, Bp, T1, T2


def _combine(P, k):
    """The kernel's recombination (tc_combine): P[a][b] are the 16 fp32 bit patterns 2^23 + P_ab."""
    M = 1 << 32
    v = [[(OFF + P[a][b]) % M for b in range(4)] for a in range(4)]
    w = [sum(v[a][s - a] for a in range(4) if 0 <= s - a < 4) % M for s in range(7)]
    n = [sum(1 for a in range(4) if 0 <= s - a < 4) for s in range(7)]  # terms per digit: 1 2 3 4 3 2 1
    x0 = (w[0] + (w[1] << 8) - (n[0] * OFF + ((n[1] * OFF) << 8))) % M
    x2 = (w[4] + (w[5] << 8) - (n[4] * OFF + ((n[5] * OFF) << 8))) % M
    x3 = (w[6] - n[6] * OFF) % M
    if k * 65025 * (4 * 256 + 3) < M:
        x1 = (w[2] + (w[3] << 8) - (n[2] * OFF + ((n[3] * OFF) << 8))) % M
        return (x0 + (x1 << 16) + (x2 << 32) + (x3 << 48)) % (1 << 64)
    y2, y3 = (w[2] - n[2] * OFF) % M, (w[3] - n[3] * OFF) % M
    return (x0 + (y2 << 16) + (y3 << 24) + (x2 << 32) + (x3 << 48)) % (1 << 64)


def test_tensor_variants_of_the_lane_group_classes():
    """Which lane mappings run the extensions on the tensor cores: the default of the 1024-, 1536- and
    2048-bit classes (32 numbers per block: 4 lanes in one warp, or 8 over two warps), a variant of
    the 512-bit class, none of the 3072- and 4096-bit classes."""
    want = {1024: (4, 128), 1536: (8, 256), 2048: (8, 256)}
    for L, (lanes, threads) in want.items():
        v = mr.mr_lane_variant_info(L, 0)
        assert v == {"lanes_per_number": lanes, "threads": threads, "numbers_per_block": 32, "tensor": True}, L
    n512 = len(mr.mr_class_variants(512))
    assert any(mr.mr_lane_variant_info(512, v)["tensor"] for v in range(n512))
    assert not mr.mr_lane_variant_info(512, 0)["tensor"]
    for L in (3072, 4096):
        assert not any(mr.mr_lane_variant_info(L, v)["tensor"] for v in range(len(mr.mr_class_variants(L))))


@pytest.mark.parametrize("L", [512, 1024, 1536, 2048])
def test_byte_slice_products_are_exact_and_recombine(L):
    k, B, Bp, T1, T2 = _class(L)
    # every coefficient and matrix entry fits four bytes' worth of 30 bits, and the largest possible
    # slice sum (k products of two bytes) plus the 2^23 offset stays below 2^24
    assert max(B + Bp) < 1 << 30
    assert k * 255 * 255 < 1 << 23
    r = SplitMix64(0x7443 + L)
    for T, rows, cols in ((T1, B, Bp), (T2, Bp, B)):
        Tn = np.array(T, dtype=np.int64)
        Ts = [(Tn >> (8 * b)) & 255 for b in range(4)]
        for trial in range(3):
            xi = [r.below(m) for m in rows]
            if trial == 1:
                xi = [m - 1 for m in rows]  # the largest coefficients
            x = np.array(xi, dtype=np.int64)
            Xs = [(x >> (8 * a)) & 255 for a in range(4)]
            P = [[Xs[a] @ Ts[b] for b in range(4)] for a in range(4)]  # slice sums, per output channel
            assert max(int(P[a][b].max()) for a in range(4) for b in range(4)) + (1 << 23) < 1 << 24
            for j in range(k):
                exact = sum(xi[i] * T[i][j] for i in range(k))
                assert exact < 1 << 64
                assert _combine([[int(P[a][b][j]) for b in range(4)] for a in range(4)], k) == exact, (L, j)
