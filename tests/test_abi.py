"""The C-ABI library loads, exports every declared symbol, and its host-side
setup (base choice and every precomputed table) equals the oracle's RNS model
value by value.  No GPU needed: nothing here launches device work."""
import os
import re

import pytest

from oracle import rns
from synth import SplitMix64, load_keys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mr.h")

mr = pytest.importorskip("paper_1305_3699_gb300.mr", reason="libmrmod.so not built")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mr_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    syms = declared_symbols()
    assert len(syms) >= 14
    for s in syms:
        assert hasattr(mr.lib, s), s
    assert sorted(mr.EXPORTED) == syms


CLASSES = [512, 1024, 1536, 2048, 3072, 4096, 8192, 16384]


@pytest.mark.parametrize("L", CLASSES)
def test_class_tables_match_model(L):
    c = rns.make_class(L)
    Lc, k = mr.mr_class_for_bits(L)
    assert (Lc, k) == (L, c.k)
    assert mr.mr_debug_class_table(L, "B") == c.B
    assert mr.mr_debug_class_table(L, "Bp") == c.Bp
    b = mr.mr_debug_class_table(L, "bound")
    assert b[0] | (b[1] << 32) == c.bound
    m_limbs = mr.mr_debug_class_table(L, "M")
    assert int.from_bytes(b"".join(v.to_bytes(4, "little") for v in m_limbs), "little") == c.M
    for name in ("M_mi_inv", "Minv_Bp", "Mp_mj_inv", "Mp_B"):
        assert mr.mr_debug_class_table(L, name) == c.t[name], name
    for name in ("M_mi_Bp", "Mp_mj_B"):
        flat = [v for row in c.t[name] for v in row]
        assert mr.mr_debug_class_table(L, name) == flat, name


def test_class_for_bits_boundaries():
    assert mr.mr_class_for_bits(1)[0] == 512
    assert mr.mr_class_for_bits(512)[0] == 512
    assert mr.mr_class_for_bits(513)[0] == 1024
    assert mr.mr_class_for_bits(4096)[0] == 4096
    assert mr.mr_class_for_bits(4097) == (8192, 295)
    assert mr.mr_class_for_bits(16384) == (16384, 599)
    with pytest.raises(mr.MRError):
        mr.mr_class_for_bits(16385)


def test_large_class_slice_widths():
    """The large classes report, per compiled slice width, the threads that hold one number's
    channels: one lane in every warp of every channel slice (4 channels per warp)."""
    for L, k in ((8192, 295), (16384, 599)):
        lanes = mr.mr_class_variants(L)
        assert len(lanes) >= 1 and all(n > 0 for n in lanes)
        nw = 8  # variant 0: 8 warps, slices of 32 channels
        assert lanes[0] == -(-k // (4 * nw)) * nw


def test_trial_table_matches_oracle():
    """Trial-division tables built by the library's host code: the first 10,000 primes (the
    oracle's sieve), 2^(32w) mod p for every limb w < 128 (Python's pow), Barrett factors."""
    from oracle import primality
    t = mr.mr_debug_trial_table()
    ps = primality.first_primes(10000)
    assert t.shape == (131, 10016)
    assert [int(v) for v in t[128, :10000]] == list(ps)
    assert not t[:129, 10000:].any()
    r = SplitMix64(4321)
    for _ in range(300):
        j, w = r.below(10000), r.below(128)
        assert int(t[w, j]) == pow(2, 32 * w, ps[j]), (w, j)
    mu_words = t[129:131].reshape(-1)  # rows 129-130: the uint64 factors, low word first
    for j in (0, 1, 2, 4999, 9999):
        mu = int(mu_words[2 * j]) | (int(mu_words[2 * j + 1]) << 32)
        assert mu == ((1 << 64) - 1) // ps[j], j


def test_large_class_wave_policy():
    """The variant a large-class launch picks on 152 SMs with one block per SM, by waves x time per
    group: the 8192-bit class fits 15 groups per wave at 32 channels per block (integer form, 1.0),
    21 at 48 (integer form, 1.33) and 15 in the tensor-core form (0.495), which wins at every group
    count (two of its waves, 0.99, against one wide integer wave, 1.33, for 16-21 groups); the
    16384-bit class has one width (8 groups per wave) in two forms and picks the tensor-core form."""
    cases = {256: (2, 8), 480: (2, 15), 512: (2, 15), 672: (2, 15), 960: (2, 15), 1344: (2, 15)}
    for n, want in cases.items():
        assert mr.mr_debug_big_variant(8192, n) == want, n
    assert mr.mr_debug_big_variant(16384, 256) == (1, 8)
    assert mr.mr_debug_big_variant(16384, 1000) == (1, 8)
    with pytest.raises(mr.MRError) as e:
        mr.mr_debug_big_variant(1024, 100)
    assert e.value.code == 1  # not a large class


def test_crt_bin_block_matches_definition():
    """The binary Garner block of 16384-bit keys (8192-bit halves, W = 256) built by the library's
    host code: P2 is the least multiple of p not below 2^(32W), qr = qinv 2^(32(W+1)) mod p,
    q's limbs, pinv p = -1 mod 2^32; also for unbalanced halves."""
    keys = load_keys("mod16384_x4")[:2]
    cases = [(k["p"], k["q"], k["qinv"]) for k in keys]
    r = SplitMix64(0x43)
    p_small = keys[0]["p"] >> 200 | 1  # an odd number below the class size (the block does not need a prime)
    cases.append((p_small, keys[0]["q"], r.below(p_small)))
    W = 256
    for p, q, qinv in cases:
        blk = mr.mr_debug_crt_bin_host(p, q, qinv, W)
        assert len(blk) == 3 * W + 2
        val = lambda a, b: sum(v << (32 * i) for i, v in enumerate(blk[a:b]))
        P2 = val(0, W + 1)
        assert P2 % p == 0 and P2 >= 1 << (32 * W) and P2 - p < 1 << (32 * W)
        assert val(W + 1, 2 * W + 1) == (qinv * (1 << (32 * (W + 1)))) % p
        assert val(2 * W + 1, 3 * W + 1) == q
        assert (blk[3 * W + 1] * p) % (1 << 32) == (1 << 32) - 1


def _key_cases():
    r = SplitMix64(1234)
    out = []
    for bits in (3, 64, 511, 512, 700, 1024, 1536, 2048, 3000, 4096, 8000, 16384):
        N = r.randbits(bits) | 1 | (1 << (bits - 1))
        out.append(N)
    out += [k["p"] for k in load_keys("rsa2048_x16")[:2]] + [k["N"] for k in load_keys("rsa1024_x64")[:2]]
    return out


@pytest.mark.parametrize("N", _key_cases(), ids=lambda N: f"{N.bit_length()}b")
def test_key_tables_match_model(N):
    L, _ = mr.mr_class_for_bits(N.bit_length())
    c = rns.make_class(L)
    key = rns.make_key(c, N)
    assert mr.mr_debug_key_table_host(N, "kxi") == key.t["kxi"]
    assert mr.mr_debug_key_table_host(N, "NMinv_Bp") == key.t["NMinv_Bp"]
    for name in ("one", "r2", "r2h"):
        v = key.t[name]
        assert mr.mr_debug_key_table_host(N, name) == v.b + v.bp, name


def test_key_setup_errors():
    with pytest.raises(mr.MRError) as e:
        mr.mr_debug_key_table_host(1 << 100, "kxi")
    assert e.value.code == 2  # MR_ERR_EVEN_MODULUS
    with pytest.raises(mr.MRError) as e:
        mr.mr_debug_key_table_host((1 << 16384) + 1, "kxi")
    assert e.value.code == 4  # MR_ERR_SIZE
    c = rns.make_class(512)
    with pytest.raises(mr.MRError) as e:
        mr.mr_debug_key_table_host(c.B[3] * 1000003, "kxi")
    assert e.value.code == 3  # MR_ERR_NOT_COPRIME
    with pytest.raises(mr.MRError) as e:
        mr.mr_debug_key_table_host(12345679, "no_such_table")
    assert e.value.code == 1


def _tile_off(R, r, k):
    """Byte offset of element (r, k) of an R-row tensor-core tile: 8-row x 16-byte core matrices,
    column groups of 8 outermost (the K-major layout without swizzling)."""
    return (k // 8) * (R // 8) * 128 + (r // 8) * 128 + (r % 8) * 16 + (k % 8) * 2


@pytest.mark.parametrize("L", [8192, 16384])
def test_tc_slice_table_recombines_to_scaled_matrices(L):
    """The tensor-core operand table: at a seeded sample of (slice, matrix, input channel, column),
    the four fp16 slices at their tile positions are integers in [0, 127] and recombine,
    sum_b 2^(7b) s_b, to the extension matrix entry times 2^64 mod its prime (the device's scaled
    form); past channel k every slice is zero."""
    from synth import SplitMix64
    k = mr.mr_class_for_bits(L)[1]
    B = mr.mr_debug_class_table(L, "B")
    Bp = mr.mr_debug_class_table(L, "Bp")
    T1 = mr.mr_debug_class_table(L, "M_mi_Bp")  # row i, column j
    T2 = mr.mr_debug_class_table(L, "Mp_mj_B")  # row j, column i
    t = mr.mr_debug_tc_slices(L)
    slices, nch = (k + 31) // 32, (k + 63) // 64
    assert t.size == slices * 2 * nch * 128 * 64
    r = SplitMix64(L)

    def at(c, e, i, j, b):
        byte = ((c * 2 + e) * nch + i // 64) * 16384 + _tile_off(128, 32 * b + j, i % 64)
        return float(t[byte // 2])

    for _ in range(400):
        c, e, i, j = r.below(slices), r.below(2), r.below(nch * 64), r.below(32)
        vals = [at(c, e, i, j, b) for b in range(4)]
        assert all(v == int(v) and 0 <= v <= 127 for v in vals)
        col = 32 * c + j
        if i >= k or col >= k:
            assert vals == [0.0] * 4
            continue
        got = sum(int(v) << (7 * b) for b, v in enumerate(vals))
        if e == 0:
            want = T1[i * k + col] * (1 << 64) % Bp[col]
        else:
            want = T2[i * k + col] * (1 << 64) % B[col]
        assert got == want, (c, e, i, j)


def test_big_variant_info():
    """The 16384-bit class compiles the integer form (variant 0) and the tensor-core form (variant 1)
    of its base extensions, both with 32-channel slices (19 blocks per group); the 8192-bit class's
    integer variants have 32- and 48-channel slices."""
    assert mr.mr_big_variant_info(16384, 0) == {"slice_channels": 32, "slices": 19, "tensor": False}
    assert mr.mr_big_variant_info(16384, 1) == {"slice_channels": 32, "slices": 19, "tensor": True}
    assert mr.mr_big_variant_info(8192, 0)["slice_channels"] == 32
    assert mr.mr_big_variant_info(8192, 1)["slice_channels"] == 48
    assert mr.mr_big_variant_info(8192, 2) == {"slice_channels": 32, "slices": 10, "tensor": True}
    with pytest.raises(mr.MRError):
        mr.mr_big_variant_info(1024, 0)


def test_lane_group_factor_estimate_bound():
    """The lane-group kernels estimate a' = floor(sum xi'_j / m'_j) from (xi'_j >> 17) floor(2^39 / m'_j)
    (Q = 22 fixed-point bits, offset 1/4).  Each term is below its exact value by less than
    2^39 / m'_j + (m'_j - 1) / 2^17 units of 2^-22; the estimate is exact when the k terms together
    stay below 1/4 (2^20 units), and the sum must fit 32 bits.  Checked on every lane-group class's
    actual primes B'."""
    Q, S = 22, 17
    for L in (512, 1024, 1536, 2048, 3072, 4096):
        k = mr.mr_class_for_bits(L)[1]
        bp = mr.mr_debug_class_table(L, "Bp")
        assert len(bp) == k
        err = sum(2 ** (Q + S) / m + (m - 1) / 2 ** S for m in bp)
        assert err < 2 ** (Q - 2), (L, err / 2 ** Q)
        assert k * 2 ** Q < 2 ** 32, L
