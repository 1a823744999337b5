"""Message-level RSA (mr_rsa_encrypt_message / mr_rsa_decrypt_message) against the oracle's
message_blocks: every ciphertext block equals the oracle's encryption of the same block, and
decryption gives the bytes back."""
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
def ctx(mr):
    c = mr.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("keyset", ["rsa1024_x64", "rsa2048_x16", "mix_x256"])
def test_message_round_trip(mr, ctx, keyset):
    k = load_keys(keyset)[3]
    h = ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
    r = SplitMix64(0x6D73 + len(keyset))
    B = plain.message_block_bytes(k["N"])
    for length in (1, B - 1, B, B + 1, 37 * B + 5):
        msg = bytes(r.below(256) for _ in range(length))
        nb, B2, W = ctx.mr_rsa_message_blocks(h, length)
        assert B2 == B and nb == -(-length // B) and W == (k["N"].bit_length() + 31) // 32
        m_dev = torch.tensor(list(msg), dtype=torch.uint8, device="cuda")
        c = torch.full((nb, W), -1, dtype=torch.int32, device="cuda")
        st = torch.full((nb,), 255, dtype=torch.uint8, device="cuda")
        ctx.mr_rsa_encrypt_message(h, m_dev, c, st)
        back = torch.zeros(length, dtype=torch.uint8, device="cuda")
        ctx.mr_rsa_decrypt_message(h, c, back, st)
        torch.cuda.synchronize()
        want = [plain.rsa_encrypt(v, k["e"], k["N"]) for v in plain.message_blocks(msg, k["N"])]
        assert mr.from_tensor(c) == want, length
        assert bytes(back.cpu().tolist()) == msg, length
        assert st.cpu().tolist() == [0] * nb


def test_message_argument_errors(mr, ctx):
    k = load_keys("rsa1024_x64")[0]
    h = ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
    nb, B, W = ctx.mr_rsa_message_blocks(h, 300)
    c = torch.zeros((nb + 1, W), dtype=torch.int32, device="cuda")
    out = torch.zeros(300, dtype=torch.uint8, device="cuda")
    with pytest.raises(mr.MRError) as e:
        ctx.mr_rsa_decrypt_message(h, c, out)  # one row too many for 300 bytes
    assert e.value.code == 1
    pub = ctx.mr_rsa_key_setup(k["N"], k["e"])
    with pytest.raises(mr.MRError) as e:
        ctx.mr_rsa_decrypt_message(pub, c[:nb], out)  # no private parts
    assert e.value.code == 10
