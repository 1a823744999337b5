"""Host-side pieces of the serving loop (no GPU): seeded Poisson arrivals and the per-request
device-footprint estimate used for admission."""
import math

import numpy as np
import pytest

pytest.importorskip("torch")


def _serve():
    try:
        from paper_1305_3699_gb300 import serve
    except OSError:  # the library is built by __graft_entry__.build(); skip when it is absent
        pytest.skip("library not built")
    return serve


def test_poisson_arrivals_seeded_sorted_mean_rate():
    serve = _serve()
    a = serve.poisson_arrivals(200_000.0, 20_000, 7)
    b = serve.poisson_arrivals(200_000.0, 20_000, 7)
    assert np.array_equal(a, b)
    assert (np.diff(a) > 0).all()
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert abs(gaps.mean() * 200_000.0 - 1.0) < 0.03          # mean gap 1/rate
    assert abs(np.median(gaps) * 200_000.0 - math.log(2)) < 0.05  # exponential: median = ln 2 / rate


def test_footprint_grows_with_size_and_decrypt_counts_two_halves():
    serve = _serve()
    f = {b: serve.request_footprint_bytes(b, 0, 128) for b in (1024, 2048, 3072, 4096)}
    assert f[1024] < f[2048] < f[3072] < f[4096]
    # a decryption holds the window tables of two half-size exponentiations
    assert serve.request_footprint_bytes(2048, 1, 128) > serve.request_footprint_bytes(1024, 0, 128)
