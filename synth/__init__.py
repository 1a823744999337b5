"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module draws random numbers and converts integers to and from the
little-endian uint32 limb layout used at the C boundary.  It holds none of
the method's arithmetic: no modular reduction, no residue number system, no
exponentiation.  Key material is drawn by the oracle (``oracle.keygen``) and
stored under ``synth/keys``; this module only reads those files.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014): a 64-bit Weyl sequence with increment
0x9E3779B97F4A7C15 followed by the published three-step finaliser.  The paper's
own random-bit layer is a hardware entropy source; it cannot be replayed, so
every input here is drawn from this deterministic generator instead.
"""
from __future__ import annotations

import gzip
import json
import math
import os
from typing import Iterable, List, Sequence

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Deterministic 64-bit generator; ``fork(label)`` gives an independent substream."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next64(self) -> int:
        self.state = (self.state + GAMMA) & MASK64
        return _mix64(self.state)

    def fork(self, label: int) -> "SplitMix64":
        # A substream seeded from (current seed, label) without consuming this stream.
        return SplitMix64(_mix64((self.state ^ _mix64((label * GAMMA + 1) & MASK64)) & MASK64))

    def randbits(self, n: int) -> int:
        """n uniform bits; 64-bit words are concatenated least significant first."""
        if n <= 0:
            return 0
        words = (n + 63) // 64
        v = 0
        for w in range(words):
            v |= self.next64() << (64 * w)
        return v & ((1 << n) - 1)

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection on bit_length(n-1)-bit draws."""
        if n <= 0:
            raise ValueError("below(n) needs n > 0")
        if n == 1:
            return 0
        b = (n - 1).bit_length()
        while True:
            v = self.randbits(b)
            if v < n:
                return v

    def between(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + self.below(hi - lo + 1)

    def uniform01(self) -> float:
        """Float in [0, 1) from the top 53 bits of one draw."""
        return (self.next64() >> 11) * (1.0 / (1 << 53))

    def exponential(self, rate: float) -> float:
        """Exponential gap with the given rate (inverse-CDF of one uniform draw)."""
        return -math.log1p(-self.uniform01()) / rate


# ----------------------------------------------------------------------------
# limb layout at the C boundary: little-endian uint32, fixed count per value
# ----------------------------------------------------------------------------

def limbs_for_bits(bits: int) -> int:
    return max(1, (bits + 31) // 32)


def to_limbs(x: int, n_limbs: int) -> np.ndarray:
    if x < 0 or x.bit_length() > 32 * n_limbs:
        raise ValueError(f"value of {x.bit_length()} bits does not fit {n_limbs} limbs")
    b = x.to_bytes(4 * n_limbs, "little")
    return np.frombuffer(b, dtype="<u4").astype(np.uint32)


def from_limbs(a: Sequence[int] | np.ndarray) -> int:
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return int.from_bytes(arr.astype("<u4").tobytes(), "little")


def pack(values: Iterable[int], n_limbs: int) -> np.ndarray:
    vals = list(values)
    out = np.zeros((len(vals), n_limbs), dtype=np.uint32)
    for i, v in enumerate(vals):
        out[i] = to_limbs(v, n_limbs)
    return out


def unpack(arr: np.ndarray) -> List[int]:
    arr = np.asarray(arr, dtype=np.uint32)
    if arr.ndim == 1:
        return [from_limbs(arr)]
    return [from_limbs(row) for row in arr]


# ----------------------------------------------------------------------------
# stored keys (written by oracle/make_keys.py; read here as plain data)
# ----------------------------------------------------------------------------

KEY_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "keys")

_RSA_FIELDS = ("N", "e", "p", "q", "d", "dp", "dq", "qinv")


def load_keys(name: str) -> List[dict]:
    """Load a stored key set: a list of dicts with int fields N, e, p, q, d, dp, dq, qinv, bits."""
    path = os.path.join(KEY_DIR, name + ".json.gz")
    with gzip.open(path, "rt") as f:
        doc = json.load(f)
    out = []
    for k in doc["keys"]:
        rec = {"bits": int(k["bits"])}
        for fld in _RSA_FIELDS:
            if fld in k:
                rec[fld] = int(k[fld], 16)
        out.append(rec)
    return out


def key_set_info(name: str) -> dict:
    path = os.path.join(KEY_DIR, name + ".json.gz")
    with gzip.open(path, "rt") as f:
        doc = json.load(f)
    return {k: v for k, v in doc.items() if k != "keys"}


def save_keys(name: str, keys: List[dict], meta: dict) -> str:
    os.makedirs(KEY_DIR, exist_ok=True)
    path = os.path.join(KEY_DIR, name + ".json.gz")
    doc = dict(meta)
    doc["keys"] = [{**{f: format(k[f], "x") for f in _RSA_FIELDS if f in k}, "bits": k["bits"]} for k in keys]
    with gzip.GzipFile(path, "wb", mtime=0) as f:
        f.write(json.dumps(doc, indent=0, sort_keys=True).encode())
    return path
