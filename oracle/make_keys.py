"""Write the stored synthetic RSA key sets under synth/keys (calls only the oracle).

Usage:  python -m oracle.make_keys [set ...]      (default: every set)

Each key j of a set is drawn from SplitMix64(seed).fork(j) by ``oracle.keygen``,
so any single key can be regenerated independently.  Seeds follow the workload
index: 0x4D520000 + i.

Sets:
  rsa1024_x64   64 RSA-1024 keys, e = 65537             (RSA-1024 encryption workload)
  rsa2048_x16   16 RSA-2048 keys, e = 65537             (RSA-2048 CRT decryption workload)
  mod16384_x4    4 moduli, each a product of two 8192-bit primes (long-exponent workload)
  mix_x256     256 keys: 102 x 1024, 77 x 2048, 51 x 3072, 26 x 4096 bits (ragged / serving)
  test_small    assorted small keys for tests (512 and 768 bits)
"""
from __future__ import annotations

import multiprocessing as mp
import sys
import time

from synth import SplitMix64, save_keys

from .keygen import gen_rsa_key

SEED_BASE = 0x4D520000


def _mix_sizes():
    return [1024] * 102 + [2048] * 77 + [3072] * 51 + [4096] * 26


SETS = {
    "rsa1024_x64": dict(seed=SEED_BASE + 1, sizes=[1024] * 64),
    "rsa2048_x16": dict(seed=SEED_BASE + 2, sizes=[2048] * 16),
    "mod16384_x4": dict(seed=SEED_BASE + 3, sizes=[16384] * 4),
    "mix_x256": dict(seed=SEED_BASE + 4, sizes=_mix_sizes()),
    "rsa8192_x2": dict(seed=SEED_BASE + 7, sizes=[8192] * 2),
    "test_small": dict(seed=SEED_BASE + 99, sizes=[512] * 4 + [768] * 4),
}


def _one(args):
    seed, j, bits = args
    rng = SplitMix64(seed).fork(j)
    return j, gen_rsa_key(rng, bits, e=65537, rounds=40)


def make(name: str, pool) -> None:
    spec = SETS[name]
    t0 = time.time()
    tasks = [(spec["seed"], j, b) for j, b in enumerate(spec["sizes"])]
    # largest first so the pool's tail is short
    order = sorted(tasks, key=lambda t: -t[2])
    res = dict(pool.imap_unordered(_one, order))
    keys = [res[j] for j in range(len(tasks))]
    meta = {"name": name, "seed": spec["seed"], "e": 65537, "mr_rounds": 40,
            "recipe": "SplitMix64(seed).fork(j); oracle.keygen.gen_rsa_key(rng, bits)"}
    path = save_keys(name, keys, meta)
    print(f"{name}: {len(keys)} keys in {time.time() - t0:.1f}s -> {path}", flush=True)


def main(argv):
    names = argv or list(SETS)
    ctx = mp.get_context("spawn")
    with ctx.Pool() as pool:
        for n in names:
            make(n, pool)


if __name__ == "__main__":
    main(sys.argv[1:])
