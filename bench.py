"""Benchmark of the RNS exponentiation library on synthetic, seeded workloads.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]

Workloads (--workload):
  rsa2048_crt   (default) one step = one mr_rsa_decrypt_crt call over 4096 ciphertexts (uniform
                in [0, N)) over 16 seeded RSA-2048 keys: 8192 RNS exponentiations of 1024-bit
                numbers with full-length CRT exponents plus 4096 Garner recombinations
  ragged        65,536 encrypt/decrypt requests over 256 keys of 1024-4096 bits (40/30/20/10%),
                per-size plain launches against the persistent, graph-captured plan
  serving       Poisson arrivals at 200k requests/s of the same mix: throughput, p50/p99 latency
  modexp16384   256 exponentiations modulo 16384-bit RSA moduli with 16128-bit exponents
  rsa1024_enc   64 RSA-1024 public encryptions (e = 65537), one graph replay per step
  mr1024        Miller-Rabin: 4096 odd 1024-bit candidates x 8 seeded witnesses
The metric is modular exponentiations per second over all ranks; with N > 1 (launched under
torchrun) every rank runs its own batch (weak scaling, no collective on the data path).
`--impl reference` times the CPU oracle (plain Python integers, its own square-and-multiply) on
the same workload instead.

Everything is printed on stderr except the single JSON result line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "modexp/s: RSA-2048 CRT decrypt and ragged mixed-size batch vs per-size launches"
UNIT = "modexp/s"
N_CT = 4096
KEYSET = "rsa2048_x16"
SEED = 0x4D520002
# Peak of the 32x32->64-bit multiply-add pipe: SMs x 64 per clock x max SM clock
IMAD_PER_CLK_PER_SM = 64   # int32 multiplies per clock per SM (integer multiply pipe)
# DRAM bytes (read + write) of one exponentiation launch of the RSA-2048 CRT workload, from an ncu
# capture on this workload, per kernel form of the 1024-bit class: the integer form
# (dram__bytes_read.sum + dram__bytes_write.sum); None for the tensor-core form, whose code changed
# after its last capture (25.3 MB per launch then, profiles/modexp_tc_k36_rsa2048_crt_4096.md)
TRAFFIC_BYTES_PER_LAUNCH = {"integer": 2_861_568 + 24_110_080, "tensor": None}
# long-exponent workload: 256 exponentiations modulo 16384-bit RSA moduli with 16128-bit exponents
BIG_KEYSET = "mod16384_x4"
BIG_N = 256
BIG_EBITS = 16128
BIG_SEED = 0x4D520003


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ----------------------------------------------------------------- workload
def workload(rank: int = 0):
    from synth import SplitMix64, load_keys
    keys = load_keys(KEYSET)
    r = SplitMix64(SEED + 0x1000 * rank)
    per = N_CT // len(keys)
    idx = [i // per for i in range(N_CT)]
    cts = [r.below(keys[i]["N"]) for i in idx]
    return keys, idx, cts


def algorithmic_products_per_modexp(k: int, W: int, WX: int, ebits: int, w: int, chunks: int) -> int:
    """32x32->64 products the method performs for one exponentiation (reductions not counted).

    Per RNS Montgomery multiplication: 2k^2 (the two base extensions) + 7k
    (x*y in both bases, xi, the two products of r_j, xi'_j, a'*|M'|).  One
    exponentiation with fixed w-bit windows: `chunks` entry products, 2^w - 2
    table products, w squarings + 1 multiplication per window after the first,
    one exit product; plus binary->RNS (chunks * W * 2k) and RNS->binary (k * WX).
    """
    per_mm = 2 * k * k + 7 * k
    nwin = max(1, math.ceil(ebits / w))
    mms = chunks + (2 ** w - 2) + (w + 1) * (nwin - 1) + 1
    return mms * per_mm + chunks * W * 2 * k + k * WX


def mms_sliding(e: int, w: int, chunks: int) -> int:
    """RNS Montgomery multiplications of one exponentiation on the sliding-window schedule the
    lane-group kernel runs when every number of a warp has the same exponent e (windows of up to
    w + 1 bits that start and end on a set bit; table of the 2^w odd powers, built with x^2):
    `chunks` entry products, 2^w table products, the squarings and window products, one exit."""
    ws = w + 1
    mms = chunks + (1 << w) + 1
    top = e.bit_length() - 1
    lo = max(top - ws + 1, 0)
    while not (e >> lo) & 1:
        lo += 1
    pos = lo
    while pos > 0:
        i, z = pos - 1, 0
        while i - z >= 0 and not (e >> (i - z)) & 1:
            z += 1
        if i - z < 0:
            mms += z
            pos = 0
        else:
            t = i - z
            lo = max(t - ws + 1, 0)
            while not (e >> lo) & 1:
                lo += 1
            mms += z + (t - lo + 1) + 1
            pos = lo
    return mms


def algorithmic_products_sliding(k: int, W: int, WX: int, e: int, w: int, chunks: int) -> int:
    """As algorithmic_products_per_modexp, on the sliding-window schedule (mms_sliding)."""
    return mms_sliding(e, w, chunks) * (2 * k * k + 7 * k) + chunks * W * 2 * k + k * WX


# Channels per base of the 31-bit-channel reading of the method: channel primes are the largest
# primes below 2^31 and k is the smallest count with M >= (k+1)^2 2^L and M' >= (k+1) 2^L (the
# closure bound of the uncorrected extension B -> B'); tests/test_bench_accounting.py recomputes them.
K31 = {512: 17, 1024: 34, 1536: 50, 2048: 67, 3072: 100, 4096: 133, 8192: 265, 16384: 530}


def ops_31bit_count(L: int, ebits: int, w: int) -> int:
    """int32-multiply operations of one L-bit exponentiation under the 31-bit-channel accounting.

    k = K31[L]; per RNS Montgomery multiplication 2 [2k(k+1) + 8k] (the two base extensions onto
    k+1 channels, a redundant one included, and 8k channel products; a 32x32->64 product counts
    as two operations); |e| + ceil(|e|/w) + 2^w + 2 multiplications per exponentiation; plus the
    conversions, 2 W (2k+1) + 2 k (W+1) products.  Channel reductions are not counted.
    """
    k, W = K31[L], L // 32
    mms = ebits + math.ceil(ebits / w) + 2 ** w + 2
    return mms * 2 * (2 * k * (k + 1) + 8 * k) + 2 * (2 * W * (2 * k + 1) + 2 * k * (W + 1))


def tensor_ops_31bit_count(L: int, n: int, ebits: int, w: int) -> int:
    """Tensor operations of the base extensions of n L-bit exponentiations under the same
    accounting with byte slices: per multiplication 2 extensions x 16 slice pairs x 2 n k (k+1)."""
    k = K31[L]
    mms = ebits + math.ceil(ebits / w) + 2 ** w + 2
    return mms * 2 * 16 * 2 * n * k * (k + 1)


# ------------------------------------------------------------- clock sampler
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.rows = []
        self.proc = None
        self.mark = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50",
                 "-i", gpu_index], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), line.strip()))

    def window(self, t0, t1):
        out = []
        for t, line in self.rows:
            if t0 <= t <= t1:
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    out.append(f)
        return out

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = self.window(t0, t1)
        note = None
        if not rows:  # a timed region shorter than the sampling interval: the samples next to it
            rows = self.window(t0 - 0.2, t1 + 0.2)
            note = "no sample inside the timed region; samples within 0.2 s of it"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples in the timed region"], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        out = {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": len(rows),
               "power_w_max": max((num(r[3]) or 0) for r in rows)}
        if note:
            out["note"] = note
        return out


# --------------------------------------------------------- CPU oracle timing
def _oracle_decrypt_chunk(args):
    from oracle import plain
    t0 = time.perf_counter()
    out = [plain.rsa_decrypt_crt(c, p, q, dp, dq, qi) for (c, p, q, dp, dq, qi) in args]
    return time.perf_counter() - t0, len(out)


def oracle_throughput(keys, idx, cts, seconds: float, steps: int = 1, warmup: int = 0):
    """Time the oracle's CRT decryption on every host core over a bounded sample.

    Returns (modexp/s of the timed steps, cores, sample description, per-step seconds)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    tasks = [(cts[j], keys[idx[j]]["p"], keys[idx[j]]["q"], keys[idx[j]]["dp"], keys[idx[j]]["dq"],
              keys[idx[j]]["qinv"]) for j in range(len(cts))]
    ctxm = mp.get_context("spawn")
    with ctxm.Pool(cores) as pool:
        # calibrate: one decryption per core
        t0 = time.perf_counter()
        pool.map(_oracle_decrypt_chunk, [[tasks[j]] for j in range(cores)])
        per = max(1e-4, (time.perf_counter() - t0))
        n = max(cores, min(len(tasks), int(seconds / per) * cores))
        n = (n // cores) * cores
        sample = tasks[:n]
        chunks = [sample[i::cores] for i in range(cores)]
        times = []
        for s in range(warmup + steps):
            t0 = time.perf_counter()
            pool.map(_oracle_decrypt_chunk, chunks)
            dt = time.perf_counter() - t0
            if s >= warmup:
                times.append(dt)
    value = 2 * n / statistics.mean(times)
    desc = (f"first {n} of the {len(cts)} ciphertexts of the workload ({2 * n} modexps), "
            f"oracle.plain.rsa_decrypt_crt on {cores} processes")
    return value, cores, desc, times


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: every rank's work counts, the whole job ends with the last one."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sm_max_mhz() -> float:
    """Maximum SM clock: MEASURED_PEAKS.json's figure when present, else the GB300 maximum."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("sm_max_mhz", 2070.0))
    except (OSError, ValueError):
        return 2070.0


def measured_peak(key: str, default: float) -> float:
    """A figure of MEASURED_PEAKS.json (measured on this machine's GPUs), else `default`."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get(key, default))
    except (OSError, ValueError):
        return default


def big_variant_used(mr, L: int, n_items: int) -> int:
    """The variant a large-class call of n_items runs: MR_VARIANT_<L> when set, else the library's
    wave policy on this GPU (one block per SM)."""
    env = os.environ.get(f"MR_VARIANT_{L}")
    if env is not None and env.isdigit():
        return int(env)
    return mr.mr_debug_big_variant(L, n_items)[0]


def window_for_bits(bits: int, max_w: int = 5) -> int:
    """The library's window width for an exponent of `bits` bits: minimises squarings +
    multiplications + table entries over w = 1..max_w (5 for the lane-group classes, 8 for the
    large ones, lower when MR_MAX_WINDOW is set)."""
    cap = os.environ.get("MR_MAX_WINDOW")
    if cap and cap.isdigit() and 1 <= int(cap) < max_w:
        max_w = int(cap)
    if bits <= 1:
        return 1
    best, bw = None, 1
    for w in range(1, max_w + 1):
        nwin = (bits + w - 1) // w
        cost = (nwin - 1) * w + nwin + (1 << w) - 2
        if best is None or cost < best:
            best, bw = cost, w
    return bw


def big_workload(rank: int = 0, ebits: int = BIG_EBITS):
    from synth import SplitMix64, load_keys
    keys = load_keys(BIG_KEYSET)
    r = SplitMix64(BIG_SEED + 0x1000 * rank)
    idx = [i % len(keys) for i in range(BIG_N)]
    xs = [r.below(keys[i]["N"]) for i in idx]
    es = [r.randbits(ebits - 1) | (1 << (ebits - 1)) for _ in range(BIG_N)]
    return keys, idx, xs, es


def big_crt_workload(rank: int = 0):
    """256 ciphertexts uniform below four seeded 16384-bit RSA moduli (64 per key)."""
    from synth import SplitMix64, load_keys
    keys = load_keys(BIG_KEYSET)
    r = SplitMix64(BIG_SEED + 0x77 + 0x1000 * rank)
    idx = [i % len(keys) for i in range(BIG_N)]
    cts = [r.below(keys[i]["N"]) for i in idx]
    return keys, idx, cts


def _oracle_modexp_chunk(args):
    from oracle import plain
    t0 = time.perf_counter()
    out = [plain.modexp(x, e, N) for (x, e, N) in args]
    return time.perf_counter() - t0, len(out)


def oracle_big_throughput(keys, idx, xs, es, steps: int = 1, warmup: int = 0,
                          what: str = "16384-bit moduli, 16128-bit exponents"):
    """The oracle's exponentiation on every host core, one item per core per step."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    n = min(len(xs), cores)
    tasks = [[(xs[j], es[j], keys[idx[j]]["N"])] for j in range(n)]
    times = []
    with mp.get_context("spawn").Pool(cores) as pool:
        for s in range(warmup + steps):
            t0 = time.perf_counter()
            pool.map(_oracle_modexp_chunk, tasks)
            if s >= warmup:
                times.append(time.perf_counter() - t0)
    value = n / statistics.mean(times)
    desc = (f"first {n} of the {len(xs)} items of the workload ({what}), "
            f"oracle.plain.modexp, one item per process on {cores} processes")
    return value, cores, desc, times


def _oracle_mixed_chunk(args):
    from oracle import plain
    t0 = time.perf_counter()
    for op, x, k in args:
        if op == 0:
            plain.rsa_encrypt(x, k["e"], k["N"])
        else:
            plain.rsa_decrypt_crt(x, k["p"], k["q"], k["dp"], k["dq"], k["qinv"])
    return time.perf_counter() - t0, len(args)


def oracle_mixed_throughput(keys, idx, ops, xs, seconds: float = 10.0):
    """The oracle on a bounded prefix of a mixed request list, on every host core: modexp/s
    (an encryption counts one exponentiation, a CRT decryption two)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(cores) as pool:
        probe = [[(ops[j], xs[j], keys[idx[j]])] for j in range(cores)]
        t0 = time.perf_counter()
        pool.map(_oracle_mixed_chunk, probe)
        per = max(1e-4, time.perf_counter() - t0)
        n = max(cores, min(len(xs), int(seconds / per) * cores))
        tasks = [(ops[j], xs[j], keys[idx[j]]) for j in range(n)]
        t0 = time.perf_counter()
        pool.map(_oracle_mixed_chunk, [tasks[i::cores] for i in range(cores)])
        dt = time.perf_counter() - t0
    modexps = sum(1 if ops[j] == 0 else 2 for j in range(n))
    desc = f"first {n} requests of the mix ({modexps} modexps), oracle.plain on {cores} processes"
    return modexps / dt, cores, desc


def _oracle_mr_chunk(args):
    from oracle import primality
    t0 = time.perf_counter()
    for n, ws in args:
        primality.miller_rabin(n, ws)
    return time.perf_counter() - t0, len(args)


# --------------------------------------------------------------- reference
def _reference_line(args, workload, value, unit, cores, desc, times, config=None):
    line = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int (Python)", "data": "synthetic",
            "impl": "reference", "config": dict({"workload": workload, "sample_per_step": desc}, **(config or {})),
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _pool_steps(fn, chunks, steps, warmup):
    """Run fn over chunks on every host core, `warmup + steps` times; per-step seconds of the timed ones."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    times = []
    with mp.get_context("spawn").Pool(cores) as pool:
        for s_ in range(warmup + max(1, steps)):
            t0 = time.perf_counter()
            pool.map(fn, [chunks[i::cores] for i in range(cores) if chunks[i::cores]])
            if s_ >= warmup:
                times.append(time.perf_counter() - t0)
    return cores, times


def run_reference_extra(args):
    """The oracle on the other workloads' inputs (same seeds as the GPU arm), bounded samples."""
    from synth import SplitMix64, load_keys
    if args.workload in ("ragged", "serving"):
        keys, idx, ops, xs = ragged_workload(0)
        times, value, cores, desc = [], 0.0, 1, ""
        for _ in range(max(1, args.steps)):
            t0 = time.perf_counter()
            value, cores, desc = oracle_mixed_throughput(keys, idx, ops, xs, seconds=min(10.0, args.cpu_seconds))
            times.append(time.perf_counter() - t0)
        return _reference_line(args, "ragged_mix_65536" if args.workload == "ragged" else "serving_poisson_200k",
                               value, UNIT, cores, desc, times)
    if args.workload == "class_modexp":
        mods, idx, xs, es = class_workload(args.bits, args.items)
        value, cores, desc, times = oracle_big_throughput([{"N": N} for N in mods], idx, xs, es,
                                                          steps=max(1, args.steps), warmup=0,
                                                          what=f"{args.bits}-bit moduli and exponents")
        return _reference_line(args, f"modexp{args.bits}_class", value, UNIT, cores, desc, times)
    if args.workload == "rsa1024_enc":
        from oracle import plain
        keys = load_keys("rsa1024_x64")
        r = SplitMix64(0x4D520001)
        msgs = [r.below(k["N"]) for k in keys]
        times = []
        for _ in range(args.warmup + max(1, args.steps)):
            t0 = time.perf_counter()
            for m, k in zip(msgs, keys):
                plain.rsa_encrypt(m, k["e"], k["N"])
            times.append(time.perf_counter() - t0)
        times = times[args.warmup:]
        return _reference_line(args, "rsa1024_encrypt_64", len(msgs) / statistics.mean(times), UNIT, 1,
                               "the 64 messages, oracle.plain.rsa_encrypt, one process", times)
    if args.workload == "mr1024":
        rounds, n = 8, 4096
        keys = load_keys(KEYSET)
        primes = [k[h] for k in keys for h in ("p", "q")]
        r = SplitMix64(0x4D520006)
        cands = [primes[i % len(primes)] if i % 2 == 0 else (r.randbits(1024) | 1 | (1 << 1023)) for i in range(n)]
        wit = [[2 + r.below(c - 3) for _ in range(rounds)] for c in cands]
        sample = [(cands[j], wit[j]) for j in range(min(n, 256))]
        cores, times = _pool_steps(_oracle_mr_chunk, sample, args.steps, args.warmup)
        return _reference_line(args, "miller_rabin_1024x4096x8", len(sample) * rounds / statistics.mean(times),
                               "MR rounds/s", cores, f"first {len(sample)} candidates x {rounds} rounds", times)
    if args.workload == "primegen1024":
        rounds, n = 8, 16384
        r = SplitMix64(0x4D520007)
        cands = [r.randbits(1024) | 1 | (1 << 1023) for _ in range(n)]
        wit = [[2 + r.below(c - 3) for _ in range(rounds)] for c in cands]
        sample = [(cands[j], wit[j]) for j in range(1024)]
        cores, times = _pool_steps(_oracle_prime_chunk, sample, args.steps, args.warmup)
        return _reference_line(args, "primegen_1024x16384x8", len(sample) / statistics.mean(times), "candidates/s",
                               cores, f"first {len(sample)} candidates, prime_test_verdict", times)
    if args.workload == "keygen2048":
        n_keys, pool, rounds = 16, 2048, 4
        r = SplitMix64(0x4D520008)
        pools = [[r.randbits(1024) | (3 << 1022) | 1 for _ in range(pool)] for _ in range(2 * n_keys)]
        wits = [[[r.between(2, c - 2) for _ in range(rounds)] for c in pl] for pl in pools]
        sample = [(pools[2 * k], wits[2 * k], pools[2 * k + 1], wits[2 * k + 1]) for k in range(n_keys)]
        cores, times = _pool_steps(_oracle_keygen_chunk, sample, args.steps, args.warmup)
        return _reference_line(args, "keygen_rsa2048_16x2x2048", n_keys / statistics.mean(times), "RSA-2048 keys/s",
                               cores, f"all {n_keys} keys, rsa_key_from_pools", times)
    return None


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    extra = run_reference_extra(args)
    if extra is not None:
        return extra
    if args.workload == "modexp16384":
        keys, idx, xs, es = big_workload(0)
        value, cores, desc, times = oracle_big_throughput(keys, idx, xs, es, steps=args.steps, warmup=args.warmup)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int (Python)", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": "modexp16384_long_exponent", "items": BIG_N, "sample_per_step": desc},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "rsa16384_crt":
        keys, idx, cts = big_crt_workload(0)
        budget = max(4.0, 90.0 / max(1, args.steps + args.warmup))
        value, cores, desc, times = oracle_throughput(keys, idx, cts, budget, steps=args.steps, warmup=args.warmup)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int (Python)", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": "rsa16384_crt_decrypt", "ciphertexts": BIG_N, "sample_per_step": desc},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    keys, idx, cts = workload(0)
    budget = max(4.0, 90.0 / max(1, args.steps + args.warmup))
    value, cores, desc, times = oracle_throughput(keys, idx, cts, budget, steps=args.steps, warmup=args.warmup)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int (Python arbitrary precision)",
        "data": "synthetic (seeded keys and ciphertexts)", "impl": "reference",
        "config": {"workload": "rsa2048_crt_decrypt", "ciphertexts": N_CT, "keys": 16,
                   "modexps_per_step": 2 * N_CT, "sample_per_step": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- ours
def run_ours(args, rank, world, local_rank, emit=True):
    import torch
    import torch.distributed as dist

    from paper_1305_3699_gb300 import mr

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    keys, idx, cts = workload(rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("timing the CPU oracle on a bounded sample ...")
        v, cores, desc, _ = oracle_throughput(keys, idx, cts, args.cpu_seconds)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    ctx = mr.Context(local_rank)
    if args.constant_time:
        ctx.mr_set_constant_time(True)
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
    kl = mr.KeyList([hk[i] for i in idx])
    c_dev = mr.to_tensor(cts, 64, device=dev)
    m_dev = torch.zeros_like(c_dev)
    status = torch.zeros(N_CT, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def step():
        ctx.mr_rsa_decrypt_crt(kl, c_dev, m_dev, status, stream=stream)

    R = max(1, args.repeats)  # calls per step, each after an L2 flush and inside its own events
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    # check on every run: a seeded sample of decryptions against the plain definition, and every
    # plaintext re-encrypted with e = 65537 gives back its ciphertext
    got_all = mr.from_tensor(m_dev)
    got = got_all[0]
    for j in range(0, N_CT, N_CT // 32):
        kj = keys[idx[j]]
        assert got_all[j] == pow(cts[j], kj["d"], kj["N"]), "benchmark output mismatch"
    assert all(pow(m, keys[i]["e"], keys[i]["N"]) == c for m, i, c in zip(got_all, idx, cts)), \
        "benchmark output mismatch (re-encryption)"
    assert int(status.sum()) == 0

    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    gpu_index = vis[local_rank] if local_rank < len(vis) else (vis[0] if vis else str(local_rank))
    sampler = ClockSampler(gpu_index) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    ctx.mr_profile_enable(True)
    ctx.mr_profile_read()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps * R)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    with torch.cuda.stream(stream):
        for s in range(args.steps * R):
            flush.zero_()  # evict L2 between timed calls (outside the call's events)
            evs[s][0].record(stream)
            step()
            evs[s][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall1 = time.time()
    prof = ctx.mr_profile_read()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = 2 * N_CT * R * world * args.steps / (total_ms / 1e3)

    # end to end through the C ABI with host buffers: H2D of the ciphertexts, the call, D2H of the plaintexts
    c_host = c_dev.cpu().pin_memory()
    m_host = torch.empty_like(c_host).pin_memory()
    e2e_ms = []
    with torch.cuda.stream(stream):
        for s in range(max(3, args.steps // 4)):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            c_dev.copy_(c_host, non_blocking=True)
            step()
            m_host.copy_(m_dev, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
    assert mr.from_tensor(m_host[:1])[0] == got
    e2e_val = 2 * N_CT * world / (statistics.mean(e2e_ms) / 1e3)
    clocks = sampler.summary(t_wall0, t_wall1) if sampler else None
    if sampler:
        sampler.stop()

    # roofline of the dominant kernel (exponentiation).  Work is counted in int32-multiply ops: one
    # 32x32->64 product of the method is two of them (low and high word), the unit of the integer
    # multiply pipe's table rate (64 per clock per SM); the peak is that rate at the maximum SM clock.
    # The same figure against a measured dependent-free mad.wide.u32 stream is reported beside it.
    (mx_launch, mx_ms), (crt_launch, crt_ms) = prof
    props = torch.cuda.get_device_properties(dev)
    L_half, k = mr.mr_class_for_bits(1024)
    W = 32
    WX = len(mr.mr_debug_class_table(L_half, "M"))
    w = window_for_bits(max(max(keys[i]["dp"].bit_length(), keys[i]["dq"].bit_length()) for i in idx))
    # every warp holds halves of one key (256 ciphertexts per key, items ordered by exponent), so
    # the kernel runs the sliding-window schedule (w >= 4) for all of them
    prods = 0
    ops31 = 0
    n_mm = 0  # RNS Montgomery multiplications of the launch (all 8192 exponentiations)
    for i in idx:
        for dpq in (keys[i]["dp"], keys[i]["dq"]):
            if w >= 4:
                prods += algorithmic_products_sliding(k, W, WX, dpq, w, 2)
                n_mm += mms_sliding(dpq, w, 2)
            else:
                prods += algorithmic_products_per_modexp(k, W, WX, dpq.bit_length(), w, 2)
                n_mm += 2 + (2 ** w - 2) + (w + 1) * (math.ceil(dpq.bit_length() / w) - 1) + 1
            ops31 += ops_31bit_count(1024, dpq.bit_length(), w)
    ops_per_launch = 2 * prods  # one exponentiation launch per call covers all 8192 halves
    max_mhz = sm_max_mhz()
    peak = props.multi_processor_count * IMAD_PER_CLK_PER_SM * max_mhz * 1e6
    mx_avg_ms = mx_ms / max(1, mx_launch)
    achieved = ops_per_launch / (mx_avg_ms / 1e3)
    wide_rate = ctx.mr_imad_peak(0, stream)
    lo_rate = ctx.mr_imad_peak(1, stream)
    pair_rate = ctx.mr_imad_peak(2, stream)
    hi_rate = ctx.mr_imad_peak(3, stream)
    tensor = {"tcgen05_kind_f16_ops_per_s": ctx.mr_tensor_peak(0, stream),
              "mma_sync_s8_ops_per_s": ctx.mr_tensor_peak(1, stream),
              "mma_sync_f16_ops_per_s": ctx.mr_tensor_peak(2, stream),
              "tcgen05_kind_i8": "not available on sm_103a (ptxas: feature not supported on this target)"}
    achieved31 = ops31 / (mx_avg_ms / 1e3)
    # the kernel form the 1024-bit class runs by default: the base extensions on the tensor cores
    # (8-bit slices, exact fp32 sums) or as mad.wide dot products on the integer pipe
    vinfo = mr.mr_lane_variant_info(L_half, 0)
    form = "tensor" if vinfo["tensor"] else "integer"
    kname = (f"modexp_kernel<k={k},TPI={vinfo['lanes_per_number']}"
             + (", base extensions on tcgen05 (8-bit slices)>" if vinfo["tensor"] else ">"))
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T int32-mul/s",
                "frac": achieved / peak, "traffic": TRAFFIC_BYTES_PER_LAUNCH[form],
                "kernel": kname, "kernel_ms": mx_avg_ms,
                "int32_mul_ops_per_launch": ops_per_launch, "wide_products_per_launch": prods,
                "count": f"implemented: k = {k} channels per base, 2k^2+7k products per multiplication, "
                         "the kernel's window schedule",
                "frac_31bit_count": achieved31 / peak, "achieved_31bit_count": achieved31 / 1e12,
                "int32_mul_ops_per_launch_31bit_count": ops31,
                "count_31bit": f"k = {K31[1024]} channels of primes below 2^31, 2[2k(k+1)+8k] per "
                               "multiplication, |e|+ceil(|e|/w)+2^w+2 multiplications, conversions",
                "peak_def": f"{props.multi_processor_count} SMs x {IMAD_PER_CLK_PER_SM} int32-mul/clk x "
                            f"{max_mhz:.0f} MHz (a 32x32->64 product counts 2)",
                "microbench": {"mad_wide_per_s": wide_rate, "mad_lo_per_s": lo_rate,
                               "carry_pair_products_per_s": pair_rate, "mad_hi_per_s": hi_rate,
                               "peak_int32_mul_per_s": 2 * wide_rate, "frac": achieved / (2 * wide_rate),
                               "tensor_peaks": tensor},
                "crt_kernel_ms": crt_ms / max(1, crt_launch)}
    if vinfo["tensor"]:
        # the two extensions' slice products: 16 pairs of 8-bit slices, 2 k^2 operations each, per
        # number and multiplication; executed: the 128-row products with the zero columns and the offset
        # column (2 x 128 x (16 ceil(k/4)) x (4 (ceil(k/4)/4 + 1) 4) per block of 32 numbers)
        npt = -(-k // 4)
        kcols = 4 * ((npt // 4 + 1) * 4)
        t_alg = n_mm * 2 * 16 * 2 * k * k
        t_exec = (n_mm / 32) * 2 * 2 * 128 * (16 * npt) * kcols
        tpeak = measured_peak("bf16_tflops", 1.9e15 / 1e12) * 1e12
        t_s = mx_avg_ms / 1e3
        roofline["extensions"] = "tcgen05.mma kind::f16, fp32 accumulators in tensor memory (exact below 2^24)"
        roofline["count"] += "; the two extensions (2k^2 of the products) run on the tensor cores"
        roofline["tensor"] = {"achieved": t_alg / t_s / 1e12, "peak": tpeak / 1e12, "unit": "TFLOP/s",
                              "frac": t_alg / t_s / tpeak, "tensor_ops_per_launch": t_alg,
                              "executed_tensor_ops_per_launch": t_exec, "frac_executed": t_exec / t_s / tpeak,
                              "peak_def": "MEASURED_PEAKS bf16 burst (fp16 and bf16 share the tensor rate)",
                              "count": "2 extensions x 16 slice pairs x 2 k^2 per number and multiplication"}
    if clocks and clocks.get("sm_mhz"):
        roofline["frac_at_observed_clock"] = achieved / (props.multi_processor_count * IMAD_PER_CLK_PER_SM *
                                                          clocks["sm_mhz"] * 1e6)
    ctx.close()
    # the other configurations of the metric, each in a context of its own, at N = 1 only
    extra = {}
    if world == 1 and not args.no_extra and emit:
        for name, fn, sub in (("rsa2048_crt_constant_time", run_ours,
                               dict(steps=5, warmup=2, repeats=2, constant_time=True, no_extra=True)),
                              ("ragged_mix_65536", run_ragged, dict(steps=5, warmup=2)),
                              ("modexp16384_long_exponent", run_big, dict(steps=3, warmup=1, workload="modexp16384")),
                              ("rsa1024_encrypt_64", run_enc1024, dict(steps=200, warmup=5)),
                              ("serving_poisson_200k", run_serving_bench, dict(steps=10, warmup=1))):
            sa = argparse.Namespace(**{**vars(args), **sub, "no_cpu_baseline": True})
            t0 = time.time()
            try:
                extra[name] = fn(sa, rank, world, local_rank, emit=False)
            except Exception as ex:  # a failed sub-record is reported, the headline line still prints
                extra[name] = {"error": f"{type(ex).__name__}: {ex}"}
            log(f"{name}: {time.time() - t0:.1f} s")
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (seeded keys and ciphertexts)",
            "config": {"workload": "rsa2048_crt_decrypt", "ciphertexts_per_gpu": N_CT, "keys": 16,
                       "modexps_per_step_per_gpu": 2 * N_CT * R, "calls_per_step": R,
                       "modexps_per_call": 2 * N_CT, "decrypt_per_s": value / 2,
                       "k": k, "window": w, "l2": "flushed before every timed call (512 MB write)",
                       "parallelism": f"items partitioned over {world} GPU(s)"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(c_host.numel() * 4),
                    "d2h_bytes_per_step": int(m_host.numel() * 4)},
            "clocks": clocks,
            "gpu_launches": int(mx_launch + crt_launch),
            "configs": extra,
        }
        if args.constant_time:
            line["config"]["schedule"] = "constant time (regular fixed windows, masked table reads)"
        if not emit:
            return line
        print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- one size class
def class_workload(bits: int, n: int, rank: int = 0):
    """n exponentiations modulo 16 seeded odd `bits`-bit moduli (top bit set), bases uniform below the
    modulus, full-length exponents drawn per item (so the kernel runs fixed windows)."""
    from synth import SplitMix64
    r = SplitMix64(0x434C4153 + bits + 0x1000 * rank)
    mods = [r.randbits(bits) | 1 | (1 << (bits - 1)) for _ in range(16)]
    idx = [i % 16 for i in range(n)]
    xs = [r.below(mods[i]) for i in idx]
    es = [r.randbits(bits - 1) | (1 << (bits - 1)) for _ in range(n)]
    return mods, idx, xs, es


def run_class_modexp(args, rank, world, local_rank, emit=True):
    """`--items` exponentiations of one lane-group size class (`--bits`), one mr_modexp_batch call per
    step: the per-class profiling case of the lane-group kernel (bank conflicts, occupancy)."""
    import torch

    from paper_1305_3699_gb300 import mr

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    bits, n = args.bits, args.items
    mods, idx, xs, es = class_workload(bits, n, rank)
    L, k = mr.mr_class_for_bits(bits)
    W = L // 32
    ctx = mr.Context(local_rank)
    hk = [ctx.mr_rns_setup(N) for N in mods]
    kl = mr.KeyList([hk[i] for i in idx])
    nl = (bits + 31) // 32
    x_dev = mr.to_tensor(xs, nl, device=dev)
    e_dev = mr.to_tensor(es, nl, device=dev)
    out = torch.zeros_like(x_dev)
    status = torch.zeros(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        ctx.mr_modexp_batch(kl, x_dev, e_dev, out, status, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    got = mr.from_tensor(out)
    for j in range(0, n, max(1, n // 32)):
        assert got[j] == pow(xs[j], es[j], mods[idx[j]]), "benchmark output mismatch"
    assert int(status.sum()) == 0
    ctx.mr_profile_enable(True)
    ctx.mr_profile_read()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.zero_()
            evs[s][0].record(stream)
            step()
            evs[s][1].record(stream)
    torch.cuda.synchronize()
    (mx_launch, mx_ms), _ = ctx.mr_profile_read()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), world, dev)
    value = n * world * args.steps / (total_ms / 1e3)
    props = torch.cuda.get_device_properties(dev)
    WX = len(mr.mr_debug_class_table(L, "M"))
    w = window_for_bits(32 * nl)
    prods = sum(algorithmic_products_per_modexp(k, W, WX, 32 * nl, w, 1) for _ in range(n))
    ops31 = sum(ops_31bit_count(L, e.bit_length(), w) for e in es)
    peak = props.multi_processor_count * IMAD_PER_CLK_PER_SM * sm_max_mhz() * 1e6
    kms = mx_ms / max(1, mx_launch)
    ctx.close()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded moduli, bases, exponents)",
            "config": {"workload": f"modexp{bits}_class", "items_per_gpu": n, "keys": 16, "class_bits": L, "k": k,
                       "window": w, "l2": "flushed between timed steps (512 MB write)",
                       "parallelism": f"items partitioned over {world} GPU(s)"},
            "roofline": {"bound": "alu", "achieved": 2 * prods / (kms / 1e3) / 1e12, "peak": peak / 1e12,
                         "unit": "T int32-mul/s", "frac": 2 * prods / (kms / 1e3) / peak, "traffic": None,
                         "kernel": f"modexp_kernel<k={k}>", "kernel_ms": kms,
                         "count": f"implemented: k = {k}, 2k^2+7k products per multiplication, fixed windows",
                         "frac_31bit_count": ops31 / (kms / 1e3) / peak if L in K31 else None},
            "cpu_baseline": None, "gpu_launches": int(mx_launch)}
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- ragged mix
MIX = ((1024, 4), (2048, 3), (3072, 2), (4096, 1))  # sizes and weights (40/30/20/10%)
N_RAGGED = 65536


def ragged_workload(rank: int = 0, n: int = N_RAGGED):
    """Requests over the 256 mixed-size keys: size by the 40/30/20/10 mix, key uniform within the
    size, half encryptions (e = 65537) and half CRT decryptions, inputs uniform in [0, N)."""
    from synth import SplitMix64, load_keys
    keys = load_keys("mix_x256")
    by_bits = {}
    for i, k in enumerate(keys):
        by_bits.setdefault(k["bits"], []).append(i)
    r = SplitMix64(0x4D520004 + 0x1000 * rank)
    cum = []
    acc = 0
    for bits, w in MIX:
        acc += w
        cum.append((acc, bits))
    idx, ops, xs = [], [], []
    for _ in range(n):
        u = r.below(acc)
        bits = next(b for c, b in cum if u < c)
        pool = by_bits[bits]
        ki = pool[r.below(len(pool))]
        idx.append(ki)
        ops.append(r.below(2))
        xs.append(r.below(keys[ki]["N"]))
    return keys, idx, ops, xs


def run_enc1024(args, rank, world, local_rank, emit=True):
    """RSA-1024 public encryption of 64 messages (one per key, e = 65537): the call is launch- and
    latency-bound, so one step is one replay of a CUDA-graph-captured plan; reports throughput and
    the per-call latency."""
    import torch
    import torch.distributed as dist

    from paper_1305_3699_gb300 import mr
    from synth import SplitMix64, load_keys

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    keys = load_keys("rsa1024_x64")
    r = SplitMix64(0x4D520001 + 0x1000 * rank)
    msgs = [r.below(k["N"]) for k in keys]
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import plain
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 2.0:
            for m, k in zip(msgs, keys):
                plain.rsa_encrypt(m, k["e"], k["N"])
            reps += 1
        dt = time.perf_counter() - t0
        cpu = {"value": reps * len(msgs) / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{reps} passes over the 64 messages, oracle.plain.rsa_encrypt, one process"}
    ctx = mr.Context(local_rank)
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"]) for k in keys]
    kl = mr.KeyList(hk)
    m_dev = mr.to_tensor(msgs, 32, device=dev)
    c_dev = torch.zeros_like(m_dev)
    stream = torch.cuda.Stream(device=dev)
    plan = ctx.mr_plan_create(kl, [mr.MR_OP_ENCRYPT] * len(msgs), m_dev, c_dev,
                              flags=mr.MR_PLAN_GRAPH | mr.MR_PLAN_CONCURRENT)
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            plan.launch(stream)
    torch.cuda.synchronize()
    got = mr.from_tensor(c_dev[:2])
    for j in range(2):
        assert got[j] == pow(msgs[j], keys[j]["e"], keys[j]["N"]), "benchmark output mismatch"
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            evs[s][0].record(stream)
            plan.launch(stream)
            evs[s][1].record(stream)
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = len(msgs) * world * args.steps / (total_ms / 1e3)
    # end to end: H2D of the messages, the graph replay, D2H of the ciphertexts
    m_host, c_host = m_dev.cpu().pin_memory(), torch.empty_like(m_dev.cpu()).pin_memory()
    e2e = []
    with torch.cuda.stream(stream):
        for _ in range(max(10, args.steps // 4)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m_dev.copy_(m_host, non_blocking=True)
            plan.launch(stream)
            c_host.copy_(c_dev, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e.append(a.elapsed_time(b))
    info = plan.info()
    plan.free()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded keys and messages)",
            "config": {"workload": "rsa1024_encrypt_64", "messages": len(msgs), "keys": len(keys),
                       "launch": "one CUDA-graph replay of a prepared plan per step",
                       "latency_ms_p50": statistics.median(step_ms), "latency_ms_max": max(step_ms),
                       "kernels_per_step": info["kernels"],
                       "roofline": "not meaningful: 64 numbers occupy 16 warps of the GPU"},
            "cpu_baseline": cpu,
            "e2e": {"value": len(msgs) * world / (statistics.mean(e2e) / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(m_host.numel() * 4), "d2h_bytes_per_step": int(c_host.numel() * 4),
                    "latency_ms_p50": statistics.median(e2e)},
            "gpu_launches": info["kernels"] * args.steps}
    ctx.close()
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_mr1024(args, rank, world, local_rank):
    """Miller-Rabin batch: 4096 odd 1024-bit candidates (the primes p, q of the 2048-bit keys and
    seeded random odd numbers, half each) x 8 rounds with seeded witnesses in [2, n-2], one
    mr_miller_rabin_batch call per step; a round is one exponentiation a^d mod n plus up to s-1
    squarings."""
    import torch
    import torch.distributed as dist

    from paper_1305_3699_gb300 import mr
    from synth import SplitMix64, load_keys

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    rounds, n = 8, 4096
    keys = load_keys(KEYSET)
    primes = [k[h] for k in keys for h in ("p", "q")]
    r = SplitMix64(0x4D520006 + 0x1000 * rank)
    cands = [primes[i % len(primes)] if i % 2 == 0 else (r.randbits(1024) | 1 | (1 << 1023)) for i in range(n)]
    wit = [[2 + r.below(c - 3) for _ in range(rounds)] for c in cands]
    ctx = mr.Context(local_rank)
    cand_t = mr.to_tensor(cands, 32, device=dev)
    wit_t = mr.to_tensor([a for ws in wit for a in ws], 32, device=dev)
    flags = torch.zeros(n, dtype=torch.uint8, device=dev)
    mask = torch.zeros(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        ctx.mr_miller_rabin_batch(cand_t, wit_t, rounds, flags, mask, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
    torch.cuda.synchronize()
    f = flags.cpu().tolist()
    assert all(f[i] == 1 for i in range(0, n, 2)), "a prime was reported composite"
    from oracle import primality
    for i in (1, 3, 5):
        assert f[i] == (1 if all(primality.miller_rabin(cands[i], wit[i])) else 0)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            evs[s][0].record(stream)
            step()
            evs[s][1].record(stream)
    torch.cuda.synchronize()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), world, dev)
    value = n * rounds * world * args.steps / (total_ms / 1e3)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import multiprocessing as mpr
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        sample = [(cands[j], wit[j]) for j in range(min(n, 4 * cores))]
        with mpr.get_context("spawn").Pool(cores) as pool:
            t0 = time.perf_counter()
            pool.map(_oracle_mr_chunk, [sample[i::cores] for i in range(cores)])
            dt = time.perf_counter() - t0
        cpu = {"value": len(sample) * rounds / dt, "unit": "MR rounds/s", "cores": cores, "kind": "oracle",
               "sample": f"first {len(sample)} candidates x {rounds} rounds, oracle.primality on {cores} processes"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "MR rounds/s (one exponentiation each)", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic (seeded candidates and witnesses)",
                "config": {"workload": "miller_rabin_1024x4096x8", "candidates": n, "rounds": rounds,
                           "composites_found": int(n - sum(f))},
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def _oracle_prime_chunk(args):
    from oracle import primality
    t0 = time.perf_counter()
    for n, ws in args:
        primality.prime_test_verdict(n, ws)
    return time.perf_counter() - t0, len(args)


def run_primegen1024(args, rank, world, local_rank):
    """Key-generation primality search: 16384 seeded random odd 1024-bit candidates, each sieved by
    trial division with the first 10,000 primes and, when it survives, tested with 8 Miller-Rabin
    rounds (seeded witnesses in [2, n-2]); one mr_prime_test_batch call per step.  The same
    candidates through mr_miller_rabin_batch alone (no sieve) are timed beside it."""
    import torch
    import torch.distributed as dist

    from paper_1305_3699_gb300 import mr
    from synth import SplitMix64

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    rounds, n = 8, 16384
    r = SplitMix64(0x4D520007 + 0x1000 * rank)
    cands = [r.randbits(1024) | 1 | (1 << 1023) for _ in range(n)]
    wit = [[2 + r.below(c - 3) for _ in range(rounds)] for c in cands]
    ctx = mr.Context(local_rank)
    cand_t = mr.to_tensor(cands, 32, device=dev)
    wit_t = mr.to_tensor([a for ws in wit for a in ws], 32, device=dev)
    verdict = torch.zeros(n, dtype=torch.uint8, device=dev)
    surv = torch.zeros(1, dtype=torch.int32, device=dev)
    flags = torch.zeros(n, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        ctx.mr_prime_test_batch(cand_t, wit_t, rounds, verdict, survivors=surv, stream=stream)

    def step_mr_only():
        ctx.mr_miller_rabin_batch(cand_t, wit_t, rounds, flags, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
            step_mr_only()
    torch.cuda.synchronize()
    v = verdict.cpu().tolist()
    from oracle import primality
    for i in range(0, n, n // 16):
        assert v[i] == primality.prime_test_verdict(cands[i], wit[i]), "benchmark output mismatch"
    f = flags.cpu().tolist()
    assert all((v[i] == 2) == (f[i] == 1) for i in range(n) if v[i] > 0), "sieve and Miller-Rabin disagree"

    def timed(fn):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for s_ in range(args.steps):
                evs[s_][0].record(stream)
                fn()
                evs[s_][1].record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), world, dev)

    ctx.mr_profile_enable(True)
    ctx.mr_profile_read()
    total_ms = timed(step)
    prof = ctx.mr_profile_read()
    mr_only_ms = timed(step_mr_only)
    value = n * world * args.steps / (total_ms / 1e3)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import multiprocessing as mpr
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        sample = [(cands[j], wit[j]) for j in range(min(n, 64 * cores))]
        with mpr.get_context("spawn").Pool(cores) as pool:
            t0 = time.perf_counter()
            pool.map(_oracle_prime_chunk, [sample[i::cores] for i in range(cores)])
            dt = time.perf_counter() - t0
        cpu = {"value": len(sample) / dt, "unit": "candidates/s", "cores": cores, "kind": "oracle",
               "sample": f"first {len(sample)} candidates, oracle.primality.prime_test_verdict on {cores} processes"}
    if rank == 0:
        (mx_n, mx_ms), (tr_n, tr_ms) = prof
        line = {"metric": METRIC, "value": value, "unit": "candidates/s (trial division + Miller-Rabin)",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic (seeded random odd candidates and witnesses)",
                "config": {"workload": "primegen_1024x16384x8", "candidates": n, "rounds": rounds,
                           "trial_primes": 10000, "survivors": int(surv.item()),
                           "probable_primes": sum(1 for x in v if x == 2),
                           "trial_kernel_ms": tr_ms / max(1, tr_n), "mr_kernel_ms": mx_ms / max(1, mx_n),
                           "miller_rabin_only_ms": mr_only_ms / args.steps,
                           "sieve_speedup": mr_only_ms / total_ms},
                "cpu_baseline": cpu, "gpu_launches": int(mx_n + tr_n)}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def _oracle_keygen_chunk(args):
    from oracle import keygen
    t0 = time.perf_counter()
    for pp, wp, pq, wq in args:
        keygen.rsa_key_from_pools(pp, wp, pq, wq, 65537)
    return time.perf_counter() - t0, len(args)


def run_keygen2048(args, rank, world, local_rank):
    """RSA-2048 key generation on the device: 16 keys, each from pools of 2048 seeded random odd
    1024-bit candidates for p and for q (top two bits set), 4 Miller-Rabin rounds with seeded
    witnesses; one mr_rsa_keygen_batch call per step (trial division and Miller-Rabin on every
    candidate, then the key assembly with Arazi's inversion)."""
    import torch
    import torch.distributed as dist

    from paper_1305_3699_gb300 import mr
    from synth import SplitMix64

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n_keys, pool, rounds, H = 16, 2048, 4, 32
    r = SplitMix64(0x4D520008 + 0x1000 * rank)
    pools = [[r.randbits(1024) | (3 << 1022) | 1 for _ in range(pool)] for _ in range(2 * n_keys)]
    wits = [[[r.between(2, c - 2) for _ in range(rounds)] for c in pl] for pl in pools]
    ctx = mr.Context(local_rank)
    cand_t = mr.to_tensor([c for pl in pools for c in pl], H, device=dev)
    wit_t = mr.to_tensor([w for wl in wits for ws in wl for w in ws], H, device=dev)
    out = torch.zeros((n_keys, 9 * H), dtype=torch.int32, device=dev)
    st = torch.zeros(n_keys, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def step():
        ctx.mr_rsa_keygen_batch(cand_t, wit_t, rounds, n_keys, pool, out, status=st, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
    torch.cuda.synchronize()
    from oracle import keygen
    rows = out.cpu().numpy().astype("int64") & 0xFFFFFFFF
    for k in (0, n_keys - 1):
        want = keygen.rsa_key_from_pools(pools[2 * k], wits[2 * k], pools[2 * k + 1], wits[2 * k + 1], 65537)
        got_n = sum(int(v) << (32 * i) for i, v in enumerate(rows[k][:2 * H]))
        assert (want is None and int(st[k]) == 5) or (want is not None and got_n == want["N"]), "keygen mismatch"
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ctx.mr_profile_enable(True)
    ctx.mr_profile_read()
    with torch.cuda.stream(stream):
        for s_ in range(args.steps):
            evs[s_][0].record(stream)
            step()
            evs[s_][1].record(stream)
    torch.cuda.synchronize()
    prof = ctx.mr_profile_read()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), world, dev)
    made = int((st == 0).sum())
    value = made * world * args.steps / (total_ms / 1e3)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import multiprocessing as mpr
        cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
        sample = [(pools[2 * k], wits[2 * k], pools[2 * k + 1], wits[2 * k + 1]) for k in range(n_keys)]
        with mpr.get_context("spawn").Pool(cores) as pool_:
            t0 = time.perf_counter()
            pool_.map(_oracle_keygen_chunk, [sample[i::cores] for i in range(cores) if sample[i::cores]])
            dt = time.perf_counter() - t0
        cpu = {"value": n_keys / dt, "unit": "keys/s", "cores": cores, "kind": "oracle",
               "sample": f"all {n_keys} keys, oracle.keygen.rsa_key_from_pools on {cores} processes"}
    if rank == 0:
        (mx_n, mx_ms), (tr_n, tr_ms) = prof
        line = {"metric": METRIC, "value": value, "unit": "RSA-2048 keys/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32",
                "data": "synthetic (seeded candidate pools and witnesses)",
                "config": {"workload": "keygen_rsa2048_16x2x2048", "keys": n_keys, "pool": pool, "rounds": rounds,
                           "keys_made": made, "mr_kernel_ms": mx_ms / max(1, mx_n),
                           "trial_kernel_ms": tr_ms / max(1, tr_n)},
                "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_ragged(args, rank, world, local_rank, emit=True):
    """Ragged batch: one prepared plan per launch mode over the same 65,536 requests (emit=False:
    return the JSON line instead of printing it)."""
    import torch
    from paper_1305_3699_gb300 import mr
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    keys, idx, ops, xs = ragged_workload(rank)
    ctx = mr.Context(local_rank)
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
    kl = mr.KeyList([hk[i] for i in idx])
    inp = mr.to_tensor(xs, 128, device=dev)
    out = torch.zeros_like(inp)
    status = torch.zeros(len(xs), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    modexps = sum(1 if o == 0 else 2 for o in ops)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("timing the CPU oracle on a bounded sample ...")
        v, cores, desc = oracle_mixed_throughput(keys, idx, ops, xs)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    # every mode runs the same tuned kernels: tune each size class of the mix once, with its item
    # count and longest exponent in this workload
    per_class = {}
    for i, o in zip(idx, ops):
        k = keys[i]
        L = mr.mr_class_for_bits(k["N"].bit_length() if o == 0 else k["p"].bit_length())[0]
        ebits = k["e"].bit_length() if o == 0 else max(k["dp"].bit_length(), k["dq"].bit_length())
        c = per_class.setdefault(L, [0, 0])
        c[0] += 1 if o == 0 else 2
        c[1] = max(c[1], ebits)
    tuning = {}
    if not args.no_autotune:
        for L, (cnt, eb) in sorted(per_class.items()):
            tuning[L] = ctx.mr_autotune(L, max(256, min(cnt, 8192)), eb)
    modes = {"per_size_plain": 0,
             "ragged_concurrent_graph": mr.MR_PLAN_CONCURRENT | mr.MR_PLAN_GRAPH,
             "ragged_persistent_graph": mr.MR_PLAN_CONCURRENT | mr.MR_PLAN_PERSISTENT | mr.MR_PLAN_GRAPH}
    res = {}
    ref = None
    for name, flags in modes.items():
        plan = ctx.mr_plan_create(kl, ops, inp, out, status, flags=flags)
        info = plan.info()
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                plan.launch(stream)
        torch.cuda.synchronize()
        if ref is None:
            ref = out.clone()
        assert torch.equal(out, ref), "launch modes disagree"
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for s in range(args.steps):
                flush.zero_()
                evs[s][0].record(stream)
                plan.launch(stream)
                evs[s][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        res[name] = {"ms_per_step": ms, "modexp_per_s": modexps / (ms / 1e3), "kernels": info["kernels"],
                     "groups": info["groups"], "products": info["products"]}
        plan.free()
    # every mode gave the same outputs (checked above); a seeded sample of 256 against the plain
    # definition
    from synth import SplitMix64
    rs = SplitMix64(0x5241474745)
    sample = sorted({rs.below(len(xs)) for _ in range(256)})
    got = mr.from_tensor(out[sample])
    for j, g in zip(sample, got):
        k = keys[idx[j]]
        assert g == pow(xs[j], k["e"] if ops[j] == 0 else k["d"], k["N"]), "ragged output mismatch"
    assert int(status.sum()) == 0
    for r in res.values():
        r["exact"] = True
    # roofline of the whole step (several kernels) under both multiplication counts
    import torch as _t
    props = _t.cuda.get_device_properties(dev)
    peak = props.multi_processor_count * IMAD_PER_CLK_PER_SM * sm_max_mhz() * 1e6
    prods = 0
    ops31 = 0
    for i, o in zip(idx, ops):
        k = keys[i]
        if o == 0:
            L, kk = mr.mr_class_for_bits(k["N"].bit_length())
            WX = len(mr.mr_debug_class_table(L, "M"))
            w = window_for_bits(k["e"].bit_length())
            prods += algorithmic_products_per_modexp(kk, L // 32, WX, k["e"].bit_length(), w, 1)
            ops31 += ops_31bit_count(L, k["e"].bit_length(), w)
        else:
            L, kk = mr.mr_class_for_bits(k["p"].bit_length())
            WX = len(mr.mr_debug_class_table(L, "M"))
            for h in (k["dp"], k["dq"]):
                w = window_for_bits(h.bit_length())
                prods += (algorithmic_products_sliding(kk, L // 32, WX, h, w, 2) if w >= 4 else
                          algorithmic_products_per_modexp(kk, L // 32, WX, h.bit_length(), w, 2))
                ops31 += ops_31bit_count(L, h.bit_length(), w)
    best = min(res, key=lambda m: res[m]["ms_per_step"])
    # the value is the faster of the two single-replay plan forms (both one CUDA-graph launch per step)
    vmode = min(("ragged_concurrent_graph", "ragged_persistent_graph"), key=lambda m: res[m]["ms_per_step"])
    rp = res[vmode]
    for r in res.values():
        r["frac"] = 2 * prods / (r["ms_per_step"] / 1e3) / peak
        r["frac_31bit_count"] = ops31 / (r["ms_per_step"] / 1e3) / peak
    roofline = {"bound": "alu", "achieved": 2 * prods / (rp["ms_per_step"] / 1e3) / 1e12, "peak": peak / 1e12,
                "unit": "T int32-mul/s", "frac": 2 * prods / (rp["ms_per_step"] / 1e3) / peak, "traffic": None,
                "kernel": f"whole step of the {vmode} plan (all kernels)",
                "frac_31bit_count": ops31 / (rp["ms_per_step"] / 1e3) / peak,
                "int32_mul_ops_per_step": 2 * prods, "int32_mul_ops_per_step_31bit_count": ops31,
                "count": "implemented k, 2k^2+7k products per multiplication, the kernels' window schedules",
                "count_31bit": "k of primes below 2^31 (34/67/100/133 for 1024-4096 bits), "
                               "2[2k(k+1)+8k] per multiplication, |e|+ceil(|e|/w)+2^w+2 multiplications"}
    line = {"metric": METRIC, "value": rp["modexp_per_s"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rp["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded keys and inputs)",
            "config": {"workload": "ragged_mix_65536", "requests": len(xs), "modexps_per_step": modexps,
                       "keys": 256, "mix_bits": [b for b, _ in MIX], "mix_weights": [w for _, w in MIX],
                       "l2": "flushed between timed steps (512 MB write)", "modes": res,
                       "fastest_mode": best, "value_mode": vmode,
                       "exact": "all modes identical; 256 seeded samples equal x^e mod N",
                       "autotune": {str(L): v for L, v in tuning.items()},
                       "speedup_vs_per_size_plain": res["per_size_plain"]["ms_per_step"] / rp["ms_per_step"],
                       "speedup_concurrent_vs_per_size_plain":
                           res["per_size_plain"]["ms_per_step"] / res["ragged_concurrent_graph"]["ms_per_step"],
                       "speedup_persistent_vs_per_size_plain":
                           res["per_size_plain"]["ms_per_step"] / res["ragged_persistent_graph"]["ms_per_step"]},
            "roofline": roofline, "cpu_baseline": cpu}
    ctx.close()
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_big(args, rank, world, local_rank, emit=True):
    """Large-class workloads over four 16384-bit RSA keys, one call per step:
      modexp16384   256 exponentiations x^e mod N with uniform 16128-bit exponents (mr_modexp_batch;
                    the 16384-bit class runs as one cooperative launch of 8 groups x 19 channel slices)
      rsa16384_crt  256 CRT decryptions (mr_rsa_decrypt_crt): 512 exponentiations modulo the 8192-bit
                    primes in the 8192-bit class, then the binary Garner recombination"""
    import torch
    import torch.distributed as dist

    from paper_1305_3699_gb300 import mr

    crt = args.workload == "rsa16384_crt"
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if crt:
        keys, idx, xs = big_crt_workload(rank)
        es = None
    else:
        keys, idx, xs, es = big_workload(rank, args.ebits)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("timing the CPU oracle on a bounded sample ...")
        if crt:
            v, cores, desc, _ = oracle_throughput(keys, idx, xs, args.cpu_seconds)
        else:
            v, cores, desc, _ = oracle_big_throughput(keys, idx, xs, es)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    ctx = mr.Context(local_rank)
    if crt:
        hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
    else:
        hk = [ctx.mr_rns_setup(k["N"]) for k in keys]
    kl = mr.KeyList([hk[i] for i in idx])
    W, EL = 512, (args.ebits + 31) // 32
    x_dev = mr.to_tensor(xs, W, device=dev)
    e_dev = None if crt else mr.to_tensor(es, EL, device=dev)
    out = torch.zeros_like(x_dev)
    status = torch.zeros(BIG_N, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        if crt:
            ctx.mr_rsa_decrypt_crt(kl, x_dev, out, status, stream=stream)
        else:
            ctx.mr_modexp_batch(kl, x_dev, e_dev, out, status, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()
    got = mr.from_tensor(out[:2])
    for j in range(2):
        k = keys[idx[j]]
        if crt:
            assert pow(got[j], k["e"], k["N"]) == xs[j], "benchmark output mismatch"
        else:
            assert got[j] == pow(xs[j], es[j], k["N"]), "benchmark output mismatch"
    assert int(status.sum()) == 0
    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    gpu_index = vis[local_rank] if local_rank < len(vis) else (vis[0] if vis else str(local_rank))
    sampler = ClockSampler(gpu_index) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    ctx.mr_profile_enable(True)
    ctx.mr_profile_read()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.zero_()
            evs[s][0].record(stream)
            step()
            evs[s][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall1 = time.time()
    prof = ctx.mr_profile_read()
    total_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), world, dev)
    per_item = 2 if crt else 1  # exponentiations per item
    value = per_item * BIG_N * world * args.steps / (total_ms / 1e3)
    # end to end: H2D of the inputs, the call, D2H of the results
    x_host = x_dev.cpu().pin_memory()
    e_host = None if crt else e_dev.cpu().pin_memory()
    o_host = torch.empty_like(x_host).pin_memory()
    e2e_ms = []
    with torch.cuda.stream(stream):
        for _ in range(max(2, args.steps // 2)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            x_dev.copy_(x_host, non_blocking=True)
            if e_host is not None:
                e_dev.copy_(e_host, non_blocking=True)
            step()
            o_host.copy_(out, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e2e_ms.append(a.elapsed_time(b))
    e2e_val = per_item * BIG_N * world / (statistics.mean(e2e_ms) / 1e3)
    clocks = sampler.summary(t_wall0, t_wall1) if sampler else None
    if sampler:
        sampler.stop()
    if crt:
        L, k = mr.mr_class_for_bits(8192)
        WX = len(mr.mr_debug_class_table(L, "M"))
        Wm = L // 32
        ebits = max(max(keys[i]["dp"].bit_length(), keys[i]["dq"].bit_length()) for i in idx)
        w = window_for_bits(ebits, 8)
        prods = sum(algorithmic_products_per_modexp(k, Wm, WX, keys[i][h].bit_length(), w, 2)
                    for i in idx for h in ("dp", "dq"))
    else:
        L, k = mr.mr_class_for_bits(16384)
        WX = len(mr.mr_debug_class_table(L, "M"))
        w = window_for_bits(args.ebits, 8)
        prods = sum(algorithmic_products_per_modexp(k, W, WX, e.bit_length(), w, 1) for e in es)
    ops31 = (sum(ops_31bit_count(L, keys[i][h].bit_length(), w) for i in idx for h in ("dp", "dq")) if crt else
             sum(ops_31bit_count(L, e.bit_length(), w) for e in es))
    (mx_launch, mx_ms), (crt_launch, crt_ms) = prof
    mx_avg_ms = mx_ms / max(1, mx_launch)
    props = torch.cuda.get_device_properties(dev)
    max_mhz = sm_max_mhz()
    peak = props.multi_processor_count * IMAD_PER_CLK_PER_SM * max_mhz * 1e6
    achieved = 2 * prods / (mx_avg_ms / 1e3)
    variant = big_variant_used(mr, L, len(idx) * (2 if crt else 1))
    vinfo = mr.mr_big_variant_info(L, variant)
    wide_rate = ctx.mr_imad_peak(0, stream)
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "T int32-mul/s",
                "frac": achieved / peak, "traffic": None, "kernel": f"big_modexp_kernel<k={k}> (channel-slice width: the variant with the fewest estimated waves)",
                "kernel_ms": mx_avg_ms, "int32_mul_ops_per_launch": 2 * prods, "window": w,
                "peak_def": f"{props.multi_processor_count} SMs x {IMAD_PER_CLK_PER_SM} int32-mul/clk x "
                            f"{max_mhz:.0f} MHz (a 32x32->64 product counts 2)",
                "microbench": {"mad_wide_per_s": wide_rate, "peak_int32_mul_per_s": 2 * wide_rate,
                               "frac": achieved / (2 * wide_rate)},
                "count": f"implemented: k = {k} channels per base, 2k^2+7k products per multiplication, "
                         "fixed windows",
                "frac_31bit_count": ops31 / (mx_avg_ms / 1e3) / peak,
                "achieved_31bit_count": ops31 / (mx_avg_ms / 1e3) / 1e12,
                "int32_mul_ops_per_launch_31bit_count": ops31,
                "count_31bit": f"k = {K31[L]} channels of primes below 2^31, 2[2k(k+1)+8k] per multiplication, "
                               "|e|+ceil(|e|/w)+2^w+2 multiplications, conversions"}
    if vinfo["tensor"]:
        # the base extensions ran on the tensor cores: the dominant unit is the tensor pipe.  Algorithmic
        # work: per multiplication 2 extensions x 16 fp16 slice pairs x 2 n k^2 (n numbers, k channels);
        # executed: the padded products the kernel issues (128 x 128 x 16 per step, 19 blocks per group)
        nums = len(idx) * (2 if crt else 1)
        ebits_all = ([keys[i][h].bit_length() for i in idx for h in ("dp", "dq")] if crt else
                     [e.bit_length() for e in es])
        mms = [1 + (2 ** w - 2) + (w + 1) * (max(1, math.ceil(b / w)) - 1) + 1 + (1 if crt else 0) for b in ebits_all]
        tensor_alg = sum(m * 2 * 16 * 2 * k * k for m in mms)
        groups = math.ceil(nums / 32)
        kp = math.ceil(k / 64) * 64
        tensor_exec = max(mms) * groups * vinfo["slices"] * 2 * (kp // 16) * 2 * 128 * 128 * 16
        tensor31 = sum(mm31 * 2 * 16 * 2 * K31[L] * (K31[L] + 1) for mm31 in
                       (b + math.ceil(b / w) + 2 ** w + 2 for b in ebits_all))
        t_s = mx_avg_ms / 1e3
        tpeak = measured_peak("bf16_tflops_sustained", 1700.0) * 1e12
        tc_probe = ctx.mr_tensor_peak(0, stream)
        imad = {k2: roofline[k2] for k2 in ("bound", "achieved", "peak", "unit", "frac", "frac_31bit_count")}
        roofline = {"bound": "tensor", "achieved": tensor_alg / t_s / 1e12, "peak": tpeak / 1e12, "unit": "TFLOP/s",
                    "frac": tensor_alg / t_s / tpeak, "traffic": None,
                    "kernel": f"big_modexp_kernel<k={k}, base extensions on tcgen05 (fp16 slices)>",
                    "kernel_ms": mx_avg_ms, "window": w,
                    "tensor_ops_per_launch": tensor_alg,
                    "count": f"2 extensions x 16 slice pairs x 2 n k^2 per multiplication, k = {k}",
                    "executed_tensor_ops_per_launch": tensor_exec, "frac_executed": tensor_exec / t_s / tpeak,
                    "frac_31bit_count": tensor31 / t_s / tpeak, "tensor_ops_per_launch_31bit_count": tensor31,
                    "count_31bit": f"2 x 16 x 2 n k(k+1) per multiplication, k = {K31[L]}, "
                                   "|e|+ceil(|e|/w)+2^w+2 multiplications",
                    "peak_def": "MEASURED_PEAKS bf16 sustained (a seconds-long kernel; fp16 and bf16 share the "
                                "tensor rate)",
                    "tcgen05_f16_probe_tflops": tc_probe / 1e12, "frac_of_probe": tensor_alg / t_s / tc_probe,
                    "integer_pipe_equivalent": imad}
    roofline["variant"] = {"index": variant, **vinfo}
    if crt:
        roofline["crt_kernel"] = "crt_bin_kernel (binary Garner, one warp per decryption)"
        roofline["crt_kernel_ms"] = crt_ms / max(1, crt_launch)
        config = {"workload": "rsa16384_crt_decrypt", "ciphertexts_per_gpu": BIG_N, "keys": len(keys),
                  "modulus_bits": 16384, "half_bits": 8192, "modexps_per_step": 2 * BIG_N, "k_half": k,
                  "decrypt_per_s": value / 2}
        data = "synthetic (seeded 16384-bit RSA keys and ciphertexts)"
    else:
        config = {"workload": "modexp16384_long_exponent", "items_per_gpu": BIG_N, "keys": len(keys),
                  "modulus_bits": 16384, "exponent_bits": args.ebits, "k": k}
        data = "synthetic (seeded 16384-bit RSA moduli, bases and exponents)"
    config.update({"l2": "flushed between timed steps (512 MB write)",
                   "parallelism": f"items partitioned over {world} GPU(s)"})
    h2d = x_host.numel() * 4 + (0 if e_host is None else e_host.numel() * 4)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": data, "config": config,
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(o_host.numel() * 4)},
            "clocks": clocks, "gpu_launches": prof[0][0] + prof[1][0]}
    ctx.close()
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serving_bench(args, rank, world, local_rank, emit=True):
    """Serving workload: Poisson arrivals at 200k requests/s over the 256 mixed-size keys, served by
    the continuous-batching loop of paper_1305_3699_gb300.serve."""
    import numpy as np
    import torch

    from paper_1305_3699_gb300 import mr
    from paper_1305_3699_gb300.serve import Server, poisson_arrivals
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    rate = 200_000.0
    n = max(4096, int(rate * max(1.0, args.steps * 0.2)))
    keys, idx, ops, xs = ragged_workload(rank, n)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("timing the CPU oracle on a bounded sample ...")
        v, cores, desc = oracle_mixed_throughput(keys, idx, ops, xs)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}
    ctx = mr.Context(local_rank)
    hk = [ctx.mr_rsa_key_setup(k["N"], k["e"], k["p"], k["q"], k["dp"], k["dq"], k["qinv"]) for k in keys]
    rows = np.zeros((n, 128), dtype=np.uint32)
    for i, x in enumerate(xs):
        rows[i] = np.frombuffer(x.to_bytes(512, "little"), dtype="<u4")
    rows = rows.view(np.int32)
    arrivals = poisson_arrivals(rate, n, 0x4D520005 + rank)
    srv = Server(ctx, hk, capacity=args.serve_capacity, slots=args.serve_slots,
                 latency_mappings=args.serve_mappings == "widest")
    # warm-up on a slice
    w = min(n, 8192)
    srv.run(arrivals[:w] - arrivals[0], np.array(idx[:w]), np.array(ops[:w]), rows[:w])
    out, status, lat, stats = srv.run(arrivals, np.array(idx), np.array(ops), rows)
    modexps = sum((1 if ops[i] == 0 else 2) for i in range(n) if not np.isnan(lat[i]))
    # spot check of served results against the plain definition
    for j in list(range(0, n, max(1, n // 8)))[:8]:
        kj = keys[idx[j]]
        want = pow(xs[j], kj["e"] if ops[j] == 0 else kj["d"], kj["N"])
        got = int.from_bytes(out[j].view(np.uint32).astype("<u4").tobytes(), "little")
        assert got == want, "serving result mismatch"
    line = {"metric": METRIC, "value": modexps / stats["wall_s"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic (seeded keys, inputs, arrivals)",
            "config": {"workload": "serving_poisson_200k", "offered_req_per_s": rate, "slot_capacity": srv.capacity,
                       "slots": len(srv.slots), "lanes_per_number": {str(L): t for L, t in srv.mappings.items()},
                       **stats},
            "cpu_baseline": cpu}
    ctx.close()
    if not emit:
        return line
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="ragged workload: keep the default configurations")
    ap.add_argument("--serve-capacity", type=int, default=4096, help="serving workload: requests per batch slot")
    ap.add_argument("--serve-slots", type=int, default=3, help="serving workload: batch slots in flight")
    ap.add_argument("--serve-mappings", default="widest", choices=["widest", "default"],
                    help="serving workload: each class's widest lane mapping, or its default one")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--repeats", type=int, default=8,
                    help="rsa2048_crt: calls per step (each after an L2 flush, each inside its own events)")
    ap.add_argument("--constant-time", action="store_true",
                    help="rsa2048_crt: constant-time exponentiation schedule (mr_set_constant_time)")
    ap.add_argument("--no-extra", action="store_true",
                    help="rsa2048_crt: skip the ragged, long-exponent, RSA-1024 and serving sub-records")
    ap.add_argument("--bits", type=int, default=1536, help="class_modexp workload: modulus bits")
    ap.add_argument("--items", type=int, default=4096, help="class_modexp workload: exponentiations per call")
    ap.add_argument("--ebits", type=int, default=BIG_EBITS,
                    help="exponent bits of the modexp16384 workload (smaller values for profiling runs)")
    ap.add_argument("--workload", default="rsa2048_crt", choices=["rsa2048_crt", "ragged", "serving", "modexp16384", "rsa16384_crt",
                                                             "rsa1024_enc", "mr1024", "primegen1024", "keygen2048",
                                                             "class_modexp"])
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", init_method="env://")
    try:
        if args.workload == "ragged":
            return run_ragged(args, rank, world, local_rank)
        if args.workload in ("modexp16384", "rsa16384_crt"):
            return run_big(args, rank, world, local_rank)
        if args.workload == "rsa1024_enc":
            return run_enc1024(args, rank, world, local_rank)
        if args.workload == "mr1024":
            return run_mr1024(args, rank, world, local_rank)
        if args.workload == "primegen1024":
            return run_primegen1024(args, rank, world, local_rank)
        if args.workload == "keygen2048":
            return run_keygen2048(args, rank, world, local_rank)
        if args.workload == "serving":
            return run_serving_bench(args, rank, world, local_rank)
        if args.workload == "class_modexp":
            return run_class_modexp(args, rank, world, local_rank)
        return run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
