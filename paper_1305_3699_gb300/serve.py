"""Continuous-batching request loop over the RNS exponentiation library.

Requests (RSA encryptions and CRT decryptions of any supported size, each with
its own key) arrive over time.  The loop keeps every key's RNS tables resident
on the device (they are set up once), and whenever a batch slot is free it
admits the requests that have arrived -- up to the slot's capacity and to a
device-memory budget estimated per request -- uploads their inputs, launches
one mixed call on the slot's stream, and reads the results back.  Several
slots are in flight at once, so requests that arrive while others are on the
GPU start as soon as a slot frees up and their work overlaps with the earlier
batches.  Latency is measured from a request's arrival time to the moment the
host sees its result.

All arithmetic runs in the library's kernels; this module only moves rows
between host and device buffers and calls mr_rsa_mixed.
"""
from __future__ import annotations

import ctypes
import math
import time
from collections import deque
from typing import List, Optional, Sequence

import numpy as np

from . import mr


def request_footprint_bytes(bits: int, op: int, row_limbs: int) -> int:
    """Device bytes one request holds while in flight: its input and output rows, and the
    window tables of its exponentiations (2^5 entries x 2k residues of 4 bytes per number)."""
    L = bits if op == mr.MR_OP_ENCRYPT else (bits + 1) // 2
    _, k = mr.mr_class_for_bits(max(L, 1))
    per_modexp = 32 * 2 * k * 4
    return 2 * row_limbs * 4 + per_modexp * (1 if op == mr.MR_OP_ENCRYPT else 2)


class _Slot:
    def __init__(self, torch, device, capacity: int, row_limbs: int):
        self.d_in = torch.zeros((capacity, row_limbs), dtype=torch.int32, device=device)
        self.d_out = torch.zeros_like(self.d_in)
        self.d_status = torch.zeros(capacity, dtype=torch.uint8, device=device)
        self.h_in = torch.zeros((capacity, row_limbs), dtype=torch.int32).pin_memory()
        self.h_out = torch.zeros_like(self.h_in).pin_memory()
        self.h_status = torch.zeros(capacity, dtype=torch.uint8).pin_memory()
        self.stream = torch.cuda.Stream(device=device)
        self.event = torch.cuda.Event()
        self.ids: Optional[np.ndarray] = None
        self.bytes = 0


class Server:
    """Continuous batching of mixed RSA requests.

    ctx          an mr.Context
    keys         the key handles requests refer to (resident on the device)
    capacity     requests per batch slot
    slots        batch slots in flight at once
    hbm_budget   device bytes all in-flight requests may hold (admission limit)
    """

    def __init__(self, ctx: "mr.Context", keys: Sequence["mr.Key"], capacity: int = 2048, slots: int = 3,
                 row_limbs: int = 128, hbm_budget: int = 1 << 30, flags: int = mr.MR_PLAN_PERSISTENT,
                 latency_mappings: bool = True):
        import torch
        self.torch = torch
        self.ctx = ctx
        self.keys = list(keys)
        self.mappings = {}
        if latency_mappings:
            # below full load, more lanes per number shorten each exponentiation's chain of
            # multiplications: take the widest compiled lane mapping of every class in use
            classes = set()
            for k in self.keys:
                classes.add(mr.mr_class_for_bits(k.N.bit_length())[0])
                if getattr(k, "half_bits", 0):
                    classes.add(mr.mr_class_for_bits(k.half_bits)[0])
            for L in sorted(classes):
                lanes = mr.mr_class_variants(L)
                if lanes:
                    v = max(range(len(lanes)), key=lambda i: lanes[i])
                    ctx.mr_set_variant(L, v)
                    self.mappings[L] = lanes[v]
        self.key_ptrs = np.array([k.handle for k in self.keys], dtype=np.uint64)
        self.key_bits = np.array([k.N.bit_length() for k in self.keys], dtype=np.int64)
        self.capacity, self.row_limbs, self.hbm_budget, self.flags = capacity, row_limbs, hbm_budget, flags
        dev = torch.device("cuda", ctx.device)
        self.slots = [_Slot(torch, dev, capacity, row_limbs) for _ in range(slots)]
        self.in_flight_bytes = 0

    def _launch(self, slot: _Slot, ids: np.ndarray, rows: np.ndarray, key_idx: np.ndarray, ops: np.ndarray,
                foot: np.ndarray):
        n = len(ids)
        slot.ids = ids
        slot.bytes = int(foot[ids].sum())
        self.in_flight_bytes += slot.bytes
        slot.h_in.numpy()[:n] = rows[ids]
        kp = np.ascontiguousarray(self.key_ptrs[key_idx[ids]])
        op = np.ascontiguousarray(ops[ids].astype(np.uint8))
        with self.torch.cuda.stream(slot.stream):
            slot.d_in[:n].copy_(slot.h_in[:n], non_blocking=True)
            rc = mr.lib.mr_rsa_mixed(self.ctx.handle, kp.ctypes.data_as(ctypes.c_void_p),
                                     op.ctypes.data_as(ctypes.c_void_p), n, slot.d_in.data_ptr(), self.row_limbs,
                                     slot.d_out.data_ptr(), self.row_limbs, slot.d_status.data_ptr(), self.flags,
                                     slot.stream.cuda_stream)
            self.ctx._check(rc)
            slot.h_out[:n].copy_(slot.d_out[:n], non_blocking=True)
            slot.h_status[:n].copy_(slot.d_status[:n], non_blocking=True)
            slot.event.record(slot.stream)
        slot._keep = (kp, op)

    def run(self, arrivals: np.ndarray, key_idx: np.ndarray, ops: np.ndarray, rows: np.ndarray,
            max_queue_s: float = 1.0):
        """Serve requests i with arrival time arrivals[i] (seconds from start, sorted), key
        keys[key_idx[i]], operation ops[i] and input row rows[i].  Returns (out rows, status,
        latency per request in seconds (nan when rejected), stats)."""
        n = len(arrivals)
        out = np.zeros((n, self.row_limbs), dtype=np.int32)
        status = np.zeros(n, dtype=np.uint8)
        lat = np.full(n, np.nan)
        foot = np.array([request_footprint_bytes(int(self.key_bits[key_idx[i]]), int(ops[i]), self.row_limbs)
                         for i in range(n)], dtype=np.int64)
        ready = deque()
        nxt = 0
        done = 0
        rejected = 0
        batches = 0
        busy: List[_Slot] = []
        idle = list(self.slots)
        t0 = time.perf_counter()
        while done + rejected < n:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[nxt] <= now:
                ready.append(nxt)
                nxt += 1
            for s in list(busy):
                if s.event.query():
                    t = time.perf_counter() - t0
                    k = len(s.ids)
                    out[s.ids] = s.h_out.numpy()[:k]
                    status[s.ids] = s.h_status.numpy()[:k]
                    lat[s.ids] = t - arrivals[s.ids]
                    done += k
                    self.in_flight_bytes -= s.bytes
                    busy.remove(s)
                    idle.append(s)
            # drop requests that waited too long for admission
            while ready and now - arrivals[ready[0]] > max_queue_s:
                i = ready.popleft()
                status[i] = 9  # MR_ERR_BUSY
                rejected += 1
            if ready and idle:
                take = []
                budget = self.hbm_budget - self.in_flight_bytes
                while ready and len(take) < self.capacity and foot[ready[0]] <= budget:
                    i = ready.popleft()
                    budget -= foot[i]
                    take.append(i)
                if take:
                    s = idle.pop()
                    self._launch(s, np.array(take, dtype=np.int64), rows, key_idx, ops, foot)
                    busy.append(s)
                    batches += 1
                    continue
            if not busy and not ready and nxt < n:
                wait = arrivals[nxt] - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        wall = time.perf_counter() - t0
        ok = ~np.isnan(lat)
        stats = {"requests": n, "completed": int(ok.sum()), "rejected": rejected, "batches": batches,
                 "wall_s": wall, "throughput_req_s": float(ok.sum()) / wall,
                 "p50_ms": float(np.percentile(lat[ok], 50) * 1e3) if ok.any() else None,
                 "p99_ms": float(np.percentile(lat[ok], 99) * 1e3) if ok.any() else None,
                 "mean_ms": float(np.mean(lat[ok]) * 1e3) if ok.any() else None}
        return out, status, lat, stats


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    """Sorted arrival times (s) of a Poisson process of the given rate (seeded exponential gaps)."""
    from synth import SplitMix64
    r = SplitMix64(seed)
    t = 0.0
    out = np.empty(n)
    for i in range(n):
        t += r.exponential(rate)
        out[i] = t
    return out
