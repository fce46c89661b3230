"""Autotuner for batched searches: picks the overlap-save segment length L,
the persistent grid (CTAs per SM) and, for L = 1024, the templates each CTA
applies to a segment before the next (templates per block) by timing
fdas_correlate_batched on a probe set of trials, and caches the choice per
(GPU, search shape)."""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import fdas_make_templates
from .batch import BatchSearch

# (L, CTAs per SM, templates per block); 0 = the default
DEFAULT_CANDIDATES = ((1024, 0, 0), (1024, 0, 26), (1024, 0, 13), (2048, 0, 0), (2048, 1, 0),
                      (4096, 0, 0))


def _cache_path() -> str:
    return os.environ.get("FDAS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "fdas_gb300",
                                       "autotune.json"))


def _key(ns, M, zmin, zmax, zstep, interbin, candidates) -> str:
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    sizes = np.unique(np.asarray(ns, np.int64), return_counts=True)
    blob = json.dumps([name, [int(x) for x in sizes[0]], [int(x) for x in sizes[1]], M, zmin,
                       zmax, zstep, interbin, [list(c) for c in candidates]])
    return hashlib.sha256(blob.encode()).hexdigest()[:24]


def autotune(ns_probe, M: int, zmin: int, zmax: int, zstep: int, interbin: int = 1,
             candidates=DEFAULT_CANDIDATES, reps: int = 3, use_cache: bool = True,
             cache_path: str | None = None, device="cuda"):
    """Return {"L": ..., "ctas_per_sm": ..., "templates_per_block": ..., "ms": {...}} for the
    fastest candidate; candidates are (L, ctas_per_sm) or (L, ctas_per_sm, templates_per_block)."""
    path = cache_path or _cache_path()
    key = _key(ns_probe, M, zmin, zmax, zstep, interbin, candidates)
    if use_cache and os.path.exists(path):
        try:
            with open(path) as fh:
                hit = json.load(fh).get(key)
            if hit:
                return hit
        except (OSError, ValueError):
            pass
    rng = np.random.default_rng(0)
    timings = {}
    for cand in candidates:
        L, cps = int(cand[0]), int(cand[1])
        tpb = int(cand[2]) if len(cand) > 2 else 0
        if 2 * ((abs(zmax) + 1) // 2 + 8) > M - 2 or M > L // 2:
            continue
        bs = BatchSearch(ns_probe, L, M, zmin, zmax, zstep, interbin=interbin,
                         ctas_per_sm=cps, templates_per_block=tpb, pool_bytes=1 << 62,
                         device=device)
        spec = (rng.standard_normal(bs.spec.numel()) + 1j * rng.standard_normal(bs.spec.numel()))
        bs.spec.copy_(torch.from_numpy((spec / np.sqrt(2)).astype(np.complex64)))
        torch.cuda.synchronize()
        fdas_make_templates(bs.p, bs.bank)
        bs.correlate_wave(0)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        best = float("inf")
        for _ in range(reps):
            ev[0].record()
            for k in range(len(bs.waves)):
                bs.correlate_wave(k)
            ev[1].record()
            torch.cuda.synchronize()
            best = min(best, ev[0].elapsed_time(ev[1]))
        timings["%d/%d/%d" % (L, cps, tpb)] = best
        del bs
        torch.cuda.empty_cache()
    choice = min(timings, key=timings.get)
    L, cps, tpb = (int(x) for x in choice.split("/"))
    res = {"L": L, "ctas_per_sm": cps, "templates_per_block": tpb, "ms": timings}
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            data = {}
            if os.path.exists(path):
                with open(path) as fh:
                    data = json.load(fh)
            data[key] = res
            with open(path, "w") as fh:
                json.dump(data, fh, indent=1)
        except (OSError, ValueError):
            pass
    return res
