"""Launch-shape autotuner for the persistent walk kernel.

The walk's results do not depend on the launch shape (integer tallies,
counter-based random numbers), so the shape is a pure speed choice: threads
per block, paths per work unit and the regroup threshold (idle lanes that
trigger a refill).  The tuner times candidate shapes on a sample of the batch
with CUDA events and keeps the fastest; winners are cached in a JSON file
keyed by GPU name and a description of the workload.
"""
import hashlib
import json
import os
import time
from dataclasses import replace
from typing import Optional

import torch

from . import api

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "sss_b300_autotune.json")
# Around the shapes sweeps on the 81-band spectral field found best (256
# threads, 512- or 1024-path units, refill at 6-8 idle lanes; the built-in
# default is 256 / 1024 / 8).
CANDIDATES = [
    dict(block_threads=bt, unit_paths=up, regroup=rg)
    for bt in (256, 128)
    for up in (1024, 512, 2048)
    for rg in (8, 6, 5, 10)
]


def _key(m: api.Media, o: api.WalkOptions) -> str:
    desc = dict(gpu=torch.cuda.get_device_name(m.alpha.device), K=m.K,
                uneven=m.n_paths is not None, uniform_paths=m.uniform_paths,
                slab=m.thickness_mm is not None, n_rel=round(m.n_rel, 4), nbins=o.nbins,
                mode=o.mode, sumsq=o.want_sumsq)
    return hashlib.sha1(json.dumps(desc, sort_keys=True).encode()).hexdigest()[:16]


def _sample(m: api.Media, max_inst: int) -> api.Media:
    if m.n_inst <= max_inst:
        return m
    idx = torch.linspace(0, m.n_inst - 1, max_inst, device=m.alpha.device).long()
    pick = lambda t: t[:, idx].contiguous()
    return api.Media(pick(m.alpha), pick(m.sigma_t), pick(m.g), pick(m.w),
                     None if m.n_paths is None else m.n_paths[idx].contiguous(),
                     m.uniform_paths,
                     None if m.thickness_mm is None else m.thickness_mm[idx].contiguous(),
                     m.n_rel)


def _time(m: api.Media, o: api.WalkOptions, reps: int) -> float:
    ws = api.alloc_workspace(m, o)
    out = api.alloc_tallies(m, o)
    api.walk(m, o, workspace=ws, out=out)   # warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        api.walk(m, o, workspace=ws, out=out)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune(m: api.Media, o: api.WalkOptions, max_inst: int = 1 << 17, reps: int = 3,
         cache_path: Optional[str] = DEFAULT_CACHE, candidates=CANDIDATES) -> api.WalkOptions:
    """Returns `o` with the fastest launch shape for this workload."""
    key = _key(m, o)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        return replace(o, **cache[key]["shape"])
    sm = _sample(m, max_inst)
    results = []
    for cand in candidates:
        oc = replace(o, **cand)
        results.append((_time(sm, oc, reps), cand))
    results.sort(key=lambda r: r[0])
    best_ms, best = results[0]
    cache[key] = {"shape": best, "ms": best_ms, "when": time.time(),
                  "all": [(ms, c) for ms, c in results]}
    if cache_path:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return replace(o, **best)
