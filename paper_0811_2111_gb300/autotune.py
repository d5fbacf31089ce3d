"""Work-plan autotuner of the batched engine, with an on-disk cache.

The batched kernel cuts every lattice into bands of rows, one CTA per band
(about `target_band_sites` sites each, clusters of 8 CTAs).  The best band
size depends on the mix of lattice sides and on the GPU, so this module times
a few candidate plans on a throw-away batch of the same shape and caches the
winner per (GPU, lattice sides, sweeps per round, precision).  The plan never
changes results: a lattice evolves bit-identically under every plan.

Cache file: $XY_GB300_AUTOTUNE_CACHE, else ~/.cache/xy_gb300/autotune.json.
"""
import hashlib
import json
import os

CANDIDATES = (1024, 2048, 4096, 8192, 16384)


def cache_path():
    p = os.environ.get("XY_GB300_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "xy_gb300", "autotune.json")


def _key(device_name, Ls, sweeps_per_round, sincos):
    h = hashlib.sha1(",".join(str(int(v)) for v in sorted(Ls)).encode()).hexdigest()[:16]
    return f"{device_name}|{h}|n{len(Ls)}|spr{sweeps_per_round}|{sincos}"


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass          # a read-only home only costs a re-tune next time


def tune_batch(Ls, betas, ladders=None, sweeps_per_round=10, sincos="accurate", rounds=6,
               candidates=CANDIDATES, device=None, use_cache=True):
    """Best target_band_sites for this batch shape (timed, then cached)."""
    import torch
    from .lattice import Batch

    dev = torch.device(device if device is not None else "cuda")
    name = torch.cuda.get_device_name(dev)
    key = _key(name, Ls, sweeps_per_round, sincos)
    cache = _load() if use_cache else {}
    if key in cache:
        return int(cache[key]["target_band_sites"])
    times = {}
    for target in candidates:
        with Batch(Ls, betas, seed=0x5EED, ladders=ladders, sweeps_per_round=sweeps_per_round,
                   sincos=sincos, target_band_sites=target, device=dev) as b:
            b.reserve(rounds + 2)
            b.run(2)                                      # warm-up (graph capture, caches)
            s = b.stream
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            b.run(rounds)
            e1.record(s)
            e1.synchronize()
            times[target] = e0.elapsed_time(e1) / rounds
    best = min(times, key=times.get)
    if use_cache:
        cache[key] = {"target_band_sites": best, "ms_per_round": times}
        _store(cache)
    return best
