"""Work-plan autotuner of the sweep engines, with an on-disk cache.

A plan never changes results: every plan gives the same angles, accept
counts and (exact) record sums, bit for bit (tested).  It only changes how
the work is cut and scheduled, and the best cut depends on the lattice
sizes and on the GPU, so this module times the candidate plans on a
throw-away copy of the workload and caches the fastest per (GPU, library
version, workload shape, precision).

Single lattices (``tune_lattice``; xy_params): the algorithm (all sweeps of
a call in one persistent launch, one launch per sweep, or two sweeps per
launch with temporal blocking) and the tile kernel's CTAs per SM (3 at up to
80 registers a thread, 4 at up to 64: more warps, or 2 at up to 128: more
independent work in flight per warp, fewer warps).

Batches (``tune_batch``; xy_batch_params): the CTAs per grouped tile launch
(lattices of one side are launched in groups, one graph branch each, so
that the groups' sweeps overlap), the grouped tile kernel's CTAs per SM, and
(only where banded lattices exist) the band size of the cluster kernel.

Cache file: $XY_GB300_AUTOTUNE_CACHE, else ~/.cache/xy_gb300/autotune.json.
"""
import hashlib
import json
import os

LATTICE_CANDIDATES = (("persistent", 3), ("persistent", 4), ("persistent", 2), ("fused", 3),
                      ("fused", 4), ("fused", 2), ("fused2", 3))
GROUP_CTAS = (64, 128, 256, 512)
BATCH_CTAS_PER_SM = (3, 4, 2)
BAND_TARGETS = (2048, 8192)


def cache_path():
    p = os.environ.get("XY_GB300_AUTOTUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "xy_gb300", "autotune.json")


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


def _device_key(dev):
    import torch
    from . import _lib as X
    return f"{torch.cuda.get_device_name(dev)}|v{X.xy_version()}"


def _events(stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    return e0, e1


def tune_lattice(L, beta=1.1, sincos="accurate", sweeps=100, repeats=3, device=None,
                 use_cache=True, candidates=LATTICE_CANDIDATES):
    """Fastest (algorithm, ctas_per_sm) for sweeping one L x L lattice.

    Returns dict(algorithm, ctas_per_sm, ms_per_sweep: {"algorithm/ctas": ms}).
    Lattices whose side the fused kernels do not take (L % 128 != 0) have one
    plan, the two-pass kernels."""
    import torch
    from .lattice import Lattice

    if L % 128 != 0:
        return {"algorithm": "two_pass", "ctas_per_sm": 0, "ms_per_sweep": {}}
    dev = torch.device(device if device is not None else "cuda")
    key = f"lattice|{_device_key(dev)}|L{L}|{sincos}|" + ",".join(f"{a}/{c}" for a, c in candidates)
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]
    times = {}
    for algorithm, ctas in candidates:
        with Lattice(L, beta, 0x5EED, sincos=sincos, algorithm=algorithm, ctas_per_sm=ctas,
                     device=dev) as lat:
            lat.reserve(sweeps * (repeats + 1) + 10)
            lat.sweep(10)                                  # warm-up (attributes, caches)
            best = None
            for _ in range(repeats):
                e0, e1 = _events(lat.stream)
                e0.record(lat.stream)
                lat.sweep(sweeps)
                e1.record(lat.stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1) / sweeps
                best = ms if best is None else min(best, ms)
        times[f"{algorithm}/{ctas}"] = best
    win = min(times, key=times.get)
    algorithm, ctas = win.split("/")
    result = {"algorithm": algorithm, "ctas_per_sm": int(ctas), "ms_per_sweep": times}
    if use_cache:
        cache[key] = result
        _store(cache)
    return result


def tune_batch(Ls, betas, ladders=None, sweeps_per_round=10, sincos="accurate", rounds=6,
               device=None, use_cache=True, group_ctas=GROUP_CTAS,
               ctas_per_sm=BATCH_CTAS_PER_SM, band_targets=BAND_TARGETS):
    """Fastest batch work plan for this batch shape (timed, then cached).

    Returns dict(group_ctas, ctas_per_sm, target_band_sites,
    ms_per_round: {"group/ctas/target": ms})."""
    import torch
    from .lattice import Batch

    dev = torch.device(device if device is not None else "cuda")
    # band sizes only matter where the plan has banded lattices (sides the tile
    # kernels and the whole-lattice kernel do not take)
    banded = any(not (L % 32 == 0 or L * L * 12 <= 112 * 1024) for L in Ls)
    targets = band_targets if banded else (8192,)
    cands = [(g, c, t) for g in group_ctas for c in ctas_per_sm for t in targets]
    h = hashlib.sha1(",".join(str(int(v)) for v in sorted(Ls)).encode()).hexdigest()[:16]
    key = (f"batch|{_device_key(dev)}|{h}|n{len(Ls)}|spr{sweeps_per_round}|{sincos}|"
           + ",".join("/".join(map(str, c)) for c in cands))
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]
    times = {}
    for g, c, t in cands:
        with Batch(Ls, betas, seed=0x5EED, ladders=ladders, sweeps_per_round=sweeps_per_round,
                   sincos=sincos, target_band_sites=t, group_ctas=g, ctas_per_sm=c,
                   device=dev) as b:
            b.reserve(rounds + 2)
            b.run(2)                                      # warm-up (graph capture, caches)
            e0, e1 = _events(b.stream)
            e0.record(b.stream)
            b.run(rounds)
            e1.record(b.stream)
            e1.synchronize()
            times[f"{g}/{c}/{t}"] = e0.elapsed_time(e1) / rounds
    win = min(times, key=times.get)
    g, c, t = (int(v) for v in win.split("/"))
    result = {"group_ctas": g, "ctas_per_sm": c, "target_band_sites": t, "ms_per_round": times}
    if use_cache:
        cache[key] = result
        _store(cache)
    return result
