"""Autotuner for the mixed form: supercell shape x threads per supercell.

The push kernel's speed depends on the supercell edge (tile reuse, frame
length, shared memory per CTA, hence CTAs per SM) and on the threads per
supercell, in a way that depends on the particles per cell and the shape.
The tuner times each supported candidate on a sample of the workload
(push + frame maintenance, CUDA events inside the step graph, after warm-up)
and caches the winner per (workload signature, GPU name, library build).

    best = autotune.tune(make_ctx, candidates, steps=5)   # make_ctx(sc, threads) -> loaded Context
"""
from __future__ import annotations

import hashlib
import json
import os
import time
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_CACHE = os.path.join(HERE, "_build", "autotune_cache.json")

# (supercell edges, threads per supercell) the library instantiates
CANDIDATES = [((4, 4, 4), 128), ((4, 4, 4), 256), ((8, 4, 4), 128), ((8, 4, 4), 256),
              ((8, 8, 4), 128), ((8, 8, 4), 256), ((8, 8, 8), 256)]


@dataclass
class Trial:
    sc: tuple
    threads: int
    ms_per_step: float  # push + frame maintenance
    ok: bool = True
    error: str = ""


def feasible(candidates, grids):
    """Candidates whose supercell edges divide every box."""
    out = []
    for sc, t in candidates:
        if all(g[0] % sc[0] == 0 and g[1] % sc[1] == 0 and g[2] % sc[2] == 0 for g in grids):
            out.append((tuple(sc), int(t)))
    return out


def signature(grids, ppc, shapes, nspecies, extra=""):
    """Key of a tuning result: box sizes, mean particles per cell, shapes."""
    g = sorted(tuple(int(v) for v in b) for b in grids)
    text = json.dumps([g[:16], len(g), round(float(ppc), 1), list(shapes), int(nspecies), extra])
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def library_tag():
    lib = os.path.join(HERE, "_build", "libpic.so")
    try:
        st = os.stat(lib)
        return f"{int(st.st_mtime)}-{st.st_size}"
    except OSError:
        return "none"


def load_cache(path=DEFAULT_CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache, path=DEFAULT_CACHE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(trials):
    good = [t for t in trials if t.ok]
    if not good:
        raise RuntimeError("autotune: no candidate ran: " + "; ".join(t.error for t in trials))
    return min(good, key=lambda t: t.ms_per_step)


def time_candidate(make_ctx, sc, threads, steps, warmup):
    """Build a context for (sc, threads), warm up, and time `steps` steps of
    push + frame maintenance with the library's in-graph stage events."""
    ctx = make_ctx(sc, threads)
    try:
        ctx.step(warmup)
        ctx.stage_timing(True)
        ctx.step(steps)
        ms, n = ctx.stage_times()
        return (ms[0] + ms[1]) / max(n, 1)
    finally:
        ctx.close()


def tune(make_ctx, candidates, key=None, steps=5, warmup=2, cache_path=DEFAULT_CACHE, gpu_name=None,
         timer=time_candidate, log=None):
    """Return (sc, threads, trials) of the fastest candidate; results are cached
    under key (+ GPU name + library build) when key is given."""
    full_key = None
    if key is not None:
        full_key = f"{key}|{gpu_name or ''}|{library_tag()}"
        hit = load_cache(cache_path).get(full_key)
        if hit:
            return tuple(hit["sc"]), int(hit["threads"]), []
    trials = []
    for sc, t in candidates:
        t0 = time.perf_counter()
        try:
            ms = timer(make_ctx, sc, t, steps, warmup)
            trials.append(Trial(tuple(sc), t, float(ms)))
        except Exception as e:  # noqa: BLE001 - a candidate that cannot run is skipped
            trials.append(Trial(tuple(sc), t, float("inf"), ok=False, error=str(e)))
        if log:
            log(f"autotune {sc} x {t}: {trials[-1].ms_per_step:.3f} ms/step "
                f"({time.perf_counter() - t0:.1f} s)")
    best = pick(trials)
    if full_key is not None:
        cache = load_cache(cache_path)
        cache[full_key] = {"sc": list(best.sc), "threads": best.threads, "ms": best.ms_per_step,
                           "trials": [[list(t.sc), t.threads, t.ms_per_step] for t in trials if t.ok]}
        save_cache(cache, cache_path)
    return best.sc, best.threads, trials
