"""Autotuner of the tracking launch shape (lanes per point) for a batch of pairs.

The library picks 8 lanes per point at radius 4 and 5, the fastest shape on the
single-pair and mixed-batch workloads. A batch of other sizes,
steps or parameters may prefer another shape, so ``tune`` times rlof_track_many
on the caller's frames for every lane count the library honours at the batch's
radius, keeps the fastest, and records it in a JSON cache keyed by the GPU, the
tracking parameters and the batch's size class (its point count rounded to a
power of two). ``BatchTracker(..., lanes="auto")`` looks the choice up;
``BatchTracker.autotune`` tunes and applies it.
"""
from __future__ import annotations

import json
import math
import os
import tempfile

CACHE_VERSION = 1


def candidates(radius: int) -> tuple:
    """Lane counts the library honours at this radius (8 and 16 only with the
    compile-time layouts of radius 4 and 5)."""
    return (8, 16, 32) if radius in (4, 5) else (32,)


def cache_file() -> str:
    return os.environ.get("DGF_TUNE_CACHE") or os.path.join(
        os.path.expanduser("~"), ".cache", "paper_1901_09971_gb300", "tune.json")


def size_class(n_points: int) -> int:
    return int(round(math.log2(max(1, int(n_points)))))


def key(gpu: str, params, n_points: int) -> str:
    """Cache key: GPU name, the parameters that shape the kernel's work, size class."""
    return (f"{gpu}|r{params.radius}|L{params.levels}|it{params.max_iter}|m{params.model}|s{params.storage}"
            f"|cross{int(params.cross_tau > 0)}|pts2^{size_class(n_points)}")


def load_cache(path: str | None = None) -> dict:
    path = path or cache_file()
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    if not isinstance(data, dict) or data.get("version") != CACHE_VERSION:
        return {}
    entries = data.get("entries")
    return entries if isinstance(entries, dict) else {}


def save_cache(entries: dict, path: str | None = None) -> None:
    """Writes the cache atomically (a temporary file renamed over the old one)."""
    path = path or cache_file()
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump({"version": CACHE_VERSION, "entries": entries}, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(k: str, path: str | None = None) -> int | None:
    rec = load_cache(path).get(k)
    if isinstance(rec, dict) and rec.get("lanes") in (8, 16, 32):
        return int(rec["lanes"])
    return None


def choose(timings: dict) -> int:
    """The fastest lane count (ties go to the smaller count)."""
    return min(sorted(timings), key=lambda lanes: timings[lanes])


def tune(measure, radius: int, k: str, path: str | None = None) -> dict:
    """Times every candidate with ``measure(lanes) -> ms``, records the fastest under
    key ``k`` and returns the record {"lanes", "ms"}."""
    timings = {lanes: float(measure(lanes)) for lanes in candidates(radius)}
    rec = {"lanes": choose(timings), "ms": {str(lanes): t for lanes, t in timings.items()}}
    entries = load_cache(path)
    entries[k] = rec
    save_cache(entries, path)
    return rec
