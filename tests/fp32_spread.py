"""Tracking parity bars derived from FP32 restatements of the oracle (test helper).

Gauss-Newton tracking with a stopping rule, an iteration cap and lost-point tests
is a discontinuous function of its rounding: an FP32 implementation that takes
exactly the oracle's steps still ends some trajectories in another state than
FP64 does (another basin, TRACKED vs MAXITER at the cap, OOB vs SINGULAR), and a
point that hits the iteration cap stops wherever its last step left it. How often
that happens depends on the workload, so the bars are not fixed percentages: they
are measured on every call from an ensemble of FP32 restatements of the oracle
(oracle/degraf_oracle.c compiled with the tracking iteration in FP32) run on the
same inputs, the key-points unmoved and moved by one FP32 ulp in each of the eight
directions (nine members; an FP32 implementation cannot tell these inputs apart).

A tracked result is compared with the FP64 oracle in three categories:
  status  - the final status differs;
  tracked - both TRACKED and the endpoints differ by more than 1e-2 px;
  maxiter - both MAXITER (tracked, but stopped by the cap) and the endpoints differ
            by more than 1e-2 px.
The GPU passes when, in each category, its count is at most the largest count of
the ensemble times 1.1 (another summation order and solver; the ensemble's own
counts spread by a few percent) plus three standard deviations of a Poisson count
plus 3; when its disagreements are the rounding-sensitive points: at least 85%
of them (once there are 20 or more) lie in the union of the ensemble's
disagreements; and when the bulk of its tracked points is as close to FP64 as the
FP32 restatement's: the median and the 90th percentile of the endpoint difference
over the points TRACKED on both sides at most 1.5 times those of the restatement on
the unmoved key-points (plus 1e-6 px; the moved members track slightly different
points, whose true flows differ by the flow field's slope times an ulp), once 100
or more points are compared.
A mistake that moves points by more than 1e-2 px, moves a different set of points,
or shifts the bulk by more than rounding does, fails one of the three.
"""
from __future__ import annotations

import dataclasses

import numpy as np

import oracle

TOL_FLOW = 1e-2
CATEGORIES = ("status", "tracked", "maxiter")
PERCENTILES = (50, 90)
MIN_FOR_QUANTILES = 100  # points compared before the bulk bar applies


def disagreements(flow, status, flow64, status64, tol: float = TOL_FLOW) -> dict:
    """Masks of the three categories of disagreement with the FP64 result."""
    e = np.hypot(*(np.asarray(flow, np.float64) - flow64).T)
    same = status == status64
    far = same & (e > tol)
    return {"status": ~same, "tracked": far & (status == oracle.TRACKED),
            "maxiter": far & (status == oracle.MAXITER)}


def ulp_neighbours(pts32: np.ndarray):
    """The key-points and their eight one-ulp FP32 neighbours (as float64 arrays)."""
    out = []
    for dx in (0, 1, -1):
        for dy in (0, 1, -1):
            q = pts32.copy()
            if dx:
                q[:, 0] = np.nextafter(q[:, 0], np.float32(np.inf * dx))
            if dy:
                q[:, 1] = np.nextafter(q[:, 1], np.float32(np.inf * dy))
            out.append(q.astype(np.float64))
    return out


@dataclasses.dataclass
class Spread:
    """FP64 reference and the FP32 ensemble's disagreements with it."""
    flow64: np.ndarray
    status64: np.ndarray
    counts: dict        # category -> per-member counts
    union: np.ndarray   # points where any member disagrees in any category
    quantiles: dict     # percentile (50, 90) -> endpoint difference on tracked points, unmoved member

    def bound(self, cat: str) -> float:
        m = max(self.counts[cat])
        return 1.1 * m + 3.0 * np.sqrt(m) + 3.0


def spread(track, pts: np.ndarray) -> Spread:
    """track(pts64, precision) -> (flow, status, ...) runs the oracle (FP64 or the FP32
    restatement) on the key-points pts; returns the FP64 result and the spread."""
    pts32 = np.asarray(pts, np.float32)
    r64 = track(pts32.astype(np.float64), "f64")
    f64, s64 = r64[0], r64[1]
    counts = {c: [] for c in CATEGORIES}
    quantiles = {}
    union = np.zeros(len(pts32), bool)
    for k, q in enumerate(ulp_neighbours(pts32)):
        r = track(q, "f32")
        d = disagreements(r[0], r[1], f64, s64)
        for c in CATEGORIES:
            counts[c].append(int(d[c].sum()))
            union |= d[c]
        if k == 0:  # the unmoved key-points
            quantiles = tracked_quantiles(r[0], r[1], f64, s64)
    return Spread(f64, s64, counts, union, quantiles)


def tracked_quantiles(flow, status, flow64, status64) -> dict:
    """Percentiles of the endpoint difference over the points TRACKED on both sides."""
    both = (status == oracle.TRACKED) & (status64 == oracle.TRACKED)
    if not both.any():
        return {p: 0.0 for p in PERCENTILES}
    e = np.hypot(*(np.asarray(flow, np.float64) - flow64).T)[both]
    return {p: float(np.percentile(e, p)) for p in PERCENTILES}


def check(flow, status, sp: Spread, label: str = "") -> dict:
    """Assert the bars for a result (flow, status) against its spread; returns the
    figures (also printed)."""
    d = disagreements(flow, status, sp.flow64, sp.status64)
    got = {c: int(d[c].sum()) for c in CATEGORIES}
    anyd = d["status"] | d["tracked"] | d["maxiter"]
    n_out = int(anyd.sum())
    explained = int((anyd & sp.union).sum())
    both = (status == oracle.TRACKED) & (sp.status64 == oracle.TRACKED)
    e = np.hypot(*(np.asarray(flow, np.float64) - sp.flow64).T)
    qs = tracked_quantiles(flow, status, sp.flow64, sp.status64)
    fig = {"n": len(status), "counts": got, "bounds": {c: round(float(sp.bound(c)), 1) for c in CATEGORIES},
           "ensemble": sp.counts, "outliers": n_out, "explained": explained,
           "within_tracked": float(np.mean(e[both] <= TOL_FLOW)) if both.any() else 1.0,
           "quantiles": {p: float(f"{v:.3g}") for p, v in qs.items()},
           "fp32_quantiles": {p: float(f"{v:.3g}") for p, v in sp.quantiles.items()}}
    print(f"{label}: {fig}")
    if both.sum() >= MIN_FOR_QUANTILES:  # a few points' percentiles are single FP32 roundings
        for p in PERCENTILES:
            lim = 1.5 * sp.quantiles[p] + 1e-6
            assert qs[p] <= lim, f"{label}: percentile {p} of the tracked endpoint difference {qs[p]:.3g} above {lim:.3g}"
    for c in CATEGORIES:
        assert got[c] <= sp.bound(c), f"{label}: {c} disagreements {got[c]} above the FP32 bound {sp.bound(c):.1f}"
    if n_out >= 20:
        assert explained >= 0.85 * n_out, f"{label}: only {explained} of {n_out} disagreements are rounding-sensitive"
    else:
        assert n_out - explained <= 3, f"{label}: {n_out - explained} disagreements outside the FP32 ensemble's"
    return fig


def frames_spread(I1, I2, pts, prm: oracle.RlofParams, init_flow=None, nthreads: int = 0) -> Spread:
    """spread() for plain tracking of frames I1 -> I2 (optionally from a prior flow)."""
    def track(q, precision):
        return oracle.rlof_track(I1, I2, q, prm, nthreads, init_flow=init_flow, precision=precision)
    return spread(track, pts)


def pyramids_spread(pyr1, pyr2, W, H, pts, prm: oracle.RlofParams, nthreads: int = 0) -> Spread:
    """spread() for tracking on given pyramid buffers (e.g. rounded to FP16)."""
    def track(q, precision):
        return oracle.rlof_track_on_pyramids(pyr1, pyr2, W, H, q, prm, nthreads, precision=precision)
    return spread(track, pts)


def fp16_pyramid(img, levels: int) -> np.ndarray:
    """The oracle's pyramid buffer with every value rounded to FP16 (round to nearest
    even), the values an FP16-storage pyramid holds."""
    return oracle.pyramid_buffer(img, levels).astype(np.float16).astype(np.float64)


# ------------------------------------------------ forward-backward filter

FB_CATEGORIES = ("status", "error")


@dataclasses.dataclass
class FbSpread:
    """FP64 forward-backward result and the FP32 ensemble's disagreements with it."""
    status64: np.ndarray
    err64: np.ndarray
    counts: dict
    union: np.ndarray
    quantiles: dict

    def bound(self, cat: str) -> float:
        m = max(self.counts[cat])
        return 1.1 * m + 3.0 * np.sqrt(m) + 3.0


def fb_disagreements(status, err, status64, err64) -> dict:
    """status: the final status (with FB_REJECTED) differs; error: both round-trip
    errors finite and more than twice the flow tolerance apart."""
    fin = np.isfinite(err) & np.isfinite(err64)
    d = np.zeros(len(err64))
    d[fin] = np.abs(np.asarray(err, np.float64)[fin] - err64[fin])
    return {"status": status != status64, "error": fin & (d > 2 * TOL_FLOW)}


def _fb_quantiles(err, err64) -> dict:
    fin = np.isfinite(err) & np.isfinite(err64)
    if not fin.any():
        return {p: 0.0 for p in PERCENTILES}
    d = np.abs(np.asarray(err, np.float64)[fin] - err64[fin])
    return {p: float(np.percentile(d, p)) for p in PERCENTILES}


def fb_spread(I1, I2, pts, prm: oracle.RlofParams, fb_max: float, nthreads: int = 0) -> FbSpread:
    """The oracle's forward-backward filter in FP64 and its FP32 ensemble."""
    pts32 = np.asarray(pts, np.float32)
    _, s64, e64 = oracle.rlof_track_fb(I1, I2, pts32.astype(np.float64), prm, fb_max, nthreads)
    counts = {c: [] for c in FB_CATEGORIES}
    union = np.zeros(len(pts32), bool)
    quantiles = {}
    for k, q in enumerate(ulp_neighbours(pts32)):
        _, s, e = oracle.rlof_track_fb(I1, I2, q, prm, fb_max, nthreads, precision="f32")
        d = fb_disagreements(s, e, s64, e64)
        for c in FB_CATEGORIES:
            counts[c].append(int(d[c].sum()))
            union |= d[c]
        if k == 0:
            quantiles = _fb_quantiles(e, e64)
    return FbSpread(s64, e64, counts, union, quantiles)


def check_fb(status, err, sp: FbSpread, label: str = "") -> dict:
    """The bars of check() for the forward-backward filter's statuses and errors."""
    d = fb_disagreements(status, err, sp.status64, sp.err64)
    got = {c: int(d[c].sum()) for c in FB_CATEGORIES}
    anyd = d["status"] | d["error"]
    n_out, explained = int(anyd.sum()), int((anyd & sp.union).sum())
    qs = _fb_quantiles(err, sp.err64)
    fig = {"n": len(status), "counts": got, "bounds": {c: round(float(sp.bound(c)), 1) for c in FB_CATEGORIES},
           "ensemble": sp.counts, "outliers": n_out, "explained": explained,
           "quantiles": {p: float(f"{v:.3g}") for p, v in qs.items()},
           "fp32_quantiles": {p: float(f"{v:.3g}") for p, v in sp.quantiles.items()}}
    print(f"{label}: {fig}")
    fin = int((np.isfinite(err) & np.isfinite(sp.err64)).sum())
    if fin >= MIN_FOR_QUANTILES:
        for p in PERCENTILES:
            lim = 1.5 * sp.quantiles[p] + 1e-6
            assert qs[p] <= lim, f"{label}: percentile {p} of the round-trip error difference {qs[p]:.3g} above {lim:.3g}"
    for c in FB_CATEGORIES:
        assert got[c] <= sp.bound(c), f"{label}: {c} disagreements {got[c]} above the FP32 bound {sp.bound(c):.1f}"
    if n_out >= 20:
        assert explained >= 0.85 * n_out, f"{label}: only {explained} of {n_out} disagreements are rounding-sensitive"
    else:
        assert n_out - explained <= 3, f"{label}: {n_out - explained} disagreements outside the FP32 ensemble's"
    return fig
