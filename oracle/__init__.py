"""FP64 CPU oracle of DeGraF detection, RLOF tracking and EPIC interpolation (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the benchmark's
CPU-baseline leg may use this module; the CUDA product path never imports it.
The arithmetic lives in ``degraf_oracle.c``; this wrapper marshals arrays, except for
three compositions written here in a few numpy lines each: the forward-backward round
trip (``rlof_track_fb``), the global-motion prior's initial flow (``gm_prior_flow``)
and the two-pass sequence of ``rlof_track_gm``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "degraf_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
# The same source with the tracking iteration in FP32 (-DORACLE_REAL=float): a
# measuring device for the GPU parity bars, never a reference value; "f32fma" also
# lets the compiler fuse multiply-adds (another FP32 rounding pattern).
_VARIANTS = {"f64": ("liboracle.so", []),
             "f32": ("liboracle_f32.so", ["-DORACLE_REAL=float"]),
             "f32fma": ("liboracle_f32fma.so", ["-DORACLE_REAL=float", "-ffp-contract=fast"])}

TRACKED, OOB, SMALL_EIG, SINGULAR, MAXITER = 0, 1, 2, 3, 4


def build(force: bool = False, precision: str = "f64") -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction, so x86 and Arm
    hosts give the same bits). precision "f64" is the oracle; "f32" compiles the
    same source with the tracking iteration in FP32 and "f32fma" does so with fused
    multiply-adds (test infrastructure that measures what FP32 rounding alone does
    to the iteration)."""
    if precision not in _VARIANTS:
        raise ValueError(precision)
    name, extra = _VARIANTS[precision]
    out = os.path.join(_LIBDIR, name)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    if precision == "f32fma" and platform.machine() in ("x86_64", "AMD64"):
        extra = extra + ["-mfma"]  # FMA is part of the base instruction set on Arm
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-fno-fast-math", *extra, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, out)
    return out


class _RlofParams(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("radius", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("model", ctypes.c_int), ("eps", ctypes.c_double), ("hampel_a", ctypes.c_double),
                ("hampel_b", ctypes.c_double), ("hampel_c", ctypes.c_double),
                ("min_eig", ctypes.c_double), ("cross_tau", ctypes.c_double)]


@dataclasses.dataclass
class RlofParams:
    levels: int = 3
    radius: int = 4
    max_iter: int = 30
    model: int = 4
    eps: float = 1e-3
    hampel_a: float = 8.0
    hampel_b: float = 16.0
    hampel_c: float = 32.0
    min_eig: float = 1e-3
    cross_tau: float = 0.0  # adaptive cross-based support threshold; 0: square support

    def _c(self) -> _RlofParams:
        return _RlofParams(self.levels, self.radius, self.max_iter, self.model, self.eps,
                           self.hampel_a, self.hampel_b, self.hampel_c, self.min_eig, self.cross_tau)


_libs: dict = {}


def lib(precision: str = "f64"):
    _lib = _libs.get(precision)
    if _lib is None:
        _lib = ctypes.CDLL(build(precision=precision))
        _libs[precision] = _lib
        P, I, L, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
        _lib.oracle_degraf_count.argtypes = [I, I, I, I, I]
        _lib.oracle_degraf_count.restype = L
        _lib.oracle_degraf_detect.argtypes = [P, I, I, I, I, I, I, P, P, P]
        _lib.oracle_degraf_detect.restype = I
        _lib.oracle_pyramid_size.argtypes = [I, I, I]
        _lib.oracle_pyramid_size.restype = L
        _lib.oracle_pyramid.argtypes = [P, I, I, I, P]
        _lib.oracle_pyramid.restype = I
        _lib.oracle_hampel_psi.argtypes = [D, D, D, D]
        _lib.oracle_hampel_psi.restype = D
        _lib.oracle_rlof_track.argtypes = [P, P, I, I, P, I, ctypes.POINTER(_RlofParams), P, P, P,
                                           P, I]
        _lib.oracle_rlof_track.restype = I
        _lib.oracle_degraf_detect_f64.argtypes = [P, I, I, I, I, I, P]
        _lib.oracle_degraf_detect_f64.restype = I
        _lib.oracle_degraf_vjp.argtypes = [P, I, I, I, I, I, P, P]
        _lib.oracle_degraf_vjp.restype = I
        _lib.oracle_rlof_vjp.argtypes = [P, P, I, I, P, I, ctypes.POINTER(_RlofParams), P, P, P, P, P, P, P]
        _lib.oracle_rlof_vjp.restype = I
        _lib.oracle_rlof_track_init.argtypes = [P, P, I, I, P, I, ctypes.POINTER(_RlofParams), P, P, P, P,
                                                P, I]
        _lib.oracle_rlof_track_init.restype = I
        _lib.oracle_rlof_track_pyr.argtypes = [P, P, I, I, P, I, ctypes.POINTER(_RlofParams), P, P, P, P, I]
        _lib.oracle_rlof_track_pyr.restype = I
        _lib.oracle_cross_mask.argtypes = [P, I, I, D, D, I, D, P]
        _lib.oracle_cross_mask.restype = I
        _lib.oracle_gm_fit_affine.argtypes = [P, P, P, I, I, D, D, P]
        _lib.oracle_gm_fit_affine.restype = I
        _lib.oracle_epic_cost.argtypes = [P, I, I, I, I, P]
        _lib.oracle_epic_cost.restype = I
        _lib.oracle_epic_interpolate.argtypes = [P, I, I, P, P, P, I, ctypes.POINTER(_EpicParams), P, P, P, P, P,
                                                 P, P, P]
        _lib.oracle_epic_interpolate.restype = I
        _lib.oracle_max_threads.argtypes = []
        _lib.oracle_max_threads.restype = I
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def degraf_count(W: int, H: int, win_w: int, win_h: int, step: int) -> int:
    return int(lib().oracle_degraf_count(W, H, win_w, win_h, step))


def degraf_detect(img: np.ndarray, win_w: int, win_h: int | None = None, step: int = 1):
    """Key-points of a uint8 frame: (pts [N,2] f64, sums [N,7] i64, neg [N] bool).

    sums columns: S_pos, sum j I, sum i I, m, S_neg, sum j (1+m-I), sum i (1+m-I).
    """
    win_h = win_w if win_h is None else win_h
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    n = degraf_count(W, H, win_w, win_h, step)
    pts = np.zeros((n, 2), np.float64)
    sums = np.zeros((n, 7), np.int64)
    neg = np.zeros(n, np.uint8)
    rc = lib().oracle_degraf_detect(_ptr(img), W, H, W, win_w, win_h, step, _ptr(pts), _ptr(sums),
                                    _ptr(neg))
    if rc:
        raise ValueError("oracle_degraf_detect: bad arguments")
    return pts, sums, neg.astype(bool)


def level_sizes(W: int, H: int, levels: int):
    out = []
    for _ in range(levels):
        out.append((W, H))
        W, H = W // 2, H // 2
    return out


def pyramid(img: np.ndarray, levels: int):
    """[(I_l, Ix_l, Iy_l)] per level, float64 arrays [H_l, W_l]."""
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    buf = np.zeros(int(lib().oracle_pyramid_size(W, H, levels)), np.float64)
    if lib().oracle_pyramid(_ptr(img), W, H, levels, _ptr(buf)):
        raise ValueError("oracle_pyramid: bad arguments")
    out, off = [], 0
    for (Wl, Hl) in level_sizes(W, H, levels):
        n = Wl * Hl
        out.append(tuple(buf[off + i * n: off + (i + 1) * n].reshape(Hl, Wl) for i in range(3)))
        off += 3 * n
    return out


def hampel_psi(r: float, a: float, b: float, c: float) -> float:
    return float(lib().oracle_hampel_psi(r, a, b, c))


def rlof_track(I1: np.ndarray, I2: np.ndarray, pts: np.ndarray, params: RlofParams,
               nthreads: int = 0, init_flow: np.ndarray | None = None, precision: str = "f64"):
    """Track pts [n,2] from I1 to I2: (flow [n,2], status [n] u8, iters [n] i32, illum [n,2]).

    init_flow [n,2] (optional): initial level-0 flow per point (the global-motion
    prior); tracking then starts the coarsest level at init_flow / 2^(levels-1).
    precision "f32" runs the FP32 build of the same iteration (see build())."""
    I1 = np.ascontiguousarray(I1, dtype=np.float64)
    I2 = np.ascontiguousarray(I2, dtype=np.float64)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    H, W = I1.shape
    n = pts.shape[0]
    flow = np.zeros((n, 2), np.float64)
    status = np.zeros(n, np.uint8)
    iters = np.zeros(n, np.int32)
    illum = np.zeros((n, 2), np.float64)
    prm = params._c()
    init = None if init_flow is None else np.ascontiguousarray(init_flow, dtype=np.float64).reshape(n, 2)
    rc = lib(precision).oracle_rlof_track_init(_ptr(I1), _ptr(I2), W, H, _ptr(pts), n, ctypes.byref(prm),
                                      _ptr(init) if init is not None else None, _ptr(flow), _ptr(status),
                                      _ptr(iters), _ptr(illum), int(nthreads))
    if rc:
        raise ValueError("oracle_rlof_track: bad arguments")
    return flow, status, iters, illum


def pyramid_buffer(img: np.ndarray, levels: int) -> np.ndarray:
    """The pyramid of a frame as one flat float64 buffer (per level I, Ix, Iy), the
    layout rlof_track_on_pyramids reads."""
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    buf = np.zeros(int(lib().oracle_pyramid_size(W, H, levels)), np.float64)
    if lib().oracle_pyramid(_ptr(img), W, H, levels, _ptr(buf)):
        raise ValueError("oracle_pyramid: bad arguments")
    return buf


def rlof_track_on_pyramids(pyr1: np.ndarray, pyr2: np.ndarray, W: int, H: int, pts: np.ndarray,
                           params: RlofParams, nthreads: int = 0, precision: str = "f64"):
    """rlof_track on given pyramid buffers (pyramid_buffer's layout), e.g. with their
    values rounded to a storage format first: (flow, status, iters, illum)."""
    pyr1 = np.ascontiguousarray(pyr1, dtype=np.float64)
    pyr2 = np.ascontiguousarray(pyr2, dtype=np.float64)
    size = int(lib().oracle_pyramid_size(W, H, params.levels))
    if pyr1.size != size or pyr2.size != size:
        raise ValueError("pyramid buffers do not match W, H and the level count")
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    n = pts.shape[0]
    flow = np.zeros((n, 2), np.float64)
    status = np.zeros(n, np.uint8)
    iters = np.zeros(n, np.int32)
    illum = np.zeros((n, 2), np.float64)
    prm = params._c()
    rc = lib(precision).oracle_rlof_track_pyr(_ptr(pyr1), _ptr(pyr2), W, H, _ptr(pts), n, ctypes.byref(prm),
                                              _ptr(flow), _ptr(status), _ptr(iters), _ptr(illum), int(nthreads))
    if rc:
        raise ValueError("oracle_rlof_track_pyr: bad arguments")
    return flow, status, iters, illum


def gm_fit_affine(pts: np.ndarray, flow: np.ndarray, status: np.ndarray, iters: int = 8, c0: float = 32.0,
                  c_min: float = 2.0):
    """Global affine motion q = A p + t from first-pass tracks (Tukey IRLS, annealed
    threshold; see the C source). Returns (a [6] float64, made) with
    q_x = a0 x + a1 y + a2, q_y = a3 x + a4 y + a5; made is False when no estimate
    could be formed (a is then the identity motion)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    n = pts.shape[0]
    flow = np.ascontiguousarray(flow, dtype=np.float64).reshape(n, 2)
    status = np.ascontiguousarray(status, dtype=np.uint8).reshape(n)
    a = np.zeros(6, np.float64)
    rc = lib().oracle_gm_fit_affine(_ptr(pts), _ptr(flow), _ptr(status), n, int(iters), float(c0), float(c_min),
                                    _ptr(a))
    if rc < 0:
        raise ValueError("oracle_gm_fit_affine: bad arguments")
    return a, rc == 0


def rlof_track_gm(I1: np.ndarray, I2: np.ndarray, pts: np.ndarray, params: RlofParams, stride: int = 4,
                  extra_levels: int = 2, iters: int = 8, c0: float = 32.0, c_min: float = 2.0, nthreads: int = 0,
                  precision: str = "f64"):
    """Tracking with the global-motion prior (Section 3, RLOF(IM-GM); the paper
    gives no formula, so this is the reading): (1) a sparse first pass tracks
    every stride-th point with extra_levels more pyramid levels, which reaches
    large motions; (2) gm_fit_affine fits the global affine motion to its converged
    points; (3) every point is tracked with the configured levels, starting from
    the prior's flow A p + t - p. Returns (flow, status, iters, illum, a, made)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    sub = pts[::stride]
    deep = dataclasses.replace(params, levels=params.levels + extra_levels)
    fs, ss, _, _ = rlof_track(I1, I2, sub, deep, nthreads, precision=precision)
    a, made = gm_fit_affine(sub, fs, ss, iters, c0, c_min)
    flow, status, its, illum = rlof_track(I1, I2, pts, params, nthreads, init_flow=gm_prior_flow(a, pts),
                                          precision=precision)
    return flow, status, its, illum, a, made


def cross_mask(img: np.ndarray, px: float, py: float, radius: int, tau: float) -> np.ndarray:
    """The adaptive cross-based support of a point at (px, py) on img (level 0):
    uint8 [2r+1, 2r+1], 1 for kept support samples (see the C source)."""
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    side = 2 * radius + 1
    m = np.zeros((side, side), np.uint8)
    if lib().oracle_cross_mask(_ptr(img), W, H, float(px), float(py), int(radius), float(tau), _ptr(m)) < 0:
        raise ValueError("oracle_cross_mask: bad arguments")
    return m


FB_REJECTED = 5


def rlof_track_fb(I1: np.ndarray, I2: np.ndarray, pts: np.ndarray, params: RlofParams, fb_max: float = 0.0,
                  nthreads: int = 0, precision: str = "f64"):
    """Forward-backward consistency (not in the paper's text; a common filter on
    sparse tracks): points are tracked from I1 to I2 (flow f), their end points
    p + f back from I2 to I1 (flow b) with the same parameters; the round-trip error
    is |f + b| where both passes tracked the point (TRACKED or MAXITER), else +inf.
    With fb_max > 0, forward-tracked points whose error exceeds fb_max get status
    FB_REJECTED (5); their flow is kept. Returns (flow, status, fb_err)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    f, s, _, _ = rlof_track(I1, I2, pts, params, nthreads, precision=precision)
    b, sb, _, _ = rlof_track(I2, I1, pts + f, params, nthreads, precision=precision)
    fwd = (s == TRACKED) | (s == MAXITER)
    bwd = (sb == TRACKED) | (sb == MAXITER)
    err = np.where(fwd & bwd, np.hypot(*(f + b).T), np.inf)
    status = s.copy()
    if fb_max > 0:
        status[fwd & (err > fb_max)] = FB_REJECTED
    return f, status, err


def gm_prior_flow(a: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Initial level-0 flow of each point under the affine motion a: A p + t - p."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 2)
    x, y = pts[:, 0], pts[:, 1]
    return np.stack([a[0] * x + a[1] * y + a[2] - x, a[3] * x + a[4] * y + a[5] - y], 1)


def degraf_detect_f64(img: np.ndarray, win_w: int, win_h: int | None = None, step: int = 1):
    """Key-points of a real-valued image (same definition; for finite differences)."""
    win_h = win_w if win_h is None else win_h
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    pts = np.zeros((degraf_count(W, H, win_w, win_h, step), 2), np.float64)
    if lib().oracle_degraf_detect_f64(_ptr(img), W, H, win_w, win_h, step, _ptr(pts)):
        raise ValueError("oracle_degraf_detect_f64: bad arguments")
    return pts


def degraf_vjp(img: np.ndarray, win_w: int, win_h: int | None, step: int, grad_pts: np.ndarray) -> np.ndarray:
    """sum_k grad_pts[k] . d(point_k)/d(img) as an image (float64 [H, W])."""
    win_h = win_w if win_h is None else win_h
    img = np.ascontiguousarray(img, dtype=np.float64)
    H, W = img.shape
    g = np.ascontiguousarray(grad_pts, dtype=np.float64).reshape(-1, 2)
    out = np.zeros((H, W), np.float64)
    if lib().oracle_degraf_vjp(_ptr(img), W, H, win_w, win_h, step, _ptr(g), _ptr(out)):
        raise ValueError("oracle_degraf_vjp: bad arguments")
    return out


def rlof_vjp(I1, I2, pts, params: RlofParams, flow, illum, status, grad_flow, grad_illum=None):
    """Implicit-function VJP of tracking: (grad_I1, grad_I2) float64 [H, W]."""
    I1 = np.ascontiguousarray(I1, dtype=np.float64)
    I2 = np.ascontiguousarray(I2, dtype=np.float64)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    flow = np.ascontiguousarray(flow, dtype=np.float64).reshape(-1, 2)
    illum = np.ascontiguousarray(illum, dtype=np.float64).reshape(-1, 2)
    status = np.ascontiguousarray(status, dtype=np.uint8)
    gf = np.ascontiguousarray(grad_flow, dtype=np.float64).reshape(-1, 2)
    gi = None if grad_illum is None else np.ascontiguousarray(grad_illum, dtype=np.float64).reshape(-1, 2)
    H, W = I1.shape
    g1 = np.zeros((H, W), np.float64)
    g2 = np.zeros((H, W), np.float64)
    prm = params._c()
    rc = lib().oracle_rlof_vjp(_ptr(I1), _ptr(I2), W, H, _ptr(pts), pts.shape[0], ctypes.byref(prm), _ptr(flow),
                               _ptr(illum), _ptr(status), _ptr(gf), None if gi is None else _ptr(gi), _ptr(g1),
                               _ptr(g2))
    if rc:
        raise ValueError("oracle_rlof_vjp: bad arguments")
    return g1, g2


def max_threads() -> int:
    return int(lib().oracle_max_threads())


class _EpicParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("model", ctypes.c_int), ("cost_base", ctypes.c_int),
                ("cost_gain", ctypes.c_int), ("a", ctypes.c_double), ("min_spread", ctypes.c_double)]


@dataclasses.dataclass
class EpicParams:
    k: int = 128           # nearest seeds per fit (Section 3 "Parameters")
    model: int = 1         # 1: locally affine fit, 0: weighted mean
    cost_base: int = 4     # edge cost of a flat pixel
    cost_gain: int = 1     # multiplier of |Gx| + |Gy| (integer Sobel responses)
    a: float = 0.1         # kernel decay per flat pixel of geodesic travel
    min_spread: float = 1.0  # px; smallest weighted spread of the neighbours for an affine fit

    def _c(self) -> _EpicParams:
        return _EpicParams(self.k, self.model, self.cost_base, self.cost_gain, self.a, self.min_spread)


@dataclasses.dataclass
class EpicResult:
    dense: np.ndarray      # float64 [H, W, 2]
    labels: np.ndarray     # int32 [H, W], seed of each pixel, -1 where no seed exists
    dist: np.ndarray       # int64 [H, W], geodesic distance to that seed, -1 where none
    knn_idx: np.ndarray    # int32 [n, k], the neighbourhood of each seed, nearest first
    knn_dist: np.ndarray   # int64 [n, k], their seed-graph distances
    knn_count: np.ndarray  # int32 [n], neighbourhood size (0 for matches that are not seeds)
    models: np.ndarray     # float64 [n, 6], (A00, A01, A10, A11, b0, b1) per seed
    fit_kind: np.ndarray   # uint8 [n], 0 not a seed, 1 affine, 2 weighted mean


def epic_cost(img: np.ndarray, cost_base: int, cost_gain: int) -> np.ndarray:
    """Edge cost map of EPIC's geodesic distance (int64 [H, W]; see the C source)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    out = np.zeros((H, W), np.int64)
    if lib().oracle_epic_cost(_ptr(img), W, H, int(cost_base), int(cost_gain), _ptr(out)) < 0:
        raise ValueError("oracle_epic_cost: bad arguments")
    return out


def epic_interpolate(img: np.ndarray, pts: np.ndarray, flow: np.ndarray, status: np.ndarray,
                     params: EpicParams = EpicParams()) -> EpicResult:
    """Dense flow from sparse matches by edge-preserving interpolation (Section 2,
    "Interpolation"; the reading is stated in the C source)."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    H, W = img.shape
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    n = pts.shape[0]
    flow = np.ascontiguousarray(flow, dtype=np.float64).reshape(n, 2)
    status = np.ascontiguousarray(status, dtype=np.uint8).reshape(n)
    k = int(params.k)
    r = EpicResult(np.zeros((H, W, 2)), np.zeros((H, W), np.int32), np.zeros((H, W), np.int64),
                   np.full((n, k), -1, np.int32), np.full((n, k), -1, np.int64), np.zeros(n, np.int32),
                   np.zeros((n, 6)), np.zeros(n, np.uint8))
    prm = params._c()
    rc = lib().oracle_epic_interpolate(_ptr(img), W, H, _ptr(pts), _ptr(flow), _ptr(status), n,
                                       ctypes.byref(prm), _ptr(r.dense), _ptr(r.labels), _ptr(r.dist),
                                       _ptr(r.knn_idx), _ptr(r.knn_dist), _ptr(r.knn_count), _ptr(r.models),
                                       _ptr(r.fit_kind))
    if rc == -1:
        raise ValueError("oracle_epic_interpolate: bad arguments")
    if rc < 0:
        raise MemoryError("oracle_epic_interpolate: out of memory")
    return r
