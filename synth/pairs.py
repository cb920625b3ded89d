"""Synthetic grayscale frame pairs with known flow.

The paper evaluates on KITTI frame pairs (about 1242x375, Section 3). KITTI is not
available here, so seeded synthetic pairs of the same shape stand in for it:

* texture: a sum of 64 random Gaussian blobs plus 3-octave value noise (lattice
  spacings 32, 16, 8 px; cubic smoothstep interpolation; amplitudes 1, 1/2, 1/4),
  mapped affinely to [16, 240] and rounded to uint8;
* translation pairs: frame 2 is frame 1 bilinearly warped by a constant
  translation, plus N(0, 2) noise, rounded half to even and clipped to [0, 255];
  frame-2 pixels whose source lies outside frame 1 take fresh texture;
* radial pairs (driving-scene shape): radial expansion about the image centre
  reaching ``max_disp`` px at the corners, plus rigid textured rectangles with
  their own translations painted in index order; frame-2 pixels whose source is
  hidden or outside the frame take fresh texture.

Every draw comes from ``numpy.random.Generator(PCG64(seed))``. The texture is a
continuous function that is separable into per-axis factors, so grids of any
separable coordinate set (translated or radially scaled) evaluate as small
matrix products. Nothing here is part of the method under test.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import ndimage

# The four frame sizes of the mixed-size batch workload (W, H).
CONFIG_SIZES = ((640, 480), (1024, 436), (1242, 375), (1280, 720))
BATCH_STEPS = (2, 3, 4, 6)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def _lattice_weights(coords: np.ndarray, spacing: float, pad: int, n: int) -> np.ndarray:
    """[n, len(coords)] interpolation matrix of 1-D value noise with smoothstep."""
    u = coords / spacing + pad
    i = np.clip(np.floor(u).astype(np.int64), 0, n - 2)
    t = np.clip(u - i, 0.0, 1.0)
    s = t * t * (3.0 - 2.0 * t)
    w = np.zeros((n, coords.size))
    cols = np.arange(coords.size)
    w[i, cols] = 1.0 - s
    w[i + 1, cols] = s
    return w


class Texture:
    """Continuous random texture on a W x H extent (blobs + value noise)."""

    OCTAVES = ((32.0, 1.0), (16.0, 0.5), (8.0, 0.25))

    def __init__(self, rng: np.random.Generator, W: int, H: int, n_blobs: int = 64):
        self.cx = rng.uniform(0.0, W, n_blobs)
        self.cy = rng.uniform(0.0, H, n_blobs)
        self.sigma = rng.uniform(W / 64.0, W / 8.0, n_blobs)
        self.amp = rng.uniform(-1.0, 1.0, n_blobs)
        self.octaves = []
        pad = 4
        for spacing, amp in self.OCTAVES:
            nx = int(math.ceil(W / spacing)) + 2 * pad + 2
            ny = int(math.ceil(H / spacing)) + 2 * pad + 2
            self.octaves.append((spacing, amp, pad, rng.uniform(-1.0, 1.0, (ny, nx))))

    def raw(self, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
        """Texture value on the grid ys x xs (float64, unmapped)."""
        xs = np.asarray(xs, dtype=np.float64)
        ys = np.asarray(ys, dtype=np.float64)
        two_s2 = 2.0 * self.sigma[:, None] ** 2
        ex = np.exp(-((xs[None, :] - self.cx[:, None]) ** 2) / two_s2)
        ey = np.exp(-((ys[None, :] - self.cy[:, None]) ** 2) / two_s2)
        out = (ey * self.amp[:, None]).T @ ex
        for spacing, amp, pad, vals in self.octaves:
            wx = _lattice_weights(xs, spacing, pad, vals.shape[1])
            wy = _lattice_weights(ys, spacing, pad, vals.shape[0])
            out += amp * (wy.T @ vals @ wx)
        return out

    def raw_at(self, x: np.ndarray, y: np.ndarray) -> np.ndarray:
        """Texture value at the points (x[i], y[i]) (float64, unmapped); equal to
        ``raw`` on grid points up to rounding."""
        x = np.asarray(x, dtype=np.float64).ravel()
        y = np.asarray(y, dtype=np.float64).ravel()
        two_s2 = 2.0 * self.sigma[:, None] ** 2
        out = self.amp @ np.exp(-(((x[None, :] - self.cx[:, None]) ** 2) + (y[None, :] - self.cy[:, None]) ** 2)
                                / two_s2)
        for spacing, amp, pad, vals in self.octaves:
            wx = _lattice_weights(x, spacing, pad, vals.shape[1])
            wy = _lattice_weights(y, spacing, pad, vals.shape[0])
            out += amp * np.einsum("ip,ij,jp->p", wy, vals, wx)
        return out


def _quantise(v: np.ndarray) -> np.ndarray:
    """Round half to even and clip to uint8."""
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


@dataclasses.dataclass
class Pair:
    """One synthetic frame pair and the parameters its workload runs with."""

    I1: np.ndarray            # uint8 [H, W]
    I2: np.ndarray            # uint8 [H, W]
    flow_gt: np.ndarray       # float32 [H, W, 2], forward flow of frame-1 pixels
    occluded: np.ndarray      # bool [H, W], frame-1 pixel not visible in frame 2
    win: int = 8
    step: int = 4
    levels: int = 3
    radius: int = 4
    max_iter: int = 30
    seed: int = 0

    @property
    def W(self) -> int:
        return self.I1.shape[1]

    @property
    def H(self) -> int:
        return self.I1.shape[0]


class _Mapper:
    """Affine map of raw texture values onto [16, 240] fixed by frame 1."""

    def __init__(self, raw1: np.ndarray):
        self.lo = float(raw1.min())
        self.hi = float(raw1.max())

    def __call__(self, v: np.ndarray) -> np.ndarray:
        return 16.0 + 224.0 * (v - self.lo) / max(self.hi - self.lo, 1e-12)


def make_translation_pair(W: int, H: int, t=(3.5, -1.25), seed: int = 0,
                          noise_sigma: float = 2.0, **params) -> Pair:
    """Frame 2 = frame 1 bilinearly warped by the constant translation t."""
    rng = _rng(seed)
    tex = Texture(rng, W, H)
    fresh = Texture(rng, W, H)
    xs, ys = np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64)
    raw1 = tex.raw(xs, ys)
    m = _Mapper(raw1)
    I1 = _quantise(m(raw1))
    tx, ty = float(t[0]), float(t[1])
    X, Y = np.meshgrid(xs, ys)
    sx, sy = X - tx, Y - ty
    inside = (sx >= 0) & (sx <= W - 1) & (sy >= 0) & (sy <= H - 1)
    warped = ndimage.map_coordinates(I1.astype(np.float64), [sy, sx], order=1, mode="nearest")
    v2 = np.where(inside, warped, m(fresh.raw(xs, ys)))
    v2 = v2 + rng.normal(0.0, noise_sigma, size=(H, W))
    I2 = _quantise(v2)
    flow = np.empty((H, W, 2), np.float32)
    flow[..., 0] = tx
    flow[..., 1] = ty
    occ = ~((X + tx >= 0) & (X + tx <= W - 1) & (Y + ty >= 0) & (Y + ty <= H - 1))
    return Pair(I1, I2, flow, occ, seed=seed, **params)


def make_radial_pair(W: int, H: int, seed: int = 0, max_disp: float = 150.0, n_rects: int = 3,
                     rect_w=(80, 300), rect_h=(40, 150), rect_t: float = 60.0,
                     noise_sigma: float = 2.0, **params) -> Pair:
    """Radial expansion about the centre plus rigid translating rectangles."""
    rng = _rng(seed)
    bg = Texture(rng, W, H)
    fresh = Texture(rng, W, H)
    c = np.array([(W - 1) / 2.0, (H - 1) / 2.0])
    k = max_disp / math.hypot(c[0], c[1])
    rects = []
    for _ in range(n_rects):
        rw = int(rng.integers(min(rect_w[0], W), min(rect_w[1], W) + 1))
        rh = int(rng.integers(min(rect_h[0], H), min(rect_h[1], H) + 1))
        x0 = int(rng.integers(0, W - rw + 1))
        y0 = int(rng.integers(0, H - rh + 1))
        tx, ty = rng.uniform(-rect_t, rect_t, 2)
        rects.append((x0, y0, rw, rh, float(tx), float(ty), Texture(rng, rw, rh)))
    xs, ys = np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64)

    # frame 1: background then rectangles in index order (the last one on top)
    raw1 = bg.raw(xs, ys)
    owner1 = np.full((H, W), -1, np.int64)
    for i, (x0, y0, rw, rh, tx, ty, rt) in enumerate(rects):
        raw1[y0:y0 + rh, x0:x0 + rw] = rt.raw(np.arange(rw, dtype=np.float64),
                                              np.arange(rh, dtype=np.float64))
        owner1[y0:y0 + rh, x0:x0 + rw] = i
    m = _Mapper(raw1)
    I1 = _quantise(m(raw1))

    # frame 2: rectangles at their moved footprints, else the radially mapped
    # background where its source is visible in frame 1, else fresh texture
    sxs = c[0] + (xs - c[0]) / (1.0 + k)
    sys_ = c[1] + (ys - c[1]) / (1.0 + k)
    v2 = m(bg.raw(sxs, sys_))
    SX, SY = np.meshgrid(sxs, sys_)
    visible = (SX >= 0) & (SX <= W - 1) & (SY >= 0) & (SY <= H - 1)
    for (x0, y0, rw, rh, _, _, _) in rects:
        visible &= ~((SX >= x0) & (SX < x0 + rw) & (SY >= y0) & (SY < y0 + rh))
    v2 = np.where(visible, v2, m(fresh.raw(xs, ys)))
    X2, Y2 = np.meshgrid(xs, ys)
    owner2 = np.full((H, W), -1, np.int64)
    for i, (x0, y0, rw, rh, tx, ty, rt) in enumerate(rects):
        ux, uy = xs - (x0 + tx), ys - (y0 + ty)
        cover = ((X2 >= x0 + tx) & (X2 < x0 + tx + rw) & (Y2 >= y0 + ty) & (Y2 < y0 + ty + rh))
        if cover.any():
            v2 = np.where(cover, m(rt.raw(ux, uy)), v2)
            owner2[cover] = i
    v2 = v2 + rng.normal(0.0, noise_sigma, size=(H, W))
    I2 = _quantise(v2)

    # ground truth at frame-1 pixels and their visibility in frame 2
    X1, Y1 = X2, Y2
    flow = np.empty((H, W, 2), np.float64)
    flow[..., 0] = k * (X1 - c[0])
    flow[..., 1] = k * (Y1 - c[1])
    for i, (x0, y0, rw, rh, tx, ty, _) in enumerate(rects):
        sel = owner1 == i
        flow[sel, 0] = tx
        flow[sel, 1] = ty
    TX, TY = X1 + flow[..., 0], Y1 + flow[..., 1]
    inb = (TX >= 0) & (TX <= W - 1) & (TY >= 0) & (TY <= H - 1)
    ix = np.clip(np.rint(TX), 0, W - 1).astype(np.int64)
    iy = np.clip(np.rint(TY), 0, H - 1).astype(np.int64)
    occ = ~inb | (owner2[iy, ix] != owner1)
    return Pair(I1, I2, flow.astype(np.float32), occ, seed=seed, **params)


def make_batch_specs(n_pairs: int, seed: int):
    """(W, H, step) per pair of the mixed-size batch workload, drawn uniformly."""
    rng = _rng(seed)
    out = []
    for _ in range(n_pairs):
        W, H = CONFIG_SIZES[int(rng.integers(0, len(CONFIG_SIZES)))]
        out.append((W, H, BATCH_STEPS[int(rng.integers(0, len(BATCH_STEPS)))]))
    return out


def make_pair(config: int, index: int = 0, size=None) -> Pair:
    """Pair ``index`` of workload ``config`` (seed = 1000 * config + index).

    1: 256x128 translation (3.5, -1.25); window 8, step 4; 3 levels, 9x9 support.
    2: 1242x375 radial expansion (150 px at the corners) + 3 rectangles;
       window 7, step 3; 5 levels, 11x11 support.
    3: mixed-size batch member (size and step drawn per pair), translation flow,
       window 8; 3 levels, 9x9 support.
    4, 5: 1242x375 translation flow; window 8, step 4; 3 levels, 9x9 support.
    ``size`` overrides (W, H) for reduced-size test cases.
    """
    seed = 1000 * config + index
    if config == 1:
        W, H = size or (256, 128)
        return make_translation_pair(W, H, seed=seed, win=8, step=4, levels=3, radius=4)
    if config == 2:
        W, H = size or (1242, 375)
        return make_radial_pair(W, H, seed=seed, win=7, step=3, levels=5, radius=5)
    if config == 3:
        (W0, H0, step), = make_batch_specs(1, seed)
        W, H = size or (W0, H0)
        return make_translation_pair(W, H, seed=seed, win=8, step=step, levels=3, radius=4)
    if config in (4, 5):
        W, H = size or (1242, 375)
        return make_translation_pair(W, H, seed=seed, win=8, step=4, levels=3, radius=4)
    raise ValueError(f"unknown workload {config}")


def render(W: int, H: int, seed: int, shift=(0.0, 0.0)) -> np.ndarray:
    """Unquantised texture frame (float64, about [16, 240]) sampled at x - shift.

    ``render(W, H, s, t)`` is ``render(W, H, s)`` translated by ``t``, exactly for
    any real ``t`` (the texture is a continuous function), which gives frame pairs
    with a known sub-pixel translation and no interpolation or rounding error.
    """
    rng = _rng(seed)
    tex = Texture(rng, W, H)
    xs, ys = np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64)
    m = _Mapper(tex.raw(xs, ys))
    return m(tex.raw(xs - shift[0], ys - shift[1]))


def render_affine(W: int, H: int, seed: int, A, c) -> np.ndarray:
    """Frame 2 of an analytic affine motion of ``render(W, H, seed)``: the frame-1
    point x moves to c + A (x - c), so the true flow at x is (A - I)(x - c). The
    texture is evaluated at each pixel's exact source point A^-1 (x - c) + c (no
    interpolation or rounding), with frame 1's intensity mapping."""
    rng = _rng(seed)
    tex = Texture(rng, W, H)
    xs, ys = np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64)
    m = _Mapper(tex.raw(xs, ys))
    Ai = np.linalg.inv(np.asarray(A, dtype=np.float64))
    Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
    sx = c[0] + Ai[0, 0] * (X - c[0]) + Ai[0, 1] * (Y - c[1])
    sy = c[1] + Ai[1, 0] * (X - c[0]) + Ai[1, 1] * (Y - c[1])
    return m(tex.raw_at(sx, sy).reshape(H, W))
