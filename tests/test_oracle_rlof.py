"""Pins of the oracle's RLOF tracker (Section 2 "Sparse point tracking", Section 3
"Parameters"). The paper gives no RLOF formulas, so the pins are facts any correct
robust pyramidal Lucas-Kanade with a gain/offset illumination model must satisfy:
exact recovery of integer translations and of gain/offset changes, equality with an
independently written textbook Lucas-Kanade in the non-robust special case,
rejection of gross outliers by the Hampel norm, and the lost-point rules. CPU only."""
import numpy as np
import pytest
from scipy import ndimage

import oracle
import synth

W, H = 160, 96
HUGE = dict(hampel_a=1e30, hampel_b=1e30, hampel_c=2e30)


@pytest.fixture(scope="module")
def frame1():
    return synth.render(W, H, 5)


def shifted(I1, t, gain=1.0, offset=0.0, fill_seed=77):
    """I2(x) = gain * I1(x - t) + offset for integer t; uncovered pixels get fresh texture."""
    I2 = synth.render(W, H, fill_seed)
    tx, ty = t
    y, x = np.mgrid[0:H, 0:W]
    ok = (x - tx >= 0) & (x - tx < W) & (y - ty >= 0) & (y - ty < H)
    I2[ok] = I1[(y - ty)[ok], (x - tx)[ok]]
    return gain * I2 + offset


def interior_points(n=200, margin=30, seed=0):
    rng = np.random.default_rng(seed)
    return np.stack([rng.uniform(margin, W - margin, n), rng.uniform(margin, H - margin, n)], 1)


def test_hampel_psi_knots():
    a, b, c = 8.0, 16.0, 32.0
    psi = lambda r: oracle.hampel_psi(r, a, b, c)  # noqa: E731
    assert psi(0.0) == 0.0 and psi(3.0) == 3.0 and psi(-a) == -a
    assert psi(b) == a and psi(12.0) == a and psi(-12.0) == -a
    assert psi((b + c) / 2) == a / 2 and psi(c) == 0.0 and psi(c + 1e-9) == 0.0
    assert psi(-1e6) == 0.0
    # continuous at every knot
    for k in (a, b, c):
        assert abs(psi(k - 1e-9) - psi(k + 1e-9)) < 1e-6


@pytest.mark.parametrize("t", [(5, -3), (9, -7), (-12, 4)])
def test_integer_translation_is_exact(frame1, t):
    """Bilinear sampling is exact at an integer shift, so d = t is a fixed point
    with zero residual; coarse-to-fine must reach it from |t| beyond the level-0
    support radius."""
    pts = interior_points()
    prm = oracle.RlofParams(levels=3, radius=4, model=2, eps=1e-10, max_iter=100)
    flow, st, _, _ = oracle.rlof_track(frame1, shifted(frame1, t), pts, prm)
    assert np.all(st == oracle.TRACKED)
    assert np.abs(flow - np.array(t)).max() < 1e-9


def test_single_level_cannot_reach_large_translation(frame1):
    """Without the pyramid a shift far beyond the support is not recovered."""
    pts = interior_points()
    prm = oracle.RlofParams(levels=1, radius=4, model=2, eps=1e-10, max_iter=100)
    flow, st, _, _ = oracle.rlof_track(frame1, shifted(frame1, (9, -7)), pts, prm)
    ok = (st == oracle.TRACKED) & (np.abs(flow - [9, -7]).max(1) < 1e-6)
    assert ok.mean() < 0.8


@pytest.mark.parametrize("t", [(4, -4), (5, -3)])
def test_gain_offset_is_exact(frame1, t):
    """Model 4: I2 = 1.2 I1(x - t) - 10 gives the fixed point d = t, m = 0.2, c = -10."""
    pts = interior_points()
    prm = oracle.RlofParams(levels=3, radius=4, model=4, eps=1e-10, max_iter=100)
    flow, st, _, illum = oracle.rlof_track(frame1, shifted(frame1, t, 1.2, -10.0), pts, prm)
    assert np.all(st == oracle.TRACKED)
    assert np.abs(flow - np.array(t)).max() < 1e-9
    assert np.abs(illum - [0.2, -10.0]).max() < 1e-8


def test_translation_model_is_biased_by_gain(frame1):
    """Model 2 has no illumination terms, so the same gain change moves its answer."""
    pts = interior_points()
    prm = oracle.RlofParams(levels=3, radius=4, model=2, eps=1e-10, max_iter=100, **HUGE)
    flow, st, _, _ = oracle.rlof_track(frame1, shifted(frame1, (4, -4), 1.2, -10.0), pts, prm)
    ok = st == oracle.TRACKED
    assert np.median(np.abs(flow[ok] - [4, -4]).max(1)) > 1e-3


def textbook_lk(I1, I2, p, radius, eps, max_iter):
    """One-level Lucas-Kanade, written independently with SciPy primitives:
    d <- d + G^-1 sum grad T (T - J(p + d)), G = sum grad T grad T^T, with Sobel/8
    template gradients and clamp-to-edge bilinear sampling."""
    gx = ndimage.sobel(I1, axis=1, mode="nearest") / 8.0
    gy = ndimage.sobel(I1, axis=0, mode="nearest") / 8.0
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    ky, kx = np.meshgrid(k, k, indexing="ij")
    cy, cx = p[1] + ky.ravel(), p[0] + kx.ravel()

    def sample(img, yy, xx):
        return ndimage.map_coordinates(img, [yy, xx], order=1, mode="nearest")

    T, Tx, Ty = sample(I1, cy, cx), sample(gx, cy, cx), sample(gy, cy, cx)
    A = np.stack([Tx, Ty], 1)
    G = A.T @ A
    d = np.zeros(2)
    for _ in range(max_iter):
        J = sample(I2, cy + d[1], cx + d[0])
        step = np.linalg.solve(G, A.T @ (T - J))
        d += step
        if np.hypot(*step) < eps:
            break
    return d


def test_non_robust_single_level_equals_textbook_lk(frame1):
    I2 = synth.render(W, H, 5, shift=(1.3, -0.6))
    pts = interior_points(40, seed=3)
    prm = oracle.RlofParams(levels=1, radius=5, model=2, eps=1e-12, max_iter=60, **HUGE)
    flow, st, _, _ = oracle.rlof_track(frame1, I2, pts, prm)
    for k in range(pts.shape[0]):
        ref = textbook_lk(frame1, I2, pts[k], 5, 1e-12, 60)
        assert st[k] in (oracle.TRACKED, oracle.MAXITER)
        assert np.abs(flow[k] - ref).max() < 1e-9


def test_subpixel_translation_recovered(frame1):
    """Analytic sub-pixel shift: the error left is the bilinear model error of a
    smooth texture (bound measured once: max 0.05 px for model 2, 0.10 px for 4)."""
    pts = interior_points()
    for t in [(0.4, -0.7), (2.3, 1.6)]:
        I2 = synth.render(W, H, 5, shift=t)
        for model, bound in ((2, 0.07), (4, 0.12)):
            prm = oracle.RlofParams(levels=3, radius=4, model=model, eps=1e-6, max_iter=100)
            flow, st, _, _ = oracle.rlof_track(frame1, I2, pts, prm)
            e = np.hypot(*(flow - np.array(t)).T)
            assert np.all(st == oracle.TRACKED)
            assert np.median(e) < 0.02 and e.max() < bound


@pytest.mark.parametrize("p", [(80.0, 48.0), (70.0, 40.0), (100.0, 50.0), (60.0, 60.0)])
def test_hampel_rejects_gross_outliers(p):
    """A 2x2 block of +120 corruption inside the support: at an integer point and an
    integer shift every sample hits one pixel, the corrupted residuals lie beyond c
    so their weights are 0, and d = t stays an exact fixed point that coarse-to-fine
    reaches. The L2 norm (all weights 1) is pulled away from t."""
    rng = np.random.default_rng(1)

    def texture():
        v = ndimage.gaussian_filter(rng.uniform(0, 255, (H, W)), 1.5)
        return 16 + 224 * (v - v.min()) / (v.max() - v.min())

    I1 = texture()
    t = (5, -3)
    I2 = texture()
    y, x = np.mgrid[0:H, 0:W]
    ok = (x - t[0] >= 0) & (x - t[0] < W) & (y - t[1] >= 0) & (y - t[1] < H)
    I2[ok] = I1[(y - t[1])[ok], (x - t[0])[ok]]
    cy, cx = int(p[1]) + t[1], int(p[0]) + t[0]
    I2[cy - 1: cy + 1, cx + 1: cx + 3] += 120.0
    pts = np.array([p])
    robust = oracle.RlofParams(levels=3, radius=4, model=2, eps=1e-10, max_iter=100)
    flow, st, _, _ = oracle.rlof_track(I1, I2, pts, robust)
    assert st[0] == oracle.TRACKED and np.abs(flow[0] - t).max() < 1e-9
    plain = oracle.RlofParams(levels=3, radius=4, model=2, eps=1e-10, max_iter=100, **HUGE)
    flow2, _, _, _ = oracle.rlof_track(I1, I2, pts, plain)
    assert np.abs(flow2[0] - t).max() > 5e-2


def test_lost_point_rules(frame1):
    prm = oracle.RlofParams(levels=2, radius=4, model=4)
    # flat frames: the gradient matrix is zero
    flat = np.full((H, W), 100.0)
    _, st, it, _ = oracle.rlof_track(flat, flat, np.array([[50.0, 40.0]]), prm)
    assert st[0] == oracle.SMALL_EIG and it[0] == 0
    # a point pushed out of the frame by a large shift
    I2 = shifted(frame1, (-12, 0))
    flow, st, _, _ = oracle.rlof_track(frame1, I2, np.array([[3.0, 40.0]]),
                                       oracle.RlofParams(levels=3, radius=4, model=2))
    assert st[0] == oracle.OOB and np.all(flow[0] == 0)
    # a point that starts outside the frame
    _, st, _, _ = oracle.rlof_track(frame1, frame1, np.array([[-5.0, 40.0]]), prm)
    assert st[0] == oracle.OOB
    # one iteration is not enough to converge: tracked, but flagged
    flow, st, it, _ = oracle.rlof_track(frame1, shifted(frame1, (2, 1)), np.array([[80.0, 48.0]]),
                                        oracle.RlofParams(levels=1, radius=4, model=2, max_iter=1))
    assert st[0] == oracle.MAXITER and it[0] == 1 and np.all(flow[0] != 0)


def test_identical_frames_give_zero_flow(frame1):
    pts = interior_points()
    flow, st, it, illum = oracle.rlof_track(frame1, frame1, pts, oracle.RlofParams(levels=3, radius=5))
    assert np.all(st == oracle.TRACKED) and np.abs(flow).max() < 1e-12 and np.abs(illum).max() < 1e-12


def test_affine_warp_recovered(frame1):
    """Analytic affine motion about the frame centre (2% zoom, 1.2 degree rotation):
    every point's flow is its centre's motion (A - I)(p - c) up to the bias of a
    translation model over a deforming support, which is first order in A - I.
    Bounds measured once: median 0.10 / 0.14 px, max 0.38 / 0.43 px (models 2 / 4)
    at flows up to 1.32 px; halving A - I halves each point's error (median ratio
    2.00). A swapped axis or a flipped sign leaves errors of the flow's own size."""
    pts = interior_points()
    c = np.array([W / 2, H / 2])

    def errors(s, model):
        th = np.deg2rad(1.2 * s)
        A = (1 + 0.02 * s) * np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
        I2 = synth.render_affine(W, H, 5, A, c)
        prm = oracle.RlofParams(levels=3, radius=4, model=model, eps=1e-8, max_iter=200)
        flow, st, _, _ = oracle.rlof_track(frame1, I2, pts, prm)
        assert np.all(st == oracle.TRACKED)
        return np.hypot(*(flow - (pts - c) @ (A - np.eye(2)).T).T)

    for model, med, top in ((2, 0.12, 0.45), (4, 0.16, 0.5)):
        e1, e2 = errors(1.0, model), errors(0.5, model)
        assert np.median(e1) < med and e1.max() < top
        assert 1.9 < np.median(e1 / np.maximum(e2, 1e-9)) < 2.1


def test_converged_state_is_a_fixed_point(frame1):
    """At convergence the robust normal equations vanish: sum_k psi(r_k) a_k = 0 with
    r_k = J(p + f + k) - (1 + m) T(p + k) - c and a_k = (Tx, Ty, -T, -1) at level 0.
    Recomputed here from the oracle's flow and gain/offset with SciPy's bilinear
    sampling and Sobel filter and a Hampel psi written from its definition, the
    Newton step H^-1 sum psi a (H = sum w a a^T) must be below 1e-8 (d, m) and
    1e-6 (c, in intensity levels). Noise and a corrupted block put residuals in
    every zone of the Hampel norm."""
    a_, b_, c_ = 8.0, 16.0, 32.0
    r = 4
    I2 = 1.1 * synth.render(W, H, 5, shift=(1.7, -0.9)) + 5 + np.random.default_rng(11).normal(0, 10, (H, W))
    I2[40:47, 60:67] += 120.0
    gx0, gy0 = np.meshgrid(np.arange(50.0, 76.0, 1.5), np.arange(34.0, 54.0, 1.5))  # supports over the block
    pts = np.concatenate([interior_points(), np.stack([gx0.ravel(), gy0.ravel()], 1)])
    prm = oracle.RlofParams(levels=3, radius=r, model=4, eps=1e-10, max_iter=200, hampel_a=a_, hampel_b=b_,
                            hampel_c=c_)
    flow, st, _, illum = oracle.rlof_track(frame1, I2, pts, prm)
    done = np.flatnonzero(st == oracle.TRACKED)
    assert done.size >= 30

    def psi(x):
        ax = np.abs(x)
        return np.where(ax <= a_, x, np.where(ax <= b_, a_ * np.sign(x),
                                              np.where(ax <= c_, a_ * np.sign(x) * (c_ - ax) / (c_ - b_), 0.0)))

    def sample(img, yy, xx):
        return ndimage.map_coordinates(img, [yy, xx], order=1, mode="nearest")

    gx = ndimage.sobel(frame1, axis=1, mode="nearest") / 8.0
    gy = ndimage.sobel(frame1, axis=0, mode="nearest") / 8.0
    k = np.arange(-r, r + 1, dtype=np.float64)
    ky, kx = (v.ravel() for v in np.meshgrid(k, k, indexing="ij"))
    zones = np.zeros(4)
    for i in done:
        cy, cx = pts[i, 1] + ky, pts[i, 0] + kx
        T, Tx, Ty = sample(frame1, cy, cx), sample(gx, cy, cx), sample(gy, cy, cx)
        m, c = illum[i]
        res = sample(I2, cy + flow[i, 1], cx + flow[i, 0]) - (1 + m) * T - c
        w = np.where(res == 0, 1.0, psi(res) / np.where(res == 0, 1.0, res))
        a = np.stack([Tx, Ty, -T, -np.ones_like(T)], 1)
        step = np.linalg.solve((a * w[:, None]).T @ a, a.T @ psi(res))
        assert np.abs(step[:3]).max() < 1e-8 and abs(step[3]) < 1e-6, (i, step)
        ar = np.abs(res)
        zones += [(ar <= a_).sum(), ((ar > a_) & (ar <= b_)).sum(), ((ar > b_) & (ar <= c_)).sum(), (ar > c_).sum()]
    assert np.all(zones > 0), zones


def test_tiny_case_is_the_root_of_the_robust_normal_equations():
    """One point, 5x5 support, one level, gain/offset model: the oracle's converged
    state (d, m, c) is the root of sum_k psi(r_k) a_k = 0 that mpmath's multidimensional
    Newton finds in 30-digit arithmetic, with bilinear sampling (taps clamped), Sobel/8
    template gradients and the Hampel psi written here from their definitions. Frame 2
    is shifted, brightened and corrupted in one support pixel so that residuals fall
    in every Hampel zone."""
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 30
    Wt, Ht, r = 16, 14, 2
    I1 = synth.render(Wt, Ht, 21)
    I2 = 1.08 * synth.render(Wt, Ht, 21, shift=(0.6, -0.35)) + 3.0
    I2[8, 8] += 60.0
    I2[6, 9] -= 14.0
    p = np.array([[7.4, 6.7]])
    prm = oracle.RlofParams(levels=1, radius=r, model=4, eps=1e-14, max_iter=500)
    flow, st, _, illum = oracle.rlof_track(I1, I2, p, prm)
    assert st[0] == oracle.TRACKED
    a_, b_, c_ = mp.mpf(8), mp.mpf(16), mp.mpf(32)

    def psi(x):
        ax = abs(x)
        if ax <= a_:
            return x
        s = 1 if x > 0 else -1
        if ax <= b_:
            return a_ * s
        return a_ * s * (c_ - ax) / (c_ - b_) if ax <= c_ else mp.mpf(0)

    def pix(img, x, y):
        return mp.mpf(float(img[min(max(y, 0), img.shape[0] - 1), min(max(x, 0), img.shape[1] - 1)]))

    def bilinear(img, x, y):
        x0, y0 = int(mp.floor(x)), int(mp.floor(y))
        fx, fy = x - x0, y - y0
        return ((1 - fx) * (1 - fy) * pix(img, x0, y0) + fx * (1 - fy) * pix(img, x0 + 1, y0)
                + (1 - fx) * fy * pix(img, x0, y0 + 1) + fx * fy * pix(img, x0 + 1, y0 + 1))

    def sobel(img, axis):
        out = np.zeros_like(img)
        for y in range(img.shape[0]):
            for x in range(img.shape[1]):
                v = 0.0
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        w = (dx if axis == 1 else dy) * (2 if (dy if axis == 1 else dx) == 0 else 1)
                        v += w * float(img[min(max(y + dy, 0), img.shape[0] - 1), min(max(x + dx, 0), img.shape[1] - 1)])
                out[y, x] = v / 8.0
        return out

    gx, gy = sobel(I1, 1), sobel(I1, 0)
    px, py = mp.mpf(p[0, 0]), mp.mpf(p[0, 1])
    ks = [(kx, ky) for ky in range(-r, r + 1) for kx in range(-r, r + 1)]
    tmpl = [(bilinear(I1, px + kx, py + ky), bilinear(gx, px + kx, py + ky), bilinear(gy, px + kx, py + ky))
            for kx, ky in ks]
    zones = set()

    def F(dx, dy, m, c):
        out = [mp.mpf(0)] * 4
        for (kx, ky), (T, Tx, Ty) in zip(ks, tmpl):
            res = bilinear(I2, px + dx + kx, py + dy + ky) - (1 + m) * T - c
            zones.add(0 if abs(res) <= a_ else 1 if abs(res) <= b_ else 2 if abs(res) <= c_ else 3)
            w = psi(res)
            for i, a in enumerate((Tx, Ty, -T, mp.mpf(-1))):
                out[i] += w * a
        return out

    # Newton from a start away from the oracle's answer (0.05 px, 1% gain, 0.5 offset);
    # measured: it lands within 2.1e-13 of the oracle
    start = [mp.mpf(flow[0, 0]) + mp.mpf("0.05"), mp.mpf(flow[0, 1]) - mp.mpf("0.04"),
             mp.mpf(illum[0, 0]) + mp.mpf("0.01"), mp.mpf(illum[0, 1]) - mp.mpf("0.5")]
    root = mpmath.findroot(F, start, tol=mp.mpf(10) ** -25)
    got = np.array([flow[0, 0], flow[0, 1], illum[0, 0], illum[0, 1]])
    assert np.abs(np.array([float(v) for v in root]) - got).max() < 1e-9
    assert zones == {0, 1, 2, 3}, zones
