"""Pins of the oracle's adjoints (the gradients of key-points and of tracked flow
with respect to the frames) to central finite differences of the pinned forward
oracle. CPU only."""
import numpy as np
import pytest

import oracle
import synth


def fd_dot(fun, img, pixels, h):
    """Central differences of the scalar fun(img) at the given (y, x) pixels."""
    out = []
    for (y, x) in pixels:
        a = img.copy()
        b = img.copy()
        a[y, x] += h
        b[y, x] -= h
        out.append((fun(a) - fun(b)) / (2 * h))
    return np.array(out)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_degraf_vjp_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    H, W, w, h, step = 16, 21, 5, 4, 2
    img = rng.uniform(0, 60, (H, W))
    img[rng.random((H, W)) < 0.08] += 150  # sparse bright pixels: both centroids occur
    n = oracle.degraf_count(W, H, w, h, step)
    g = rng.normal(size=(n, 2))
    neg = oracle.degraf_detect(np.clip(np.rint(img), 0, 255).astype(np.uint8), w, h, step)[2]
    assert 0 < neg.sum() < n  # both selections are exercised

    def L(im):
        return float(np.sum(g * oracle.degraf_detect_f64(im, w, h, step)))

    vjp = oracle.degraf_vjp(img, w, h, step, g)
    pixels = [(y, x) for y in range(H) for x in range(W)]
    fd = fd_dot(L, img, pixels, 1e-5).reshape(H, W)
    assert np.abs(vjp - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_degraf_vjp_positive_centroid_closed_form():
    """A bright window keeps C_pos: d(x)/dI_ij = (j - x) / S exactly."""
    rng = np.random.default_rng(5)
    img = rng.uniform(180, 250, (6, 7))
    g = np.array([[1.0, 0.0]])
    vjp = oracle.degraf_vjp(img, 7, 6, 1, g)
    S = img.sum()
    cx = (img * np.arange(7)[None, :]).sum() / S
    assert np.allclose(vjp, (np.arange(7)[None, :] - cx) / S * np.ones((6, 1)), atol=1e-15)


def track_params(model, hampel=True):
    kw = {} if hampel else dict(hampel_a=1e30, hampel_b=1e30, hampel_c=2e30)
    return oracle.RlofParams(levels=2, radius=3, model=model, eps=1e-13, max_iter=200, **kw)


@pytest.mark.parametrize("model,perturb", [(2, 0.0), (4, 0.0), (4, 20.0), (2, 20.0)])
def test_rlof_vjp_matches_finite_differences(model, perturb):
    """Smooth frames with a sub-pixel shift (all samples inliers), and with a block of
    +20 residuals that puts samples in the descending Hampel segment."""
    W, H = 64, 48
    I1 = synth.render(W, H, 11)
    I2 = synth.render(W, H, 11, shift=(0.35, -0.6))
    if model == 4:  # a gain and offset change the illumination terms absorb
        I2 = I2 * 1.05 + 2.0
    if perturb:
        I2[20:24, 30:33] += perturb
    pts = np.array([[31.5, 19.5], [24.8, 20.2], [36.1, 25.7]])
    prm = track_params(model)
    flow, st, _, illum = oracle.rlof_track(I1, I2, pts, prm)
    assert np.all(st == oracle.TRACKED)
    rng = np.random.default_rng(model)
    gflow = rng.normal(size=flow.shape)
    g1, g2 = oracle.rlof_vjp(I1, I2, pts, prm, flow, illum, st, gflow)

    def L1(im):
        f, s, _, _ = oracle.rlof_track(im, I2, pts, prm)
        assert np.all(s == oracle.TRACKED)
        return float(np.sum(gflow * f))

    def L2(im):
        f, s, _, _ = oracle.rlof_track(I1, im, pts, prm)
        assert np.all(s == oracle.TRACKED)
        return float(np.sum(gflow * f))

    # pixels under the supports (template side and search side)
    pix = [(y, x) for y in range(17, 30, 2) for x in range(20, 41, 3)]
    fd1 = fd_dot(L1, I1, pix, 1e-3)
    fd2 = fd_dot(L2, I2, pix, 1e-3)
    a1 = np.array([g1[y, x] for (y, x) in pix])
    a2 = np.array([g2[y, x] for (y, x) in pix])
    scale = max(np.abs(fd1).max(), np.abs(fd2).max())
    assert scale > 1e-3
    assert np.abs(a1 - fd1).max() <= 2e-4 * scale
    assert np.abs(a2 - fd2).max() <= 2e-4 * scale


@pytest.mark.parametrize("model", [2, 4])
def test_rlof_vjp_matches_fd_on_256_random_pixels(model):
    """The differentiation check as stated for that workload: central differences
    with h = 1e-2 intensity at 256 random pixels of both frames (those off every
    support must come out zero), 12 random points, random upstream weights; within
    1e-5 of the largest entry (measured: 2.5e-8 for model 2, 5.5e-7 for model 4)."""
    W, H = 64, 48
    I1 = synth.render(W, H, 11)
    I2 = synth.render(W, H, 11, shift=(0.35, -0.6))
    if model == 4:
        I2 = I2 * 1.05 + 2.0
    rng = np.random.default_rng(100 + model)
    pts = np.stack([rng.uniform(14, W - 14, 12), rng.uniform(12, H - 12, 12)], 1)
    prm = track_params(model)
    flow, st, _, illum = oracle.rlof_track(I1, I2, pts, prm)
    assert np.all(st == oracle.TRACKED)
    gflow = rng.normal(size=flow.shape)
    g1, g2 = oracle.rlof_vjp(I1, I2, pts, prm, flow, illum, st, gflow)
    pix = [(int(i // W), int(i % W)) for i in rng.choice(W * H, 256, replace=False)]
    fd1 = fd_dot(lambda im: float(np.sum(gflow * oracle.rlof_track(im, I2, pts, prm)[0])), I1, pix, 1e-2)
    fd2 = fd_dot(lambda im: float(np.sum(gflow * oracle.rlof_track(I1, im, pts, prm)[0])), I2, pix, 1e-2)
    a1 = np.array([g1[y, x] for (y, x) in pix])
    a2 = np.array([g2[y, x] for (y, x) in pix])
    scale = max(np.abs(fd1).max(), np.abs(fd2).max())
    assert scale > 1e-3 and (np.abs(a1) > 0).sum() > 20 and (np.abs(a1) == 0).sum() > 20
    assert np.abs(a1 - fd1).max() <= 1e-5 * scale
    assert np.abs(a2 - fd2).max() <= 1e-5 * scale


def test_rlof_vjp_zero_for_lost_points_and_outlier_samples():
    W, H = 64, 48
    I1 = synth.render(W, H, 11)
    I2 = synth.render(W, H, 11, shift=(0.35, -0.6))
    pts = np.array([[30.3, 22.6]])
    prm = track_params(2)
    flow, st, _, illum = oracle.rlof_track(I1, I2, pts, prm)
    g1, g2 = oracle.rlof_vjp(I1, I2, pts, prm, flow, illum, np.array([oracle.OOB], np.uint8), np.ones((1, 2)))
    assert not g1.any() and not g2.any()
    g1, g2 = oracle.rlof_vjp(I1, I2, pts, prm, flow, illum, st, np.ones((1, 2)))
    assert g2.any() and np.all(g2[:10] == 0)  # nothing outside the support
