"""Pins of the oracle's global-motion prior (Section 3 "Parameters", RLOF(IM-GM): a
global affine motion fitted robustly to first-pass tracks and used as every
point's initial flow). The paper prints no formula, so the pins are the
mathematics of the reading: exact recovery of an affine motion, rejection of gross
outliers where least squares fails, the degenerate cases, zero prior = plain
tracking, and large affine motions tracked only with the prior."""
import numpy as np
import pytest

import oracle
import synth


def affine_flow(a, pts):
    x, y = pts[:, 0], pts[:, 1]
    return np.stack([a[0] * x + a[1] * y + a[2] - x, a[3] * x + a[4] * y + a[5] - y], 1)


A_TRUE = np.array([1.08, -0.03, -21.5, 0.02, 1.05, 7.25])


def grid_points(W=640, H=360, step=16):
    ys, xs = np.mgrid[4:H - 4:step, 4:W - 4:step]
    return np.stack([xs.ravel() + 0.37, ys.ravel() + 0.61], 1).astype(np.float64)


def test_fit_recovers_exact_affine_and_ignores_lost_points():
    pts = grid_points()
    flow = affine_flow(A_TRUE, pts)
    status = np.zeros(len(pts), np.uint8)
    rng = np.random.default_rng(1)
    lost = rng.choice(len(pts), 50, replace=False)
    status[lost] = rng.choice([oracle.OOB, oracle.SINGULAR, oracle.MAXITER], 50)
    flow[lost] += rng.uniform(-80, 80, (50, 2))  # garbage on points that are not TRACKED
    a, made = oracle.gm_fit_affine(pts, flow, status)
    assert made
    np.testing.assert_allclose(a, A_TRUE, rtol=0, atol=1e-9)
    np.testing.assert_allclose(oracle.gm_prior_flow(a, pts), affine_flow(A_TRUE, pts), atol=1e-7)


def test_fit_rejects_gross_outliers_where_least_squares_fails():
    pts = grid_points()
    flow = affine_flow(A_TRUE, pts)
    rng = np.random.default_rng(7)
    out = rng.choice(len(pts), int(0.3 * len(pts)), replace=False)
    flow[out] += rng.uniform(-100, 100, (len(out), 2))
    status = np.zeros(len(pts), np.uint8)
    inl = np.setdiff1d(np.arange(len(pts)), out)
    a_ls, _ = oracle.gm_fit_affine(pts, flow, status, iters=1)  # plain least squares
    a, made = oracle.gm_fit_affine(pts, flow, status)
    assert made
    err_ls = np.abs(affine_flow(a_ls, pts[inl]) - affine_flow(A_TRUE, pts[inl])).max()
    err = np.abs(affine_flow(a, pts[inl]) - affine_flow(A_TRUE, pts[inl])).max()
    assert err_ls > 1.0
    assert err < 1e-6  # outliers end with weight exactly 0


def test_one_reweighting_is_tukey_weighted_least_squares():
    """Two IRLS iterations: a least-squares fit, then a weighted least-squares fit
    with Tukey biweights (1 - (e / c)^2)^2 of its residuals e at c = c0 (zero beyond);
    both steps recomputed here with numpy's least squares."""
    pts = grid_points(step=24)
    rng = np.random.default_rng(5)
    flow = affine_flow(A_TRUE, pts) + rng.normal(0, 3.0, (len(pts), 2))
    flow[rng.choice(len(pts), 40, replace=False)] += rng.uniform(-60, 60, (40, 2))
    status = np.zeros(len(pts), np.uint8)
    c0 = 16.0
    a, made = oracle.gm_fit_affine(pts, flow, status, iters=2, c0=c0, c_min=1.0)
    assert made
    X = np.c_[pts, np.ones(len(pts))]
    Q = pts + flow
    a0 = np.linalg.lstsq(X, Q, rcond=None)[0]  # [3, 2]: columns are the x and y rows
    e = np.hypot(*(X @ a0 - Q).T)
    w = np.where(e < c0, (1 - (e / c0) ** 2) ** 2, 0.0)
    a1 = np.linalg.lstsq(X * np.sqrt(w)[:, None], Q * np.sqrt(w)[:, None], rcond=None)[0]
    expect = np.r_[a1[:, 0], a1[:, 1]]
    assert 0 < np.mean(w > 0) < 1
    np.testing.assert_allclose(a, expect, rtol=0, atol=1e-8)


def test_fit_degenerate_cases_fall_back_to_identity():
    ident = np.array([1, 0, 0, 0, 1, 0], float)
    pts = grid_points()[:2]
    a, made = oracle.gm_fit_affine(pts, np.ones((2, 2)), np.zeros(2, np.uint8))
    assert not made and np.array_equal(a, ident)
    line = np.stack([np.arange(20.0), 2 * np.arange(20.0) + 1], 1)  # collinear: singular
    a, made = oracle.gm_fit_affine(line, np.ones((20, 2)), np.zeros(20, np.uint8))
    assert not made and np.array_equal(a, ident)
    a, made = oracle.gm_fit_affine(np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(0, np.uint8))
    assert not made
    with pytest.raises(ValueError):
        oracle.gm_fit_affine(pts, np.ones((2, 2)), np.zeros(2, np.uint8), iters=0)
    np.testing.assert_array_equal(oracle.gm_prior_flow(ident, grid_points()), 0.0)


def test_zero_prior_is_plain_tracking():
    p = synth.make_pair(1)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, model=4)
    f0, s0, i0, l0 = oracle.rlof_track(p.I1, p.I2, pts, prm)
    f1, s1, i1, l1 = oracle.rlof_track(p.I1, p.I2, pts, prm, init_flow=np.zeros_like(pts))
    for u, v in ((f0, f1), (s0, s1), (i0, i1), (l0, l1)):
        np.testing.assert_array_equal(u, v)


def test_prior_reaches_large_motion_plain_tracking_loses():
    """37 px of global translation (9 px at the coarsest of 3 levels, beyond a 9x9
    support): plain tracking converges to wrong flows; the exact prior and the
    two-pass method (sparse deep first pass, fit, retrack) reach the accuracy that
    plain tracking has on a small motion."""
    t = (37.3, -21.6)
    p = synth.make_translation_pair(640, 360, t=t, seed=11)
    a_true = np.array([1.0, 0.0, t[0], 0.0, 1.0, t[1]])
    pts, _, _ = oracle.degraf_detect(p.I1, 8, 8, 8)
    gt = affine_flow(a_true, pts)
    visible = np.all((pts + gt >= 6) & (pts + gt <= np.array([p.W, p.H]) - 7), axis=1)
    prm = oracle.RlofParams(levels=3, radius=4, model=4)

    def good(flow, status):  # tracked into the right basin (the textured pair's EPE is ~0.4 px)
        ok = (status == oracle.TRACKED) & (np.hypot(*(flow - gt).T) < 2.0)
        return np.mean(ok[visible])

    f0, s0, _, _ = oracle.rlof_track(p.I1, p.I2, pts, prm)
    f1, s1, _, _ = oracle.rlof_track(p.I1, p.I2, pts, prm, init_flow=oracle.gm_prior_flow(a_true, pts))
    f2, s2, _, _, a_fit, made = oracle.rlof_track_gm(p.I1, p.I2, pts, prm)
    small = synth.make_translation_pair(640, 360, t=(3.5, -1.25), seed=11)
    f3, s3, _, _ = oracle.rlof_track(small.I1, small.I2, pts, prm)
    gs = np.mean((s3 == oracle.TRACKED) & (np.hypot(*(f3 - np.array([3.5, -1.25])).T) < 2.0))
    print(f"good: plain {good(f0, s0):.3f}, exact prior {good(f1, s1):.3f}, two-pass {good(f2, s2):.3f}, "
          f"small motion plain {gs:.3f}; fitted prior max error "
          f"{np.abs(oracle.gm_prior_flow(a_fit, pts) - gt).max():.3f} px")
    assert made
    assert np.abs(oracle.gm_prior_flow(a_fit, pts) - gt).max() < 0.2
    assert good(f0, s0) < 0.3
    assert good(f1, s1) > 0.95 * gs
    assert good(f2, s2) > 0.95 * gs


def test_two_pass_prior_keeps_small_motion_results():
    """On the small-motion workload the prior is near zero motion and the tracks
    stay as good as plain tracking."""
    p = synth.make_pair(1)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, model=4)
    gt = np.array([3.5, -1.25])
    f0, s0, _, _ = oracle.rlof_track(p.I1, p.I2, pts, prm)
    f1, s1, _, _, a, made = oracle.rlof_track_gm(p.I1, p.I2, pts, prm)
    assert made and np.abs(oracle.gm_prior_flow(a, pts) - gt).max() < 0.2
    g0 = np.mean((s0 == oracle.TRACKED) & (np.hypot(*(f0 - gt).T) < 2.0))
    g1 = np.mean((s1 == oracle.TRACKED) & (np.hypot(*(f1 - gt).T) < 2.0))
    assert g1 >= g0 - 0.01
