"""Pins of the oracle's forward-backward consistency filter (not in the paper's text;
a common filter on sparse tracks before interpolation): identical frames give a
round-trip error of exactly 0; on a translation pair with an occluding patch the
filter rejects the points that land on the patch and keeps the visible ones; lost
points carry an infinite error; without a threshold no status changes."""
import numpy as np

import oracle
import synth

T = (3.5, -1.25)
PATCH = (120, 60, 200, 140)  # x0, y0, x1, y1 of fresh texture pasted into frame 2


def occlusion_pair(W=320, H=200):
    I1 = synth.render(W, H, 21)
    I2 = synth.render(W, H, 21, shift=T)
    fresh = synth.render(W, H, 99)
    x0, y0, x1, y1 = PATCH
    I2[y0:y1, x0:x1] = fresh[y0:y1, x0:x1]
    q = lambda a: np.clip(np.rint(a), 0, 255).astype(np.uint8)  # frames are 8-bit like every workload
    return q(I1), q(I2)


PRM = oracle.RlofParams(levels=3, radius=4, model=4)


def test_identical_frames_round_trip_exactly():
    I1, _ = occlusion_pair()
    pts, _, _ = oracle.degraf_detect(I1, 8, 8, 4)
    f, s, err = oracle.rlof_track_fb(I1, I1, pts, PRM, 1.0)
    tr = (s == oracle.TRACKED) | (s == oracle.MAXITER)
    assert tr.mean() > 0.9
    assert np.all(err[tr] == 0.0) and np.all(f[tr] == 0.0)


def test_occluded_points_are_rejected_visible_points_kept():
    I1, I2 = occlusion_pair()
    pts, _, _ = oracle.degraf_detect(I1, 8, 8, 4)
    f, s, err = oracle.rlof_track_fb(I1, I2, pts, PRM, 1.0)
    q = pts + np.array(T)
    x0, y0, x1, y1 = PATCH
    on_patch = (q[:, 0] >= x0 - 1) & (q[:, 0] < x1 + 1) & (q[:, 1] >= y0 - 1) & (q[:, 1] < y1 + 1)
    near = (q[:, 0] >= x0 - 6) & (q[:, 0] < x1 + 6) & (q[:, 1] >= y0 - 6) & (q[:, 1] < y1 + 6)
    fwd = (s == oracle.TRACKED) | (s == oracle.MAXITER) | (s == oracle.FB_REJECTED)
    rej_occ = np.mean(s[fwd & on_patch] == oracle.FB_REJECTED)
    rej_vis = np.mean(s[fwd & ~near] == oracle.FB_REJECTED)
    print(f"rejected: on the patch {rej_occ:.3f}, visible {rej_vis:.3f}; "
          f"visible median error {np.median(err[fwd & ~near]):.4f} px")
    assert (fwd & on_patch).sum() > 100
    assert rej_occ >= 0.95 and rej_vis <= 0.03
    assert np.median(err[fwd & ~near]) < 0.05  # 8-bit frames: 0.011 px measured (0.0003 px unquantised)


def test_lost_points_have_infinite_error_and_no_threshold_changes_nothing():
    I1, I2 = occlusion_pair()
    pts, _, _ = oracle.degraf_detect(I1, 8, 8, 4)
    pts = np.vstack([pts, [[-50.0, 10.0]]])  # outside the frame: lost
    f0, s0, _, _ = oracle.rlof_track(I1, I2, pts, PRM)
    f, s, err = oracle.rlof_track_fb(I1, I2, pts, PRM, 0.0)
    np.testing.assert_array_equal(s, s0)
    np.testing.assert_array_equal(f, f0)
    lost = ~((s0 == oracle.TRACKED) | (s0 == oracle.MAXITER))
    assert lost[-1] and np.all(np.isinf(err[lost]))
    assert not np.any(np.isnan(err))  # finite, or infinite where the backward pass lost the point
