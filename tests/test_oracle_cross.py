"""Pins of the oracle's adaptive cross-based support (Section 3 "Parameters": RLOF with
the adaptive cross based support region; the paper prints no formula, so the pins
are the geometry of the reading): inside a region separated from its surroundings
by more than tau the cross is the window's intersection with the region; a uniform
image keeps the whole window; the mask grows with tau and mirrors with the image;
a huge tau is the square support bit for bit; and at a motion boundary the cross
tracks the foreground where the square support is pulled toward the background."""
import numpy as np

import oracle

R = 4


def texture(x, y, phase):
    """Smooth, low-amplitude texture (|variation| <= 16), continuous in x and y."""
    return 8.0 * np.sin(0.7 * x + 0.3 * y + phase) + 8.0 * np.cos(0.4 * x - 0.9 * y + 2 * phase)


def two_region_frame(W, H, rect, shift=(0.0, 0.0)):
    """Background ~60 and a rectangle ~190 (x0, y0, x1, y1), the rectangle and its
    texture translated by shift."""
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    x0, y0, x1, y1 = rect
    inside = (x >= x0 + shift[0]) & (x < x1 + shift[0]) & (y >= y0 + shift[1]) & (y < y1 + shift[1])
    bg = 60.0 + texture(x, y, 0.0)
    fg = 190.0 + texture(x - shift[0], y - shift[1], 1.3)
    return np.clip(np.rint(np.where(inside, fg, bg)), 0, 255).astype(np.uint8)


RECT = (30, 20, 70, 52)


def test_cross_inside_a_region_is_its_intersection_with_the_window():
    img = two_region_frame(100, 80, RECT)
    x0, y0, x1, y1 = RECT
    for (cx, cy) in [(31, 21), (69, 51), (33, 40), (50, 22), (66, 48), (45, 35)]:
        m = oracle.cross_mask(img, cx, cy, R, 40.0)
        ky, kx = np.mgrid[-R:R + 1, -R:R + 1]
        expect = ((cx + kx >= x0) & (cx + kx < x1) & (cy + ky >= y0) & (cy + ky < y1)).astype(np.uint8)
        np.testing.assert_array_equal(m, expect, err_msg=f"centre {(cx, cy)}")


def test_row_arms_are_measured_from_their_own_arm_pixel():
    """Centre column 100 + 20 (y - cy), the rest of each row 20 above its centre-column
    pixel; tau 25. The vertical arm keeps rows cy - 1 .. cy + 1 (|20| <= 25, |40| > 25);
    each of those rows differs from its own arm pixel by 20 and is kept whole, although
    rows cy +- 1 lie 40 or 0 away from the centre pixel."""
    W, H, cx, cy = 21, 21, 10, 10
    y = np.arange(H)[:, None].repeat(W, 1).astype(np.float64)
    img = 100.0 + 20.0 * (y - cy)
    img[:, np.arange(W) != cx] += 20.0
    m = oracle.cross_mask(img, cx, cy, R, 25.0)
    expect = np.zeros((2 * R + 1, 2 * R + 1), np.uint8)
    expect[R - 1:R + 2, :] = 1
    np.testing.assert_array_equal(m, expect)


def test_uniform_image_keeps_the_whole_window_and_the_border_clamps():
    img = np.full((40, 50), 77, np.uint8)
    for c in [(25, 20), (0, 0), (49, 39)]:
        np.testing.assert_array_equal(oracle.cross_mask(img, *c, R, 1.0), 1)


def test_mask_grows_with_tau_and_mirrors_with_the_image():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, (60, 60)).astype(np.float64)
    for c in [(20.3, 31.7), (40.5, 12.2), (30.0, 30.0)]:
        prev = np.zeros((2 * R + 1, 2 * R + 1), np.uint8)
        for tau in (5.0, 20.0, 60.0, 120.0, 300.0):
            m = oracle.cross_mask(img, *c, R, tau)
            assert np.all(m >= prev) and m[R, R] == 1
            prev = m
        assert np.all(prev == 1)
        # mirrored image, mirrored centre (pixel centres at integers): mirrored mask
        cx, cy = int(np.floor(c[0] + 0.5)), int(np.floor(c[1] + 0.5))
        mirrored = oracle.cross_mask(img[:, ::-1].copy(), 59 - cx, cy, R, 60.0)
        np.testing.assert_array_equal(mirrored, oracle.cross_mask(img, cx, cy, R, 60.0)[:, ::-1])


def test_huge_tau_is_the_square_support():
    import synth
    p = synth.make_pair(1)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    a = oracle.rlof_track(p.I1, p.I2, pts, oracle.RlofParams(levels=3, radius=4, model=4))
    b = oracle.rlof_track(p.I1, p.I2, pts, oracle.RlofParams(levels=3, radius=4, model=4, cross_tau=1e9))
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_cross_support_tracks_a_motion_boundary():
    """A bright textured rectangle moves by (3.25, 1.5) px over a static background.
    Points inside the rectangle within 1..3 px of its edges: their square window
    straddles the boundary and is pulled toward zero motion; the cross keeps the
    rectangle's samples only."""
    t = (3.25, 1.5)
    W, H = 100, 80
    I1 = two_region_frame(W, H, RECT)
    I2 = two_region_frame(W, H, RECT, shift=t)
    x0, y0, x1, y1 = RECT
    pts = []
    for d in (1.2, 2.4, 3.1):
        for s in np.linspace(0.3, 0.7, 5):
            pts += [(x0 + d, y0 + s * (y1 - y0)), (x1 - 1 - d, y0 + s * (y1 - y0)),
                    (x0 + s * (x1 - x0), y0 + d), (x0 + s * (x1 - x0), y1 - 1 - d)]
    pts = np.array(pts)
    sq = oracle.rlof_track(I1, I2, pts, oracle.RlofParams(levels=2, radius=R, model=2))
    cr = oracle.rlof_track(I1, I2, pts, oracle.RlofParams(levels=2, radius=R, model=2, cross_tau=40.0))
    # MAXITER points are tracked (the cap was hit, the estimate stands)
    for f, st in (sq[:2], cr[:2]):
        assert np.all((st == oracle.TRACKED) | (st == oracle.MAXITER))
    e_sq = np.hypot(*(sq[0] - np.array(t)).T)
    e_cr = np.hypot(*(cr[0] - np.array(t)).T)
    print(f"median EPE: square {np.median(e_sq):.3f}, cross {np.median(e_cr):.3f}; within 0.5 px: "
          f"square {np.mean(e_sq < 0.5):.2f}, cross {np.mean(e_cr < 0.5):.2f}")
    assert np.median(e_cr) < 0.15 and np.median(e_sq) > 3 * np.median(e_cr)
    assert np.mean(e_cr < 0.5) >= 0.8 and np.mean(e_sq < 0.5) <= 0.6
