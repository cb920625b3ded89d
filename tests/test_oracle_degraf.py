"""Pins of the oracle's DeGraF detection (Section 2, Eq. 1-2) to facts the paper and
the mathematics fix: exact-integer brute force on tiny images, closed forms and
invariants. CPU only."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import golden


def brute_force(img, w, h, step):
    """Eq. 1-2 evaluated with Python integers and exact fractions."""
    H, W = img.shape
    out = []
    for oy in range(0, H - h + 1, step):
        for ox in range(0, W - w + 1, step):
            win = [[int(img[oy + i, ox + j]) for j in range(w)] for i in range(h)]
            m = max(max(r) for r in win)
            S = sum(sum(r) for r in win)
            Sn = sum(1 + m - v for r in win for v in r)
            if Sn > S:
                cx = Fraction(sum(j * (1 + m - win[i][j]) for i in range(h) for j in range(w)), Sn)
                cy = Fraction(sum(i * (1 + m - win[i][j]) for i in range(h) for j in range(w)), Sn)
            else:
                cx = Fraction(sum(j * win[i][j] for i in range(h) for j in range(w)), S)
                cy = Fraction(sum(i * win[i][j] for i in range(h) for j in range(w)), S)
            out.append((ox + cx, oy + cy, S, m, Sn > S))
    return out


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    W, H = int(rng.integers(1, 33)), int(rng.integers(1, 33))
    w, h = int(rng.integers(1, 10)), int(rng.integers(1, 10))
    step = int(rng.integers(1, 10))
    hi = int(rng.choice([2, 16, 256]))
    img = rng.integers(0, hi, size=(H, W)).astype(np.uint8)
    pts, sums, neg = oracle.degraf_detect(img, w, h, step)
    ref = brute_force(img, w, h, step)
    assert len(ref) == pts.shape[0] == oracle.degraf_count(W, H, w, h, step)
    for k, (cx, cy, S, m, use_neg) in enumerate(ref):
        assert abs(pts[k, 0] - float(cx)) <= 1e-12 * max(1, float(cx))
        assert abs(pts[k, 1] - float(cy)) <= 1e-12 * max(1, float(cy))
        assert sums[k, 0] == S and sums[k, 3] == m and bool(neg[k]) == use_neg


def test_grid_count_closed_form():
    # the paper's own KITTI setting (Section 3: w = h = 3, delta = 9) on 1240x376
    assert oracle.degraf_count(1240, 376, 3, 3, 9) == (((1240 - 3) // 9) + 1) * (((376 - 3) // 9) + 1)
    assert oracle.degraf_count(1242, 375, 7, 7, 3) == 50676
    assert oracle.degraf_count(256, 128, 8, 8, 4) == 1953
    assert oracle.degraf_count(1242, 375, 8, 8, 4) == 28428
    assert oracle.degraf_count(6, 100, 7, 7, 3) == 0
    assert oracle.degraf_count(7, 7, 7, 7, 3) == 1


def test_point_inside_its_window_and_row_major():
    rng = np.random.default_rng(7)
    img = rng.integers(0, 256, size=(40, 57)).astype(np.uint8)
    w, step = 7, 3
    pts, _, _ = oracle.degraf_detect(img, w, w, step)
    nu = (57 - w) // step + 1
    for k in range(pts.shape[0]):
        ox, oy = (k % nu) * step, (k // nu) * step
        assert ox <= pts[k, 0] <= ox + w - 1 and oy <= pts[k, 1] <= oy + w - 1


@pytest.mark.parametrize("value", [0, 1, 77, 255])
def test_constant_window_centre(value):
    img = np.full((9, 9), value, np.uint8)
    pts, sums, neg = oracle.degraf_detect(img, 8, 6, 1)
    assert np.allclose(pts[0], [3.5, 2.5], atol=1e-14)
    # S_pos + S_neg = n (1 + m) for every window
    n = 8 * 6
    assert np.all(sums[:, 0] + sums[:, 4] == n * (1 + sums[:, 3]))


def test_sum_invariant_and_selection_rule():
    rng = np.random.default_rng(3)
    img = rng.integers(0, 256, size=(50, 60)).astype(np.uint8)
    for (w, h, step) in [(7, 7, 3), (8, 8, 4), (3, 3, 9), (5, 2, 1)]:
        _, s, neg = oracle.degraf_detect(img, w, h, step)
        n = w * h
        assert np.all(s[:, 0] + s[:, 4] == n * (1 + s[:, 3]))
        assert np.all(s[:, 1] + s[:, 5] == (1 + s[:, 3]) * h * w * (w - 1) // 2)
        assert np.all(s[:, 2] + s[:, 6] == (1 + s[:, 3]) * w * h * (h - 1) // 2)
        # C_neg wins exactly when the mean intensity is below (1 + m) / 2
        assert np.array_equal(neg, 2 * s[:, 0] < n * (1 + s[:, 3]))


def test_mirror_symmetry():
    rng = np.random.default_rng(11)
    for _ in range(20):
        win = rng.integers(0, 256, size=(7, 7)).astype(np.uint8)
        p, _, n1 = oracle.degraf_detect(win, 7, 7, 1)
        q, _, n2 = oracle.degraf_detect(win[:, ::-1].copy(), 7, 7, 1)
        assert n1[0] == n2[0]
        assert abs(q[0, 0] - (6 - p[0, 0])) < 1e-12 and abs(q[0, 1] - p[0, 1]) < 1e-12
        r, _, n3 = oracle.degraf_detect(win[::-1, :].copy(), 7, 7, 1)
        assert n1[0] == n3[0] and abs(r[0, 1] - (6 - p[0, 1])) < 1e-12


def test_single_bright_pixel_closed_form():
    w, h, v, i0, j0 = 8, 6, 200, 4, 1
    win = np.zeros((h, w), np.uint8)
    win[i0, j0] = v
    p, s, neg = oracle.degraf_detect(win, w, h, 1)
    n = w * h
    Sn = n * (1 + v) - v
    assert neg[0] and s[0, 4] == Sn
    x = ((1 + v) * h * w * (w - 1) / 2 - j0 * v) / Sn
    y = ((1 + v) * w * h * (h - 1) / 2 - i0 * v) / Sn
    assert np.allclose(p[0], [x, y], atol=1e-13)


def test_ramp_closed_forms():
    w = 8
    j = np.arange(w)
    # bright ramp: C_pos is chosen, c_x = sum j (a j + b) / sum (a j + b)
    a, b = 5, 200
    win = np.tile(a * j + b, (w, 1)).astype(np.uint8)
    p, _, neg = oracle.degraf_detect(win, w, w, 1)
    sj, sj2 = w * (w - 1) / 2, (w - 1) * w * (2 * w - 1) / 6
    assert not neg[0]
    assert abs(p[0, 0] - (a * sj2 + b * sj) / (a * sj + b * w)) < 1e-13
    assert abs(p[0, 1] - (w - 1) / 2) < 1e-13
    # dark ramp 0..7: m = 7, weights 8 - j, C_neg is chosen at 84 / 36
    win = np.tile(j, (w, 1)).astype(np.uint8)
    p, _, neg = oracle.degraf_detect(win, w, w, 1)
    assert neg[0] and abs(p[0, 0] - 84 / 36) < 1e-13


def test_all_zero_window_uses_negative_centroid():
    p, s, neg = oracle.degraf_detect(np.zeros((5, 5), np.uint8), 5, 5, 1)
    assert neg[0] and s[0, 0] == 0 and np.allclose(p[0], [2, 2])


@pytest.mark.parametrize("case", golden.degraf_cases(), ids=lambda c: c[0])
def test_hand_worked_examples(case):
    """Key-points worked by hand from Eq. 1-2 (tests/golden/degraf_hand_worked.txt):
    an inverted-intensity centroid, a positive one, a tie (kept positive) and a grid of
    two windows; the oracle equals the exact fractions to FP64 rounding."""
    _, img, ww, wh, step, expect = case
    pts, _, _ = oracle.degraf_detect(img, ww, wh, step)
    assert pts.shape == (len(expect), 2)
    for (x, y), (ex, ey) in zip(pts, expect):
        assert abs(x - float(ex)) <= 1e-12 and abs(y - float(ey)) <= 1e-12
