"""The FP32 restatement of the oracle (oracle/degraf_oracle.c compiled with the tracking
iteration in FP32) and the parity bars derived from it (tests/fp32_spread.py).

The restatement is a measuring device, not a reference: it takes the FP64 oracle's
steps with every tracking quantity rounded to FP32, so its departures from FP64 show
what FP32 rounding alone does to a discontinuous iteration (Section 2, "Sparse point
tracking": robust Gauss-Newton with a stopping rule and lost-point tests). These
tests pin it (it is FP32, it is the same iteration) and show that the bars built
from it accept a correct FP32 implementation and reject planted mistakes.
"""
import numpy as np
import pytest

import fp32_spread as fs
import oracle
import synth


def test_fp32_build_recovers_an_integer_shift_exactly():
    """Integer shift of a frame: the residual vanishes at the shift, a fixed point that
    FP32 represents exactly, so the FP32 build converges onto it as the FP64 one does
    (both stop within the stopping rule's eps of it)."""
    p = synth.make_pair(1)
    I2 = np.roll(np.roll(p.I1, -2, axis=0), 3, axis=1)
    pts = np.array([[x, y] for x in range(40, 216, 16) for y in range(30, 100, 12)], np.float64)
    prm = oracle.RlofParams(levels=3, radius=4, model=2, eps=1e-4, max_iter=60)
    for precision in ("f64", "f32"):
        f, s, _, _ = oracle.rlof_track(p.I1, I2, pts, prm, precision=precision)
        ok = s == oracle.TRACKED
        assert ok.mean() > 0.9
        assert np.abs(f[ok] - [3, -2]).max() < prm.eps, precision


def test_fp32_build_is_fp32_and_the_same_iteration():
    """On the 256x128 workload the FP32 build differs from FP64 by FP32 rounding (a
    median endpoint difference between 1e-7 and 1e-4 px, never zero everywhere) and
    otherwise takes the same path: statuses and iteration counts agree on almost
    every point."""
    p = synth.make_pair(1)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    pts = pts.astype(np.float32).astype(np.float64)
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    f64, s64, i64, _ = oracle.rlof_track(p.I1, p.I2, pts, prm)
    f32, s32, i32, _ = oracle.rlof_track(p.I1, p.I2, pts, prm, precision="f32")
    both = (s64 == oracle.TRACKED) & (s32 == oracle.TRACKED)
    e = np.hypot(*(f32 - f64).T)[both]
    print(f"FP32 vs FP64: median {np.median(e):.2e} px, max {e.max():.2e} px, status agree {np.mean(s32 == s64):.4f}, "
          f"iterations agree {np.mean(i32 == i64):.4f}")
    assert 1e-7 < np.median(e) < 1e-4 and e.max() <= fs.TOL_FLOW
    assert np.mean(s32 == s64) >= 0.995 and np.mean(i32[both] == i64[both]) >= 0.9
    # the flows are FP32 values
    assert np.array_equal(f32.astype(np.float32).astype(np.float64), f32)


@pytest.fixture(scope="module")
def c1():
    p = synth.make_pair(1)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    return p, pts.astype(np.float32), prm, fs.frames_spread(p.I1, p.I2, pts, prm)


@pytest.fixture(scope="module")
def c2():
    p = synth.make_pair(2)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    return p, pts.astype(np.float32), prm, fs.frames_spread(p.I1, p.I2, pts, prm)


@pytest.mark.parametrize("case", ["c1", "c2"])
def test_fp32_flip_rates_on_the_workloads(case, request):
    """The measured spread itself (printed; it sets the bars): FP32 rounding alone
    changes the final status of under 1% of the points and leaves fewer than 0.1% of
    the points TRACKED on both sides more than 1e-2 px apart, while points stopped by
    the iteration cap part ways far more often (they had not converged)."""
    p, pts, prm, sp = request.getfixturevalue(case)
    n = len(pts)
    print(f"{case}: n {n}, FP32 ensemble counts {sp.counts}, union {int(sp.union.sum())}, "
          f"tracked quantiles {sp.quantiles}")
    assert max(sp.counts["status"]) <= 0.01 * n
    assert max(sp.counts["tracked"]) <= 0.001 * n
    assert max(sp.counts["maxiter"]) <= 0.5 * np.sum(sp.status64 == oracle.MAXITER)
    assert sp.quantiles[50] < 1e-4


@pytest.mark.parametrize("case", ["c1", "c2"])
def test_bars_accept_another_correct_fp32_run(case, request):
    """A correct FP32 implementation that the ensemble does not include, the FP32
    restatement compiled with fused multiply-adds (another rounding pattern, as on
    a GPU), passes the bars; it is not bit-identical to the ensemble's member."""
    p, pts, prm, sp = request.getfixturevalue(case)
    q = pts.astype(np.float64)
    f, s, _, _ = oracle.rlof_track(p.I1, p.I2, q, prm, precision="f32fma")
    g, _, _, _ = oracle.rlof_track(p.I1, p.I2, q, prm, precision="f32")
    assert not np.array_equal(f, g)
    fs.check(f, s, sp, f"{case} FP32 with FMA")


@pytest.mark.parametrize("case", ["c1", "c2"])
@pytest.mark.parametrize("mistake", ["template 0.02 px off", "stopping rule 20x looser", "offset sign"])
def test_bars_reject_planted_mistakes(case, mistake, request):
    """Mistakes planted in an FP32 run of the oracle on the CPU fail the bars."""
    p, pts, prm, sp = request.getfixturevalue(case)
    I1, I2, q = p.I1, p.I2, pts.astype(np.float64)
    if mistake == "template 0.02 px off":
        q = q + np.array([0.02, 0.0])
    elif mistake == "stopping rule 20x looser":
        prm = oracle.RlofParams(**{**prm.__dict__, "eps": 20 * prm.eps})
    else:  # frame 2 offset by one intensity level the wrong way round: I2 - 1 instead of
        # the same frame; with the gain/offset model the offset absorbs it exactly, so
        # this plants it in the 2-unknown model where nothing absorbs it
        prm = oracle.RlofParams(**{**prm.__dict__, "model": 2})
        sp = fs.frames_spread(I1, I2, q, prm)
        I2 = np.clip(I2.astype(np.int32) - 1, 0, 255).astype(np.uint8)
    f, s, _, _ = oracle.rlof_track(I1, I2, q, prm, precision="f32")
    with pytest.raises(AssertionError):
        fs.check(f, s, sp, f"{case} {mistake}")


def _level_planes(W, H, levels):
    out, off = [], 0
    for (w, h) in oracle.level_sizes(W, H, levels):
        n = w * h
        out.append([(off + i * n, off + (i + 1) * n) for i in range(3)])
        off += 3 * n
    return out


def _keep_8_bits(x):
    """Round to 8 significant bits (bfloat16's precision), nearest even."""
    b = x.astype(np.float32).view(np.uint32)
    b = (b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return b.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("config", [1, 4])
def test_fp16_storage_bars_catch_a_one_level_rounding_mistake(config):
    """FP16 storage: tracking on pyramids rounded to FP16 (FP32 arithmetic) passes the
    bars against the FP64 oracle on exact pyramids; the same with level 1's intensity
    planes of both frames kept to 8 significant bits instead of FP16's 11 fails them."""
    p = synth.make_pair(config)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    if config == 4:
        pts = pts[::3]
    pts = pts.astype(np.float32).astype(np.float64)
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    sp = fs.frames_spread(p.I1, p.I2, pts, prm)
    b1 = fs.fp16_pyramid(p.I1, p.levels)
    b2 = fs.fp16_pyramid(p.I2, p.levels)
    f, s, _, _ = oracle.rlof_track_on_pyramids(b1, b2, p.W, p.H, pts, prm, precision="f32")
    fs.check(f, s, sp, f"workload {config} FP16 storage")
    a, b = _level_planes(p.W, p.H, p.levels)[1][0]
    e1, e2 = oracle.pyramid_buffer(p.I1, p.levels), oracle.pyramid_buffer(p.I2, p.levels)
    b1[a:b], b2[a:b] = _keep_8_bits(e1[a:b]), _keep_8_bits(e2[a:b])
    f, s, _, _ = oracle.rlof_track_on_pyramids(b1, b2, p.W, p.H, pts, prm, precision="f32")
    with pytest.raises(AssertionError):
        fs.check(f, s, sp, f"workload {config} FP16 storage with level 1 at 8 bits")


def test_pyramid_input_tracking_equals_frame_input_tracking():
    """rlof_track_on_pyramids on the oracle's own pyramids is rlof_track, bit for bit."""
    p = synth.make_pair(1)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    a = oracle.rlof_track(p.I1, p.I2, pts, prm)
    b = oracle.rlof_track_on_pyramids(oracle.pyramid_buffer(p.I1, p.levels), oracle.pyramid_buffer(p.I2, p.levels),
                                      p.W, p.H, pts, prm)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
