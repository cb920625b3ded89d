"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs.

Bars: bit-exact integer window sums, key-point count and order; key-points within
1e-4 px; FP32 pyramid bit-exact, FP16 pyramid equal to the oracle value rounded to
FP16; tracked flow within 1e-2 px endpoint error on points that converge
(TRACKED) on both sides, with status agreement and the converged-point fraction
within tolerance asserted per workload (an iterative, discontinuous method can
take another branch on a few FP32 trajectories; those are counted and printed).
"""
import numpy as np
import pytest
import torch

import golden
import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_PTS = 1e-4
TOL_FLOW = 1e-2


@pytest.fixture(scope="module")
def dgf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_09971_gb300 as m
    m.load()
    return m


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------- detection

DETECT_CASES = [
    ((256, 128), 8, 8, 4),       # workload 1
    ((1242, 375), 7, 7, 3),      # workload 2
    ((1240, 376), 3, 3, 9),      # the paper's KITTI setting (no overlap: direct path)
    ((1280, 720), 8, 8, 2),
    ((1024, 436), 8, 8, 3),      # batch steps: shared-row column sums
    ((641, 483), 8, 8, 6),
    ((333, 211), 7, 7, 3),       # ragged, workload-2 window
    ((301, 155), 6, 6, 2),       # square window without a column-sum specialisation
    ((97, 61), 5, 9, 2),         # ragged tiles, non-square window
    ((200, 100), 64, 64, 1),     # largest window
    ((300, 90), 64, 33, 70),     # step beyond the window
    ((7, 7), 7, 7, 3),           # one window
]


@pytest.mark.parametrize("size,ww,wh,step", DETECT_CASES)
def test_detect_parity(dgf, size, ww, wh, step):
    W, H = size
    rng = np.random.default_rng(W * 7 + H)
    img = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    if W >= 256:
        img = synth.make_translation_pair(W, H, seed=W + H).I1
    pts_o, sums_o, _ = oracle.degraf_detect(img, ww, wh, step)
    pts_g, sums_g = dgf.detect(to_dev(img), ww, step, win_h=wh, with_sums=True)
    torch.cuda.synchronize()
    assert pts_g.shape[0] == pts_o.shape[0]
    assert np.array_equal(sums_g.cpu().numpy().astype(np.int64), sums_o[:, :4])
    err = np.abs(pts_g.cpu().numpy().astype(np.float64) - pts_o).max()
    assert err <= TOL_PTS
    # two correctly rounded FP32 steps (quotient, then origin): within one FP32 ulp
    g = pts_g.cpu().numpy()
    ulp = np.maximum(np.spacing(np.abs(pts_o).astype(np.float32)), np.spacing(np.abs(g))).astype(np.float64)
    diff = np.abs(g.astype(np.float64) - pts_o)
    assert np.all(diff <= ulp)
    # and the rounding budget itself: half an ulp of the result (the origin added) plus
    # half an ulp of the local centroid (its quotient, from exact FP32 operands or, for
    # sums from 2^24 on, from FP64), below one ulp of the window size
    assert np.all(diff <= 0.5 * ulp + float(np.spacing(np.float32(max(ww, wh)))))


@pytest.mark.parametrize("case", golden.degraf_cases(), ids=lambda c: c[0])
def test_detect_hand_worked_examples(dgf, case):
    """The kernel on the hand-worked key-points of tests/golden (Eq. 1-2: inverted and
    positive centroids, a tie, a grid of two windows): within the FP32 rounding budget
    of the exact fractions (half an ulp of the result plus one ulp of the window size)."""
    _, img, ww, wh, step, expect = case
    pts = dgf.detect(to_dev(img), ww, step, win_h=wh)
    torch.cuda.synchronize()
    g = pts.cpu().numpy()
    exact = np.array([[float(x), float(y)] for x, y in expect])
    assert g.shape == exact.shape
    ulp = np.maximum(np.spacing(np.abs(exact).astype(np.float32)), np.spacing(np.abs(g))).astype(np.float64)
    budget = 0.5 * ulp + float(np.spacing(np.float32(max(ww, wh))))
    assert np.all(np.abs(g.astype(np.float64) - exact) <= budget)


def test_detect_pitched_frame(dgf):
    H, W, pitch = 90, 150, 192
    rng = np.random.default_rng(2)
    big = rng.integers(0, 256, size=(H, pitch)).astype(np.uint8)
    dev = to_dev(big)[:, :W]
    assert dev.stride(0) == pitch
    pts_g = dgf.detect(dev, 7, 3).cpu().numpy()
    pts_o, _, _ = oracle.degraf_detect(big[:, :W].copy(), 7, 7, 3)
    assert np.abs(pts_g - pts_o).max() <= TOL_PTS


def test_detect_empty(dgf):
    pts = dgf.detect(torch.zeros((5, 40), dtype=torch.uint8, device="cuda"), 8, 4)
    assert pts.shape == (0, 2)


# ----------------------------------------------------------------- pyramid

@pytest.mark.parametrize("size,levels", [((256, 128), 3), ((1242, 375), 5), ((97, 61), 4),
                                         ((640, 480), 6), ((33, 1030), 5), ((9, 9), 1)])
@pytest.mark.parametrize("storage", [0, 1])
def test_pyramid_parity(dgf, size, levels, storage):
    W, H = size
    rng = np.random.default_rng(W + H + levels)
    img = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    ref = oracle.pyramid(img, levels)
    lay = dgf.pyramid_layout(W, H, levels, storage, True)
    buf = dgf.build_pyramid(to_dev(img), levels, storage, True)
    buf2 = dgf.build_pyramid(to_dev(img), levels, storage, False)
    lay2 = dgf.pyramid_layout(W, H, levels, storage, False)
    torch.cuda.synchronize()
    dt = np.float32 if storage == 0 else np.float16
    for l, (planes, planes2, oref) in enumerate(zip(dgf.pyramid_planes(buf, lay),
                                                    dgf.pyramid_planes(buf2, lay2), ref)):
        for g, o in zip(planes, oref):
            assert np.array_equal(g.cpu().numpy(), o.astype(dt)), f"level {l}"
        assert np.array_equal(planes2[0].cpu().numpy(), oref[0].astype(dt))


# ----------------------------------------------------------------- tracking

def compare_tracks(flow_g, st_g, flow_o, st_o):
    """Return (status agreement, converged-both mask, endpoint error per point)."""
    agree = np.mean(st_g == st_o)
    both = (st_g == oracle.TRACKED) & (st_o == oracle.TRACKED)
    e = np.hypot(*(flow_g.astype(np.float64) - flow_o).T)
    return agree, both, e


def run_both(dgf, I1, I2, pts64, prm_o, storage=0, lanes=0):
    H, W = I1.shape
    prm = dgf.RlofParams(levels=prm_o.levels, radius=prm_o.radius, max_iter=prm_o.max_iter,
                         model=prm_o.model, storage=storage, eps=prm_o.eps, hampel_a=prm_o.hampel_a,
                         hampel_b=prm_o.hampel_b, hampel_c=prm_o.hampel_c, min_eig=prm_o.min_eig)
    pts32 = pts64.astype(np.float32)
    prev = dgf.set_lanes(lanes)
    try:
        p1 = dgf.build_pyramid(to_dev(I1), prm.levels, storage, True)
        p2 = dgf.build_pyramid(to_dev(I2), prm.levels, storage, False)
        flow, st, it, il = dgf.track(p1, p2, W, H, to_dev(pts32), prm, with_iters=True, with_illum=True)
        torch.cuda.synchronize()
    finally:
        dgf.set_lanes(prev)
    fo, so, io, lo = oracle.rlof_track(I1, I2, pts32.astype(np.float64), prm_o)
    return (flow.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy(), il.cpu().numpy()), (fo, so, io, lo)


@pytest.mark.parametrize("config,model,lanes", [(1, 4, 0), (1, 2, 0), (1, 4, 16), (1, 4, 32),
                                                (2, 4, 0), (2, 2, 0)])
def test_track_parity_workloads(dgf, config, model, lanes):
    p = synth.make_pair(config)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=model)
    (fg, sg, ig, lg), (fo, so, io, lo) = run_both(dgf, p.I1, p.I2, pts, prm, lanes=lanes)
    agree, both, e = compare_tracks(fg, sg, fo, so)
    within = np.mean(e[both] <= TOL_FLOW)
    bad = np.flatnonzero(both & (e > TOL_FLOW))
    print(f"workload {config} model {model}: status agree {agree:.5f}, converged both {both.sum()}, "
          f"within {TOL_FLOW}: {within:.5f}, mismatches {bad[:10]} epe {e[bad[:10]]}")
    if config == 1:
        # the final status is a discontinuous function of rounding at the stopping
        # rule and the iteration cap: an FP32 restatement of the oracle already
        # flips 0.05-0.5% of statuses against FP64, so 3 of 1,953 may differ
        assert agree >= 0.998 and within == 1.0
    else:
        assert agree >= 0.99 and within >= 0.999
    # the lost-point outputs are zero on the GPU as in the oracle
    lost = (sg != oracle.TRACKED) & (sg != oracle.MAXITER)
    assert np.all(fg[lost] == 0)
    if model == 4:
        # illumination (gain m, offset c in intensity levels) on the points whose flow
        # agrees: the stopping rule bounds only the flow update, so c is looser
        ok = both & (e <= TOL_FLOW)
        assert np.abs(lg[ok, 0] - lo[ok, 0]).max() < 5e-3
        assert np.abs(lg[ok, 1] - lo[ok, 1]).max() < 0.5


@pytest.mark.parametrize("radius,levels,n,model", [(1, 1, 1, 2), (1, 2, 200, 2), (2, 2, 33, 4), (3, 3, 257, 4),
                                                   (6, 4, 100, 4), (7, 2, 65, 4), (4, 6, 500, 4), (5, 5, 3, 4)])
def test_track_parity_shapes(dgf, radius, levels, n, model):
    """Ragged point counts (group and block tails), every radius path, 1..6 levels,
    on a noise-free translation pair (supports this small make the 4-unknown
    problem ill-posed under noise, where FP32 and FP64 trajectories part ways)."""
    W, H = 640, 480
    p = synth.make_translation_pair(W, H, t=(2.5, -1.75), seed=radius * 10 + levels, noise_sigma=0.0)
    rng = np.random.default_rng(n)
    pts = np.stack([rng.uniform(0, W - 1, n), rng.uniform(0, H - 1, n)], 1)
    prm = oracle.RlofParams(levels=levels, radius=radius, model=model)
    (fg, sg, _, _), (fo, so, _, _) = run_both(dgf, p.I1, p.I2, pts, prm)
    agree, both, e = compare_tracks(fg, sg, fo, so)
    assert np.sum(sg != so) <= max(1, 0.01 * n)
    assert np.sum(e[both] > TOL_FLOW) <= max(1, 0.01 * both.sum())


@pytest.mark.parametrize("config", [1, 4])
def test_track_fp16_storage_error(dgf, config):
    """FP16 storage: endpoint error against the FP64 oracle is reported beside the
    FP32-storage error on the same points (no fixed bar; the converged points must
    stay close)."""
    p = synth.make_pair(config)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    if config == 4:
        pts = pts[::7]  # a sample of the 1242x375 pair keeps the oracle fast
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, model=4)
    res = {}
    for storage in (0, 1):
        (fg, sg, _, _), (fo, so, _, _) = run_both(dgf, p.I1, p.I2, pts, prm, storage=storage)
        agree, both, e = compare_tracks(fg, sg, fo, so)
        res[storage] = (agree, both, e)
        print(f"workload {config} storage {'f16' if storage else 'f32'}: status agree {agree:.4f}, "
              f"EPE vs FP64 oracle on converged points: mean {e[both].mean():.2e} median {np.median(e[both]):.2e} "
              f"p99 {np.percentile(e[both], 99):.2e} max {e[both].max():.2e}")
    agree, both, e = res[1]
    assert agree >= 0.97 and np.median(e[both]) < 0.05


def test_track_exact_shift(dgf):
    """Integer shift of a float-exact frame: both sides return the shift itself."""
    p = synth.make_pair(1)
    I1 = p.I1
    I2 = np.roll(np.roll(I1, -2, axis=0), 3, axis=1)
    pts = np.array([[x, y] for x in range(40, 216, 16) for y in range(30, 100, 12)], np.float64)
    prm = oracle.RlofParams(levels=3, radius=4, model=2, eps=1e-4, max_iter=60)
    (fg, sg, _, _), (fo, so, _, _) = run_both(dgf, I1, I2, pts, prm)
    ok = (sg == 0) & (so == 0)
    assert ok.mean() > 0.9
    assert np.abs(fg[ok] - [3, -2]).max() < 1e-2 and np.abs(fo[ok] - [3, -2]).max() < 1e-2


def test_track_empty_and_errors(dgf):
    z = torch.zeros((64, 64), dtype=torch.uint8, device="cuda")
    p1 = dgf.build_pyramid(z, 4, 0, True)
    p2 = dgf.build_pyramid(z, 4, 0, False)
    pts = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
    flow, st = dgf.track(p1, p2, 64, 64, pts, dgf.RlofParams(levels=4, radius=3))
    assert flow.shape == (0, 2)
    one = torch.zeros((1, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(dgf.DegrafError) as ei:  # coarsest level 8x8 < 2 r + 2 = 10
        dgf.track(p1, p2, 64, 64, one, dgf.RlofParams(levels=4, radius=4))
    assert ei.value.code == -3
    torch.cuda.synchronize()
