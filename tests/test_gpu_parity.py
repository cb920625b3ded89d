"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same
seeded inputs.

Bars: bit-exact integer window sums, key-point count and order; key-points within
1e-4 px; FP32 pyramid bit-exact, FP16 pyramid equal to the oracle value rounded to
FP16; tracked flow within 1e-2 px of the FP64 oracle on the points TRACKED or
MAXITER on both sides, and the same statuses, except where an FP32 restatement of
the oracle also parts from FP64: the number of disagreements of each kind is
bounded by what an ensemble of FP32 restatements shows on the same inputs, most of
the GPU's disagreements must be points where that ensemble disagrees too, and the
bulk of the tracked points must be as close to FP64 as the restatement's
(tests/fp32_spread.py states the bars).
"""
import numpy as np
import pytest
import torch

import fp32_spread as fs
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


@pytest.mark.parametrize("ww,step", [(8, 2), (8, 3), (8, 4), (8, 6), (7, 3), (6, 2), (5, 3)])
def test_detect_window_maximum_at_every_position(dgf, ww, step):
    """The window maximum m (the negative centroid's weights 1 + m - I) is exact
    wherever in the window it sits: low-valued frames (0..60) with sparse peaks
    (61..254) put a window's maximum at every row and byte position, odd or even,
    first or last, of the column-sum and packed-row paths."""
    rng = np.random.default_rng(ww * 100 + step)
    H, W = 157, 389
    img = rng.integers(0, 61, size=(H, W)).astype(np.uint8)
    peaks = rng.random((H, W)) < 0.02
    img[peaks] = rng.integers(61, 255, size=int(peaks.sum())).astype(np.uint8)
    pts_o, sums_o, _ = oracle.degraf_detect(img, ww, ww, step)
    pts_g, sums_g = dgf.detect(to_dev(img), ww, step, with_sums=True)
    torch.cuda.synchronize()
    sg = sums_g.cpu().numpy().astype(np.int64)
    assert np.array_equal(sg, sums_o[:, :4])
    m = sums_o[:, 3]
    assert np.unique(m).size > 100 and np.mean(m <= 60) > 0.05  # maxima of every kind occur
    assert np.abs(pts_g.cpu().numpy().astype(np.float64) - pts_o).max() <= TOL_PTS


def test_detect_pitched_frame(dgf):
    H, W, pitch = 90, 150, 192
    rng = np.random.default_rng(2)
    big = rng.integers(0, 256, size=(H, pitch)).astype(np.uint8)
    dev = to_dev(big)[:, :W]
    assert dev.stride(0) == pitch
    pts_g = dgf.detect(dev, 7, 3).cpu().numpy()
    pts_o, _, _ = oracle.degraf_detect(big[:, :W].copy(), 7, 7, 3)
    assert np.abs(pts_g - pts_o).max() <= TOL_PTS


@pytest.mark.parametrize("W,pitch", [(160, 192), (1024, 1024), (150, 192)])
def test_bulk_and_word_staging_agree_with_the_oracle(dgf, W, pitch):
    """Detection and the pyramid stage frame rows with bulk copies when the frame's
    base, pitch and width are multiples of 16 (the first two cases) and with word
    copies otherwise (the last): key-points, exact sums and FP32 pyramid planes equal
    the oracle's either way, and no block gave up waiting for its copies."""
    H = 90
    rng = np.random.default_rng(W + pitch)
    big = rng.integers(0, 256, size=(H, pitch)).astype(np.uint8)
    dev = to_dev(big)[:, :W]
    assert dev.stride(0) == pitch and dev.data_ptr() % 16 == 0
    dgf.device_status(reset=True)
    pts_g, sums_g = dgf.detect(dev, 7, 3, with_sums=True)
    pts_o, sums_o, _ = oracle.degraf_detect(big[:, :W].copy(), 7, 7, 3)
    assert np.array_equal(sums_g.cpu().numpy().astype(np.int64), sums_o[:, :4])
    assert np.abs(pts_g.cpu().numpy() - pts_o).max() <= TOL_PTS
    buf = dgf.build_pyramid(dev, 3, 0, True)
    lay = dgf.pyramid_layout(W, H, 3, 0, True)
    for planes, oref in zip(dgf.pyramid_planes(buf, lay), oracle.pyramid(big[:, :W].copy(), 3)):
        for g, o in zip(planes, oref):
            assert np.array_equal(g.cpu().numpy(), o.astype(np.float32))
    assert dgf.device_status() == 0


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
    # the replicated border around every plane holds the clamped values
    A, es = dgf.PYR_APRON, (4 if storage == 0 else 2)
    flat = buf.cpu().numpy().view(dt)
    for l, oref in enumerate(ref):
        Wl, Hl, p = lay["W"][l], lay["H"][l], lay["pitch"][l]
        ys, xs = np.meshgrid(np.arange(-A, Hl + A), np.arange(-A, Wl + A), indexing="ij")
        for key, o in zip(("off_I", "off_Ix", "off_Iy"), oref):
            padded = flat[lay[key][l] // es + ys * p + xs]
            assert np.array_equal(padded, np.pad(o, A, mode="edge").astype(dt)), f"level {l} {key} border"


# ----------------------------------------------------------------- tracking

def run_gpu(dgf, I1, I2, pts64, prm_o, storage=0, lanes=0):
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
    return flow.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy(), il.cpu().numpy()


@pytest.fixture(scope="module")
def workload_spreads():
    """FP64 oracle results and FP32 spreads of the two workloads, per model."""
    cache = {}

    def get(config, model):
        if (config, model) not in cache:
            p = synth.make_pair(config)
            pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
            pts = pts.astype(np.float32).astype(np.float64)
            prm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=model)
            cache[(config, model)] = (p, pts, prm, fs.frames_spread(p.I1, p.I2, pts, prm))
        return cache[(config, model)]
    return get


@pytest.mark.parametrize("config,model,lanes", [(1, 4, 0), (1, 2, 0), (1, 4, 16), (1, 4, 32),
                                                (2, 4, 0), (2, 2, 0)])
def test_track_parity_workloads(dgf, workload_spreads, config, model, lanes):
    p, pts, prm, sp = workload_spreads(config, model)
    fg, sg, ig, lg = run_gpu(dgf, p.I1, p.I2, pts, prm, lanes=lanes)
    fs.check(fg, sg, sp, f"workload {config} model {model} lanes {lanes}")
    # the lost-point outputs are zero on the GPU as in the oracle
    lost = (sg != oracle.TRACKED) & (sg != oracle.MAXITER)
    assert np.all(fg[lost] == 0)
    if model == 4:
        # illumination (gain m, offset c in intensity levels) on the points TRACKED on
        # both sides whose flows agree: the stopping rule bounds only the flow update,
        # so c is looser
        _, _, _, lo = oracle.rlof_track(p.I1, p.I2, pts, prm)
        e = np.hypot(*(fg.astype(np.float64) - sp.flow64).T)
        ok = (sg == oracle.TRACKED) & (sp.status64 == oracle.TRACKED) & (e <= fs.TOL_FLOW)
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
    pts = np.stack([rng.uniform(0, W - 1, n), rng.uniform(0, H - 1, n)], 1).astype(np.float32).astype(np.float64)
    prm = oracle.RlofParams(levels=levels, radius=radius, model=model)
    fg, sg, _, _ = run_gpu(dgf, p.I1, p.I2, pts, prm)
    fs.check(fg, sg, fs.frames_spread(p.I1, p.I2, pts, prm), f"radius {radius} levels {levels} n {n}")


@pytest.mark.parametrize("config", [1, 4])
def test_track_fp16_storage(dgf, config):
    """FP16 storage: against the FP64 oracle on exact pyramids the FP16-storage path
    meets the FP32 path's bars (the same spread, so no looser), and against the oracle
    run on the FP16-rounded pyramids it meets that computation's FP32 spread; the
    endpoint error of both storages against FP64 is printed."""
    p = synth.make_pair(config)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    if config == 4:
        pts = pts[::3]  # a third of the 1242x375 pair keeps the oracle ensembles fast
    pts = pts.astype(np.float32).astype(np.float64)
    prm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    sp = fs.frames_spread(p.I1, p.I2, pts, prm)
    res = {}
    for storage in (0, 1):
        fg, sg, _, _ = run_gpu(dgf, p.I1, p.I2, pts, prm, storage=storage)
        res[storage] = fs.check(fg, sg, sp, f"workload {config} storage {'f16' if storage else 'f32'} vs FP64")
    sp16 = fs.pyramids_spread(fs.fp16_pyramid(p.I1, p.levels), fs.fp16_pyramid(p.I2, p.levels), p.W, p.H, pts, prm)
    fs.check(fg, sg, sp16, f"workload {config} storage f16 vs the oracle on FP16-rounded pyramids")
    both = (sg == oracle.TRACKED) & (sp.status64 == oracle.TRACKED)
    e = np.hypot(*(fg.astype(np.float64) - sp.flow64).T)[both]
    print(f"workload {config} FP16 storage vs FP64: mean {e.mean():.2e} median {np.median(e):.2e} "
          f"p99 {np.percentile(e, 99):.2e} max {e.max():.2e} px")


def test_track_exact_shift(dgf):
    """Integer shift of a float-exact frame: both sides return the shift itself."""
    p = synth.make_pair(1)
    I1 = p.I1
    I2 = np.roll(np.roll(I1, -2, axis=0), 3, axis=1)
    pts = np.array([[x, y] for x in range(40, 216, 16) for y in range(30, 100, 12)], np.float64)
    prm = oracle.RlofParams(levels=3, radius=4, model=2, eps=1e-4, max_iter=60)
    fg, sg, _, _ = run_gpu(dgf, I1, I2, pts, prm)
    fo, so, _, _ = oracle.rlof_track(I1, I2, pts, prm)
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
