"""GPU parity of tracking with the global-motion prior (rlof_track_gm) against the
oracle's reading (Section 3, RLOF(IM-GM)): the affine fit on the GPU's own first
pass equals the oracle's fit on the same tracks; the first and the main pass meet
the tracking bars against the oracle run with the same inputs; the two-pass result
tracks a 37 px motion as well as plain tracking tracks a small one; and a fit that
cannot be formed leaves plain tracking bit for bit."""
import numpy as np
import pytest
import torch

import fp32_spread
import oracle
import synth

pytestmark = pytest.mark.gpu

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


def bars(fg, sg, I1, I2, pts64, oprm, label, init_flow=None):
    """The tracking bars (derived from FP32 restatements of the oracle, see
    tests/fp32_spread.py) for a pass started from init_flow."""
    return fp32_spread.check(fg, sg, fp32_spread.frames_spread(I1, I2, pts64, oprm, init_flow=init_flow), label)


def run_gm(dgf, p, pts32, prm, gm):
    pyr_levels = prm.levels + gm.extra_levels
    p1 = dgf.build_pyramid(to_dev(p.I1), pyr_levels, prm.storage, True)
    p2 = dgf.build_pyramid(to_dev(p.I2), pyr_levels, prm.storage, False)
    n = pts32.shape[0]
    ws = torch.zeros(dgf.gm_workspace_bytes(n, gm), dtype=torch.uint8, device="cuda")
    flow, status, a, made = dgf.track_gm(p1, p2, p.W, p.H, pyr_levels, to_dev(pts32), prm, gm, workspace=ws)
    torch.cuda.synchronize()
    n_sub = (n + gm.stride - 1) // gm.stride
    st_off = (256 + 8 * n_sub + 255) // 256 * 256
    sub_flow = ws[256:256 + 8 * n_sub].view(torch.float32).reshape(n_sub, 2).cpu().numpy()
    sub_status = ws[st_off:st_off + n_sub].cpu().numpy()
    return (flow.cpu().numpy(), status.cpu().numpy(), a.cpu().numpy(), int(made.item()), sub_flow, sub_status,
            (p1, p2, pyr_levels))


def test_gm_large_motion_parity_and_quality(dgf):
    t = (37.3, -21.6)
    p = synth.make_translation_pair(640, 360, t=t, seed=11)
    pts, _, _ = oracle.degraf_detect(p.I1, 8, 8, 8)
    pts32 = pts.astype(np.float32)
    pts64 = pts32.astype(np.float64)
    prm = dgf.RlofParams(levels=3, radius=4, model=4)
    gm = dgf.GmParams()
    fg, sg, a, made, sub_flow, sub_status, _ = run_gm(dgf, p, pts32, prm, gm)
    assert made == 1
    oprm = oracle.RlofParams(levels=3, radius=4, model=4)
    deep = oracle.RlofParams(levels=3 + gm.extra_levels, radius=4, model=4)
    sub = pts64[::gm.stride]
    # first pass against the oracle on the same points and deeper pyramid
    bars(sub_flow, sub_status, p.I1, p.I2, sub, deep, "first pass")
    # the fit on the GPU's first-pass tracks
    a_o, made_o = oracle.gm_fit_affine(sub, sub_flow, sub_status, gm.iters, gm.c0, gm.c_min)
    assert made_o
    d = np.abs(oracle.gm_prior_flow(a, pts64) - oracle.gm_prior_flow(a_o, pts64)).max()
    print(f"affine: GPU {a}, oracle {a_o}, prior difference {d:.2e} px")
    assert d < 1e-6
    # main pass against the oracle started from the same prior
    bars(fg, sg, p.I1, p.I2, pts64, oprm, "main pass", init_flow=oracle.gm_prior_flow(a, pts64))
    # the two-pass oracle reaches the same motion
    _, _, _, _, a2, made2 = oracle.rlof_track_gm(p.I1, p.I2, pts64, oprm)
    assert made2 and np.abs(oracle.gm_prior_flow(a, pts64) - oracle.gm_prior_flow(a2, pts64)).max() < 0.05
    # quality: the right basin for the large motion as often as plain tracking on a small one
    gt = np.array(t)
    visible = np.all((pts64 + gt >= 6) & (pts64 + gt <= np.array([p.W, p.H]) - 7), axis=1)
    good = np.mean(((sg == oracle.TRACKED) & (np.hypot(*(fg - gt).T) < 2.0))[visible])
    small = synth.make_translation_pair(640, 360, t=(3.5, -1.25), seed=11)
    fs, ss = dgf.track(dgf.build_pyramid(to_dev(small.I1), 3, 0, True), dgf.build_pyramid(to_dev(small.I2), 3, 0, False),
                       small.W, small.H, to_dev(pts32), prm)
    fs, ss = fs.cpu().numpy(), ss.cpu().numpy()
    good_small = np.mean((ss == oracle.TRACKED) & (np.hypot(*(fs - np.array([3.5, -1.25])).T) < 2.0))
    print(f"good: gm {good:.3f}, small-motion plain {good_small:.3f}")
    assert good > 0.95 * good_small


@pytest.mark.parametrize("config,extra", [(1, 1), (2, 0)])  # 5 levels of 256x128 would be 16x8
def test_gm_workloads_parity(dgf, config, extra):
    """The small-motion and the driving-scene workloads with the prior: main pass
    against the oracle run from the GPU's prior."""
    p = synth.make_pair(config)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    pts32 = pts.astype(np.float32)
    prm = dgf.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    gm = dgf.GmParams(extra_levels=extra)
    fg, sg, a, made, _, _, _ = run_gm(dgf, p, pts32, prm, gm)
    assert made == 1
    oprm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    pts64 = pts32.astype(np.float64)
    bars(fg, sg, p.I1, p.I2, pts64, oprm, f"workload {config} with the prior",
         init_flow=oracle.gm_prior_flow(a, pts64))


def test_gm_without_a_fit_is_plain_tracking(dgf):
    """A first pass of one point cannot form a fit: the prior stays the identity
    motion and the main pass equals plain tracking bit for bit."""
    p = synth.make_pair(1)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    pts32 = pts.astype(np.float32)
    prm = dgf.RlofParams(levels=p.levels, radius=p.radius, model=4)
    gm = dgf.GmParams(stride=len(pts32) + 1, extra_levels=0)
    fg, sg, a, made, _, _, (p1, p2, _) = run_gm(dgf, p, pts32, prm, gm)
    assert made == 0 and np.array_equal(a, [1, 0, 0, 0, 1, 0])
    f0, s0 = dgf.track(p1, p2, p.W, p.H, to_dev(pts32), prm)
    np.testing.assert_array_equal(fg, f0.cpu().numpy())
    np.testing.assert_array_equal(sg, s0.cpu().numpy())


def test_gm_with_cross_support_driving_scene(dgf):
    """The paper's tracking configuration (Section 3: RLOF(IM-GM) with the adaptive
    cross-based support) on the driving scene: the fit on the GPU's own first pass
    equals the oracle's fit on the same tracks, and the main pass meets the cross
    support's bars for this scene (tau 20) against the oracle run from the same prior."""
    p = synth.make_pair(2)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    pts32 = pts.astype(np.float32)
    pts64 = pts32.astype(np.float64)
    tau = 20.0
    prm = dgf.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4, cross_tau=tau)
    gm = dgf.GmParams(extra_levels=0)
    fg, sg, a, made, sub_flow, sub_status, _ = run_gm(dgf, p, pts32, prm, gm)
    assert made == 1
    a_o, made_o = oracle.gm_fit_affine(pts64[::gm.stride], sub_flow, sub_status, gm.iters, gm.c0, gm.c_min)
    assert made_o
    assert np.abs(oracle.gm_prior_flow(a, pts64) - oracle.gm_prior_flow(a_o, pts64)).max() < 1e-6
    oprm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4, cross_tau=tau)
    bars(fg, sg, p.I1, p.I2, pts64, oprm, "prior + cross support", init_flow=oracle.gm_prior_flow(a, pts64))


def test_gm_fp16_storage(dgf):
    """FP16 pyramid storage with the prior on the 256x128 pair: the fitted motion is
    within 0.01 px of the FP32-storage fit and the main pass meets the FP32 path's
    bars against the FP64 oracle run from the same prior."""
    p = synth.make_pair(1)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    pts32 = pts.astype(np.float32)
    pts64 = pts32.astype(np.float64)
    gm = dgf.GmParams(extra_levels=1)
    res = {}
    for storage in (dgf.F32, dgf.F16):
        prm = dgf.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4, storage=storage)
        res[storage] = run_gm(dgf, p, pts32, prm, gm)
    a32, a16 = res[dgf.F32][2], res[dgf.F16][2]
    d = np.abs(oracle.gm_prior_flow(a16, pts64) - oracle.gm_prior_flow(a32, pts64)).max()
    print(f"prior difference FP16 vs FP32 storage: {d:.2e} px")
    assert res[dgf.F16][3] == 1 and d < 0.01
    fg, sg = res[dgf.F16][0], res[dgf.F16][1]
    oprm = oracle.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    bars(fg, sg, p.I1, p.I2, pts64, oprm, "FP16 storage main pass", init_flow=oracle.gm_prior_flow(a16, pts64))
