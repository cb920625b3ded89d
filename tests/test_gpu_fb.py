"""GPU parity of the forward-backward consistency filter (rlof_track_fb) against the
oracle's composition of two tracking passes: statuses (with FB_REJECTED) and
round-trip errors (within twice the flow tolerance where both sides have one)
meet bars derived from FP32 restatements of the oracle (tests/fp32_spread.py),
identical frames give an error of exactly 0, and the occluding patch is rejected
as in the oracle."""
import numpy as np
import pytest
import torch

import fp32_spread
import oracle
import synth
from test_oracle_fb import PATCH, PRM, T, occlusion_pair

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def dgf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_09971_gb300 as m
    m.load()
    return m


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_fb(dgf, I1, I2, pts, levels, radius, fb_max, model=4, storage=0):
    """GPU filter; also returns the backward pass's statuses from the workspace."""
    H, W = I1.shape
    n = len(pts)
    prm = dgf.RlofParams(levels=levels, radius=radius, model=model, storage=storage)
    p1 = dgf.build_pyramid(to_dev(I1), levels, storage, True)
    p2 = dgf.build_pyramid(to_dev(I2), levels, storage, True)
    ws = torch.empty(int(dgf.load().dgf_fb_workspace(n)), dtype=torch.uint8, device="cuda")
    f, s, e = dgf.track_fb(p1, p2, W, H, to_dev(pts.astype(np.float32)), prm, fb_max, workspace=ws)
    torch.cuda.synchronize()
    r256 = lambda v: (v + 255) // 256 * 256
    off = 2 * r256(8 * n)  # end points, backward flow, then backward statuses
    return f.cpu().numpy(), s.cpu().numpy(), e.cpu().numpy(), ws[off:off + n].cpu().numpy()


def test_fb_occlusion_pair_parity(dgf):
    I1, I2 = occlusion_pair()
    pts, _, _ = oracle.degraf_detect(I1, 8, 8, 4)
    pts = pts.astype(np.float32).astype(np.float64)
    q = pts + np.array(T)
    x0, y0, x1, y1 = PATCH
    on_patch = (q[:, 0] >= x0 - 1) & (q[:, 0] < x1 + 1) & (q[:, 1] >= y0 - 1) & (q[:, 1] < y1 + 1)
    for fb_max in (1.0, 0.0):
        fg, sg, eg, _ = run_fb(dgf, I1, I2, pts, 3, 4, fb_max)
        # points landing on the patch's fresh texture converge to arbitrary places,
        # differently in FP32 and FP64: the FP32 ensemble shows how often
        fp32_spread.check_fb(sg, eg, fp32_spread.fb_spread(I1, I2, pts, PRM, fb_max), f"occlusion pair fb_max {fb_max}")
        if fb_max > 0:
            fwd = np.isin(sg, [oracle.TRACKED, oracle.MAXITER, oracle.FB_REJECTED])
            assert np.mean(sg[fwd & on_patch] == oracle.FB_REJECTED) >= 0.95


def test_fb_driving_scene_parity(dgf):
    p = synth.make_pair(2)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    pts = pts.astype(np.float32).astype(np.float64)
    prm_o = oracle.RlofParams(levels=p.levels, radius=p.radius, model=4)
    fg, sg, eg, _ = run_fb(dgf, p.I1, p.I2, pts, p.levels, p.radius, 1.0)
    fp32_spread.check_fb(sg, eg, fp32_spread.fb_spread(p.I1, p.I2, pts, prm_o, 1.0), "driving scene fb_max 1")


def test_fb_identical_frames_zero_error(dgf):
    I1, _ = occlusion_pair()
    pts, _, _ = oracle.degraf_detect(I1, 8, 8, 4)
    fg, sg, eg, _ = run_fb(dgf, I1, I1, pts, 3, 4, 1.0)
    tr = (sg == oracle.TRACKED) | (sg == oracle.MAXITER)
    assert tr.mean() > 0.9 and np.all(eg[tr] == 0.0) and np.all(fg[tr] == 0.0)


def test_fb_fp16_storage(dgf):
    """FP16 pyramid storage: the filter meets the FP32 path's bars against the FP64
    oracle, and the occluding patch is still rejected."""
    I1, I2 = occlusion_pair()
    pts, _, _ = oracle.degraf_detect(I1, 8, 8, 4)
    pts = pts.astype(np.float32).astype(np.float64)
    fg, sg, eg, _ = run_fb(dgf, I1, I2, pts, 3, 4, 1.0, storage=dgf.F16)
    fp32_spread.check_fb(sg, eg, fp32_spread.fb_spread(I1, I2, pts, PRM, 1.0), "occlusion pair FP16 storage")
    q = pts + np.array(T)
    x0, y0, x1, y1 = PATCH
    on_patch = (q[:, 0] >= x0 - 1) & (q[:, 0] < x1 + 1) & (q[:, 1] >= y0 - 1) & (q[:, 1] < y1 + 1)
    fwd = np.isin(sg, [oracle.TRACKED, oracle.MAXITER, oracle.FB_REJECTED])
    assert np.mean(sg[fwd & on_patch] == oracle.FB_REJECTED) >= 0.95
