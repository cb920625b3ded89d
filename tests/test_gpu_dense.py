"""The composed DeGraF-Flow pipeline (DenseFlow): detection, pyramids, tracking with
the global-motion prior or plain or with the forward-backward filter, and EPIC
interpolation. Each stage has its own parity tests against the oracle; here the
pipeline must equal the same calls made one by one, bit for bit, and on the
256x128 translation pair the dense field must be as accurate as the sparse tracks
it interpolates."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dgf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_09971_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("mode", ["gm", "plain", "fb"])
def test_pipeline_equals_its_stages(dgf, mode):
    p = synth.make_pair(1)
    f1, f2 = torch.from_numpy(p.I1).cuda(), torch.from_numpy(p.I2).cuda()
    prm = dgf.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    gm = dgf.GmParams(extra_levels=0) if mode == "gm" else None
    fb = 1.0 if mode == "fb" else 0.0
    df = dgf.DenseFlow(p.W, p.H, p.win, p.step, prm, gm=gm, fb_max=fb)
    dense, (pts, flow, status) = df.run(f1, f2)
    torch.cuda.synchronize()
    q = dgf.detect(f1, p.win, p.step)
    p1 = dgf.build_pyramid(f1, prm.levels, dgf.F32, True)
    p2 = dgf.build_pyramid(f2, prm.levels, dgf.F32, mode == "fb")
    if mode == "gm":
        fl, st = dgf.track_gm(p1, p2, p.W, p.H, prm.levels, q, prm, gm)[:2]
    elif mode == "fb":
        fl, st, _ = dgf.track_fb(p1, p2, p.W, p.H, q, prm, fb)
    else:
        fl, st = dgf.track(p1, p2, p.W, p.H, q, prm)
    ref = dgf.epic_interpolate(f1, q, fl, st)
    torch.cuda.synchronize()
    assert torch.equal(pts, q) and torch.equal(flow, fl) and torch.equal(status, st)
    assert torch.equal(dense, ref)
    e = np.hypot(*(dense.cpu().numpy().astype(np.float64) - p.flow_gt).transpose(2, 0, 1))[~p.occluded]
    ok = status.cpu().numpy() == dgf.TRACKED
    es = np.hypot(*(flow.cpu().numpy()[ok].astype(np.float64) - np.array([3.5, -1.25])).T)
    print(f"{mode}: dense EPE median {np.median(e):.3f} px (sparse tracks {np.median(es):.3f} px)")
    # the frame-2 noise (sigma 2 levels) limits the tracks to about 0.3 px; the
    # interpolation must not add to that
    assert np.median(e) <= np.median(es) + 0.02


@pytest.mark.parametrize("mode", ["gm", "plain"])
def test_pipeline_replays_from_a_captured_cuda_graph(dgf, mode):
    """No stage of a run waits on the host (EPIC's labelling settles on the device),
    so a whole run captures into one CUDA graph; replayed on new frame contents it
    gives what an eager run gives, bit for bit, and no device-side failure is
    reported."""
    p, q = synth.make_pair(1), synth.make_pair(1, index=1)
    prm = dgf.RlofParams(levels=p.levels, radius=p.radius, max_iter=p.max_iter, model=4)
    gm = dgf.GmParams(extra_levels=0) if mode == "gm" else None
    df = dgf.DenseFlow(p.W, p.H, p.win, p.step, prm, gm=gm)
    f1, f2 = torch.from_numpy(p.I1).cuda(), torch.from_numpy(p.I2).cuda()
    dgf.device_status(reset=True)
    df.run(f1, f2)  # eager first: looks up the device status word
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        dense_g, (_, flow_g, status_g) = df.run(f1, f2)
    f1.copy_(torch.from_numpy(q.I1))
    f2.copy_(torch.from_numpy(q.I2))
    g.replay()
    torch.cuda.synchronize()
    got = (dense_g.clone(), flow_g.clone(), status_g.clone())
    ref = dgf.DenseFlow(p.W, p.H, p.win, p.step, prm, gm=gm)
    dense_e, (_, flow_e, status_e) = ref.run(f1, f2)
    torch.cuda.synchronize()
    assert torch.equal(got[0], dense_e) and torch.equal(got[1], flow_e) and torch.equal(got[2], status_e)
    assert dgf.device_status() == 0
