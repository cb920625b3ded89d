"""The torch binding refuses caller buffers the kernels would read or write past:
wrong shapes, dtypes, pyramid layouts and gradient planes raise ValueError before
any launch, and the library is left usable."""
import pytest
import torch

pytestmark = pytest.mark.gpu

W, H, WIN, STEP, LEVELS = 96, 64, 8, 4, 3


@pytest.fixture(scope="module")
def dgf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_09971_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def scene(dgf):
    g = torch.Generator().manual_seed(5)
    f1 = torch.randint(0, 256, (H, W), generator=g, dtype=torch.uint8).cuda()
    f2 = torch.roll(f1, shifts=(1, 2), dims=(0, 1)).contiguous()
    prm = dgf.RlofParams(levels=LEVELS, radius=4)
    pts = dgf.detect(f1, WIN, STEP)
    p1 = dgf.build_pyramid(f1, LEVELS, dgf.F32, True)
    p2 = dgf.build_pyramid(f2, LEVELS, dgf.F32, True)
    return f1, f2, prm, pts, p1, p2


def test_detect_out_checked(dgf, scene):
    f1 = scene[0]
    n = dgf.degraf_count(W, H, WIN, STEP)
    with pytest.raises(ValueError):
        dgf.detect(f1, WIN, STEP, out=torch.empty((n - 1, 2), device="cuda"))
    with pytest.raises(ValueError):
        dgf.detect(f1, WIN, STEP, out=torch.empty((n, 2), dtype=torch.float64, device="cuda"))
    out = torch.empty((n, 2), device="cuda")
    assert dgf.detect(f1, WIN, STEP, out=out).data_ptr() == out.data_ptr()


def test_pyramid_out_checked(dgf, scene):
    f1 = scene[0]
    nbytes = dgf.pyramid_bytes(W, H, LEVELS, dgf.F32, True)
    with pytest.raises(ValueError):  # a float buffer's element count is not its size in bytes
        dgf.build_pyramid(f1, LEVELS, dgf.F32, True, out=torch.empty(nbytes, dtype=torch.float32, device="cuda"))


def test_track_points_and_outputs_checked(dgf, scene):
    _, _, prm, pts, p1, p2 = scene
    n = pts.shape[0]
    with pytest.raises(ValueError):  # flattened points: n floats, not n pairs
        dgf.track(p1, p2, W, H, pts.reshape(-1)[:n].contiguous(), prm)
    with pytest.raises(ValueError):
        dgf.track(p1, p2, W, H, pts[::2], prm)  # not contiguous
    short = (torch.empty((n - 1, 2), device="cuda"), torch.empty(n, dtype=torch.uint8, device="cuda"), None, None)
    with pytest.raises(ValueError):
        dgf.track(p1, p2, W, H, pts, prm, out=short)
    flow, status = dgf.track(p1, p2, W, H, pts, prm)
    torch.cuda.synchronize()
    assert flow.shape == (n, 2) and status.shape == (n,)


def test_track_pyramid_layouts_checked(dgf, scene):
    f1, _, prm, pts, p1, p2 = scene
    deeper = dgf.build_pyramid(f1, LEVELS + 1, dgf.F32, True)
    with pytest.raises(ValueError):  # frame 1's gradients sit at other offsets in a deeper pyramid
        dgf.track(deeper, p2, W, H, pts, prm)
    f2_only = dgf.build_pyramid(scene[1], LEVELS, dgf.F32, False)
    flow, _ = dgf.track(p1, f2_only, W, H, pts, prm)  # frame 2's intensities: any superset layout
    flow2, _ = dgf.track(p1, p2, W, H, pts, prm)
    torch.cuda.synchronize()
    assert torch.equal(flow, flow2)
    with pytest.raises(ValueError):  # the backward pass reads frame 2's gradients
        dgf.track_fb(p1, f2_only, W, H, pts, prm, 1.0)
    with pytest.raises(ValueError):
        dgf.track_gm(p1, p2, W, H, LEVELS + 1, pts, prm, dgf.GmParams(extra_levels=1))


def test_epic_inputs_checked(dgf, scene):
    f1, _, prm, pts, p1, p2 = scene
    flow, status = dgf.track(p1, p2, W, H, pts, prm)
    with pytest.raises(ValueError):
        dgf.epic_interpolate(f1, pts, flow[:-1].contiguous(), status)
    with pytest.raises(ValueError):
        dgf.epic_interpolate(f1, pts, flow, status[:-1].contiguous())
    with pytest.raises(ValueError):
        dgf.epic_interpolate(f1, pts, flow, status, out=torch.empty((H, W, 2), dtype=torch.float64, device="cuda"))
    dense = dgf.epic_interpolate(f1, pts, flow, status)
    torch.cuda.synchronize()
    assert dense.shape == (H, W, 2) and torch.isfinite(dense).all()


def test_backward_planes_checked(dgf, scene):
    f1, _, prm, pts, p1, p2 = scene
    flow, status, illum = dgf.track(p1, p2, W, H, pts, prm, with_illum=True)
    g = torch.ones_like(flow)
    with pytest.raises(ValueError):  # transposed gradient plane
        dgf.track_backward(p1, p2, W, H, pts, prm, flow, illum, status, g,
                           grad_I1=torch.zeros((W, H), device="cuda"))
    with pytest.raises(ValueError):  # planes whose rows are spaced differently
        dgf.track_backward(p1, p2, W, H, pts, prm, flow, illum, status, g,
                           grad_I2=torch.zeros((H, W + 32), device="cuda")[:, :W])
    with pytest.raises(ValueError):
        dgf.track_backward(p1, p2, W, H, pts, prm, flow, illum, status, g[:-1])
    with pytest.raises(ValueError):
        dgf.detect_backward(f1, WIN, STEP, g[:-1])
    g1, g2 = dgf.track_backward(p1, p2, W, H, pts, prm, flow, illum, status, g)
    torch.cuda.synchronize()
    assert torch.isfinite(g1).all() and torch.isfinite(g2).all()


def test_host_buffer_path_equals_the_device_path(dgf):
    """track_pair / HostPairTracker (host frames in, host results out) give exactly
    what BatchTracker gives on device copies of the same frames, call after call;
    track_pair keeps its device buffers between calls of one size (the second call
    leaves the device's free memory unchanged) and hands back tensors the caller owns."""
    import numpy as np
    import synth
    pair = synth.make_pair(1)
    prm = dgf.RlofParams(levels=3, radius=4, max_iter=30, model=4)
    ref = dgf.BatchTracker([(pair.W, pair.H, pair.win, pair.step)], prm)
    ref.run([torch.from_numpy(pair.I1).cuda()], [torch.from_numpy(pair.I2).cuda()], use_graph=False)
    want = [t[0].cpu() for t in (ref.pts, ref.flow, ref.status)]
    first = dgf.track_pair(pair.I1, pair.I2, pair.win, pair.step, prm)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    second = dgf.track_pair(pair.I1, pair.I2, pair.win, pair.step, prm)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    for got in (first, second):
        for a, b in zip(got, want):
            assert not a.is_cuda and torch.equal(a, b)
    assert first[1].data_ptr() != second[1].data_ptr()  # the caller's own copies
    ht = dgf.HostPairTracker(pair.W, pair.H, pair.win, pair.step, prm)
    out = (torch.empty((ht.n, 2)).pin_memory(), torch.empty((ht.n, 2)).pin_memory(),
           torch.empty(ht.n, dtype=torch.uint8).pin_memory())
    for _ in range(2):
        got = ht.run(torch.from_numpy(pair.I1).pin_memory(), np.ascontiguousarray(pair.I2), out=out)
        assert all(g.data_ptr() == o.data_ptr() for g, o in zip(got, out))
        for a, b in zip(got, want):
            assert torch.equal(a, b)
    with pytest.raises(ValueError):
        ht.run(pair.I1[:, :-1], pair.I2)
    with pytest.raises(ValueError):
        ht.run(pair.I1, pair.I2, out=(out[0][:-1], out[1], out[2]))
