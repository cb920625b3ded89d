"""GPU parity of the adjoints against the FP64 oracle's VJPs (which
tests/test_oracle_adjoint.py pins to finite differences).

The tracking adjoint is compared with the oracle VJP evaluated at the GPU's own
converged state (its flow, illumination and status, with the level-0 position in
the FP32 the kernel forms it in), so the difference measures the FP32 adjoint
arithmetic alone. Bars: DeGraF adjoint within 1e-5 of the
largest gradient magnitude (FP32 quotients of exact integer sums); tracking
adjoint within 1e-2 relative error in the 2-norm over the image and per pixel
within 1e-2 of the largest magnitude."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dgf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1901_09971_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("case", ["random", "workload"])
def test_degraf_backward_matches_oracle(dgf, case):
    rng = np.random.default_rng(7)
    if case == "random":
        img = rng.integers(0, 60, (61, 97)).astype(np.uint8)
        img[rng.random(img.shape) < 0.08] = 230
        w, h, step = 5, 4, 2
    else:
        img = synth.make_pair(1).I1
        w = h = 8
        step = 4
    H, W = img.shape
    n = dgf.degraf_count(W, H, w, step, win_h=h)
    g = rng.normal(size=(n, 2)).astype(np.float32)
    frame = torch.from_numpy(img).cuda()
    got = dgf.detect_backward(frame, w, step, torch.from_numpy(g).cuda(), win_h=h)
    torch.cuda.synchronize()
    ref = oracle.degraf_vjp(img.astype(np.float64), w, h, step, g.astype(np.float64))
    assert np.abs(got.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def test_degraf_autograd_accumulates(dgf):
    img = synth.make_pair(1).I1
    frame = torch.from_numpy(img).float().cuda().requires_grad_(True)
    pts = dgf.DeGraFDetect.apply(frame, 8, 4)
    w = torch.randn_like(pts)
    (pts * w).sum().backward()
    ref = oracle.degraf_vjp(img.astype(np.float64), 8, 8, 4, w.cpu().numpy().astype(np.float64))
    assert np.abs(frame.grad.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


def kernel_state_flow(pts, flow):
    """The flow at which the oracle's VJP evaluates the state the kernel differentiates.

    The adjoint kernel forms the level-0 position q = p + d in FP32 and takes the
    bilinear cell of each tap from it (an integer decided in floating point); the
    oracle forms p + d in FP64. A position within FP32 rounding below an integer
    column (558.99997 rounds to 559.0) then lands in the neighbouring cell on the
    two sides, and the interpolant's slopes, hence the point's whole VJP, differ.
    So the oracle gets d' = fl32(p + d) - p (exact in FP64): its p + d' is the
    kernel's position, and the comparison measures the adjoint's arithmetic alone.
    """
    P = np.asarray(pts, np.float32)
    return (P + np.asarray(flow, np.float32)).astype(np.float64) - P.astype(np.float64)


@pytest.mark.parametrize("model", [4, 2])
def test_rlof_backward_matches_oracle_vjp(dgf, model):
    """The differentiation workload's shape: a 1242x375 translation pair, step 4,
    3 levels, 9x9 support, random upstream weights w ~ N(0, 1) per point."""
    p = synth.make_pair(5)
    prm = dgf.RlofParams(levels=3, radius=4, max_iter=30, model=model)
    f1 = torch.from_numpy(p.I1).float().cuda().requires_grad_(True)
    f2 = torch.from_numpy(p.I2).float().cuda().requires_grad_(True)
    pts = dgf.detect(torch.from_numpy(p.I1).cuda(), p.win, p.step)
    flow, status = dgf.RLOFTrack.apply(f1, f2, pts, prm)
    rng = np.random.default_rng(model)
    w = torch.from_numpy(rng.normal(size=tuple(flow.shape)).astype(np.float32)).cuda()
    (flow * w).sum().backward()
    torch.cuda.synchronize()
    st = status.cpu().numpy()
    assert (st == 0).mean() > 0.7
    # oracle VJP at the GPU's converged state (illumination from a forward with it)
    pyr1 = dgf.build_pyramid(torch.from_numpy(p.I1).cuda(), 3, 0, True)
    pyr2 = dgf.build_pyramid(torch.from_numpy(p.I2).cuda(), 3, 0, False)
    fl, st2, il = dgf.track(pyr1, pyr2, p.W, p.H, pts, prm, with_illum=True)
    assert torch.equal(fl, flow) and torch.equal(st2, status)
    P = pts.cpu().numpy()
    r1, r2 = oracle.rlof_vjp(p.I1, p.I2, P, oracle.RlofParams(levels=3, radius=4, model=model),
                             kernel_state_flow(P, fl.cpu().numpy()), il.cpu().numpy(), st, w.cpu().numpy())
    for got, ref in ((f1.grad.cpu().numpy(), r1), (f2.grad.cpu().numpy(), r2)):
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"model {model}: relative 2-norm error {rel:.2e}")
        assert rel <= 1e-2
        assert np.abs(got - ref).max() <= 1e-2 * np.abs(ref).max()


def test_rlof_backward_skips_lost_points(dgf):
    p = synth.make_pair(1)
    prm = dgf.RlofParams(levels=3, radius=4)
    pyr1 = dgf.build_pyramid(torch.from_numpy(p.I1).cuda(), 3, 0, True)
    pyr2 = dgf.build_pyramid(torch.from_numpy(p.I2).cuda(), 3, 0, False)
    pts = dgf.detect(torch.from_numpy(p.I1).cuda(), 8, 4)
    flow, st, il = dgf.track(pyr1, pyr2, p.W, p.H, pts, prm, with_illum=True)
    lost = torch.full_like(st, 1)  # every point OOB: no gradient at all
    g1, g2 = dgf.track_backward(pyr1, pyr2, p.W, p.H, pts, prm, flow, il, lost, torch.ones_like(flow))
    torch.cuda.synchronize()
    assert not g1.any() and not g2.any()
