"""GPU test of rlof_track_pair_noalloc, the entry point for callers that cannot
allocate device memory while they track (it keeps the pyramids in a fixed scratch
array inside the library instead of a caller workspace).

It is called through the C ABI and must give exactly what rlof_track_many gives
with a caller workspace, on two calls in a row (the second call reuses the scratch
the first one left behind). The file is named to be collected last."""
import ctypes

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


def descriptor(dgf, f1, f2, win, step, out):
    from paper_1901_09971_gb300 import _abi
    H, W = f1.shape
    pts, flow, status, iters = out
    return _abi.PairC(f1.data_ptr(), f2.data_ptr(), W, H, f1.stride(0), win, step, pts.data_ptr(),
                      flow.data_ptr(), status.data_ptr(), iters.data_ptr())


def outputs(n):
    return (torch.empty((n, 2), dtype=torch.float32, device="cuda"),
            torch.empty((n, 2), dtype=torch.float32, device="cuda"),
            torch.empty(n, dtype=torch.uint8, device="cuda"),
            torch.empty(n, dtype=torch.uint8, device="cuda"))


def test_noalloc_matches_workspace_path_twice(dgf):
    lib = dgf.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [(synth.make_pair(2), dgf.RlofParams(levels=5, radius=5, max_iter=30, model=4)),
             (synth.make_pair(1), dgf.RlofParams(levels=3, radius=4, max_iter=30, model=4))]
    for pair, prm in cases:  # two calls in a row through the shared scratch
        f1 = torch.from_numpy(pair.I1).cuda()
        f2 = torch.from_numpy(pair.I2).cuda()
        n = dgf.degraf_count(pair.W, pair.H, pair.win, pair.step)
        got = outputs(n)
        desc = descriptor(dgf, f1, f2, pair.win, pair.step, got)
        c_prm = prm.c()
        rc = lib.rlof_track_pair_noalloc(ctypes.byref(desc), ctypes.byref(c_prm), stream)
        assert rc == 0, lib.dgf_strerror(rc)
        ref = dgf.BatchTracker([(pair.W, pair.H, pair.win, pair.step)], prm)
        ref.run([f1], [f2], use_graph=False)
        torch.cuda.synchronize()
        for a, b in zip(got, (ref.pts[0], ref.flow[0], ref.status[0], ref.iters[0])):
            assert torch.equal(a, b)
        assert (got[2] == 0).float().mean().item() > 0.5  # most points converge


def test_noalloc_rejects_frames_beyond_the_scratch(dgf):
    lib = dgf.load()
    from paper_1901_09971_gb300 import _abi
    W, H = 4096, 2048  # its two pyramids need far more than the fixed scratch
    n = dgf.degraf_count(W, H, 8, 8)
    fake = 1 << 20  # never dereferenced: the call returns before enqueuing anything
    desc = _abi.PairC(fake, fake, W, H, W, 8, 8, fake, fake, fake, 0)
    c_prm = dgf.RlofParams(levels=5, radius=5).c()
    assert lib.dgf_track_many_workspace(ctypes.byref(desc), 1, ctypes.byref(c_prm)) > (24 << 20)
    assert n > 0
    assert lib.rlof_track_pair_noalloc(ctypes.byref(desc), ctypes.byref(c_prm), None) == _abi.DGF_ERR_WORKSPACE
