"""GPU test of rlof_track_pair_noalloc, the entry point for callers that cannot
allocate device memory while they track (it keeps the pyramids in a fixed scratch
array inside the library instead of a caller workspace).

It is called through the C ABI and must give exactly what rlof_track_many gives
with a caller workspace, on calls in a row (each reuses the scratch the previous
one left behind), with FP32 and FP16 pyramids, up to the largest frame the scratch
holds; a second call must leave the device's free memory unchanged; and the first
frame size whose pyramids need more than the scratch is rejected before anything
runs, with real buffers passed so that a regression in that check could only give
wrong outputs, never touch memory the test does not own. The file is named to be
collected last."""
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


def descriptor(f1, f2, win, step, out):
    from paper_1901_09971_gb300 import _abi
    H, W = f1.shape
    pts, flow, status, iters = out
    return _abi.PairC(f1.data_ptr(), f2.data_ptr(), W, H, f1.stride(0), win, step, pts.data_ptr(),
                      flow.data_ptr(), status.data_ptr(), iters.data_ptr())


def outputs(n, fill=None):
    out = (torch.empty((n, 2), dtype=torch.float32, device="cuda"),
           torch.empty((n, 2), dtype=torch.float32, device="cuda"),
           torch.empty(n, dtype=torch.uint8, device="cuda"),
           torch.empty(n, dtype=torch.uint8, device="cuda"))
    if fill is not None:
        for t in out:
            t.view(torch.uint8).fill_(fill)
    return out


_QUERY_BUF = []


def workspace_bytes(lib, W, H, win, step, prm):
    """dgf_track_many_workspace of one W x H pair: a host-side size query that reads
    no buffer (it still wants non-null, aligned pointers, so it gets a real one)."""
    from paper_1901_09971_gb300 import _abi
    if not _QUERY_BUF:
        _QUERY_BUF.append(torch.zeros(256, dtype=torch.uint8, device="cuda"))
    a = _QUERY_BUF[0].data_ptr()
    desc = _abi.PairC(a, a, W, H, W, win, step, a, a, a, a)
    c_prm = prm.c()
    n = int(lib.dgf_track_many_workspace(ctypes.byref(desc), 1, ctypes.byref(c_prm)))
    assert n > 0, "size query rejected its arguments"
    return n


def noalloc_call(dgf, f1, f2, win, step, prm, out):
    lib = dgf.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    desc = descriptor(f1, f2, win, step, out)
    c_prm = prm.c()
    return lib.rlof_track_pair_noalloc(ctypes.byref(desc), ctypes.byref(c_prm), stream)


def reference(dgf, f1, f2, win, step, prm):
    H, W = f1.shape
    ref = dgf.BatchTracker([(W, H, win, step)], prm)
    ref.run([f1], [f2], use_graph=False)
    return ref.pts[0], ref.flow[0], ref.status[0], ref.iters[0]


def cases(dgf):
    big = synth.make_translation_pair(1280, 720, seed=77)
    big.win, big.step = 8, 3
    return [
        ("1242x375, 5 FP32 levels", synth.make_pair(2), dgf.RlofParams(levels=5, radius=5, max_iter=30, model=4)),
        ("256x128, 3 FP32 levels", synth.make_pair(1), dgf.RlofParams(levels=3, radius=4, max_iter=30, model=4)),
        ("1280x720, 5 FP32 levels", big, dgf.RlofParams(levels=5, radius=5, max_iter=30, model=4)),
        ("1280x720, 5 FP16 levels", big, dgf.RlofParams(levels=5, radius=5, max_iter=30, model=4, storage=dgf.F16)),
    ]


def test_noalloc_matches_workspace_path_calls_in_a_row(dgf):
    from paper_1901_09971_gb300 import _abi
    lib = dgf.load()
    for name, pair, prm in cases(dgf):  # calls in a row through the shared scratch
        assert workspace_bytes(lib, pair.W, pair.H, pair.win, pair.step, prm) <= _abi.DGF_NOALLOC_SCRATCH_BYTES, name
        f1 = torch.from_numpy(pair.I1).cuda()
        f2 = torch.from_numpy(pair.I2).cuda()
        n = dgf.degraf_count(pair.W, pair.H, pair.win, pair.step)
        got = outputs(n, fill=0xA5)
        rc = noalloc_call(dgf, f1, f2, pair.win, pair.step, prm, got)
        assert rc == 0, lib.dgf_strerror(rc)
        ref = reference(dgf, f1, f2, pair.win, pair.step, prm)
        torch.cuda.synchronize()
        for a, b in zip(got, ref):
            assert torch.equal(a, b), name
        assert (got[2] == 0).float().mean().item() > 0.5, name  # most points converge


def test_a_second_call_allocates_nothing(dgf):
    """Free device memory is the same before and after a call once one call has run
    (the first call on a device may make the runtime load the library's module)."""
    pair = synth.make_pair(2)
    prm = dgf.RlofParams(levels=5, radius=5, max_iter=30, model=4)
    f1 = torch.from_numpy(pair.I1).cuda()
    f2 = torch.from_numpy(pair.I2).cuda()
    out = outputs(dgf.degraf_count(pair.W, pair.H, pair.win, pair.step))
    assert noalloc_call(dgf, f1, f2, pair.win, pair.step, prm, out) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert noalloc_call(dgf, f1, f2, pair.win, pair.step, prm, out) == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_the_first_size_beyond_the_scratch(dgf):
    """At 720 rows, 5 FP32 levels: the widest frame whose pyramids fit is tracked like
    the workspace path; one column more is rejected with DGF_ERR_WORKSPACE and the
    outputs (real buffers, filled with a sentinel) are left untouched."""
    from paper_1901_09971_gb300 import _abi
    lib = dgf.load()
    prm = dgf.RlofParams(levels=5, radius=5, max_iter=30, model=4)
    H, win, step = 720, 8, 8
    limit = _abi.DGF_NOALLOC_SCRATCH_BYTES
    W = next(w for w in range(1280, 4096) if workspace_bytes(lib, w + 1, H, win, step, prm) > limit)
    assert workspace_bytes(lib, W + 1, H, win, step, prm) > limit >= workspace_bytes(lib, W, H, win, step, prm)
    print(f"widest {H}-row frame in the scratch: {W} columns")
    big = synth.make_translation_pair(W + 1, H, seed=5)
    for width, accepted in ((W, True), (W + 1, False)):
        f1 = torch.from_numpy(np.ascontiguousarray(big.I1[:, :width])).cuda()
        f2 = torch.from_numpy(np.ascontiguousarray(big.I2[:, :width])).cuda()
        n = dgf.degraf_count(width, H, win, step)
        got = outputs(n, fill=0x5A)
        rc = noalloc_call(dgf, f1, f2, win, step, prm, got)
        torch.cuda.synchronize()
        if accepted:
            assert rc == 0, lib.dgf_strerror(rc)
            for a, b in zip(got, reference(dgf, f1, f2, win, step, prm)):
                assert torch.equal(a, b)
        else:
            assert rc == _abi.DGF_ERR_WORKSPACE
            for t in got:
                assert bool((t.view(torch.uint8) == 0x5A).all())
