"""CPU checks of the C ABI: the library builds, loads and exports every entry point
include/degraf.h declares; host-side size queries and argument checks behave as
documented (these paths return before any CUDA call); the product package never
touches the oracle."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

import oracle
import paper_1901_09971_gb300 as dgf
from paper_1901_09971_gb300 import _abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "degraf.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_][a-z0-9_ ]*\**\s+\**([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declarations_are_exported():
    lib = dgf.load()
    names = declared_functions()
    assert "rlof_track" in names and "degraf_detect" in names and "pyramid_build" in names
    assert sorted(_abi.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    assert set(names) <= exported


def declared_arity():
    """Parameter count of every prototype in the header (comments removed)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for name, args in re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(([^()]*)\)\s*;", text):
        args = args.strip()
        out[name] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_argtypes_match_the_header():
    """The ctypes declarations pass exactly as many arguments as each prototype takes."""
    lib = dgf.load()
    arity = declared_arity()
    assert set(arity) == set(_abi.EXPORTS)
    for name in _abi.EXPORTS:
        assert len(getattr(lib, name).argtypes) == arity[name], name


def test_count_matches_oracle():
    for (W, H, w, h, s) in [(1242, 375, 7, 7, 3), (256, 128, 8, 8, 4), (1240, 376, 3, 3, 9), (5, 5, 7, 7, 1),
                            (64, 64, 64, 64, 1), (100, 37, 9, 2, 5)]:
        assert dgf.degraf_count(W, H, w, s, win_h=h) == oracle.degraf_count(W, H, w, h, s)
    assert dgf.load().dgf_degraf_count(100, 100, 65, 8, 1) == -1
    assert dgf.load().dgf_degraf_count(100, 100, 8, 8, 0) == -1


@pytest.mark.parametrize("storage", [0, 1])
def test_pyramid_layout(storage):
    es = 4 if storage == 0 else 2
    a = dgf.pyramid_layout(1242, 375, 5, storage, True)
    b = dgf.pyramid_layout(1242, 375, 5, storage, False)
    assert a["W"] == [1242, 621, 310, 155, 77] and a["H"] == [375, 187, 93, 46, 23]
    assert a["off_I"] == b["off_I"]  # intensity planes independent of the gradient planes
    A = _abi.PYR_APRON
    spans = []
    for l in range(5):
        p = a["pitch"][l]
        assert p * es % 128 == 0 and p >= a["W"][l] + 2 * A
        for off in (a["off_I"][l], a["off_Ix"][l], a["off_Iy"][l]):
            assert off % 128 == 0  # every row of the level starts on a 128-byte boundary
            first = off - (A * p + A) * es  # pixel (-A, -A) of the replicated border
            last = off + ((a["H"][l] + A - 1) * p + a["W"][l] + A) * es  # one past (W + A - 1, H + A - 1)
            assert first >= 0
            spans.append((first, last))
    spans.sort()
    assert all(e0 <= s1 for (_, e0), (s1, _) in zip(spans, spans[1:])) and spans[-1][1] <= a["bytes"]
    assert a["bytes"] > b["bytes"] and dgf.pyramid_bytes(1242, 375, 5, storage, True) == a["bytes"]
    assert dgf.pyramid_bytes(1242, 375, 7, storage, True) == 0
    assert dgf.pyramid_bytes(3, 3, 3, storage, True) == 0  # empty coarsest level


def test_strerror_and_defaults():
    lib = dgf.load()
    for code in range(0, -7, -1):
        assert lib.dgf_strerror(code)
    assert lib.dgf_strerror(-99) == b"unknown status"
    p = _abi.RlofParamsC()
    lib.dgf_rlof_params_default(ctypes.byref(p))
    assert (p.version, p.levels, p.radius, p.max_iter, p.model) == (_abi.RLOF_PARAMS_VERSION, 3, 4, 30, 4)
    assert abs(p.eps - 1e-3) < 1e-9 and (p.hampel_a, p.hampel_b, p.hampel_c) == (8.0, 16.0, 32.0)
    assert p.cross_tau == 0.0  # square support unless asked for
    # a negative threshold or a stale parameter version is rejected before any launch
    fake = ctypes.c_void_p(1 << 20)
    bad = dgf.RlofParams(cross_tau=-1.0).c()
    assert lib.rlof_track(fake, fake, 64, 64, fake, 10, ctypes.byref(bad), fake, fake, None, None, None) == -1
    old = dgf.RlofParams().c()
    old.version = 1
    assert lib.rlof_track(fake, fake, 64, 64, fake, 10, ctypes.byref(old), fake, fake, None, None, None) == -1


def test_host_side_errors_return_before_launch():
    lib = dgf.load()
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every call below fails its checks first
    p = dgf.RlofParams(levels=5, radius=5).c()
    bad = dgf.RlofParams(levels=5, radius=5).c()
    bad.version = 7
    assert lib.rlof_track(fake, fake, 1242, 375, fake, 10, ctypes.byref(bad), fake, fake, None, None, None) == -1
    bad = dgf.RlofParams(levels=5, radius=9).c()
    assert lib.rlof_track(fake, fake, 1242, 375, fake, 10, ctypes.byref(bad), fake, fake, None, None, None) == -1
    bad = dgf.RlofParams(hampel_a=8, hampel_b=16, hampel_c=16).c()
    assert lib.rlof_track(fake, fake, 1242, 375, fake, 10, ctypes.byref(bad), fake, fake, None, None, None) == -1
    # coarsest level 38x11 is lower than 2r + 2 = 12
    deep = dgf.RlofParams(levels=6, radius=5).c()
    assert lib.rlof_track(fake, fake, 1242, 375, fake, 10, ctypes.byref(deep), fake, fake, None, None, None) == -3
    # null outputs with points to track
    assert lib.rlof_track(fake, fake, 1242, 375, fake, 10, ctypes.byref(p), None, fake, None, None, None) == -1
    # nothing to track: success without a launch
    assert lib.rlof_track(None, None, 1242, 375, None, 0, ctypes.byref(p), None, None, None, None, None) == 0
    # pyramid buffer too small / misaligned
    assert lib.pyramid_build(fake, 1242, 375, 1242, 5, 0, 1, fake, 1024, None) == -2
    assert lib.pyramid_build(fake, 1242, 375, 1242, 5, 0, 1, ctypes.c_void_p((1 << 20) + 64), 1 << 30, None) == -1
    assert lib.pyramid_build(fake, 1242, 375, 1000, 5, 0, 1, fake, 1 << 30, None) == -1
    # detection: bad window, and an empty grid (no launch)
    assert lib.degraf_detect(fake, 100, 100, 100, 0, 7, 3, fake, None, None) == -1
    assert lib.degraf_detect(fake, 5, 5, 5, 7, 7, 3, None, None, None) == 0


def test_batch_host_checks_return_before_launch():
    lib = dgf.load()
    prm = dgf.RlofParams(levels=3, radius=4).c()
    pairs = (_abi.PairC * 2)()
    fake = 1 << 20
    for i, (W, H, step) in enumerate([(640, 480, 2), (1242, 375, 6)]):
        pairs[i] = _abi.PairC(fake, fake, W, H, W, 8, step, fake, fake, fake, 0)
    need = lib.dgf_track_many_workspace(pairs, 2, ctypes.byref(prm))
    b = [dgf.pyramid_bytes(W, H, 3, 0, True) + dgf.pyramid_bytes(W, H, 3, 0, False)
         for (W, H) in [(640, 480), (1242, 375)]]
    assert need == sum(b)
    # short workspace, misaligned workspace, bad pair, bad parameters: no launch
    assert lib.rlof_track_many(pairs, 2, ctypes.byref(prm), ctypes.c_void_p(fake), need - 1, 7, 0, None) == -2
    assert lib.rlof_track_many(pairs, 2, ctypes.byref(prm), ctypes.c_void_p(fake + 8), need, 7, 0, None) == -1
    bad = (_abi.PairC * 1)(_abi.PairC(fake, 0, 640, 480, 640, 8, 2, fake, fake, fake, 0))
    assert lib.dgf_track_many_workspace(bad, 1, ctypes.byref(prm)) == 0
    deep = dgf.RlofParams(levels=6, radius=5).c()
    assert lib.rlof_track_many(pairs, 2, ctypes.byref(deep), ctypes.c_void_p(fake), 1 << 40, 7, 0, None) == -3
    assert lib.rlof_track_many(pairs, 0, ctypes.byref(prm), None, 0, 7, 0, None) == 0
    assert lib.rlof_track_many(pairs, 2, ctypes.byref(prm), ctypes.c_void_p(fake), need, 8, 0, None) == -1


def test_batch_tracker_run_needs_bound_frames():
    bt = dgf.BatchTracker([(64, 48, 8, 4)], dgf.RlofParams(levels=2, radius=4), device="cpu")
    with pytest.raises(ValueError):
        bt.run()


def test_gm_host_checks_return_before_launch():
    lib = dgf.load()
    prm = dgf.RlofParams(levels=3, radius=4).c()
    g = _abi.GmParamsC()
    lib.dgf_gm_params_default(ctypes.byref(g))
    assert (g.stride, g.extra_levels, g.iters, g.c0, g.c_min) == (4, 2, 8, 32.0, 2.0)
    n = 1000
    need = lib.dgf_gm_workspace(n, ctypes.byref(g))
    n_sub = (n + 3) // 4
    assert need >= 256 + 8 * n_sub + n_sub and need % 256 == 0
    fake = ctypes.c_void_p(1 << 20)

    def call(W=640, H=480, pyr_levels=5, ws=need, gp=g, p=prm, npts=n):
        return lib.rlof_track_gm(fake, fake, W, H, pyr_levels, fake, npts, ctypes.byref(p), ctypes.byref(gp), fake,
                                 fake, None, None, fake, ws, None)

    assert call(ws=need - 1) == -2                 # short workspace
    assert call(pyr_levels=4) == -1                # pyramid shallower than levels + extra_levels
    assert call(pyr_levels=7) == -1                # beyond DGF_MAX_LEVELS
    assert call(W=100, H=40) == -3                 # first pass's coarsest level too small
    assert call(npts=0) == 0
    bad = _abi.GmParamsC(_abi.GM_PARAMS_VERSION, 0, 2, 8, 32.0, 2.0)  # stride 0
    assert call(gp=bad) == -1 and lib.dgf_gm_workspace(n, ctypes.byref(bad)) == 0
    bad = _abi.GmParamsC(_abi.GM_PARAMS_VERSION, 4, 2, 0, 32.0, 2.0)  # no iterations
    assert call(gp=bad) == -1
    bad = _abi.GmParamsC(_abi.GM_PARAMS_VERSION, 4, 2, 8, 32.0, 0.0)  # c_min 0
    assert call(gp=bad) == -1


def test_fb_host_checks_return_before_launch():
    lib = dgf.load()
    prm = dgf.RlofParams(levels=3, radius=4).c()
    fake = ctypes.c_void_p(1 << 20)
    W, H, n = 640, 480, 1000
    full = dgf.pyramid_bytes(W, H, 3, 0, True)
    ws = lib.dgf_fb_workspace(n)
    assert ws >= 2 * 8 * n + n and ws % 256 == 0 and lib.dgf_fb_workspace(-1) == 0

    def call(nbytes=full, wsb=ws, fb_max=1.0, npts=n):
        return lib.rlof_track_fb(fake, fake, nbytes, W, H, fake, npts, ctypes.byref(prm), fb_max, fake, fake, None,
                                 fake, wsb, None)

    assert call(nbytes=dgf.pyramid_bytes(W, H, 3, 0, False)) == -1  # frame 2 pyramid without gradients
    assert call(wsb=ws - 1) == -2
    assert call(fb_max=-1.0) == -1
    assert call(npts=0) == 0


def test_epic_host_checks_return_before_launch():
    lib = dgf.load()
    d = _abi.EpicParamsC()
    assert lib.dgf_epic_params_default(ctypes.byref(d)) == 0
    assert (d.version, d.k, d.model, d.cost_base, d.cost_gain, d.a, d.min_spread) == \
        (_abi.EPIC_PARAMS_VERSION, 128, 1, 4, 1, 0.1, 1.0)
    py = dgf.EpicParams()
    assert (py.k, py.model, py.cost_base, py.cost_gain, py.a, py.min_spread) == (128, 1, 4, 1, 0.1, 1.0)
    fake = ctypes.c_void_p(1 << 20)
    W, H, n = 640, 480, 5000
    ws = lib.dgf_epic_workspace(W, H, n)
    assert ws % 256 == 0 and ws >= W * H * (8 + 4 + 4 * 12) + n * 48
    assert lib.dgf_epic_workspace(5000, 3193, 10) == 0 and lib.dgf_epic_workspace(W, H, -1) == 0
    assert lib.dgf_epic_workspace(W, H, 1 << 24) == 0

    def call(prm=None, w=W, h=H, pitch=W, npts=n, wsb=ws, pts=fake, dense=fake, dbg=None):
        prm = prm if prm is not None else dgf.EpicParams().c()
        return lib.epic_interpolate(fake, w, h, pitch, pts, fake, fake, npts, ctypes.byref(prm), dense,
                                    ctypes.byref(dbg) if dbg is not None else None, fake, wsb, None)

    assert call(wsb=ws - 1) == -2
    assert call(w=5000, h=3193) == -1 and call(pitch=W - 1) == -1 and call(npts=-1) == -1
    assert call(pts=None) == -1 and call(dense=ctypes.c_void_p((1 << 20) + 4)) == -1
    for bad in (dict(k=0), dict(k=257), dict(model=2), dict(cost_base=0), dict(cost_gain=33), dict(a=-1.0),
                dict(min_spread=float("nan"))):
        assert call(prm=dgf.EpicParams(**bad).c()) == -1, bad
    v = dgf.EpicParams().c()
    v.version = 99
    assert call(prm=v) == -1
    half = _abi.EpicDebugC(None, None, fake.value, None, None, None, None, None)  # knn_idx without knn_dist
    assert call(dbg=half) == -1


def test_dense_flow_rejects_prior_with_filter():
    """DenseFlow runs the global-motion prior or the forward-backward filter, not both;
    the check comes before any device allocation."""
    with pytest.raises(ValueError):
        dgf.DenseFlow(64, 48, 8, 4, dgf.RlofParams(), gm=dgf.GmParams(), fb_max=1.0, device="cpu")


def test_adjoint_rejects_the_cross_support():
    """The tracking adjoint is defined for the square support only."""
    lib = dgf.load()
    fake = ctypes.c_void_p(1 << 20)
    prm = dgf.RlofParams(cross_tau=20.0).c()
    ws = lib.dgf_rlof_backward_workspace(64, 64)
    rc = lib.rlof_track_backward(fake, fake, 64, 64, fake, 10, ctypes.byref(prm), fake, fake, fake, fake, None, fake,
                                 ws, fake, fake, 64, None)
    assert rc == -1


@pytest.mark.parametrize("which", ["pts", "flow", "illum", "grad_flow", "grad_illum", "grad_I1", "grad_I2"])
def test_adjoint_rejects_misaligned_float_arrays(which):
    """A float array off its 4-byte alignment is refused before any launch."""
    lib = dgf.load()
    good, bad = ctypes.c_void_p(1 << 20), ctypes.c_void_p((1 << 20) + 2)
    prm = dgf.RlofParams().c()
    ws = lib.dgf_rlof_backward_workspace(64, 64)
    a = {k: good for k in ("pts", "flow", "illum", "grad_flow", "grad_illum", "grad_I1", "grad_I2")}
    a[which] = bad
    rc = lib.rlof_track_backward(good, good, 64, 64, a["pts"], 10, ctypes.byref(prm), a["flow"], a["illum"], good,
                                 a["grad_flow"], a["grad_illum"], good, ws, a["grad_I1"], a["grad_I2"], 64, None)
    assert rc == -1
    if which in ("pts", "grad_I1"):  # the detection adjoint's float arrays: grad_pts and grad_img
        rc = lib.degraf_detect_backward(good, 64, 64, 64, 8, 8, 4, bad if which == "pts" else good, good,
                                        lib.dgf_degraf_backward_workspace(64, 64, 8, 8, 4),
                                        bad if which == "grad_I1" else good, 64, None)
        assert rc == -1


def test_missing_library_raises_instead_of_falling_back(monkeypatch, tmp_path):
    """Without libdegraf.so every entry point raises: there is no CPU path to fall back to."""
    from paper_1901_09971_gb300 import _abi, build
    missing = str(tmp_path / "libdegraf.so")
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(build, "LIB", missing)
    monkeypatch.setattr(build, "build", lambda *a, **k: missing)  # a build that produced nothing
    with pytest.raises(RuntimeError, match="libdegraf.so not found"):
        _abi.load()
    with pytest.raises(RuntimeError):
        dgf.degraf_count(64, 64, 8, 4)
    with pytest.raises(RuntimeError):
        dgf.pyramid_bytes(64, 64, 3)


def test_product_package_never_loads_the_oracle():
    code = ("import sys; sys.path.insert(0, %r); import paper_1901_09971_gb300 as d; d.load(); "
            "import bench; assert 'oracle' not in sys.modules, 'oracle imported'" % ROOT)
    subprocess.run([sys.executable, "-c", code], check=True, cwd=ROOT)
    pkg = os.path.join(ROOT, "paper_1901_09971_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert "oracle" not in open(os.path.join(dirpath, f)).read().lower(), f


def test_probe_host_checks_and_flop_count():
    """The measurement probes reject bad sizes before any launch; the FP32 probe's FLOP
    count is 2 per FMA: 8 chains x 8 steps per trip, two FMAs per packed lane."""
    lib = dgf.load()
    assert lib.dgf_fp32_probe(None, 1, 256, 1, 1, None) == _abi.DGF_ERR_ARG
    assert lib.dgf_fp32_probe(ctypes.c_void_p(16), 1, 300, 1, 1, None) == _abi.DGF_ERR_ARG
    assert lib.dgf_fp32_probe(ctypes.c_void_p(16), 1, 48, 1, 1, None) == _abi.DGF_ERR_ARG
    assert lib.dgf_fp32_probe_flops(3, 256, 10, 0) == 2 * 64 * 10 * 256 * 3
    assert lib.dgf_fp32_probe_flops(3, 256, 10, 1) == 4 * 64 * 10 * 256 * 3
    assert lib.dgf_epic_exp_neg(None, None, -1, None) == _abi.DGF_ERR_ARG
    assert lib.dgf_epic_exp_neg(None, None, 5, None) == _abi.DGF_ERR_ARG
    assert lib.dgf_epic_exp_neg(None, None, 0, None) == _abi.DGF_OK
    assert lib.dgf_device_status(None, 0) == _abi.DGF_ERR_ARG


def test_noalloc_scratch_size_matches_the_header():
    text = open(HEADER).read()
    assert re.search(r"#define DGF_PYR_APRON (\d+)", text).group(1) == str(_abi.PYR_APRON)
    m = re.search(r"#define DGF_NOALLOC_SCRATCH_BYTES \((\d+)u << (\d+)\)", text)
    assert m and int(m.group(1)) << int(m.group(2)) == _abi.DGF_NOALLOC_SCRATCH_BYTES


def test_rlof_track_function_rejects_keypoints_that_require_grad():
    """The flow's derivative with respect to the key-points is not computed, so the
    autograd Function refuses key-points that require grad (before any launch)."""
    import torch
    f = torch.zeros((64, 64))
    pts = torch.zeros((3, 2), requires_grad=True)
    with pytest.raises(ValueError, match="key-points require grad"):
        dgf.RLOFTrack.apply(f, f, pts, dgf.RlofParams(levels=2, radius=3))
