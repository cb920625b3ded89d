"""GPU parity of the batched pipeline (rlof_track_many): every pair's key-points,
flow, status and iteration counts equal those of the single-pair path bit for bit
(same arithmetic, only the scheduling differs), and the single-pair path is held
to the FP64 oracle by the same bars as tests/test_gpu_parity.py."""
import numpy as np
import pytest
import torch

import fp32_spread as fs
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


def frames_for(specs, seed0):
    out = []
    for i, (W, H, win, step) in enumerate(specs):
        p = synth.make_translation_pair(W, H, seed=seed0 + i)
        out.append((p.I1, p.I2))
    return out


def single_pair_path(dgf, I1, I2, win, step, prm):
    f1 = torch.from_numpy(I1).cuda()
    f2 = torch.from_numpy(I2).cuda()
    H, W = I1.shape
    tr = dgf.PairTracker(W, H, win, step, prm)
    pts, flow, st, it = tr.run(f1, f2)
    torch.cuda.synchronize()
    return pts.cpu().numpy(), flow.cpu().numpy(), st.cpu().numpy(), it.cpu().numpy()


def run_batch(dgf, specs, frames, prm, use_graph):
    bt = dgf.BatchTracker(specs, prm)
    d1 = [torch.from_numpy(a).cuda() for a, _ in frames]
    d2 = [torch.from_numpy(b).cuda() for _, b in frames]
    bt.run(d1, d2, use_graph=use_graph)
    torch.cuda.synchronize()
    return bt, d1, d2


def assert_same_as_single(dgf, bt, frames, specs, prm):
    for i, ((I1, I2), (W, H, win, step)) in enumerate(zip(frames, specs)):
        pts, flow, st, it = single_pair_path(dgf, I1, I2, win, step, prm)
        assert np.array_equal(bt.pts[i].cpu().numpy(), pts), f"pair {i} points"
        assert np.array_equal(bt.flow[i].cpu().numpy(), flow), f"pair {i} flow"
        assert np.array_equal(bt.status[i].cpu().numpy(), st), f"pair {i} status"
        assert np.array_equal(bt.iters[i].cpu().numpy(), it), f"pair {i} iterations"


SMALL_SPECS = [(320, 240, 8, 2), (256, 109, 8, 3), (310, 93, 7, 4), (320, 180, 8, 6), (97, 61, 7, 3),
               (160, 120, 8, 4)]


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_single_pair_path_and_oracle(dgf, use_graph):
    prm = dgf.RlofParams(levels=3, radius=4, max_iter=30, model=4)
    frames = frames_for(SMALL_SPECS, 3100)
    bt, _, _ = run_batch(dgf, SMALL_SPECS, frames, prm, use_graph)
    assert_same_as_single(dgf, bt, frames, SMALL_SPECS, prm)
    oprm = oracle.RlofParams(levels=3, radius=4, max_iter=30, model=4)
    for i, ((I1, I2), (W, H, win, step)) in enumerate(zip(frames, SMALL_SPECS)):
        pts_o, _, _ = oracle.degraf_detect(I1, win, win, step)
        pts = bt.pts[i].cpu().numpy()
        assert pts.shape == pts_o.shape and np.abs(pts - pts_o).max() <= 1e-4
        sg, fg = bt.status[i].cpu().numpy(), bt.flow[i].cpu().numpy()
        fs.check(fg, sg, fs.frames_spread(I1, I2, pts.astype(np.float64), oprm), f"pair {i}")


def test_graph_replay_sees_new_frame_contents(dgf):
    prm = dgf.RlofParams(levels=3, radius=4, max_iter=30, model=4)
    specs = SMALL_SPECS[:3]
    frames = frames_for(specs, 3200)
    bt, d1, d2 = run_batch(dgf, specs, frames, prm, True)
    first = [f.cpu().numpy().copy() for f in bt.flow]
    frames2 = frames_for(specs, 3300)
    for k, (a, b) in enumerate(frames2):  # same buffers, new contents: the cached graph replays
        d1[k].copy_(torch.from_numpy(a))
        d2[k].copy_(torch.from_numpy(b))
    bt.run(d1, d2, use_graph=True)
    torch.cuda.synchronize()
    assert any(not np.array_equal(first[k], bt.flow[k].cpu().numpy()) for k in range(len(specs)))
    assert_same_as_single(dgf, bt, frames2, specs, prm)


def test_bound_frames_run_without_arguments(dgf):
    """bind() + run(): descriptors built once; new contents written into the bound
    buffers are tracked, and the results equal an explicit run on the same frames."""
    prm = dgf.RlofParams(levels=3, radius=4, max_iter=30, model=4)
    specs = SMALL_SPECS[:3]
    frames = frames_for(specs, 3500)
    bt, d1, d2 = run_batch(dgf, specs, frames, prm, True)
    bt.bind(d1, d2)
    frames2 = frames_for(specs, 3600)
    for k, (a, b) in enumerate(frames2):
        d1[k].copy_(torch.from_numpy(a))
        d2[k].copy_(torch.from_numpy(b))
    bt.run(use_graph=True)
    torch.cuda.synchronize()
    bound = [(f.cpu().numpy().copy(), s.cpu().numpy().copy()) for f, s in zip(bt.flow, bt.status)]
    bt.run(d1, d2, use_graph=False)
    torch.cuda.synchronize()
    for k in range(len(specs)):
        np.testing.assert_array_equal(bound[k][0], bt.flow[k].cpu().numpy())
        np.testing.assert_array_equal(bound[k][1], bt.status[k].cpu().numpy())
    assert_same_as_single(dgf, bt, frames2, specs, prm)


def test_more_pairs_than_one_chunk(dgf):
    """70 pairs: two chunks of the persistent launch, each with its own counter."""
    prm = dgf.RlofParams(levels=2, radius=4, max_iter=20, model=2)
    specs = [(64 + (i % 5) * 8, 48 + (i % 3) * 8, 8, 3 + (i % 2)) for i in range(70)]
    frames = frames_for(specs, 3400)
    bt, _, _ = run_batch(dgf, specs, frames, prm, False)
    assert_same_as_single(dgf, bt, frames, specs, prm)


def test_mixed_size_batch_of_64_pairs(dgf):
    """The mixed-size batch workload: 64 pairs of 640x480 .. 1280x720, steps 2..6,
    window 8, 3 levels, 9x9 support; every pair equals the single-pair path, and
    4,000 sampled points of each of four pairs meet the oracle bars."""
    specs = [(W, H, 8, step) for (W, H, step) in synth.make_batch_specs(64, 3000)]
    frames = []
    for i, (W, H, win, step) in enumerate(specs):
        p = synth.make_translation_pair(W, H, seed=3000 + i)
        frames.append((p.I1, p.I2))
    prm = dgf.RlofParams(levels=3, radius=4, max_iter=30, model=4)
    bt, _, _ = run_batch(dgf, specs, frames, prm, True)
    assert sum(bt.n) > 1_000_000
    assert_same_as_single(dgf, bt, frames, specs, prm)
    oprm = oracle.RlofParams(levels=3, radius=4, max_iter=30, model=4)
    rng = np.random.default_rng(0)
    for i in (0, 17, 42, 63):
        I1, I2 = frames[i]
        idx = np.sort(rng.choice(bt.n[i], size=min(4000, bt.n[i]), replace=False))
        pts = bt.pts[i].cpu().numpy()[idx]
        sg, fg = bt.status[i].cpu().numpy()[idx], bt.flow[i].cpu().numpy()[idx]
        fs.check(fg, sg, fs.frames_spread(I1, I2, pts.astype(np.float64), oprm), f"batch pair {i}")


def test_autotune_picks_a_shape_and_every_shape_tracks_alike(dgf, tmp_path, monkeypatch):
    """The autotuner times every lane count the library honours at radius 4, keeps
    the fastest for the tracker and in its cache (which lanes="auto" then reads);
    every shape meets the oracle bars on every pair of the batch (the shapes sum the
    normal equations in different orders, so FP32 trajectories may part where an
    FP32 restatement of the oracle's also does)."""
    monkeypatch.setenv("DGF_TUNE_CACHE", str(tmp_path / "tune.json"))
    prm = dgf.RlofParams(levels=3, radius=4, max_iter=30, model=4)
    frames = frames_for(SMALL_SPECS, 500)
    bt, d1, d2 = run_batch(dgf, SMALL_SPECS, frames, prm, True)
    rec = bt.autotune(reps=2)
    assert rec["lanes"] in (8, 16, 32) and set(rec["ms"]) == {"8", "16", "32"} and bt.lanes == rec["lanes"]
    assert dgf.BatchTracker(SMALL_SPECS, prm, lanes="auto").lanes == rec["lanes"]
    oprm = oracle.RlofParams(levels=3, radius=4, max_iter=30, model=4)
    spreads = [fs.frames_spread(I1, I2, bt.pts[i].cpu().numpy().astype(np.float64), oprm)
               for i, (I1, I2) in enumerate(frames)]
    for lanes in (8, 16, 32):
        bt.lanes = lanes
        bt.run()
        torch.cuda.synchronize()
        for i, sp in enumerate(spreads):
            fs.check(bt.flow[i].cpu().numpy(), bt.status[i].cpu().numpy(), sp, f"lanes {lanes} pair {i}")
