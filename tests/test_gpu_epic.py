"""GPU parity of the EPIC interpolation (epic_interpolate) against the oracle's
reading (Section 2 "Interpolation"; k from Section 3): the cost map, geodesic
labels and distances, and the k-nearest lists are exact integers on both sides and
must agree bit for bit; the fits run in FP64 on both sides, so models agree to
rounding and the FP32 dense field to its own rounding; edge cases (no seed, one
seed, duplicates, k above the seed count, a pitched frame, the weighted-mean model)
and the largest frame and point count of the mixed batch."""
import numpy as np
import pytest
import torch

import oracle
import synth
from test_oracle_epic import random_matches, textured

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


def run_both(dgf, img, pts, flow, status, k=128, model=1, frame=None, **kw):
    """GPU (debug outputs) and oracle on the same float32 inputs."""
    pts32, flow32 = pts.astype(np.float32), flow.astype(np.float32)
    prm = dgf.EpicParams(k=k, model=model, **kw)
    fr = to_dev(img) if frame is None else frame
    dgf.device_status(reset=True)
    dense, d = dgf.epic_interpolate(fr, to_dev(pts32), to_dev(flow32), to_dev(status.astype(np.uint8)), prm,
                                    debug=True)
    torch.cuda.synchronize()
    assert dgf.device_status() == 0  # the labelling settled and every search fitted its layout
    g = {key: v.cpu().numpy() for key, v in d.items()}
    g["dense"] = dense.cpu().numpy()
    o = oracle.epic_interpolate(img, pts32.astype(np.float64), flow32.astype(np.float64), status,
                                oracle.EpicParams(k=k, model=model, **kw))
    return g, o


def assert_parity(g, o, dense_tol=1e-4, model_tol=1e-9):
    np.testing.assert_array_equal(g["labels"], o.labels)
    np.testing.assert_array_equal(g["dist"], o.dist)
    np.testing.assert_array_equal(g["knn_count"], o.knn_count)
    for s in np.flatnonzero(o.knn_count):
        c = o.knn_count[s]
        np.testing.assert_array_equal(g["knn_idx"][s, :c], o.knn_idx[s, :c])
        np.testing.assert_array_equal(g["knn_dist"][s, :c], o.knn_dist[s, :c])
    np.testing.assert_array_equal(g["fit_kind"], o.fit_kind)
    scale = np.maximum(1.0, np.abs(o.models))
    assert np.max(np.abs(g["models"] - o.models) / scale) <= model_tol
    err = np.abs(g["dense"].astype(np.float64) - o.dense)
    print(f"max dense difference {err.max():.3g} px")
    assert err.max() <= dense_tol


@pytest.mark.parametrize("seed,k", [(0, 5), (1, 12), (2, 200), (3, 1)])
def test_small_random_matches_exact(dgf, seed, k):
    W, H = 41, 29
    img = textured(W, H, seed)
    pts, flow, status = random_matches(W, H, 60, seed)
    g, o = run_both(dgf, img, pts, flow, status, k=k)
    assert_parity(g, o)


def test_ragged_tiles_and_weighted_mean_model(dgf):
    W, H = 101, 67  # several 32 x 32 tiles with ragged right and bottom edges
    img = textured(W, H, 5)
    pts, flow, status = random_matches(W, H, 400, 5)
    for model in (1, 0):
        g, o = run_both(dgf, img, pts, flow, status, k=64, model=model)
        assert_parity(g, o)


def tracked_pair(config):
    p = synth.make_pair(config)
    pts, _, _ = oracle.degraf_detect(p.I1, p.win, p.win, p.step)
    pts = pts.astype(np.float32).astype(np.float64)
    f, s, _, _ = oracle.rlof_track(p.I1, p.I2, pts, oracle.RlofParams(levels=p.levels, radius=p.radius,
                                                                        max_iter=p.max_iter, model=4))
    return p, pts, f, s


@pytest.mark.parametrize("config", [1, 2])
def test_tracked_workloads_exact(dgf, config):
    """The 256x128 translation pair and the 1242x375 driving scene (50,676 points),
    seeds from the oracle's tracking."""
    p, pts, f, s = tracked_pair(config)
    g, o = run_both(dgf, p.I1, pts, f, s)
    assert (o.fit_kind == 1).mean() > 0.5
    assert_parity(g, o, dense_tol=1e-3)


def test_largest_batch_frame_exact(dgf):
    """1280x720 radial scene with DeGraF step 2 (227,409 points), ground-truth flows at the points
    as the sparse input, a tenth of them lost."""
    p = synth.make_pair(2, size=(1280, 720))
    pts, _, _ = oracle.degraf_detect(p.I1, 8, 8, 2)
    assert len(pts) == 227409
    pts = pts.astype(np.float32).astype(np.float64)
    xi, yi = np.rint(pts[:, 0]).astype(int), np.rint(pts[:, 1]).astype(int)
    flow = p.flow_gt[yi, xi].astype(np.float64)
    status = np.where(np.random.default_rng(0).random(len(pts)) < 0.1, oracle.OOB, oracle.TRACKED).astype(np.uint8)
    g, o = run_both(dgf, p.I1, pts, flow, status)
    assert_parity(g, o, dense_tol=1e-3)


def test_edge_cases(dgf):
    img = textured(30, 20, 9)
    pts = np.array([[10.3, 7.6], [20.0, 5.0], [10.1, 7.9]])
    flow = np.array([[1.5, -2.0], [9.0, 9.0], [4.0, 4.0]])
    # one seed (the third shares its pixel and has a higher index): fills the image
    g, o = run_both(dgf, img, pts, flow, np.array([0, 1, 0], np.uint8))
    assert_parity(g, o)
    assert np.all(g["labels"] == 0) and g["fit_kind"].tolist() == [2, 0, 0]
    np.testing.assert_array_equal(g["dense"].reshape(-1, 2), np.tile(flow[0].astype(np.float32), (600, 1)))
    # no seed
    g, o = run_both(dgf, img, pts, flow, np.array([1, 2, 3], np.uint8))
    assert np.all(g["labels"] == -1) and np.all(g["dense"] == 0) and np.all(g["dist"] == -1)
    # no matches at all
    dense = dgf.epic_interpolate(to_dev(img), torch.zeros((0, 2), device="cuda"), torch.zeros((0, 2), device="cuda"),
                                 torch.zeros(0, dtype=torch.uint8, device="cuda"))
    assert torch.all(dense == 0)
    # k far above the number of seeds, and a frame that is a view of a wider buffer
    W, H = 70, 45
    big = textured(W + 13, H, 11)
    pts, flow, status = random_matches(W, H, 30, 11)
    fr = to_dev(big)[:, :W]
    g, o = run_both(dgf, np.ascontiguousarray(big[:, :W]), pts, flow, status, k=256, frame=fr)
    assert_parity(g, o)
    assert g["knn_count"].max() < 30


def test_hub_seed_takes_the_retry_path(dgf):
    """A seed in the middle of a flat frame inside a ring of 1,600 seeds: its cell
    borders 604 ring cells, so its search discovers more seeds at once than the fast
    hash holds; the search is redone with the large layout and must still match the
    oracle exactly (on a flat frame, with many equal distances and ring seeds that
    share pixels, which also exercises the index tie-break and the pixel rule)."""
    W = H = 601
    img = np.full((H, W), 100, np.uint8)
    ang = np.linspace(0, 2 * np.pi, 1600, endpoint=False)
    ring = np.stack([300 + 285 * np.cos(ang), 300 + 285 * np.sin(ang)], 1)
    pts = np.vstack([[[300.2, 299.9]], ring])
    rng = np.random.default_rng(12)
    flow = rng.normal(0, 1, pts.shape)
    status = np.zeros(len(pts), np.uint8)
    g, o = run_both(dgf, img, pts, flow, status)
    print(f"searches redone with the large layout: {int(g['retried'][0])}")
    assert g["retried"][0] >= 1
    assert_parity(g, o)


def test_large_k_layout(dgf):
    """k = 256 takes the larger fast layout."""
    W, H = 160, 120
    img = textured(W, H, 13)
    pts, flow, status = random_matches(W, H, 700, 13)
    g, o = run_both(dgf, img, pts, flow, status, k=256)
    assert_parity(g, o)
