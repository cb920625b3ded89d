"""Pins of the oracle's EPIC interpolation (Section 2 "Interpolation": an affine model
fitted to the k nearest sparse vectors under a geodesic distance that penalises
crossing image edges, the edges taken from image gradients; the paper prints no
formulas, so the pins check the reading stated in the C source against independent
computations): the cost map against scipy's Sobel filter; the geodesic distances,
Voronoi labels, seed graph and k-nearest lists against scipy's Dijkstra on graphs
built here; the fit against weighted least squares by numpy; closed forms (an
exactly affine flow field is reproduced everywhere; collinear seeds fall back to
the weighted mean; one seed fills the image); and edge preservation at a step edge
between two motions."""
import numpy as np
import pytest
from scipy import ndimage
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import dijkstra

import oracle

PRM = oracle.EpicParams()


def textured(W, H, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    base = 120 + 40 * np.sin(0.21 * x + 0.5) * np.cos(0.17 * y) + rng.normal(0, 6, (H, W))
    return np.clip(np.rint(base), 0, 255).astype(np.uint8)


def grid_graph(cost):
    """4-connected pixel grid, the step between neighbours costing the sum of their costs."""
    H, W = cost.shape
    idx = np.arange(H * W).reshape(H, W)
    a = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    b = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    c = cost.ravel()
    w = (c[a] + c[b]).astype(np.float64)
    return coo_matrix((np.concatenate([w, w]), (np.concatenate([a, b]), np.concatenate([b, a]))),
                      shape=(H * W, H * W)).tocsr()


def seeds_of(pts, status, W, H):
    """(seed index, pixel) pairs: tracked matches, a pixel held by its lowest index."""
    out, held = [], set()
    for i, (p, s) in enumerate(zip(pts, status)):
        if s not in (oracle.TRACKED, oracle.MAXITER):
            continue
        x = min(max(int(np.floor(p[0] + 0.5)), 0), W - 1)
        y = min(max(int(np.floor(p[1] + 0.5)), 0), H - 1)
        if (x, y) in held:
            continue
        held.add((x, y))
        out.append((i, y * W + x))
    return out


def brute_force(img, pts, status, prm):
    """Labels, distances and k-nearest lists from scipy's Dijkstra on graphs built here."""
    H, W = img.shape
    cost = prm.cost_base + prm.cost_gain * (np.abs(ndimage.sobel(img.astype(np.int64), 1, mode="nearest"))
                                            + np.abs(ndimage.sobel(img.astype(np.int64), 0, mode="nearest")))
    seeds = seeds_of(pts, status, W, H)
    ids = np.array([s for s, _ in seeds])
    D_all = dijkstra(grid_graph(cost), indices=[p for _, p in seeds])  # [n_seeds, H*W]
    # lexicographic (distance, seed index): seed indices ascend with the rows
    order = np.lexsort((np.broadcast_to(ids[:, None], D_all.shape), D_all), axis=0)[0]
    D = D_all[order, np.arange(H * W)].astype(np.int64).reshape(H, W)
    lab = ids[order].reshape(H, W)
    # seed graph
    c = cost
    best = {}
    for (dy, dx) in ((0, 1), (1, 0)):
        la, lb = lab[:H - dy, :W - dx], lab[dy:, dx:]
        w = D[:H - dy, :W - dx] + c[:H - dy, :W - dx] + c[dy:, dx:] + D[dy:, dx:]
        for s, t, ww in zip(la[la != lb], lb[la != lb], w[la != lb]):
            key = (min(s, t), max(s, t))
            best[key] = min(best.get(key, np.inf), ww)
    pos = {s: j for j, s in enumerate(ids)}
    r = [pos[s] for s, _ in best] + [pos[t] for _, t in best]
    q = [pos[t] for _, t in best] + [pos[s] for s, _ in best]
    w = list(best.values()) * 2
    G = coo_matrix((np.array(w, np.float64), (r, q)), shape=(len(ids), len(ids))).tocsr()
    Dg = dijkstra(G)
    knn = {}
    for j, s in enumerate(ids):
        ok = np.isfinite(Dg[j])
        cand = np.lexsort((ids[ok], Dg[j][ok]))[:prm.k]
        knn[s] = (ids[ok][cand], Dg[j][ok][cand].astype(np.int64))
    return cost, lab, D, knn


def random_matches(W, H, n, seed, lost=0.15):
    rng = np.random.default_rng(seed)
    pts = rng.uniform([0, 0], [W - 1, H - 1], (n, 2))
    pts[5] = pts[3] + 0.2  # same pixel as a lower-index seed (usually): dropped
    flow = rng.normal(0, 3, (n, 2))
    status = np.where(rng.random(n) < lost, oracle.OOB, oracle.TRACKED).astype(np.uint8)
    status[rng.random(n) < 0.1] = oracle.MAXITER
    return pts, flow, status


def test_cost_map_is_the_sobel_gradient_l1_norm():
    img = textured(37, 23, 1)
    got = oracle.epic_cost(img, 5, 3)
    sx = ndimage.sobel(img.astype(np.int64), axis=1, mode="nearest")
    sy = ndimage.sobel(img.astype(np.int64), axis=0, mode="nearest")
    np.testing.assert_array_equal(got, 5 + 3 * (np.abs(sx) + np.abs(sy)))


@pytest.mark.parametrize("seed,k", [(0, 5), (1, 12), (2, 200)])
def test_voronoi_graph_and_neighbourhoods_match_scipy_dijkstra(seed, k):
    W, H = 41, 29
    img = textured(W, H, seed)
    pts, flow, status = random_matches(W, H, 60, seed)
    prm = oracle.EpicParams(k=k)
    r = oracle.epic_interpolate(img, pts, flow, status, prm)
    cost, lab, D, knn = brute_force(img, pts, status, prm)
    np.testing.assert_array_equal(r.labels, lab)
    np.testing.assert_array_equal(r.dist, D)
    seeds = {s for s, _ in seeds_of(pts, status, W, H)}
    for i in range(len(pts)):
        if i not in seeds:
            assert r.knn_count[i] == 0 and r.fit_kind[i] == 0
            continue
        idx, dd = knn[i]
        assert r.knn_count[i] == len(idx)
        np.testing.assert_array_equal(r.knn_idx[i, :len(idx)], idx)
        np.testing.assert_array_equal(r.knn_dist[i, :len(idx)], dd)
        assert idx[0] == i and dd[0] == 0


def test_fit_is_weighted_least_squares():
    W, H = 60, 44
    img = textured(W, H, 4)
    pts, flow, status = random_matches(W, H, 90, 4)
    prm = oracle.EpicParams(k=16, min_spread=0.0)
    r = oracle.epic_interpolate(img, pts, flow, status, prm)
    checked = 0
    for s in np.flatnonzero(r.fit_kind == 1)[:25]:
        nb = r.knn_idx[s, :r.knn_count[s]]
        w = np.exp(-prm.a * r.knn_dist[s, :r.knn_count[s]] / (2 * prm.cost_base))
        X = np.c_[pts[nb] - pts[s], np.ones(len(nb))] * np.sqrt(w)[:, None]
        sol = np.linalg.lstsq(X, flow[nb] * np.sqrt(w)[:, None], rcond=None)[0]  # [3, 2]
        A, b = sol[:2].T, sol[2]
        np.testing.assert_allclose(r.models[s], [A[0, 0], A[0, 1], A[1, 0], A[1, 1], b[0], b[1]], atol=1e-8)
        checked += 1
    assert checked >= 20
    # the dense field applies each pixel's seed model
    yy, xx = np.mgrid[0:H, 0:W]
    lab = r.labels
    m = r.models[lab]
    dx, dy = xx - pts[lab, 0], yy - pts[lab, 1]
    np.testing.assert_allclose(r.dense[..., 0], m[..., 0] * dx + m[..., 1] * dy + m[..., 4], atol=1e-9)
    np.testing.assert_allclose(r.dense[..., 1], m[..., 2] * dx + m[..., 3] * dy + m[..., 5], atol=1e-9)


def test_an_affine_flow_field_is_reproduced_everywhere():
    W, H = 120, 80
    img = textured(W, H, 7)
    rng = np.random.default_rng(7)
    pts = np.stack(np.meshgrid(np.arange(3, W - 3, 4.0), np.arange(3, H - 3, 4.0)), -1).reshape(-1, 2)
    pts += rng.uniform(-1, 1, pts.shape)
    A = np.array([[0.03, -0.02], [0.015, 0.04]])
    b = np.array([2.5, -1.75])
    flow = pts @ A.T + b
    status = np.zeros(len(pts), np.uint8)
    # a slow decay, so that every neighbourhood spreads enough on this strong texture
    r = oracle.epic_interpolate(img, pts, flow, status, oracle.EpicParams(a=0.002))
    assert np.all(r.fit_kind == 1)
    yy, xx = np.mgrid[0:H, 0:W]
    truth = np.stack([xx, yy], -1) @ A.T + b
    np.testing.assert_allclose(r.dense, truth, atol=1e-9)


def test_collinear_seeds_fall_back_to_the_weighted_mean_and_model_0_is_the_mean():
    W, H = 50, 30
    img = textured(W, H, 8)
    pts = np.array([[x, 15.0] for x in range(4, 46, 3)])
    rng = np.random.default_rng(8)
    flow = rng.normal(0, 2, pts.shape)
    status = np.zeros(len(pts), np.uint8)
    for prm in (PRM, oracle.EpicParams(model=0)):
        r = oracle.epic_interpolate(img, pts, flow, status, prm)
        assert np.all(r.fit_kind == 2)
        for s in range(len(pts)):
            nb = r.knn_idx[s, :r.knn_count[s]]
            w = np.exp(-prm.a * r.knn_dist[s, :r.knn_count[s]] / (2 * prm.cost_base))
            np.testing.assert_allclose(r.models[s, 4:], (w[:, None] * flow[nb]).sum(0) / w.sum(), atol=1e-12)
            np.testing.assert_array_equal(r.models[s, :4], 0.0)


def test_one_seed_fills_the_image_and_no_seed_gives_zero():
    img = textured(30, 20, 9)
    pts = np.array([[10.3, 7.6], [20.0, 5.0]])
    flow = np.array([[1.5, -2.0], [9.0, 9.0]])
    r = oracle.epic_interpolate(img, pts, flow, np.array([0, 1], np.uint8), PRM)
    assert np.all(r.labels == 0) and r.dist[8, 10] == 0
    np.testing.assert_array_equal(r.dense.reshape(-1, 2), np.tile(flow[0], (600, 1)))
    assert r.fit_kind.tolist() == [2, 0]
    r = oracle.epic_interpolate(img, pts, flow, np.array([1, 2], np.uint8), PRM)
    assert np.all(r.labels == -1) and np.all(r.dist == -1) and np.all(r.dense == 0)
    r = oracle.epic_interpolate(img, np.zeros((0, 2)), np.zeros((0, 2)), np.zeros(0, np.uint8), PRM)
    assert np.all(r.labels == -1)


def test_edges_keep_the_two_motions_apart():
    """Left of a step edge the seeds move by (2, 1), right of it by (-3, 0.5). With
    edge costs the pixels away from the edge keep their side's motion; with a flat
    cost (gain 0) the fits mix the two sides near the edge."""
    W, H, xe = 96, 64, 47
    rng = np.random.default_rng(10)
    img = np.where(np.arange(W)[None, :] <= xe, 60, 190) + rng.integers(-3, 4, (H, W))
    img = img.astype(np.uint8)
    pts = np.stack(np.meshgrid(np.arange(1, W - 1, 3.0), np.arange(1, H - 1, 3.0)), -1).reshape(-1, 2)
    pts += rng.uniform(-0.4, 0.4, pts.shape)
    left = pts[:, 0] < xe + 0.5
    flow = np.where(left[:, None], [2.0, 1.0], [-3.0, 0.5])
    status = np.zeros(len(pts), np.uint8)
    truth = np.where((np.arange(W) <= xe)[None, :, None], [2.0, 1.0], [-3.0, 0.5])
    near = np.abs(np.arange(W) - xe - 0.5) < 6
    for gain, ok in ((1, True), (0, False)):
        r = oracle.epic_interpolate(img, pts, flow, status, oracle.EpicParams(cost_gain=gain))
        e = np.hypot(*(r.dense - truth).transpose(2, 0, 1))
        away = np.abs(np.arange(W) - xe - 0.5)[None, :].repeat(H, 0) >= 2
        print(f"gain {gain}: max error 2+ px from the edge {e[away].max():.3f}, "
              f"mean within 6 px {e[:, near].mean():.3f}")
        if ok:
            assert e[away].max() < 0.05
        else:
            assert e[:, near].mean() > 0.5
