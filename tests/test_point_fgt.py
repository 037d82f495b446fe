"""Discrete (point) Gauss transform with proxy grids (Algorithm 2) through the C ABI, against the
direct sum."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")

pytestmark = pytest.mark.gpu


def _clustered(rng, n, d, k=6):
    c = rng.uniform(-0.4, 0.4, size=(k, d))
    w = np.exp(rng.uniform(np.log(0.01), np.log(0.1), size=k))
    lab = rng.integers(0, k, n)
    return c[lab] + w[lab, None] * rng.standard_normal((n, d))


def check(d, delta, tol, src, tgt, n_s, seed=0, prec=0):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0.5, 1.5, len(src))
    plan = F.PointPlan(d, delta, tol, src, tgt, n_s=n_s, prec=prec)
    u = plan(torch.from_numpy(q).cuda()).cpu().numpy()
    info = plan.info()
    plan.close()
    uo = oracle.point_fgt(d, delta, src, q, tgt)
    err = np.abs(u - uo).max() / max(np.abs(uo).max(), 1e-300)
    assert np.all(np.isfinite(u))
    assert err <= 10 * tol, (err, info)
    return info


@pytest.mark.parametrize("d,delta,tol", [(2, 1e-3, 1e-6), (2, 1e-4, 1e-10), (3, 1e-3, 1e-6), (3, 3e-3, 1e-10)])
def test_uniform_points(d, delta, tol):
    rng = np.random.default_rng(d)
    pts = rng.uniform(-0.5, 0.5, size=(20000, d))
    info = check(d, delta, tol, pts, pts, n_s=32)
    assert info["n_dense_boxes"] > 0 and info["n_direct_pairs"] >= 0


@pytest.mark.parametrize("d", [2, 3])
def test_clustered_sources_and_separate_targets(d):
    rng = np.random.default_rng(10 + d)
    src = _clustered(rng, 30000, d)
    tgt = np.concatenate([_clustered(rng, 10000, d), rng.uniform(-0.6, 0.6, size=(5000, d))])
    info = check(d, 1e-3, 1e-8, src, tgt, n_s=40)
    assert info["n_dense_boxes"] > 0 and info["n_direct_pairs"] > 0


def test_all_direct_and_all_plane_wave():
    rng = np.random.default_rng(5)
    pts = rng.uniform(-0.5, 0.5, size=(8000, 3))
    info = check(3, 1e-3, 1e-7, pts, pts, n_s=10 ** 9)       # no dense box: every pair direct
    assert info["n_dense_boxes"] == 0
    info = check(3, 1e-3, 1e-7, pts, pts, n_s=1)             # nearly every box dense
    assert info["n_dense_boxes"] > 0


def test_empty_and_tiny_sets():
    rng = np.random.default_rng(6)
    pts = rng.uniform(-0.5, 0.5, size=(100, 2))
    plan = F.PointPlan(2, 1e-2, 1e-6, pts[:0], pts, n_s=8)
    u = plan(torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert u.shape == (100,) and (u == 0).all().item()
    plan.close()
    check(2, 1e-2, 1e-6, pts[:1], pts, n_s=8)
    check(2, 1e-2, 1e-6, pts, pts[:1], n_s=8)


@pytest.mark.parametrize("d,delta,tol", [(2, 1e-3, 1e-6), (3, 1e-3, 1e-6), (3, 3e-3, 1e-7)])
def test_split_uniform_points(d, delta, tol):
    """FP32 Lagrange weights, anterpolation, interpolation and expansions: the same bound."""
    rng = np.random.default_rng(20 + d)
    pts = rng.uniform(-0.5, 0.5, size=(20000, d))
    info = check(d, delta, tol, pts, pts, n_s=32, prec=F.PREC_SPLIT)
    assert info["prec"] == F.PREC_SPLIT and info["n_dense_boxes"] > 0


@pytest.mark.parametrize("d", [2, 3])
def test_split_clustered(d):
    """Crowded boxes: many source and target segments per box, with sparse colleagues."""
    rng = np.random.default_rng(30 + d)
    src = _clustered(rng, 60000, d)
    tgt = np.concatenate([_clustered(rng, 10000, d), rng.uniform(-0.6, 0.6, size=(5000, d))])
    info = check(d, 1e-3, 1e-6, src, tgt, n_s=40, prec=F.PREC_SPLIT)
    assert info["n_dense_boxes"] > 0 and info["n_direct_pairs"] > 0


def test_split_nodes_and_box_edges():
    """Points on proxy nodes' coordinates and on box faces (Lagrange weights at a node, s = +-1)."""
    rng = np.random.default_rng(41)
    pts = rng.uniform(-0.5, 0.5, size=(4000, 3))
    pts[:50] = 0.0                       # the centre of the root; a node coordinate for odd k_p
    pts[50:100, 0] = pts[50:100, 0].round(1)
    for prec in (F.PREC_FP64, F.PREC_SPLIT):
        check(3, 1e-3, 1e-6, pts, pts, n_s=8, prec=prec)


def test_split_rejects_tight_tolerance():
    pts = np.zeros((4, 3))
    with pytest.raises(F.FGTError):
        F.PointPlan(3, 1e-3, 1e-8, pts, pts, prec=F.PREC_SPLIT)
    with pytest.raises(F.FGTError):
        F.PointPlan(3, 1e-3, 1e-6, pts, pts, prec=7)


def test_split_all_direct():
    """No dense box: every pair through the FP32 direct sum from local coordinates."""
    rng = np.random.default_rng(43)
    pts = rng.uniform(-0.5, 0.5, size=(6000, 3))
    info = check(3, 1e-3, 1e-6, pts, pts, n_s=10 ** 9, prec=F.PREC_SPLIT)
    assert info["n_dense_boxes"] == 0 and info["n_direct_pairs"] > 0
