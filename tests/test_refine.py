"""Refinement and coarsening (Algorithms 5 and 6) through the C ABI: the error monitor and the
child-to-parent interpolation against numpy, and the refined output tree against the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")
R = pytest.importorskip("paper_2305_07165_gb300.refine")

pytestmark = pytest.mark.gpu


def _legendre_coeffs(vals, d, k):
    """Tensor Legendre coefficients of the interpolant (numpy's Vandermonde, solved)."""
    x, _ = np.polynomial.legendre.leggauss(k)
    V = np.polynomial.legendre.legvander(x, k - 1)       # V[t, n] = P_n(x_t)
    Vi = np.linalg.inv(V)
    c = vals.reshape((-1,) + (k,) * d)                    # [..., j_d, ..., j_1]
    for ax in range(1, d + 1):
        c = np.moveaxis(np.tensordot(c, Vi, axes=([ax], [1])), -1, ax)
    return c


@pytest.mark.parametrize("d,k", [(2, 8), (3, 6), (3, 12), (2, 16)])
def test_error_monitor_matches_the_legendre_tail(d, k):
    rng = np.random.default_rng(d * 100 + k)
    vals = rng.standard_normal((7, k ** d))
    err, sq = R.leaf_errors(torch.from_numpy(vals).cuda(), d, k)
    c = _legendre_coeffs(vals, d, k)
    idx = np.indices((k,) * d)                            # idx[0] = alpha_d ... idx[-1] = alpha_1
    tail = (idx ** 2).sum(axis=0) >= k * k
    ref = np.sqrt((c[:, tail] ** 2).mean(axis=1))
    assert np.abs(err.cpu().numpy() - ref).max() <= 1e-12 * ref.max()
    w = np.polynomial.legendre.leggauss(k)[1]
    W_ = w
    for _ in range(d - 1):
        W_ = np.multiply.outer(w, W_).reshape(-1)
    assert np.abs(sq.cpu().numpy() - (vals ** 2 * W_).sum(axis=1)).max() <= 1e-12 * (vals ** 2).sum()


@pytest.mark.parametrize("d,k", [(2, 8), (3, 5), (3, 8)])
def test_merge_children_is_exact_for_polynomials(d, k):
    """Children sampled from one polynomial of degree < k: the parent values are the polynomial."""
    rng = np.random.default_rng(k)
    coef = rng.standard_normal((k,) * d) * 0.3
    parent = W.Tree(d, np.array([1], dtype=np.int32), np.zeros((1, d), dtype=np.int32))
    kids_l = np.full(1 << d, 2, dtype=np.int32)
    kids_c = np.array([[(c >> a) & 1 for a in range(d)] for c in range(1 << d)], dtype=np.int32)
    kids = W.Tree(d, kids_l, kids_c)

    def poly(X):
        # a polynomial of degree < k in each coordinate of the parent box's local frame
        s = (X + 0.25) * 4.0                                  # parent box [-1/2, 0]^d -> [-1, 1]^d
        v = np.zeros(X.shape[:-1])
        for alpha in np.ndindex(*coef.shape):
            term = coef[alpha]
            for a in range(d):
                term = term * np.polynomial.legendre.legval(s[..., a], np.eye(k)[alpha[a]])
            v = v + term
        return v
    cv = poly(W.node_positions(kids, k))
    pv = R.merge_children(torch.from_numpy(cv).cuda(), np.arange(1 << d), d, k)
    ref = poly(W.node_positions(parent, k))
    assert np.abs(pv.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()


def test_refine_then_coarsen_two_sharp_gaussians():
    """The setting of the paper's output-tree example (Section 4.3), at a CPU-friendly size: two
    Gaussians of alpha = 1e-4, delta = 4e-3, k = 8, FP64.  Refinement must leave every output
    leaf within the monitor's bound and agree with the oracle at the output boxes; coarsening
    must keep that agreement to the requested precision."""
    d, k, delta, eps = 2, 8, 4e-3, 1e-9
    centers, alphas = np.array([[0.1, -0.05], [-0.2, 0.15]]), np.array([1e-4, 1e-4])
    tr = W.gaussian_refined_tree(d, centers, np.sqrt(alphas), rho=1.0, beta=4.0, max_level=7, min_level=2)
    sigma = W.gaussian_sum(W.node_positions(tr, k), centers, alphas)
    plan = F.Plan(d, k, delta, 1e-11, tr.level, tr.coord)
    lev, crd, u, rounds = R.refine(plan, torch.from_numpy(sigma).cuda(), eps, max_level=int(tr.level.max()) + 2)
    assert rounds >= 2 and len(lev) > tr.n_leaves
    err, sq = R.leaf_errors(u, d, k)
    norm = R._norm(sq, lev, d)
    assert (err.cpu().numpy() <= eps * norm).all() or (lev.max() == tr.level.max() + 2)
    uo = oracle.box_fgt_boxes(d, k, delta, False, tr.level, tr.coord, sigma, lev, crd)
    ug = u.cpu().numpy()
    assert np.abs(ug - uo).max() <= 1e-9 * np.abs(uo).max()
    cl, cc, cu = R.coarsen(lev, crd, u, d, k, eps, norm=norm)
    assert len(cl) < len(lev)
    uc = oracle.box_fgt_boxes(d, k, delta, False, tr.level, tr.coord, sigma, cl, cc)
    assert np.abs(cu.cpu().numpy() - uc).max() <= 1e-7 * np.abs(uc).max()
    plan.close()


def _u_exact(x, centers, alphas, delta):
    """u = int_B exp(-|x - y|^2 / delta) sum_i exp(-|y - c_i|^2 / alpha_i) dy in free space: per axis
    the product of the two Gaussians is a Gaussian in y, integrated over [-1/2, 1/2] by erf."""
    from scipy.special import erf
    out = np.zeros(len(x))
    for c, a in zip(centers, alphas):
        s = np.sqrt(a * delta / (a + delta))
        term = np.ones(len(x))
        for ax in range(x.shape[1]):
            mu = (a * x[:, ax] + delta * c[ax]) / (a + delta)
            term *= (np.exp(-(x[:, ax] - c[ax]) ** 2 / (a + delta)) * s * np.sqrt(np.pi) / 2
                     * (erf((0.5 - mu) / s) - erf((-0.5 - mu) / s)))
        out += term
    return out


def test_refinement_recovers_the_potential_between_nodes():
    """The setting of the paper's example (Section 4.3): two Gaussians with alpha = 1e-4, delta =
    4e-3, k = 8, eps = 1e-12, the source tree built to resolve sigma (Algorithm 3).  The potential's
    interpolant on the source tree misses u between the nodes by far more than eps (the diffused
    peaks are too wide for the coarse boxes); after refinement (Algorithm 5) the relative l2 error
    at equispaced points drops by more than three orders of magnitude."""
    d, k, delta, eps = 2, 8, 4e-3, 1e-12
    centers, alphas = np.array([[-0.13, 0.07], [0.21, -0.18]]), np.array([1e-4, 1e-4])
    level, coord, sigma = F.build_gaussian_tree(d, k, centers, alphas, eps=eps, max_level=11)
    plan = F.Plan(d, k, delta, 1e-12, level, coord)
    g = (np.arange(200) + 0.5) / 200 - 0.5
    pts = np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    ue = _u_exact(pts, centers, alphas, delta)
    u0 = plan(sigma)
    e_in = np.linalg.norm(R.interpolate(level, coord, u0, d, k, pts) - ue) / np.linalg.norm(ue)
    lev, crd, u, rounds = R.refine(plan, sigma, eps)
    e_ref = np.linalg.norm(R.interpolate(lev, crd, u, d, k, pts) - ue) / np.linalg.norm(ue)
    plan.close()
    assert len(lev) > len(level) and rounds >= 2
    assert e_ref <= 1e-3 * e_in and e_ref <= 1e-10, (e_in, e_ref)
