"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each check targets a way the oracle could plausibly be wrong: a transposed
1D kernel matrix or a wrong Lagrange basis (Gaussian closed form on an
adaptive tree), a dropped image or a too-short image sum (periodic constants
and Fourier eigenfunctions), a truncation radius that is too small (sigma = 1
at small delta), an off-by-one in the leaf layout (brute-force 2D/3D
quadrature with an independent Legendre-basis interpolant), and ordering or
index mistakes (invariants).
"""
import itertools
import os

import numpy as np
import pytest
from scipy.special import erf

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gauss_legendre_rule_matches_numpy():
    for n in (1, 2, 5, 8, 16, 24, 32, 48):
        x, w = oracle.gauss_legendre(n)
        xr, wr = np.polynomial.legendre.leggauss(n)
        assert np.abs(x - xr).max() < 1e-14
        assert np.abs(w - wr).max() < 1e-14


def _u_const_free(X, delta):
    """u for sigma = 1 on B, free space: product of erf differences (exact)."""
    s = np.sqrt(delta)
    return np.prod(0.5 * np.sqrt(np.pi * delta) * (erf((0.5 - X) / s) + erf((0.5 + X) / s)), axis=-1)


@pytest.mark.parametrize("d,p,delta,seed", [(2, 8, 1e-2, 1), (2, 5, 1e-4, 2), (3, 6, 1e-2, 3),
                                            (3, 4, 3e-1, 4), (2, 7, 1.0, 5)])
def test_constant_density_free_space(d, p, delta, seed):
    tr = W.random_balanced_tree(d, seed, max_level=4 if d == 2 else 3, min_level=1)
    X = W.node_positions(tr, p)
    u = oracle.box_fgt(d, p, delta, False, tr.level, tr.coord, np.ones((tr.n_leaves, p ** d)))
    ex = _u_const_free(X, delta)
    assert np.abs(u - ex).max() <= 1e-13 * np.abs(ex).max()


@pytest.mark.parametrize("d,p,delta,seed", [(2, 8, 1e-2, 1), (2, 6, 2e-1, 2), (3, 5, 1e-2, 3),
                                            (3, 4, 1e-3, 4)])
def test_constant_density_periodic(d, p, delta, seed):
    # sigma = 1 with the periodic kernel: u = (pi delta)^(d/2) everywhere.
    tr = W.random_balanced_tree(d, seed, max_level=4 if d == 2 else 3, periodic=True, min_level=1)
    u = oracle.box_fgt(d, p, delta, True, tr.level, tr.coord, np.ones((tr.n_leaves, p ** d)))
    ex = (np.pi * delta) ** (d / 2)
    assert np.abs(u - ex).max() <= 1e-13 * ex


@pytest.mark.parametrize("d,level,p,n,delta", [(2, 3, 16, 2, 1e-2), (2, 2, 14, 1, 1e-1),
                                               (3, 2, 12, 2, 1e-2), (3, 1, 12, 1, 5e-2)])
def test_trig_density_periodic_eigenfunction(d, level, p, n, delta):
    # Paper eq. (sigmap) and the Fourier form of the periodic kernel (eq. gp:fourier):
    # convolution multiplies the n-th Fourier mode by sqrt(pi delta) exp(-(pi sqrt(delta) n)^2)
    # in each dimension.
    tr = W.uniform_tree(d, level, periodic=True)
    X = W.node_positions(tr, p)
    s = W.trig_density(X, n)
    u = oracle.box_fgt(d, p, delta, True, tr.level, tr.coord, s)
    ex = (np.sqrt(np.pi * delta) * np.exp(-np.pi ** 2 * delta * n ** 2)) ** d * s
    assert np.abs(u - ex).max() <= 1e-11 * np.abs(ex).max()


def _gauss_closed_form(X, centers, alphas, delta):
    """Free-space u for sigma = sum_i exp(-|y-c_i|^2/alpha_i) restricted to B:
    per dimension int_{-1/2}^{1/2} exp(-(x-y)^2/delta) exp(-(y-c)^2/alpha) dy
      = exp(-(x-c)^2/(alpha+delta)) (s sqrt(pi)/2) [erf((1/2-mu)/s) - erf((-1/2-mu)/s)],
    s^2 = alpha delta/(alpha+delta), mu = (alpha x + delta c)/(alpha+delta)."""
    u = np.zeros(X.shape[:-1])
    for c, a in zip(centers, alphas):
        f = np.ones(X.shape[:-1])
        for i in range(X.shape[-1]):
            x = X[..., i]
            s = np.sqrt(a * delta / (a + delta))
            mu = (a * x + delta * c[i]) / (a + delta)
            f *= np.exp(-(x - c[i]) ** 2 / (a + delta)) * 0.5 * s * np.sqrt(np.pi) * (
                erf((0.5 - mu) / s) - erf((-0.5 - mu) / s))
        u += f
    return u


@pytest.mark.parametrize("d,p,delta", [(2, 16, 1e-2), (2, 16, 1e-3), (3, 12, 1e-2)])
def test_gaussian_density_free_space_closed_form(d, p, delta):
    rng = np.random.default_rng(7)
    centers = rng.uniform(-0.3, 0.3, size=(3, d))
    alphas = np.array([0.02, 0.01, 0.005]) if d == 2 else np.array([0.03, 0.02])
    centers = centers[: len(alphas)]
    widths = np.sqrt(alphas)
    tr = W.gaussian_refined_tree(d, centers, widths, rho=1.5 if d == 2 else 2.5, beta=3.0,
                                 max_level=5 if d == 2 else 3, min_level=2 if d == 2 else 1)
    X = W.node_positions(tr, p)
    s = W.gaussian_sum(X, centers, alphas)
    u = oracle.box_fgt(d, p, delta, False, tr.level, tr.coord, s)
    ex = _gauss_closed_form(X, centers, alphas, delta)
    # the oracle integrates the interpolant of sigma; this tree resolves sigma to ~1e-9
    assert np.abs(u - ex).max() <= 1e-8 * np.abs(ex).max()


def _brute_force(d, p, delta, periodic, tr, sigma, nq=40, targets=None):
    """Non-separable brute force: a d-dimensional tensor Gauss rule over each
    source leaf, the interpolant evaluated through a Legendre-series fit
    (numpy), the kernel evaluated on the full d-dimensional distance."""
    eta = W.leaf_nodes(p)
    V = np.polynomial.legendre.legvander(eta, p - 1)          # V[j, n] = P_n(eta_j)
    Vinv = np.linalg.inv(V)
    xq, wq = np.polynomial.legendre.leggauss(nq)
    Pq = np.polynomial.legendre.legvander(xq, p - 1)            # [nq, p]
    targets = np.arange(tr.n_leaves) if targets is None else np.asarray(targets)
    X = W.node_positions(tr, p)[targets].reshape(-1, d)
    u = np.zeros(len(X))
    nimg = int(np.ceil(np.sqrt(45.0 * delta))) + 1          # images beyond this are < 1e-19
    shifts = list(itertools.product(range(-nimg, nimg + 1), repeat=d)) if periodic else [(0,) * d]
    for s in range(tr.n_leaves):
        L = 2.0 ** -tr.level[s]
        c = -0.5 + (tr.coord[s] + 0.5) * L
        vals = sigma[s].reshape((p,) * d)                        # axes (j_d, ..., j_1)
        coef = vals
        for ax in range(d):                                      # Legendre coefficients per axis
            coef = np.moveaxis(np.tensordot(Vinv, coef, axes=([1], [ax])), 0, ax)
        sq = coef
        for ax in range(d):                                      # values at the quadrature grid
            sq = np.moveaxis(np.tensordot(Pq, sq, axes=([1], [ax])), 0, ax)
        grids = np.meshgrid(*([xq] * d), indexing="ij")           # axis a <-> x_{d-a}
        Y = np.stack([c[i] + 0.5 * L * grids[d - 1 - i] for i in range(d)], axis=-1).reshape(-1, d)
        Wq = np.ones(1)
        for _ in range(d):
            Wq = np.multiply.outer(Wq, wq).reshape(-1)
        Wq = Wq * (0.5 * L) ** d * sq.reshape(-1)
        for sh in shifts:
            # skip images whose whole leaf lies beyond exp(-r^2/delta) < 1e-19 of B
            gap = np.maximum(np.abs(c - np.asarray(sh, dtype=np.float64)) - 0.5 * L - 0.5, 0.0)
            if np.sum(gap ** 2) > 45.0 * delta:
                continue
            diff = X[:, None, :] - Y[None, :, :] + np.asarray(sh, dtype=np.float64)
            u += np.exp(-np.sum(diff ** 2, axis=-1) / delta) @ Wq
    return u.reshape(len(targets), p ** d)


@pytest.mark.parametrize("d,p,delta,periodic,seed", [(2, 5, 5e-2, False, 11), (2, 4, 2e-1, True, 12),
                                                     (3, 3, 1e-1, False, 13), (3, 3, 3e-2, True, 14)])
def test_brute_force_tiny_trees(d, p, delta, periodic, seed):
    if d == 3 and periodic:
        # 15 leaves: level 1 with one box split (keeps the image sum affordable)
        tr = W.refine_tree(3, lambda lev, c: lev == 0 or (lev == 1 and c == (0, 1, 0)), 2, periodic=True)
    else:
        tr = W.random_balanced_tree(d, seed, max_level=2, split_prob=0.5, periodic=periodic, min_level=1)
    assert tr.n_leaves <= 64
    sig = W.random_sigma(tr, p, seed)
    # 3D: a few target leaves of each level (the brute force is O(targets x sources x images))
    tg = np.arange(tr.n_leaves) if d == 2 else np.array([0, 1, tr.n_leaves - 2, tr.n_leaves - 1])
    u = oracle.box_fgt(d, p, delta, periodic, tr.level, tr.coord, sig, targets=tg)
    ub = _brute_force(d, p, delta, periodic, tr, sig, nq=32 if d == 2 else 20, targets=tg)
    assert np.abs(u - ub).max() <= 1e-11 * np.abs(ub).max()


def test_linearity():
    tr = W.random_balanced_tree(3, 21, max_level=3, min_level=1)
    p = 4
    a = W.random_sigma(tr, p, 1)
    b = W.random_sigma(tr, p, 2)
    f = lambda s: oracle.box_fgt(3, p, 3e-3, False, tr.level, tr.coord, s)
    ua, ub, uab = f(a), f(b), f(2.0 * a - 3.0 * b)
    assert np.abs(uab - (2.0 * ua - 3.0 * ub)).max() <= 1e-13 * np.abs(uab).max()


def test_periodic_shift_invariance():
    # translating sigma by one leaf on a uniform periodic tree translates u by one leaf
    d, lev, p, delta = 2, 3, 6, 4e-3
    tr = W.uniform_tree(d, lev, periodic=True)
    sig = W.random_sigma(tr, p, 5)
    n = 1 << lev
    idx = {tuple(c): i for i, c in enumerate(tr.coord)}
    perm = np.array([idx[((c[0] + 1) % n, (c[1] + 3) % n)] for c in tr.coord])
    u = oracle.box_fgt(d, p, delta, True, tr.level, tr.coord, sig)
    us = oracle.box_fgt(d, p, delta, True, tr.level, tr.coord, sig[perm])
    assert np.abs(us - u[perm]).max() <= 1e-13 * np.abs(u).max()


def test_reflection_symmetry():
    # x_1 -> -x_1 on a uniform tree maps leaf c -> n-1-c and reverses node index j_1
    d, lev, p, delta = 3, 2, 5, 1e-2
    tr = W.uniform_tree(d, lev)
    sig = W.random_sigma(tr, p, 9)
    n = 1 << lev
    idx = {tuple(c): i for i, c in enumerate(tr.coord)}
    perm = np.array([idx[(n - 1 - c[0], c[1], c[2])] for c in tr.coord])
    flip = lambda a: a.reshape(-1, p, p, p)[:, :, :, ::-1].reshape(a.shape)
    u = oracle.box_fgt(d, p, delta, False, tr.level, tr.coord, sig)
    ur = oracle.box_fgt(d, p, delta, False, tr.level, tr.coord, flip(sig[perm]))
    assert np.abs(ur - flip(u[perm])).max() <= 1e-13 * np.abs(u).max()


def test_positivity_for_positive_density():
    tr = W.gaussian_refined_tree(2, [[0.1, -0.2]], [0.05], rho=1.0, beta=4.0, max_level=6, min_level=2)
    p = 8
    s = W.gaussian_sum(W.node_positions(tr, p), [[0.1, -0.2]], [0.05 ** 2]) + 0.01
    u = oracle.box_fgt(2, p, 1e-3, False, tr.level, tr.coord, s)
    assert u.min() > 0


def test_target_subset_matches_full():
    tr = W.random_balanced_tree(2, 31, max_level=4, min_level=1)
    p = 6
    sig = W.random_sigma(tr, p, 3)
    full = oracle.box_fgt(2, p, 1e-3, False, tr.level, tr.coord, sig)
    sub = np.array([0, tr.n_leaves - 1, tr.n_leaves // 2])
    part = oracle.box_fgt(2, p, 1e-3, False, tr.level, tr.coord, sig, targets=sub, threads=2)
    assert np.array_equal(part, full[sub])


def test_golden_values():
    """Stored oracle values (written by tests/golden/make_golden.py, which calls
    only the oracle), so later changes to the oracle's arithmetic are caught."""
    import json
    with open(os.path.join(GOLDEN, "oracle_small.json")) as f:
        g = json.load(f)
    for key, c in g.items():
        u = oracle.box_fgt(c["d"], c["p"], c["delta"], c["periodic"], np.array(c["level"]),
                           np.array(c["coord"]), np.array(c["sigma"]))
        ref = np.array(c["u"])
        assert np.abs(u - ref).max() <= 1e-13 * np.abs(ref).max(), key


def _children(tree, depth=1):
    """Boxes `depth` levels below every leaf (an output tree refining the source tree)."""
    d = tree.d
    lev, crd = tree.level.copy(), tree.coord.copy()
    for _ in range(depth):
        off = np.array([[(c >> a) & 1 for a in range(d)] for c in range(1 << d)], dtype=np.int32)
        crd = (2 * crd[:, None, :] + off[None, :, :]).reshape(-1, d)
        lev = np.repeat(lev + 1, 1 << d)
    return W.Tree(d, lev.astype(np.int32), crd.astype(np.int32), tree.periodic)


@pytest.mark.parametrize("d,p,delta,depth", [(2, 8, 1e-2, 1), (2, 6, 1e-4, 2), (3, 5, 1e-2, 1)])
def test_target_boxes_constant_density_free_space(d, p, delta, depth):
    """u at the nodes of boxes refining the tree (Algorithm 5's output tree): sigma = 1 gives
    the product of erf differences at any point."""
    tr = W.random_balanced_tree(d, 11, max_level=3 if d == 2 else 2, min_level=1)
    out = _children(tr, depth)
    u = oracle.box_fgt_boxes(d, p, delta, False, tr.level, tr.coord, np.ones((tr.n_leaves, p ** d)),
                             out.level, out.coord)
    ex = _u_const_free(W.node_positions(out, p), delta)
    assert np.abs(u - ex).max() <= 1e-13 * np.abs(ex).max()


@pytest.mark.parametrize("d,p,delta", [(2, 16, 1e-2), (3, 12, 1e-2)])
def test_target_boxes_periodic_eigenfunction_and_coarser_boxes(d, p, delta):
    """Periodic trig density: u = lambda sigma_p at the nodes of finer and of coarser boxes."""
    tr = W.uniform_tree(d, 2, periodic=True)
    s = W.trig_density(W.node_positions(tr, p), 1)
    lam = (np.sqrt(np.pi * delta) * np.exp(-np.pi ** 2 * delta)) ** d
    for out in (_children(tr, 1), W.uniform_tree(d, 1, periodic=True)):
        u = oracle.box_fgt_boxes(d, p, delta, True, tr.level, tr.coord, s, out.level, out.coord)
        ex = lam * W.trig_density(W.node_positions(out, p), 1)
        assert np.abs(u - ex).max() <= 1e-10 * np.abs(ex).max()


def test_target_boxes_gaussian_density_closed_form():
    d, p, delta = 2, 16, 1e-3
    centers, alphas = np.array([[0.1, -0.2], [-0.25, 0.15]]), np.array([0.02, 0.01])
    tr = W.gaussian_refined_tree(d, centers, np.sqrt(alphas), rho=1.5, beta=3.0, max_level=5, min_level=2)
    s = W.gaussian_sum(W.node_positions(tr, p), centers, alphas)
    out = _children(tr, 1)
    u = oracle.box_fgt_boxes(d, p, delta, False, tr.level, tr.coord, s, out.level, out.coord)
    ex = _gauss_closed_form(W.node_positions(out, p), centers, alphas, delta)
    assert np.abs(u - ex).max() <= 1e-8 * np.abs(ex).max()


def test_point_fgt_single_source_and_superposition():
    """The discrete transform: one unit source gives the Gaussian itself; two sources add; a common
    shift of all points changes nothing; delta enters as exp(-r^2/delta)."""
    rng = np.random.default_rng(3)
    for d in (2, 3):
        x = rng.uniform(-0.5, 0.5, size=(50, d))
        y1, y2 = rng.uniform(-0.5, 0.5, size=(2, d))
        for delta in (1e-3, 3e-2, 1.0):
            g1 = np.exp(-((x - y1) ** 2).sum(axis=1) / delta)
            g2 = np.exp(-((x - y2) ** 2).sum(axis=1) / delta)
            u1 = oracle.point_fgt(d, delta, y1[None, :], [1.0], x)
            assert np.abs(u1 - g1).max() <= 1e-15
            u12 = oracle.point_fgt(d, delta, np.stack([y1, y2]), [2.0, -0.5], x)
            assert np.abs(u12 - (2 * g1 - 0.5 * g2)).max() <= 1e-14
            s = rng.uniform(-1, 1, size=d)
            us = oracle.point_fgt(d, delta, np.stack([y1, y2]) + s, [2.0, -0.5], x + s)
            assert np.abs(us - u12).max() <= 1e-13
