"""Pins of the oracle's tree construction (paper Section 4, Algorithm 3, eq. funerr), on the CPU.

What fixes the tree, checked here without reusing the oracle's own routines:
  * a polynomial density of total degree < k has a zero tail, so the tree is the root
    (or the uniform tree at min_level);
  * every leaf of the refinement loop passes the monitor, and its parent failed it (or was
    below min_level): the monitor recomputed from the node values by an independent
    least-squares Legendre fit, against the threshold the oracle used at that level;
  * that threshold is eps ||sigma||_2, ||sigma||_2 computed separably by 1D quadrature;
  * the final tree tiles B, is level-restricted (leaves sharing a boundary point, across the
    faces of B when periodic, differ by at most one level), refines the loop's leaves, and is
    the coarsest such tree (every box the restriction split had a neighbour two levels finer).
"""
import itertools

import numpy as np
import pytest

from oracle import tree as OT


def _indep_monitor(vals, d, k):
    """e of eq. (funerr) from node values by a least-squares fit of the tensor Legendre basis
    (numpy's Vandermonde matrices; exact interpolation on the k^d Gauss nodes)."""
    eta, _ = np.polynomial.legendre.leggauss(k)
    V1 = np.polynomial.legendre.legvander(eta, k - 1)         # [node j][degree n]
    V = V1
    for _ in range(d - 1):
        V = np.kron(V, V1)                                    # node / degree index: last axis fastest
    c = np.linalg.solve(V, vals.T).T                           # [box][alpha_d .. alpha_1], alpha_1 fastest
    idx = np.array(list(itertools.product(range(k), repeat=d)))
    tail = (idx ** 2).sum(axis=1) >= k * k
    if not tail.any():
        return np.zeros(len(vals))
    return np.sqrt(np.mean(c[:, tail] ** 2, axis=1))


def _touch(la, ca, lb, cb, periodic):
    """Closed boxes (level, coord) share at least one boundary point (minimum image if periodic)."""
    for a in range(len(ca)):
        lo1, hi1 = ca[a] / 2.0 ** la, (ca[a] + 1) / 2.0 ** la
        lo2, hi2 = cb[a] / 2.0 ** lb, (cb[a] + 1) / 2.0 ** lb
        ok = any(lo1 <= hi2 + s and lo2 + s <= hi1 for s in ((-1.0, 0.0, 1.0) if periodic else (0.0,)))
        if not ok:
            return False
    return True


def _contains(lp, cp, l, c):
    return l >= lp and all((c[a] >> (l - lp)) == cp[a] for a in range(len(c)))


@pytest.mark.parametrize("d,k", [(2, 6), (3, 4)])
def test_polynomial_density_gives_the_root_or_the_min_level(d, k):
    def poly(x):                                   # total degree k - 1: every ||alpha||_2 <= k - 1
        return 1.0 + x[..., 0] ** (k - 1) + 0.5 * x[..., 0] * x[..., 1] ** (k - 2) - 0.3 * x[..., d - 1] ** 2
    lev, crd = OT.build_tree_fn(d, k, poly, eps=1e-13, min_level=0, max_level=6)
    assert len(lev) == 1 and lev[0] == 0
    lev, crd = OT.build_tree_fn(d, k, poly, eps=1e-13, min_level=2, max_level=6)
    assert len(lev) == 4 ** d and np.all(lev == 2)


@pytest.mark.parametrize("d,k,periodic,eps", [(2, 8, False, 1e-8), (2, 6, True, 1e-7), (3, 6, False, 1e-6),
                                              (3, 4, True, 1e-5)])
def test_refinement_loop_and_level_restriction(d, k, periodic, eps):
    rng = np.random.default_rng(3 * d + k)
    centers = rng.uniform(-0.4, 0.4, size=(3, d))
    alphas = np.array([3e-3, 1e-3, 6e-4])
    max_level = 7 if d == 2 else 5
    lev, crd, info = OT.build_tree(d, k, centers, alphas, periodic=periodic, eps=eps, min_level=1,
                                   max_level=max_level, return_unbalanced=True)
    # leaves of the loop pass the monitor; their parents failed it (or sat below min_level)
    for it in info:
        l, c = it["level"], np.array(it["coord"])
        x = OT.box_nodes(d, k, np.array([l]), c[None, :])
        e = _indep_monitor(OT.gaussian_density(x, centers, alphas, periodic=periodic), d, k)[0]
        assert l == max_level or e <= it["thr"] * (1 + 1e-9)
        par = it["parent"]
        if par is not None and not par[2]:
            xp = OT.box_nodes(d, k, np.array([l - 1]), (c >> 1)[None, :])
            ep = _indep_monitor(OT.gaussian_density(xp, centers, alphas, periodic=periodic), d, k)[0]
            assert ep > par[1] * (1 - 1e-9)
    # the threshold is eps ||sigma||_2: at the deepest level, where the interpolant resolves sigma,
    # against the norm of sigma over B computed separably (each product of two Gaussians by 1D
    # adaptive quadrature of its per-axis factors)
    from scipy.integrate import quad
    def g1(x, c, a):
        t = x - c
        if periodic:
            t = t - np.rint(t)
        return np.exp(-t * t / a)
    norm2 = 0.0
    for i in range(len(alphas)):
        for j in range(len(alphas)):
            prod = 1.0
            for ax in range(d):
                pts = sorted({float(np.clip(centers[i][ax], -0.5, 0.5)), float(np.clip(centers[j][ax], -0.5, 0.5))})
                prod *= quad(lambda x: g1(x, centers[i][ax], alphas[i]) * g1(x, centers[j][ax], alphas[j]),
                             -0.5, 0.5, points=pts, limit=200, epsabs=0, epsrel=1e-12)[0]
            norm2 += prod
    deepest = max(it["level"] for it in info)
    thr = [it["thr"] for it in info if it["level"] == deepest][0]
    assert abs(thr - eps * np.sqrt(norm2)) <= 1e-4 * eps * np.sqrt(norm2), (thr, eps * np.sqrt(norm2))
    loop = [(it["level"], tuple(it["coord"])) for it in info]
    leaves = list(zip(lev.tolist(), [tuple(c) for c in crd.tolist()]))
    # tiles B: volumes add to 1 and no leaf contains another
    assert abs(sum(0.5 ** (d * l) for l, _ in leaves) - 1.0) < 1e-12
    assert len(set(leaves)) == len(leaves)
    # level-restricted
    for i, (la, ca) in enumerate(leaves):
        for lb, cb in leaves[i + 1:]:
            if abs(la - lb) > 1:
                assert not _touch(la, ca, lb, cb, periodic), ((la, ca), (lb, cb))
    # refines the loop's leaves
    for l, c in loop:
        assert any(_contains(l, c, lb, cb) for lb, cb in leaves)
    # coarsest: the restriction only splits a box that touches a leaf two or more levels finer, so
    # the parent of every leaf it created touches such a leaf in the final tree
    loop_set = set(loop)
    for l, c in leaves:
        if (l, c) in loop_set:
            continue
        pl, pc = l - 1, tuple(v >> 1 for v in c)
        assert any(lb >= pl + 2 and _touch(pl, pc, lb, cb, periodic) for lb, cb in leaves), (l, c)


def test_tail_mask_counts():
    """N_{k,2} of eq. (funerr): the multi-indices of [0, k)^d with ||alpha||_2 >= k."""
    assert OT.tail_mask(2, 4).sum() == 1           # only (3, 3)
    assert OT.tail_mask(2, 3).sum() == 0
    brute = sum(1 for a in itertools.product(range(8), repeat=3) if sum(v * v for v in a) >= 64)
    assert OT.tail_mask(3, 8).sum() == brute
