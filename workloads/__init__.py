"""Seeded synthetic inputs for the box Gauss transform: trees and node values.

This module is shared by the tests, the benchmark and the oracle's callers.  It
holds none of the transform's arithmetic: it builds leaf lists (uniform, or
refined geometrically around Gaussian bumps and then 2:1 balanced) and samples
a density at the tensor-product Gauss-Legendre nodes of every leaf (the layout
the transform's interface prescribes: node t of a leaf with centre c and side
L sits at c + (L/2) eta_t, eta the ascending Gauss-Legendre nodes on [-1, 1],
node index j_1 fastest).  Node positions come from ``numpy.polynomial``.

Densities follow the paper's test densities (Section 6, eqs. (sigmap),
(sigmaf)): sums of Gaussians exp(-|x - c_i|^2 / alpha_i) and products of
sin / cos of 2 pi n x_i, plus seeded uniform noise where a workload asks for it.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Tree:
    d: int
    level: np.ndarray            # int32 [n_leaves]
    coord: np.ndarray            # int32 [n_leaves, d]
    periodic: bool = False

    @property
    def n_leaves(self) -> int:
        return int(len(self.level))


@dataclass
class Workload:
    name: str
    d: int
    p: int
    delta: float
    periodic: bool
    tree: Tree
    sigma: np.ndarray            # float64 [n_leaves, p**d]
    meta: dict = field(default_factory=dict)

    @property
    def n_points(self) -> int:
        return self.tree.n_leaves * self.p ** self.d


# ----------------------------------------------------------------------------- trees

def uniform_tree(d: int, level: int, periodic: bool = False) -> Tree:
    n = 1 << level
    grids = np.meshgrid(*([np.arange(n)] * d), indexing="ij")
    # x_1 fastest in leaf order as well (reversed axis order in the flattening)
    coord = np.stack([g.T.reshape(-1) for g in grids], axis=1).astype(np.int32)
    return Tree(d, np.full(len(coord), level, dtype=np.int32), coord, periodic)


def _box_center(level, c):
    return -0.5 + (np.asarray(c, dtype=np.float64) + 0.5) * 2.0 ** (-level)


def _box_point_dist(level, c, x, periodic):
    L = 2.0 ** (-level)
    ctr = _box_center(level, c)
    dc = np.abs(ctr - x)
    if periodic:
        dc = np.minimum(dc, 1.0 - dc)
    gap = np.maximum(dc - 0.5 * L, 0.0)
    return float(np.sqrt(np.sum(gap * gap)))


def refine_tree(d, should_split, max_level, periodic=False, balance=True) -> Tree:
    """Top-down refinement: split a box while should_split(level, coord) holds."""
    leaves = []
    stack = [(0, (0,) * d)]
    while stack:
        lev, c = stack.pop()
        if lev < max_level and should_split(lev, c):
            for ch in itertools.product((0, 1), repeat=d):
                stack.append((lev + 1, tuple(2 * ci + bi for ci, bi in zip(c, ch))))
        else:
            leaves.append((lev, c))
    if balance:
        leaves = balance_leaves(d, leaves, periodic)
    leaves.sort(key=lambda t: (t[0], t[1][::-1]))
    lev = np.array([t[0] for t in leaves], dtype=np.int32)
    crd = np.array([t[1] for t in leaves], dtype=np.int32).reshape(len(leaves), d)
    return Tree(d, lev, crd, periodic)


def balance_leaves(d, leaves, periodic=False):
    """Refine until leaves sharing a boundary point (corners included, across the
    periodic wrap when asked) differ by at most one level."""
    leafset = set(leaves)
    queue = list(leafset)
    offsets = [o for o in itertools.product((-1, 0, 1), repeat=d) if any(o)]

    def covering_leaf(lev, c):
        for up in range(lev + 1):
            key = (lev - up, tuple(ci >> up for ci in c))
            if key in leafset:
                return key
        return None

    while queue:
        t = queue.pop()
        if t not in leafset:
            continue
        lev, c = t
        n = 1 << lev
        for o in offsets:
            nc = []
            ok = True
            for ci, oi in zip(c, o):
                v = ci + oi
                if v < 0 or v >= n:
                    if not periodic:
                        ok = False
                        break
                    v %= n
                nc.append(v)
            if not ok:
                continue
            s = covering_leaf(lev, tuple(nc))
            if s is not None and s[0] < lev - 1:
                leafset.discard(s)
                sl, sc = s
                for ch in itertools.product((0, 1), repeat=d):
                    kid = (sl + 1, tuple(2 * ci + bi for ci, bi in zip(sc, ch)))
                    leafset.add(kid)
                    queue.append(kid)
                queue.append(t)
                break
    return list(leafset)


def gaussian_refined_tree(d, centers, widths, rho, beta=4.0, max_level=12, periodic=False, min_level=0,
                          balance=True):
    """Split a box while it is wider than rho*w_i and lies within beta*w_i of centre c_i."""
    centers = np.asarray(centers, dtype=np.float64)
    widths = np.asarray(widths, dtype=np.float64)

    def should_split(lev, c):
        if lev < min_level:
            return True
        L = 2.0 ** (-lev)
        for ci, wi in zip(centers, widths):
            if L > rho * wi and _box_point_dist(lev, c, ci, periodic) < beta * wi:
                return True
        return False

    return refine_tree(d, should_split, max_level, periodic, balance=balance)


# ----------------------------------------------------------------------------- nodes / densities

def leaf_nodes(p: int):
    """Ascending Gauss-Legendre nodes on [-1, 1] (numpy's rule)."""
    x, _ = np.polynomial.legendre.leggauss(p)
    return x


def node_positions(tree: Tree, p: int) -> np.ndarray:
    """x[n_leaves, p**d, d]: positions of every leaf node, node index j_1 fastest."""
    d = tree.d
    eta = leaf_nodes(p)
    L = 2.0 ** (-tree.level.astype(np.float64))
    ctr = -0.5 + (tree.coord.astype(np.float64) + 0.5) * L[:, None]
    idx = np.stack(np.meshgrid(*([np.arange(p)] * d), indexing="ij"), axis=-1)  # [p]*d + [d], axis0 = j_1
    idx = idx.transpose(*reversed(range(d)), d).reshape(-1, d)                  # j_1 fastest
    e = eta[idx]                                                                 # [p^d, d]
    return ctr[:, None, :] + 0.5 * L[:, None, None] * e[None, :, :]


def gaussian_sum(x, centers, alphas, amps=None, periodic=False):
    """sum_i a_i exp(-|x - c_i|^2 / alpha_i); periodic: minimum-image distance to each centre."""
    centers = np.asarray(centers, dtype=np.float64)
    alphas = np.asarray(alphas, dtype=np.float64)
    amps = np.ones(len(centers)) if amps is None else np.asarray(amps, dtype=np.float64)
    out = np.zeros(x.shape[:-1])
    for c, a, w in zip(centers, alphas, amps):
        dx = x - c
        if periodic:
            dx = dx - np.round(dx)
        out += w * np.exp(-np.sum(dx * dx, axis=-1) / a)
    return out


def trig_density(x, n):
    """Paper eq. (sigmap): prod over odd i of sin(2 pi n x_i), even i of cos(2 pi n x_i)."""
    out = np.ones(x.shape[:-1])
    for i in range(x.shape[-1]):
        f = np.sin if i % 2 == 0 else np.cos   # i = 0 is the paper's x_1 (odd)
        out = out * f(2.0 * np.pi * n * x[..., i])
    return out


# ----------------------------------------------------------------------------- named workloads

def config_2d_free_uniform(seed=0, p=8, level=3, delta=1e-2, n_gauss=3):
    """2D free space, uniform level-3 tree (64 leaves), p=8, delta=1e-2, 3 Gaussians
    with centres U(B) and widths U[0.05, 0.2] (alpha = width^2)."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-0.5, 0.5, size=(n_gauss, 2))
    widths = rng.uniform(0.05, 0.2, size=n_gauss)
    tree = uniform_tree(2, level)
    sigma = gaussian_sum(node_positions(tree, p), centers, widths ** 2)
    return Workload("2d-free-uniform-l3-p8", 2, p, delta, False, tree, sigma,
                    dict(seed=seed, centers=centers, alphas=widths ** 2))


def _tune_rho(d, centers, widths, target_leaves, beta, max_level, periodic):
    lo, hi = 0.05, 50.0
    best = None
    for _ in range(40):
        mid = np.sqrt(lo * hi)
        tr = gaussian_refined_tree(d, centers, widths, mid, beta, max_level, periodic)
        if best is None or abs(tr.n_leaves - target_leaves) < abs(best[1].n_leaves - target_leaves):
            best = (mid, tr)
        if tr.n_leaves > target_leaves:
            lo = mid
        else:
            hi = mid
        if abs(tr.n_leaves - target_leaves) <= 0.03 * target_leaves:
            break
    return best


def config_3d_free_adaptive(seed=0, p=8, delta=1e-3, n_gauss=8, target_points=2_000_000,
                            beta=4.0, max_level=11):
    """3D free space, adaptive 2:1-balanced tree refined around 8 Gaussians with
    centres U([-0.4,0.4]^3) and widths log-U[1e-3, 1e-1] (alpha = width^2); the
    refinement ratio is tuned so that N = n_leaves p^3 is close to target_points."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-0.4, 0.4, size=(n_gauss, 3))
    widths = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), size=n_gauss))
    rho, tree = _tune_rho(3, centers, widths, target_points / p ** 3, beta, max_level, False)
    sigma = gaussian_sum(node_positions(tree, p), centers, widths ** 2)
    return Workload(f"3d-free-adaptive-p{p}", 3, p, delta, False, tree, sigma,
                    dict(seed=seed, centers=centers, alphas=widths ** 2, rho=rho, beta=beta))


def config_3d_periodic_uniform(seed=0, p=8, level=5, delta=1e-3, n_gauss=16, noise=1.0):
    """3D periodic, uniform level-5 tree (32768 leaves), p=8 (16.8M points), 16
    Gaussians (centres U(B), widths log-U[1e-2, 1e-1]) plus i.i.d. U[-1,1] noise."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-0.5, 0.5, size=(n_gauss, 3))
    widths = np.exp(rng.uniform(np.log(1e-2), np.log(1e-1), size=n_gauss))
    tree = uniform_tree(3, level, periodic=True)
    x = node_positions(tree, p)
    sigma = gaussian_sum(x, centers, widths ** 2, periodic=True)
    if noise:
        sigma = sigma + rng.uniform(-noise, noise, size=sigma.shape)
    return Workload(f"3d-periodic-uniform-l{level}-p{p}", 3, p, delta, True, tree, sigma,
                    dict(seed=seed, centers=centers, alphas=widths ** 2, noise=noise))


# centres of the paper's free-space density (Section 6, eqs. sigmaf / xi3d); in 2D their projections
# on the x_1 x_2 plane
PAPER_SIGMA_F_CENTRES_3D = np.array([(-0.3, -0.4, -0.06), (-0.2, 0.0, -0.25), (0.18, -0.1, -0.03),
                                     (-0.09, 0.3, 0.17), (-0.38, -0.05, -0.17)])


def paper_sigma_f(d=3, p=16, delta=1e-3, n_g=5, alpha1=None, target_points=None, beta=4.0, max_level=10):
    """The paper's free-space experiment (Section 6): sigma_f = sum_i exp(-|x - x_i|^2 / alpha_i)
    with its five centres, alpha_i = alpha_1 / i (alpha_1 = 4e-3 in 3D, 1e-5 in 2D), k = 16
    nodes per axis.  The tree is refined geometrically around the centres (widths sqrt(alpha_i))
    and 2:1 balanced; with target_points set, the refinement ratio is tuned to about that size."""
    if alpha1 is None:
        alpha1 = 4e-3 if d == 3 else 1e-5
    centers = PAPER_SIGMA_F_CENTRES_3D[:n_g, :d]
    alphas = alpha1 / np.arange(1, n_g + 1)
    widths = np.sqrt(alphas)
    if target_points is None:
        rho, tree = 1.0, gaussian_refined_tree(d, centers, widths, 1.0, beta, max_level)
    else:
        rho, tree = _tune_rho(d, centers, widths, target_points / p ** d, beta, max_level, False)
    sigma = gaussian_sum(node_positions(tree, p), centers, alphas)
    return Workload(f"paper-sigma-f-{d}d-p{p}", d, p, delta, False, tree, sigma,
                    dict(centers=centers, alphas=alphas, rho=rho, beta=beta))


def paper_sigma_p(d=3, p=16, delta=1e-3, n_p=4, level=3):
    """The paper's periodic experiment (Section 6, eq. sigmap): trig density with n_p = 4 in 3D
    (32 in 2D) on a uniform tree, k = 16."""
    tree = uniform_tree(d, level, periodic=True)
    sigma = trig_density(node_positions(tree, p), n_p)
    return Workload(f"paper-sigma-p-{d}d-p{p}-l{level}", d, p, delta, True, tree, sigma, dict(n_p=n_p))


def batched_configs(seed=0, n=256, max_points=1 << 18):
    """n independent free-space transforms: d in {2,3}, tree depth U{2..7}, p in {8,12,16},
    delta log-U[1e-5, 1e-1], sigma a sum of 1..8 Gaussians (widths log-U[1e-2, 2e-1]).  Each
    transform is capped at max_points (the depth is lowered until the tree fits)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        d = int(rng.choice([2, 3]))
        depth = int(rng.integers(2, 8))
        p = int(rng.choice([8, 12, 16]))
        delta = float(np.exp(rng.uniform(np.log(1e-5), np.log(1e-1))))
        ng = int(rng.integers(1, 9))
        centers = rng.uniform(-0.4, 0.4, size=(ng, d))
        widths = np.exp(rng.uniform(np.log(1e-2), np.log(2e-1), size=ng))
        while True:  # size the depth on the unbalanced tree, balance only the final one
            tree = gaussian_refined_tree(d, centers, widths, rho=1.0, beta=3.0, max_level=depth, min_level=1,
                                         balance=False)
            if tree.n_leaves * p ** d * 1.5 <= max_points or depth <= 1:
                break
            depth -= 1
        tree = gaussian_refined_tree(d, centers, widths, rho=1.0, beta=3.0, max_level=depth, min_level=1)
        sigma = gaussian_sum(node_positions(tree, p), centers, widths ** 2)
        out.append(Workload(f"batch{i}-{d}d-p{p}-L{depth}", d, p, delta, False, tree, sigma,
                            dict(seed=seed, index=i)))
    return out


def serving_mix(seed=0, n=24, max_points=1 << 22):
    """n distinct request geometries for the serving loop: d in {2, 3}, free space or periodic
    (3 in 10), tol 1e-6 or 1e-10 (1 in 4, stored in meta["tol"]), delta log-U[1e-4, 1e-2],
    sizes log-spread from about 4K points up to max_points.  Free-space trees are refined around
    1..8 Gaussians (as in batched_configs), periodic ones are uniform (level drawn to the size)
    with a periodic Gaussian sum."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        d = int(rng.choice([2, 3]))
        per = bool(rng.uniform() < 0.3)
        tol = 1e-10 if rng.uniform() < 0.25 else 1e-6
        delta = float(np.exp(rng.uniform(np.log(1e-4), np.log(1e-2))))
        p = int(rng.choice([8, 12]))
        target = float(np.exp(rng.uniform(np.log(4096), np.log(max_points))))
        ng = int(rng.integers(1, 9))
        centers = rng.uniform(-0.4, 0.4, size=(ng, d))
        widths = np.exp(rng.uniform(np.log(1e-2), np.log(2e-1), size=ng))
        if per:
            level = max(1, int(round(np.log(max(target / p ** d, 1.0)) / np.log(2 ** d))))
            while (1 << (d * level)) * p ** d > max_points and level > 1:
                level -= 1
            tree = uniform_tree(d, level, periodic=True)
            sigma = gaussian_sum(node_positions(tree, p), centers, widths ** 2, periodic=True)
        else:
            depth = 9 if d == 2 else 7
            while True:
                tree = gaussian_refined_tree(d, centers, widths, rho=1.0, beta=3.0, max_level=depth, min_level=1,
                                             balance=False)
                if tree.n_leaves * p ** d * 1.5 <= min(target, max_points) or depth <= 2:
                    break
                depth -= 1
            tree = gaussian_refined_tree(d, centers, widths, rho=1.0, beta=3.0, max_level=depth, min_level=1)
            sigma = gaussian_sum(node_positions(tree, p), centers, widths ** 2)
        out.append(Workload(f"serve{i}-{d}d-{'per' if per else 'free'}-p{p}", d, p, delta, per, tree, sigma,
                            dict(seed=seed, index=i, tol=tol)))
    return out


def random_balanced_tree(d, seed, max_level=4, split_prob=0.45, periodic=False, min_level=0):
    """Random refinement (each box split with probability split_prob, seeded) then 2:1 balance."""
    rng = np.random.default_rng(seed)
    memo = {}

    def should_split(lev, c):
        if lev < min_level:
            return True
        key = (lev, c)
        if key not in memo:
            memo[key] = rng.uniform() < split_prob
        return memo[key]

    return refine_tree(d, should_split, max_level, periodic)


def random_sigma(tree: Tree, p: int, seed: int):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(tree.n_leaves, p ** tree.d))
