"""Adaptive tree construction for a continuous density (paper Section 4, Algorithm 3, eq. funerr).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): plain numpy, FP64, written from the
algorithm's steps.  The tests compare the tree the GPU builds against this one, leaf for leaf.

Steps, in the algorithm's order, for level l = 0, 1, ...:
  * every box B at level l: the density at its k^d tensor Gauss-Legendre nodes;
  * its Legendre coefficients c_alpha (the val -> pol map of Definition val2pol, per axis
    c_n = (2n+1)/2 sum_j w_j P_n(eta_j) v_j);
  * the error monitor of eq. (funerr): e = sqrt(mean of |c_alpha|^2 over ||alpha||_2 >= k), the
    mean taken over the N_{k,2} multi-indices of that tail inside the k^d cube;
  * B is subdivided into its 2^d children when e > eps ||sigma||_2 (and always below min_level,
    never at max_level);
then the leaves are refined until the tree is level-restricted (leaves that share a boundary
point differ by at most one level; across the faces of B when periodic).

Reading of ||sigma||_2 (the paper does not say over which boxes it is taken): the L2 norm of the
density over the current partition of B -- the leaves already final plus the boxes of level l --
each box's integral of sigma^2 taken by its own tensor Gauss-Legendre rule.

The density is sigma(x) = sum_i a_i exp(-|x - c_i|^2 / alpha_i), minimum-image distance to each
centre when periodic (the paper's sigma_f form).
"""
from __future__ import annotations

import itertools

import numpy as np


def gaussian_density(x, centers, alphas, amps=None, periodic=False):
    """sum_i a_i exp(-|x - c_i|^2 / alpha_i) at points x[..., d]."""
    centers = np.asarray(centers, dtype=np.float64)
    alphas = np.asarray(alphas, dtype=np.float64)
    amps = np.ones(len(alphas)) if amps is None else np.asarray(amps, dtype=np.float64)
    out = np.zeros(x.shape[:-1])
    for c, a, w in zip(centers, alphas, amps):
        dx = x - c
        if periodic:
            dx = dx - np.rint(dx)
        out = out + w * np.exp(-np.sum(dx * dx, axis=-1) / a)
    return out


def val2pol_matrix(k):
    """T[n][j] = (2n+1)/2 w_j P_n(eta_j) on the k Gauss-Legendre nodes (Definition val2pol)."""
    eta, w = np.polynomial.legendre.leggauss(k)
    P = np.polynomial.legendre.legvander(eta, k - 1).T     # P[n][j] = P_n(eta_j)
    return (2 * np.arange(k)[:, None] + 1) / 2.0 * w[None, :] * P


def tail_mask(d, k):
    """Multi-indices alpha in [0, k)^d with ||alpha||_2 >= k (the tail of eq. funerr), as a
    boolean array indexed [alpha_d, ..., alpha_1]."""
    a = np.arange(k)
    grids = np.meshgrid(*([a] * d), indexing="ij")
    return sum(g * g for g in grids) >= k * k


def box_nodes(d, k, level, coord):
    """Tensor Gauss-Legendre nodes of boxes (level [n], coord [n, d]), node index t_1 fastest:
    returns x [n, k^d, d]."""
    eta, _ = np.polynomial.legendre.leggauss(k)
    L = np.ldexp(1.0, -np.asarray(level))
    centre = -0.5 + (np.asarray(coord, dtype=np.float64) + 0.5) * L[:, None]
    idx = np.array(list(itertools.product(range(k), repeat=d)))[:, ::-1]   # [t][axis], axis 0 fastest
    return centre[:, None, :] + 0.5 * L[:, None, None] * eta[idx][None, :, :]


def monitor(vals, d, k):
    """Error monitor e (eq. funerr) and the quadrature integral of v^2 on the reference box
    [-1, 1]^d, for node values vals [n, k^d] (t_1 fastest)."""
    T = val2pol_matrix(k)
    _, w = np.polynomial.legendre.leggauss(k)
    n = vals.shape[0]
    c = vals.reshape((n,) + (k,) * d)           # [n, t_d, ..., t_1]
    for ax in range(1, d + 1):                  # c_alpha: apply T along every axis
        c = np.moveaxis(np.tensordot(c, T, axes=([ax], [1])), -1, ax)
    mask = tail_mask(d, k)
    if mask.any():
        e = np.sqrt(np.mean(np.abs(c[:, mask]) ** 2, axis=1))
    else:                                        # k too small for a tail: nothing to monitor
        e = np.zeros(n)
    wt = w
    for _ in range(d - 1):
        wt = np.multiply.outer(w, wt)
    sq = np.sum(vals.reshape((n,) + (k,) * d) ** 2 * wt[None], axis=tuple(range(1, d + 1)))
    return e, sq


def _neighbours(d, level, c, periodic):
    """Boxes at `level` sharing a boundary point with box c (corners included), wrapped when periodic."""
    n = 1 << level
    out = []
    for off in itertools.product((-1, 0, 1), repeat=d):
        if not any(off):
            continue
        q = []
        for a in range(d):
            v = c[a] + off[a]
            if v < 0 or v >= n:
                if not periodic:
                    break
                v %= n
            q.append(v)
        else:
            out.append(tuple(q))
    return out


def balance(d, leaves, periodic):
    """Level restriction: split any leaf that has a neighbour leaf two or more levels finer,
    until none does.  leaves: set of (level, coord tuple)."""
    leaves = set(leaves)
    changed = True
    while changed:
        changed = False
        for (l, c) in sorted(leaves, key=lambda t: -t[0]):
            if (l, c) not in leaves:
                continue
            for q in _neighbours(d, l, c, periodic):
                # the leaf covering neighbour position q at a level coarser than l - 1
                for up in range(2, l + 1):
                    pc = tuple(v >> up for v in q)
                    if (l - up, pc) in leaves:
                        leaves.discard((l - up, pc))
                        for ch in itertools.product((0, 1), repeat=d):
                            leaves.add((l - up + 1, tuple(2 * pc[a] + ch[d - 1 - a] for a in range(d))))
                        changed = True
                        break
    return leaves


def build_tree(d, k, centers, alphas, amps=None, periodic=False, eps=1e-10, min_level=0, max_level=12,
               return_unbalanced=False):
    """Algorithm 3 for a sum of Gaussians.  Returns (level [n], coord [n, d]) of the leaves of the
    level-restricted tree sorted by (level, coord), and with return_unbalanced also the leaves the
    refinement loop produced before the level restriction, each with its own monitor and threshold
    and its parent's."""
    def fn(x):
        return gaussian_density(x, centers, alphas, amps, periodic)
    return build_tree_fn(d, k, fn, periodic, eps, min_level, max_level, return_unbalanced)


def build_tree_fn(d, k, density, periodic=False, eps=1e-10, min_level=0, max_level=12, return_unbalanced=False):
    """Algorithm 3 for a density given as a function of points x[..., d] (see build_tree)."""
    active = [(0, (0,) * d)]
    final = []
    final_sq = 0.0
    history = []           # (leaf level, coord, parent e, parent threshold) for the unbalanced leaves' parents
    parents = {}
    for l in range(max_level + 1):
        if not active:
            break
        lev = np.full(len(active), l)
        crd = np.array([c for _, c in active], dtype=np.int64)
        vals = density(box_nodes(d, k, lev, crd))
        e, sq = monitor(vals, d, k)
        vol = (0.5 * np.ldexp(1.0, -l)) ** d
        norm2 = final_sq + float(np.sum(sq)) * vol
        thr = eps * np.sqrt(norm2)
        nxt = []
        for i, (_, c) in enumerate(active):
            split = l < max_level and (l < min_level or e[i] > thr)
            if split:
                for ch in itertools.product((0, 1), repeat=d):
                    kid = tuple(2 * c[a] + ch[d - 1 - a] for a in range(d))
                    nxt.append((l + 1, kid))
                    parents[(l + 1, kid)] = (float(e[i]), float(thr), l < min_level)
            else:
                final.append((l, c))
                final_sq += float(sq[i]) * vol
                history.append((l, c, float(e[i]), float(thr)))
        active = nxt
    bal = sorted(balance(d, final, periodic))
    level = np.array([l for l, _ in bal], dtype=np.int32)
    coord = np.array([c for _, c in bal], dtype=np.int32).reshape(-1, d)
    if not return_unbalanced:
        return level, coord
    info = [dict(level=l, coord=c, e=ev, thr=tv, parent=parents.get((l, c))) for l, c, ev, tv in history]
    return level, coord, info
