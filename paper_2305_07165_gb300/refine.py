"""Output-tree refinement and coarsening (the paper's Algorithms 5 and 6).

A level-restricted tree that resolves the density sigma need not resolve the potential u: a
sharp feature diffused a short distance can be too sharp for the input grid (Section 4.3), and a
smooth potential can be over-resolved.  ``refine`` evaluates u on an output tree that starts as
the source tree and subdivides every leaf whose error monitor (eq. funerr, computed on the GPU by
``fgt_leaf_errors``) exceeds eps * ||u||_2, at most down to the source tree's deepest level, until
no leaf is flagged; each round evaluates the transform only at the new leaves (an output tree of
the subdivided leaves' children, ``fgt_plan_set_output_tree``) and keeps the others' values.  ``coarsen`` walks the levels bottom-up and merges 2^d sibling
leaves into their parent when the parent's values (the children's interpolant at its nodes,
``fgt_merge_children``) pass the same monitor.  The tree bookkeeping is host logic; the
transform, the monitor and the interpolation run in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _check, lib


def leaf_errors(vals, d, k, stream=None):
    """(error monitor [n], quadrature sum of squares on [-1,1]^d [n]) of n boxes' node values
    (CUDA float64 [n, k**d])."""
    import torch
    vals = vals.contiguous()
    n = vals.shape[0]
    err = torch.empty(n, dtype=torch.float64, device=vals.device)
    sq = torch.empty(n, dtype=torch.float64, device=vals.device)
    st = stream if stream is not None else torch.cuda.current_stream(vals.device)
    _check(lib().fgt_leaf_errors(d, k, n, ctypes.c_void_p(vals.data_ptr()), ctypes.c_void_p(err.data_ptr()),
                                 ctypes.c_void_p(sq.data_ptr()), ctypes.c_void_p(st.cuda_stream)))
    return err, sq


def merge_children(vals, child_rows, d, k, stream=None):
    """Parent node values from 2^d children each (rows child_rows[p * 2^d + c] of vals, child c
    in the half (c >> a) & 1 along axis a)."""
    import torch
    rows = torch.as_tensor(np.ascontiguousarray(child_rows, dtype=np.int64)).to(vals.device)
    n_par = rows.numel() >> d
    out = torch.empty((n_par, k ** d), dtype=torch.float64, device=vals.device)
    st = stream if stream is not None else torch.cuda.current_stream(vals.device)
    _check(lib().fgt_merge_children(d, k, n_par, ctypes.c_void_p(rows.data_ptr()), ctypes.c_void_p(vals.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream)))
    return out


def _norm(sq, level, d):
    """||u||_2 over B = [-1/2, 1/2]^d from the per-leaf quadrature sums on [-1,1]^d."""
    scale = (0.5 * np.ldexp(1.0, -np.asarray(level, dtype=np.int64))) ** d
    return float(np.sqrt(np.sum(sq.cpu().numpy() * scale)))


def _children(level, coord, d):
    off = np.array([[(c >> a) & 1 for a in range(d)] for c in range(1 << d)], dtype=np.int32)
    return (np.repeat(level + 1, 1 << d).astype(np.int32),
            (2 * coord[:, None, :] + off[None, :, :]).reshape(-1, d).astype(np.int32))


def refine(plan, sigma, eps, max_level=None, max_rounds=64):
    """Algorithm 5.  plan: a Plan on the source tree (its output tree is changed, and restored to
    the source tree at the end); sigma: CUDA [n_leaves, k**d].  Returns (level, coord, u) of the
    refined output tree and the number of rounds.  The first round evaluates u on the source tree;
    each later round evaluates it only at the children of the leaves flagged in the round before
    (an output tree of those children alone) and keeps every other leaf's values.  Leaves are not
    subdivided below max_level (default: the source tree's deepest)."""
    import torch
    d, k = plan.d, plan.k
    level = np.asarray(plan._src_level, dtype=np.int32).copy()
    coord = np.asarray(plan._src_coord, dtype=np.int32).reshape(-1, d).copy()
    lmax = int(level.max()) if max_level is None else int(max_level)
    plan.set_output_tree(None)
    u = plan(sigma)
    err, sq = leaf_errors(u, d, k)
    err, sq = err.cpu().numpy(), sq.cpu().numpy()
    rounds = 1
    while True:
        norm = float(np.sqrt(np.sum(sq * (0.5 * np.ldexp(1.0, -level.astype(np.int64))) ** d)))
        flag = (err > eps * norm) & (level < lmax)
        if not flag.any() or rounds >= max_rounds:
            plan.set_output_tree(None)
            return level, coord, u, rounds
        cl, cc = _children(level[flag], coord[flag], d)
        plan.set_output_tree(cl, cc)
        un = plan(sigma)                      # the new leaves only
        rounds += 1
        en, sn = leaf_errors(un, d, k)
        keep = np.where(~flag)[0]
        u = torch.cat([u[torch.as_tensor(keep, device=u.device)], un])
        level = np.concatenate([level[keep], cl])
        coord = np.concatenate([coord[keep], cc])
        err = np.concatenate([err[keep], en.cpu().numpy()])
        sq = np.concatenate([sq[keep], sn.cpu().numpy()])


def interpolate(level, coord, u, d, k, points):
    """The tensor Lagrange interpolant of node values u [n, k**d] (CUDA or numpy; node index t_1
    fastest, Gauss-Legendre nodes) at points [m, d] of B, on the host.  Returns [m]."""
    u = u.cpu().numpy() if hasattr(u, "cpu") else np.asarray(u)
    level = np.asarray(level, dtype=np.int64)
    coord = np.asarray(coord, dtype=np.int64).reshape(-1, d)
    x = np.polynomial.legendre.leggauss(k)[0]
    pts = np.asarray(points, dtype=np.float64).reshape(-1, d)
    # the leaf containing each point, level by level (keys level * 2^60 + packed coordinates)
    def pack(l, c):
        kk = np.asarray(l, dtype=np.int64) << 60
        for a in range(d):
            kk = kk | (np.asarray(c[..., a], dtype=np.int64) << (20 * a))
        return kk
    keys = pack(level, coord)
    order = np.argsort(keys)
    sk = keys[order]
    leaf = np.full(len(pts), -1, dtype=np.int64)
    for l in range(int(level.min()), int(level.max()) + 1):
        todo = leaf < 0
        if not todo.any():
            break
        c = np.minimum(np.floor((pts[todo] + 0.5) * (1 << l)), (1 << l) - 1).astype(np.int64)
        kq = pack(np.full(len(c), l), c)
        pos = np.clip(np.searchsorted(sk, kq), 0, len(sk) - 1)
        hit = sk[pos] == kq
        idx = np.where(todo)[0]
        leaf[idx[hit]] = order[pos[hit]]
    L = np.ldexp(1.0, -level[leaf])
    s = (pts - (-0.5 + (coord[leaf] + 0.5) * L[:, None])) / (0.5 * L[:, None])
    vals = u[leaf].reshape((len(pts),) + (k,) * d)          # [m, t_d, ..., t_1]
    for a in range(d):                                      # contract t_1 (last axis) first
        lag = np.ones((len(pts), k))
        for j in range(k):
            for m in range(k):
                if m != j:
                    lag[:, j] *= (s[:, a] - x[m]) / (x[j] - x[m])
        vals = np.einsum("m...j,mj->m...", vals, lag)
    return vals


def coarsen(level, coord, u, d, k, eps, norm=None):
    """Algorithm 6: returns (level, coord, u) with every set of 2^d sibling leaves whose parent
    passes the error monitor (e <= eps * ||u||_2) merged into the parent, bottom-up."""
    import torch
    level = np.asarray(level, dtype=np.int32)
    coord = np.asarray(coord, dtype=np.int32).reshape(-1, d)
    if norm is None:
        _, sq = leaf_errors(u, d, k)
        norm = _norm(sq, level, d)
    for l in range(int(level.max()) - 1, -1, -1):
        sel = np.where(level == l + 1)[0]
        if len(sel) == 0:
            continue
        parent = coord[sel] >> 1
        key = {}
        for i, c in zip(sel, map(tuple, parent)):
            key.setdefault(c, []).append(i)
        groups = [(c, ids) for c, ids in key.items() if len(ids) == 1 << d]
        if not groups:
            continue
        rows = np.zeros((len(groups), 1 << d), dtype=np.int64)
        for g, (c, ids) in enumerate(groups):
            for i in ids:
                ch = sum(((int(coord[i, a]) & 1) << a) for a in range(d))
                rows[g, ch] = i
        pv = merge_children(u, rows.reshape(-1), d, k)
        err, _ = leaf_errors(pv, d, k)
        ok = err.cpu().numpy() <= eps * norm
        if not ok.any():
            continue
        drop = np.zeros(len(level), dtype=bool)
        drop[rows[ok].reshape(-1)] = True
        keep = np.where(~drop)[0]
        new_coord = np.array([groups[g][0] for g in np.where(ok)[0]], dtype=np.int32).reshape(-1, d)
        level = np.concatenate([level[keep], np.full(len(new_coord), l, dtype=np.int32)])
        coord = np.concatenate([coord[keep], new_coord])
        u = torch.cat([u[torch.as_tensor(keep, device=u.device)], pv[torch.as_tensor(np.where(ok)[0], device=u.device)]])
    return level, coord, u
