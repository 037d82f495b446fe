"""Output-tree refinement and coarsening (the paper's Algorithms 5 and 6).

A level-restricted tree that resolves the density sigma need not resolve the potential u: a
sharp feature diffused a short distance can be too sharp for the input grid (Section 4.3), and a
smooth potential can be over-resolved.  ``refine`` evaluates u on an output tree that starts as
the source tree and subdivides every leaf whose error monitor (eq. funerr, computed on the GPU by
``fgt_leaf_errors``) exceeds eps * ||u||_2, at most down to the source tree's deepest level, until
no leaf is flagged; each round re-evaluates the transform on the new output tree
(``fgt_plan_set_output_tree``).  ``coarsen`` walks the levels bottom-up and merges 2^d sibling
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
    """Algorithm 5.  plan: a Plan on the source tree (its output tree is changed); sigma: CUDA
    [n_leaves, k**d].  Returns (level, coord, u) of the refined output tree and the number of
    rounds.  Leaves are not subdivided below max_level (default: the source tree's deepest)."""
    d, k = plan.d, plan.k
    level = np.asarray(plan._src_level, dtype=np.int32).copy()
    coord = np.asarray(plan._src_coord, dtype=np.int32).reshape(-1, d).copy()
    lmax = int(level.max()) if max_level is None else int(max_level)
    rounds = 0
    while True:
        plan.set_output_tree(level, coord)
        u = plan(sigma)
        rounds += 1
        err, sq = leaf_errors(u, d, k)
        flag = (err.cpu().numpy() > eps * _norm(sq, level, d)) & (level < lmax)
        if not flag.any() or rounds >= max_rounds:
            return level, coord, u, rounds
        cl, cc = _children(level[flag], coord[flag], d)
        level = np.concatenate([level[~flag], cl])
        coord = np.concatenate([coord[~flag], cc])


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
