"""Output trees (Algorithm 5): u at the nodes of a tree refining the source tree, through the C
ABI, against the oracle evaluated at the same target boxes."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")

pytestmark = pytest.mark.gpu


def refine(tree, pick, depth=1):
    """Subdivide the leaves selected by pick(i) `depth` times (the rest stay)."""
    d = tree.d
    off = np.array([[(c >> a) & 1 for a in range(d)] for c in range(1 << d)], dtype=np.int32)
    lev, crd = [], []
    for i in range(tree.n_leaves):
        if pick(i):
            l, c = np.array([tree.level[i]]), tree.coord[i][None, :]
            for _ in range(depth):
                c = (2 * c[:, None, :] + off[None, :, :]).reshape(-1, d)
                l = np.repeat(l + 1, 1 << d)
            lev.append(l)
            crd.append(c)
        else:
            lev.append(np.array([tree.level[i]]))
            crd.append(tree.coord[i][None, :])
    return W.Tree(d, np.concatenate(lev).astype(np.int32), np.concatenate(crd).astype(np.int32), tree.periodic)


def run(d, p, delta, tol, tree, sigma, out, bc=0, prec=0):
    plan = F.Plan(d, p, delta, tol, tree.level, tree.coord, bc=bc, prec=prec)
    plan.set_output_tree(out.level, out.coord)
    u = plan(torch.from_numpy(sigma).cuda())
    torch.cuda.synchronize()
    u = u.cpu().numpy()
    plan.close()
    uo = oracle.box_fgt_boxes(d, p, delta, bool(bc), tree.level, tree.coord, sigma, out.level, out.coord)
    err = np.abs(u - uo).max() / np.abs(uo).max()
    assert u.shape == uo.shape and np.all(np.isfinite(u))
    assert err <= 10 * tol, err
    return u


@pytest.mark.parametrize("delta,tol,prec", [(1e-2, 1e-10, 0), (1e-3, 1e-6, 1), (1e-4, 1e-9, 0)])
def test_2d_every_leaf_refined(delta, tol, prec):
    tr = W.random_balanced_tree(2, 4, max_level=5, min_level=1)
    run(2, 8, delta, tol, tr, W.random_sigma(tr, 8, 41), refine(tr, lambda i: True), prec=prec)


@pytest.mark.parametrize("delta,tol,prec", [(1e-3, 1e-6, 1), (1e-3, 1e-10, 0), (1e-2, 1e-8, 2), (3e-4, 1e-8, 0)])
def test_3d_some_leaves_refined_one_and_two_levels(delta, tol, prec):
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    rng = np.random.default_rng(3)
    pick = set(rng.choice(tr.n_leaves, tr.n_leaves // 3, replace=False).tolist())
    out1 = refine(tr, lambda i: i in pick)
    sig = W.random_sigma(tr, 6, 42)
    run(3, 6, delta, tol, tr, sig, out1, prec=prec)
    # two levels for a few leaves: blocks of K = 4k (uniform) next to single leaves
    few = set(list(pick)[:5])
    run(3, 6, delta, tol, tr, sig, refine(tr, lambda i: i in few, depth=2), prec=prec)


@pytest.mark.parametrize("delta", [1e-3, 3e-2])
def test_periodic_refined(delta):
    tr = W.random_balanced_tree(3, 9, max_level=3, min_level=2, split_prob=0.3, periodic=True)
    out = refine(tr, lambda i: i % 2 == 0)
    run(3, 4, delta, 1e-9, tr, W.random_sigma(tr, 4, 43), out, bc=1)


def test_identity_output_tree_equals_the_plain_transform():
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    sig = torch.from_numpy(W.random_sigma(tr, 6, 44)).cuda()
    plan = F.Plan(3, 6, 1e-3, 1e-8, tr.level, tr.coord)
    u0 = plan(sig).clone()
    plan.set_output_tree(tr.level, tr.coord)
    u1 = plan(sig).clone()
    plan.set_output_tree(None)
    u2 = plan(sig)
    torch.cuda.synchronize()
    assert (u1 - u0).abs().max().item() <= 1e-13 * u0.abs().max().item()
    assert (u2 - u0).abs().max().item() <= 1e-13 * u0.abs().max().item()
    plan.close()
