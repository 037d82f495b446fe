"""FP64-accurate form and evaluation on the BF16 tensor cores (precision FP64_TC, 3D, fused mode):
every FP64 operand cut into six 8-bit digits, the slice products accumulated exactly in FP32 on the
tensor cores, recombined in 64-bit integers.  Against the oracle at 10 tol (tol 1e-10 and 1e-6),
against the plain FP64 path of the same problem (agreement at FP64 level, 1e-12 of max |u|), for
blocks of K = 8 .. 64 nodes a side, free space and periodic, anchors with one block (slot stored)
and several (slot added to), a second call on the same plan, and the allocation-free call (which
keeps the FP64 kernels)."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")

pytestmark = pytest.mark.gpu


def _u(monkeypatch, sliced, tree, p, delta, tol, sig, bc=0, prec=None, noalloc=False):
    monkeypatch.setenv("FGT_OZAKI", "1" if sliced else "0")
    plan = F.Plan(3, p, delta, tol, tree.level, tree.coord, bc=bc, prec=F.PREC_FP64_TC if prec is None else prec)
    info = plan.info()
    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    u = plan(s).cpu().numpy()
    u2 = plan(s).cpu().numpy()
    un = None
    if noalloc and 16 * info["modes_1d"] ** 2 * info["modes_half"] * info["n_anchor_boxes"] <= (48 << 20):
        o = torch.empty_like(s)
        plan.execute_noalloc(s, o)
        un = o.cpu().numpy()
    plan.close()
    return u, u2, info, un


CASES = [
    # (tree, p, delta, tol, bc)
    ("uniform3", 8, 1e-2, 1e-10, 0),    # level 3 under l_c = 1: K = 32 blocks, one per anchor
    ("uniform3p", 8, 1e-3, 1e-10, 1),   # periodic, l_c = 2: K = 16, n1 = 65
    ("uniform3", 4, 1e-2, 1e-6, 0),     # k = 4
    ("random", 6, 1e-3, 1e-10, 0),      # K = 6 .. 24 mixed, several blocks per anchor
    ("randomp", 4, 1e-3, 1e-10, 1),
    ("uniform4", 4, 1e-2, 1e-10, 0),    # K = 64 blocks (k = 4, 16 leaves a side)
    ("random5", 4, 1e-4, 1e-10, 0),     # cutoff level 4 with empty boxes: the line-stencil gather
    ("random5p", 4, 1e-4, 1e-10, 1),
]


def _tree(name):
    if name.startswith("uniform"):
        return W.uniform_tree(3, int(name[7]), periodic=name.endswith("p"))
    if name.startswith("random5"):
        return W.random_balanced_tree(3, 32, max_level=5, min_level=3, split_prob=0.15, periodic=name.endswith("p"))
    return W.random_balanced_tree(3, 31, max_level=4, min_level=2, split_prob=0.3, periodic=name.endswith("p"))


@pytest.mark.parametrize("name,p,delta,tol,bc", CASES)
def test_sliced_fp64_tensor_core(monkeypatch, name, p, delta, tol, bc):
    tr = _tree(name)
    sig = W.random_sigma(tr, p, 51)
    u, u2, info, un = _u(monkeypatch, True, tr, p, delta, tol, sig, bc, noalloc=True)
    assert F.device_status() == 0
    u0, _, info0, _ = _u(monkeypatch, True, tr, p, delta, tol, sig, bc, prec=F.PREC_FP64)
    scale = np.abs(u0).max()
    assert np.abs(u - u0).max() <= 1e-12 * scale
    assert np.abs(u2 - u).max() <= 1e-12 * scale   # rewrites (atomic sums differ in order), does not accumulate
    if un is not None:  # the allocation-free call keeps the FP64 (DMMA) kernels
        assert np.abs(un - u0).max() <= 1e-12 * scale
    # fewer launches than the FP64 path is not implied; the sliced path is six stage launches
    assert info["launches"] >= 6
    rng = np.random.default_rng(8)
    tg = np.sort(rng.choice(tr.n_leaves, min(40, tr.n_leaves), replace=False))
    uo = oracle.box_fgt(3, p, delta, bool(bc), tr.level, tr.coord, sig, targets=tg)
    assert np.abs(u[tg] - uo).max() <= 10 * tol * np.abs(uo).max()


def test_sliced_matches_dmma_path(monkeypatch):
    """The same FP64_TC plan with the sliced stages and with the DMMA kernels (FGT_OZAKI=0)."""
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    sig = W.random_sigma(tr, 6, 52)
    u, _, _, _ = _u(monkeypatch, True, tr, 6, 1e-3, 1e-10, sig)
    ud, _, _, _ = _u(monkeypatch, False, tr, 6, 1e-3, 1e-10, sig)
    assert np.abs(u - ud).max() <= 1e-12 * np.abs(ud).max()


def test_sliced_full_size_periodic():
    """The 16.8M-point periodic level-5 workload at tol 1e-10 (64 blocks of K = 64, n1 = 65),
    sampled target leaves against the oracle."""
    w = W.config_3d_periodic_uniform(seed=0)
    plan = F.Plan(3, w.p, w.delta, 1e-10, w.tree.level, w.tree.coord, bc=1, prec=F.PREC_FP64_TC)
    u = plan(torch.from_numpy(w.sigma).cuda()).cpu().numpy()
    plan.close()
    assert F.device_status() == 0
    rng = np.random.default_rng(11)
    tg = np.sort(rng.choice(w.tree.n_leaves, 16, replace=False))
    uo = oracle.box_fgt(3, w.p, w.delta, True, w.tree.level, w.tree.coord, w.sigma, targets=tg)
    assert np.all(np.isfinite(u))
    assert np.abs(u[tg] - uo).max() <= 10 * 1e-10 * np.abs(uo).max()
