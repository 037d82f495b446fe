"""The split-precision evaluation with all three contractions on the fifth-generation tensor cores
(eval7_kernel: tcgen05.mma in 3xTF32, the incoming expansions staged by tensor-map copies from the
padded layout the gather writes), against the oracle (10 tol of max |u|) and against the CUDA-core
evaluation of the same plan (FP32-level agreement), for blocks of K = 8, 16 and 32 nodes per axis,
free space and periodic, small trees and the full-size workloads."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")

pytestmark = pytest.mark.gpu


def _run(monkeypatch, on, tree, p, delta, sig, bc=0, tol=1e-6, noalloc=False):
    monkeypatch.setenv("FGT_EVAL7", "1" if on else "0")
    plan = F.Plan(3, p, delta, tol, tree.level, tree.coord, bc=bc, prec=F.PREC_SPLIT)
    info = plan.info()
    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    u = plan(s).cpu().numpy()
    un = None
    if noalloc and 16 * info["modes_1d"] ** 2 * info["modes_half"] * info["n_anchor_boxes"] <= (48 << 20):
        o = torch.empty_like(s)   # the expansions of this plan fit the allocation-free scratch array
        plan.execute_noalloc(s, o)
        un = o.cpu().numpy()
    plan.close()
    return u, info, un


CASES = [
    # (tree, p, delta, bc): uniform level 4 at delta 3e-3 -> K = 32 blocks; at 1e-3 -> K = 16 (periodic);
    # random adaptive trees -> K = 8 / 16 / 32 mixes
    ("uniform4", 8, 3e-3, 0),
    ("uniform4p", 8, 1e-3, 1),
    ("random", 8, 3e-3, 0),
    ("random", 8, 1e-3, 0),
    ("randomp", 8, 4e-3, 1),
]


def _tree(name):
    if name.startswith("uniform4"):
        return W.uniform_tree(3, 4, periodic=name.endswith("p"))
    return W.random_balanced_tree(3, 31, max_level=4, min_level=2, split_prob=0.3, periodic=name.endswith("p"))


@pytest.mark.parametrize("name,p,delta,bc", CASES)
def test_all_stage_tcgen05_evaluation(monkeypatch, name, p, delta, bc):
    tr = _tree(name)
    sig = W.random_sigma(tr, p, 41)
    u7, info, un = _run(monkeypatch, True, tr, p, delta, sig, bc, noalloc=True)
    assert info["n_tc_eval_blocks"] == info["n_form_blocks"] > 0
    assert F.device_status() == 0
    u0, info0, _ = _run(monkeypatch, False, tr, p, delta, sig, bc)
    assert info0["n_tc_eval_blocks"] == 0
    scale = np.abs(u0).max()
    assert np.abs(u7 - u0).max() <= 2e-6 * scale
    # the allocation-free call keeps the plain layout and the CUDA-core evaluation
    if un is not None:
        assert np.abs(un - u0).max() <= 2e-6 * scale
    rng = np.random.default_rng(5)
    tg = np.sort(rng.choice(tr.n_leaves, min(48, tr.n_leaves), replace=False))
    uo = oracle.box_fgt(3, p, delta, bool(bc), tr.level, tr.coord, sig, targets=tg)
    assert np.abs(u7[tg] - uo).max() <= 10 * 1e-6 * np.abs(uo).max()


def _sample(w, n, seed):
    rng = np.random.default_rng(seed)
    tg = set(rng.choice(w.tree.n_leaves, n, replace=False).tolist())
    lev = w.tree.level.astype(np.float64)
    centre = (w.tree.coord + 0.5) / (2.0 ** lev)[:, None] - 0.5
    for c in w.meta.get("centers", [])[:8]:
        tg.add(int(np.argmin(((centre - c) ** 2).sum(axis=1))))
    return np.array(sorted(tg))


@pytest.mark.parametrize("which", ["adaptive", "periodic"])
def test_all_stage_tcgen05_evaluation_full_size(monkeypatch, which):
    """The benchmark's workloads (2.09M-point adaptive tree, 16.8M-point periodic level 5) with the
    tcgen05 evaluation, against the oracle on sampled target leaves."""
    w = (W.config_3d_free_adaptive(seed=0, p=8, delta=1e-3) if which == "adaptive"
         else W.config_3d_periodic_uniform(seed=0))
    u7, info, _ = _run(monkeypatch, True, w.tree, w.p, w.delta, w.sigma, int(w.periodic))
    assert info["n_tc_eval_blocks"] == info["n_form_blocks"] > 0
    assert F.device_status() == 0
    tg = _sample(w, 24, 9)
    uo = oracle.box_fgt(3, w.p, w.delta, w.periodic, w.tree.level, w.tree.coord, w.sigma, targets=tg)
    assert np.all(np.isfinite(u7))
    assert np.abs(u7[tg] - uo).max() <= 10 * 1e-6 * np.abs(uo).max()
