"""The split-precision form with all three contractions on the fifth-generation tensor cores
(form7_kernel: tcgen05.mma in 3xTF32, the packed density staged by tensor-map copies with the
swizzle of a K-float row), against the oracle (10 tol of max |u|) and against the CUDA-core form
of the same plan (FP32-level agreement), for blocks of K = 8, 16 and 32 nodes per axis, anchors
with one block (slot stored) and with several (slot added to), free space and periodic."""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")

pytestmark = pytest.mark.gpu


def _run(monkeypatch, form7, tree, p, delta, sig, bc=0, tol=1e-6, noalloc=False, eval7=True):
    monkeypatch.setenv("FGT_FORM7", "1" if form7 else "0")
    monkeypatch.setenv("FGT_EVAL7", "1" if eval7 else "0")
    plan = F.Plan(3, p, delta, tol, tree.level, tree.coord, bc=bc, prec=F.PREC_SPLIT)
    info = plan.info()
    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    u = plan(s).cpu().numpy()
    u2 = plan(s).cpu().numpy()   # a second call: the slots are rewritten, not accumulated
    un = None
    if noalloc and 16 * info["modes_1d"] ** 2 * info["modes_half"] * info["n_anchor_boxes"] <= (48 << 20):
        o = torch.empty_like(s)
        plan.execute_noalloc(s, o)
        un = o.cpu().numpy()
    plan.close()
    return u, u2, info, un


CASES = [
    ("uniform4", 8, 3e-3, 0),    # K = 32, one block per anchor (slots stored)
    ("uniform4p", 8, 1e-3, 1),   # K = 16, one block per anchor, periodic
    ("random", 8, 3e-3, 0),      # K = 8 / 16 / 32 mixed, several blocks per anchor (slots added to)
    ("random", 8, 1e-3, 0),
    ("randomp", 8, 4e-3, 1),
]


def _tree(name):
    if name.startswith("uniform4"):
        return W.uniform_tree(3, 4, periodic=name.endswith("p"))
    return W.random_balanced_tree(3, 31, max_level=4, min_level=2, split_prob=0.3, periodic=name.endswith("p"))


@pytest.mark.parametrize("name,p,delta,bc", CASES)
@pytest.mark.parametrize("eval7", [True, False])
def test_all_stage_tcgen05_form(monkeypatch, name, p, delta, bc, eval7):
    tr = _tree(name)
    sig = W.random_sigma(tr, p, 43)
    u7, u7b, info, un = _run(monkeypatch, True, tr, p, delta, sig, bc, noalloc=True, eval7=eval7)
    assert info["n_tc_form_blocks"] == info["n_form_blocks"] > 0
    assert F.device_status() == 0
    u0, _, info0, _ = _run(monkeypatch, False, tr, p, delta, sig, bc, eval7=False)
    assert info0["n_tc_form_blocks"] == 0
    scale = np.abs(u0).max()
    assert np.abs(u7 - u0).max() <= 2e-6 * scale
    assert np.abs(u7b - u7).max() <= 1e-6 * scale
    if un is not None:   # the allocation-free call falls back to the CUDA-core form
        assert np.abs(un - u0).max() <= 2e-6 * scale
    rng = np.random.default_rng(6)
    tg = np.sort(rng.choice(tr.n_leaves, min(48, tr.n_leaves), replace=False))
    uo = oracle.box_fgt(3, p, delta, bool(bc), tr.level, tr.coord, sig, targets=tg)
    assert np.abs(u7[tg] - uo).max() <= 10 * 1e-6 * np.abs(uo).max()


@pytest.mark.parametrize("which", ["adaptive", "periodic"])
def test_all_stage_tcgen05_form_full_size(monkeypatch, which):
    """Both tcgen05 kernels on the benchmark's workloads (2.09M-point adaptive tree, 16.8M-point
    periodic level 5), against the oracle on sampled target leaves."""
    w = (W.config_3d_free_adaptive(seed=0, p=8, delta=1e-3) if which == "adaptive"
         else W.config_3d_periodic_uniform(seed=0))
    u7, _, info, _ = _run(monkeypatch, True, w.tree, w.p, w.delta, w.sigma, int(w.periodic))
    assert info["n_tc_form_blocks"] == info["n_form_blocks"] == info["n_tc_eval_blocks"] > 0
    assert F.device_status() == 0
    rng = np.random.default_rng(10)
    tg = np.sort(rng.choice(w.tree.n_leaves, 24, replace=False))
    uo = oracle.box_fgt(3, w.p, w.delta, w.periodic, w.tree.level, w.tree.coord, w.sigma, targets=tg)
    assert np.all(np.isfinite(u7))
    assert np.abs(u7[tg] - uo).max() <= 10 * 1e-6 * np.abs(uo).max()


def test_default_mixes_tcgen05_and_cuda_core_forms(monkeypatch):
    """By default the tcgen05 form takes the blocks of K = 16 and 32 and the CUDA-core form the
    K = 8 ones, in one plan: the density is packed block by block in the order each kernel reads."""
    monkeypatch.delenv("FGT_FORM7", raising=False)
    monkeypatch.delenv("FGT_EVAL7", raising=False)
    tr = _tree("random")
    sig = W.random_sigma(tr, 8, 44)
    plan = F.Plan(3, 8, 3e-3, 1e-6, tr.level, tr.coord, prec=F.PREC_SPLIT)
    info = plan.info()
    u = plan(torch.from_numpy(sig).cuda()).cpu().numpy()
    plan.close()
    assert 0 < info["n_tc_form_blocks"] < info["n_form_blocks"]
    u0, _, _, _ = _run(monkeypatch, False, tr, 8, 3e-3, sig, eval7=False)
    assert np.abs(u - u0).max() <= 2e-6 * np.abs(u0).max()
    uo = oracle.box_fgt(3, 8, 3e-3, False, tr.level, tr.coord, sig)
    assert np.abs(u - uo).max() <= 10 * 1e-6 * np.abs(uo).max()
