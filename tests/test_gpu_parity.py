"""GPU (CUDA, through the C ABI) against the CPU oracle, element by element.

Acceptance: max |u_gpu - u_oracle| <= 10 tol max |u_oracle| (the bar stated for
this transform), on seeded inputs spanning several blocks, ragged (adaptive)
trees, both boundary conditions, d = 2 and 3, both execution modes and both
precisions (split only at tol >= 1e-7).
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")

pytestmark = pytest.mark.gpu


def gpu_u(d, p, delta, tol, tree, sigma, bc=0, prec=0, mode=0):
    plan = F.Plan(d, p, delta, tol, tree.level, tree.coord, bc=bc, prec=prec, mode=mode)
    s = torch.from_numpy(np.ascontiguousarray(sigma)).cuda()
    u = plan(s)
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    info = plan.info()
    plan.close()
    return out, info


def check(d, p, delta, tol, tree, sigma, bc=0, prec=0, mode=0, targets=None):
    u, info = gpu_u(d, p, delta, tol, tree, sigma, bc, prec, mode)
    if targets is None:
        uo = oracle.box_fgt(d, p, delta, bool(bc), tree.level, tree.coord, sigma)
        ug = u
    else:
        uo = oracle.box_fgt(d, p, delta, bool(bc), tree.level, tree.coord, sigma, targets=targets)
        ug = u[targets]
    assert np.all(np.isfinite(u))
    err = np.abs(ug - uo).max() / np.abs(uo).max()
    assert err <= 10 * tol, (err, info)
    return err, info


@pytest.mark.parametrize("tol", [1e-6, 1e-9, 1e-10])
def test_2d_free_uniform_level3(tol):
    w = W.config_2d_free_uniform(seed=0)
    check(2, w.p, w.delta, tol, w.tree, w.sigma)


@pytest.mark.parametrize("delta,tol", [(1e-1, 1e-6), (1e-2, 1e-10), (1e-3, 1e-6), (1e-3, 1e-10), (1e-4, 1e-10)])
@pytest.mark.parametrize("mode", [0, 1])
def test_2d_free_adaptive(delta, tol, mode):
    tr = W.random_balanced_tree(2, 4, max_level=6, min_level=1)
    sig = W.random_sigma(tr, 6, 11)
    check(2, 6, delta, tol, tr, sig, mode=mode)


@pytest.mark.parametrize("delta,tol", [(1e-1, 1e-8), (1e-2, 1e-10), (3e-3, 1e-8), (2e-4, 1e-8)])
def test_2d_periodic_adaptive(delta, tol):
    tr = W.random_balanced_tree(2, 7, max_level=5, min_level=1, periodic=True, split_prob=0.35)
    sig = W.random_sigma(tr, 6, 12)
    check(2, 6, delta, tol, tr, sig, bc=1)


@pytest.mark.parametrize("delta,tol", [(1e-1, 1e-6), (1e-2, 1e-10), (1e-3, 1e-6), (1e-3, 1e-10), (3e-4, 1e-8)])
@pytest.mark.parametrize("mode", [0, 1])
def test_3d_free_adaptive(delta, tol, mode):
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    sig = W.random_sigma(tr, 4, 13)
    check(3, 4, delta, tol, tr, sig, mode=mode)


@pytest.mark.parametrize("delta,tol", [(5e-2, 1e-8), (5e-3, 1e-10), (1e-3, 1e-6), (1e-3, 1e-10)])
def test_3d_periodic(delta, tol):
    tr = W.random_balanced_tree(3, 9, max_level=3, min_level=2, split_prob=0.3, periodic=True)
    sig = W.random_sigma(tr, 4, 14)
    check(3, 4, delta, tol, tr, sig, bc=1)


@pytest.mark.parametrize("d,delta", [(2, 1e-3), (3, 1e-3), (3, 1e-2)])
def test_split_precision(d, delta):
    if d == 2:
        tr = W.random_balanced_tree(2, 4, max_level=6, min_level=1)
        p = 8
    else:
        tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
        p = 6
    sig = W.random_sigma(tr, p, 15)
    check(d, p, delta, 1e-6, tr, sig, prec=1)


@pytest.mark.parametrize("d,delta", [(2, 3e-3), (2, 2e-4), (3, 1e-3), (3, 2e-3)])
def test_split_precision_periodic(d, delta):
    """Split precision with periodic wrap-around of the cutoff-level gather (runs of boxes along
    x_1 whose neighbours wrap, cutoff grids of 4 to 32 boxes per axis)."""
    if d == 2:
        tr = W.random_balanced_tree(2, 7, max_level=6, min_level=2, periodic=True, split_prob=0.35)
        p = 8
    else:
        tr = W.random_balanced_tree(3, 9, max_level=4, min_level=2, split_prob=0.25, periodic=True)
        p = 4
    sig = W.random_sigma(tr, p, 19)
    _, info = check(d, p, delta, 1e-6, tr, sig, bc=1, prec=1)
    assert info["cutoff_level"] >= 2


@pytest.mark.parametrize("delta,tol", [(1e-3, 1e-6), (1e-3, 1e-10), (1e-2, 1e-10), (3e-4, 1e-8)])
def test_fp64_tensor_core(delta, tol):
    """FP64 contractions on the tensor cores (DMMA): against the oracle, and against the
    CUDA-core FP64 path, which does the same FP64 products in another order."""
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    sig = W.random_sigma(tr, 6, 23)
    check(3, 6, delta, tol, tr, sig, prec=F.PREC_FP64_TC)
    u_tc, info = gpu_u(3, 6, delta, tol, tr, sig, prec=F.PREC_FP64_TC)
    assert info["prec"] == F.PREC_FP64_TC
    u_64, _ = gpu_u(3, 6, delta, tol, tr, sig, prec=F.PREC_FP64)
    assert np.abs(u_tc - u_64).max() <= 1e-12 * np.abs(u_64).max()


def test_fp64_tensor_core_periodic_and_large_blocks():
    tr = W.random_balanced_tree(3, 9, max_level=3, min_level=2, split_prob=0.3, periodic=True)
    check(3, 4, 1e-3, 1e-10, tr, W.random_sigma(tr, 4, 24), bc=1, prec=F.PREC_FP64_TC)
    tr3 = W.uniform_tree(3, 3)  # K = 32 blocks under the level-1 cutoff boxes
    check(3, 8, 1e-2, 1e-8, tr3, W.random_sigma(tr3, 8, 25), prec=F.PREC_FP64_TC)


def test_split_precision_large_blocks():
    """Split precision, uniform subtrees of K = 32 nodes per axis under each cutoff-level box:
    one block per CTA, sigma streamed from global memory in the first contraction."""
    tr = W.uniform_tree(3, 3)
    sig = W.random_sigma(tr, 8, 21)
    check(3, 8, 1e-2, 1e-6, tr, sig, prec=1)


def test_3d_uniform_p8_sampled():
    """3D free space, uniform level-4 tree, p = 8 (2M points): sampled targets."""
    tr = W.uniform_tree(3, 4)
    rng = np.random.default_rng(3)
    sig = rng.uniform(-1, 1, size=(tr.n_leaves, 512))
    tg = np.sort(rng.choice(tr.n_leaves, 24, replace=False))
    check(3, 8, 1e-3, 1e-10, tr, sig, targets=tg)
    check(3, 8, 1e-3, 1e-6, tr, sig, targets=tg, prec=1)


def test_single_leaf_and_root_cases():
    # one leaf (the root): free space is direct-only; periodic uses the root Fourier series
    tr = W.uniform_tree(2, 0)
    sig = W.random_sigma(tr, 8, 3)
    check(2, 8, 1e-2, 1e-8, tr, sig)
    check(2, 8, 1e-2, 1e-8, tr, sig, bc=1)
    tr3 = W.uniform_tree(3, 0)
    check(3, 6, 2e-2, 1e-8, tr3, W.random_sigma(tr3, 6, 4), bc=1)


def test_linearity_and_repeat():
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    plan = F.Plan(3, 4, 1e-3, 1e-8, tr.level, tr.coord)
    a = torch.from_numpy(W.random_sigma(tr, 4, 1)).cuda()
    b = torch.from_numpy(W.random_sigma(tr, 4, 2)).cuda()
    ua, ub, uab = plan(a).clone(), plan(b).clone(), plan(2 * a - 3 * b).clone()
    ua2 = plan(a)
    torch.cuda.synchronize()
    # repeatable up to the order of the atomic additions into the anchor expansions
    assert (ua - ua2).abs().max().item() <= 1e-13 * ua.abs().max().item()
    assert (uab - (2 * ua - 3 * ub)).abs().max().item() <= 1e-12 * uab.abs().max().item()
    plan.close()


def test_host_entry_point_matches_device():
    tr = W.random_balanced_tree(2, 4, max_level=5, min_level=1)
    sig = W.random_sigma(tr, 6, 5)
    plan = F.Plan(2, 6, 1e-3, 1e-8, tr.level, tr.coord)
    ud = plan(torch.from_numpy(sig).cuda()).cpu()
    sh = torch.from_numpy(sig).pin_memory()
    uh = torch.empty_like(sh).pin_memory()
    plan.execute_host(sh, uh)
    assert (uh - ud).abs().max().item() <= 1e-13 * ud.abs().max().item()
    plan.close()


def test_invalid_tree_rejected_on_gpu_plan():
    lev = np.array([1, 1, 1], dtype=np.int32)
    crd = np.array([[0, 0], [1, 0], [0, 1]], dtype=np.int32)
    with pytest.raises(F.FGTError) as e:
        F.Plan(2, 4, 1e-3, 1e-6, lev, crd)
    assert e.value.status == 2


def test_split_precision_tensor_core_evaluation(monkeypatch):
    """The tensor-core (3xTF32) evaluation kernel, off by default, selected with FGT_TC_EVAL=1."""
    monkeypatch.setenv("FGT_TC_EVAL", "1")
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    sig = W.random_sigma(tr, 8, 16)
    check(3, 8, 1e-3, 1e-6, tr, sig, prec=1)
    check(3, 8, 1e-2, 1e-6, tr, sig, prec=1)


@pytest.mark.parametrize("prec", [1, 0])
def test_autotune_keeps_the_result(prec):
    """The autotuner only changes launch shapes: the tuned plan gives the same transform."""
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    p, tol = 8, 1e-6
    sig = torch.from_numpy(W.random_sigma(tr, p, 26)).cuda()
    plan = F.Plan(3, p, 1e-3, tol, tr.level, tr.coord, prec=prec)
    u0 = plan(sig).clone()
    knobs = plan.autotune(sig, reps=2)
    assert knobs["ms"] > 0 and plan.tuning() == knobs
    u1 = plan(sig)
    torch.cuda.synchronize()
    assert (u1 - u0).abs().max().item() <= 10 * tol * u0.abs().max().item()
    plan.set_tuning(form_group=2, eval_rows16=16, eval_rows_large=8, near_phase=0)
    u2 = plan(sig)
    torch.cuda.synchronize()
    assert (u2 - u0).abs().max().item() <= 10 * tol * u0.abs().max().item()
    plan.close()


def test_split_precision_tensor_core_evaluation_stages_2_3(monkeypatch):
    """Evaluation with its second and third contractions in 3xTF32 on the tensor cores
    (selected with FGT_TC_EVAL4=1): K = 8, 16 and 32 blocks, n1 up to 35."""
    monkeypatch.setenv("FGT_TC_EVAL4", "1")
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    sig = W.random_sigma(tr, 8, 27)
    check(3, 8, 1e-3, 1e-6, tr, sig, prec=1)
    check(3, 8, 1e-2, 1e-6, tr, sig, prec=1)
    tr3 = W.uniform_tree(3, 3)
    check(3, 8, 1e-2, 1e-6, tr3, W.random_sigma(tr3, 8, 28), prec=1)


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (0, 1e-6), (0, 1e-10)])
def test_evaluation_half_range_axis_last(monkeypatch, prec, tol):
    """The evaluation contracted m1, m2, then the half-range m3 (FGT_EVAL5=1): adaptive blocks of
    K = 6 to 24 (p = 6), K = 32 blocks, and a periodic tree."""
    monkeypatch.setenv("FGT_EVAL5", "1")
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    check(3, 6, 1e-3, tol, tr, W.random_sigma(tr, 6, 29), prec=prec)
    check(3, 6, 1e-2, tol, tr, W.random_sigma(tr, 6, 30), prec=prec)
    tr3 = W.uniform_tree(3, 3)
    check(3, 8, 1e-2, tol, tr3, W.random_sigma(tr3, 8, 31), prec=prec)
    trp = W.random_balanced_tree(3, 9, max_level=4, min_level=2, split_prob=0.25, periodic=True)
    check(3, 4, 1e-3, tol, trp, W.random_sigma(trp, 4, 32), bc=1, prec=prec)


def _sample_targets(w, n, seed):
    """Seeded target leaves, plus the leaf nearest to each Gaussian centre and leaves on the faces."""
    rng = np.random.default_rng(seed)
    tg = set(rng.choice(w.tree.n_leaves, n, replace=False).tolist())
    lev = w.tree.level.astype(np.float64)
    centre = (w.tree.coord + 0.5) / (2.0 ** lev)[:, None] - 0.5
    for c in w.meta.get("centers", [])[:8]:
        tg.add(int(np.argmin(((centre - c) ** 2).sum(axis=1))))
    on_face = np.where(np.any((w.tree.coord == 0) | (w.tree.coord == (2 ** w.tree.level)[:, None] - 1), axis=1))[0]
    tg.update(rng.choice(on_face, min(4, len(on_face)), replace=False).tolist())
    return np.array(sorted(tg))


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (0, 1e-10), (2, 1e-6), (2, 1e-10)])
def test_full_size_adaptive_workload_sampled(prec, tol):
    """The benchmark's 3D free-space adaptive workload (2.09M points, delta 1e-3) as the
    benchmark runs it, checked on sampled target leaves."""
    w = W.config_3d_free_adaptive(seed=0, p=8, delta=1e-3)
    check(3, w.p, w.delta, tol, w.tree, w.sigma, prec=prec, targets=_sample_targets(w, 24, 5))


@pytest.fixture(scope="module")
def periodic_full():
    """3D periodic, uniform level 5 (16.8M points): the workload and the oracle on sampled leaves."""
    w = W.config_3d_periodic_uniform(seed=0)
    tg = _sample_targets(w, 24, 6)
    uo = oracle.box_fgt(3, w.p, w.delta, True, w.tree.level, w.tree.coord, w.sigma, targets=tg)
    return w, tg, uo


@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (0, 1e-10), (0, 1e-6), (2, 1e-6), (2, 1e-10)])
def test_full_size_periodic_workload_sampled(periodic_full, prec, tol):
    """The benchmark's headline workload in every form it times, sampled target leaves."""
    w, tg, uo = periodic_full
    u, info = gpu_u(3, w.p, w.delta, tol, w.tree, w.sigma, bc=1, prec=prec)
    assert np.all(np.isfinite(u))
    err = np.abs(u[tg] - uo).max() / np.abs(uo).max()
    assert err <= 10 * tol, (err, info)


@pytest.mark.parametrize("delta", [1e-4, 1e-2])
def test_full_size_adaptive_delta_sweep_sampled(delta):
    """The benchmark's delta sweep on the 2.09M-point adaptive tree (same tree and density, delta
    1e-4 and 1e-2), every form it times, against the oracle on sampled target leaves."""
    w = W.config_3d_free_adaptive(seed=0, p=8, delta=1e-3)
    tg = _sample_targets(w, 24, 7)
    uo = oracle.box_fgt(3, w.p, delta, False, w.tree.level, w.tree.coord, w.sigma, targets=tg)
    for prec, tol in [(1, 1e-6), (0, 1e-6), (0, 1e-10), (2, 1e-6), (2, 1e-10)]:
        u, info = gpu_u(3, w.p, delta, tol, w.tree, w.sigma, prec=prec)
        assert np.all(np.isfinite(u))
        err = np.abs(u[tg] - uo).max() / np.abs(uo).max()
        assert err <= 10 * tol, (prec, tol, err, info)


@pytest.mark.parametrize("delta", [1e-10, 1e-6, 1e-3, 1e-1, 1.0])
@pytest.mark.parametrize("prec,tol", [(1, 1e-6), (0, 1e-10)])
def test_paper_free_space_density_k16(delta, prec, tol):
    """The paper's free-space experiment shape (Section 6): sigma_f with its five centres,
    alpha_i = 4e-3 / i, k = 16 nodes per axis, delta from 1e-10 (all direct) to 1 (root expansion)."""
    w = W.paper_sigma_f(d=3, p=16, target_points=200_000)
    check(3, 16, delta, tol, w.tree, w.sigma, prec=prec)


@pytest.mark.parametrize("delta", [1e-4, 1e-3, 1e-2])
def test_paper_periodic_density_k16(delta):
    """The paper's periodic density (eq. sigmap, n_p = 4) at k = 16: an eigenfunction of the
    periodic kernel, so u = (sqrt(pi delta) exp(-pi^2 delta n_p^2))^3 sigma up to interpolation."""
    w = W.paper_sigma_p(d=3, p=16, n_p=4, level=2)
    check(3, 16, delta, 1e-10, w.tree, w.sigma, bc=1)
    lam = (np.sqrt(np.pi * delta) * np.exp(-np.pi ** 2 * delta * 16)) ** 3
    ug, _ = gpu_u(3, 16, delta, 1e-10, w.tree, w.sigma, bc=1)
    assert np.abs(ug - lam * w.sigma).max() <= 1e-8 * np.abs(lam * w.sigma).max()


def _split_u(monkeypatch, tc6, tree, p, delta, sig, bc=0, tuning=None):
    monkeypatch.setenv("FGT_TC_EVAL6", "1" if tc6 else "0")
    plan = F.Plan(3, p, delta, 1e-6, tree.level, tree.coord, bc=bc, prec=F.PREC_SPLIT)
    if tuning:
        plan.set_tuning(**tuning)
    u = plan(torch.from_numpy(np.ascontiguousarray(sig)).cuda()).cpu().numpy()
    plan.close()
    return u


@pytest.mark.parametrize("p,delta,bc,rows16", [(8, 1e-3, 0, 8), (8, 1e-3, 0, 4), (8, 1e-2, 0, 16), (6, 1e-3, 0, 8),
                                               (4, 1e-3, 1, 8)])
def test_split_evaluation_stage1_on_tcgen05(monkeypatch, p, delta, bc, rows16):
    """Split precision, 3D, blocks of K <= 16: the evaluation whose first contraction runs on the
    fifth-generation tensor cores (tcgen05.mma kind::tf32 in 3xTF32, accumulators in tensor memory)
    selected with FGT_TC_EVAL6=1, against the CUDA-core kernel and against the oracle; K = 8 and 16 blocks, rows
    per CTA 4, 8 and 16, ragged K (p = 6), a periodic tree; no wait of the kernel may run out."""
    tr = W.random_balanced_tree(3, 21 + p, max_level=4, min_level=2, split_prob=0.2, periodic=bool(bc))
    sig = W.random_sigma(tr, p, 40 + p)
    tun = {"eval_rows16": rows16}
    u6 = _split_u(monkeypatch, True, tr, p, delta, sig, bc, tun)
    u2 = _split_u(monkeypatch, False, tr, p, delta, sig, bc, tun)
    assert F.device_status() == 0
    uo = oracle.box_fgt(3, p, delta, bool(bc), tr.level, tr.coord, sig)
    scale = np.abs(uo).max()
    assert np.all(np.isfinite(u6))
    assert np.abs(u6 - uo).max() <= 10 * 1e-6 * scale
    # both kernels compute the same FP32-accurate contractions: they agree far inside the bound
    assert np.abs(u6 - u2).max() <= 1e-6 * scale


def test_split_evaluation_tcgen05_full_size_workload(monkeypatch):
    """The 2.09M-point adaptive benchmark workload (K = 8 and 16 blocks on tcgen05) against the
    CUDA-core evaluation, every point, and the status word stays clear over repeated calls."""
    w = W.config_3d_free_adaptive(seed=0, p=8, delta=1e-3)
    u6 = _split_u(monkeypatch, True, w.tree, w.p, w.delta, w.sigma)
    u2 = _split_u(monkeypatch, False, w.tree, w.p, w.delta, w.sigma)
    assert F.device_status() == 0
    assert np.abs(u6 - u2).max() <= 1e-6 * np.abs(u2).max()


def test_split_evaluation_tcgen05_plan_without_operand_copy(monkeypatch):
    """A plan with tcgen05 evaluation ranges run through the allocation-free call, which has no
    operand copy of the expansions: those ranges fall back to the CUDA-core kernel, same result."""
    monkeypatch.setenv("FGT_TC_EVAL6", "1")
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    s = torch.from_numpy(W.random_sigma(tr, 4, 13)).cuda()
    plan = F.Plan(3, 4, 1e-3, 1e-6, tr.level, tr.coord, prec=F.PREC_SPLIT)
    ref = plan(s)
    out = torch.empty_like(s)
    plan.execute_noalloc(s, out)
    torch.cuda.synchronize()
    assert F.device_status() == 0
    assert (out - ref).abs().max().item() <= 1e-6 * ref.abs().max().item()
    plan.close()


def test_tensor_core_wait_time_out_is_reported():
    """The time-out path of the tcgen05 kernels' waits: a wait that nothing completes gives up after
    its limit and sets the device status word, which the host reads once and which then reads clear;
    the context stays usable (a transform right after matches the oracle)."""
    assert F.device_status() == 0
    F.selftest_tc_timeout()
    assert F.device_status() == 1
    assert F.device_status() == 0
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    check(3, 4, 1e-3, 1e-8, tr, W.random_sigma(tr, 4, 13))


def test_pipelined_host_calls_match_device_results():
    """fgt_execute_host_async: several calls in flight on one plan (copy-in, transform and copy-out
    overlapped across calls, two staging buffers in turn), each output equal to the device-buffer
    transform of its own input; host_sync waits for all of them."""
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
    plan = F.Plan(3, 4, 1e-3, 1e-6, tr.level, tr.coord, prec=F.PREC_SPLIT)
    sig = [torch.from_numpy(W.random_sigma(tr, 4, 60 + i)).pin_memory() for i in range(5)]
    outs = [torch.full_like(s, float("nan")).pin_memory() for s in sig]
    for s, o in zip(sig, outs):
        plan.execute_host_async(s, o)
    plan.host_sync()
    for s, o in zip(sig, outs):
        ref = plan(s.cuda()).cpu()
        # the same transform (atomics make the last bits depend on the order of the sums)
        assert (o - ref).abs().max().item() <= 1e-6 * ref.abs().max().item()
    plan.close()
