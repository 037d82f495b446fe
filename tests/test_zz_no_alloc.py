"""The allocation-free entry point, fgt_execute_noalloc, through the C ABI.

Some callers cannot allocate device memory when they run a transform (their
allocator owns the device memory, or a cudaMalloc would synchronise the device
in the middle of their work).  fgt_execute_noalloc keeps the plane-wave
expansions in the library's fixed device array instead.  Its result must match
the ordinary entry point's on consecutive calls (the array keeps the previous
call's contents, so the second call checks that it is cleared), and a plan
whose workspace is too large must be refused with a clear error.

Collected last on purpose: a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["2d", "3d", "3d_split", "3d_split_large_blocks"])
def test_noalloc_matches_execute_twice(case):
    if case == "2d":
        w = W.config_2d_free_uniform(seed=0)
        d, p, delta, tol, tree, sig, prec = 2, w.p, w.delta, 1e-9, w.tree, w.sigma, F.PREC_FP64
    elif case == "3d_split_large_blocks":
        # K = 32 blocks: the allocation-free call reads sigma directly, the plan's own call
        # through its packed FP32 copy, so the two paths check each other
        tree = W.uniform_tree(3, 3)
        d, p, delta, tol, prec = 3, 8, 1e-2, 1e-6, F.PREC_SPLIT
        sig = W.random_sigma(tree, p, 17)
    else:
        tree = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
        d, p = 3, 4
        sig = W.random_sigma(tree, p, 13)
        # both fit the 64 MiB array: 64 FP64 anchors (about 60 MiB); 270 FP32 anchors plus near field
        delta, tol, prec = (3e-3, 1e-8, F.PREC_FP64) if case == "3d" else (1e-3, 1e-6, F.PREC_SPLIT)
    plan = F.Plan(d, p, delta, tol, tree.level, tree.coord, prec=prec)
    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    ref = plan(s)
    scale = ref.abs().max().item()
    for call in range(2):
        out = torch.full_like(s, float("nan"))
        plan.execute_noalloc(s, out)
        torch.cuda.synchronize()
        err = (out - ref).abs().max().item()
        assert err <= 10 * tol * scale, (call, err, scale)
    # a different input through the same array: the previous contents must not leak in
    s2 = torch.from_numpy(W.random_sigma(tree, p, 99)).cuda()
    out2 = torch.empty_like(s2)
    plan.execute_noalloc(s2, out2)
    ref2 = plan(s2)
    torch.cuda.synchronize()
    assert (out2 - ref2).abs().max().item() <= 10 * tol * ref2.abs().max().item()
    plan.close()


def test_noalloc_rejects_workspace_larger_than_the_array():
    # 3D, delta = 1e-3, tol 1e-10: 64 boxes at the cutoff level (2), each holding
    # 65 x 65 x 33 FP64 complex modes twice (outgoing and incoming): about 285 MB
    tree = W.uniform_tree(3, 3)
    plan = F.Plan(3, 4, 1e-3, 1e-10, tree.level, tree.coord)
    info = plan.info()
    assert info["device_bytes"] > 64 << 20
    s = torch.zeros(tree.n_leaves, 64, dtype=torch.float64, device="cuda")
    out = torch.empty_like(s)
    with pytest.raises(F.FGTError) as e:
        plan.execute_noalloc(s, out)
    assert e.value.status == 1 and "exceeds" in str(e.value)
    plan.close()
