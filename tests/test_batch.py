"""Batched execution (one CUDA graph launch, one branch per transform) against
each transform run alone, for a mix of d, k, delta, tol, boundary conditions and
precisions; graph reuse on the same buffers and recapture on new ones."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
F = pytest.importorskip("paper_2305_07165_gb300")

pytestmark = pytest.mark.gpu


def _mix(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        d = int(rng.choice([2, 3]))
        k = int(rng.choice([4, 6, 8])) if d == 2 else int(rng.choice([3, 4, 6]))
        per = bool(rng.integers(2))
        tol = float(rng.choice([1e-6, 1e-10]))
        prec = F.PREC_SPLIT if (tol >= 1e-7 and rng.integers(2)) else F.PREC_FP64
        delta = float(10 ** rng.uniform(-4, -1))
        tr = W.random_balanced_tree(d, int(rng.integers(1 << 30)), max_level=5 if d == 2 else 3, min_level=1,
                                    split_prob=0.4, periodic=per)
        plan = F.Plan(d, k, delta, tol, tr.level, tr.coord, bc=int(per), prec=prec)
        sig = torch.from_numpy(W.random_sigma(tr, k, int(rng.integers(1 << 30)))).cuda()
        out.append((plan, sig, tol))
    return out


def test_batch_matches_single_transforms():
    mix = _mix(14)
    plans = [m[0] for m in mix]
    sig = [m[1] for m in mix]
    ref = [p(s).clone() for p, s in zip(plans, sig)]
    outs = [torch.full_like(s, float("nan")) for s in sig]
    b = F.Batch(plans)
    b(sig, outs)
    b(sig, outs)                      # graph reused
    torch.cuda.synchronize()
    for (p, s, tol), r, o in zip(mix, ref, outs):
        assert (o - r).abs().max().item() <= 1e-12 * r.abs().max().item()
    outs2 = [torch.empty_like(s) for s in sig]  # new pointers: recaptured
    b(sig, outs2)
    torch.cuda.synchronize()
    for r, o in zip(ref, outs2):
        assert (o - r).abs().max().item() <= 1e-12 * r.abs().max().item()
    b.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_persistent_batch_matches_single_transforms(seed):
    """The batch as ONE persistent kernel over a device queue of every transform's (phase, block)
    items: each result equals its transform run alone (FP64 to rounding; split precision to the
    FP32 level, the queue using the CUDA-core kernels where a plan alone takes the tcgen05 ones),
    repeatedly and after new buffers, and no dependency wait ran out."""
    mix = _mix(16, seed=seed)
    plans = [m[0] for m in mix]
    sig = [m[1] for m in mix]
    ref = [p(s).clone() for p, s in zip(plans, sig)]
    b = F.Batch(plans, mode=F.BATCH_PERSISTENT)
    info = b.info()
    assert info["mode"] == F.BATCH_PERSISTENT and info["items"] > len(plans) and info["grid"] >= 1
    for outs in ([torch.full_like(s, float("nan")) for s in sig], [torch.empty_like(s) for s in sig]):
        for _ in range(2):
            b(sig, outs)
        torch.cuda.synchronize()
        assert b.status() == 0
        for (p, s, tol), r, o in zip(mix, ref, outs):
            bound = (1e-12 if p.info()["prec"] == F.PREC_FP64 else 2e-6) * r.abs().max().item()
            assert (o - r).abs().max().item() <= bound
    b.close()
    for p in plans:
        p.close()


def test_persistent_batch_wait_time_out_is_reported():
    """A dependency wait of the persistent kernel that runs out (a counter nothing increments, a
    limit of about a millisecond) reports FGT_ERR_TIMEOUT instead of hanging."""
    assert F.selftest_batch_timeout() == F.ERR_TIMEOUT


def test_persistent_batch_refuses_hierarchical_plans():
    tr = W.random_balanced_tree(2, 3, max_level=3, min_level=1)
    p = F.Plan(2, 4, 1e-2, 1e-6, tr.level, tr.coord, mode=F.MODE_HIERARCHICAL)
    with pytest.raises(F.FGTError, match="hierarchical"):
        F.Batch([p], mode=F.BATCH_PERSISTENT)
    p.close()
