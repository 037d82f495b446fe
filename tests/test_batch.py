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
