"""The bounds-checked build (libfgt_checked.so) on the parity cases: every instrumented global access
of the kernels must fall inside the buffers registered for its call, so the check counter stays at
zero, and the results still match the oracle.

The checked library is loaded in a child process (FGT_LIB=checked is read when the binding first
loads its library)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, os.environ["FGT_ROOT"])
import numpy as np, torch
import oracle, workloads as W, paper_2305_07165_gb300 as F
out = {"cases": []}
assert F.check_status()["checked"] == 1

def run(name, d, p, delta, tol, tree, sig, bc=0, prec=0, mode=0, noalloc=False):
    plan = F.Plan(d, p, delta, tol, tree.level, tree.coord, bc=bc, prec=prec, mode=mode)
    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    if noalloc:
        plan.info()
        u = torch.empty_like(s)
        plan.execute_noalloc(s, u)
    else:
        u = plan(s)
    torch.cuda.synchronize()
    st = F.check_status()
    uo = oracle.box_fgt(d, p, delta, bool(bc), tree.level, tree.coord, sig)
    err = float(np.abs(u.cpu().numpy() - uo).max() / np.abs(uo).max())
    out["cases"].append(dict(name=name, err=err, bound=10 * tol, **st))
    plan.close()

tr3 = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.2)
tr2 = W.random_balanced_tree(2, 5, max_level=6, min_level=2, split_prob=0.3)
trp = W.random_balanced_tree(3, 9, max_level=4, min_level=2, split_prob=0.25, periodic=True)
run("3d free fp64", 3, 4, 1e-3, 1e-8, tr3, W.random_sigma(tr3, 4, 1))
run("3d free split", 3, 8, 1e-3, 1e-6, tr3, W.random_sigma(tr3, 8, 2), prec=1)
run("3d free fp64-tc", 3, 4, 1e-3, 1e-8, tr3, W.random_sigma(tr3, 4, 3), prec=2)
run("3d free hierarchical", 3, 4, 1e-3, 1e-8, tr3, W.random_sigma(tr3, 4, 4), mode=1)
run("3d periodic split", 3, 4, 1e-3, 1e-6, trp, W.random_sigma(trp, 4, 5), bc=1, prec=1)
run("2d free fp64", 2, 8, 1e-3, 1e-10, tr2, W.random_sigma(tr2, 8, 6))
run("2d free split", 2, 8, 1e-3, 1e-6, tr2, W.random_sigma(tr2, 8, 7), prec=1)
run("3d allocation-free", 3, 4, 3e-3, 1e-8, tr3, W.random_sigma(tr3, 4, 8), noalloc=True)
tr32 = W.uniform_tree(3, 3)
run("3d K=32 blocks split", 3, 8, 1e-2, 1e-6, tr32, W.random_sigma(tr32, 8, 9), prec=1)
# the discrete transform
rng = np.random.default_rng(3)
pts = rng.uniform(-0.5, 0.5, size=(20000, 3))
q = rng.uniform(0.5, 1.5, len(pts))
for prec in (0, 1):
    pp = F.PointPlan(3, 1e-3, 1e-6, pts, pts, n_s=32, prec=prec)
    u = pp(torch.from_numpy(q).cuda()).cpu().numpy()
    st = F.check_status()
    uo = oracle.point_fgt(3, 1e-3, pts, q, pts)
    out["cases"].append(dict(name=f"point 3d prec {prec}", err=float(np.abs(u - uo).max() / np.abs(uo).max()),
                             bound=1e-5, **st))
    pp.close()
print("RESULT " + json.dumps(out))
"""


def test_checked_build_parity_without_out_of_range_access():
    env = dict(os.environ, FGT_LIB="checked", FGT_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("RESULT ")][-1]
    cases = json.loads(line[len("RESULT "):])["cases"]
    assert len(cases) == 11
    for c in cases:
        assert c["checked"] == 1, c
        assert c["count"] == 0 and c["site"] == 0, c   # no access outside its buffers
        assert c["err"] <= c["bound"], c
