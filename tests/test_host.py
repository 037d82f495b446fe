"""CPU tests of the product's host side: C-ABI exports, the 1D-table building
blocks against the paper's tables and closed forms, tree validation, and the
planner's lists and tables (through a host-only plan and a numpy restatement of
each device step) against the oracle."""
import os
import re

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import spherical_jn

import oracle
import paper_2305_07165_gb300 as F
import workloads as W
from hostref import HostState

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def test_library_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "fgt.h")).read()
    names = set(re.findall(r"^\s*(?:fgt_status|void|const char \*|size_t|int32_t)\s+\**(fgt_\w+)\s*\(", hdr, re.M))
    assert len(names) >= 18, names
    L = F.lib()
    for n in sorted(names):
        assert hasattr(L, n), n
    # the bounds-checked build exports the same interface
    import ctypes
    from paper_2305_07165_gb300 import build as B
    Lc = ctypes.CDLL(B.CHECKED_LIB)
    for n in sorted(names):
        assert hasattr(Lc, n), n


def _read_table(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return rows


def test_table1_number_of_plane_waves():
    # Paper Table 1: D0 and n_f(R) for R = 2 D0, 3 D0, 4 D0
    for eps, d0, n2, n3, n4 in _read_table("table1_nf.txt"):
        D0 = F.params(1e-2, eps)["D0"]
        assert abs(D0 - d0) < 0.006
        assert [F.nf_for_range(eps, m * D0) for m in (2, 3, 4)] == [n2, n3, n4]


def test_table2_number_of_fourier_terms():
    # Paper Table 2: n_p for delta in {1e-1, 1e-2, 1e-3} and six tolerances
    eps = [1e-2, 1e-4, 1e-6, 1e-8, 1e-10, 1e-12]
    for row in _read_table("table2_np.txt"):
        delta, vals = row[0], row[1:]
        assert [F.params(delta, e, F.BC_PERIODIC)["n_p"] for e in eps] == vals


def test_cutoff_level_rule():
    # l_c: largest level with side 2^-l_c >= D0 sqrt(delta)
    for delta in (1e-6, 1e-4, 1e-3, 1e-2, 1e-1, 1.0):
        for eps in (1e-6, 1e-10):
            p = F.params(delta, eps)
            cut = p["D0"] * np.sqrt(delta)
            lc = p["cutoff_level"]
            assert 2.0 ** -lc >= cut or lc == 0
            assert 2.0 ** -(lc + 1) < cut
            assert p["R"] >= p["D0"]


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8, 1e-10, 1e-12])
@pytest.mark.parametrize("mult", [2.0, 3.0, 4.0])
def test_theorem1_error_bound_symmetric_modes(eps, mult):
    """Theorem 1: |G - PW| <= eps on |x| <= R sqrt(delta).  The transform uses the
    symmetric range m = -(M-1)..M-1 (one term fewer than the paper's [-M, M-1]); the
    proof's truncation bound covers exactly that symmetric tail."""
    D0 = np.sqrt(np.log(3 / eps))
    R = mult * D0
    h = 2 * np.pi / (R + D0)
    M = int(np.ceil(D0 * (R + D0) / np.pi))
    x = np.linspace(-R, R, 4001)          # x / sqrt(delta)
    for lo in (-M, -(M - 1)):
        m = np.arange(lo, M)
        pw = (h / (2 * np.sqrt(np.pi)) * np.exp(-(m * h) ** 2 / 4)[None, :] * np.exp(1j * np.outer(x, m) * h)).sum(1)
        assert np.abs(np.exp(-x ** 2) - pw).max() <= eps


def test_gauss_legendre_rule():
    for k in (1, 2, 3, 8, 12, 16):
        x, w = F.gauss_legendre(k)
        xr, wr = np.polynomial.legendre.leggauss(k)
        assert np.abs(x - xr).max() < 2e-16 * k and (np.abs(w - wr) / wr).max() < 1e-14
    # numpy's own weights lose ~1e-12 relative at high order; check those against 40-digit roots
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for k in (33, 64):
        x, w = F.gauss_legendre(k)
        for i in range(0, k, 7):
            z = mp.findroot(lambda t: mp.legendre(k, t), x[i])
            wt = 2 / ((1 - z ** 2) * mp.diff(lambda t: mp.legendre(k, t), z) ** 2)
            assert abs(x[i] - float(z)) < 2e-16 and abs(w[i] - float(wt)) < 1e-13 * float(wt)


@pytest.mark.parametrize("x", [0.0, 1e-9, 1e-3, 0.3, np.pi, 2 * np.pi, 10.0, 47.3, 95.0, -7.5, 300.0])
def test_spherical_bessel(x):
    assert np.abs(F.spherical_bessel(x, 20) - spherical_jn(np.arange(21), x)).max() < 1e-15


@pytest.mark.parametrize("t", [0.0, 0.5, -3.0, 12.0, 40.0])
def test_fourier_integrals_of_legendre(t):
    # I[P_n](t) = int_{-1}^{1} exp(i t x) P_n(x) dx (eq. pwintegrals), checked by quadrature
    I = F.legendre_fourier_integrals(t, 12)
    for n in range(13):
        P = np.polynomial.legendre.Legendre.basis(n)
        re = quad(lambda x: np.cos(t * x) * P(x), -1, 1, limit=400, epsabs=1e-14)[0]
        im = quad(lambda x: np.sin(t * x) * P(x), -1, 1, limit=400, epsabs=1e-14)[0]
        assert abs(I[n] - (re + 1j * im)) < 1e-12


@pytest.mark.parametrize("lam", [0.002, 0.03, 0.1, 0.125, 0.13, 0.5, 3.0])
def test_gaussian_integrals_of_legendre(lam):
    # J_lambda[P_n](t) = int_{-1}^{1} exp(-(t-x)^2/lambda^2) P_n(x) dx (eq. gsintegrals): erf seeds plus
    # the five-term recurrence (lambda <= 1/8) or quadrature, against adaptive quadrature
    for t in (-3.0, -1.5, -1.0, -0.6, 0.0, 0.37, 0.99, 1.0, 1.25, 2.0):
        J = F.legendre_gauss_integrals(lam, t, 15)
        for n in range(16):
            P = np.polynomial.legendre.Legendre.basis(n)
            pts = [t] if -1 < t < 1 else None
            ref = quad(lambda x: np.exp(-(t - x) ** 2 / lam ** 2) * P(x), -1, 1, points=pts, limit=400,
                       epsabs=1e-16, epsrel=1e-13)[0]
            assert abs(J[n] - ref) <= 1e-13 * lam * np.sqrt(np.pi), (lam, t, n)


def _tree(level, coord):
    return np.array(level, dtype=np.int32), np.array(coord, dtype=np.int32)


def test_tree_validation_errors():
    with pytest.raises(F.FGTError) as e:           # gap
        F.analyze(2, 4, 1e-3, 1e-6, *_tree([1, 1, 1], [[0, 0], [1, 0], [0, 1]]))
    assert e.value.status == 2
    with pytest.raises(F.FGTError) as e:           # overlap
        F.analyze(2, 4, 1e-3, 1e-6, *_tree([0, 1], [[0, 0], [1, 1]]))
    assert e.value.status == 2
    with pytest.raises(F.FGTError) as e:           # out of range
        F.analyze(2, 4, 1e-3, 1e-6, *_tree([0], [[1, 0]]))
    assert e.value.status == 2
    # unbalanced: level-1 leaves next to level-3 leaves
    lev, crd = [1, 1, 1], [[1, 0], [0, 1], [1, 1]]
    for c in [(0, 0), (1, 0), (0, 1)]:
        lev.append(2); crd.append(list(c))
    for c in [(2, 2), (3, 2), (2, 3), (3, 3)]:
        lev.append(3); crd.append(list(c))
    with pytest.raises(F.FGTError) as e:
        F.analyze(2, 4, 1e-3, 1e-6, *_tree(lev, crd))
    assert e.value.status == 2
    # balanced in free space but not across the periodic wrap
    tr = W.refine_tree(2, lambda l, c: l == 0 or (l == 1 and c == (0, 0)) or (l == 2 and c == (0, 0)), 3,
                       balance=True, periodic=False)
    F.analyze(2, 4, 1e-3, 1e-6, tr.level, tr.coord, bc=F.BC_FREE)
    with pytest.raises(F.FGTError):
        F.analyze(2, 4, 1e-3, 1e-6, tr.level, tr.coord, bc=F.BC_PERIODIC)
    trp = W.refine_tree(2, lambda l, c: l == 0 or (l == 1 and c == (0, 0)) or (l == 2 and c == (0, 0)), 3,
                        balance=True, periodic=True)
    F.analyze(2, 4, 1e-3, 1e-6, trp.level, trp.coord, bc=F.BC_PERIODIC)
    with pytest.raises(F.FGTError) as e:           # bad arguments
        F.analyze(2, 4, -1.0, 1e-6, *_tree([0], [[0, 0]]))
    assert e.value.status == 1
    with pytest.raises(F.FGTError):
        F.analyze(2, 4, 1e-3, 1e-8, *_tree([0], [[0, 0]]), prec=F.PREC_SPLIT)


def _planner_vs_oracle(d, tr, p, delta, tol, bc=0, mode=0, prec=0, seed=1):
    sig = W.random_sigma(tr, p, seed)
    hp = F.HostPlan(d, p, delta, tol, tr.level, tr.coord, bc=bc, mode=mode, prec=prec)
    hs = HostState(hp)
    u = hs.transform(sig)
    uo = oracle.box_fgt(d, p, delta, bool(bc), tr.level, tr.coord, sig)
    err = np.abs(u - uo).max() / np.abs(uo).max()
    assert err <= 10 * tol, (err, hs.info)
    return hs.info


@pytest.mark.parametrize("delta,tol", [(1e-1, 1e-6), (1e-2, 1e-10), (1e-3, 1e-6), (1e-3, 1e-10), (1e-4, 1e-10)])
@pytest.mark.parametrize("mode", [0, 1])
def test_planner_2d_free(delta, tol, mode):
    tr = W.random_balanced_tree(2, 4, max_level=5, min_level=1)
    _planner_vs_oracle(2, tr, 6, delta, tol, mode=mode)


@pytest.mark.parametrize("delta,tol", [(1e-1, 1e-8), (1e-2, 1e-8), (3e-3, 1e-8), (2e-4, 1e-8)])
def test_planner_2d_periodic(delta, tol):
    tr = W.random_balanced_tree(2, 7, max_level=4, min_level=1, periodic=True, split_prob=0.3)
    info = _planner_vs_oracle(2, tr, 6, delta, tol, bc=1)
    assert info["fourier"] == (info["cutoff_level"] <= 1)


@pytest.mark.parametrize("delta,tol", [(1e-1, 1e-6), (1e-2, 1e-10), (1e-3, 1e-6), (1e-3, 1e-10)])
def test_planner_3d_free(delta, tol):
    tr = W.random_balanced_tree(3, 21, max_level=3, min_level=1, split_prob=0.25)
    _planner_vs_oracle(3, tr, 3, delta, tol)


def test_planner_fp64_tensor_core_precision(monkeypatch):
    """FGT_PREC_FP64_TC plans the same FP64 tables as FGT_PREC_FP64 (only its kernels differ) and
    reports itself.  In 3D fused mode its form and evaluation are the six sliced tensor-core stages,
    which add two intermediate arrays, the digit planes of the largest stage's operand and of the 1D
    matrices to the device footprint; with FGT_OZAKI=0 (the DMMA kernels) it is the FP64 one."""
    tr = W.random_balanced_tree(3, 21, max_level=3, min_level=1, split_prob=0.25)
    info = _planner_vs_oracle(3, tr, 3, 1e-3, 1e-10, prec=F.PREC_FP64_TC)
    assert info["prec"] == F.PREC_FP64_TC
    a = F.analyze(3, 3, 1e-3, 1e-10, tr.level, tr.coord, prec=F.PREC_FP64_TC)
    b = F.analyze(3, 3, 1e-3, 1e-10, tr.level, tr.coord, prec=F.PREC_FP64)
    assert (a["n_f"], a["cutoff_level"]) == (b["n_f"], b["cutoff_level"])
    assert b["device_bytes"] < a["device_bytes"] <= 3 * b["device_bytes"]   # + intermediates, digit planes
    assert a["launches"] == 12 + 1 + (a["n_direct_pairs"] > 0)   # six stages of two launches, gather, near field
    monkeypatch.setenv("FGT_OZAKI", "0")
    c = F.analyze(3, 3, 1e-3, 1e-10, tr.level, tr.coord, prec=F.PREC_FP64_TC)
    assert abs(c["device_bytes"] - b["device_bytes"]) <= 0.01 * b["device_bytes"]
    assert c["form_flops"] == a["form_flops"] == b["form_flops"]
    with pytest.raises(F.FGTError):
        F.analyze(3, 3, 1e-3, 1e-10, tr.level, tr.coord, prec=3)


@pytest.mark.parametrize("delta", [5e-2, 5e-3, 1e-3])
def test_planner_3d_periodic(delta):
    tr = W.random_balanced_tree(3, 9, max_level=3, min_level=1, split_prob=0.3, periodic=True)
    _planner_vs_oracle(3, tr, 3, delta, 1e-8, bc=1)


def test_planner_split_precision_tables():
    tr = W.random_balanced_tree(2, 4, max_level=5, min_level=1)
    _planner_vs_oracle(2, tr, 6, 1e-3, 1e-6, prec=1)


def test_direct_only_and_root_cases():
    # l_max <= l_c: every interaction is direct; a single leaf (the root)
    tr = W.uniform_tree(2, 2)
    info = _planner_vs_oracle(2, tr, 6, 1e-4, 1e-10)
    assert info["n_form_blocks"] == 0 and info["n_direct_pairs"] > 0
    root = W.uniform_tree(3, 0)
    info = _planner_vs_oracle(3, root, 4, 1e-2, 1e-8)
    assert info["n_direct_pairs"] == 1
    info = _planner_vs_oracle(3, root, 4, 2e-2, 1e-8, bc=1)
    assert info["fourier"] == 1


def test_analyze_reports_footprint():
    w = W.config_2d_free_uniform()
    a = F.analyze(2, 8, 1e-2, 1e-9, w.tree.level, w.tree.coord)
    assert a["cutoff_level"] == 1 and a["n_f"] == 44 and a["n_leaves"] == 64
    assert a["n_pw_leaves"] == 64 and a["n_direct_pairs"] == 0 and a["device_bytes"] > 0
    h = F.analyze(2, 8, 1e-2, 1e-9, w.tree.level, w.tree.coord, mode=F.MODE_HIERARCHICAL)
    assert h["device_bytes"] > a["device_bytes"]


def test_tuning_knobs_validated_on_a_host_plan():
    import ctypes
    tr = W.random_balanced_tree(3, 21, max_level=3, min_level=1, split_prob=0.25)
    hp = F.HostPlan(3, 4, 1e-3, 1e-6, tr.level, tr.coord, prec=F.PREC_SPLIT)
    t = F.Tuning()
    assert F.lib().fgt_plan_get_tuning(hp._h, ctypes.byref(t)) == 0
    assert (t.form_group, t.eval_rows16, t.eval_rows_large, t.near_phase) == (8, 8, 4, 2) and t.ms == 0.0
    for field, bad in (("form_group", 0), ("form_group", 9), ("near_phase", 1), ("eval_rows16", 0)):
        u = F.Tuning(**{k: getattr(t, k) for k in ("form_group", "eval_rows16", "eval_rows_large", "near_phase")})
        setattr(u, field, bad)
        assert F.lib().fgt_plan_set_tuning(hp._h, ctypes.byref(u)) == 1
    u = F.Tuning(form_group=4, eval_rows16=16, eval_rows_large=8, near_phase=4)
    assert F.lib().fgt_plan_set_tuning(hp._h, ctypes.byref(u)) == 0
    assert F.lib().fgt_plan_get_tuning(hp._h, ctypes.byref(t)) == 0
    assert (t.form_group, t.eval_rows16, t.eval_rows_large, t.near_phase) == (4, 16, 8, 4)


def test_output_tree_validation():
    """fgt_plan_set_output_tree accepts non-overlapping output leaves, each inside one source leaf
    (they need not cover the source leaves, as in a refinement round that re-evaluates the
    subdivided leaves alone), and refuses the rest."""
    import ctypes
    lev, crd = np.array([1, 1, 1, 1], dtype=np.int32), np.array([[0, 0], [1, 0], [0, 1], [1, 1]], dtype=np.int32)
    hp = F.HostPlan(2, 4, 1e-2, 1e-6, lev, crd)

    def try_tree(l, c):
        t, keep = F._tree_struct(2, 4, np.array(l, dtype=np.int32), np.array(c, dtype=np.int32))
        return F.lib().fgt_plan_set_output_tree(hp._h, ctypes.byref(t))

    kids = [[2 * x + a, 2 * y + b] for (x, y) in crd.tolist() for b in (0, 1) for a in (0, 1)]
    assert try_tree([2] * 16, kids) == 0                                  # every leaf refined once
    assert try_tree([1, 1, 1] + [2] * 4, crd.tolist()[:3] + kids[12:]) == 0  # one leaf refined
    assert try_tree([0], [[0, 0]]) == 2                                   # coarser than the source
    assert try_tree([1, 1, 1], crd.tolist()[:3]) == 0                     # a source leaf left out: allowed
    assert try_tree([2] * 4, kids[4:8]) == 0                              # only one leaf's children
    assert try_tree([2] * 3, kids[4:7]) == 0                              # a source leaf partly covered
    assert try_tree([1, 1, 1, 1, 2], crd.tolist() + [[0, 0]]) == 2         # overlapping leaves
    assert try_tree([1, 1, 1, 1, 1], crd.tolist() + [[0, 0]]) == 2         # repeated leaf
    assert F.lib().fgt_plan_set_output_tree(hp._h, None) == 0


def test_point_plan_argument_checks():
    """fgt_point_plan_create rejects bad precisions and split below tol 1e-7 before touching the device."""
    import ctypes
    L = F.lib()
    pts = np.zeros((4, 3))
    h = ctypes.c_void_p()

    def create(tol, prec, d=3):
        return L.fgt_point_plan_create(d, 1e-3, tol, 4, pts.ctypes.data, 4, pts.ctypes.data, 8, prec,
                                       ctypes.byref(h))
    assert create(1e-6, 7) == 1
    assert create(1e-8, F.PREC_SPLIT) == 1
    assert create(1e-6, F.PREC_FP64_TC) == 1
    assert create(1e-6, F.PREC_FP64, d=4) == 1
    assert h.value is None


def test_batch_rejects_a_plan_listed_twice():
    """A batch runs its transforms as concurrent branches, each writing its own plan's workspace:
    the same plan twice would race with itself, so the batch is refused (before any device work)."""
    tr = W.random_balanced_tree(2, 3, max_level=3, min_level=1)
    hp = F.HostPlan(2, 4, 1e-2, 1e-6, tr.level, tr.coord)
    with pytest.raises(F.FGTError, match="listed twice"):
        F.Batch([hp, hp])
    with pytest.raises(F.FGTError, match="not a device plan"):
        F.Batch([hp])
    hp.close()
