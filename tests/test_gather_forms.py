"""The three forms of the out->in gather at the cutoff level (eq. diagonaltranslation), from a
host-only plan's arrays, on random outgoing expansions: the per-anchor source lists with their
offset codes (the definition: psi_T = sum over source boxes S = T + o of the separable phase
P_1(o_1) P_2(o_2) P_3(o_3) times phi_S), the runs along x_1 with their 9 neighbouring lines, and
the stencil form over a full cutoff grid (3D, 4 or 8 boxes a side; FP64 plans), restated here as
the kernels compute them, must agree."""
import numpy as np
import pytest

import workloads as W

F = pytest.importorskip("paper_2305_07165_gb300")

SRC = np.dtype([("slot", "<i4"), ("code", "<i4")])
SEGW = 8
SEG = np.dtype([("tgt", "<i4", SEGW), ("src", "<i4", (9, SEGW + 2))])


def modes(n1, nh):
    m3, m2, m1 = np.meshgrid(np.arange(nh), np.arange(n1), np.arange(n1), indexing="ij")
    return m1.ravel(), m2.ravel(), m3.ravel()


@pytest.mark.parametrize("bc,level,delta,lc", [(1, 4, 2e-3, 2), (0, 4, 2e-3, 2), (1, 4, 1e-3, 3), (0, 4, 1e-3, 3),
                                               (0, -5, 1e-4, 4), (1, -5, 1e-4, 4)])
def test_gather_forms_agree(bc, level, delta, lc):
    """level > 0: a uniform tree (every cutoff box an anchor); level < 0: a random tree to depth
    -level, whose cutoff grid has empty boxes (an FP64_TC plan: the grid form with zeros there)."""
    if level > 0:
        tr = W.uniform_tree(3, level, periodic=bool(bc))
        prec = F.PREC_FP64
    else:
        tr = W.random_balanced_tree(3, 32, max_level=-level, min_level=3, split_prob=0.15, periodic=bool(bc))
        prec = F.PREC_FP64_TC
    hp = F.HostPlan(3, 2, delta, 1e-6, tr.level, tr.coord, bc=bc, prec=prec)
    info = hp.info()
    n1, nh = info["modes_1d"], info["modes_half"]
    assert info["cutoff_level"] == lc
    nb = 1 << lc
    Pf = hp.array("Pf", np.complex128).reshape(3, n1)
    Ph = hp.array("Ph", np.complex128).reshape(3, nh)
    dst = hp.array("gather_dst", np.int32)
    ptr = hp.array("gather_ptr", np.int64)
    src = hp.array("gather_src", SRC)
    nslot = int(dst.max()) + 1
    m1, m2, m3 = modes(n1, nh)
    rng = np.random.default_rng(4)
    phi = rng.standard_normal((nslot, m1.size)) + 1j * rng.standard_normal((nslot, m1.size))
    # the definition: per-anchor source lists
    ref = np.zeros_like(phi)
    for t, T in enumerate(dst):
        for s in src[ptr[t]:ptr[t + 1]]:
            c = int(s["code"])
            o1, o2, o3 = c % 3, (c // 3) % 3, c // 9
            ref[T] += Pf[o1, m1] * Pf[o2, m2] * Ph[o3, m3] * phi[s["slot"]]
    # the runs along x_1 (gather2): lines l = (o2 + 1) + 3 (o3 + 1), positions x0 - 1 + i
    segs = hp.array("gather_segs", SEG)
    sw = min(SEGW, nb)
    run = np.full_like(phi, np.nan)
    for g in segs:
        w = np.zeros((sw + 2, m1.size), complex)
        for l in range(9):
            f = Pf[l % 3, m2] * Ph[l // 3, m3]
            for i in range(sw + 2):
                if g["src"][l][i] >= 0:
                    w[i] += f * phi[g["src"][l][i]]
        for t in range(sw):
            if g["tgt"][t] >= 0:
                run[g["tgt"][t]] = Pf[0, m1] * w[t] + Pf[1, m1] * w[t + 1] + Pf[2, m1] * w[t + 2]
    assert np.allclose(run, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    # the stencil form over the full grid: axis by axis, neighbours wrapped (periodic) or absent
    grid = hp.array("gather_grid", np.int32)
    assert grid.size == nb ** 3 and sorted(v for v in grid.tolist() if v >= 0) == list(range(nslot))
    buf = np.where((grid >= 0)[:, None], phi[np.maximum(grid, 0)], 0)   # [box][mode], zero where empty
    for ax, P, m in ((0, Pf, m1), (1, Pf, m2), (2, Ph, m3)):
        stride = nb ** ax
        out = np.zeros_like(buf)
        for b in range(nb ** 3):
            x = (b // stride) % nb
            for o in (-1, 0, 1):
                xs = x + o
                if not 0 <= xs < nb:
                    if not bc:
                        continue
                    xs %= nb
                out[b] += P[o + 1, m] * buf[b + (xs - x) * stride]
        buf = out
    sten = np.empty_like(phi)
    sten[grid[grid >= 0]] = buf[grid >= 0]
    assert np.allclose(sten, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    hp.close()
