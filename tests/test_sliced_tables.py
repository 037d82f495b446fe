"""The planner's side of the sliced FP64 tensor-core stages (precision FP64_TC, 3D), on the CPU: the
digit planes of every stage's 1D matrix, read back from a host-only plan, reconstruct the real form
of the block's complex 1D matrix (rebuilt here from the plan's FP64 tables) to the 47-bit rounding
the slicing promises, every digit is a balanced 8-bit one, padding is zero, and the jobs cover
every (row, column) of every stage of every block exactly once.  The form's last stage runs over
groups of an anchor's blocks (their contractions concatenated), which must take every block once."""
import numpy as np
import pytest

import workloads as W

F = pytest.importorskip("paper_2305_07165_gb300")

BLOCK = np.dtype([("slot", "<i4"), ("K", "<i4"), ("dl", "<i4"), ("flags", "<i4"), ("mat", "<i4", 3),
                  ("pad", "<i4"), ("leaf0", "<i8")])
JOB = np.dtype([("blk", "<i4"), ("tile", "<i2"), ("part", "<i2"), ("scr", "<i8"), ("boff", "<i8"),
                ("aoff", "<i8"), ("eoff", "<i4"), ("roff", "<i4"), ("flags", "<i4"), ("nks", "<i2"), ("np", "<i2")])
GROUP = np.dtype([("slot", "<i4"), ("n", "<i4"), ("K", "<i4", 10), ("q0", "<i4", 11), ("blk", "<i4", 10),
                  ("pad", "<i4"), ("scr", "<i8", 10)])
S = 6


def dims(kind, K, n1, nh):
    R, Q, N = {0: (K * K, K, 2 * nh), 1: (nh * K, 2 * K, 2 * n1), 2: (nh * n1, 2 * K, 2 * n1),
               3: (nh * n1, 2 * n1, 2 * K), 4: (K * nh, 2 * n1, 2 * K), 5: (K * K, 2 * nh, K)}[kind]
    P = -(-N // 32)
    Nc = -(-N // P)
    return R, Q, N, P, Nc, -(-Nc // 16) * 16, -(-Q // 16)


def real_form(kind, blk, k, n1, nh, tab):
    """The stage's 1D matrix as a real Q x N matrix: complex entries a + ib act on (re, im) pairs
    as [[a, b], [-b, a]] (column c' of the output, row c of the input)."""
    K = int(blk["K"])
    axis = {0: 2, 1: 1, 2: 0, 3: 0, 4: 1, 5: 2}[kind]
    mat = int(blk["mat"][axis])
    R, Q, N, *_ = dims(kind, K, n1, nh)
    B = np.zeros((Q, N))
    if kind <= 2:
        n = nh if kind == 0 else n1
        T = tab["Fh"] if kind == 0 else tab["Ff"]
        M = np.array([[T[((mat + J // k) * n + m) * k + J % k] for J in range(K)] for m in range(n)])  # [m][J]
        if kind == 0:
            B[:, 0::2], B[:, 1::2] = M.real.T, M.imag.T
        else:
            B[:K, 0::2], B[K:, 0::2], B[:K, 1::2], B[K:, 1::2] = M.real.T, -M.imag.T, M.imag.T, M.real.T
    else:
        n = nh if kind == 5 else n1
        T = tab["Eh"] if kind == 5 else tab["Ef"]
        M = np.array([[T[((mat + I // k) * k + I % k) * n + m] for m in range(n)] for I in range(K)])  # [I][m]
        if kind == 3:
            B[0::2, :K], B[1::2, :K], B[0::2, K:], B[1::2, K:] = M.real.T, -M.imag.T, M.imag.T, M.real.T
        elif kind == 4:
            B[:n1, :K], B[n1:, :K], B[:n1, K:], B[n1:, K:] = M.real.T, -M.imag.T, M.imag.T, M.real.T
        else:
            B[:nh], B[nh:] = M.real.T, -M.imag.T
    return B


def group_form(g, blocks, k, n1, nh, tab):
    """Stage 2 over a group: the members' real-form matrices stacked along the contraction."""
    Q = int(g["q0"][g["n"]])
    B = np.zeros((Q, 2 * n1))
    for m in range(int(g["n"])):
        b = blocks[g["blk"][m]]
        assert int(b["K"]) == int(g["K"][m]) and int(b["slot"]) == int(g["slot"])
        q0 = int(g["q0"][m])
        B[q0:q0 + 2 * int(b["K"])] = real_form(2, b, k, n1, nh, tab)
    return B


def bf16_to_float(h):
    return (h.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("name,k,delta,tol,bc", [("random", 4, 1e-3, 1e-10, 0), ("uniformp", 3, 1e-3, 1e-10, 1),
                                                 ("random", 6, 1e-2, 1e-6, 0)])
def test_sliced_digit_tables(name, k, delta, tol, bc):
    tr = (W.uniform_tree(3, 3, periodic=True) if name == "uniformp"
          else W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.25))
    hp = F.HostPlan(3, k, delta, tol, tr.level, tr.coord, bc=bc, prec=F.PREC_FP64_TC)
    info = hp.info()
    n1, nh = info["modes_1d"], info["modes_half"]
    assert info["n_sliced_jobs"] > 0
    tab = {nm: hp.array(nm, np.complex128) for nm in ("Ff", "Fh", "Ef", "Eh")}
    btab = hp.array("oz_btab", np.uint16)
    bexp = hp.array("oz_bexp", np.int32)
    blocks = {0: hp.array("blocks", BLOCK), 1: hp.array("eval_blocks", BLOCK)}
    total = 0
    groups = hp.array("oz_groups", GROUP)
    # the groups of stage 2 take every form block once, members of one slot, contraction <= 160
    members = sorted(int(b) for g in groups for b in g["blk"][: g["n"]])
    assert members == list(range(len(blocks[0])))
    for g in groups:
        assert 1 <= g["n"] <= 10 and g["q0"][0] == 0 and g["q0"][g["n"]] <= 160
        assert all(g["q0"][m + 1] - g["q0"][m] == 2 * g["K"][m] for m in range(g["n"]))
    for kind in range(6):
        jobs = hp.array(f"oz_jobs{kind}", JOB)
        blks = groups if kind == 2 else blocks[0 if kind < 3 else 1]
        covered, checked = {}, set()
        for j in jobs:
            b = blks[j["blk"]]
            if kind == 2:
                R, Q, N, P, Nc, Np, nks = dims(2, 8, n1, nh)
                Q = int(b["q0"][b["n"]])
                nks = -(-Q // 16)
            else:
                K = int(b["K"])
                R, Q, N, P, Nc, Np, nks = dims(kind, K, n1, nh)
            assert 0 <= j["tile"] < -(-R // 128) and 0 <= j["part"] < P
            assert (int(j["nks"]), int(j["np"])) == (nks, Np)   # the warps' copies of the step counts
            covered.setdefault(int(j["blk"]), set()).add((int(j["tile"]), int(j["part"])))
            if (int(j["boff"]), int(j["eoff"])) in checked:   # tiles of a block share its table
                continue
            checked.add((int(j["boff"]), int(j["eoff"])))
            B = group_form(b, blocks[0], k, n1, nh, tab) if kind == 2 else real_form(kind, b, k, n1, nh, tab)
            Bp = np.zeros((nks * 16, Np))                     # this part's columns, padded
            c = int(j["part"]) * Nc + np.arange(Np)
            ok = (np.arange(Np) < Nc) & (c < N)
            Bp[:Q, ok] = B[:, c[ok]]
            f = bexp[j["eoff"]: j["eoff"] + Np].astype(np.int64)
            q = np.arange(nks * 16)[:, None]
            nl = np.arange(Np)[None, :]
            ks, kk = q // 16, q % 16
            off = (ks * S * Np * 16 + (nl >> 3) * 128 + (kk >> 3) * 64 + (nl & 7) * 8 + (kk & 7))   # plane 0
            base = int(j["boff"]) // 2
            d = np.stack([bf16_to_float(btab[base + off + s * Np * 16]) for s in range(S)])
            assert np.all(d == np.round(d)) and np.all(np.abs(d) <= 128)
            val = np.ldexp(np.tensordot(2.0 ** (-7 - 8 * np.arange(S)), d, axes=1), f[None, :])
            assert np.all(np.abs(val - Bp) <= np.ldexp(1.0, f - 48)[None, :]), kind
        sj = hp.array(f"oz_slice_jobs{kind}", JOB)
        # the first evaluation stage slices each anchor's expansion once (the operand is the slot);
        # every other stage slices each block's own operand
        owner = (lambda b: int(blks[b]["slot"])) if kind == 3 else (lambda b: int(b))
        assert ({(owner(j["blk"]), int(j["tile"])) for j in sj} ==
                {(owner(b), t) for b, ts in covered.items() for t, _ in ts})
        assert len(sj) == len({(owner(j["blk"]), int(j["tile"])) for j in sj})
        def steps(bi):
            if kind == 2:
                return -(-int(blks[bi]["q0"][blks[bi]["n"]]) // 16)
            return dims(kind, int(blks[bi]["K"]), n1, nh)[6]
        ends = sorted((int(j["aoff"]), int(j["aoff"]) + steps(j["blk"]) * S * 4096) for j in sj)
        assert all(a1 <= b0 for (_, a1), (b0, _) in zip(ends, ends[1:]))      # digit planes do not overlap
        where = {(owner(x["blk"]), int(x["tile"])): (int(x["aoff"]), int(x["roff"])) for x in sj}
        for j in jobs:   # the products read their tile's planes and exponents
            assert (int(j["aoff"]), int(j["roff"])) == where[(owner(j["blk"]), int(j["tile"]))]
        for bi in range(len(blks)):
            R, Q, N, P, *_ = dims(kind, 8 if kind == 2 else int(blks[bi]["K"]), n1, nh)
            assert covered.get(bi) == {(t, p) for t in range(-(-R // 128)) for p in range(P)}
        total += len(jobs)
    assert total == info["n_sliced_jobs"]
    hp.close()


def slice_rows(A, e):
    """Six balanced base-256 digits of each entry of A against its row exponent e (the largest
    entry of row r lies in [2^(e_r - 1), 2^e_r)): A ~ 2^e_r sum_s d_s 2^(-7 - 8 s), |d_s| <= 128."""
    N = np.rint(np.ldexp(A, (47 - e)[:, None])).astype(np.int64)   # |N| <= 2^47
    d = []
    for _ in range(S - 1):
        lo = ((N + 128) % 256) - 128
        d.append(lo)
        N = (N - lo) // 256
    d.append(N)
    return np.stack(d[::-1])                                           # d[0] the leading digit


@pytest.mark.parametrize("kind", [1, 4])
def test_sliced_products_meet_their_bound(kind):
    """The scheme end to end on one job's real table: a seeded operand A (rows spanning 2^-20 .. 2^20,
    a zero row, ragged magnitudes) sliced by rows, the 21 digit-pair products with s + t <= 5 summed
    per diagonal D = s + t (each partial sum below 2^24: exact in FP32), recombined as
    V = sum_D P_D 2^(8 (5 - D)) (|V| < 2^62) and scaled by 2^(e_r + f_n - 54).  The result meets the
    bound of the two 47-bit roundings and the dropped pairs, a few units of 2^(e_r + f_n - 47) per
    term of the contraction, and lies far inside tol 1e-10."""
    tr = W.random_balanced_tree(3, 21, max_level=4, min_level=2, split_prob=0.25)
    k = 4
    hp = F.HostPlan(3, k, 1e-3, 1e-10, tr.level, tr.coord, bc=0, prec=F.PREC_FP64_TC)
    info = hp.info()
    n1, nh = info["modes_1d"], info["modes_half"]
    tab = {nm: hp.array(nm, np.complex128) for nm in ("Ff", "Fh", "Ef", "Eh")}
    btab = hp.array("oz_btab", np.uint16)
    bexp = hp.array("oz_bexp", np.int32)
    blocks = hp.array("blocks" if kind < 3 else "eval_blocks", BLOCK)
    jobs = hp.array(f"oz_jobs{kind}", JOB)
    j = jobs[int(np.argmax([int(blocks[x["blk"]]["K"]) for x in jobs]))]   # a job of the largest block
    b = blocks[j["blk"]]
    R, Q, N, P, Nc, Np, nks = dims(kind, int(b["K"]), n1, nh)
    # B's digits and column exponents as the products read them
    f = bexp[j["eoff"]: j["eoff"] + Np].astype(np.int64)
    q = np.arange(nks * 16)[:, None]
    nl = np.arange(Np)[None, :]
    off = ((q // 16) * S * Np * 16 + (nl >> 3) * 128 + ((q % 16) >> 3) * 64 + (nl & 7) * 8 + (q % 16 & 7))
    bd = np.stack([bf16_to_float(btab[int(j["boff"]) // 2 + off + s * Np * 16]) for s in range(S)]).astype(np.int64)
    Bt = real_form(kind, b, k, n1, nh, tab)
    c = int(j["part"]) * Nc + np.arange(Np)
    live = (np.arange(Np) < Nc) & (c < N)
    Bp = np.zeros((nks * 16, Np))
    Bp[:Q, live] = Bt[:, c[live]]
    # a seeded operand tile: 128 rows, the contraction padded to whole 16-deep steps with zeros
    rng = np.random.default_rng(11)
    A = np.zeros((128, nks * 16))
    A[:, :Q] = rng.standard_normal((128, Q)) * np.ldexp(1.0, rng.integers(-20, 21, 128))[:, None]
    A[5] = 0.0
    A[7, :Q] *= np.ldexp(1.0, -rng.integers(0, 40, Q))                      # ragged within a row
    amax = np.abs(A).max(axis=1)
    e = np.where(amax > 0, np.frexp(np.where(amax > 0, amax, 1.0))[1], 0).astype(np.int64)
    ad = slice_rows(A, e)
    assert np.abs(ad).max() <= 128 and np.abs(bd).max() <= 128
    Pd = np.zeros((S, 128, Np), dtype=np.int64)
    for s in range(S):
        for t in range(S - s):
            Pd[s + t] += ad[s] @ bd[t]
    assert np.abs(Pd).max() < 2 ** 24                                        # exact FP32 accumulation
    V = sum(Pd[D] << (8 * (S - 1 - D)) for D in range(S))
    assert np.abs(V).max() < 2 ** 62
    C = np.ldexp(V.astype(np.float64), e[:, None] + f[None, :] - 54)
    ref = A @ Bp
    err = np.abs(C - ref)[:, live]
    scale = np.ldexp(1.0, e[:, None] + f[None, :])[:, live]
    assert np.all(err <= 8 * Q * scale * 2.0 ** -47), (err / scale).max()
    assert np.all(C[5] == 0)
    assert (err / np.maximum(np.abs(A) @ np.abs(Bp), 1e-300)[:, live]).max() < 1e-12
    hp.close()
