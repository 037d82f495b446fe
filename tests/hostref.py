"""Host FP64 restatement of each device step, driven by a host-only plan's own
lists and tables (numpy einsum instead of the CUDA kernels).

It checks the planner (parameters, f flags, P- and D-lists, 1D tables, phase
vectors) against the oracle without a GPU, and gives the per-kernel GPU tests
a reference for each step.  Test infrastructure only.
"""
import numpy as np

BLOCK = np.dtype([("slot", "<i4"), ("K", "<i4"), ("dl", "<i4"), ("flags", "<i4"), ("mat", "<i4", (3,)),
                  ("pad", "<i4"), ("leaf0", "<i8")])
GSRC = np.dtype([("slot", "<i4"), ("code", "<i4")])
NSRC = np.dtype([("leaf", "<i8"), ("tab", "<i4", (3,)), ("pad", "<i4")])
SHIFT = np.dtype([("parent", "<i4"), ("child", "<i4", (8,))])


class HostState:
    def __init__(self, hp):
        self.info = info = hp.info()
        self.d, self.k = info["d"], info["k"]
        self.n1, self.nh = info["modes_1d"], info["modes_half"]
        self.fourier = info["fourier"]
        cdt = np.complex64 if info["prec"] == 1 else np.complex128  # FP32 expansions only in split precision
        k, n1, nh = self.k, self.n1, self.nh
        self.blocks = hp.array("blocks", BLOCK)
        self.bleaves = hp.array("block_leaves", np.int64)
        self.Ff = hp.array("Ff", cdt).reshape(-1, n1, k)
        self.Fh = hp.array("Fh", cdt).reshape(-1, nh, k)
        self.Ef = hp.array("Ef", cdt).reshape(-1, k, n1)
        self.Eh = hp.array("Eh", cdt).reshape(-1, k, nh)
        self.gdst = hp.array("gather_dst", np.int32)
        self.gptr = hp.array("gather_ptr", np.int64)
        self.gsrc = hp.array("gather_src", GSRC)
        self.Pf = hp.array("Pf", cdt).reshape(3, n1)
        self.Ph = hp.array("Ph", cdt).reshape(3, nh)
        self.ntgt = hp.array("near_tgt", np.int64)
        self.nflags = hp.array("near_flags", np.int32)
        self.nptr = hp.array("near_ptr", np.int64)
        self.nsrc = hp.array("near_src", NSRC)
        self.ntab = hp.array("near_tab", np.float64).reshape(-1, k, k)
        self.merge, self.push = [], []
        for name, dst in (("merge", self.merge), ("push", self.push)):
            i = 0
            while True:
                try:
                    items = hp.array(f"{name}{i}_items", SHIFT)
                except Exception:
                    break
                dst.append((items, hp.array(f"{name}{i}_qf", cdt).reshape(2, n1),
                            hp.array(f"{name}{i}_qh", cdt).reshape(2, nh)))
                i += 1
        self.slot_shape = (nh, n1, n1) if self.d == 3 else (nh, n1)
        nslot = 0
        if len(self.blocks):
            nslot = int(self.blocks["slot"].max()) + 1
        for items, _, _ in self.merge + self.push:
            if len(items):
                nslot = max(nslot, int(items["parent"].max()) + 1, int(items["child"].max()) + 1)
        self.n_slots = nslot

    # block matrices: concatenate the per-offset matrices along the node axis
    def _fmat(self, blk, a, half):
        nl = 1 << int(blk["dl"])
        src = self.Fh if half else self.Ff
        return np.concatenate([src[blk["mat"][a] + o] for o in range(nl)], axis=1)  # [modes, K]

    def _emat(self, blk, a, half):
        nl = 1 << int(blk["dl"])
        src = self.Eh if half else self.Ef
        return np.concatenate([src[blk["mat"][a] + o] for o in range(nl)], axis=0)  # [K, modes]

    def _block_leaves(self, blk):
        nl = 1 << int(blk["dl"])
        n = nl ** self.d
        return self.bleaves[blk["leaf0"]: blk["leaf0"] + n].reshape((nl,) * self.d)  # axes (o_d, .., o_1)

    def _dense(self, blk, sigma):
        """sigma of a block as a dense [K]*d array, axes (J_d, ..., J_1)."""
        d, k = self.d, self.k
        lv = self._block_leaves(blk)
        nl = lv.shape[0]
        if d == 3:
            s = sigma[lv].reshape(nl, nl, nl, k, k, k)          # o3 o2 o1 j3 j2 j1
            return s.transpose(0, 3, 1, 4, 2, 5).reshape(nl * k, nl * k, nl * k)
        s = sigma[lv].reshape(nl, nl, k, k)
        return s.transpose(0, 2, 1, 3).reshape(nl * k, nl * k)

    def form(self, sigma):
        phi = np.zeros((self.n_slots,) + self.slot_shape, dtype=np.complex128)
        for blk in self.blocks:
            S = self._dense(blk, sigma)
            if self.d == 3:
                o = np.einsum("cz,by,ax,zyx->cba", self._fmat(blk, 2, True), self._fmat(blk, 1, False),
                              self._fmat(blk, 0, False), S)
            else:
                o = np.einsum("by,ax,yx->ba", self._fmat(blk, 1, True), self._fmat(blk, 0, False), S)
            phi[blk["slot"]] += o
        return phi

    def _phase(self, tabf, tabh, b):
        n1, nh = self.n1, self.nh
        if self.d == 3:
            return tabh[b[2]][:, None, None] * tabf[b[1]][None, :, None] * tabf[b[0]][None, None, :]
        return tabh[b[1]][:, None] * tabf[b[0]][None, :]

    def merge_up(self, phi):
        for items, qf, qh in self.merge:
            for it in items:
                acc = 0
                for c in range(1 << self.d):
                    b = [(c >> a) & 1 for a in range(3)]
                    acc = acc + self._phase(qf, qh, b) * phi[it["child"][c]]
                phi[it["parent"]] = acc
        return phi

    def gather(self, phi):
        if self.fourier or len(self.gdst) == 0:
            return phi
        psi = np.zeros_like(phi)
        for i, dst in enumerate(self.gdst):
            acc = 0
            for q in range(self.gptr[i], self.gptr[i + 1]):
                code = int(self.gsrc[q]["code"])
                b = [code % 3, (code // 3) % 3, code // 9]
                acc = acc + self._phase(self.Pf, self.Ph, b) * phi[self.gsrc[q]["slot"]]
            psi[dst] = acc
        return psi

    def push_down(self, psi):
        for items, qf, qh in self.push:
            for it in items:
                for c in range(1 << self.d):
                    b = [(c >> a) & 1 for a in range(3)]
                    psi[it["child"][c]] = self._phase(qf, qh, b) * psi[it["parent"]]
        return psi

    def evaluate(self, psi, u):
        d, k = self.d, self.k
        for blk in self.blocks:
            lv = self._block_leaves(blk)
            nl = lv.shape[0]
            if d == 3:
                v = np.einsum("zc,yb,xa,cba->zyx", self._emat(blk, 2, True), self._emat(blk, 1, False),
                              self._emat(blk, 0, False), psi[blk["slot"]]).real
                v = v.reshape(nl, k, nl, k, nl, k).transpose(0, 2, 4, 1, 3, 5).reshape(nl ** 3, k ** 3)
            else:
                v = np.einsum("yb,xa,ba->yx", self._emat(blk, 1, True), self._emat(blk, 0, False),
                              psi[blk["slot"]]).real
                v = v.reshape(nl, k, nl, k).transpose(0, 2, 1, 3).reshape(nl ** 2, k ** 2)
            idx = lv.reshape(-1)
            if blk["flags"] & 1:
                u[idx] += v
            else:
                u[idx] = v
        return u

    def near(self, sigma, u):
        d, k = self.d, self.k
        for i, t in enumerate(self.ntgt):
            acc = np.zeros((k,) * d)
            for q in range(self.nptr[i], self.nptr[i + 1]):
                ns = self.nsrc[q]
                s = sigma[ns["leaf"]].reshape((k,) * d)
                T = [self.ntab[ns["tab"][a]] for a in range(d)]
                if d == 3:
                    acc += np.einsum("ck,bj,ai,kji->cba", T[2], T[1], T[0], s)
                else:
                    acc += np.einsum("bj,ai,ji->ba", T[1], T[0], s)
            if self.nflags[i] & 1:
                u[t] += acc.reshape(-1)
            else:
                u[t] = acc.reshape(-1)
        return u

    def transform(self, sigma):
        sigma = np.asarray(sigma, dtype=np.float64).reshape(-1, self.k ** self.d)
        # the device clears u first when the near field or a cutoff-level block adds into it;
        # otherwise every entry must be stored by exactly one writer (NaN shows a missed one)
        zero_u = len(self.ntgt) > 0 or any(int(b["flags"]) & 1 for b in self.blocks)
        u = np.zeros(sigma.shape) if zero_u else np.full(sigma.shape, np.nan)
        if len(self.blocks):
            phi = self.merge_up(self.form(sigma))
            psi = self.push_down(self.gather(phi))
            u = self.evaluate(psi, u)
        return self.near(sigma, u)
