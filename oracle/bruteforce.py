"""Determinant-space brute force for tiny closed-shell systems (oracle pin).

The Hamiltonian is built in the full Sz = 0 determinant space from spin-summed
excitation operators E_pq = a+_{p alpha} a_{q alpha} + a+_{p beta} a_{q beta}:

    H = sum_pq h_pq E_pq + 1/2 sum_pqrs (pq|rs) (E_pq E_rs - delta_qr E_ps)

(textbook second quantisation; with density fitting the two-electron part is
1/2 sum_Q L_Q L_Q with L_Q = sum_pq B[Q,p,q] E_pq).  Cluster and EOM operators
follow the paper's definitions (Sec. 2): T1 = t^i_a E^a_i,
T2 = 1/2 t^{ij}_{ab} E^a_i E^b_j, and likewise R1, R2.  The similarity
transform exp(-T) H exp(T) is applied to vectors by the terminating series of
the nilpotent T, so nothing here depends on any coupled-cluster algebra.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


class DetSpace:
    """Sz = 0 determinants of ``o`` alpha and ``o`` beta electrons in ``nmo``
    spatial orbitals; index = ia * nstr + ib."""

    def __init__(self, nmo: int, o: int):
        self.nmo, self.o = nmo, o
        self.strings = [sum(1 << p for p in c) for c in itertools.combinations(range(nmo), o)]
        self.index = {s: k for k, s in enumerate(self.strings)}
        self.nstr = len(self.strings)
        self.dim = self.nstr * self.nstr
        occmask = (1 << o) - 1
        lvl = np.array([bin(s & ~occmask).count("1") for s in self.strings])
        self.level = (lvl[:, None] + lvl[None, :]).reshape(-1)
        self.ref = self.index[occmask] * self.nstr + self.index[occmask]
        self._E = {}

    def _string_op(self, p, q):
        """a+_p a_q on the single-spin string space (sparse)."""
        rows, cols, vals = [], [], []
        for k, s in enumerate(self.strings):
            if not (s >> q) & 1:
                continue
            sign = (-1) ** bin(s & ((1 << q) - 1)).count("1")
            s1 = s & ~(1 << q)
            if (s1 >> p) & 1:
                continue
            sign *= (-1) ** bin(s1 & ((1 << p) - 1)).count("1")
            s2 = s1 | (1 << p)
            rows.append(self.index[s2]); cols.append(k); vals.append(sign)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.nstr, self.nstr))

    def E(self, p, q):
        """Spin-summed E_pq on the determinant space."""
        key = (p, q)
        if key not in self._E:
            e = self._string_op(p, q)
            eye = sp.identity(self.nstr, format="csr")
            self._E[key] = (sp.kron(e, eye) + sp.kron(eye, e)).tocsr()
        return self._E[key]

    def hamiltonian(self, h, B):
        """Sparse H from one-electron h and DF factors B (no nuclear term)."""
        nmo = self.nmo
        hp = h - 0.5 * np.einsum("Qpq,Qqs->ps", B, B)
        H = sp.csr_matrix((self.dim, self.dim))
        for p in range(nmo):
            for q in range(nmo):
                if hp[p, q] != 0.0:
                    H = H + hp[p, q] * self.E(p, q)
        for Q in range(B.shape[0]):
            L = sp.csr_matrix((self.dim, self.dim))
            for p in range(nmo):
                for q in range(nmo):
                    L = L + B[Q, p, q] * self.E(p, q)
            H = H + 0.5 * (L @ L)
        return H.tocsr()

    # --- excitation operators applied to vectors -------------------------
    def apply_excitation(self, x1, x2, vec):
        """(sum_ai x1[i,a] E_ai + 1/2 sum x2[i,j,a,b] E_ai E_bj) vec."""
        o = self.o
        v = self.nmo - o
        out = np.zeros_like(vec)
        ebj = {}
        for j in range(o):
            for b in range(v):
                ebj[j, b] = self.E(o + b, j) @ vec
        for i in range(o):
            for a in range(v):
                acc = x1[i, a] * vec
                if x2 is not None:
                    w = np.zeros_like(vec)
                    for j in range(o):
                        for b in range(v):
                            c = x2[i, j, a, b]
                            if c != 0.0:
                                w = w + c * ebj[j, b]
                    acc = acc + 0.5 * w
                out = out + self.E(o + a, i) @ acc
        return out

    def exp_apply(self, t1, t2, vec, sign=1.0):
        """exp(sign * T) vec by the terminating series (T is nilpotent)."""
        out = vec.copy()
        term = vec.copy()
        for k in range(1, 2 * self.o + 2):
            term = sign * self.apply_excitation(t1, t2, term) / k
            if not np.any(term):
                break
            out = out + term
        return out

    def reference(self, dtype=float):
        e0 = np.zeros(self.dim, dtype=dtype)
        e0[self.ref] = 1.0
        return e0

    def project_sd(self, vec):
        """Keep the singly and doubly excited components only."""
        out = vec.copy()
        out[(self.level < 1) | (self.level > 2)] = 0.0
        return out


def hbar_apply(ds, H, t1, t2, vec):
    """exp(-T) H exp(T) vec."""
    w = ds.exp_apply(t1, t2, vec, +1.0)
    w = H @ w
    return ds.exp_apply(t1, t2, w, -1.0)


def cc_residual_state(ds, H, t1, t2):
    """P_SD exp(-T) H exp(T) |0>: the CC residual as a determinant vector."""
    return ds.project_sd(hbar_apply(ds, H, t1, t2, ds.reference()))


def eom_sigma_state(ds, H, t1, t2, r1, r2):
    """P_SD [Hbar, R] |0> (connected EOM sigma) as a determinant vector."""
    e0 = ds.reference()
    Rk = ds.apply_excitation(r1, r2, e0)
    a = hbar_apply(ds, H, t1, t2, Rk)
    b = ds.apply_excitation(r1, r2, hbar_apply(ds, H, t1, t2, e0))
    return ds.project_sd(a - b)


def amplitudes_state(ds, x1, x2):
    """(X1 + X2)|0> for closed-shell singles/doubles coefficient arrays."""
    return ds.apply_excitation(x1, x2, ds.reference())


def singlet_sd_basis(ds):
    """Orthonormal basis (columns) of span{E_ai|0>, E_ai E_bj|0>}: the singlet
    singles-and-doubles space of the closed-shell reference."""
    o = ds.o
    v = ds.nmo - o
    e0 = ds.reference()
    cols = []
    for i in range(o):
        for a in range(v):
            cols.append(ds.E(o + a, i) @ e0)
    pairs = [(i, a) for i in range(o) for a in range(v)]
    for x in range(len(pairs)):
        for y in range(x, len(pairs)):
            (i, a), (j, b) = pairs[x], pairs[y]
            cols.append(ds.E(o + a, i) @ (ds.E(o + b, j) @ e0))
    M = np.array(cols).T
    U, s, _ = np.linalg.svd(M, full_matrices=False)
    return U[:, s > 1e-10 * s[0]]


def cisd_excitation_energies(ds, H):
    """Eigenvalues of the singlet S+D block of H minus E_HF (T = 0 EOM)."""
    Qb = singlet_sd_basis(ds)
    e0 = ds.reference()
    ehf = e0 @ (H @ e0)
    M = Qb.T @ (H @ Qb)
    return np.sort(np.linalg.eigvalsh(0.5 * (M + M.T))) - ehf


def fci_singlet_energies(ds, H):
    """Singlet FCI energies for a 2-electron system (o = 1): H in the span of
    |0>, E_ai|0>, E_ai E_bj|0>, which is the whole singlet space there."""
    e0 = ds.reference()
    Qb = np.column_stack([e0, singlet_sd_basis(ds)])
    Qb, _ = np.linalg.qr(Qb)
    M = Qb.T @ (H @ Qb)
    return np.sort(np.linalg.eigvalsh(0.5 * (M + M.T)))
