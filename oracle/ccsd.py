"""Closed-shell CCSD residual and ground-state amplitudes (oracle).

The paper defines the ground state by projecting exp(-T) H exp(T)|0> onto
singly and doubly excited determinants (Sec. 2) and uses the Bartlett/Stanton
closed-shell formalism without printing it.  Here the residual is written in
the T1-dressed frame: H~ = exp(-T1) H exp(T1) (``hamiltonian.dress``), after
which only T2 appears, and the closed-shell doubles/singles projections are
the standard biorthogonal spin-adapted CCSD equations (the closed-shell
formulation of Koch et al. and Scuseria et al.):

  Omega_ai   = F_ai + sum_ckd u^{cd}_{ki} (ad|kc) - sum_ckl u^{ac}_{kl} (ki|lc)
               + sum_ck u^{ac}_{ik} F_kc
  Omega_aibj = (ai|bj) + A + B + P^{ab}_{ij} (C + D + E)

with u^{ab}_{ij} = 2 t^{ab}_{ij} - t^{ba}_{ij}, L_pqrs = 2(pq|rs) - (ps|rq),
P^{ab}_{ij} f_aibj = f_aibj + f_bjai and

  A = sum_cd t^{cd}_{ij} (ac|bd)
  B = sum_kl t^{ab}_{kl} [(ki|lj) + sum_cd t^{cd}_{ij} (kc|ld)]
  C = -1/2 sum_ck t^{bc}_{kj} [(ki|ac) - 1/2 sum_dl t^{ad}_{li} (kd|lc)]
      - sum_ck t^{bc}_{ki} [(kj|ac) - 1/2 sum_dl t^{ad}_{lj} (kd|lc)]
  D = 1/2 sum_ck u^{bc}_{jk} [L_aikc + 1/2 sum_dl u^{ad}_{il} L_ldkc]
  E = sum_c t^{ac}_{ij} [F_bc - sum_dkl u^{bd}_{kl} (ld|kc)]
      - sum_k t^{ab}_{ik} [F_kj + sum_cdl u^{cd}_{lj} (kd|lc)]

Amplitude arrays are stored t1[i,a] and t2[i,j,a,b] = t^{ab}_{ij}
(t2[i,j,a,b] = t2[j,i,b,a]).  All integrals are evaluated from DF factors, so
the same code serves a Hamiltonian whose factors are not symmetric in (p,q)
(the dressed one) and the derivative Hamiltonian [H~, R1] used by EOM.

Pins (tests/test_oracle_ccsd.py): the residual equals the determinant-space
projection of exp(-T) H exp(T)|0> for random T; converged CCSD at o = 1 equals
FCI; MP2 energy matches second-order perturbation theory by brute force.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as hm

_SL = {"o": None, "v": None}


def _sl(o, c):
    return slice(0, o) if c == "o" else slice(o, None)


class DFHam:
    """Hamiltonian given by a Fock matrix F and a sum of DF products:
    (pq|rs) = sum_{(L,R) in pairs} sum_Q L[Q,p,q] R[Q,r,s].

    ``ladder_fn`` (optional) overrides the vvvv contraction
    x -> sum_cd x[i,j,c,d] (ac|bd).
    """

    def __init__(self, F, pairs, o, ladder_fn=None):
        self.F, self.pairs, self.o = F, pairs, o
        self.ladder_fn = ladder_fn

    def g(self, spec):
        o = self.o
        s = [_sl(o, c) for c in spec]
        out = None
        for L, R in self.pairs:
            blk = np.einsum("Qpq,Qrs->pqrs", L[:, s[0], s[1]], R[:, s[2], s[3]], optimize=True)
            out = blk if out is None else out + blk
        return out

    def gc(self, subs, x, spec):
        """einsum(subs, x, g[spec]) evaluated directly from the DF factors
        (``subs`` names the integral's four indices as its second operand)."""
        o = self.o
        sl = [_sl(o, c) for c in spec]
        lhs, out = subs.split("->")
        a, gidx = lhs.split(",")
        expr = f"{a},Q{gidx[0]}{gidx[1]},Q{gidx[2]}{gidx[3]}->{out}"
        res = None
        for L, R in self.pairs:
            blk = np.einsum(expr, x, L[:, sl[0], sl[1]], R[:, sl[2], sl[3]], optimize=True)
            res = blk if res is None else res + blk
        return res

    def f(self, spec):
        o = self.o
        return self.F[_sl(o, spec[0]), _sl(o, spec[1])]

    def ladder(self, x):
        if self.ladder_fn is not None:
            return self.ladder_fn(x)
        return ladder_dense(x, self.pairs, self.o)


def ladder_dense(x, pairs, o, chunk=32):
    """sum_cd x[i,j,c,d] (ac|bd), (ac|bd) formed in chunks of a from DF."""
    no = x.shape[0]
    v = x.shape[2]
    out = np.zeros(x.shape, dtype=np.result_type(x, pairs[0][0]))
    xm = x.reshape(no * no, v * v)
    for a0 in range(0, v, chunk):
        a1 = min(v, a0 + chunk)
        g = None
        for L, R in pairs:
            blk = np.einsum("Qac,Qbd->acbd", L[:, o + a0:o + a1, o:], R[:, o:, o:], optimize=True)
            g = blk if g is None else g + blk
        # out[ij, a, b] = sum_{cd} x[ij, c, d] g[a, c, b, d]
        gm = g.transpose(1, 3, 0, 2).reshape(v * v, (a1 - a0) * v)
        out[:, :, a0:a1, :] = (xm @ gm).reshape(no, no, a1 - a0, v)
    return out


def make_ham(h, B, o):
    """DFHam of a Hamiltonian (h, B): Fock from the closed-shell formula."""
    return DFHam(hm.fock(h, B, o), [(B, B)], o)


def uamp(t2):
    """u^{ab}_{ij} = 2 t^{ab}_{ij} - t^{ba}_{ij}."""
    return 2.0 * t2 - t2.swapaxes(2, 3)


def omega(t2, H):
    """Dressed-frame CCSD residual (Omega1[i,a], Omega2[i,j,a,b]) for T2 only."""
    e = np.einsum
    u = uamp(t2)
    # singles
    O1 = H.f("vo").T.copy()
    O1 = O1 + H.gc("kicd,adkc->ia", u, "vvov")
    O1 = O1 - H.gc("klac,kilc->ia", u, "ooov")
    O1 = O1 + e("ikac,kc->ia", u, H.f("ov"), optimize=True)
    # doubles
    O2 = H.g("vovo").transpose(1, 3, 0, 2).copy()          # (ai|bj) -> [i,j,a,b]
    O2 = O2 + H.ladder(t2)
    W = H.g("oooo") + H.gc("ijcd,kcld->kilj", t2, "ovov")
    O2 = O2 + e("klab,kilj->ijab", t2, W, optimize=True)
    Wc = H.g("oovv") - 0.5 * H.gc("liad,kdlc->kiac", t2, "ovov")
    C = -0.5 * e("kjbc,kiac->ijab", t2, Wc, optimize=True) - e("kibc,kjac->ijab", t2, Wc, optimize=True)
    # L_aikc = 2(ai|kc) - (ac|ki);  L_ldkc = 2(ld|kc) - (lc|kd)
    Wd = (2.0 * H.g("voov") - H.g("vvoo").transpose(0, 3, 2, 1)
          + H.gc("ilad,ldkc->aikc", u, "ovov") - 0.5 * H.gc("ilad,lckd->aikc", u, "ovov"))
    D = 0.5 * e("jkbc,aikc->ijab", u, Wd, optimize=True)
    Fvv = H.f("vv") - H.gc("klbd,ldkc->bc", u, "ovov")
    Foo = H.f("oo") + H.gc("ljcd,kdlc->kj", u, "ovov")
    E = e("ijac,bc->ijab", t2, Fvv, optimize=True) - e("ikab,kj->ijab", t2, Foo, optimize=True)
    CDE = C + D + E
    O2 = O2 + CDE + CDE.transpose(1, 0, 3, 2)
    return O1, O2


def residual(t1, t2, h, B, o):
    """CCSD residual <mu~| exp(-T) H exp(T) |0> for mu = singles, doubles."""
    hd, Bd = hm.dress(h, B, t1, o)
    return omega(t2, make_ham(hd, Bd, o))


def energy(t1, t2, eps, B, o):
    """CCSD correlation energy sum_ijab (2(ia|jb) - (ib|ja)) (t^{ab}_{ij} + t^a_i t^b_j)
    (HF Fock diagonal, so no f_ia t^a_i term)."""
    g = np.einsum("Qia,Qjb->iajb", B[:, :o, o:], B[:, :o, o:], optimize=True)
    tau = t2 + np.einsum("ia,jb->ijab", t1, t1)
    return float(np.einsum("ijab,iajb->", tau, 2.0 * g - g.transpose(0, 3, 2, 1)))


def denominators(eps, o):
    eo, ev = eps[:o], eps[o:]
    d1 = eo[:, None] - ev[None, :]
    d2 = eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    return d1, d2


def mp1_t2(eps, B, o):
    """First-order amplitudes t^{ab}_{ij} = (ai|bj) / (f_ii + f_jj - f_aa - f_bb)
    (Eq. T1 of the paper: G^{ij}_{ab} = <ab|ij> = (ai|bj)).  Formed one occupied i at a
    time (the same sums; it keeps the large systems within host memory)."""
    v = len(eps) - o
    eo, ev = eps[:o], eps[o:]
    Bia = np.ascontiguousarray(B[:, o:, :o].transpose(0, 2, 1))      # [Q, i, a] = B[Q, a, i]
    t = np.empty((o, o, v, v))
    for i in range(o):
        g = np.einsum("Qa,Qjb->jab", Bia[:, i, :], Bia, optimize=True)   # (ai|bj)
        t[i] = g / (eo[i] + eo[:, None, None] - ev[None, :, None] - ev[None, None, :])
    return t


def solve_ccsd(eps, B, o, tol=1e-11, maxiter=200):
    """Converged closed-shell CCSD amplitudes by Jacobi updates with DIIS.

    Returns (t1, t2, energy, max|residual|)."""
    h = hm.hcore_from_fock(eps, B, o)
    d1, d2 = denominators(eps, o)
    t1 = np.zeros(d1.shape)
    t2 = mp1_t2(eps, B, o)
    hist_t, hist_r = [], []
    for it in range(maxiter):
        r1, r2 = residual(t1, t2, h, B, o)
        err = max(np.abs(r1).max(), np.abs(r2).max())
        if err < tol:
            break
        t1n = t1 + r1 / d1
        t2n = t2 + r2 / d2
        vec = np.concatenate([t1n.ravel(), t2n.ravel()])
        res = np.concatenate([(r1 / d1).ravel(), (r2 / d2).ravel()])
        hist_t.append(vec); hist_r.append(res)
        hist_t, hist_r = hist_t[-8:], hist_r[-8:]
        m = len(hist_r)
        if m >= 2:
            A = -np.ones((m + 1, m + 1)); A[m, m] = 0.0
            A[:m, :m] = np.array([[x @ y for y in hist_r] for x in hist_r])
            rhs = np.zeros(m + 1); rhs[m] = -1.0
            c = np.linalg.lstsq(A, rhs, rcond=None)[0][:m]
            vec = sum(ci * x for ci, x in zip(c, hist_t))
        t1 = vec[:t1.size].reshape(t1.shape)
        t2 = vec[t1.size:].reshape(t2.shape)
        t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    return t1, t2, energy(t1, t2, eps, B, o), err
