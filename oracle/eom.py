"""Closed-shell singlet EOM-CCSD sigma vectors (oracle).

Definition (Sec. 2): the EOM-CCSD eigenproblem is Hbar R|0> = E R|0> with
Hbar = exp(-T) H exp(T); its excitation energies are the eigenvalues of the
map R -> sigma(R) = <mu~| [Hbar, R] |0>, mu = singles, doubles.  Because all
excitation operators commute, [Hbar, R] is the derivative of
exp(-(T + e R)) H exp(T + e R) at e = 0, so sigma is exactly the
Jacobian-vector product of the CCSD residual Omega(T) in direction R.

Two evaluations:

* ``sigma_jvp``: the definition itself, by complex-step differentiation of
  ``ccsd.residual`` (Omega is a polynomial with real coefficients, so
  Im Omega(T + i h R) / h is its derivative to rounding for tiny h);
* ``Sigma``: explicit terms with R-independent intermediates (the form the
  library evaluates).  The R2 part is the product rule applied to each term of
  the dressed residual; the R1 part is the dressed residual evaluated with the
  Hamiltonian [H~, R1] (``hamiltonian.commutator_r1``), because the residual
  is linear in the Hamiltonian and d/de exp(-(T1+eR1)) H exp(T1+eR1) =
  [H~, R1].

Pins (tests/test_oracle_eom.py): both agree with the determinant-space
P_SD [Hbar, R]|0> for random T and R; at T = 0 the spectrum equals the singlet
CISD excitation energies; at o = 1 with converged CCSD it equals FCI.
"""
from __future__ import annotations

import numpy as np

from . import ccsd
from . import hamiltonian as hm


def sigma_jvp(t1, t2, r1, r2, h, B, o, step=1e-30):
    """sigma = d/de Omega(T + e R) at e = 0 by complex step."""
    o1, o2 = ccsd.residual(t1 + 1j * step * r1, t2 + 1j * step * r2, h, B, o)
    return o1.imag / step, o2.imag / step


class Sigma:
    """Explicit closed-shell EOM-CCSD sigma at fixed ground-state T.

    ``ladder_r2`` (optional) replaces the vvvv contraction applied to R2,
    sum_cd r^{cd}_{ij} (ac|bd); the PNO-basis sigma passes its own.
    """

    def __init__(self, t1, t2, h, B, o):
        e = np.einsum
        self.o = o
        self.t2 = t2
        self.hd, self.Bd = hm.dress(h, B, t1, o)
        H = ccsd.make_ham(self.hd, self.Bd, o)
        self.H = H
        u = ccsd.uamp(t2)
        self.u = u
        g_ovov = H.g("ovov")
        self.g_ovov = g_ovov
        self.L_ovov = 2.0 * g_ovov - g_ovov.transpose(0, 3, 2, 1)
        self.g_vvov = H.g("vvov")
        self.g_ooov = H.g("ooov")
        # R-independent intermediates of the dressed residual
        self.W = H.g("oooo") + e("ijcd,kcld->kilj", t2, g_ovov, optimize=True)
        self.Wc = H.g("oovv") - 0.5 * e("liad,kdlc->kiac", t2, g_ovov, optimize=True)
        L_voov = 2.0 * H.g("voov") - H.g("vvoo").transpose(0, 3, 2, 1)
        self.Wd = L_voov + 0.5 * e("ilad,ldkc->aikc", u, self.L_ovov, optimize=True)
        self.Fvv = H.f("vv") - e("klbd,ldkc->bc", u, g_ovov, optimize=True)
        self.Foo = H.f("oo") + e("ljcd,kdlc->kj", u, g_ovov, optimize=True)
        self.Fov = H.f("ov")
        # T2 contracted with the rank-o part of the R1-derivative ladder
        self.Y1 = e("ijcd,kcbd->ijkb", t2, H.g("ovvv"), optimize=True)
        self.Y2 = e("ijcd,ackd->ijak", t2, self.g_vvov, optimize=True)

    # ------------------------------------------------------------------
    def r2_part(self, r2, ladder_r2=None):
        """Product-rule derivative of the dressed residual in direction R2."""
        e = np.einsum
        t, u = self.t2, self.u
        ur = ccsd.uamp(r2)
        g = self.g_ovov
        s1 = (e("kicd,adkc->ia", ur, self.g_vvov, optimize=True)
              - e("klac,kilc->ia", ur, self.g_ooov, optimize=True)
              + e("ikac,kc->ia", ur, self.Fov, optimize=True))
        lad = self.H.ladder(r2) if ladder_r2 is None else ladder_r2(r2)
        X = e("ijcd,kcld->kilj", r2, g, optimize=True)
        s2 = e("klab,kilj->ijab", r2, self.W, optimize=True) + e("klab,kilj->ijab", t, X, optimize=True)
        Xc = -0.5 * e("liad,kdlc->kiac", r2, g, optimize=True)
        C = (-0.5 * e("kjbc,kiac->ijab", r2, self.Wc, optimize=True) - e("kibc,kjac->ijab", r2, self.Wc, optimize=True)
             - 0.5 * e("kjbc,kiac->ijab", t, Xc, optimize=True) - e("kibc,kjac->ijab", t, Xc, optimize=True))
        Xd = 0.5 * e("ilad,ldkc->aikc", ur, self.L_ovov, optimize=True)
        D = 0.5 * e("jkbc,aikc->ijab", ur, self.Wd, optimize=True) + 0.5 * e("jkbc,aikc->ijab", u, Xd, optimize=True)
        Fvv_r = -e("klbd,ldkc->bc", ur, g, optimize=True)
        Foo_r = e("ljcd,kdlc->kj", ur, g, optimize=True)
        E = (e("ijac,bc->ijab", r2, self.Fvv, optimize=True) - e("ikab,kj->ijab", r2, self.Foo, optimize=True)
             + e("ijac,bc->ijab", t, Fvv_r, optimize=True) - e("ikab,kj->ijab", t, Foo_r, optimize=True))
        CDE = C + D + E
        s2 = s2 + CDE + CDE.transpose(1, 0, 3, 2)
        return s1, s2, lad

    def r1_part(self, r1):
        """Dressed residual evaluated with the Hamiltonian [H~, R1]."""
        o = self.o
        hp, Bp = hm.commutator_r1(self.hd, self.Bd, r1, o)
        Bd = self.Bd
        # Fock of [H~, R1]: derivative of h + 2J - K, each DF product split
        J = (np.einsum("Qpq,Qkk->pq", Bp, Bd[:, :o, :o]) + np.einsum("Qpq,Qkk->pq", Bd, Bp[:, :o, :o]))
        K = (np.einsum("Qpk,Qkq->pq", Bp[:, :, :o], Bd[:, :o, :]) + np.einsum("Qpk,Qkq->pq", Bd[:, :, :o], Bp[:, :o, :]))
        Fp = hp + 2.0 * J - K

        def ladder_rank_o(x):
            # vv block of B' is -rho_vo B~_ov (rank o), so
            # sum_cd x (ac|bd)' = -sum_k r1[k,a] Y1[ijkb] - sum_k r1[k,b] Y2[ijak]
            assert x is self.t2
            return (-np.einsum("ka,ijkb->ijab", r1, self.Y1, optimize=True)
                    - np.einsum("kb,ijak->ijab", r1, self.Y2, optimize=True))

        Hp = ccsd.DFHam(Fp, [(Bp, Bd), (Bd, Bp)], o, ladder_fn=ladder_rank_o)
        return ccsd.omega(self.t2, Hp)

    def __call__(self, r1, r2, ladder_r2=None):
        a1, a2, lad = self.r2_part(r2, ladder_r2)
        b1, b2 = self.r1_part(r1)
        return a1 + b1, a2 + b2 + lad
