"""The PNO-space sigma evaluated pair by pair, without canonical R2 or sigma2 (oracle O2).

Test infrastructure: only tests/, the smoke check and the benchmark's CPU legs use it.

What it computes (Sec. 2): the same map as ``pno.PNOSigma``, sigma_bar = P sigma(P R) in
PNO/OSV coordinates, sigma being the closed-shell EOM-CCSD Jacobian of ``eom.Sigma``
(the derivative of the T1-dressed CCSD residual) and P the projector onto the
state-averaged PNO/OSV spaces.  ``PNOSigma`` back-transforms to the canonical o^2 v^2
space and applies the canonical sigma; here every term of ``eom.Sigma`` is evaluated with
the R-dependent factor as one PNO block R(k,l) (rows on k) or one canonical singles row
r_k = U^k r_bar^k, and the rest projected into the PNO spaces it connects.  No canonical
R2 or sigma2 and no integral with three or four virtual indices is formed: those enter
through the density-fitting factors B^Q, (pq|rs) = sum_Q B^Q_pq B^Q_rs.  The only o^2 v^2
arrays are the amplitudes t, u = 2t - t(ab swapped) and the integrals (kc|ld).

Terms of the doubles block of stored pair ij (U = U^{ij}, S(p,q) = U_p^T U_q):
  4-virtual ladder   sum_Q Bb_Q R Bb_Q^T,  Bb_Q = U^T B^Q_vv U
  T2 ladder          sum_kl <gb[kl], R> U^T t^{kl} U,  gb[kl] = U^T G^{kl} U, G^{kl}_cd = (kc|ld)
  virtual Fock       R Fb^T + Fb R, Fb = U^T F~vv U
  occupied ladder    sum_kl W[k,i,l,j] S(ij,kl) R(k,l) S(kl,ij)
  and, for the ordered pairs (i,j) and (j,i) (P-symmetrisation of C + D + E):
  rings C1..C4, D1, D2 through the mixed-pair blocks MC, MD, MZ, MZd (``_MC`` ... ``_MZd``),
  occupied Fock E2, the global terms E3 (v x v FvR) and E4 (o x o FoR), and the R1 terms.
Terms of the singles block of occupied i: the R2 -> sigma1 terms (s1 of eom.Sigma) and
the R1 -> sigma1 singles-singles block.

Pins (tests/test_oracle_pno_direct.py): equal to ``PNOSigma`` to 1e-12 with T1 = 0 and
T1 != 0, with empty and full PNO spaces, and for any subset of output blocks (which is how
samples of the large workload are computed on the host).
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as hm

e = lambda *a: np.einsum(*a, optimize=True)


class PNOSigmaDirect:
    def __init__(self, t1, t2, h, B, o, space):
        sp = self.sp = space
        self.o = o
        v = self.v = space.v
        self.has_t1 = t1 is not None and bool(np.any(t1 != 0))
        hd, Bd = hm.dress(h, B, t1, o) if self.has_t1 else (h, B)
        F = hm.fock(hd, Bd, o)
        self.Foo, self.Fov, self.Fvv = F[:o, :o].copy(), F[:o, o:].copy(), F[o:, o:].copy()
        self.Boo = np.ascontiguousarray(Bd[:, :o, :o])
        self.Bov = np.ascontiguousarray(Bd[:, :o, o:])
        self.Bvo = np.ascontiguousarray(Bd[:, o:, :o])
        nq = self.Bov.shape[0]
        self.t = t2
        self.u = np.multiply(t2, 2.0)
        self.u -= t2.swapaxes(2, 3)                                   # u = 2 t - t(ab swapped)
        # (kc|ld) at [k,c,l,d]
        Bm = self.Bov.reshape(nq, o * v)
        self.g = np.empty((o * v, o * v))
        for r0 in range(0, o * v, 3600):
            self.g[r0:r0 + 3600] = Bm[:, r0:r0 + 3600].T @ Bm
        self.g = self.g.reshape(o, v, o, v)
        self._pid = {}
        for p, (i, j) in enumerate(sp.pairs):
            self._pid[i, j] = self._pid[j, i] = p
        t, u, g = self.t, self.u, self.g
        # R-independent intermediates (eom.Sigma), built from the DF factors and (kc|ld)
        self.W = e("Qki,Qlj->kilj", self.Boo, self.Boo)
        for k in range(o):
            self.W[k] += e("ijcd,cld->ilj", t, g[k])                  # sum_cd t^{cd}_{ij} (kc|ld)
        # FvvI = Fvv - sum u[k,l,b,d] (ld|kc),  FooI = Foo + sum u[l,j,c,d] (kd|lc),
        # Xv = Fvv - sum u[k,l,a,c] (kd|lc),     Xo = Foo + sum u[k,i,c,d] (md|kc):
        # the outer occupied index summed one slice at a time (whole-array contractions
        # would copy u and (kc|ld), 10 GB each at o = 60, v = 600)
        self.FvvI, self.FooI = self.Fvv.copy(), self.Foo.copy()
        self.Xv, self.Xo = self.Fvv.copy(), self.Foo.copy()
        for k in range(o):
            gk = np.ascontiguousarray(g[:, :, k, :])                   # (ld|kc) at [l,d,c]
            self.FvvI -= e("lbd,ldc->bc", u[k], gk)
            self.FooI += e("jcd,mdc->mj", u[k], gk)                    # l = k here
            self.Xv -= e("lac,dlc->ad", u[k], g[k])
            self.Xo += e("icd,mdc->mi", u[k], gk)
        self.g_ooov = e("Qki,Qlc->kilc", self.Boo, self.Bov)          # (ki|lc)
        self.g_ovoo = e("Qkc,Qlj->kclj", self.Bov, self.Boo)          # (kc|lj)
        self.g_oovo = e("Qki,Qbj->kibj", self.Boo, self.Bvo)          # (ki|bj)
        self.g_vooo = e("Qai,Qkj->aikj", self.Bvo, self.Boo)          # (ai|kj)
        # B^Q_ab, stored contiguous (after the o^2 v^2 contractions above, whose temporaries
        # are the host-memory peak of this setup)
        self.Bvv = np.ascontiguousarray(Bd[:, o:, o:])

    # -- bases -----------------------------------------------------------------------
    def U(self, x, y):
        return self.sp.U[min(x, y), max(x, y)]

    def n(self, x, y):
        return self.U(x, y).shape[1]

    def _R(self, vec, x, y):
        """R^{xy} in the PNO basis of pair {x, y}, rows on x."""
        blk = self.sp.block(vec, self._pid[x, y])
        return blk if x <= y else blk.T

    # -- mixed-pair ring blocks ------------------------------------------------------------
    def _rf(self, kind, x, y):
        """(ov x n) factor of pair {x, y} for its occupied index x, rows (l, d):
          TU: sum_a t[l,x,a,d] U[a,A]           UU: sum_a u[x,l,a,d] U[a,A]
          GU: sum_c (xd|lc) U[c,C]              LU: sum_c L[l,d,x,c] U[c,C]
        with L[p,q,r,s] = 2 (pq|rs) - (ps|rq).  The rank-(ov) parts of the ring
        intermediates are products of two of them (``_MC`` ... ``_MZd``)."""
        key = (kind, x, y)
        if key not in self._cache:
            Uq = self.U(x, y)
            o, v, g = self.o, self.v, self.g
            if kind == "TU":
                f = e("lad,aA->ldA", self.t[:, x], Uq)
            elif kind == "UU":
                f = e("lad,aA->ldA", self.u[x], Uq)
            elif kind == "GU":
                f = e("dlc,cC->ldC", g[x], Uq)
            else:
                L = 2.0 * g[:, :, x, :] - g[x].transpose(1, 0, 2)       # L[l,d,x,c] = 2 (ld|xc) - (lc|xd)
                f = e("ldc,cC->ldC", L, Uq)
            self._cache[key] = f.reshape(o * v, -1)
        return self._cache[key]

    def _kiac(self, k, i):
        """(ki|ac) = sum_Q B^Q_ki B^Q_ac (v x v), kept for the rest of the sigma call.  One
        pass over B_vv gives it for every occupied index of the requested output blocks."""
        key = ("kiac", k, i)
        if key not in self._cache:
            occ = sorted(set(self._occ) | {i})
            blk = np.tensordot(self.Boo[:, k, occ], self.Bvv, axes=(0, 0))
            for n_, x in enumerate(occ):
                self._cache[("kiac", k, x)] = blk[n_]
        return self._cache[key]

    def _MC(self, i, j, k):
        """U(i,j)^T Wc[k,i] U(k,j), Wc[k,i,a,c] = (ki|ac) - 1/2 sum_{l,d} t[l,i,a,d] (kd|lc)."""
        kiac = self._kiac(k, i)
        return self.U(i, j).T @ kiac @ self.U(k, j) - 0.5 * self._rf("TU", i, j).T @ self._rf("GU", k, j)

    def _MD(self, i, j, k):
        """U(i,j)^T Wd[.,i,k,.] U(j,k), Wd[a,i,k,c] = 2 (ai|kc) - (ki|ac) + 1/2 sum u[i,l,a,d] L[l,d,k,c]."""
        X = 2.0 * e("Qa,Qc->ac", self.Bvo[:, :, i], self.Bov[:, k, :]) - self._kiac(k, i)
        return self.U(i, j).T @ X @ self.U(j, k) + 0.5 * self._rf("UU", i, j).T @ self._rf("LU", k, j)

    def _MZ(self, k, i, j):
        """U(k,i)^T Zt[k,j] U(i,j), Zt[k,j][d,b] = sum_{m,c} (md|kc) t[m,j,b,c]."""
        return self._rf("GU", k, i).T @ self._rf("TU", j, i)

    def _MZd(self, k, i, j):
        """U(i,k)^T Zd[k,j] U(i,j), Zd[k,j][d,b] = sum_{m,c} L[k,d,m,c] u[j,m,b,c]."""
        return self._rf("LU", k, i).T @ self._rf("UU", j, i)

    # -- sigma --------------------------------------------------------------------------
    def __call__(self, vec, pairs=None, singles=None):
        """sigma_bar of the packed vector.  With `pairs` (stored-pair indices) and/or
        `singles` (occupied indices) only those output blocks are evaluated, the rest
        of the result is zero."""
        sp, o, v, g = self.sp, self.o, self.v, self.g
        self._cache = {}
        pairs = range(len(sp.pairs)) if pairs is None else pairs
        singles = range(o) if singles is None else singles
        self._occ = sorted({x for p in pairs if sp.n_ij[p] for x in sp.pairs[p]})
        out = np.zeros(sp.length)
        r1 = [sp.Ui[i] @ vec[sp.off_i[i]:sp.off_i[i + 1]] for i in range(o)]
        # R1-dependent v x v global of the ordered-pair R1 terms:
        # Lam[b,c] = sum_{m,d} (2 (bc|md) - (bd|mc)) r_m,d
        rho = sum(e("Qd,d->Q", self.Bov[:, m, :], r1[m]) for m in range(o))
        self._Lam = 2.0 * e("Qbc,Q->bc", self.Bvv, rho)
        for m in range(o):
            self._Lam -= e("Qbd,d,Qc->bc", self.Bvv, r1[m], self.Bov[:, m, :])
        # R-dependent globals: FvR = -sum_kl U ur(k,l) U^T G^{lk},  FoR[k,j] = sum_l <U^T X_k U, ur(l,j)>
        # with ur = 2 R - R^T, G^{lk}[d,c] = (ld|kc), X_k[c,d] = (kd|lc)
        FvR = np.zeros((v, v))
        FoR = np.zeros((o, o))
        for k in range(o):
            for l in range(o):
                if not self.n(k, l):
                    continue
                Ukl = self.U(k, l)
                R = self._R(vec, k, l)
                ur = 2.0 * R - R.T
                FvR -= Ukl @ ur @ (Ukl.T @ g[l, :, k, :])
                for m in range(o):
                    FoR[m, l] += np.sum((Ukl.T @ g[m, :, k, :].T @ Ukl) * ur)
        for p in pairs:
            if sp.n_ij[p]:
                # the (ov x n) ring factors of one output block are dropped before the next
                # (at o = 60, v = 600 those of a few blocks fill the host memory)
                self._cache = {key: x for key, x in self._cache.items() if key[0] == "kiac"}
                out[sp.off_ij[p]:sp.off_ij[p + 1]] = self._pair_block(vec, p, r1, FvR, FoR).ravel()
        for i in singles:
            if sp.n_i[i]:
                out[sp.off_i[i]:sp.off_i[i + 1]] = sp.Ui[i].T @ self._singles_canonical(vec, i, r1)
        return out

    def _pair_block(self, vec, p, r1, FvR, FoR):
        sp, t = self.sp, self.t
        i, j = sp.pairs[p]
        Up = sp.U[i, j]
        R = sp.block(vec, p)
        # 4-virtual ladder
        BU = e("Qad,dB->QaB", self.Bvv, Up)
        Bb = e("aA,QaC->QAC", Up, BU)
        sig = e("QAC,CD,QBD->AB", Bb, R, Bb)
        # T2 ladder
        Bh = e("Qkc,cC->QkC", self.Bov, Up)
        gb = e("QkC,QlD->klCD", Bh, Bh)
        tb = e("aA,klab,bB->klAB", Up, t, Up)
        sig += e("klAB,klCD,CD->AB", tb, gb, R)
        # virtual Fock
        Fb = Up.T @ self.FvvI @ Up
        sig += R @ Fb.T + Fb @ R
        # occupied ladder
        for q, (k, l) in enumerate(sp.pairs):
            if not sp.n_ij[q]:
                continue
            Spq = Up.T @ sp.U[k, l]
            Rq = sp.block(vec, q)
            sig += self.W[k, i, l, j] * (Spq @ Rq @ Spq.T)
            if k != l:
                sig += self.W[l, i, k, j] * (Spq @ Rq.T @ Spq.T)
        # P-symmetrised terms: ordered (i,j) as is and (j,i) transposed (both orders of ii)
        for ordr, (x, y) in enumerate(((i, j), (j, i))):
            C = self._ordered(vec, x, y, FvR, FoR, r1)
            sig += C if ordr == 0 else C.T
        # R1 terms outside the symmetrised part
        sig += self._r1_direct(p, r1)
        return sig

    def _ordered(self, vec, i, j, FvR, FoR, r1):
        """Contribution of the ordered pair (i, j) (C + D + E of eom.Sigma and the ordered
        R1 terms), in the basis of pair {i, j} with rows on i."""
        o, t = self.o, self.t
        Uij = self.U(i, j)
        R = lambda x, y: self._R(vec, x, y)
        C = np.zeros((Uij.shape[1], Uij.shape[1]))
        for k in range(o):
            if self.n(k, j):
                Skj = self.U(k, j).T @ Uij
                C += -0.5 * self._MC(i, j, k) @ R(k, j).T @ Skj          # C1
                C += 0.5 * Skj.T @ R(k, j) @ self._MZ(k, j, i)            # C4
            if self.n(k, i):
                Ski = self.U(k, i).T @ Uij
                C += -1.0 * self._MC(j, i, k) @ R(k, i).T @ Ski          # C2
                C += 0.25 * Ski.T @ R(k, i) @ self._MZ(k, i, j)           # C3
                Rik = R(i, k)
                C += Ski.T @ (0.5 * Rik - 0.25 * Rik.T) @ self._MZd(k, i, j)   # D2
                C += -self.FooI[k, j] * (Ski.T @ Rik @ Ski)                 # E2
            if self.n(j, k):
                Rjk = R(j, k)
                C += self._MD(i, j, k) @ (Rjk.T - 0.5 * Rjk) @ (self.U(j, k).T @ Uij)   # D1
            C += -FoR[k, j] * (Uij.T @ t[i, k] @ Uij)                       # E4
        C += (Uij.T @ t[i, j]) @ FvR.T @ Uij                                # E3
        C += self._r1_ordered(i, j, Uij, r1)
        return C

    # -- R1 couplings ---------------------------------------------------------------------
    def _r1_direct(self, p, r1):
        """sigma_bar^{ij} from R1, the terms outside the P-symmetrised part."""
        sp, o, t = self.sp, self.o, self.t
        i, j = sp.pairs[p]
        Up = sp.U[i, j]
        # sum_c r_i,c (ac|bj) + sum_c r_j,c (ai|bc), projected
        sig = e("aA,Qac,c,Qb,bB->AB", Up, self.Bvv, r1[i], self.Bvo[:, :, j], Up)
        sig += e("aA,Qa,Qbc,c,bB->AB", Up, self.Bvo[:, :, i], self.Bvv, r1[j], Up)
        # sum_kl U^T t^{kl} U [(kc|lj) r_i,c + (ki|lc) r_j,c]
        H = e("kcl,c->kl", self.g_ovoo[:, :, :, j], r1[i]) + e("klc,c->kl", self.g_ooov[:, i, :, :], r1[j])
        sig += e("aA,klab,bB,kl->AB", Up, t, Up, H)
        # outer products with U^T r_k: wa[k,B] = -sum_b ((ki|bj) + Y1[i,j,k,b]) U[b,B],
        # wb[k,A] = -sum_a ((ai|kj) + Y2[i,j,a,k]) U[a,A], Y1 = sum_cd t[i,j,c,d] (kc|bd),
        # Y2 = sum_cd t[i,j,c,d] (ac|kd)
        BUt = e("Qbd,bB->QdB", self.Bvv, Up)
        wa = -(self.g_oovo[:, i, :, j] @ Up + e("Qkc,cd,QdB->kB", self.Bov, t[i, j], BUt))
        wb = -(self.g_vooo[:, i, :, j].T @ Up + e("Qkd,cd,QcA->kA", self.Bov, t[i, j], BUt))
        for k in range(o):
            s = Up.T @ r1[k]
            sig += np.outer(s, wa[k]) + np.outer(wb[k], s)
        return sig

    def _r1_ordered(self, x, y, Up, r1):
        """R1 terms of the ordered pair (x, y), rows on x."""
        o, v, t, u = self.o, self.v, self.t, self.u
        n = Up.shape[1]
        BUt = e("Qbd,bB->QdB", self.Bvv, Up)                      # sum_b B[Q,b,d] U[b,B]
        ut = e("kbc,bB->kcB", u[y], Up)                           # sum_b u[y,k,b,c] U[b,B]
        ty = e("kbc,bB->kcB", t[:, y], Up)                        # sum_b t[k,y,b,c] U[b,B]
        tx = e("kbc,bB->kcB", t[:, x], Up)
        C = np.zeros((n, n))
        # sum U[a,A] [(ad|kc) ut - 1/2 (ac|kd) (ut + ty)][k,c,B] r_x,d
        C += e("aA,Qad,d,Qkc,kcB->AB", Up, self.Bvv, r1[x], self.Bov, ut)
        C += -0.5 * e("QcA,Qkd,d,kcB->AB", BUt, self.Bov, r1[x], ut + ty)
        # - sum U[a,A] (ac|kd) r_y,d tx[k,c,B]
        C += -e("QcA,Qkd,d,kcB->AB", BUt, self.Bov, r1[y], tx)
        # U^T t[x,y] Lam^T U, Lam[b,c] = sum_{m,d} (2 (bc|md) - (bd|mc)) r_m,d (formed once
        # per sigma call)
        C += Up.T @ t[x, y] @ self._Lam.T @ Up
        # - sum_k gam[k] U^T t[x,k] U, gam[k] = sum_{m,d} (2 (ky|md) - (kd|my)) r_m,d
        for k in range(o):
            gam = sum(2.0 * self.g_ooov[k, y, m] @ r1[m] - self.g_ovoo[k, :, m, y] @ r1[m] for m in range(o))
            C += -gam * (Up.T @ t[x, k] @ Up)
        # outer products (U^T r_m) qb[m]: qb = sum_b Qb[m,x,y,b] U[b,B],
        # Qb[m,x,y,b] = Q2[m,y,x,b] + 1/2 Q2[m,x,y,b] - Q5[m,x,y,b] + 1/2 Q6[m,x,y,b],
        # Q2[m,i,j,b] = sum (ki|mc) t[k,j,b,c], Q5[m,i,j,b] = sum (mi|kc) u[j,k,b,c],
        # Q6[m,i,j,b] = sum (mc|ki) u[j,k,b,c]
        Q2 = lambda a, b_: e("kmc,kbc->mb", self.g_ooov[:, a], t[:, b_])
        qb = (Q2(y, x) + 0.5 * Q2(x, y) - e("mkc,kbc->mb", self.g_ooov[:, x], u[y])
              + 0.5 * e("mck,kbc->mb", self.g_ovoo[:, :, :, x], u[y])) @ Up
        for m in range(o):
            C += np.outer(Up.T @ r1[m], qb[m])
        if self.has_t1:
            # F~ov terms: - (Fov t[x,y]^T U)[m] outer U^T r_m and - sum_m U^T t[x,m] U (Fov[m] . r_y)
            e2a = -(self.Fov @ t[x, y].T) @ Up
            for m in range(o):
                C += np.outer(e2a[m], Up.T @ r1[m])
                C += -(self.Fov[m] @ r1[y]) * (Up.T @ t[x, m] @ Up)
        return C

    def _singles_canonical(self, vec, i, r1):
        """Canonical sigma1 row i (then projected by the caller): the R2 -> sigma1 terms
        s1 of eom.Sigma and the R1 -> sigma1 singles-singles terms."""
        o, v, u, g = self.o, self.v, self.u, self.g
        s = np.zeros(v)
        for k in range(o):
            for l in range(o):
                if not self.n(k, l):
                    continue
                Ukl = self.U(k, l)
                R = self._R(vec, k, l)
                ur = Ukl @ (2.0 * R - R.T) @ Ukl.T                    # canonical ur^{kl}, v x v
                if l == i:
                    # sum_cd ur[k,i,c,d] (ad|kc)
                    s += e("cd,Qad,Qc->a", ur, self.Bvv, self.Bov[:, k, :])
                # - sum_c ur[k,l,a,c] (ki|lc)
                s -= ur @ self.g_ooov[k, i, l]
                if k == i:
                    # + sum_c ur[i,l,a,c] F~ov[l,c]
                    s += ur @ self.Fov[l]
        # singles-singles: sum_m Acan[i,:,m,:] r_m with
        # Acan[i,a,m,d] = sum_{k,c} u[i,k,a,c] L[k,c,m,d] + 2 (ai|md) - (mi|ad) + delta_im Xv - delta_ad Xo[m,i]
        rr = np.array(r1)                                             # [m, d]
        Lr = 2.0 * e("kcmd,md->kc", g, rr) - e("kdmc,md->kc", g, rr)
        s += e("kac,kc->a", u[i], Lr)
        s += 2.0 * e("Qa,Qmd,md->a", self.Bvo[:, :, i], self.Bov, rr)
        s -= e("Qm,Qad,md->a", self.Boo[:, :, i], self.Bvv, rr)
        s += self.Xv @ r1[i]
        s -= e("m,ma->a", self.Xo[:, i], rr)
        return s
