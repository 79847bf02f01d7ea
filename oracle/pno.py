"""CIS, CIS(D) pair densities, state-averaged PNOs/OSVs and the PNO-space
sigma (oracle).

Paper passages followed:
* CIS singles amplitudes B^i_a(k) and energies omega_k (Sec. 2, the CIS(D)
  paragraph); singlet CIS matrix A_{ia,jb} = delta_ij delta_ab (f_aa - f_ii)
  + 2 (ia|jb) - (ij|ab), amplitudes normalised so that R1|0> is a unit
  vector, i.e. 2 sum_ia (b^i_a)^2 = 1.
* CIS(D) doubles (Eq. cis_d): B^{ij}_{ab(k)} = K^{ij}_{ab(k)} /
  (omega_k + f_ii + f_jj - f_aa - f_bb), K = b^i_c (ac|bj) + b^j_c (ai|bc)
  - b^l_a (li|bj) - b^l_b (ai|lj) (G^{pq}_{rs} read as (rp|sq)).  A
  denominator of magnitude below 1e-4 Eh is replaced by +-1e-4 Eh.
* pair density D^{ij}_(k) = 2/(1+delta_ij) (B B~^T + B^T B~), B~ = 2B - B^T,
  and its state average D^{ij} = (1/N) sum_k D^{ij}_(k) (Eq. eom:sa_density);
  the one-state density D^{ij}_(k) alone gives the state-specific PNOs that the
  average replaces (Sec. 2).
* ground-state PNOs: the same density form built from the amplitudes T^{ij}
  (Methods, D_(0)); truncation projects each T^{ij} onto the kept ones.
* PNOs: eigenvectors of D^{ij} with occupation >= T_CutPNO (all of them when
  T_CutPNO = 0); OSVs of occupied i: the same for D^{ii} at T_CutOSV =
  T_CutPNO / 10 (Sec. 3); both semicanonicalised by diagonalising the
  virtual Fock block inside the kept space (Sec. 2, PNO-CCSD simulation).
* The simulation's projection (Sec. 2, PNO-EOM-CCSD Davidson): R^i ->
  U^i U^i^T R^i and R^{ij} -> U^{ij} U^{ij}^T R^{ij} U^{ij} U^{ij}^T; in PNO
  coordinates R^i_bar = U^i^T R^i, R^{ij}_bar = U^{ij}^T R^{ij} U^{ij}.

Sign convention (shared with the library by specification): every kept
semicanonical PNO/OSV vector is flipped so that its entry of largest
magnitude (the first one, on ties) is positive.  Packed vector layout:
[R1: i = 0..o-1, n_i entries each][R2: pairs i <= j in lexicographic order,
n_ij x n_ij row-major with the row index on i].
"""
from __future__ import annotations

import numpy as np

from . import ccsd

DENOM_CLAMP = 1e-4


# Row block of the large matrix products below: the products are formed a block of
# rows at a time (the same sums, in the same order per element), which keeps every
# single BLAS call to a moderate size.
ROW_BLOCK = 3600


def _rows_matmul(X, Y):
    """X @ Y, computed a block of rows of X at a time."""
    out = np.empty((X.shape[0], Y.shape[1]))
    for r0 in range(0, X.shape[0], ROW_BLOCK):
        out[r0:r0 + ROW_BLOCK] = X[r0:r0 + ROW_BLOCK] @ Y
    return out


def cis_matrix(eps, B, o):
    v = len(eps) - o
    nq = B.shape[0]
    Bov = np.ascontiguousarray(B[:, :o, o:]).reshape(nq, o * v)
    A = 2.0 * _rows_matmul(Bov.T, Bov)                       # 2 (ia|jb)
    Boo = np.ascontiguousarray(B[:, :o, :o]).reshape(nq, o * o)
    Bvv = np.ascontiguousarray(B[:, o:, o:]).reshape(nq, v * v)
    A4 = A.reshape(o, v, o, v)
    for i in range(o):                                       # - (ij|ab)
        A4[i] -= (Boo[:, i * o:(i + 1) * o].T @ Bvv).reshape(o, v, v).transpose(1, 0, 2)
    d = (eps[o:][None, :] - eps[:o][:, None])
    A[np.diag_indices_from(A)] += d.ravel()
    return A


# Above this many singles the lowest roots are found by an iterative symmetric
# eigensolver (ARPACK through SciPy) instead of a full dense diagonalisation.
CIS_DENSE_MAX = 6000


def cis(eps, B, o, nroots):
    """Lowest ``nroots`` singlet CIS roots: (omega[k], b[k,i,a]),
    2 sum b^2 = 1, sign fixed by a positive largest-magnitude entry."""
    v = len(eps) - o
    A = cis_matrix(eps, B, o)
    A = 0.5 * (A + A.T)
    if o * v <= CIS_DENSE_MAX:
        w, X = np.linalg.eigh(A)
    else:
        import scipy.sparse.linalg as sla
        w, X = sla.eigsh(A, k=nroots, which="SA", tol=1e-14)
        order = np.argsort(w)
        w, X = w[order], X[:, order]
    w, X = w[:nroots], X[:, :nroots].T.copy()
    for k in range(nroots):
        m = np.argmax(np.abs(X[k]))
        if X[k, m] < 0:
            X[k] = -X[k]
    X /= np.sqrt(2.0)
    return w, X.reshape(nroots, o, v)


def _clamp(d):
    small = np.abs(d) < DENOM_CLAMP
    return np.where(small, np.where(d < 0, -DENOM_CLAMP, DENOM_CLAMP), d)


def cisd_doubles(eps, B, o, omega, b):
    """CIS(D) doubles B^{ij}_{ab}[i,j,a,b] for one CIS root (Eq. cis_d)."""
    e = np.einsum
    v = len(eps) - o
    nq = B.shape[0]
    Bvv, Bvo, Boo = B[:, o:, o:], B[:, o:, :o], B[:, :o, :o]
    # sum_c b[i,c] (ac|bj) - sum_l b[l,a] (li|bj) = sum_Q Z[Q,i,a] B[Q,b,j] with
    # Z[Q,i,a] = sum_c b[i,c] B[Q,a,c] - sum_l b[l,a] B[Q,l,i]; the other two terms of K
    # are the same with (i,a) and (j,b) exchanged, using B[Q,a,i] on the left
    Z = e("ic,Qac->Qia", b, Bvv, optimize=True) - e("la,Qli->Qia", b, Boo, optimize=True)
    Zm = np.ascontiguousarray(Z).reshape(nq, o * v)
    Bm = np.ascontiguousarray(Bvo.transpose(0, 2, 1)).reshape(nq, o * v)      # [Q, j, b] = B[Q,b,j]
    K = _rows_matmul(Zm.T, Bm).reshape(o, v, o, v).transpose(0, 2, 1, 3)       # [i,j,a,b]
    Bl = np.ascontiguousarray(Bvo.transpose(0, 2, 1)).reshape(nq, o * v)      # [Q, i, a] = B[Q,a,i]
    K = K + _rows_matmul(Bl.T, Zm).reshape(o, v, o, v).transpose(0, 2, 1, 3)
    eo, ev = eps[:o], eps[o:]
    K = np.ascontiguousarray(K)
    for i in range(o):        # one occupied index at a time (memory)
        d = omega + eo[i] + eo[:, None, None] - ev[None, :, None] - ev[None, None, :]
        K[i] /= _clamp(d)
    return K


def pair_density(Bij, i, j):
    """D^{ij} = 2/(1+delta_ij) (B B~^T + B^T B~) with B~ = 2B - B^T."""
    Bt = 2.0 * Bij - Bij.T
    return (2.0 / (1.0 + (i == j))) * (Bij @ Bt.T + Bij.T @ Bt)


def sa_densities(eps, B, o, nroots, omegas=None, bs=None):
    """State-averaged densities D[i,j] (dict over i <= j) plus CIS data."""
    if omegas is None:
        omegas, bs = cis(eps, B, o, nroots)
    D = {}
    for k in range(nroots):
        Bd = cisd_doubles(eps, B, o, omegas[k], bs[k])
        for i in range(o):
            for j in range(i, o):
                Dk = pair_density(Bd[i, j], i, j)
                D[i, j] = D.get((i, j), 0.0) + Dk / nroots
    return D, omegas, bs


def _truncate_semicanonical(Dm, thresh, fvv):
    n, U = np.linalg.eigh(Dm)
    keep = np.ones(len(n), bool) if thresh == 0.0 else (n >= thresh)
    occ = n[keep]
    U = U[:, keep]
    if U.shape[1] == 0:
        return U, np.zeros(0), occ, n
    fbar, Z = np.linalg.eigh(U.T @ fvv @ U)
    U = U @ Z
    for c in range(U.shape[1]):
        m = np.argmax(np.abs(U[:, c]))
        if U[m, c] < 0:
            U[:, c] = -U[:, c]
    return U, fbar, occ, n


def gs_truncate_t2(t2, o, t_gs):
    """Ground-state PNO truncation of T2 (Methods): for each pair i <= j the ground-state
    pair density D_(0)^{ij} = 2/(1+delta_ij) (T T~^T + T^T T~), T~ = 2T - T^T, is
    diagonalised; P^{ij} projects onto its eigenvectors with occupation >= t_gs (all of
    them when t_gs = 0), and T^{ij} -> P T^{ij} P, T^{ji} -> P T^{ji} P."""
    out = np.array(t2, copy=True)
    for i in range(o):
        for j in range(i, o):
            D = pair_density(t2[i, j], i, j)
            w, U = np.linalg.eigh(D)
            Uk = U if t_gs == 0 else U[:, w >= t_gs]
            P = Uk @ Uk.T
            out[i, j] = P @ t2[i, j] @ P
            if i != j:
                out[j, i] = P @ t2[j, i] @ P
    return out


def ss_densities(eps, B, o, root, nroots, omegas=None, bs=None):
    """State-specific densities (Methods: the PNOs of one state, the construction the
    state average replaces): D[i,j] from the CIS(D) doubles of CIS root `root` alone
    (0-based, among the lowest `nroots`), with weight 1."""
    if omegas is None:
        omegas, bs = cis(eps, B, o, nroots)
    Bd = cisd_doubles(eps, B, o, omegas[root], bs[root])
    D = {}
    for i in range(o):
        for j in range(i, o):
            D[i, j] = pair_density(Bd[i, j], i, j)
    return D, omegas, bs


class PNOSpace:
    """PNO/OSV bases of one system and the packed-vector maps."""

    def __init__(self, eps, B, o, nroots, t_pno, t_osv=None, D=None, cis=None):
        """D: pair densities (default: the state average of the lowest nroots); cis:
        (omegas, vectors) of the CIS roots that seed the Davidson guesses when D is given."""
        self.o = o
        self.v = len(eps) - o
        self.eps = eps
        if t_osv is None or t_osv < 0:
            t_osv = t_pno / 10.0
        if D is None:
            D, self.cis_omega, self.cis_b = sa_densities(eps, B, o, nroots)
        elif cis is not None:
            self.cis_omega, self.cis_b = cis
        self.D = D
        fvv = np.diag(eps[o:])
        self.U, self.fbar, self.occ, self.alleig = {}, {}, {}, {}
        for i in range(o):
            for j in range(i, o):
                U, fb, oc, n = _truncate_semicanonical(D[i, j], t_pno, fvv)
                self.U[i, j], self.fbar[i, j], self.occ[i, j], self.alleig[i, j] = U, fb, oc, n
        self.Ui, self.fbar_i = {}, {}
        for i in range(o):
            U, fb, _, _ = _truncate_semicanonical(D[i, i], t_osv, fvv)
            self.Ui[i], self.fbar_i[i] = U, fb
        self.pairs = [(i, j) for i in range(o) for j in range(i, o)]
        self.n_i = np.array([self.Ui[i].shape[1] for i in range(o)])
        self.n_ij = np.array([self.U[p].shape[1] for p in self.pairs])
        self.off_i = np.concatenate([[0], np.cumsum(self.n_i)])
        base = self.off_i[-1]
        self.off_ij = base + np.concatenate([[0], np.cumsum(self.n_ij ** 2)])
        self.length = int(self.off_ij[-1])

    # -- packed layout --------------------------------------------------
    def pack(self, r1, r2):
        """Project canonical (r1[i,a], r2[i,j,a,b]) into the packed vector."""
        out = np.zeros(self.length)
        for i in range(self.o):
            out[self.off_i[i]:self.off_i[i + 1]] = self.Ui[i].T @ r1[i]
        for p, (i, j) in enumerate(self.pairs):
            U = self.U[i, j]
            out[self.off_ij[p]:self.off_ij[p + 1]] = (U.T @ r2[i, j] @ U).ravel()
        return out

    def block(self, vec, p):
        n = self.n_ij[p]
        return vec[self.off_ij[p]:self.off_ij[p + 1]].reshape(n, n)

    def unpack(self, vec):
        """Back-transform the packed vector to canonical r1, r2."""
        o, v = self.o, self.v
        r1 = np.zeros((o, v))
        r2 = np.zeros((o, o, v, v))
        for i in range(o):
            r1[i] = self.Ui[i] @ vec[self.off_i[i]:self.off_i[i + 1]]
        for p, (i, j) in enumerate(self.pairs):
            U = self.U[i, j]
            R = U @ self.block(vec, p) @ U.T
            r2[i, j] = R
            r2[j, i] = R.T
        return r1, r2

    def project(self, r1, r2):
        """Canonical P(R): the simulation's projector."""
        return self.unpack(self.pack(r1, r2))

    def symmetrize(self, vec):
        """Make the diagonal-pair blocks symmetric (R^{ii} is symmetric by
        definition; keeps trial vectors inside the valid amplitude space)."""
        out = vec.copy()
        for p, (i, j) in enumerate(self.pairs):
            if i == j:
                Bk = self.block(out, p)
                out[self.off_ij[p]:self.off_ij[p + 1]] = (0.5 * (Bk + Bk.T)).ravel()
        return out

    def valid_basis(self):
        """Orthonormal basis (columns) of the packed vectors with symmetric
        diagonal-pair blocks."""
        cols = []
        n0 = self.off_ij[0]
        for k in range(n0):
            e = np.zeros(self.length); e[k] = 1.0; cols.append(e)
        for p, (i, j) in enumerate(self.pairs):
            n = self.n_ij[p]
            for a in range(n):
                for b in range(n if i != j else a + 1):
                    e = np.zeros(self.length)
                    if i != j or a == b:
                        e[self.off_ij[p] + a * n + b] = 1.0
                    else:
                        e[self.off_ij[p] + a * n + b] = e[self.off_ij[p] + b * n + a] = np.sqrt(0.5)
                    cols.append(e)
        return np.array(cols).T

    def denominators(self, omega):
        """omega + f_ii - fbar_a (singles), omega + f_ii + f_jj - fbar_a - fbar_b
        (doubles), in packed layout (Sec. 2 preconditioner)."""
        eo = self.eps[:self.o]
        out = np.zeros(self.length)
        for i in range(self.o):
            out[self.off_i[i]:self.off_i[i + 1]] = omega + eo[i] - self.fbar_i[i]
        for p, (i, j) in enumerate(self.pairs):
            fb = self.fbar[i, j]
            out[self.off_ij[p]:self.off_ij[p + 1]] = (omega + eo[i] + eo[j] - fb[:, None] - fb[None, :]).ravel()
        return out


class PNOSigma:
    """sigma in PNO coordinates: U^T sigma(U R_bar U^T) U per block.

    The ladder contraction sum_cd r^{cd}_{ij} (ac|bd) applied to R2 is taken
    in the pair's own PNO basis, sum_Q Bbar^Q R_bar Bbar^Q^T with
    Bbar^Q = U^{ij}^T B~^Q_vv U^{ij}, which equals the projected canonical
    term exactly; every other term is the canonical expression followed by the
    projection."""

    def __init__(self, sig, space):
        self.sig, self.space = sig, space
        o = space.o
        Bvv = sig.Bd[:, o:, o:]
        self.Bbar = [np.einsum("ca,Qcd,db->Qab", space.U[p], Bvv, space.U[p], optimize=True)
                     for p in space.pairs]

    def __call__(self, vec):
        sp_ = self.space
        r1, r2 = sp_.unpack(vec)
        zero = lambda x: 0.0
        a1, a2, _ = self.sig.r2_part(r2, ladder_r2=zero)
        b1, b2 = self.sig.r1_part(r1)
        out = sp_.pack(a1 + b1, a2 + b2)
        for p in range(len(sp_.pairs)):
            Rb = sp_.block(vec, p)
            Bb = self.Bbar[p]
            lad = np.einsum("Qac,cd,Qbd->ab", Bb, Rb, Bb, optimize=True)
            out[sp_.off_ij[p]:sp_.off_ij[p + 1]] += lad.ravel()
        return out
