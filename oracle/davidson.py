"""Non-symmetric Davidson solver with the PNO-space preconditioner (oracle).

Follows the paper's PNO-EOM-CCSD Davidson (Sec. 2): residuals of the current
Ritz pairs are formed in PNO/OSV coordinates, divided by
omega_k + f_ii (+ f_jj) - fbar_a (- fbar_b) in the semicanonical bases, and
added to the subspace.  Because every vector is kept in PNO coordinates, the
back-transform of the paper's step 3 is implicit.  Readings where the paper
is silent: guesses are the projected CIS vectors (R2 = 0); the residual is
r = sigma - omega x; denominators smaller than 1e-4 Eh in magnitude are
clamped to +-1e-4; Gram-Schmidt is applied twice; the diagonal-pair blocks of each new
vector are symmetrised (R^{ii} is symmetric by definition); the subspace collapses to
the current Ritz vectors when it would exceed ``max_subspace``; Ritz values
are sorted by real part and complex pairs contribute their real parts.
"""
from __future__ import annotations

import numpy as np

CLAMP = 1e-4


def _orth(V, t):
    for _ in range(2):
        t = t - V.T @ (V @ t)
    return t


def davidson(matvec, denom, guesses, nroots, res_tol=1e-7, e_tol=1e-10,
             max_iter=100, max_subspace=None, symmetrize=None):
    """Lowest ``nroots`` eigenpairs of the linear map ``matvec``.

    ``denom(omega)`` returns the packed preconditioner denominators;
    ``guesses`` is float64[k, n].  Returns (omega[nroots], X[nroots, n],
    residual norms, iterations, converged)."""
    if max_subspace is None:
        max_subspace = max(8 * nroots, 2 * guesses.shape[0])
    V = []
    for g in guesses:
        t = g.copy()
        if V:
            t = _orth(np.array(V), t)
        nrm = np.linalg.norm(t)
        if nrm > 1e-10:
            V.append(t / nrm)
    V = np.array(V)
    nroots = min(nroots, V.shape[0])
    S = np.array([matvec(x) for x in V])
    w_old = None
    for it in range(1, max_iter + 1):
        G = V @ S.T                  # G[m, n] = <v_m | sigma(v_n)>
        w, Y = np.linalg.eig(G)
        order = np.argsort(w.real)
        w, Y = w[order][:nroots], Y[:, order][:, :nroots]
        w, Y = w.real, Y.real
        X = Y.T @ V
        R = Y.T @ S - w[:, None] * X
        rn = np.linalg.norm(R, axis=1)
        dw = np.inf if w_old is None else np.max(np.abs(w - w_old))
        w_old = w.copy()
        if np.all(rn < res_tol) and dw < e_tol:
            nrm = np.linalg.norm(X, axis=1)
            return w, X / nrm[:, None], rn, it, True
        new = []
        for k in range(nroots):
            if rn[k] < res_tol:
                continue
            d = denom(w[k])
            d = np.where(np.abs(d) < CLAMP, np.where(d < 0, -CLAMP, CLAMP), d)
            t = R[k] / d
            new.append(t if symmetrize is None else symmetrize(t))
        if V.shape[0] + len(new) > max_subspace:
            Xq, _ = np.linalg.qr(X.T)
            V = Xq.T
            S = np.array([matvec(x) for x in V])
        added = []
        for t in new:
            base = np.vstack([V] + added) if added else V
            t = _orth(base, t)
            nrm = np.linalg.norm(t)
            if nrm > 1e-8:
                added.append((t / nrm)[None, :])
        if not added:
            nrm = np.linalg.norm(X, axis=1)
            return w, X / nrm[:, None], rn, it, bool(np.all(rn < res_tol))
        A = np.vstack(added)
        V = np.vstack([V, A])
        S = np.vstack([S, np.array([matvec(x) for x in A])])
    nrm = np.linalg.norm(X, axis=1)
    return w, X / nrm[:, None], rn, max_iter, False


def solve(sigma_pno, space, nroots, guesses_b=None, **kw):
    """PNO-EOM-CCSD roots from projected CIS guesses."""
    if guesses_b is None:
        guesses_b = space.cis_b
    o, v = space.o, space.v
    G = np.array([space.pack(b, np.zeros((o, o, v, v))) for b in guesses_b[:nroots]])
    return davidson(sigma_pno, space.denominators, G, nroots, symmetrize=space.symmetrize, **kw)
