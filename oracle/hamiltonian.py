"""Integrals and one-electron operators from density-fitting factors (oracle).

Conventions: orbitals p = 0..o-1 occupied, o..o+v-1 virtual; Mulliken
two-electron integrals (pq|rs) = sum_Q B[Q,p,q] B[Q,r,s], the density-fitting
form the paper uses for all calculations (Sec. 3).
"""
from __future__ import annotations

import numpy as np


def eri(B):
    """Full (pq|rs) tensor [p,q,r,s] from DF factors (small systems only)."""
    return np.einsum("Qpq,Qrs->pqrs", B, B, optimize=True)


def hcore_from_fock(eps, B, o):
    """One-electron operator h that makes diag(eps) the HF Fock matrix.

    f_pq = h_pq + sum_i [2 (pq|ii) - (pi|iq)]  (closed-shell Fock operator), so
    h = diag(eps) - sum_i [2 (pq|ii) - (pi|iq)].  With this h the synthetic
    system is a genuine Hamiltonian whose HF determinant is stationary.
    """
    J = np.einsum("Qpq,Qii->pq", B, B[:, :o, :o], optimize=True)
    K = np.einsum("Qpi,Qiq->pq", B[:, :, :o], B[:, :o, :], optimize=True)
    return np.diag(eps) - 2.0 * J + K


def fock(h, B, o):
    """Closed-shell Fock matrix of a (possibly non-symmetric) Hamiltonian given
    by one-electron h and DF factors B: F = h + 2 J - K over occupied k."""
    J = np.einsum("Qpq,Qkk->pq", B, B[:, :o, :o], optimize=True)
    K = np.einsum("Qpk,Qkq->pq", B[:, :, :o], B[:, :o, :], optimize=True)
    return h + 2.0 * J - K


def t1_kappa(t1, o, nmo):
    """Matrix kappa of the operator T1 = sum_ai t1[i,a] E_ai: kappa[a,i] = t1[i,a]."""
    kappa = np.zeros((nmo, nmo), dtype=np.result_type(t1, float))
    kappa[o:, :o] = t1.T
    return kappa


def dress(h, B, t1, o):
    """T1-similarity-transformed Hamiltonian exp(-T1) H exp(T1).

    A one-body excitation operator kappa (kappa^2 = 0) transforms every
    orbital operator linearly, so the transformed one- and two-electron
    integrals are h~ = (1 - kappa) h (1 + kappa) and B~^Q = (1 - kappa) B^Q
    (1 + kappa).  In this frame the CCSD equations contain T2 only.
    """
    nmo = h.shape[0]
    kappa = t1_kappa(t1, o, nmo)
    X = np.eye(nmo) - kappa
    Y = np.eye(nmo) + kappa
    hd = X @ h @ Y
    Bd = np.einsum("pr,Qrs,sq->Qpq", X, B, Y, optimize=True)
    return hd, Bd


def commutator_r1(h, B, r1, o):
    """Integrals of [H, R1] for R1 = sum_ai r1[i,a] E_ai.

    [sum h_pq E_pq, sum rho_rs E_rs] = sum (h rho - rho h)_pq E_pq, and the
    same rule applies to each DF factor, so the derivative of the T1 dressing
    in the direction R1 is h' = h rho - rho h, B'^Q = B^Q rho - rho B^Q (with
    rho[a,i] = r1[i,a]); the two-electron integrals of [H, R1] are
    sum_Q (B'^Q_pq B^Q_rs + B^Q_pq B'^Q_rs).
    """
    nmo = h.shape[0]
    rho = t1_kappa(r1, o, nmo)
    hp = h @ rho - rho @ h
    Bp = np.einsum("Qpr,rq->Qpq", B, rho, optimize=True) - np.einsum("pr,Qrq->Qpq", rho, B, optimize=True)
    return hp, Bp
