"""Pins of the EOM-CCSD sigma oracle."""
import numpy as np
import pytest

from synthetic import make_system
from oracle import bruteforce as bf, ccsd, eom, hamiltonian as hm


def _sym(x):
    return 0.5 * (x + x.transpose(1, 0, 3, 2))


def _sys(o, v, naux, seed):
    s = make_system(o, v, naux, seed)
    eps, B = s["eps"], s["B"]
    h = hm.hcore_from_fock(eps, B, o)
    ds = bf.DetSpace(o + v, o)
    return eps, B, h, ds, ds.hamiltonian(h, B)


@pytest.mark.parametrize("o,v,naux", [(2, 4, 12), (3, 5, 16)])
@pytest.mark.parametrize("scale", [0.0, 0.3])
def test_sigma_equals_projected_commutator(o, v, naux, scale):
    eps, B, h, ds, H = _sys(o, v, naux, 31)
    rng = np.random.default_rng(9)
    t1 = scale * rng.standard_normal((o, v))
    t2 = _sym(scale * rng.standard_normal((o, o, v, v)))
    r1 = rng.standard_normal((o, v))
    r2 = _sym(rng.standard_normal((o, o, v, v)))
    ref = bf.eom_sigma_state(ds, H, t1, t2, r1, r2)
    s1, s2 = eom.Sigma(t1, t2, h, B, o)(r1, r2)
    j1, j2 = eom.sigma_jvp(t1, t2, r1, r2, h, B, o)
    tol = 1e-12 * max(1.0, np.abs(ref).max())
    assert np.abs(bf.amplitudes_state(ds, s1, s2) - ref).max() < tol
    assert np.abs(bf.amplitudes_state(ds, j1, j2) - ref).max() < tol


def _sigma_matrix(S, o, v):
    """Dense matrix of sigma on the symmetric amplitude space."""
    idx2 = [(i, j, a, b) for i in range(o) for j in range(o) for a in range(v) for b in range(v)
            if (i, a) <= (j, b)]
    cols = []
    for i in range(o):
        for a in range(v):
            r1 = np.zeros((o, v)); r1[i, a] = 1.0
            cols.append((r1, np.zeros((o, o, v, v))))
    for (i, j, a, b) in idx2:
        r2 = np.zeros((o, o, v, v)); r2[i, j, a, b] = 1.0; r2[j, i, b, a] = 1.0
        cols.append((np.zeros((o, v)), r2))
    M = []
    for r1, r2 in cols:
        s1, s2 = S(r1, r2)
        M.append(np.concatenate([s1.ravel(), [s2[i, j, a, b] for (i, j, a, b) in idx2]]))
    return np.array(M).T


def test_t_zero_spectrum_is_cisd():
    o, v, naux = 2, 3, 10
    eps, B, h, ds, H = _sys(o, v, naux, 32)
    S = eom.Sigma(np.zeros((o, v)), np.zeros((o, o, v, v)), h, B, o)
    ev = np.sort(np.linalg.eigvals(_sigma_matrix(S, o, v)).real)
    ref = bf.cisd_excitation_energies(ds, H)
    assert len(ev) == len(ref)
    assert np.abs(ev - ref).max() < 1e-11


def test_two_electron_eom_is_fci():
    o, v, naux = 1, 4, 12
    eps, B, h, ds, H = _sys(o, v, naux, 33)
    t1, t2, ecc, err = ccsd.solve_ccsd(eps, B, o, tol=1e-13)
    S = eom.Sigma(t1, t2, h, B, o)
    ev = np.sort(np.linalg.eigvals(_sigma_matrix(S, o, v)).real)
    fci = bf.fci_singlet_energies(ds, H)
    assert np.abs(ev - (fci[1:] - fci[0])).max() < 1e-9


def test_sigma_linearity():
    o, v, naux = 3, 6, 18
    s = make_system(o, v, naux, 34)
    h = hm.hcore_from_fock(s["eps"], s["B"], o)
    rng = np.random.default_rng(3)
    t1 = 0.05 * rng.standard_normal((o, v)); t2 = _sym(0.05 * rng.standard_normal((o, o, v, v)))
    S = eom.Sigma(t1, t2, h, s["B"], o)
    x = [(rng.standard_normal((o, v)), _sym(rng.standard_normal((o, o, v, v)))) for _ in range(2)]
    a, b = 0.7, -1.3
    lhs = S(a * x[0][0] + b * x[1][0], a * x[0][1] + b * x[1][1])
    s0, s1 = S(*x[0]), S(*x[1])
    assert np.allclose(lhs[0], a * s0[0] + b * s1[0], atol=1e-12)
    assert np.allclose(lhs[1], a * s0[1] + b * s1[1], atol=1e-12)
