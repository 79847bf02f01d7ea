"""Pins of the CCSD oracle against brute force and textbook identities."""
import numpy as np
import pytest

from synthetic import make_system
from oracle import bruteforce as bf, ccsd, hamiltonian as hm


def _sys(o, v, naux, seed):
    s = make_system(o, v, naux, seed)
    eps, B = s["eps"], s["B"]
    h = hm.hcore_from_fock(eps, B, o)
    ds = bf.DetSpace(o + v, o)
    return eps, B, h, ds, ds.hamiltonian(h, B)


def _sym(x):
    return 0.5 * (x + x.transpose(1, 0, 3, 2))


def test_generator_recipe():
    s = make_system(3, 7, 11, 5)
    assert s["B"].shape == (11, 10, 10)
    assert np.allclose(s["B"], s["B"].transpose(0, 2, 1))
    assert np.all(np.diff(s["eps"][:3]) >= 0) and np.all(np.diff(s["eps"][3:]) >= 0)
    assert s["eps"][:3].max() <= -0.3 and s["eps"][3:].min() >= 0.1
    s2 = make_system(3, 7, 11, 5)
    assert np.array_equal(s["B"], s2["B"])


def test_hf_fock_is_diagonal_and_stationary():
    eps, B, h, ds, H = _sys(2, 4, 12, 3)
    assert np.allclose(hm.fock(h, B, 2), np.diag(eps), atol=1e-15)
    # Brillouin: <S|H|0> = 0 for the HF determinant
    hv = H @ ds.reference()
    assert np.abs(hv[ds.level == 1]).max() < 1e-13


@pytest.mark.parametrize("o,v,naux", [(2, 4, 12), (3, 5, 16)])
@pytest.mark.parametrize("scale", [0.0, 0.1, 0.6])
def test_residual_equals_projected_hbar(o, v, naux, scale):
    eps, B, h, ds, H = _sys(o, v, naux, 21)
    rng = np.random.default_rng(7)
    t1 = scale * rng.standard_normal((o, v))
    t2 = _sym(scale * rng.standard_normal((o, o, v, v)))
    r1, r2 = ccsd.residual(t1, t2, h, B, o)
    ref = bf.cc_residual_state(ds, H, t1, t2)
    got = bf.amplitudes_state(ds, r1, r2)
    assert np.abs(ref - got).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_residual_detects_dropped_term():
    """A planted mistake (sign flip of the exchange ring) must fail the pin."""
    o, v, naux = 2, 4, 12
    eps, B, h, ds, H = _sys(o, v, naux, 22)
    rng = np.random.default_rng(8)
    t1 = 0.1 * rng.standard_normal((o, v))
    t2 = _sym(0.3 * rng.standard_normal((o, o, v, v)))
    ref = bf.cc_residual_state(ds, H, t1, t2)
    hd, Bd = hm.dress(h, B, t1, o)
    Hd = ccsd.make_ham(hd, Bd, o)
    orig = Hd.g

    def g_bad(spec):
        blk = orig(spec)
        return -blk if spec == "oovv" else blk
    Hd.g = g_bad
    r1, r2 = ccsd.omega(t2, Hd)
    assert np.abs(bf.amplitudes_state(ds, r1, r2) - ref).max() > 1e-3


def test_mp2_energy_equals_second_order_perturbation_theory():
    """E_MP2 = sum t (2(ia|jb) - (ib|ja)) equals Rayleigh-Schroedinger PT2
    with H0 = sum_p eps_p n_p, evaluated over determinants."""
    o, v, naux = 2, 4, 12
    eps, B, h, ds, H = _sys(o, v, naux, 23)
    t2 = ccsd.mp1_t2(eps, B, o)
    e_mp2 = ccsd.energy(np.zeros((o, v)), t2, eps, B, o)
    e0 = ds.reference()
    hv = H @ e0
    e2 = 0.0
    occ0 = sum(eps[:o]) * 2
    for k in np.nonzero(ds.level == 2)[0]:
        ia, ib = divmod(k, ds.nstr)
        sa, sb = ds.strings[ia], ds.strings[ib]
        ek = sum(eps[p] for p in range(o + v) if (sa >> p) & 1) + sum(eps[p] for p in range(o + v) if (sb >> p) & 1)
        e2 += hv[k] ** 2 / (occ0 - ek)
    assert abs(e_mp2 - e2) < 1e-14 + 1e-10 * abs(e2)


def test_ccsd_two_electrons_is_fci():
    o, v, naux = 1, 5, 14
    eps, B, h, ds, H = _sys(o, v, naux, 24)
    t1, t2, ecc, err = ccsd.solve_ccsd(eps, B, o, tol=1e-12)
    assert err < 1e-11
    e0 = ds.reference()
    ehf = e0 @ (H @ e0)
    efci = bf.fci_singlet_energies(ds, H)[0]
    assert abs(ehf + ecc - efci) < 1e-10


def test_ccsd_converged_residual_zero():
    s = make_system(5, 20, 60, 1)
    t1, t2, ecc, err = ccsd.solve_ccsd(s["eps"], s["B"], 5)
    assert err < 1e-10 and ecc < 0.0
