"""Pins of the CIS / CIS(D) / PNO / Davidson oracle."""
import numpy as np
import pytest

from synthetic import make_system
from oracle import bruteforce as bf, ccsd, davidson, eom, hamiltonian as hm, pno


def _small(o=3, v=6, naux=18, seed=41):
    s = make_system(o, v, naux, seed)
    return s["eps"], s["B"], hm.hcore_from_fock(s["eps"], s["B"], o)


def test_cis_is_singles_block_of_brute_force():
    o, v, naux = 2, 4, 12
    eps, B, h = _small(o, v, naux, 42)
    ds = bf.DetSpace(o + v, o)
    H = ds.hamiltonian(h, B)
    e0 = ds.reference()
    ehf = e0 @ (H @ e0)
    cols = [ds.E(o + a, i) @ e0 for i in range(o) for a in range(v)]
    Qs, _ = np.linalg.qr(np.array(cols).T)
    ref = np.sort(np.linalg.eigvalsh(Qs.T @ (H @ Qs))) - ehf
    w, b = pno.cis(eps, B, o, o * v)
    assert np.abs(np.sort(w) - ref).max() < 1e-12
    # normalisation: R1|0> is a unit vector <=> 2 sum b^2 = 1
    for k in range(o * v):
        vec = bf.amplitudes_state(ds, b[k], None)
        assert abs(np.linalg.norm(vec) - 1.0) < 1e-12


def test_cisd_K_is_doubles_projection_of_H_R1():
    """K^{ij}_{ab} of Eq. cis_d is the biorthogonal doubles projection of
    [H, R1]|0> (the doubles of H R1|0>, since <S|H|0> = 0 for HF)."""
    o, v, naux = 2, 4, 12
    eps, B, h = _small(o, v, naux, 43)
    ds = bf.DetSpace(o + v, o)
    H = ds.hamiltonian(h, B)
    rng = np.random.default_rng(5)
    b = rng.standard_normal((o, v))
    omega = 0.37
    Bd = pno.cisd_doubles(eps, B, o, omega, b)
    eo, ev = eps[:o], eps[o:]
    den = omega + eo[:, None, None, None] + eo[None, :, None, None] - ev[None, None, :, None] - ev[None, None, None, :]
    K = Bd * den
    vec = H @ bf.amplitudes_state(ds, b, None)
    vec[ds.level != 2] = 0.0
    got = bf.amplitudes_state(ds, np.zeros((o, v)), K)
    assert np.abs(got - vec).max() < 1e-13
    assert np.allclose(K, K.transpose(1, 0, 3, 2))   # K^{ji}_{ba} = K^{ij}_{ab}


def test_pair_density_invariants():
    eps, B, h = _small()
    o = 3
    D, w, b = pno.sa_densities(eps, B, o, 3)
    Bd = pno.cisd_doubles(eps, B, o, w[0], b[0])
    for i in range(o):
        for j in range(i, o):
            Dm = D[i, j]
            assert np.allclose(Dm, Dm.T, atol=1e-15)
            n = np.linalg.eigvalsh(Dm)
            assert n.min() > -1e-14 * max(1e-30, np.trace(Dm))
            assert abs(n.sum() - np.trace(Dm)) < 1e-13 * abs(np.trace(Dm)) + 1e-30
            # closed form: with B = S + A, B B~^T + B^T B~ = 2 S^2 + 6 A A^T
            X = Bd[i, j]
            Ss, As = 0.5 * (X + X.T), 0.5 * (X - X.T)
            ref = (2.0 / (1 + (i == j))) * (2 * Ss @ Ss + 6 * As @ As.T)
            assert np.allclose(pno.pair_density(X, i, j), ref, atol=1e-14 * max(1e-30, np.abs(ref).max()))
            # D^{ji} = D^{ij}
            assert np.allclose(pno.pair_density(Bd[j, i], j, i), pno.pair_density(X, i, j), atol=1e-18)


def _setup(o, v, naux, seed, tp, nroots=3, t1scale=None):
    s = make_system(o, v, naux, seed)
    eps, B = s["eps"], s["B"]
    h = hm.hcore_from_fock(eps, B, o)
    t1, t2, _, _ = ccsd.solve_ccsd(eps, B, o)
    sig = eom.Sigma(t1, t2, h, B, o)
    sp = pno.PNOSpace(eps, B, o, nroots, tp)
    return sig, sp


def test_projector_idempotent_and_pno_sigma_equals_projected_canonical():
    sig, sp = _setup(3, 8, 24, 44, 1e-6)
    o, v = 3, 8
    rng = np.random.default_rng(11)
    r1 = rng.standard_normal((o, v))
    r2 = rng.standard_normal((o, o, v, v)); r2 = 0.5 * (r2 + r2.transpose(1, 0, 3, 2))
    p1, p2 = sp.project(r1, r2)
    q1, q2 = sp.project(p1, p2)
    assert np.allclose(p1, q1, atol=1e-14) and np.allclose(p2, q2, atol=1e-14)
    vec = sp.pack(r1, r2)
    ps = pno.PNOSigma(sig, sp)
    got = ps(vec)
    c1, c2 = sig(*sp.unpack(vec))
    ref = sp.pack(c1, c2)
    assert np.abs(got - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_pno_sigma_rotation_invariance():
    """Rotating each kept PNO space leaves U R_bar U^T and hence the
    back-transformed sigma unchanged."""
    sig, sp = _setup(3, 8, 24, 45, 1e-6)
    rng = np.random.default_rng(12)
    vec = sp.symmetrize(rng.standard_normal(sp.length))
    ps = pno.PNOSigma(sig, sp)
    s_ref = sp.unpack(ps(vec))
    r1, r2 = sp.unpack(vec)
    for key in list(sp.U):
        n = sp.U[key].shape[1]
        if n:
            Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
            sp.U[key] = sp.U[key] @ Q
    for i in list(sp.Ui):
        n = sp.Ui[i].shape[1]
        if n:
            Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
            sp.Ui[i] = sp.Ui[i] @ Q
    ps2 = pno.PNOSigma(sig, sp)
    s_rot = sp.unpack(ps2(sp.pack(r1, r2)))
    assert np.abs(s_rot[0] - s_ref[0]).max() < 1e-12
    assert np.abs(s_rot[1] - s_ref[1]).max() < 1e-12


def test_tpno_zero_is_canonical_eom():
    o, v, naux = 3, 6, 18
    sig, sp = _setup(o, v, naux, 46, 0.0)
    assert np.all(sp.n_ij == v) and np.all(sp.n_i == v)
    ps = pno.PNOSigma(sig, sp)
    w, X, rn, it, conv = davidson.solve(ps, sp, 3)
    assert conv
    M = np.array([ps(e) for e in sp.valid_basis().T]).T
    Q = sp.valid_basis()
    ev = np.sort(np.linalg.eigvals(Q.T @ M).real)
    # canonical EOM: sigma matrix on the symmetric amplitude space
    from tests.test_oracle_eom import _sigma_matrix
    evc = np.sort(np.linalg.eigvals(_sigma_matrix(sig, o, v)).real)
    assert np.abs(ev - evc).max() < 1e-10
    assert np.abs(w - evc[:3]).max() < 1e-9


def test_davidson_matches_dense_eig_of_projected_map():
    sig, sp = _setup(3, 8, 24, 47, 1e-6)
    ps = pno.PNOSigma(sig, sp)
    w, X, rn, it, conv = davidson.solve(ps, sp, 3)
    assert conv and np.all(rn < 1e-7)
    Q = sp.valid_basis()
    M = Q.T @ np.array([ps(e) for e in Q.T]).T
    ev = np.linalg.eigvals(M)
    ev = np.sort(ev.real[np.abs(ev.imag) < 1e-12])
    assert np.abs(w - ev[:3]).max() < 1e-10


def test_truncation_counts_and_threshold_rule():
    eps, B, h = _small(4, 10, 30, 48)
    sp = pno.PNOSpace(eps, B, 4, 3, 1e-7)
    for p, key in enumerate(sp.pairs):
        n = sp.alleig[key]
        assert sp.n_ij[p] == int(np.sum(n >= 1e-7))
    assert sp.length == sp.n_i.sum() + (sp.n_ij ** 2).sum()


def test_state_average_is_mean_of_state_specific_densities():
    """Eq. eom:sa_density is the mean of the one-state densities: a wrong root index or
    weight in the state-specific construction breaks the identity."""
    eps, B, _ = _small(o=3, v=6, naux=18, seed=47)
    o, nr = 3, 3
    Dsa, om, bs = pno.sa_densities(eps, B, o, nr)
    Dss = [pno.ss_densities(eps, B, o, k, nr, om, bs)[0] for k in range(nr)]
    for key, D in Dsa.items():
        mean = sum(Dk[key] for Dk in Dss) / nr
        assert np.abs(mean - D).max() <= 1e-14 * max(1.0, np.abs(D).max())
    # the states differ, so the one-state densities do too
    assert max(np.abs(Dss[0][k] - Dss[1][k]).max() for k in Dsa) > 1e-6
    # one-state densities keep the pair-density invariants (symmetric, PSD)
    for key, D in Dss[1].items():
        assert np.abs(D - D.T).max() < 1e-14 * max(1.0, np.abs(D).max())
        assert np.linalg.eigvalsh(D).min() > -1e-12 * max(1.0, np.trace(D))


def test_ground_state_pno_truncation_of_t2():
    """T -> P T P with P from the ground-state pair density (Methods): threshold 0 is the
    identity, the result lies in the kept spaces on both sides, T^{ji} = T^{ij T} holds,
    and a tighter threshold keeps more (monotone discarded norm)."""
    o, v, naux = 3, 8, 24
    s = make_system(o, v, naux, 48)
    t2 = ccsd.mp1_t2(s["eps"], s["B"], o)
    assert np.abs(pno.gs_truncate_t2(t2, o, 0.0) - t2).max() < 1e-13 * np.abs(t2).max()
    errs = []
    for thr in (1e-3, 1e-5, 1e-7):
        tt = pno.gs_truncate_t2(t2, o, thr)
        for i in range(o):
            for j in range(o):
                assert np.abs(tt[j, i] - tt[i, j].T).max() < 1e-14
        for i in range(o):
            for j in range(i, o):
                w, U = np.linalg.eigh(pno.pair_density(t2[i, j], i, j))
                Q = U[:, w < thr]                       # discarded directions
                assert np.abs(Q.T @ tt[i, j]).max() < 1e-12 and np.abs(tt[i, j] @ Q).max() < 1e-12
        errs.append(np.linalg.norm(tt - t2))
    assert errs[0] >= errs[1] >= errs[2] and errs[0] > 0


def test_osv_count_is_the_diagonal_density_count_at_a_tenth_of_t_pno():
    """T_CutOSV = T_CutPNO / 10 (Sec. 3) on the state-averaged D^{ii} (Eq.
    eom:sa_density): n_i equals the number of eigenvalues of D^{ii} (computed here by
    SciPy's solver) that are >= T_PNO / 10.  The case is chosen so that counting at
    T_PNO itself gives a different answer, so a threshold mix-up fails."""
    import scipy.linalg
    eps, B, h = _small(4, 12, 36, 52)
    tp = 1e-5
    sp = pno.PNOSpace(eps, B, 4, 3, tp)
    differs = False
    for i in range(4):
        w = scipy.linalg.eigvalsh(sp.D[i, i])
        assert sp.n_i[i] == int(np.sum(w >= tp / 10))
        differs = differs or int(np.sum(w >= tp)) != sp.n_i[i]
    assert differs
    # an explicit T_CutOSV overrides the default
    sp2 = pno.PNOSpace(eps, B, 4, 3, tp, t_osv=tp)
    for i in range(4):
        assert sp2.n_i[i] == int(np.sum(scipy.linalg.eigvalsh(sp.D[i, i]) >= tp))


def test_semicanonical_bases_diagonalise_the_virtual_fock_block():
    """Semicanonical PNOs/OSVs (Sec. 2, PNO-CCSD simulation): every kept basis is
    orthonormal, spans exactly the kept eigenvectors of its density (SciPy's
    eigensolver), and U^T f_vv U is diagonal with the recorded fbar on the diagonal,
    in ascending order."""
    import scipy.linalg
    o, v = 4, 12
    eps, B, h = _small(o, v, 36, 53)
    tp = 1e-6
    sp = pno.PNOSpace(eps, B, o, 3, tp)
    fvv = np.diag(eps[o:])
    sets = [(sp.U[k], sp.fbar[k], sp.D[k], tp) for k in sp.pairs]
    sets += [(sp.Ui[i], sp.fbar_i[i], sp.D[i, i], tp / 10) for i in range(o)]
    checked = 0
    for U, fb, D, thr in sets:
        n = U.shape[1]
        if n == 0:
            continue
        assert np.abs(U.T @ U - np.eye(n)).max() < 1e-12
        w, V = scipy.linalg.eigh(D)
        Vk = V[:, w >= thr]
        assert Vk.shape[1] == n
        assert np.abs(U @ U.T - Vk @ Vk.T).max() < 1e-9
        F = U.T @ fvv @ U
        assert np.abs(F - np.diag(np.diag(F))).max() < 1e-12
        assert np.abs(np.diag(F) - fb).max() < 1e-12
        assert np.all(np.diff(fb) >= 0)
        checked += 1
    assert checked > o
