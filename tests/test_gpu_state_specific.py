"""State-specific PNOs (pnoeom_opts.state_specific = k): the PNO/OSV spaces built from the
CIS(D) pair densities of CIS root k alone, the one-state construction that the paper's
state average replaces (Methods).  Compared with the oracle's ss_densities space: PNO
counts exactly, the spanned spaces, FP64 sigma in the canonical space, and the Davidson
energies.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synthetic import make_system  # noqa: E402
from oracle import ccsd, davidson, eom, hamiltonian as hm, pno  # noqa: E402
from tests.test_gpu_parity import _pack_gpu, _unpack_gpu  # noqa: E402

pytestmark = pytest.mark.gpu

O, V, NAUX, SEED, TP, NR, ROOT = 6, 30, 90, 11, 1e-6, 4, 2   # root index 2 -> state_specific = 3


@pytest.fixture(scope="module")
def both():
    import paper_1802_06738_gb300 as pkg
    pkg.build()
    ctx = pkg.Context(0)
    s = make_system(O, V, NAUX, SEED)
    eps, B = s["eps"], s["B"]
    t2 = ccsd.mp1_t2(eps, B, O)
    sig = eom.Sigma(np.zeros((O, V)), t2, hm.hcore_from_fock(eps, B, O), B, O)
    D, om, bs = pno.ss_densities(eps, B, O, ROOT, NR)
    sp = pno.PNOSpace(eps, B, O, NR, TP, D=D, cis=(om, bs))
    sp_sa = pno.PNOSpace(eps, B, O, NR, TP)
    gp = pkg.PNO(ctx, eps, B, O, opts=pkg.make_opts(t_pno=TP, nroots=NR, state_specific=ROOT + 1))
    return pkg, gp, sig, sp, sp_sa


def test_state_specific_spaces_match_oracle(both):
    pkg, gp, sig, sp, sp_sa = both
    assert np.array_equal(gp.n_ij, sp.n_ij)
    assert np.array_equal(gp.n_i, sp.n_i)
    for p, key in enumerate(sp.pairs):
        U, _ = gp.basis(p)
        assert np.abs(U @ U.T - sp.U[key] @ sp.U[key].T).max() < 1e-9
    # and they are not the state-averaged spaces
    differs = not np.array_equal(sp.n_ij, sp_sa.n_ij) or any(
        np.abs(sp.U[k] @ sp.U[k].T - sp_sa.U[k] @ sp_sa.U[k].T).max() > 1e-6 for k in sp.pairs)
    assert differs


def test_state_specific_sigma_fp64_parity(both):
    pkg, gp, sig, sp, sp_sa = both
    rng = np.random.default_rng(9)
    r1 = rng.standard_normal((O, V))
    r2 = rng.standard_normal((O, O, V, V))
    r2 = 0.5 * (r2 + r2.transpose(1, 0, 3, 2))
    x = torch.tensor(_pack_gpu(gp, r1, r2)[None, :], device="cuda:0")
    y = torch.zeros_like(x)
    gp.sigma(x, y)
    torch.cuda.synchronize()
    g1, g2 = _unpack_gpu(gp, y.cpu().numpy()[0])
    ref1, ref2 = sp.unpack(pno.PNOSigma(sig, sp)(sp.pack(r1, r2)))
    scale = max(np.abs(ref1).max(), np.abs(ref2).max())
    assert np.abs(g1 - ref1).max() < 1e-11 * scale
    assert np.abs(g2 - ref2).max() < 1e-11 * scale


def test_state_specific_davidson_matches_oracle(both):
    pkg, gp, sig, sp, sp_sa = both
    e, rn, it, conv = gp.davidson_solve(pkg.make_opts(t_pno=TP, nroots=NR, state_specific=ROOT + 1))
    assert conv
    w, X, rno, ito, convo = davidson.solve(pno.PNOSigma(sig, sp), sp, NR)
    assert convo
    assert np.abs(np.asarray(e) - np.asarray(w)).max() < 1e-8
