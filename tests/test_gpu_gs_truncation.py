"""Ground-state PNO truncation (pnoeom_opts.t_pno_gs): T2 projected onto the PNOs of its
ground-state pair densities (Methods), then the usual state-averaged excited-state
spaces.  Compared with the oracle's gs_truncate_t2 followed by the same PNO-space sigma
and Davidson solve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synthetic import make_system  # noqa: E402
from oracle import ccsd, davidson, eom, hamiltonian as hm, pno  # noqa: E402
from tests.test_gpu_parity import _pack_gpu, _unpack_gpu  # noqa: E402

pytestmark = pytest.mark.gpu

O, V, NAUX, SEED, TP, TGS, NR = 5, 20, 60, 1, 1e-7, 1e-5, 3


@pytest.fixture(scope="module")
def both():
    import paper_1802_06738_gb300 as pkg
    pkg.build()
    ctx = pkg.Context(0)
    s = make_system(O, V, NAUX, SEED)
    eps, B = s["eps"], s["B"]
    t2 = pno.gs_truncate_t2(ccsd.mp1_t2(eps, B, O), O, TGS)
    sig = eom.Sigma(np.zeros((O, V)), t2, hm.hcore_from_fock(eps, B, O), B, O)
    sp = pno.PNOSpace(eps, B, O, NR, TP)
    gp = pkg.PNO(ctx, eps, B, O, opts=pkg.make_opts(t_pno=TP, nroots=NR, t_pno_gs=TGS))
    full = pkg.PNO(ctx, eps, B, O, opts=pkg.make_opts(t_pno=TP, nroots=NR))
    return pkg, gp, full, sig, sp


def test_gs_truncated_sigma_fp64_parity(both):
    pkg, gp, full, sig, sp = both
    assert np.array_equal(gp.n_ij, sp.n_ij)   # the excited-state spaces do not depend on T
    rng = np.random.default_rng(10)
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


def test_gs_truncated_energies_match_oracle_and_move(both):
    pkg, gp, full, sig, sp = both
    e, rn, it, conv = gp.davidson_solve()
    assert conv
    w, X, rno, ito, convo = davidson.solve(pno.PNOSigma(sig, sp), sp, NR)
    assert convo
    assert np.abs(np.asarray(e) - np.asarray(w)).max() < 1e-8
    e_full, *_ = full.davidson_solve()
    assert np.abs(np.asarray(e) - np.asarray(e_full)).max() > 1e-7   # the truncation acts
