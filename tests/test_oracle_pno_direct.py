"""Pins of the per-pair PNO sigma (oracle.pno_direct.PNOSigmaDirect, "O2") against the
projected canonical sigma (oracle.pno.PNOSigma: U^T sigma(U R U^T) U, Sec. 2), which is
itself pinned against brute force.  A plausible slip in any term (a sign, an index, a
missing transpose of one of the mixed-pair blocks) moves the result far above 1e-12."""
import numpy as np
import pytest

from synthetic import make_system
from oracle import ccsd, eom, hamiltonian as hm, pno
from oracle.pno_direct import PNOSigmaDirect


def _setup(o, v, naux, seed, tp, gs):
    s = make_system(o, v, naux, seed)
    eps, B = s["eps"], s["B"]
    h = hm.hcore_from_fock(eps, B, o)
    if gs == "ccsd":
        t1, t2, _, _ = ccsd.solve_ccsd(eps, B, o)
    else:
        t1, t2 = np.zeros((o, v)), ccsd.mp1_t2(eps, B, o)
    sp = pno.PNOSpace(eps, B, o, 3, tp)
    ref = pno.PNOSigma(eom.Sigma(t1, t2, h, B, o), sp)
    return sp, ref, PNOSigmaDirect(t1, t2, h, B, o, sp)


@pytest.mark.parametrize("o,v,naux,seed,tp,gs", [
    (3, 8, 24, 61, 1e-6, "mp1"),      # ragged PNO spaces, T1 = 0
    (4, 10, 30, 62, 1e-5, "ccsd"),    # T1 != 0 (dressed, non-symmetric factors)
    (3, 7, 21, 63, 0.0, "ccsd"),      # full spaces: equals canonical EOM-CCSD
    (4, 9, 27, 64, 1e-4, "mp1"),      # some empty pair and OSV spaces
])
def test_o2_equals_projected_canonical_sigma(o, v, naux, seed, tp, gs):
    sp, ref, o2 = _setup(o, v, naux, seed, tp, gs)
    rng = np.random.default_rng(seed)
    for _ in range(2):
        x = sp.symmetrize(rng.standard_normal(sp.length))
        a, b = ref(x), o2(x)
        assert np.abs(a - b).max() <= 1e-12 * max(1.0, np.abs(a).max()), np.abs(a - b).max()


def test_o2_output_subsets():
    """Evaluating a subset of output blocks gives exactly those blocks of the full sigma."""
    sp, ref, o2 = _setup(4, 10, 30, 65, 1e-6, "mp1")
    x = sp.symmetrize(np.random.default_rng(1).standard_normal(sp.length))
    full = o2(x)
    pairs = [p for p in range(len(sp.pairs)) if sp.n_ij[p]][:3]
    part = o2(x, pairs=pairs, singles=[2])
    for p in pairs:
        assert np.array_equal(part[sp.off_ij[p]:sp.off_ij[p + 1]], full[sp.off_ij[p]:sp.off_ij[p + 1]])
    assert np.array_equal(part[sp.off_i[2]:sp.off_i[3]], full[sp.off_i[2]:sp.off_i[3]])
    others = np.ones(sp.length, bool)
    for p in pairs:
        others[sp.off_ij[p]:sp.off_ij[p + 1]] = False
    others[sp.off_i[2]:sp.off_i[3]] = False
    assert not np.any(part[others])
