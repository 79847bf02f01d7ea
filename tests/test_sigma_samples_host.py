"""CPU checks of the sampled-sigma helpers (tests/sigma_samples.py) that the large-workload
GPU test relies on, and of the fixture script's sample fields (tests/golden/make_golden.py),
on a small system:
  * the samples written from the per-pair oracle (O2) are read back exactly from the
    projected canonical sigma (oracle.pno.PNOSigma, Sec. 2) through the helpers;
  * they are read back equally when every PNO/OSV basis is rotated inside its space (the
    library's bases differ from the oracle's by such rotations and by phases);
  * every non-empty pair block and every singles row with OSVs has samples;
  * a transposed read of a pair block fails."""
import os
import sys

import numpy as np
import pytest

from synthetic import make_system
from oracle import ccsd, eom, hamiltonian as hm, pno
from tests.sigma_samples import blockwise_vector, sampled_entries

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_golden  # noqa: E402

W = dict(o=4, v=12, naux=36, nroots=3, t_pno=1e-6, seed=65)   # one empty pair, ragged others


@pytest.fixture(scope="module")
def case():
    fields = make_golden.sigma_sample_fields(W, npairs_whole=3, per_pair=5, per_row=4)
    s = make_system(W["o"], W["v"], W["naux"], W["seed"])
    eps, B, o = s["eps"], s["B"], W["o"]
    sp = pno.PNOSpace(eps, B, o, W["nroots"], W["t_pno"])
    t1, t2 = np.zeros((o, W["v"])), ccsd.mp1_t2(eps, B, o)
    ps = pno.PNOSigma(eom.Sigma(t1, t2, hm.hcore_from_fock(eps, B, o), B, o), sp)
    return fields, sp, ps


def _basis(sp):
    return lambda k: sp.Ui[-k - 1] if k < 0 else sp.U[sp.pairs[k]]


def _read(sp, basis, sig, fields):
    return sampled_entries(sp, basis, sig, fields["sigma_pair_samples"], fields["sigma_singles_samples"])


def test_samples_cover_every_nonempty_block(case):
    fields, sp, _ = case
    pairs = {f"{i},{j}" for p, (i, j) in enumerate(sp.pairs) if sp.n_ij[p]}
    assert set(fields["sigma_pair_samples"]) == pairs
    assert set(fields["sigma_singles_samples"]) == {str(i) for i in range(sp.o) if sp.n_i[i]}
    assert np.any(np.asarray(sp.n_ij) < W["v"])      # truncated spaces: the projection matters


def test_samples_read_back_from_projected_canonical_sigma(case):
    fields, sp, ps = case
    basis = _basis(sp)
    vec = blockwise_vector(sp, basis, make_golden.trial_r1(sp.o, sp.v), make_golden.trial_r2_block)
    got, ref = _read(sp, basis, ps(vec), fields)
    scale = np.abs(ref).max()
    assert scale > 0 and np.abs(got - ref).max() <= 1e-12 * scale


def test_samples_invariant_under_rotations_inside_each_space(case):
    fields, sp, ps = case
    rng = np.random.default_rng(5)
    Q = {}
    for k in [-i - 1 for i in range(sp.o)] + list(range(len(sp.pairs))):
        n = sp.n_i[-k - 1] if k < 0 else sp.n_ij[k]
        Q[k] = np.linalg.qr(rng.standard_normal((n, n)))[0] if n else np.zeros((0, 0))
    base = _basis(sp)
    rotated = lambda k: base(k) @ Q[k]

    def to_base(x, sign):    # packed vector in the rotated bases <-> in the oracle's bases
        y = x.copy()
        for i in range(sp.o):
            sl = slice(sp.off_i[i], sp.off_i[i + 1])
            y[sl] = (Q[-i - 1] if sign > 0 else Q[-i - 1].T) @ x[sl]
        for p in range(len(sp.pairs)):
            n = sp.n_ij[p]
            sl = slice(sp.off_ij[p], sp.off_ij[p + 1])
            q = Q[p] if sign > 0 else Q[p].T
            y[sl] = (q @ x[sl].reshape(n, n) @ q.T).ravel()
        return y

    vec = blockwise_vector(sp, rotated, make_golden.trial_r1(sp.o, sp.v), make_golden.trial_r2_block)
    sig = to_base(ps(to_base(vec, +1)), -1)
    got, ref = _read(sp, rotated, sig, fields)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_transposed_block_read_fails(case):
    fields, sp, ps = case
    basis = _basis(sp)
    vec = blockwise_vector(sp, basis, make_golden.trial_r1(sp.o, sp.v), make_golden.trial_r2_block)
    sig = ps(vec)
    bad = sig.copy()
    for p, (i, j) in enumerate(sp.pairs):
        n = sp.n_ij[p]
        if i != j and n:
            sl = slice(sp.off_ij[p], sp.off_ij[p + 1])
            bad[sl] = sig[sl].reshape(n, n).T.ravel()
    got, ref = _read(sp, basis, bad, fields)
    assert np.abs(got - ref).max() > 1e-3 * np.abs(ref).max()
