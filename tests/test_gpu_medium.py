"""Parity at the benchmark's full size: the medium workload (o = 20, v = 200,
naux = 600, 6 roots, T_CutPNO = 1e-7, MP1 T2; Sec. 2 and Eq. T1).

The oracle is too slow to run here, so its results are read from
tests/golden/oracle_medium.json (written by tests/golden/make_golden.py,
which calls only oracle/):
  * the PNO counts n_ij and n_i (compared exactly);
  * sigma of the seeded canonical trial vector: every singles element and
    256 seeded entries of five pair blocks, in the canonical basis;
  * the oracle's FP64 Davidson excitation energies.
The GPU side runs through the C ABI in the launch configuration of bench.py.
"""
import json
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "oracle_medium.json")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def medium():
    if not os.path.exists(GOLD):
        pytest.skip("oracle_medium.json not generated")
    import paper_1802_06738_gb300 as pkg
    from synthetic import make_system
    sys.path.insert(0, os.path.join(HERE, "golden"))
    from make_golden import trial_vector
    gold = json.load(open(GOLD))
    pkg.build()
    ctx = pkg.Context(0)
    s = make_system(gold["o"], gold["v"], gold["naux"], gold["seed"])
    opts = pkg.make_opts(t_pno=gold["t_pno"], nroots=gold["nroots"], precision=pkg.FP32, refine_fp64=1)
    gp = pkg.PNO(ctx, s["eps"], s["B"], gold["o"], opts=opts)
    return pkg, gp, gold, trial_vector


def _pack(gp, r1, r2):
    vec = np.zeros(gp.length)
    for i in range(gp.o):
        U, _ = gp.basis(-i - 1)
        vec[gp.off_i[i]:gp.off_i[i + 1]] = U.T @ r1[i]
    for p, (i, j) in enumerate(gp.pairs):
        U, _ = gp.basis(p)
        vec[gp.off_ij[p]:gp.off_ij[p + 1]] = (U.T @ r2[i, j] @ U).ravel()
    return vec


def _canonical(gp, vec, pairs):
    """Singles (o x v) and the requested pair blocks (v x v) of a packed vector, canonical basis."""
    s1 = np.zeros((gp.o, gp.v))
    for i in range(gp.o):
        U, _ = gp.basis(-i - 1)
        s1[i] = U @ vec[gp.off_i[i]:gp.off_i[i + 1]]
    blocks = {}
    for (i, j) in pairs:
        p = gp.pairs.index((min(i, j), max(i, j)))
        U, _ = gp.basis(p)
        n = gp.n_ij[p]
        R = U @ vec[gp.off_ij[p]:gp.off_ij[p + 1]].reshape(n, n) @ U.T
        blocks[(i, j)] = R if i <= j else R.T
    return s1, blocks


def test_medium_pno_counts(medium):
    _, gp, gold, _ = medium
    assert np.array_equal(np.asarray(gp.n_ij), np.asarray(gold["n_ij"]))
    assert np.array_equal(np.asarray(gp.n_i), np.asarray(gold["n_i"]))
    assert gp.length == gold["vec_len"]


# BF16: the dense pair blocks are rounded to 8 significant bits (relative 2^-9 per
# element) and the rounding errors of a block row add up to about that fraction of the
# row's absolute sum, which the bound below covers with a margin
@pytest.mark.parametrize("prec,tol", [("FP64", 1e-10), ("FP32", 1e-5), ("BF16", 2e-2)])
def test_medium_sigma_matches_oracle(medium, prec, tol):
    pkg, gp, gold, trial_vector = medium
    r1, r2 = trial_vector(gold["o"], gold["v"], gold["sigma_trial_seed"])
    x = _pack(gp, r1, r2)
    dt = torch.float64 if prec == "FP64" else torch.float32   # BF16 sigma takes float vectors
    rt = torch.tensor(x[None, :], dtype=dt, device="cuda:0")
    st = torch.zeros_like(rt)
    gp.sigma(rt, st, precision=getattr(pkg, prec))
    torch.cuda.synchronize()
    samples = gold["sigma_pair_samples"]
    pairs = [tuple(int(t) for t in k.split(",")) for k in samples]
    s1, blocks = _canonical(gp, st.double().cpu().numpy()[0], pairs)
    ref1 = np.asarray(gold["sigma_s1"])
    scale = np.abs(ref1).max()
    for key, ent in samples.items():
        scale = max(scale, max(abs(e[2]) for e in ent))
    assert np.abs(s1 - ref1).max() <= tol * scale
    for (i, j), key in zip(pairs, samples):
        got = np.array([blocks[(i, j)][a, b] for a, b, _ in samples[key]])
        ref = np.array([e[2] for e in samples[key]])
        assert np.abs(got - ref).max() <= tol * scale, (key, np.abs(got - ref).max() / scale)


@pytest.mark.parametrize("prec,refine,tol", [("FP64", 0, 1e-8), ("FP32", 1, 1e-7), ("BF16", 1, 1e-7)])
def test_medium_davidson_energies(medium, prec, refine, tol):
    pkg, gp, gold, _ = medium
    opts = pkg.make_opts(t_pno=gold["t_pno"], nroots=gold["nroots"], precision=getattr(pkg, prec),
                         refine_fp64=refine)
    e, rn, it, conv = gp.davidson_solve(opts)
    assert conv
    assert np.abs(np.asarray(e) - np.asarray(gold["energies"])).max() < tol
    if refine:
        # the unrefined energies of the low-precision phases, per root, against the oracle
        # (a BF16 solve runs BF16, then FP32, then FP64)
        ref = np.asarray(gold["energies"])
        low = gp.lowprec_energies(pkg.FP32)
        assert len(low) == gold["nroots"] and np.abs(low - ref).max() < 1e-4
        if prec == "BF16":
            low16 = gp.lowprec_energies(pkg.BF16)
            assert len(low16) == gold["nroots"] and np.abs(low16 - ref).max() < 3e-2
