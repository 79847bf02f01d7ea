"""Parity of sigma on every pair block of the medium workload (o = 20, v = 200, naux = 600,
6 roots, T_CutPNO = 1e-7, MP1 T2; Sec. 2), in the launch configuration of bench.py.

The oracle's values come from tests/golden/oracle_medium_blockwise.json (written by
tests/golden/make_golden.py medium --sigma-samples --out=oracle_medium_blockwise.json,
which calls only oracle/): sigma of the blockwise trial vector from the per-pair oracle
(O2), at seeded canonical-basis entries of every non-empty pair block (256 for eight
blocks of every size class, 8 for the others) and of every singles row (three whole).
The spaces come from dense CIS on both sides here, so the FP64 bound is that of the
canonical-trial test of this workload.  Named so that pytest collects it after the other
medium-size GPU tests.
"""
import json
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "oracle_medium_blockwise.json")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def medium():
    if not os.path.exists(GOLD):
        pytest.skip("oracle_medium_blockwise.json not generated")
    import paper_1802_06738_gb300 as pkg
    from synthetic import make_system
    from tests.sigma_samples import blockwise_vector
    sys.path.insert(0, os.path.join(HERE, "golden"))
    from make_golden import trial_r1, trial_r2_block
    gold = json.load(open(GOLD))
    pkg.build()
    ctx = pkg.Context(0)
    s = make_system(gold["o"], gold["v"], gold["naux"], gold["seed"])
    opts = pkg.make_opts(t_pno=gold["t_pno"], nroots=gold["nroots"], precision=pkg.BF16, refine_fp64=1)
    gp = pkg.PNO(ctx, s["eps"], s["B"], gold["o"], opts=opts)
    bases = {}

    def basis(k):
        if k not in bases:
            bases[k] = gp.basis(k)[0]
        return bases[k]
    vec = blockwise_vector(gp, basis, trial_r1(gp.o, gp.v), trial_r2_block)
    return pkg, ctx, gp, gold, basis, vec


def test_medium_blockwise_samples_cover_every_block(medium):
    _, _, gp, gold, _, _ = medium
    assert np.array_equal(np.asarray(gp.n_ij), np.asarray(gold["n_ij"]))
    assert np.array_equal(np.asarray(gp.n_i), np.asarray(gold["n_i"]))
    nonempty = {f"{i},{j}" for p, (i, j) in enumerate(gp.pairs) if gp.n_ij[p]}
    assert set(gold["sigma_pair_samples"]) == nonempty
    assert set(gold["sigma_singles_samples"]) == {str(i) for i in range(gp.o) if gp.n_i[i]}


@pytest.mark.parametrize("prec,tol", [("FP64", 1e-10), ("FP32", 1e-5), ("BF16", 2e-2)])
def test_medium_sigma_every_block_matches_oracle(medium, prec, tol):
    pkg, ctx, gp, gold, basis, vec = medium
    from tests.sigma_samples import sampled_entries
    dt = torch.float64 if prec == "FP64" else torch.float32   # BF16 sigma takes float vectors
    rt = torch.tensor(vec[None, :], dtype=dt, device="cuda:0")
    st = torch.zeros_like(rt)
    gp.sigma(rt, st, precision=getattr(pkg, prec))
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    got, ref = sampled_entries(gp, basis, st.double().cpu().numpy()[0], gold["sigma_pair_samples"],
                               gold["sigma_singles_samples"])
    scale = np.abs(ref).max()
    err = np.abs(got - ref).max() / scale
    assert err <= tol, (prec, err)
