"""Serving (a12): continuous batching of solves of different sizes.  Every
result must equal the same system solved alone; requests that arrive while
others are solving join the running batch; over-budget requests are refused."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_system

REQS = [  # (o, v, naux, seed, t_pno, roots, precision)
    (3, 12, 36, 41, 1e-6, 2, 0),
    (4, 16, 48, 42, 1e-7, 3, 0),
    (5, 20, 60, 43, 1e-7, 3, 1),
    (3, 10, 30, 44, 1e-6, 2, 0),
    (6, 24, 72, 45, 1e-7, 3, 1),
]


@pytest.fixture(scope="module")
def pkg():
    import paper_1802_06738_gb300 as p
    p.build()
    return p


def _opts(pkg, tp, nr, prec):
    return pkg.make_opts(t_pno=tp, nroots=nr, precision=prec, refine_fp64=1 if prec == pkg.FP32 else 0)


def test_served_results_equal_solo_results(pkg):
    ctx = pkg.Context(0)
    srv = pkg.Server(ctx, hbm_budget_bytes=0, max_active=8)
    systems = [make_system(o, v, naux, seed) for (o, v, naux, seed, *_r) in REQS]
    ids = []
    for k in range(3):                              # first wave
        o, v, naux, seed, tp, nr, prec = REQS[k]
        ids.append(srv.submit(systems[k]["eps"], systems[k]["B"], o, _opts(pkg, tp, nr, prec)))
    time.sleep(0.3)
    for k in range(3, len(REQS)):                   # second wave arrives while the first runs
        o, v, naux, seed, tp, nr, prec = REQS[k]
        ids.append(srv.submit(systems[k]["eps"], systems[k]["B"], o, _opts(pkg, tp, nr, prec)))
    for rid in ids:
        assert srv.wait(rid, 600.0) == pkg.OK
    st = srv.stats()
    assert st["merges"] >= 2 and st["rounds"] > 0
    for k, rid in enumerate(ids):
        res = srv.poll(rid)
        assert res["status"] == pkg.DONE, res
        t = res["times"]
        assert t[0] <= t[1] <= t[2] <= t[3]
        o, v, naux, seed, tp, nr, prec = REQS[k]
        solo = pkg.PNO(ctx, systems[k]["eps"], systems[k]["B"], o, opts=_opts(pkg, tp, nr, 0))
        e, rn, it, conv = solo.davidson_solve()
        assert conv
        tol = 1e-9 if prec == 0 else 1e-7
        assert np.abs(res["energies"] - e).max() < tol, (k, res["energies"], e)
        assert res["sigma_evals"] > 0
    srv.close()


def test_over_budget_request_is_refused(pkg):
    ctx = pkg.Context(0)
    srv = pkg.Server(ctx, hbm_budget_bytes=1 << 20, max_active=2)
    s = make_system(5, 20, 60, 7)
    rid = srv.submit(s["eps"], s["B"], 5, pkg.make_opts(t_pno=1e-7, nroots=3))
    assert srv.wait(rid, 10.0) == pkg.OK
    res = srv.poll(rid)
    assert res["status"] == pkg.FAILED and res["error"][0] == pkg.ERR_NOMEM
    srv.close()
