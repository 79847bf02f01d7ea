"""Failure detection without a GPU fault, through the C ABI.

* A bounded device wait that runs out: a self-test kernel waits on an mbarrier
  that nothing arrives at (a short clock budget), records the expiry in the
  status word like the tensor-core kernels do, and the next Davidson solve
  returns PNOEOM_ERR_TIMEOUT; the context stays usable afterwards.
* A Davidson solve stopped by max_iter returns PNOEOM_ERR_NOT_CONVERGED with its
  best values (finite energies and residual norms of the last iteration).
* An allocation failure injected on the host side of the library's caching
  device allocator makes pno_build return PNOEOM_ERR_NOMEM, and everything the
  failed build took is handed back (the allocator's live bytes return to their
  earlier value); the next build succeeds.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_system


@pytest.fixture(scope="module")
def pkg():
    import paper_1802_06738_gb300 as p
    p.build()
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    return pkg.Context(0)


@pytest.fixture(scope="module")
def system():
    return make_system(4, 16, 48, 31)


def _live(pkg):
    b = ctypes.c_longlong()
    assert pkg.lib().pnoeom_alloc_live_bytes(ctypes.byref(b)) == pkg.OK
    return b.value


def test_bounded_wait_expiry_reports_timeout(pkg, ctx, system):
    gp = pkg.PNO(ctx, system["eps"], system["B"], 4, opts=pkg.make_opts(t_pno=1e-6, nroots=3))
    assert ctx.device_status(clear=True) == 0
    flag = ctypes.c_int(-1)
    rc = pkg.lib().pnoeom_selftest_bounded_wait(ctx.h, 200000, None, ctypes.byref(flag))
    assert rc == pkg.OK, pkg.lib().pnoeom_last_error()
    assert flag.value == 1                       # the wait ran out
    assert ctx.device_status(clear=False) & 1    # and was recorded
    opts = pkg.make_opts(t_pno=1e-6, nroots=3)
    e, rn, it = np.zeros(3), np.zeros(3), ctypes.c_int()
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = pkg.lib().davidson_solve(ctx.h, gp.h, ctypes.byref(opts), None, dp(e), dp(rn), ctypes.byref(it))
    assert rc == pkg.ERR_TIMEOUT
    assert b"bounded wait" in pkg.lib().pnoeom_last_error()
    # the solve cleared the word; the context and handle are still usable
    assert ctx.device_status(clear=False) == 0
    e2, rn2, it2, conv = gp.davidson_solve(opts)
    assert conv and np.all(np.isfinite(e2))
    # the self-test's budget is validated on the host
    assert pkg.lib().pnoeom_selftest_bounded_wait(ctx.h, 0, None, ctypes.byref(flag)) == pkg.ERR_INVALID_ARG


def test_not_converged_returns_best_values(pkg, ctx, system):
    gp = pkg.PNO(ctx, system["eps"], system["B"], 4, opts=pkg.make_opts(t_pno=1e-6, nroots=3))
    e_ref, _, _, conv = gp.davidson_solve(pkg.make_opts(t_pno=1e-6, nroots=3))
    assert conv
    opts = pkg.make_opts(t_pno=1e-6, nroots=3, max_iter=2, res_tol=1e-12, e_tol=1e-14)
    e, rn, it, dp = np.zeros(3), np.zeros(3), ctypes.c_int(), lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = pkg.lib().davidson_solve(ctx.h, gp.h, ctypes.byref(opts), None, dp(e), dp(rn), ctypes.byref(it))
    assert rc == pkg.ERR_NOT_CONVERGED
    assert it.value == 2
    assert np.all(np.isfinite(e)) and np.all(np.isfinite(rn))
    assert rn.max() > 1e-12                      # not converged, as reported
    # best values so far: Ritz values of a two-iteration subspace, already near the roots
    assert np.abs(e - e_ref).max() < 0.1 * np.abs(e_ref).max()


@pytest.mark.parametrize("after", [0, 3, 40])
def test_injected_alloc_failure_returns_nomem_without_leak(pkg, ctx, system, after):
    torch.cuda.synchronize()
    before = _live(pkg)
    assert pkg.lib().pnoeom_inject_alloc_failure(after) == pkg.OK
    eps, B = np.ascontiguousarray(system["eps"]), np.ascontiguousarray(system["B"])
    sysd = pkg.System(4, 16, 48, eps.ctypes.data, B.ctypes.data, None, None, pkg.HOST)
    opts = pkg.make_opts(t_pno=1e-6, nroots=3)
    h = ctypes.c_void_p()
    rc = pkg.lib().pno_build(ctx.h, ctypes.byref(sysd), ctypes.byref(opts), None, ctypes.byref(h))
    msg = pkg.lib().pnoeom_last_error()
    pkg.lib().pnoeom_inject_alloc_failure(-1)
    assert rc == pkg.ERR_NOMEM
    assert b"injected" in msg
    assert not h.value
    assert _live(pkg) == before                  # the failed build released what it took
    gp = pkg.PNO(ctx, system["eps"], system["B"], 4, opts=opts)   # and the next build works
    assert gp.length > 0
