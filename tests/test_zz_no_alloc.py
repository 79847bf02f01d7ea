"""sigma_noalloc: the allocation-free sigma entry point.

Some callers cannot allocate device memory while they run (a serving loop
that cannot absorb the device-wide synchronisation of cudaMalloc/cudaFree,
or an application whose own pool allocator owns all device memory).
sigma_noalloc keeps its scratch in a fixed file-scope device array instead.
This file checks, through the C ABI, that it returns what sigma() returns,
on two calls in a row (the shared array keeps the previous call's contents),
in FP64 and FP32, and that an oversized request is refused with an error
code before anything is launched.  It is named so that pytest collects it
last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_system


@pytest.fixture(scope="module")
def built():
    import paper_1802_06738_gb300 as pkg
    pkg.build()
    ctx = pkg.Context(0)
    s = make_system(4, 16, 48, 21)
    gp = pkg.PNO(ctx, s["eps"], s["B"], 4, opts=pkg.make_opts(t_pno=1e-6, nroots=3))
    return pkg, ctx, gp


def _call_noalloc(pkg, ctx, gp, r, out, precision):
    nvec = r.shape[0]
    return pkg.lib().sigma_noalloc(ctx.h, gp.h, nvec, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   precision, None)


@pytest.mark.parametrize("precision,dtype,tol", [(0, torch.float64, 1e-12), (1, torch.float32, 2e-6)])
def test_noalloc_matches_sigma_twice(built, precision, dtype, tol):
    pkg, ctx, gp = built
    rng = np.random.default_rng(17)
    for call in range(2):      # two calls in a row: the shared scratch must not leak state
        r = torch.tensor(rng.standard_normal((3, gp.length)), dtype=dtype, device="cuda:0")
        ref = torch.zeros_like(r)
        gp.sigma(r, ref, precision=precision)
        out = torch.full_like(r, float("nan"))
        rc = _call_noalloc(pkg, ctx, gp, r, out, precision)
        assert rc == pkg.OK, pkg.lib().pnoeom_last_error()
        torch.cuda.synchronize()
        a, b = ref.double().cpu().numpy(), out.double().cpu().numpy()
        assert np.all(np.isfinite(b))
        assert np.abs(a - b).max() <= tol * np.abs(a).max()


def test_noalloc_rejects_oversized_request(built):
    pkg, ctx, gp = built
    # FP64 scratch per vector: FvR (v^2), FoR (o^2), Y and Z (v * sum n_ij each)
    per_vec = (gp.v * gp.v + gp.o * gp.o + 2 * gp.v * int(np.sum(gp.n_ij))) * 8
    nvec = (64 << 20) // per_vec + 1
    r = torch.zeros((1, gp.length), dtype=torch.float64, device="cuda:0")
    rc = pkg.lib().sigma_noalloc(ctx.h, gp.h, nvec, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(r.data_ptr()),
                                 0, None)
    assert rc == pkg.ERR_UNSUPPORTED
    assert b"scratch" in pkg.lib().pnoeom_last_error()


def _live_bytes(pkg):
    b = ctypes.c_longlong()
    assert pkg.lib().pnoeom_alloc_live_bytes(ctypes.byref(b)) == pkg.OK
    return b.value


def test_noalloc_allocates_nothing(built):
    """On a fresh handle whose sigma() scratch was sized for one vector, a sigma_noalloc
    call with more vectors leaves the library's allocator untouched and matches sigma()."""
    pkg, ctx, _ = built
    s = make_system(4, 16, 48, 21)
    fresh = pkg.PNO(ctx, s["eps"], s["B"], 4, opts=pkg.make_opts(t_pno=1e-6, nroots=3))
    rng = np.random.default_rng(23)
    one = torch.tensor(rng.standard_normal((1, fresh.length)), dtype=torch.float32, device="cuda:0")
    fresh.sigma(one, torch.zeros_like(one), precision=pkg.FP32)   # loads the kernels; scratch for 1 vector
    torch.cuda.synchronize()
    r = torch.tensor(rng.standard_normal((4, fresh.length)), dtype=torch.float32, device="cuda:0")
    out = torch.full_like(r, float("nan"))
    before = _live_bytes(pkg)
    assert _call_noalloc(pkg, ctx, fresh, r, out, pkg.FP32) == pkg.OK, pkg.lib().pnoeom_last_error()
    torch.cuda.synchronize()
    assert _live_bytes(pkg) == before
    ref = torch.zeros_like(r)
    fresh.sigma(r, ref, precision=pkg.FP32)     # sigma() now grows its scratch to 4 vectors
    torch.cuda.synchronize()
    assert _live_bytes(pkg) > before
    a, b = ref.double().cpu().numpy(), out.double().cpu().numpy()
    assert np.abs(a - b).max() <= 2e-6 * np.abs(a).max()

