"""Batches of systems in one launch sequence (a11): batched sigma equals each
member's own sigma; lockstep batched Davidson equals the individual solves;
the CUDA-graph path (side stream) equals the direct path."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_system

SIZES = [(4, 16, 48, 31), (6, 24, 72, 32), (5, 20, 60, 33), (3, 12, 36, 34)]


@pytest.fixture(scope="module")
def setup():
    import paper_1802_06738_gb300 as pkg
    pkg.build()
    ctx = pkg.Context(0)
    pnos = []
    for (o, v, naux, seed) in SIZES:
        s = make_system(o, v, naux, seed)
        pnos.append(pkg.PNO(ctx, s["eps"], s["B"], o, opts=pkg.make_opts(t_pno=1e-7, nroots=3)))
    return pkg, ctx, pnos


@pytest.mark.parametrize("precision,dtype,tol", [(0, torch.float64, 1e-12), (1, torch.float32, 3e-6)])
@pytest.mark.parametrize("use_stream", [False, True])
def test_batch_sigma_equals_individual(setup, precision, dtype, tol, use_stream):
    pkg, ctx, pnos = setup
    batch = pkg.Batch(ctx, pnos)
    rng = np.random.default_rng(2)
    rs = [torch.tensor(rng.standard_normal((k % 3 + 1, p.length)), dtype=dtype, device="cuda:0") for k, p in enumerate(pnos)]
    rs[2] = None    # a member that takes no part
    outs = [None if r is None else torch.full_like(r, float("nan")) for r in rs]
    stream = torch.cuda.Stream() if use_stream else None
    handle = None if stream is None else stream.cuda_stream
    for _ in range(2):   # the second call replays through the updated graph
        batch.sigma(rs, outs, precision=precision, stream=handle)
    torch.cuda.synchronize()
    for p, r, o in zip(pnos, rs, outs):
        if r is None:
            continue
        ref = torch.zeros_like(r)
        p.sigma(r, ref, precision=precision)
        torch.cuda.synchronize()
        a, b = ref.double().cpu().numpy(), o.double().cpu().numpy()
        assert np.abs(a - b).max() <= tol * np.abs(a).max()


@pytest.mark.parametrize("use_stream", [False, True])
def test_batch_solve_equals_individual(setup, use_stream):
    pkg, ctx, pnos = setup
    batch = pkg.Batch(ctx, pnos)
    stream = torch.cuda.Stream() if use_stream else None
    handle = None if stream is None else stream.cuda_stream
    opts = pkg.make_opts(t_pno=1e-7, nroots=3)
    e, rn, it, cv = batch.solve(opts, stream=handle)
    assert all(cv)
    for k, p in enumerate(pnos):
        ek, rk, ik, ck = p.davidson_solve(opts)
        assert ck and np.abs(ek - e[k]).max() < 1e-9


def test_batch_mixed_refined_matches_fp64(setup):
    pkg, ctx, pnos = setup
    batch = pkg.Batch(ctx, pnos)
    e64, _, _, c64 = batch.solve(pkg.make_opts(t_pno=1e-7, nroots=3))
    em, _, _, cm = batch.solve(pkg.make_opts(t_pno=1e-7, nroots=3, precision=pkg.FP32, refine_fp64=1),
                               stream=torch.cuda.Stream().cuda_stream)
    assert all(c64) and all(cm)
    assert np.abs(e64 - em).max() < 1e-7
