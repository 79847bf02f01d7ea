"""GPU parity of pno_build / sigma / davidson_solve against the FP64 oracle.

Every comparison of vectors happens in the canonical space (each side
back-transforms with its own PNO/OSV bases), so it does not depend on the
phase of individual PNOs; PNO counts are compared exactly."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synthetic import make_system
from oracle import ccsd, davidson, eom, hamiltonian as hm, pno


@pytest.fixture(scope="module")
def pkg():
    import paper_1802_06738_gb300 as p
    p.build()
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    return pkg.Context(0)


CASES = {
    # name: (o, v, naux, seed, t_pno, nroots, ground state)
    "small_ccsd_t0": (5, 20, 60, 1, 0.0, 3, "ccsd"),
    "small_ccsd": (5, 20, 60, 1, 1e-7, 3, "ccsd"),
    "mp1_ragged": (6, 30, 90, 11, 1e-6, 4, "mp1"),
    "mp1_tight": (4, 24, 40, 12, 1e-9, 3, "mp1"),
    "empty_pairs": (3, 8, 24, 13, 1e-4, 3, "mp1"),
    # T_PNO = 0 with v = 96: every pair block (96 PNOs) is above the tensor-core path's limit
    # of 80 and above the grouped kernel's 64, so every sandwich runs on the generic kernel
    "wide_t0": (3, 96, 96, 14, 0.0, 2, "mp1"),
}


def _oracle(case):
    o, v, naux, seed, tp, nr, gs = CASES[case]
    s = make_system(o, v, naux, seed)
    eps, B = s["eps"], s["B"]
    h = hm.hcore_from_fock(eps, B, o)
    if gs == "ccsd":
        t1, t2, _, _ = ccsd.solve_ccsd(eps, B, o)
    else:
        t1, t2 = np.zeros((o, v)), ccsd.mp1_t2(eps, B, o)
    sig = eom.Sigma(t1, t2, h, B, o)
    sp = pno.PNOSpace(eps, B, o, nr, tp)
    return dict(o=o, v=v, eps=eps, B=B, t1=t1 if gs == "ccsd" else None, t2=t2 if gs == "ccsd" else None,
                sig=sig, sp=sp, ps=pno.PNOSigma(sig, sp), nr=nr, tp=tp)


_cache = {}


def oracle_case(case):
    if case not in _cache:
        _cache[case] = _oracle(case)
    return _cache[case]


def _build(pkg, ctx, d, **kw):
    opts = pkg.make_opts(t_pno=d["tp"], nroots=d["nr"], **kw)
    return pkg.PNO(ctx, d["eps"], d["B"], d["o"], t1=d["t1"], t2=d["t2"], opts=opts)


def _pack_gpu(gp, r1, r2):
    o = gp.o
    vec = np.zeros(gp.length)
    for i in range(o):
        U, _ = gp.basis(-i - 1)
        vec[gp.off_i[i]:gp.off_i[i + 1]] = U.T @ r1[i]
    for p, (i, j) in enumerate(gp.pairs):
        U, _ = gp.basis(p)
        vec[gp.off_ij[p]:gp.off_ij[p + 1]] = (U.T @ r2[i, j] @ U).ravel()
    return vec


def _unpack_gpu(gp, vec):
    o, v = gp.o, gp.v
    r1 = np.zeros((o, v)); r2 = np.zeros((o, o, v, v))
    for i in range(o):
        U, _ = gp.basis(-i - 1)
        r1[i] = U @ vec[gp.off_i[i]:gp.off_i[i + 1]]
    for p, (i, j) in enumerate(gp.pairs):
        U, _ = gp.basis(p)
        n = gp.n_ij[p]
        R = U @ vec[gp.off_ij[p]:gp.off_ij[p + 1]].reshape(n, n) @ U.T
        r2[i, j] = R; r2[j, i] = R.T
    return r1, r2


@pytest.mark.parametrize("case", list(CASES))
def test_pno_spaces_match_oracle(pkg, ctx, case):
    d = oracle_case(case)
    gp = _build(pkg, ctx, d)
    sp = d["sp"]
    assert np.array_equal(gp.n_ij, sp.n_ij)
    assert np.array_equal(gp.n_i, sp.n_i)
    assert np.allclose(gp.cis_energies(), sp.cis_omega, atol=1e-12)
    for p, key in enumerate(sp.pairs):
        U, fb = gp.basis(p)
        Uo = sp.U[key]
        assert np.abs(U @ U.T - Uo @ Uo.T).max() < 1e-9
        assert np.allclose(fb, sp.fbar[key], atol=1e-10)
    for i in range(d["o"]):
        U, fb = gp.basis(-i - 1)
        assert np.abs(U @ U.T - sp.Ui[i] @ sp.Ui[i].T).max() < 1e-9


@pytest.mark.parametrize("case", list(CASES))
def test_sigma_fp64_parity(pkg, ctx, case):
    d = oracle_case(case)
    gp = _build(pkg, ctx, d)
    o, v = d["o"], d["v"]
    rng = np.random.default_rng(5)
    nvec = 3
    cans = []
    for _ in range(nvec):
        r1 = rng.standard_normal((o, v))
        r2 = rng.standard_normal((o, o, v, v)); r2 = 0.5 * (r2 + r2.transpose(1, 0, 3, 2))
        cans.append((r1, r2))
    R = np.array([_pack_gpu(gp, *c) for c in cans])
    rt = torch.tensor(R, device="cuda:0")
    st = torch.zeros_like(rt)
    gp.sigma(rt, st)
    torch.cuda.synchronize()
    S = st.cpu().numpy()
    sp, ps = d["sp"], d["ps"]
    for k, (r1, r2) in enumerate(cans):
        ref1, ref2 = sp.unpack(ps(sp.pack(r1, r2)))
        g1, g2 = _unpack_gpu(gp, S[k])
        scale = max(np.abs(ref1).max(), np.abs(ref2).max())
        assert np.abs(g1 - ref1).max() < 1e-11 * scale
        assert np.abs(g2 - ref2).max() < 1e-11 * scale


@pytest.mark.parametrize("case", ["small_ccsd", "mp1_ragged"])
def test_sigma_fp32_error_bound(pkg, ctx, case):
    d = oracle_case(case)
    gp = _build(pkg, ctx, d)
    rng = np.random.default_rng(6)
    R = rng.standard_normal((2, gp.length))
    r64 = torch.tensor(R, device="cuda:0")
    s64 = torch.zeros_like(r64)
    gp.sigma(r64, s64, precision=pkg.FP64)
    r32 = r64.float()
    s32 = torch.zeros_like(r32)
    gp.sigma(r32, s32, precision=pkg.FP32)
    torch.cuda.synchronize()
    a, b = s64.cpu().numpy(), s32.double().cpu().numpy()
    assert np.abs(a - b).max() < 2e-5 * np.abs(a).max()


@pytest.mark.parametrize("case", ["small_ccsd_t0", "small_ccsd", "mp1_ragged"])
def test_davidson_fp64_matches_oracle(pkg, ctx, case):
    d = oracle_case(case)
    gp = _build(pkg, ctx, d)
    assert gp.solve_stats() == dict(fp32=0, fp64=0)
    e, rn, it, conv = gp.davidson_solve()
    w, X, rno, ito, convo = davidson.solve(d["ps"], d["sp"], d["nr"])
    assert conv and convo
    assert np.abs(e - w).max() < 1e-8
    ev = gp.solve_stats()   # the guesses, then at least one new sigma per iteration but the last; FP64 only
    assert ev["fp32"] == 0 and ev["fp64"] >= it


def test_davidson_mixed_with_refinement(pkg, ctx):
    d = oracle_case("mp1_ragged")
    gp = _build(pkg, ctx, d, precision=pkg.FP32, refine_fp64=1)
    e, rn, it, conv = gp.davidson_solve()
    w, X, rno, ito, convo = davidson.solve(d["ps"], d["sp"], d["nr"])
    assert conv
    assert np.abs(e - w).max() < 1e-6
    ev = gp.solve_stats()   # the FP32 phase from the guesses, then the FP64 refinement
    assert ev["fp32"] >= d["nr"] and ev["fp64"] >= 1


@pytest.mark.parametrize("case", ["mp1_ragged", "wide_t0"])
def test_sigma_bf16_error_bound(pkg, ctx, case):
    """BF16 sigma (tensor-core sandwiches for blocks of at most 80 PNOs, the generic kernel
    above; BF16 dense blocks) against the oracle: relative error within 2e-2 of the largest
    element (BF16 keeps 8 significant bits; the operands are rounded once, sums in FP32)."""
    d = oracle_case(case)
    gp = _build(pkg, ctx, d)
    o, v = d["o"], d["v"]
    rng = np.random.default_rng(9)
    r1 = rng.standard_normal((o, v))
    r2 = rng.standard_normal((o, o, v, v)); r2 = 0.5 * (r2 + r2.transpose(1, 0, 3, 2))
    R = np.array([_pack_gpu(gp, r1, r2)])
    rt = torch.tensor(R, device="cuda:0", dtype=torch.float32)
    st = torch.zeros_like(rt)
    gp.sigma(rt, st, precision=pkg.BF16)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    sp, ps = d["sp"], d["ps"]
    ref1, ref2 = sp.unpack(ps(sp.pack(r1, r2)))
    g1, g2 = _unpack_gpu(gp, st.cpu().numpy()[0].astype(np.float64))
    scale = max(np.abs(ref1).max(), np.abs(ref2).max())
    err = max(np.abs(g1 - ref1).max(), np.abs(g2 - ref2).max()) / scale
    assert err < 2e-2, err
    assert err > 0.0   # the BF16 path really rounds (it is not the FP64 one)
