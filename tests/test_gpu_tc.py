"""The tensor-core tile kernel alone (pnoeom_gemm_tf32x3): tcgen05 kind::tf32 MMAs with
each FP32 operand split into a tf32 high part and a tf32 remainder (3xTF32).

Reference: the FP64 product of the same FP32 inputs.  Bound, elementwise against
scale = |alpha| |A||B| + |C|: the three kept partial products carry about 21 bits
(3e-6), and the FP32 accumulation over K adds a random-walk term 3 sqrt(K) u
(u = 2^-24).  Plain TF32 (10-bit mantissa) misses the bound of the second test by an
order of magnitude, so that test shows that the low parts are used.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SHAPES = [(128, 64, 32), (1, 1, 1), (77, 45, 13), (200, 200, 2668), (200, 2668, 200), (300, 130, 40),
          (129, 65, 33)]


@pytest.fixture(scope="module")
def ctx():
    import paper_1802_06738_gb300 as pkg
    pkg.build()
    c = pkg.Context(0)
    assert c.device_status(clear=True) == 0
    return c


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tf32x3_gemm_matches_fp64(ctx, M, N, K):
    rng = np.random.default_rng(M * 7919 + N * 31 + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    alpha = -0.75
    dA = torch.tensor(A, device="cuda:0")
    dB = torch.tensor(B, device="cuda:0")
    dC = torch.tensor(C0, device="cuda:0")
    ctx.gemm_tf32x3(dA, dB, dC, alpha)
    torch.cuda.synchronize()
    got = dC.cpu().numpy().astype(np.float64)
    ref = C0.astype(np.float64) + alpha * (A.astype(np.float64) @ B.astype(np.float64))
    scale = abs(alpha) * (np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)) + np.abs(ref)
    err = np.abs(got - ref)
    tol = 3e-6 + 3.0 * np.sqrt(K) * 2.0 ** -24
    assert np.all(err <= tol * scale + 1e-30), float((err / scale).max())
    assert ctx.device_status(clear=True) == 0


def test_tf32x3_beats_plain_tf32(ctx):
    """The split keeps far more than the 10 mantissa bits of a single tf32 product."""
    rng = np.random.default_rng(3)
    M, N, K = 128, 64, 256
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    dC = torch.zeros((M, N), device="cuda:0")
    ctx.gemm_tf32x3(torch.tensor(A, device="cuda:0"), torch.tensor(B, device="cuda:0"), dC)
    torch.cuda.synchronize()
    ref = A.astype(np.float64) @ B.astype(np.float64)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    rel = (np.abs(dC.cpu().numpy() - ref) / scale).max()
    assert rel < 5e-6
