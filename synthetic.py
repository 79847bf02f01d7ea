"""Seeded synthetic inputs for state-averaged PNO-EOM-CCSD.

This module is the only code shared by the CUDA path and the CPU oracle.  It
draws random numbers and nothing else: no integral, amplitude or energy is
computed here.

Recipe (closed-shell RHF system of ``o`` occupied and ``v`` virtual spatial
orbitals, ``naux`` density-fitting functions):

* orbital energies: occupied uniform in [-1.5, -0.3] Eh, virtual uniform in
  [0.1, 3.0] Eh, each block sorted ascending (occupied first, so orbital
  index p = 0..o-1 is occupied and p = o..o+v-1 virtual);
* density-fitting factors B[Q, p, q] = 0.05 * (Z + Z^T)/2 *
  exp(-0.1 |p - q|) * exp(-4 Q / naux) with Z[Q, p, q] ~ N(0, 1); p, q and Q
  are 0-based, so B is symmetric in (p, q);
* draw order from one NumPy PCG64 stream seeded with ``seed``: occupied
  energies, virtual energies, then Z.

The recipe mimics a molecular RI factorisation: the envelope in |p - q| gives
decaying couplings between distant orbitals, the one in Q a decaying
auxiliary spectrum.
"""
from __future__ import annotations

import numpy as np

__all__ = ["make_system", "make_trial_vectors", "CONFIGS"]


def make_system(o: int, v: int, naux: int, seed: int) -> dict:
    """Return ``{"o", "v", "naux", "eps", "B"}`` for one synthetic system.

    ``eps`` is float64[o+v]; ``B`` is float64[naux, o+v, o+v], C-contiguous.
    """
    if o < 1 or v < 1 or naux < 1:
        raise ValueError("o, v and naux must be positive")
    rng = np.random.Generator(np.random.PCG64(seed))
    eps_o = np.sort(rng.uniform(-1.5, -0.3, size=o))
    eps_v = np.sort(rng.uniform(0.1, 3.0, size=v))
    nmo = o + v
    z = rng.standard_normal(size=(naux, nmo, nmo))
    z = 0.5 * (z + z.transpose(0, 2, 1))
    p = np.arange(nmo)
    env_pq = np.exp(-0.1 * np.abs(p[:, None] - p[None, :]))
    env_q = np.exp(-4.0 * np.arange(naux) / naux)
    B = 0.05 * z * env_pq[None, :, :] * env_q[:, None, None]
    return {"o": o, "v": v, "naux": naux,
            "eps": np.concatenate([eps_o, eps_v]),
            "B": np.ascontiguousarray(B)}


def make_trial_vectors(n: int, length: int, seed: int) -> np.ndarray:
    """``n`` seeded N(0,1) vectors of ``length`` entries (float64[n, length])."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size=(n, length))


# The five workloads: (o, v, naux, roots, T_PNO, seed).  System s of the
# batched workload draws o from seed 4 and uses seed 4000 + s.
CONFIGS = {
    "small": dict(o=5, v=20, naux=60, nroots=3, t_pno=1e-7, seed=1),
    "medium": dict(o=20, v=200, naux=600, nroots=6, t_pno=1e-7, seed=2),
    "large": dict(o=60, v=600, naux=1800, nroots=6, t_pno=1e-7, seed=3),
}


def batched_sizes(nsys: int = 64, seed: int = 4) -> list:
    """(o, v, naux, seed) of the batched workload: o ~ U{5..30}, v = 10 o,
    naux = 3 v, system s seeded with 4000 + s."""
    rng = np.random.Generator(np.random.PCG64(seed))
    os_ = rng.integers(5, 31, size=nsys)
    return [(int(o), 10 * int(o), 30 * int(o), 4000 + s) for s, o in enumerate(os_)]


def poisson_requests(n: int = 600, rate: float = 20.0, seed: int = 5) -> list:
    """Arrival stream of the serving workload: Poisson arrivals of mean
    ``rate``/s; o ~ U{5..40}, v = 10 o, naux = 3 v, roots ~ U{3,6,10},
    T_PNO ~ U{1e-6, 1e-7}; request r seeded with 5000 + r."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    o = rng.integers(5, 41, size=n)
    roots = rng.choice([3, 6, 10], size=n)
    tp = rng.choice([1e-6, 1e-7], size=n)
    return [dict(t=float(t[r]), o=int(o[r]), v=10 * int(o[r]), naux=30 * int(o[r]),
                 nroots=int(roots[r]), t_pno=float(tp[r]), seed=5000 + r)
            for r in range(n)]
