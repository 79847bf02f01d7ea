"""Sampled sigma entries of the blockwise trial vector (tests/golden/make_golden.py).

Two helpers shared by the GPU test of the large workload, which compares the library's
sigma with the oracle's samples stored in tests/golden/oracle_large.json, and by a CPU
test that checks these helpers against the oracle itself on a small system.

A `space` is any object with the packed layout of Sec. 2's PNO/OSV vectors: o, v, n_i,
n_ij, off_i, off_ij and pairs (stored pairs i <= j in order).  `basis(k)` returns the
v x n basis of stored pair k (k >= 0) or the OSV basis of occupied -k - 1 (k < 0).
Entries are compared in the canonical basis, so the result does not depend on the
phases or the rotation of the vectors inside each PNO/OSV space.
"""
import numpy as np


def blockwise_vector(space, basis, r1, r2_block):
    """The canonical trial vector (singles r1[i], doubles blocks r2_block(v, i, j)) projected
    into the packed PNO/OSV layout of `space`."""
    vec = np.zeros(int(space.off_ij[-1]))
    for i in range(space.o):
        if space.n_i[i]:
            vec[space.off_i[i]:space.off_i[i + 1]] = basis(-i - 1).T @ r1[i]
    for p, (i, j) in enumerate(space.pairs):
        if space.n_ij[p]:
            U = basis(p)
            vec[space.off_ij[p]:space.off_ij[p + 1]] = (U.T @ r2_block(space.v, i, j) @ U).ravel()
    return vec


def sampled_entries(space, basis, sig, pair_samples, singles_samples):
    """(got, ref): the packed sigma `sig` back in the canonical basis at the sampled
    positions, and the stored values.  pair_samples: "i,j" -> [[a, b, value], ...] of pair
    block (i, j), i <= j; singles_samples: "i" -> [[a, value], ...] of singles row i."""
    index = {pq: p for p, pq in enumerate(space.pairs)}
    got, ref = [], []
    for key, ent in pair_samples.items():
        i, j = (int(t) for t in key.split(","))
        p = index[(i, j)]
        n = int(space.n_ij[p])
        U = basis(p)
        S = sig[space.off_ij[p]:space.off_ij[p + 1]].reshape(n, n)
        a = np.array([e[0] for e in ent], dtype=np.int64)
        b = np.array([e[1] for e in ent], dtype=np.int64)
        got.extend(np.einsum("kx,xy,ky->k", U[a], S, U[b]))
        ref.extend(float(e[2]) for e in ent)
    for key, ent in singles_samples.items():
        i = int(key)
        row = basis(-i - 1) @ sig[space.off_i[i]:space.off_i[i + 1]]
        got.extend(row[np.array([e[0] for e in ent], dtype=np.int64)])
        ref.extend(float(e[1]) for e in ent)
    return np.asarray(got), np.asarray(ref)
