"""Write oracle fixtures for the GPU tests and the benchmark.

Calls only oracle/ and the seeded generator.  For a workload it stores:
  * the PNO counts n_ij and n_i;
  * the Davidson excitation energies (the oracle's FP64 solve, Sec. 2);
  * sigma of one seeded canonical trial vector, projected (Sec. 2), for the
    singles and a sample of pair blocks, in the canonical basis (so the
    comparison does not depend on PNO phases).  For v > 32 each sampled pair
    block keeps SIGMA_SAMPLES entries at seeded positions instead of all v^2.

Usage: python tests/golden/make_golden.py medium   (about two hours on 8 cores)
       python tests/golden/make_golden.py large --pno-only
           (PNO/OSV counts and CIS energies of the large workload, ~10 minutes)
       python tests/golden/make_golden.py large --sigma-samples
           (per-pair oracle sigma of the blockwise trial vector: seeded entries of 16 pair
            blocks of every size class and of every singles row of the large workload,
            added to its fixture)
       python tests/golden/make_golden.py medium --sigma-samples --out=oracle_medium_blockwise.json
           (the same for the medium workload, in a file of its own)
       python tests/golden/make_golden.py medium --sigma-only
           (recomputes only the sigma fields of an existing fixture, ~2 minutes)
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from synthetic import make_system  # noqa: E402
from oracle import ccsd, davidson, eom, hamiltonian as hm, pno  # noqa: E402

WORKLOADS = {
    "small": dict(o=5, v=20, naux=60, nroots=3, t_pno=1e-7, seed=1, gs="ccsd"),
    "medium": dict(o=20, v=200, naux=600, nroots=6, t_pno=1e-7, seed=2, gs="mp1"),
    "large": dict(o=60, v=600, naux=1800, nroots=6, t_pno=1e-7, seed=3, gs="mp1"),
}
SAMPLE_PAIRS = {"small": [(0, 0), (0, 4), (2, 3), (4, 4)], "medium": [(0, 19), (5, 5), (7, 12), (18, 19), (19, 19)]}
SIGMA_SAMPLES = 256


def sigma_fields(s1, s2, pairs, v):
    """Sigma of the trial vector: singles whole, pair blocks whole (v <= 32) or sampled."""
    out = {"sigma_trial_seed": 123, "sigma_s1": s1.tolist()}
    if v <= 32:
        out["sigma_pairs"] = {f"{i},{j}": s2[i, j].tolist() for (i, j) in pairs}
    else:
        rng = np.random.default_rng(7)
        smp = {}
        for (i, j) in pairs:
            pos = rng.integers(0, v, size=(SIGMA_SAMPLES, 2))
            smp[f"{i},{j}"] = [[int(a), int(b), float(s2[i, j, a, b])] for a, b in pos]
        out["sigma_pair_samples"] = smp
    return out


def trial_vector(o, v, seed=123):
    """Seeded canonical trial vector (r1, symmetric r2)."""
    rng = np.random.default_rng(seed)
    r1 = rng.standard_normal((o, v))
    r2 = rng.standard_normal((o, o, v, v))
    return r1, 0.5 * (r2 + r2.transpose(1, 0, 3, 2))


def trial_r1(o, v, seed=321):
    """Seeded canonical singles of the blockwise trial vector."""
    return np.random.default_rng(seed).standard_normal((o, v))


def trial_r2_block(v, i, j, seed=321):
    """Canonical doubles block r2[i, j] (v x v) of the blockwise trial vector: pair i <= j
    draws from its own seeded stream, r2[j, i] = r2[i, j]^T, r2[i, i] symmetric."""
    a, b = min(i, j), max(i, j)
    x = np.random.default_rng([seed, a, b]).standard_normal((v, v))
    if a == b:
        x = 0.5 * (x + x.T)
    return x if i <= j else x.T


def sigma_sample_fields(w, npairs_whole=8, per_pair=8, per_row=16, t2=None, all_pairs=True):
    """Sigma of the blockwise trial vector by the per-pair oracle (oracle.pno_direct), in
    the canonical basis, for every non-empty pair block (or, with all_pairs=False, only the
    npairs_whole pairs below) and every singles row with OSVs:
      * npairs_whole pairs of every size class (sorted by n_ij, evenly spaced) keep
        SIGMA_SAMPLES seeded entries each, every other non-empty pair per_pair entries;
      * three occupied orbitals keep their whole singles row, the others per_row entries.
    w: a workload dict (o, v, naux, nroots, t_pno, seed); the ground state is MP1 unless
    t2 is given.  Returns the fixture fields."""
    from oracle.pno_direct import PNOSigmaDirect
    o, v = w["o"], w["v"]
    t0 = time.time()
    s = make_system(o, v, w["naux"], w["seed"])
    eps, B = s["eps"], s["B"]
    sp = pno.PNOSpace(eps, B, o, w["nroots"], w["t_pno"])
    sp.D = None                                               # densities not needed any more
    print(f"PNO spaces {time.time() - t0:.0f} s", flush=True)
    if t2 is None:
        t2 = ccsd.mp1_t2(eps, B, o)
    h = hm.hcore_from_fock(eps, B, o)
    o2 = PNOSigmaDirect(None, t2, h, B, o, sp)
    del s, B                                                  # O2 keeps its own blocks of B
    print(f"O2 setup {time.time() - t0:.0f} s", flush=True)
    r1 = trial_r1(o, v)
    vec = np.zeros(sp.length)
    for i in range(o):
        vec[sp.off_i[i]:sp.off_i[i + 1]] = sp.Ui[i].T @ r1[i]
    for p, (i, j) in enumerate(sp.pairs):
        if sp.n_ij[p]:
            U = sp.U[i, j]
            vec[sp.off_ij[p]:sp.off_ij[p + 1]] = (U.T @ trial_r2_block(v, i, j) @ U).ravel()
    nz = [int(p) for p in np.argsort(sp.n_ij, kind="stable") if sp.n_ij[p] > 0]
    whole = {nz[int(round(k * (len(nz) - 1) / (npairs_whole - 1)))] for k in range(npairs_whole)}
    occ = [i for i in range(o) if sp.n_i[i] > 0]
    occ_whole = {occ[0], occ[len(occ) // 2], occ[-1]}
    out_pairs = sorted(nz) if all_pairs else sorted(whole)
    sig = o2(vec, pairs=out_pairs, singles=occ)
    print(f"sigma of {len(out_pairs)} pair blocks and {len(occ)} singles rows {time.time() - t0:.0f} s", flush=True)
    rng = np.random.default_rng(7)
    smp, s1 = {}, {}
    for p in out_pairs:
        i, j = sp.pairs[p]
        U = sp.U[i, j]
        blk = U @ sig[sp.off_ij[p]:sp.off_ij[p + 1]].reshape(sp.n_ij[p], sp.n_ij[p]) @ U.T
        pos = rng.integers(0, v, size=(SIGMA_SAMPLES if p in whole else per_pair, 2))
        smp[f"{i},{j}"] = [[int(a), int(b), float(blk[a, b])] for a, b in pos]
    for i in occ:
        row = sp.Ui[i] @ sig[sp.off_i[i]:sp.off_i[i + 1]]
        cols = np.arange(v) if i in occ_whole else rng.integers(0, v, size=per_row)
        s1[str(i)] = [[int(a), float(row[a])] for a in cols]
    return {"n_ij": sp.n_ij.tolist(), "n_i": sp.n_i.tolist(),
            "sigma_trial": "blockwise (make_golden.trial_r1 / trial_r2_block, seed 321)",
            "sigma_pair_samples": smp, "sigma_singles_samples": s1, "sigma_seconds": time.time() - t0}


def sigma_samples(name, out=None):
    """Add the sigma samples of the blockwise trial vector to the workload's fixture (or to
    the fixture file `out` in this folder)."""
    path = os.path.join(HERE, out or f"oracle_{name}.json")
    if name == "large":   # O2 takes about a minute per pair block here: 16 blocks of every size class
        fields = sigma_sample_fields(WORKLOADS[name], npairs_whole=16, all_pairs=False)
    else:
        fields = sigma_sample_fields(WORKLOADS[name])
    fields.update({"workload": name, **{k: WORKLOADS[name][k] for k in ("o", "v", "naux", "nroots", "t_pno", "seed")}})
    out = json.load(open(path)) if os.path.exists(path) else {}
    out.update(fields)
    out.pop("sigma_singles_rows", None)
    json.dump(out, open(path, "w"))
    print(f"wrote sigma samples to {path}: {fields['sigma_seconds']:.0f} s", flush=True)


def pno_only(name):
    """PNO/OSV counts, CIS energies and the occupations nearest the thresholds
    (oracle PNO construction only; no sigma or solve)."""
    w = WORKLOADS[name]
    o = w["o"]
    t0 = time.time()
    s = make_system(o, w["v"], w["naux"], w["seed"])
    sp = pno.PNOSpace(s["eps"], s["B"], o, w["nroots"], w["t_pno"])
    tp, to = w["t_pno"], w["t_pno"] / 10.0
    near = lambda ev, t: float(np.min(np.abs(np.log10(np.maximum(np.abs(ev), 1e-300) / t))))
    out = {"workload": name, **{k: w[k] for k in ("o", "v", "naux", "nroots", "t_pno", "seed", "gs")},
           "n_ij": sp.n_ij.tolist(), "n_i": sp.n_i.tolist(), "vec_len": int(sp.length),
           "cis_energies": sp.cis_omega.tolist(),
           "closest_log10_gap_to_t_pno": min(near(sp.alleig[p], tp) for p in sp.pairs),
           "closest_log10_gap_to_t_osv": min(near(sp.alleig[(i, i)], to) for i in range(o)),
           "seconds": time.time() - t0}
    path = os.path.join(HERE, f"oracle_{name}.json")
    json.dump(out, open(path, "w"))
    print(f"wrote {path}: {time.time() - t0:.0f} s", flush=True)


def main(name, sigma_only=False):
    w = WORKLOADS[name]
    o, v = w["o"], w["v"]
    t0 = time.time()
    s = make_system(o, v, w["naux"], w["seed"])
    eps, B = s["eps"], s["B"]
    h = hm.hcore_from_fock(eps, B, o)
    if w["gs"] == "ccsd":
        t1, t2, _, _ = ccsd.solve_ccsd(eps, B, o)
    else:
        t1, t2 = np.zeros((o, v)), ccsd.mp1_t2(eps, B, o)
    sig = eom.Sigma(t1, t2, h, B, o)
    sp = pno.PNOSpace(eps, B, o, w["nroots"], w["t_pno"])
    ps = pno.PNOSigma(sig, sp)
    print(f"setup {time.time() - t0:.0f} s, L = {sp.length}", flush=True)
    r1, r2 = trial_vector(o, v)
    s1, s2 = sp.unpack(ps(sp.pack(r1, r2)))
    out = {"workload": name, **{k: w[k] for k in ("o", "v", "naux", "nroots", "t_pno", "seed", "gs")},
           "n_ij": sp.n_ij.tolist(), "n_i": sp.n_i.tolist(), "vec_len": int(sp.length),
           **sigma_fields(s1, s2, SAMPLE_PAIRS[name], v)}
    print(f"sigma done {time.time() - t0:.0f} s", flush=True)
    path = os.path.join(HERE, f"oracle_{name}.json")
    if sigma_only:   # keep the stored solve, replace the sigma fields
        old = json.load(open(path))
        for k in ("sigma_pairs", "sigma_pair_samples"):
            old.pop(k, None)
        old.update(out)
        json.dump(old, open(path, "w"))
        print(f"updated sigma fields of {path}", flush=True)
        return
    e, X, rn, it, conv = davidson.solve(ps, sp, w["nroots"])
    out.update({"energies": e.tolist(), "residual_norms": rn.tolist(), "iterations": int(it), "converged": bool(conv),
                "cis_energies": sp.cis_omega.tolist(), "seconds": time.time() - t0})
    json.dump(out, open(path, "w"))
    print(f"wrote {path}: energies {e}, converged {conv}, {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    if "--pno-only" in sys.argv:
        pno_only(args[0])
    elif "--sigma-samples" in sys.argv:
        outs = [a.split("=", 1)[1] for a in sys.argv[1:] if a.startswith("--out=")]
        sigma_samples(args[0], outs[0] if outs else None)
    else:
        main(args[0] if args else "small", sigma_only="--sigma-only" in sys.argv)
