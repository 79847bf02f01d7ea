"""A few sigma calls on one synthetic system, as a short program for profilers.

    python -m paper_1802_06738_gb300.profile_sigma --o 20 --v 200 --naux 600 --seed 1 \\
        --roots 6 --precision BF16 --calls 3

builds the system (occupied and virtual orbital energies and DF factors from the seeded
generator, MP1 amplitudes, state-averaged PNOs of `--roots` CIS(D) densities at
`--t-pno`), then calls sigma `--calls` times on `--roots` random vectors in the given
precision and prints the device status word.  Under ncu, select one launch with
`-k regex:<kernel> -s <launches to skip> -c 1`; each sigma call launches every kernel
of the program once (the setup launches others before them).
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--o", type=int, default=20)
    ap.add_argument("--v", type=int, default=200)
    ap.add_argument("--naux", type=int, default=600)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--roots", type=int, default=6)
    ap.add_argument("--t-pno", type=float, default=1e-7)
    ap.add_argument("--precision", default="BF16", choices=["FP64", "FP32", "BF16"])
    ap.add_argument("--calls", type=int, default=3)
    args = ap.parse_args(argv)

    import torch
    import paper_1802_06738_gb300 as pkg
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from synthetic import make_system

    prec = getattr(pkg, args.precision)
    ctx = pkg.Context(0)
    s = make_system(args.o, args.v, args.naux, args.seed)
    gp = pkg.PNO(ctx, s["eps"], s["B"], args.o, opts=pkg.make_opts(t_pno=args.t_pno, nroots=args.roots,
                                                                   precision=prec))
    dt = torch.float64 if prec == pkg.FP64 else torch.float32
    rng = np.random.default_rng(args.seed)
    R = torch.tensor(rng.standard_normal((args.roots, gp.length)), dtype=dt, device="cuda:0")
    S = torch.zeros_like(R)
    for _ in range(args.calls):
        gp.sigma(R, S, precision=prec)
    torch.cuda.synchronize()
    status = ctx.device_status()
    print(f"{args.calls} sigma calls, {args.roots} vectors of length {gp.length}, {args.precision}; "
          f"device status {status}")
    return 0 if status == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
