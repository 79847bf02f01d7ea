#!/usr/bin/env python
"""Benchmark of the GB300 state-averaged PNO-EOM-CCSD engine.

Workload (one GPU, default): the large synthetic system, o = 60 occupied, v = 600
virtual, naux = 1800 density-fitting functions, 6 roots, T_CutPNO = 1e-7, T2 from
Eq. T1 (seed 3 of the generator in synthetic.py).  A step is one sigma evaluation of
all 6 roots with the PNO-space operators resident in HBM; the metric is
sigma-evaluations per second (one sigma-eval = Hbar applied to one root vector).  The
headline runs the mixed path (BF16 dense blocks, FP32 arithmetic, the precision the
Davidson solve uses before its FP64 refinement); the plain FP64 path, full Davidson
solves (BF16 + FP64 refinement, and plain FP64) with their latencies and energies, and
the setup time are reported beside it.  --workload medium runs the medium system
(o = 20, v = 200, naux = 600, seed 2) with the FP32 mixed path.

Multi-GPU: every rank solves its own replica of the workload (independent
systems, no collective on the data path); value = all ranks' sigma-evals /
max-over-ranks time ("scaling": "weak").

--impl reference times the FP64 CPU oracle (oracle/) on the host cores on the same
workload and metric when the oracle can reach a sigma of that workload within the run's
limits; each step is one oracle sigma-eval of one root vector, after an untimed oracle
setup.  Otherwise it prints the reason as its "unavailable" line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "large": dict(o=60, v=600, naux=1800, nroots=6, t_pno=1e-7, seed=3, mixed="BF16", solves=1),
    "medium": dict(o=20, v=200, naux=600, nroots=6, t_pno=1e-7, seed=2, mixed="FP32", solves=3),
    "small": dict(o=5, v=20, naux=60, nroots=3, t_pno=1e-7, seed=1, mixed="FP32", solves=3),
}
# the metric as the benchmark's specification words it (both arms print it unchanged)
METRIC = "PNO-EOM-CCSD \u03c3-evals/s & solve p50/p99, mixed vs FP64 GPU path, |\u0394E|\u22641e-5 Eh"
# the oracle's sigma needs the canonical intermediates of the system, which it can hold
# and form in a bounded time only up to the medium workload
ORACLE_WORKLOADS = ("small", "medium")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=list(WORKLOADS))
    ap.add_argument("--solves", type=int, default=0, help="repeated Davidson solves for latency percentiles "
                                                          "(0: the workload's default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solves", action="store_true", help="skip the Davidson solves (profiling runs of the sigma steps)")
    ap.add_argument("--mixed", default="", choices=["", "BF16", "FP32"],
                    help="precision of the mixed sigma (default: the workload's own)")
    ap.add_argument("--mode", default="sigma", choices=["sigma", "batched", "serving"],
                    help="sigma: medium-workload sigma throughput (default); batched: many systems in one "
                         "launch sequence; serving: Poisson request stream through the continuous-batching server")
    ap.add_argument("--nsys", type=int, default=16, help="batched: number of systems (sample of the 64-system workload)")
    ap.add_argument("--omax", type=int, default=14, help="batched/serving: cap on o of the sampled systems")
    ap.add_argument("--nreq", type=int, default=40, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=20.0, help="serving: mean arrivals per second of the stream")
    ap.add_argument("--arms", default="mixed", help="serving: comma-separated arms to run on the same stream, "
                                                    "'mixed' and/or 'fp64' (the plain FP64 GPU path)")
    ap.add_argument("--serve-mixed", default="FP32", choices=["FP32", "BF16"],
                    help="serving: sigma precision of the mixed arm (FP64 refinement follows)")
    return ap.parse_args(argv)


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi clock / throttle sampling (every 50 ms, each line time-stamped on
    arrival by a reader thread).  Start it before the warm-up so the first samples exist
    when the timed region begins; mark() the region, and summary() keeps the samples
    inside it (or, for a region shorter than the sampling period, the nearest ones)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.rows = []                 # (arrival time, csv fields)
        self.window = None
        # raw samples (the JSON line carries their summary); PNOEOM_CLOCKS_DIR picks the folder
        import tempfile
        self.path = os.path.join(os.environ.get("PNOEOM_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"pnoeom_clocks_{os.getpid()}.csv")

    def _read(self):
        import time as _t
        with open(self.path, "w") as f:
            for line in self.proc.stdout:
                f.write(line)
                self.rows.append((_t.time(), [x.strip() for x in line.strip().split(",")]))

    def __enter__(self):
        import threading
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def wait_first(self, limit_s=5.0):
        """Block (at most limit_s) until the sampler has produced its first line."""
        import time as _t
        t_end = _t.time() + limit_s
        while self.proc is not None and not self.rows and _t.time() < t_end:
            _t.sleep(0.01)
        return self

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = list(self.rows)
        inside = rows
        where = "timed region"
        if self.window is not None:
            t0, t1 = self.window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if not inside and rows:   # region shorter than the sampling period: nearest samples
                rows.sort(key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))
                inside = rows[:2]
                where = "nearest to the timed region"
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, r in inside:
            try:
                sm.append(float(r[1])); smax = float(r[2])
                for nm, val in zip(names, r[5:9]):
                    if "Active" in val and "Not" not in val:
                        reasons.add(nm)
            except (ValueError, IndexError):
                pass
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "window": where}


def oracle_setup(w):
    """The oracle's PNO-space sigma for the workload (host, FP64)."""
    import numpy as np
    from synthetic import make_system
    from oracle import ccsd, eom, hamiltonian as hm, pno
    s = make_system(w["o"], w["v"], w["naux"], w["seed"])
    eps, B, o, v = s["eps"], s["B"], w["o"], w["v"]
    t2 = ccsd.mp1_t2(eps, B, o)
    sig = eom.Sigma(np.zeros((o, v)), t2, hm.hcore_from_fock(eps, B, o), B, o)
    sp = pno.PNOSpace(eps, B, o, w["nroots"], w["t_pno"])
    return sp, pno.PNOSigma(sig, sp)


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


# kernel classes that run on the tensor cores, per mixed precision (the rest run on the
# SIMT pipes or stream dense blocks): the E3 products (cuBLAS, TF32 in the BF16 sigma,
# the 3xTF32 tile kernel in the FP32 sigma) and, in the BF16 sigma, the sandwich terms
# (tcgen05 kind::f16 with BF16 operands)
TENSOR_CLASSES = {"BF16": {"sandwich->sigma": "bf16", "gemm->sigma": "tf32", "gemm->intermediates": "tf32"},
                  "FP32": {"gemm->sigma": "tf32", "gemm->intermediates": "tf32"}}


def roofline(dom, steps, peaks, dev_peaks, clk, mixed):
    """Roofline entry of the dominant kernel class.  The peak is the one of the unit the
    class runs on: the BF16 tensor rate of MEASURED_PEAKS.json (the sustained figure: the
    class is timed inside a loop of whole sigma calls) for the BF16 tensor-core class, half
    of it (the nominal TF32:BF16 ratio) for TF32 classes, the FP32 FMA rate measured by
    pnoeom_measure_peaks for SIMT contraction classes, and the HBM copy bandwidth of
    MEASURED_PEAKS.json for streaming classes; which bound applies is decided by the class's
    arithmetic intensity against the ridge.  The device's own tcgen05 BF16 microbenchmark
    is given beside it."""
    hbm, src = (peaks.get("hbm_gbs"), "of measured (MEASURED_PEAKS.json hbm_gbs)") if peaks.get("hbm_gbs") \
        else (6800.0, "of fallback")
    fp32 = dev_peaks.get("fp32_fma_tflops") or 0.0
    if peaks.get("bf16_tflops_sustained"):
        bf16, bsrc = peaks["bf16_tflops_sustained"], "of measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
    elif peaks.get("bf16_tflops"):
        bf16, bsrc = peaks["bf16_tflops"], "of measured (MEASURED_PEAKS.json bf16_tflops)"
    else:
        bf16, bsrc = 1900.0, "of fallback"
    kind = TENSOR_CLASSES.get(mixed, {}).get(dom["name"])
    avg_ms = dom["ms"] / steps
    intensity = dom["flops"] / max(dom["bytes"], 1.0)
    if kind == "bf16":
        alu, asrc = bf16, bsrc
    elif kind == "tf32":
        alu, asrc = bf16 / 2.0, bsrc + " x 1/2 (nominal TF32:BF16 ratio)"
    else:
        alu, asrc = fp32, "of measured: FP32 FMA (SIMT) by pnoeom_measure_peaks"
    ridge = alu * 1e12 / (hbm * 1e9) if alu else float("inf")
    common = {"kernel": dom["name"], "algorithmic_bytes_per_call": dom["bytes"], "algorithmic_flops_per_call": dom["flops"],
              "avg_ms_per_call": avg_ms, "launches_per_call": dom["launches"] / steps,
              "intensity_flop_per_byte": intensity, "ridge_flop_per_byte": ridge}
    tflops = dom["flops"] / (avg_ms * 1e-3) / 1e12
    if intensity > ridge:
        out = {"bound": "tensor" if kind else "alu", "achieved": tflops, "peak": alu, "unit": "TFLOP/s",
               "frac": tflops / alu, "peak_source": asrc, **common}
    else:
        ach = dom["bytes"] / (avg_ms * 1e-3) / 1e9
        out = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "peak_source": src, **common}
    dev_bf16 = dev_peaks.get("tc_bf16_tflops")
    if dev_bf16:
        out["vs_device_tcgen05_bf16"] = {"achieved_tflops": tflops, "peak_tflops": dev_bf16, "frac": tflops / dev_bf16,
                                         "peak_source": "of measured: tcgen05 kind::f16 issue-rate microbenchmark "
                                                        "(pnoeom_measure_peaks)"}
    return out


def fp64_roofline(prof, steps, peaks, dev_peaks):
    """Roofline entry of the dominant class of the FP64 sigma: the cuBLAS DGEMM rate
    measured by pnoeom_measure_peaks for the library-GEMM classes, the DFMA rate it
    measures for the other contraction classes, the HBM copy bandwidth of
    MEASURED_PEAKS.json for streaming classes (intensity against the ridge decides)."""
    dom = max(prof, key=lambda d: d["ms"])
    hbm, src = (peaks.get("hbm_gbs"), "of measured (MEASURED_PEAKS.json hbm_gbs)") if peaks.get("hbm_gbs") \
        else (6800.0, "of fallback")
    if dom["name"].startswith("gemm") and dev_peaks.get("cublas_dgemm_tflops"):
        alu, asrc = dev_peaks["cublas_dgemm_tflops"], "of measured: cuBLAS DGEMM by pnoeom_measure_peaks"
    else:
        alu, asrc = dev_peaks.get("fp64_fma_tflops") or 0.0, "of measured: FP64 FMA (SIMT) by pnoeom_measure_peaks"
    avg_ms = dom["ms"] / steps
    if avg_ms <= 0:
        return {"unavailable": "no class time was recorded"}
    intensity = dom["flops"] / max(dom["bytes"], 1.0)
    ridge = alu * 1e12 / (hbm * 1e9) if alu else float("inf")
    common = {"kernel": dom["name"], "algorithmic_bytes_per_call": dom["bytes"],
              "algorithmic_flops_per_call": dom["flops"], "avg_ms_per_call": avg_ms,
              "intensity_flop_per_byte": intensity, "ridge_flop_per_byte": ridge}
    if intensity > ridge:
        tf = dom["flops"] / (avg_ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": tf, "peak": alu, "unit": "TFLOP/s", "frac": tf / alu,
                "peak_source": asrc, **common}
    ach = dom["bytes"] / (avg_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "peak_source": src, **common}


def ncu_traffic(cls, workload, mixed):
    """DRAM bytes per sigma call of kernel class `cls` from the committed ncu summary (a
    line "traffic per call (bytes): <class> = <bytes>"), or None.  The summary records the
    sha256 of the kernel source it was captured with ("kernel source sha256: <hex>"); once
    that source has changed the counters no longer describe the kernel and None is returned."""
    import hashlib
    import re
    f = os.path.join(ROOT, "profiles", f"sigma_traffic_{workload}.md")
    kfile = "sandwich_tc.cu" if (mixed == "BF16" and cls == "sandwich->sigma") else "sigma_kernels.cu"
    src = os.path.join(ROOT, "paper_1802_06738_gb300", "csrc", kfile)
    if not os.path.exists(f) or not os.path.exists(src):
        return None
    text = open(f).read()
    h = re.search(r"kernel source sha256: ([0-9a-f]{64})", text)
    if h is None or h.group(1) != hashlib.sha256(open(src, "rb").read()).hexdigest():
        return None
    for line in text.splitlines():
        m = re.match(r"traffic per call \(bytes\): (\S+) = (\d+)", line.strip())
        if m and m.group(1) == cls:
            return float(m.group(2))
    return None


def cpu_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def workload_name(name, w):
    return (f"{name}: o={w['o']} v={w['v']} naux={w['naux']} roots={w['nroots']} T_PNO={w['t_pno']} "
            f"MP1 T2 (seed {w['seed']})")


def oracle_unavailable(name):
    return (f"the FP64 oracle's canonical sigma for the {name} workload needs its three- and four-virtual "
            "intermediates (about 100 GB for the v^3 o integrals at o=60, v=600); its per-pair sigma (O2) avoids "
            "them but needs the oracle's PNO construction (11 to 70 minutes on 8 host cores) and its setup "
            "before the first sample, and then about two minutes per pair block, so no bounded sample of it "
            "fits this run")


def run_reference(args, ws, rank):
    """Oracle arm: FP64 CPU sigma-evals/s on the host cores."""
    if rank != 0:
        return
    import numpy as np
    w = WORKLOADS[args.workload]
    if args.workload not in ORACLE_WORKLOADS:
        print(json.dumps({"impl": "reference", "metric": METRIC, "unavailable": oracle_unavailable(args.workload),
                          "config": {"workload": workload_name(args.workload, w)}}), flush=True)
        return
    t0 = time.time()
    sp, ps = oracle_setup(w)
    setup_s = time.time() - t0
    rng = np.random.default_rng(0)
    x = sp.symmetrize(rng.standard_normal(sp.length))
    for _ in range(min(args.warmup, 1)):
        ps(x)
    # one oracle sigma-eval takes tens of seconds: time at most 3 of them so the
    # arm ends within a few minutes ("steps" reports the number timed)
    nsteps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(nsteps):
        ps(x)
    dt = time.perf_counter() - t0
    requested = args.steps
    args.steps = nsteps
    val = args.steps / dt
    cores = cpu_threads()
    line = {"impl": "reference", "metric": METRIC,
            "value": val, "unit": "sigma-evals/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "steps_note": f"{requested} requested; the CPU oracle times at most 3 sigma-evals of one root",
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.workload, w), "vec_len": int(sp.length)},
            "cpu_baseline": {"value": val, "unit": "sigma-evals/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} oracle sigma-evals of one root vector after a {setup_s:.0f} s untimed setup"},
            "e2e": {"value": val, "unit": "sigma-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args, ws, rank, local):
    """Many systems in one launch sequence (a sample of the 64-system workload)."""
    import numpy as np
    import torch
    import paper_1802_06738_gb300 as pkg
    from synthetic import make_system, batched_sizes
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    if rank == 0:
        pkg.build()
    barrier(ws)
    sizes = [x for x in batched_sizes(64, 4) if x[0] <= args.omax][: args.nsys]
    ctx = pkg.Context(local)
    stream = torch.cuda.Stream(dev)
    h = stream.cuda_stream
    t0 = time.perf_counter()
    pnos = []
    for (o, v, naux, seed) in sizes:
        sd = make_system(o, v, naux, seed + 1000 * rank)
        pnos.append(pkg.PNO(ctx, sd["eps"], sd["B"], o, opts=pkg.make_opts(t_pno=1e-7, nroots=6, precision=pkg.FP32,
                                                                          refine_fp64=1), stream=h))
    build_s = time.perf_counter() - t0
    batch = pkg.Batch(ctx, pnos, stream=h)
    nr = 6
    rng = np.random.default_rng(3)
    rs = [torch.tensor(rng.standard_normal((nr, p.length)), dtype=torch.float32, device=dev) for p in pnos]
    outs = [torch.empty_like(r) for r in rs]
    with torch.cuda.stream(stream), Clocks(local) as clk:
        clk.wait_first()
        for _ in range(args.warmup):
            batch.sigma(rs, outs, precision=pkg.FP32, stream=h)
        stream.synchronize()
        barrier(ws)
        ev0 = torch.cuda.Event(enable_timing=True); ev1 = torch.cuda.Event(enable_timing=True)
        tw0 = time.time()
        ev0.record(stream)
        for _ in range(args.steps):
            batch.sigma(rs, outs, precision=pkg.FP32, stream=h)
        ev1.record(stream)
        stream.synchronize()
        clk.mark(tw0, time.time())
    t_sig = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, dev)
    # lockstep batched solve (mixed + FP64 refinement) vs the same systems one after another
    t0 = time.perf_counter()
    e, rn, it, cv = batch.solve(pkg.make_opts(t_pno=1e-7, nroots=nr, precision=pkg.FP32, refine_fp64=1), stream=h)
    t_batch_solve = time.perf_counter() - t0
    t0 = time.perf_counter()
    for p in pnos:
        p.davidson_solve(pkg.make_opts(t_pno=1e-7, nroots=nr, precision=pkg.FP32, refine_fp64=1), stream=h)
    t_serial_solve = time.perf_counter() - t0
    if rank != 0:
        return
    line = {"metric": "batched PNO-EOM-CCSD sigma-evals/s (all systems in one launch sequence, mixed FP32 sigma)",
            "value": ws * len(pnos) * nr * args.steps / t_sig, "unit": "sigma-evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_sig / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched sample: {len(pnos)} systems of the 64-system stream (o <= {args.omax}), "
                                   "v=10o, naux=3v, 6 roots, T_PNO=1e-7, MP1 T2",
                       "o_values": [x[0] for x in sizes], "vec_len_total": int(sum(p.length for p in pnos))},
            "solve": {"batched_lockstep_s": t_batch_solve, "one_after_another_s": t_serial_solve,
                      "converged": int(sum(cv)), "iterations": it, "build_total_s": build_s},
            "clocks": clk.summary(), "gpu_launches": None, "cpu_baseline": None}
    print(json.dumps(line), flush=True)


def serving_stream(nreq, omax, rate, seed=5, n=600):
    """The requests the serving mode submits: the first `nreq` requests with o <= omax of
    the 600-request Poisson stream, each at its own arrival time in that stream (so with
    omax >= 40 and nreq = 600 it is the whole stream; a filter thins it, and the offered
    rate is what remains)."""
    from synthetic import poisson_requests
    return [r for r in poisson_requests(n, rate, seed) if r["o"] <= omax][:nreq]


def serve_arm(pkg, ctx, reqs, systems, precision, refine):
    """One pass of the request stream through a fresh server; per-request times and stats."""
    import numpy as np
    srv = pkg.Server(ctx, hbm_budget_bytes=200 << 30, max_active=32)
    t0 = time.perf_counter()
    ids = []
    for k, r in enumerate(reqs):
        delay = r["t"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        opts = pkg.make_opts(t_pno=r["t_pno"], nroots=r["nroots"], precision=precision, refine_fp64=refine)
        ids.append(srv.submit(systems[k]["eps"], systems[k]["B"], r["o"], opts))
    for rid in ids:
        srv.wait(rid, 3600.0)
    wall = time.perf_counter() - t0
    res = [srv.poll(rid) for rid in ids]
    st = srv.stats()
    srv.close()
    tm = np.array([x["times"] for x in res])
    pct = lambda a: {"p50_s": float(np.percentile(a, 50)), "p99_s": float(np.percentile(a, 99))}
    sev = sum(x["sigma_evals"] for x in res)
    return {"wall_s": wall, "sigma_evals": sev, "sigma_evals_per_s": sev / wall,
            "latency": pct(tm[:, 3] - tm[:, 0]), "queueing": pct(tm[:, 1] - tm[:, 0]),
            "build": pct(tm[:, 2] - tm[:, 1]), "solve": pct(tm[:, 3] - tm[:, 2]),
            "achieved_rate_per_s": len(reqs) / wall,
            "completed": sum(1 for x in res if x["status"] == pkg.DONE), "server": st}


def run_serving(args, ws, rank, local):
    """Poisson request stream through the continuous-batching server, once per arm."""
    import torch
    import paper_1802_06738_gb300 as pkg
    from synthetic import make_system
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    if rank == 0:
        pkg.build()
    barrier(ws)
    reqs = serving_stream(args.nreq, args.omax, args.rate)
    systems = [make_system(r["o"], r["v"], r["naux"], r["seed"] + 1000 * rank) for r in reqs]
    ctx = pkg.Context(local)
    arms = [a.strip() for a in args.arms.split(",") if a.strip()]
    mixed = getattr(pkg, args.serve_mixed)
    out = {}
    with Clocks(local) as clk:
        clk.wait_first()
        tw0 = time.time()
        for arm in arms:
            barrier(ws)
            if arm == "mixed":
                out[arm] = serve_arm(pkg, ctx, reqs, systems, mixed, 1)
            elif arm == "fp64":
                out[arm] = serve_arm(pkg, ctx, reqs, systems, pkg.FP64, 0)
            else:
                raise SystemExit(f"unknown serving arm {arm!r}")
            out[arm]["wall_s"] = max_over_ranks(out[arm]["wall_s"], ws, dev)
        clk.mark(tw0, time.time())
    if rank != 0:
        return
    head = out[arms[0]]
    span = reqs[-1]["t"] if reqs else 0.0
    line = {"metric": f"served PNO-EOM-CCSD solves: latency p50/p99 and sigma-evals/s ({arms[0]} arm"
                      + (f": {args.serve_mixed} sigma + FP64 refinement)" if arms[0] == "mixed" else ": FP64 sigma)"),
            "value": ws * head["sigma_evals"] / head["wall_s"], "unit": "sigma-evals/s", "n_gpus": ws,
            "steps": len(reqs), "warmup": 0, "ms_per_step": 1e3 * head["wall_s"] / max(len(reqs), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if arms[0] == "fp64" else args.serve_mixed.lower(), "data": "synthetic",
            "config": {"workload": f"serving: {len(reqs)} requests of the 600-request Poisson stream (o <= {args.omax}) "
                                   f"at their own arrival times, stream rate {args.rate}/s, v=10o, naux=3v, "
                                   "roots in {3,6,10}, T_PNO in {1e-6,1e-7}",
                       "o_values": [r["o"] for r in reqs]},
            "offered_rate_per_s": len(reqs) / span if span > 0 else None,
            "arms": out, "clocks": clk.summary(), "gpu_launches": None, "cpu_baseline": None}
    if "mixed" in out and "fp64" in out:
        line["fp64_over_mixed"] = {"p50": out["fp64"]["latency"]["p50_s"] / out["mixed"]["latency"]["p50_s"],
                                   "p99": out["fp64"]["latency"]["p99_s"] / out["mixed"]["latency"]["p99_s"],
                                   "sigma_evals_per_s": out["fp64"]["sigma_evals_per_s"] / out["mixed"]["sigma_evals_per_s"]}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.mode == "batched":
        run_batched(args, ws, rank, local)
        return
    if args.mode == "serving":
        run_serving(args, ws, rank, local)
        return
    import numpy as np
    import torch
    import paper_1802_06738_gb300 as pkg
    from synthetic import make_system

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    if rank == 0:
        pkg.build()
    barrier(ws)
    w = dict(WORKLOADS[args.workload])
    if args.mixed:
        w["mixed"] = args.mixed
    o, nr = w["o"], w["nroots"]
    MIX = getattr(pkg, w["mixed"])
    nsolves = args.solves if args.solves > 0 else w["solves"]
    s = make_system(w["o"], w["v"], w["naux"], w["seed"] + 1000 * rank)
    ctx = pkg.Context(local)
    stream = torch.cuda.current_stream(dev).cuda_stream
    dev_peaks = ctx.measure_peaks(stream) if rank == 0 else {}
    opts_mixed = pkg.make_opts(t_pno=w["t_pno"], nroots=nr, precision=MIX, refine_fp64=1, max_iter=300)
    gp = pkg.PNO(ctx, s["eps"], s["B"], o, opts=opts_mixed, stream=stream)
    del s
    build_s = gp.build_seconds
    L = gp.length

    # --- full Davidson solves: latency (mixed + FP64 refinement, and plain FP64)
    lat_mixed, lat_fp64 = [], []
    e_mixed = e_fp64 = e_low = e_low16 = None
    it_mixed = it_fp64 = None
    rn_mixed = rn_fp64 = None
    ev_mixed = ev_fp64 = {"fp32": 0, "fp64": 0}
    opts_fp64 = pkg.make_opts(t_pno=w["t_pno"], nroots=nr, precision=pkg.FP64, max_iter=300)
    for k in range(0 if args.no_solves else nsolves):
        torch.cuda.synchronize(); t0 = time.perf_counter()
        e_mixed, rn_mixed, it_mixed, conv_m = gp.davidson_solve(opts_mixed, stream=stream)
        torch.cuda.synchronize(); lat_mixed.append(time.perf_counter() - t0)
        ev_mixed = gp.solve_stats()
        e_low = gp.lowprec_energies(pkg.FP32)
        e_low16 = gp.lowprec_energies(pkg.BF16) if w["mixed"] == "BF16" else []
        t0 = time.perf_counter()
        e_fp64, rn_fp64, it_fp64, conv_64 = gp.davidson_solve(opts_fp64, stream=stream)
        torch.cuda.synchronize(); lat_fp64.append(time.perf_counter() - t0)
        ev_fp64 = gp.solve_stats()

    # --- timed sigma steps, operators resident in HBM (no per-kernel instrumentation)
    rng = np.random.default_rng(1 + rank)
    R64 = torch.tensor(rng.standard_normal((nr, L)), device=dev)
    R32 = R64.float()
    S32 = torch.empty_like(R32)
    S64 = torch.empty_like(R64)
    with Clocks(local) as clk:
        clk.wait_first()
        for _ in range(args.warmup):
            gp.sigma(R32, S32, precision=MIX, stream=stream)
        barrier(ws)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True); ev1 = torch.cuda.Event(enable_timing=True)
        nvtx_push("sigma_timed")   # lets a profiler select exactly the timed launches
        tw0 = time.time()
        ev0.record()
        for _ in range(args.steps):
            gp.sigma(R32, S32, precision=MIX, stream=stream)
        ev1.record()
        torch.cuda.synchronize()
        clk.mark(tw0, time.time())
        nvtx_pop()
    barrier(ws)
    t_mixed = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, dev)

    # per-class device times, in a separate loop (CUDA events around every kernel class)
    k_cls = max(3, min(args.steps, 20))
    gp.set_timing(True)
    for _ in range(k_cls):
        gp.sigma(R32, S32, precision=MIX, stream=stream)
    torch.cuda.synchronize()
    prof = gp.sigma_timing(nr, MIX)
    gp.set_timing(False)
    tc_exec = None     # executed MMA flops of the tensor-core sandwich kernel per call
    if w["mixed"] == "BF16":
        try:
            tc_exec = gp.tc_mma_flops() * nr
        except Exception:
            tc_exec = None

    # FP64 sigma steps
    k64 = max(3, args.steps // 4)
    for _ in range(max(1, args.warmup // 2)):
        gp.sigma(R64, S64, precision=pkg.FP64, stream=stream)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(k64):
        gp.sigma(R64, S64, precision=pkg.FP64, stream=stream)
    ev1.record()
    torch.cuda.synchronize()
    t_fp64 = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, ws, dev)
    # per-class times of the FP64 sigma, in a loop of their own (outside the timed region)
    k64c = 3
    try:
        gp.set_timing(True)
        for _ in range(k64c):
            gp.sigma(R64, S64, precision=pkg.FP64, stream=stream)
        torch.cuda.synchronize()
        prof64, prof64_err = gp.sigma_timing(nr, pkg.FP64), None
    except Exception as ex:    # reported in the line; the headline does not depend on it
        prof64, prof64_err = None, str(ex)
    finally:
        gp.set_timing(False)

    # end to end through the C ABI: host vectors in pinned memory, copies inside the timed region
    Rh = R32.cpu().pin_memory()
    Sh = torch.empty_like(Rh).pin_memory()
    Rd = torch.empty_like(R32)
    Sd = torch.empty_like(R32)
    k_e2e = max(3, args.steps // 2)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        Rd.copy_(Rh, non_blocking=True)
        gp.sigma(Rd, Sd, precision=MIX, stream=stream)
        Sh.copy_(Sd, non_blocking=True)
        torch.cuda.synchronize()
    t_e2e = max_over_ranks(time.perf_counter() - t0, ws, dev)

    # mixed (and FP32) vs FP64 sigma on the same vectors
    errs = {}
    gp.sigma(R64, S64, precision=pkg.FP64, stream=stream)
    for name in ("FP32", "BF16"):
        gp.sigma(R32, S32, precision=getattr(pkg, name), stream=stream)
        torch.cuda.synchronize()
        errs[name] = float((S32.double() - S64).abs().max() / S64.abs().max())
    st = ctx.device_status()

    if rank != 0:
        return
    value = ws * nr * args.steps / t_mixed
    peaks = {}
    pf = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pf):
        peaks = json.load(open(pf))
    dom = max(prof, key=lambda d: d["ms"])
    clocks = clk.summary()
    roof = roofline(dom, k_cls, peaks, dev_peaks, clocks, w["mixed"])
    roof["timing"] = f"class times from a separate loop of {k_cls} calls with CUDA events around each class"
    if tc_exec and dom["name"] == "sandwich->sigma" and roof.get("avg_ms_per_call"):
        ex_tf = tc_exec / (roof["avg_ms_per_call"] * 1e-3) / 1e12
        roof["executed_mma"] = {"flops_per_call": tc_exec, "over_algorithmic": tc_exec / max(dom["flops"], 1.0),
                                "tflops": ex_tf, "frac_of_peak": ex_tf / roof["peak"] if roof.get("unit") == "TFLOP/s" else None,
                                "note": "2 M N K over every MMA the kernel issues, padding included (pno_tc_mma_flops)"}
    roof["traffic"] = ncu_traffic(dom["name"], args.workload, w["mixed"])
    if roof["traffic"] is not None:
        roof["traffic_per"] = ("call, from the committed ncu summary profiles/sigma_traffic_" + args.workload +
                               ".md (dram__bytes_read.sum + dram__bytes_write.sum)")
        roof["traffic_over_algorithmic"] = roof["traffic"] / max(dom["bytes"], 1.0)
    cpu = None
    if not args.no_cpu_baseline and args.gpus == 1:
        if args.workload in ORACLE_WORKLOADS:
            t0 = time.time()
            sp, ps = oracle_setup(w)
            setup_s = time.time() - t0
            x = sp.symmetrize(np.random.default_rng(0).standard_normal(sp.length))
            t0 = time.perf_counter()
            ps(x)
            dt = time.perf_counter() - t0
            cpu = {"value": 1.0 / dt, "unit": "sigma-evals/s", "cores": cpu_threads(), "kind": "oracle",
                   "sample": f"1 oracle sigma-eval of one root vector of the same workload ({dt:.1f} s) after a "
                             f"{setup_s:.0f} s untimed oracle setup"}
        else:
            cpu = {"value": None, "unit": "sigma-evals/s", "cores": cpu_threads(), "kind": "oracle",
                   "unavailable": oracle_unavailable(args.workload)}
    golden = None
    gfile = os.path.join(ROOT, "tests", "golden", f"oracle_{args.workload}.json")
    if os.path.exists(gfile):
        gold = json.load(open(gfile))
        golden = {"n_ij_match": bool(np.array_equal(gp.n_ij, gold["n_ij"])),
                  "n_i_match": bool(np.array_equal(gp.n_i, gold["n_i"]))}
        if "energies" in gold and e_mixed is not None:
            golden.update({"oracle_energies": gold["energies"],
                           "abs_err_mixed_refined": [abs(a - b) for a, b in zip(e_mixed, gold["energies"])],
                           "abs_err_fp64": [abs(a - b) for a, b in zip(e_fp64, gold["energies"])]})
    lat = lambda xs: {"p50_s": float(np.percentile(xs, 50)), "p99_s": float(np.percentile(xs, 99)), "n": len(xs),
                      **({"note": f"percentiles of {len(xs)} solves: the p99 is their maximum"} if len(xs) < 100 else {})}

    def in_solve(ev, xs):   # sigma-evals of one whole solve (setup excluded) and their rate
        n = ev["fp32"] + ev["fp64"]
        return {"sigma_evals_lowprec": ev["fp32"], "sigma_evals_fp64": ev["fp64"],
                "sigma_evals_per_s": n / float(np.percentile(xs, 50))}
    if lat_mixed:
        solve_section = {"mixed_refined": {**lat(lat_mixed), "iterations": it_mixed, **in_solve(ev_mixed, lat_mixed),
                                        "energies": list(map(float, e_mixed)),
                                        "residual_norms": list(map(float, rn_mixed)),
                                        "unrefined_fp32_phase_energies": list(map(float, e_low)),
                                        "unrefined_fp32_phase_abs_err_vs_fp64": [abs(a - b) for a, b in zip(e_low, e_fp64)],
                                        "unrefined_bf16_phase_energies": list(map(float, e_low16)),
                                        "unrefined_bf16_phase_abs_err_vs_fp64": [abs(a - b) for a, b in zip(e_low16, e_fp64)]},
                      "fp64": {**lat(lat_fp64), "iterations": it_fp64, **in_solve(ev_fp64, lat_fp64),
                               "energies": list(map(float, e_fp64)), "residual_norms": list(map(float, rn_fp64))},
                      "max_abs_dE_mixed_vs_fp64": float(np.abs(np.asarray(e_mixed) - np.asarray(e_fp64)).max()),
                      "pno_build_s": build_s}
    else:
        solve_section = {"skipped": "--no-solves (profiling run)", "pno_build_s": build_s}
    gflop_call = sum(d["flops"] for d in prof) / 1e9
    launches_call = sum(d["launches"] for d in prof) / k_cls
    line = {
        "metric": METRIC, "value": value, "unit": "sigma-evals/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_mixed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if w["mixed"] == "BF16" else "f32", "data": "synthetic",
        "dtype_detail": ("sandwich terms: BF16 operands on tcgen05 tensor cores, FP32 accumulation; E3 products: "
                         "TF32 tensor cores; dense blocks: BF16 storage, FP32 arithmetic; vectors FP32")
        if w["mixed"] == "BF16" else "FP32 SIMT arithmetic; E3 products FP32",
        "config": {"workload": workload_name(args.workload, w), "mixed_precision": w["mixed"],
                   "vec_len": int(L), "n_ij_mean": float(np.mean(gp.n_ij)), "n_ij_max": int(np.max(gp.n_ij)),
                   "nonzero_pairs": int(np.sum(np.asarray(gp.n_ij) > 0)), "n_osv_total": int(np.sum(gp.n_i)),
                   "parallelism": f"replicas x{ws}", "l2": "operator pool larger than L2 (no flush)",
                   "device_footprint_bytes": int(gp.footprint)},
        "fp64_path": {"value": ws * nr * k64 / t_fp64, "unit": "sigma-evals/s", "steps": k64,
                      "ms_per_step": 1e3 * t_fp64 / k64, "kernels": prof64,
                      "roofline": fp64_roofline(prof64, k64c, peaks, dev_peaks) if prof64 else {"unavailable": prof64_err}},
        "sigma_max_rel_err_vs_fp64": errs,
        "solve": solve_section,
        "flop_weighted": {"gflop_per_call": gflop_call, "tflops": gflop_call / (t_mixed / args.steps) / 1e3,
                          "note": "algorithmic FLOPs of all sigma kernel classes per 6-root call / CUDA-event time"},
        "energy_check": golden,
        "e2e": {"value": ws * nr * k_e2e / t_e2e, "unit": "sigma-evals/s",
                "h2d_bytes_per_step": int(Rh.numel() * 4), "d2h_bytes_per_step": int(Sh.numel() * 4)},
        "roofline": roof,
        "kernels": prof,
        "device_peaks_measured": dev_peaks,
        "device_status": st,
        "autotune": dict(zip(["candidates_group_rpc_ms", "choice"], gp.autotune_info())),
        "gpu_launches": int(round(launches_call * args.steps)),
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
