#!/usr/bin/env python3
"""Benchmark of the GB300 asymmetric-plmDCA library.

One step = the whole hot path on one synthetic protein family (N = 120
positions, B = 5000 sequences, q = 21, planted chain contacts -- 168 of the
ceil(1.5 N) = 180 asked for, all the chain offers at seed 0 -- 15 % gaps): reweighting at 0.8 identity, the batched per-site L-BFGS solve of
every g_r^(reg) to ||grad|| <= 1e-4, then Ising gauge + average + FN + APC
and the top-N contact list.  The MSA is resident in HBM before the timed
region; L2 is flushed (a 256 MiB write) between timed steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (on host cores, a bounded sample of the same workload).
Multi-GPU runs (torchrun) are independent replicas (one family per rank).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "plmDCA full-solve seconds & objective+grad evals/s vs plain FP32 path at fixed error"
MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")


def workload_name(fam):
    return (f"synthetic protein family N={fam.N} B={fam.B} q=21 "
            f"({len(fam.model.pairs)} planted chain contacts, 15% gaps)")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="auto", choices=["auto", "fp32", "split_bf16"])
    ap.add_argument("--gtol", type=float, default=1e-4)
    ap.add_argument("--lbfgs-m", type=int, default=5, help="L-BFGS memory (curvature pairs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-cmp", action="store_true",
                    help="skip timing the plain FP32 path beside the split-bf16 one")
    ap.add_argument("--workload", default="family",
                    choices=["family", "batch", "scale", "eval", "symmetric", "scores",
                             "frontend"],
                    help="family: the benchmark line; batch (64 families), scale "
                         "(N=500, B=50000), eval (full objective+gradient evaluations "
                         "of the family at a random point) and symmetric (symmetric "
                         "plmDCA on the family): separate measurements")
    ap.add_argument("--cpu-sites", type=int, default=0,
                    help="sites per CPU-oracle sample (0: the reference arm takes two per host "
                         "core, at most 32; the CPU baseline of our arm runs the whole rundown)")
    return ap.parse_args()


def peaks():
    try:
        with open(MEASURED) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms.  Started before the
    warm-up (the tool needs ~0.1 s to begin); `window` marks the timed region
    on the host clock, and only the samples nvidia-smi stamped inside it are
    kept (or, for a region shorter than the sampling period, the sample
    nearest to it)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def window(self, t0, t1):
        self.t0, self.t1 = t0, t1

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return summarize_clocks(self.lines, self.t0, self.t1)


def summarize_clocks(lines, t0=None, t1=None):
    """Median SM clock, its maximum and the throttle reasons seen, over the
    nvidia-smi samples stamped within [t0, t1] (host wall-clock seconds);
    with none inside, the one nearest to the window."""
    import datetime
    rows = []
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 10:
            continue
        try:
            ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
        except ValueError:
            continue
    if t0 is not None and rows:
        inside = [r for r in rows if t0 <= r[0] <= t1]
        if not inside:
            inside = [min(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))]
        rows = inside
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = {n for r in rows for n, v in zip(names, r[3]) if v.lower().startswith("active")}
    sm = [r[1] for r in rows]
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(r[2] for r in rows) if rows else None,
            "reasons": sorted(reasons), "samples": len(sm)}


def cpu_sample(fam, n_sites, gtol):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    the full reweighting, the L-BFGS solve of `n_sites` site problems (the
    site problems are independent), and FN+APC on the full J; the solve time
    is scaled by N / n_sites to one full solve."""
    import numpy as np
    import oracle
    S = fam.msa
    N = S.shape[1]
    t0 = time.perf_counter()
    m, w, w32, beff = oracle.reweight(S, 0.8)
    t1 = time.perf_counter()
    sites = list(np.linspace(0, N - 1, n_sites).round().astype(int))
    h, J, info = oracle.solve(S, w, beff, 0.01, 0.01, gtol=gtol, sites=sites)
    t2 = time.perf_counter()
    fn, cfn = oracle.scores(J)
    oracle.topL(cfn, N, 5)
    t3 = time.perf_counter()
    full = (t1 - t0) + (t2 - t1) * N / len(sites) + (t3 - t2)
    evals = float(np.mean(info["nevals"]))
    return full, (t3 - t0), evals, len(sites)


def cpu_full_rundown(fam, gtol, gpu):
    """The oracle's whole rundown of the workload, timed on all host cores,
    and the last timed GPU solve compared with it: every pair's FN and CFN
    against the stated error bound (gradient norms of both points by the
    oracle, strong convexity mu = 2 min(lambda_h, lambda'_J)) and the top-L
    lists (exactly identical, or ties only inside the bound)."""
    import numpy as np
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity_bounds import cfn_bound, compare_top, fn_bound
    S = fam.msa
    t0 = time.perf_counter()
    ro = oracle.plmdca(S, gtol=gtol)
    wall = time.perf_counter() - t0
    parity = None
    if gpu:
        N = S.shape[1]
        h = gpu["h"].cpu().numpy().astype(np.float64)
        J = gpu["J"].cpu().numpy().astype(np.float64)
        _, gh, gJ = oracle.objgrad(S, ro["w"], ro["beff"], h, J, 0.01, 0.01)
        gn = np.sqrt((gh ** 2).sum(1) + (gJ ** 2).reshape(N, -1).sum(1))
        mu = 2 * min(0.01, 0.5 * 0.01)
        b = fn_bound(gn, ro["info"]["gnorm"], mu)
        fn_err = np.abs(gpu["fn"].cpu().numpy() - ro["fn"])
        e = cfn_bound(ro["fn"], b)
        cfn_err = np.abs(gpu["cfn"].cpu().numpy() - ro["cfn"])
        top = gpu["top"].cpu().numpy()[:len(ro["top"])]
        identical, ok, detail = compare_top(top, ro["top"], ro["cfn"], e)
        parity = {"top_L_identical": identical, "top_L_within_bound": ok, "detail": detail,
                  "fn_within_bound": bool(np.all(fn_err <= b + 1e-9)),
                  "max_fn_err": float(fn_err.max()), "max_fn_bound": float(b.max()),
                  "max_cfn_err": float(cfn_err.max()), "max_cfn_bound": float(e.max())}
    return wall, parity


def cpu_sample_single_thread(fam, n_sites, gtol):
    """The same oracle sample on one host thread (the timing protocol asks for
    one core beside all of them); the thread count is restored after."""
    import oracle
    cores = oracle.num_threads()
    oracle.set_threads(1)
    try:
        return cpu_sample(fam, n_sites, gtol)
    finally:
        oracle.set_threads(cores)


def measure_alu_peaks(lib, stream):
    """Measured CUDA-core instruction rates (instructions/s over the GPU):
    FP32 add, FP32 FMA, FP64 add, lop3, popc (plm_measure_peak)."""
    import ctypes
    out = {}
    for kind, name in enumerate(("fadd_f32", "ffma_f32", "dadd_f64", "lop3_b32", "popc_b32")):
        v = ctypes.c_double(0.0)
        st = lib.plm_measure_peak(kind, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(v))
        out[name] = v.value if st == 0 else None
    return out


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle
    from paper_1401_4832_gb300 import synth
    fam = synth.protein_family(seed=0)
    cores = oracle.num_threads()
    # two sites per core: OpenMP balances them, so the sample's wall time
    # scales to the full solve (with one site per core the slowest site would
    # set it)
    n_sites = args.cpu_sites or min(32, 2 * cores)
    for _ in range(args.warmup):
        cpu_sample(fam, max(1, n_sites // 4), args.gtol)
    vals, walls = [], []
    for _ in range(args.steps):
        full, wall, evals, ns = cpu_sample(fam, n_sites, args.gtol)
        vals.append(full)
        walls.append(wall)
    v = statistics.mean(vals)
    sample = (f"full reweighting + L-BFGS of {ns} of {fam.N} sites (gtol {args.gtol}) scaled "
              f"x{fam.N}/{ns} + full FN/APC/top-L, FP64 oracle, {cores} OpenMP threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * statistics.mean(walls), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(fam), "N": fam.N, "B": fam.B, "q": 21, "gtol": args.gtol,
                   "parallelism": "host cores (OpenMP over sites)"},
        "cpu_baseline": {"value": v, "unit": "s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_batch(args):
    """64 families (N ~ U{50..300}, B log-uniform in [500, 20000]) in one
    batched solve vs the same families solved one after another."""
    import torch
    from paper_1401_4832_gb300 import api, synth
    fams = synth.batch_families()
    stream = torch.cuda.Stream()
    ctx = api.Context(0, stream)
    msas = [torch.from_numpy(f.msa).cuda() for f in fams]
    out = {}
    with torch.cuda.stream(stream):
        for mode in ("batched", "one_by_one"):
            times = []
            for k in range(args.warmup + args.steps):
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if mode == "batched":
                    res = api.plm_solve_batch(ctx, msas, gtol=args.gtol)
                else:
                    res = [api.plm_solve(ctx, m, gtol=args.gtol) for m in msas]
                e1.record(stream)
                torch.cuda.synchronize()
                if k >= args.warmup:
                    times.append(e0.elapsed_time(e1) / 1000.0)
            out[mode] = {"s": statistics.mean(times),
                         "sites_not_converged": sum(r[2]["n_noise"] + r[2]["n_failed"] for r in res)}
    # one profiled batched solve: per-kernel device time
    from paper_1401_4832_gb300 import _native
    lib = _native.load()
    lib.plm_profile(ctx.handle, 1)
    with torch.cuda.stream(stream):
        res = api.plm_solve_batch(ctx, msas, gtol=args.gtol)
    kern = read_profile(lib, ctx)
    lib.plm_profile(ctx.handle, 0)
    print(json.dumps({"workload": "batch: 64 synthetic families, N~U{50..300}, B log-uniform [500,20000]",
                      "families": len(fams), "sum_N": sum(f.N for f in fams),
                      "sum_BN": sum(f.B * f.N for f in fams), "results": out,
                      "batched_speedup": out["one_by_one"]["s"] / out["batched"]["s"],
                      "evals_per_solve": res[0][2]["evals"],
                      "kernels_profiled_ms": {k: v[1] for k, v in kern.items()}}), flush=True)


def run_scale(args):
    """N=500, B=50000: device time per full evaluation of both precisions
    (CUDA events, median), and one full split-BF16 solve at that size
    (reweighting + L-BFGS of all 500 sites to gtol; the solve is tuned and
    warmed once first)."""
    import torch
    from paper_1401_4832_gb300 import api, synth
    fam = synth.scale_family()
    S = torch.from_numpy(fam.msa).cuda()
    stream = torch.cuda.Stream()
    ctx = api.Context(0, stream)
    N = fam.N
    out = {}

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / 1000.0, r

    with torch.cuda.stream(stream):
        m, w, beff = api.msa_reweight(ctx, S)
        h = torch.zeros((N, 21), device="cuda")
        J = torch.zeros((N, 21, N, 21), device="cuda")
        for prec in ("split_bf16", "fp32"):
            for _ in range(2):
                api.plm_site_objective_grad(ctx, S, w, beff, h, J, prec=prec)
            ts = [timed(lambda: api.plm_site_objective_grad(ctx, S, w, beff, h, J,
                                                            prec=prec))[0]
                  for _ in range(max(3, min(args.steps, 20)))]
            out[prec] = {"s_per_eval": statistics.median(ts)}
        del h, J
        api.plm_solve(ctx, S, gtol=args.gtol, prec="split_bf16")
        t, (hs, Js, rep) = timed(lambda: api.plm_solve(ctx, S, gtol=args.gtol,
                                                       prec="split_bf16"))
        out["split_bf16_full_solve"] = {"s": t, "evals": rep["evals"], "iters": rep["iters"],
                                        "sites_converged": rep["n_converged"],
                                        "gnorm_max": rep["gnorm_max"], "gtol": args.gtol}
    print(json.dumps({"workload": "scale: N=500 B=50000 q=21 (750 chain contacts, 20% gaps)",
                      "results": out}), flush=True)
    ctx.close()


def run_eval(args):
    """Full evaluations (every site) of the family workload at a random
    point: device time per evaluation with L2 flushed before each (also the
    small case the kernel captures run on)."""
    import numpy as np
    import torch
    from paper_1401_4832_gb300 import api, synth
    fam = synth.protein_family()
    S = torch.from_numpy(fam.msa).cuda()
    stream = torch.cuda.Stream()
    ctx = api.Context(0, stream)
    m, w, beff = api.msa_reweight(ctx, S)
    N = fam.N
    rng = np.random.default_rng(0)
    h = torch.from_numpy(rng.normal(0, 0.05, (N, 21)).astype(np.float32)).cuda()
    J = rng.normal(0, 0.05, (N, 21, N, 21)).astype(np.float32)
    for r in range(N):
        J[r, :, r, :] = 0
    J = torch.from_numpy(J).cuda()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    prec = "split_bf16" if args.prec == "auto" else args.prec
    out = {}
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            api.plm_site_objective_grad(ctx, S, w, beff, h, J, prec=prec)
        times = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            f, gh, gJ = api.plm_site_objective_grad(ctx, S, w, beff, h, J, prec=prec)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1000.0)
    t = statistics.mean(times)
    print(json.dumps({"workload": "eval: " + workload_name(fam), "precision": prec, "steps": args.steps,
                      "s_per_eval": t, "s_per_eval_median": statistics.median(times),
                      "evals_per_s": 1.0 / t, "f_sum": float(f.double().sum()),
                      "note": "through plm_site_objective_grad: public-layout conversion, "
                              "bf16 split, both tensor-core kernels and the objective sums"}),
          flush=True)
    ctx.close()


def run_symmetric(args):
    """Symmetric plmDCA (one minimisation, tied blocks) on the family
    workload beside the asymmetric solve: seconds, descent steps and the
    overlap of the two contact lists (the paper compares the two, Sec. 6)."""
    import torch
    from paper_1401_4832_gb300 import api, synth
    fam = synth.protein_family()
    S = torch.from_numpy(fam.msa).cuda()
    stream = torch.cuda.Stream()
    ctx = api.Context(0, stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    prec = "split_bf16" if args.prec == "auto" else args.prec
    out = {}
    tops = {}
    with torch.cuda.stream(stream):
        for name, fn in (("asymmetric", api.plm_solve), ("symmetric", api.plm_solve_symmetric)):
            times = []
            for k in range(args.warmup + args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h, J, rep = fn(ctx, S, gtol=args.gtol, prec=prec)
                fnm, cfn, top = api.fn_apc_scores(ctx, J)
                e1.record(stream)
                torch.cuda.synchronize()
                if k >= args.warmup:
                    times.append(e0.elapsed_time(e1) / 1000.0)
            tops[name] = set(map(tuple, top.cpu().numpy().tolist()))
            out[name] = {"s": statistics.mean(times), "iters": rep["iters"],
                         "evals": rep["evals"], "gnorm_max": rep["gnorm_max"],
                         "converged": rep["n_converged"] == fam.N}
    out["top_N_overlap"] = len(tops["asymmetric"] & tops["symmetric"]) / max(1, len(tops["symmetric"]))
    print(json.dumps({"workload": "symmetric vs asymmetric: " + workload_name(fam), "precision": prec,
                      "gtol": args.gtol, "results": out}), flush=True)
    ctx.close()


def run_scores(args):
    """Every score variant of Sec. 6 on the family's solved couplings: device
    time per call (gauge + combination + score + correction + top-N)."""
    import torch
    from paper_1401_4832_gb300 import api, synth
    fam = synth.protein_family()
    S = torch.from_numpy(fam.msa).cuda()
    stream = torch.cuda.Stream()
    ctx = api.Context(0, stream)
    out = {}
    with torch.cuda.stream(stream):
        h, J, rep = api.plm_solve(ctx, S, gtol=args.gtol)
        m, w, beff = api.msa_reweight(ctx, S)
        freq = api.msa_frequencies(ctx, S, w, beff)
        ref = set(map(tuple, api.fn_apc_scores(ctx, J)[2].cpu().numpy().tolist()))
        variants = {"fro+apc": {}, "lp1+apc": dict(norm="lp", p=1.0),
                    "fro_nogap+apc": dict(exclude_gap=True), "fro+asc": dict(correction="asc"),
                    "burkoff+apc": dict(norm="burkoff", freq=freq),
                    "min+fro+apc": dict(combine="min")}
        for name, kw in variants.items():
            for _ in range(args.warmup):
                api.plm_scores(ctx, J, **kw)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                sc, co, top = api.plm_scores(ctx, J, **kw)
            e1.record(stream)
            torch.cuda.synchronize()
            got = set(map(tuple, top.cpu().numpy().tolist()))
            out[name] = {"ms_per_call": e0.elapsed_time(e1) / args.steps,
                         "top_N_overlap_with_fro_apc": len(got & ref) / max(1, len(ref))}
    print(json.dumps({"workload": "scores: " + workload_name(fam), "results": out}), flush=True)
    ctx.close()


def run_frontend(args):
    """The MSA front end on the family written as A2M text with insert
    states (host code): parse throughput, and the parsed MSA equal to the
    family's."""
    import numpy as np
    from paper_1401_4832_gb300 import api, synth
    fam = synth.protein_family()
    rng = np.random.default_rng(0)
    inv = "-ACDEFGHIKLMNPQRSTVWY"
    lines = []
    for b, row in enumerate(fam.msa):
        s = "".join(inv[x] + ("a" if rng.random() < 0.05 else "") for x in row)
        lines.append(f">seq{b}")
        lines.extend(s[k:k + 60] for k in range(0, len(s), 60))
    text = ("\n".join(lines) + "\n").encode()
    for _ in range(args.warmup):
        api.msa_parse(text)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S = api.msa_parse(text)
    dt = (time.perf_counter() - t0) / args.steps
    print(json.dumps({"workload": "frontend: A2M text of " + workload_name(fam), "bytes": len(text),
                      "s_per_parse": dt, "MB_per_s": len(text) / dt / 1e6,
                      "equal_to_family": bool(np.array_equal(S, fam.msa))}), flush=True)


def main():
    args = parse_args()
    if args.workload == "frontend":
        return run_frontend(args)
    if args.workload == "scores":
        return run_scores(args)
    if args.workload == "symmetric":
        return run_symmetric(args)
    if args.workload == "eval":
        return run_eval(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "scale":
        return run_scale(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    from paper_1401_4832_gb300 import _native, api, synth

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = local
    torch.cuda.set_device(device)
    pk, pk_kind = peaks()

    # one replica per rank (weak scaling): rank 0 generates the family (and
    # caches it on disk), the other ranks load it after the barrier and take
    # their own order of its sequences
    if dist and rank != 0:
        dist.barrier()
    fam = synth.protein_family()
    if dist and rank == 0:
        dist.barrier()
    B, N = fam.B, fam.N
    msa = torch.from_numpy(replica_msa(fam.msa, rank)).to(f"cuda:{device}")
    stream = torch.cuda.Stream(device)
    ctx = api.Context(device, stream)
    prec = args.prec
    if prec == "auto":
        prec = "split_bf16"
        try:
            api.plm_solve(ctx, msa[:64, :8].contiguous(), prec="split_bf16", max_iter=1)
        except _native.PlmError:
            prec = "fp32"
    opts = dict(gtol=args.gtol, prec=prec, lbfgs_m=args.lbfgs_m)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{device}")

    last = {}

    def step():
        h, J, rep = api.plm_solve(ctx, msa, **opts)
        fn, cfn, top = api.fn_apc_scores(ctx, J)
        last.update(h=h, J=J, fn=fn, cfn=cfn, top=top)  # kept for the oracle comparison
        return rep, top

    sampler = ClockSampler(device)
    sampler.start()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(device)
        if dist:
            dist.barrier()
        lib = _native.load()
        launches0 = lib.plm_kernel_launches()
        times, reps = [], []
        t_wall0 = time.perf_counter()
        t_epoch0 = time.time()
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(device)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rep, top = step()
            e1.record(stream)
            torch.cuda.synchronize(device)
            times.append(e0.elapsed_time(e1) / 1000.0)
            reps.append(rep)
        t_wall = time.perf_counter() - t_wall0
        sampler.window(t_epoch0, time.time())
        clocks = sampler.stop()
        launches = lib.plm_kernel_launches() - launches0
    if dist:
        dist.barrier()
    mean_t = statistics.mean(times)
    value = job_seconds_per_solve(sum(times), args.steps, world, dist,
                                  f"cuda:{device}" if dist else "cpu")
    evals = statistics.mean(r["evals"] for r in reps)

    # the plain FP32 GPU path at the same gtol (the comparison the metric names)
    fp32_cmp = None
    if prec != "fp32" and not args.no_fp32_cmp:
        def step32():
            h, J, rep = api.plm_solve(ctx, msa, gtol=args.gtol, prec="fp32")
            fn, cfn, top = api.fn_apc_scores(ctx, J)
            return rep, top
        with torch.cuda.stream(stream):
            step32()
            t32, top32 = [], None
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize(device)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                rep32, top32 = step32()
                e1.record(stream)
                torch.cuda.synchronize(device)
                t32.append(e0.elapsed_time(e1) / 1000.0)
        same = bool(torch.equal(top32.cpu(), top.cpu()))
        fp32_cmp = {"value": statistics.mean(t32), "unit": "s",
                    "speedup_of_split_bf16": statistics.mean(t32) / mean_t,
                    "evals_per_solve": rep32["evals"], "gnorm_max": rep32["gnorm_max"],
                    "top_L_identical_to_split_bf16": same}

    # end to end through the public API with host buffers: the whole rundown
    # (api.plmdca -> plmdca_run) from a pinned host MSA into pinned host
    # outputs (h, J, FN, CFN, top-N); the copies happen inside the call
    msa_host = torch.from_numpy(fam.msa).pin_memory()
    pin = dict(h=torch.empty((N, 21), dtype=torch.float32).pin_memory(),
               J=torch.empty((N, 21, N, 21), dtype=torch.float32).pin_memory(),
               fn=torch.empty((N, N), dtype=torch.float64).pin_memory(),
               cfn=torch.empty((N, N), dtype=torch.float64).pin_memory(),
               top=torch.empty((N, 2), dtype=torch.int32).pin_memory())
    e2e_times = []
    with torch.cuda.stream(stream):
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize(device)
            t0 = time.perf_counter()
            res = api.plmdca(ctx, msa_host, out=pin, **opts)
            e2e_times.append(time.perf_counter() - t0)
    e2e_top_same = bool(torch.equal(res["top"], top.cpu()))
    h2d = B * N  # the MSA
    d2h = sum(v.numel() * v.element_size() for v in pin.values())  # h, J, FN, CFN, top-N

    # per-kernel device times of one profiled solve (events on the library stream)
    import ctypes
    lib.plm_profile_report.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int]
    lib.plm_profile(ctx.handle, 1)
    with torch.cuda.stream(stream):
        flush.zero_()
        rep_p, _ = step()
    kern = read_profile(lib, ctx)
    lib.plm_profile(ctx.handle, 0)
    # the tensor-core kernels on full evaluations (every tile live; inside the
    # solve, tiles whose sites all stopped searching are skipped)
    tc_full = tc_full_evals(api, lib, ctx, stream, msa, flush, prec, reps=10)
    alu = measure_alu_peaks(lib, stream)
    per_kernel = kernel_rooflines(kern, tc_full, B, N, pk, pk_kind, alu)
    if fp32_cmp is not None:
        # the plain FP32 path's kernels on full evaluations, against the
        # measured FP32 add rate (gathers) and HBM bandwidth (the softmax pass:
        # logits read, residual written, B x 24N floats each)
        f32 = tc_full_evals(api, lib, ctx, stream, msa, flush, "fp32", reps=5)
        fr = kernel_rooflines({}, f32, B, N, pk, pk_kind, alu)
        if "softmax_resid" in f32:
            by = 2 * B * 24 * N * 4
            ach = by / f32["softmax_resid"] / 1e9
            fr["softmax_resid"] = {"bound": "hbm", "achieved": ach, "peak": pk.get("hbm_gbs", 6800.0),
                                   "unit": "GB/s", "frac": ach / pk.get("hbm_gbs", 6800.0),
                                   "launch_us_full_eval": f32["softmax_resid"] * 1e6}
        fp32_cmp["kernel_rooflines"] = fr
        fp32_cmp["s_per_full_eval"] = sum(f32.values())
    dom = max(kern, key=lambda k: kern[k][1]) if kern else None
    roof = None
    if dom:
        roof = dict(per_kernel.get(dom) or {"bound": None, "achieved": None, "peak": None,
                                            "unit": None, "frac": None, "traffic": None})
        roof["kernel"] = dom
        roof["launches_profiled"] = kern[dom][0]
        roof["share_of_profiled"] = kern[dom][1] / sum(v[1] for v in kern.values())

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        cores = oracle.num_threads()
        if args.cpu_sites:
            full, wall, oevals, ns = cpu_sample(fam, args.cpu_sites, args.gtol)
            sample = (f"full reweighting + L-BFGS of {ns} of {N} sites (gtol {args.gtol}) "
                      f"scaled x{N}/{ns} + full FN/APC/top-L; {wall:.1f} s of CPU wall time")
            parity = None
        else:
            full, parity = cpu_full_rundown(fam, args.gtol, last)
            sample = (f"the whole rundown on all {N} sites (reweighting, L-BFGS to gtol "
                      f"{args.gtol}, FN/APC/top-L), no extrapolation")
        full1, wall1, _, ns1 = cpu_sample_single_thread(fam, 2, args.gtol)
        cpu = {"value": full, "unit": "s", "cores": cores, "kind": "oracle", "sample": sample,
               "single_thread": {"value": full1, "unit": "s", "cores": 1,
                                 "sample": (f"reweighting + L-BFGS of {ns1} of {N} sites on one "
                                            f"thread scaled x{N}/{ns1} + FN/APC/top-L; "
                                            f"{wall1:.1f} s of CPU wall time")},
               "parity_of_the_timed_solve": parity}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * mean_t,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if prec == "split_bf16" else "f32", "data": "synthetic",
            "config": {"workload": workload_name(fam), "N": N, "B": B, "q": 21, "gtol": args.gtol,
                       "precision": prec, "lbfgs_m": args.lbfgs_m, "lambda_h": 0.01, "lambda_J": 0.01,
                       "x": 0.8, "l2": "flushed between timed steps (256 MiB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "evals_per_s": evals / mean_t,
            "fp32_path": fp32_cmp,
            "evals_per_solve": evals,
            "iters": statistics.mean(r["iters"] for r in reps),
            "sites_converged": reps[-1]["n_converged"], "sites_noise": reps[-1]["n_noise"],
            "sites_failed": reps[-1]["n_failed"], "gnorm_max": reps[-1]["gnorm_max"],
            "clocks": clocks,
            "e2e": {"value": statistics.mean(e2e_times), "unit": "s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "call": "api.plmdca (plmdca_run), pinned host buffers",
                    "top_N_equal_to_device_run": e2e_top_same},
            "gpu_launches": launches,
            "roofline": roof,
            "kernels_profiled_ms": {k: v[1] for k, v in kern.items()},
            "kernel_rooflines": per_kernel,
            "alu_peaks_measured": alu,
            "cpu_baseline": cpu,
            "wall_s_timed_region": t_wall,
        }
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


# DRAM bytes (read + write) per launch from one ncu capture of a full
# evaluation of this workload, valid only for the kernel source it was
# taken on (sha256 prefix of the .cu file); null once the source changes
NCU_TRAFFIC = {
    "tc_logits": ("k_tc.cu", "e10e6cc3c03733fe", 27.150848e6 + 4.660224e6),
    "tc_grad": ("k_tc.cu", "e10e6cc3c03733fe", 78.078976e6 + 3.575040e6),
}


def ncu_traffic(kernel):
    import hashlib
    ent = NCU_TRAFFIC.get(kernel)
    if not ent:
        return None
    fn = os.path.join(ROOT, "paper_1401_4832_gb300", "csrc", ent[0])
    try:
        with open(fn, "rb") as fh:
            h = hashlib.sha256(fh.read()).hexdigest()[:16]
    except OSError:
        return None
    return ent[2] if h == ent[1] else None


def replica_msa(msa, rank):
    """Multi-GPU runs are replicas (the path needs no exchange): rank r
    solves the family with its sequences in an order drawn with seed r
    (rank 0: as generated) -- its own copy of the data, the same problem and
    the same work on every rank, from one family that rank 0 generates."""
    import numpy as np
    if rank == 0:
        return msa
    perm = np.random.default_rng(int(rank)).permutation(msa.shape[0])
    return np.ascontiguousarray(msa[perm])


def job_seconds_per_solve(local_total_s, steps, world, dist=None, device="cpu"):
    """Whole-job seconds per solve: the slowest rank's total over the timed
    steps (max over ranks), divided by all the solves the job did."""
    total = float(local_total_s)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = t.item()
    return total / (steps * world)


def read_profile(lib, ctx):
    """{kernel: (launches, total ms, algorithmic bytes)} from the context's
    profile record."""
    import ctypes
    buf = ctypes.create_string_buffer(1 << 16)
    lib.plm_profile_report(ctx.handle, buf, len(buf))
    out = {}
    for ln in buf.value.decode().splitlines():
        name, cnt, ms, by = ln.split()
        out[name] = (int(cnt), float(ms), float(by))
    return out


def tc_full_evals(api, lib, ctx, stream, msa, flush, prec, reps=10):
    """Per-launch device time of the evaluation kernels on full evaluations
    (all sites, a random theta), L2 flushed before each."""
    import numpy as np
    import torch
    B, N = msa.shape
    m, w, beff = api.msa_reweight(ctx, msa)
    rng = np.random.default_rng(0)
    h = torch.from_numpy(rng.normal(0, 0.05, (N, 21)).astype(np.float32)).to(msa.device)
    J = rng.normal(0, 0.05, (N, 21, N, 21)).astype(np.float32)
    for r in range(N):
        J[r, :, r, :] = 0
    J = torch.from_numpy(J).to(msa.device)
    with torch.cuda.stream(stream):
        for _ in range(3):
            api.plm_site_objective_grad(ctx, msa, w, beff, h, J, prec=prec)
        lib.plm_profile(ctx.handle, 1)
        for _ in range(reps):
            flush.zero_()
            api.plm_site_objective_grad(ctx, msa, w, beff, h, J, prec=prec)
        kern = read_profile(lib, ctx)
        lib.plm_profile(ctx.handle, 0)
    return {k: v[1] / 1000.0 / v[0] for k, v in kern.items()}


def kernel_rooflines(kern, tc_full, B, N, pk, pk_kind, alu=None):
    """Roofline entry of every profiled kernel: HBM-bound passes from their
    algorithmic bytes over the profiled solve, tensor-core kernels from the
    dense-equivalent flops of one full evaluation (timed alone, so against
    the burst bf16 peak), ALU-bound passes against the instruction rates
    measured on this GPU (plm_measure_peak) when given."""
    q = 21
    out = {}
    alu = alu or {}
    hbm = pk.get("hbm_gbs", 6800.0)
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    derived = 152 * 128 * sm_mhz * 1e6  # one op per lane per clock
    fadd = alu.get("fadd_f32") or derived
    fadd_note = ("FP32 add rate measured on this GPU (plm_measure_peak)" if alu.get("fadd_f32")
                 else f"152 SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (derived)")
    for name, (cnt, ms, by) in kern.items():
        if by > 0:
            ach = by / (ms / 1000.0) / 1e9
            out[name] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": None,
                         "bytes_per_launch": by / cnt,
                         "peak_note": f"HBM copy bandwidth, {pk_kind}"}
    if "reweight" in kern:
        # pair tests of the bit-plane kernel: 64 x 64 tiles of the upper
        # triangle, ceil(N/32) words each, 7 integer instructions per word
        # (5 three-input logic ops folding XOR/OR over the planes, an add,
        # and one POPC); with measured rates the peak is the mix's rate, the
        # six ALU ops and the POPC each at their own measured throughput
        cnt, ms, _ = kern["reweight"]
        tiles = -(-B // 64)
        words = tiles * (tiles + 1) // 2 * 64 * 64 * (-(-N // 32))
        ops = words * 7
        if alu.get("lop3_b32") and alu.get("popc_b32"):
            t_word = max(6.0 / alu["lop3_b32"], 1.0 / alu["popc_b32"])
            peak = 7.0 / t_word / 1e12
            note = ("7 integer ops per word at the measured lop3 and popc rates "
                    f"({alu['lop3_b32'] / 1e12:.1f} and {alu['popc_b32'] / 1e12:.1f} Tops/s); "
                    "time of the whole reweighting (packing, pair counts, weights, B_eff)")
        else:
            peak = derived / 1e12
            note = (f"152 SMs x 128 lanes x {sm_mhz:.0f} MHz, one 32-bit integer op per lane "
                    "per clock (derived); time of the whole reweighting")
        ach = ops / (ms / 1000.0 / cnt) / 1e12
        out["reweight"] = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Tintop/s",
                           "frac": ach / peak, "traffic": None, "ops_per_launch": ops,
                           "peak_note": note}
    for name, avg_s in tc_full.items():
        if name in ("tc_logits", "tc_grad"):
            # the one-hot contraction as a dense GEMM (unpadded): B x Nq x (Nq + 1)
            # multiply-adds, two bf16 products (hi, lo) each
            flops = 2 * 2 * B * (N * q) * (N * q + 1)
            peak = pk.get("bf16_tflops", 1900.0)
            ach = flops / avg_s / 1e12
            out[name] = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "traffic": ncu_traffic(name),
                         "traffic_unit": "bytes per launch (ncu dram read + write)",
                         "flops_per_launch": flops,
                         "launch_us_full_eval": avg_s * 1e6,
                         "frac_of_sustained": ach / pk.get("bf16_tflops_sustained", 1700.0),
                         "peak_note": f"bf16 dense burst, {pk_kind} (the kernel is timed alone "
                                      "on full evaluations, L2 flushed before each)"}
        elif name in ("logits_gather", "grad_gather"):
            adds = B * N * N * q
            ach = adds / avg_s / 1e12
            out[name] = {"bound": "alu", "achieved": ach, "peak": fadd / 1e12, "unit": "Tadd/s",
                         "frac": ach / (fadd / 1e12), "traffic": None,
                         "launch_us_full_eval": avg_s * 1e6,
                         "peak_note": fadd_note}
        if name in out and name in ("tc_logits", "tc_grad", "logits_gather", "grad_gather"):
            # the method's own work, whatever the formulation: B N (N-1) q adds
            # (one gathered coupling per sequence, site, state and other site)
            # and one pass over the couplings or the gradient (FP32) plus the
            # MSA; the time that work needs at the FP32-add or HBM peak over
            # the measured time
            t_alg = max(B * N * (N - 1) * q / fadd,
                        (N * q * (N * q + 1) * 4 + B * N) / (hbm * 1e9))
            out[name]["algorithmic_frac"] = t_alg / avg_s
            out[name]["algorithmic_peak_note"] = fadd_note
    return out


if __name__ == "__main__":
    main()
