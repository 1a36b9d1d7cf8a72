"""Benchmark of the VBARMS hot path on GB300.

One step = the whole data-parallel path on one synthetic matrix: angle
compression (Step 1), the multilevel factorization (Steps 2-4 per level and
the last-level block ILUT) and the FGMRES(50) solve to rtol 1e-8.  The
reported metric is the setup time (compression + factorization) of the mixed
FP32 factor, with the plain FP64 factor timed beside it; the roofline object
covers the dominant factorization kernel (the numeric Schur complement).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the CPU oracle arm

Under torchrun (N > 1) every rank factors its own replica (the method does
not shard: replicas only); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "VBARMS setup s + HBM roofline frac; FP32 vs FP64 factor at FGMRES rtol 1e-8"
PROFILE_NOTE = os.path.join(ROOT, "profiles", "schur_numeric_geo500k_l6.md")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="geo500k_l6")
    p.add_argument("--scale", type=float, default=1.0, help="node-count scale of the workload (1 = full size)")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparator factor")
    p.add_argument("--group-size", type=int, default=1,
                   help="Step 3 groups of up to this many supernodes (block-sparse D_i); 1 = one per group")
    p.add_argument("--lean", action="store_true",
                   help="release each level's intermediate factors once consumed (vbarms_opts.keep_factors = 0)")
    p.add_argument("--dd", type=int, default=0,
                   help="domain decomposition (Section 5) with this many subdomains; 0 = one global VBARMS")
    p.add_argument("--overlap", type=int, default=1, help="subdomain overlap levels with --dd (0 = block Jacobi)")
    p.add_argument("--additive", action="store_true", help="with --dd: additive instead of restricted Schwarz")
    p.add_argument("--schur", type=int, default=0,
                   help="with --dd: the Schur-complement global preconditioner with this many inner GMRES steps")
    return p.parse_args()


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        return dist, rank, ws
    return None, rank, ws


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def schur_source_hash() -> str:
    src = open(os.path.join(ROOT, "paper_1508_02219_gb300", "csrc", "level.cu")).read()
    # the numeric phase: the row-plan kernel and the listed-rows kernel
    a, b = src.find("// Numeric phase."), src.find("// Last reduction: drop off-diagonal blocks of S")
    body = src[a:b] if 0 <= a < b else src
    return hashlib.sha256(body.encode()).hexdigest()[:16]


def profiled_traffic():
    """Per-launch DRAM bytes of the Schur numeric kernel from the committed
    ncu summary, or None when the kernel changed since it was captured."""
    if not os.path.exists(PROFILE_NOTE):
        return None
    txt = open(PROFILE_NOTE).read()
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"full_size_traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not h or not t or h.group(1) != schur_source_hash():
        return None
    return float(t.group(1))


def workload(name, scale, seed):
    from paper_1508_02219_gb300 import synth
    w = dict(synth.WORKLOADS[name])
    m = synth.make_workload(name, seed=seed, scale=scale)
    return m, w


def dd_config(args):
    """(nparts, overlap, restricted, inner steps) of a Section 5 run, or None;
    inner steps > 0 selects the Schur-complement preconditioner (no overlap)."""
    if not getattr(args, "dd", 0):
        return None
    ms = getattr(args, "schur", 0)
    return (args.dd, 0, True, ms) if ms else (args.dd, args.overlap, not args.additive, 0)


def dd_name(dd):
    if dd is None:
        return "vbarms"
    if dd[3]:
        return "schur"
    return "bj" if dd[1] == 0 else ("ras" if dd[2] else "asm")


def dd_keys(dd):
    """The config keys of a Section 5 run."""
    if dd is None:
        return {}
    k = {"precond": dd_name(dd), "nparts": dd[0]}
    k.update({"inner_steps": dd[3]} if dd[3] else {"overlap": dd[1]})
    return k


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


class OneCore:
    """Pin the calling thread to one host core for the oracle (the oracle is
    single-threaded; pinning keeps it on one core, as `taskset -c 0` would),
    restoring the previous affinity afterwards."""

    def __enter__(self):
        self.prev = None
        try:
            self.prev = os.sched_getaffinity(0)
            self.core = min(self.prev)
            os.sched_setaffinity(0, {self.core})
        except (AttributeError, OSError):
            self.core = None
        return self

    def __exit__(self, *exc):
        if self.prev is not None:
            os.sched_setaffinity(0, self.prev)


def oracle_setup_seconds(m, w, restart=50, dd=None, keep=False, gs=1):
    """The CPU oracle (single-threaded) on matrix m: setup seconds and FGMRES."""
    import oracle
    t0 = time.perf_counter()
    c = oracle.compress(m.n, m.rowptr, m.colind, m.val, w["tau"])
    t1 = time.perf_counter()
    if dd is None:
        P = oracle.Prec(c.A, w["nlev"], w["droptol"], w["lfil"], gs=gs)
    elif dd[3]:
        P = oracle.DDSchur(c.A, dd[0], dd[3], w["nlev"], w["droptol"], w["lfil"])
    else:
        P = oracle.DD(c.A, dd[0], dd[1], dd[2], w["nlev"], w["droptol"], w["lfil"])
    t2 = time.perf_counter()
    from paper_1508_02219_gb300 import synth
    b = synth.ones_rhs(m)
    x, its, rr, st = oracle.fgmres(c.A, P, b[c.perm], rtol=1e-8, restart=restart, maxit=1000)
    t3 = time.perf_counter()
    r = dict(compress_s=t1 - t0, factor_s=t2 - t1, solve_s=t3 - t2, its=its, relres=rr)
    if keep:
        r.update(c=c, P=P, x=x)
    return r


def run_reference(args):
    dist, rank, ws = dist_init()
    if rank != 0:
        return
    from paper_1508_02219_gb300 import synth
    if args.workload in synth.BATCHES:
        # a batch: the oracle on one 10k-node ell=5 matrix of the generator,
        # scaled by the batch's node count
        bw = synth.BATCHES[args.workload]
        total = sum(n for n, _ in synth.batch_shapes(args.workload, args.seed, args.scale))
        ms = synth.geometric(10000, 5, seed=args.seed)
        times = []
        for i in range(args.warmup + args.steps):
            r = oracle_setup_seconds(ms, dict(tau=bw["tau"], nlev=bw["nlev"], droptol=bw["droptol"],
                                              lfil=bw["lfil"]))
            if i >= args.warmup:
                times.append((r["compress_s"] + r["factor_s"]) * total / 10000)
        v = statistics.mean(times)
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
                          "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": {"workload": args.workload, "scale": args.scale},
                          "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                                           "sample": f"one 10000-node ell=5 matrix, scaled by {total} nodes"},
                          "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
              flush=True)
        return
    # the oracle on the full matrix of the workload: one step, no warm-up
    # (a step of the single-threaded oracle takes minutes; the line reports the
    # steps it ran)
    full = synth.WORKLOADS[args.workload]
    m = synth.make_workload(args.workload, seed=args.seed, scale=args.scale)
    dd = dd_config(args)
    with OneCore() as oc:
        r = oracle_setup_seconds(m, full, dd=dd, gs=getattr(args, "group_size", 1))
    v = r["compress_s"] + r["factor_s"]
    out = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": 1,
        "warmup": 0, "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "nodes": m.meta.get("nodes"), "n": m.n, "nnz": m.nnz,
                   "ell": full["ell"], "tau": full["tau"], "nlev": full["nlev"], "droptol": full["droptol"],
                   "lfil": full["lfil"], "scale": args.scale,
                   **dd_keys(dd), **({"group_size": args.group_size} if getattr(args, "group_size", 1) > 1 else {})},
        "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"the whole {args.workload} matrix (n = {m.n}), one run of the oracle's "
                                   f"compress + factor, pinned to one core",
                         "host_cpus": os.cpu_count(), "cpu_model": cpu_model(),
                         "requested_steps": args.steps, "requested_warmup": args.warmup},
        "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "detail": {"compress_s": r["compress_s"], "factor_s": r["factor_s"], "solve_s": r["solve_s"],
                   "fgmres_its": r["its"], "relres": r["relres"]},
    }
    print(json.dumps(out), flush=True)


def run_batch(args):
    """Batched factorization of a named batch of independent matrices: one
    step = compress every matrix + one vbarms_factor_batched call (one launch
    per phase for the whole batch).  No solve is timed in this mode."""
    import torch
    from paper_1508_02219_gb300 import build, synth, vbarms as V
    dist, rank, ws = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    bw = synth.BATCHES[args.workload]
    mats = synth.make_batch(args.workload, seed=args.seed, scale=args.scale)
    prec = "fp32" if bw["precision"] == "fp32" else "fp64"
    dev = torch.device("cuda", local)
    dmats = [(torch.from_numpy(m.rowptr).to(dev), torch.from_numpy(m.colind).to(dev),
              torch.from_numpy(m.val).to(dev)) for m in mats]
    torch.cuda.synchronize()

    def step():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        As = [V.vbarms_compress(m.n, rp, ci, vv, bw["tau"]) for m, (rp, ci, vv) in zip(mats, dmats)]
        e[1].record()
        Ps = V.vbarms_factor_batched(As, bw["nlev"], bw["droptol"], bw["lfil"], precision=prec)
        e[2].record()
        torch.cuda.synchronize()
        r = dict(compress_s=e[0].elapsed_time(e[1]) / 1e3, factor_s=e[1].elapsed_time(e[2]) / 1e3,
                 stats=Ps[0].stats(), kstats=Ps[0].kernel_stats(0))
        del Ps, As
        return r

    for _ in range(args.warmup):
        step()
    barrier(dist)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    l0 = V.launch_count()
    res = [step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    launches = V.launch_count() - l0
    clocks = clk.stop()
    barrier(dist)
    setup = max_over_ranks(dist, statistics.mean(r["compress_s"] + r["factor_s"] for r in res))
    kb = sum(r["kstats"]["bytes"] for r in res)
    kms = sum(r["kstats"]["ms"] for r in res)
    kl = sum(r["kstats"]["launches"] for r in res)
    peak, peak_kind = peaks()
    achieved = kb / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    roof = {"bound": "hbm", "kernel": "k_schur_numeric", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
            "traffic": None, "launches_per_step": kl / max(1, len(res)),
            "algorithmic_bytes_per_launch": kb / max(1, kl), "avg_launch_ms": kms / max(1, kl)}
    e2e = None
    if not args.no_e2e:
        pins = [(torch.from_numpy(m.rowptr).pin_memory(), torch.from_numpy(m.colind).pin_memory(),
                 torch.from_numpy(m.val).pin_memory()) for m in mats]
        ets = []
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record()
            As = [V.vbarms_compress(m.n, a.numpy(), b.numpy(), c.numpy(), bw["tau"])
                  for m, (a, b, c) in zip(mats, pins)]
            Ps = V.vbarms_factor_batched(As, bw["nlev"], bw["droptol"], bw["lfil"], precision=prec)
            tags = Ps[0].vector(Ps[0].levels, "ptag")  # device-to-host read of the batch's result
            ev[1].record()
            torch.cuda.synchronize()
            ets.append(ev[0].elapsed_time(ev[1]) / 1e3)
            del Ps, As
        e2e = {"value": max_over_ranks(dist, statistics.mean(ets)), "unit": "s",
               "h2d_bytes_per_step": int(sum(m.rowptr.nbytes + m.colind.nbytes + m.val.nbytes for m in mats)),
               "d2h_bytes_per_step": int(tags.nbytes),
               "note": "compress every matrix from pinned host CSR (copied inside the calls) + the batched factor "
                       "+ read-back of its last-level precision tags"}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        nodes = 10000
        ms = synth.geometric(nodes, 5, seed=args.seed)
        r = oracle_setup_seconds(ms, dict(tau=bw["tau"], nlev=bw["nlev"], droptol=bw["droptol"],
                                          lfil=bw["lfil"]))
        total_nodes = sum(m.meta.get("nodes", m.n) for m in mats)
        cpu = {"value": (r["compress_s"] + r["factor_s"]) * total_nodes / nodes, "unit": "s", "cores": 1,
               "kind": "oracle",
               "sample": f"one {nodes}-node ell=5 matrix of the same generator; oracle compress+factor seconds "
                         f"scaled by the batch's node count {total_nodes}",
               "host_cpus": os.cpu_count()}
    if rank == 0:
        last = res[-1]
        out = {
            "metric": METRIC, "value": setup, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": setup * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "scale": args.scale, "matrices": len(mats),
                       "nodes": [m.meta.get("nodes") for m in mats], "ell": [m.meta.get("ell") for m in mats],
                       "n": sum(m.n for m in mats), "nnz": sum(m.nnz for m in mats), "tau": bw["tau"],
                       "nlev": bw["nlev"], "droptol": bw["droptol"], "lfil": bw["lfil"], "factor_precision": prec,
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (CSR %.2f GB)" % (sum(m.nnz * 12 + m.n * 8 for m in mats) / 1e9)},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "detail": {"compress_s": statistics.mean(r["compress_s"] for r in res),
                       "factor_s": statistics.mean(r["factor_s"] for r in res), "levels": last["stats"]["levels"],
                       "phase_s": last["stats"]["phase_s"], "solve": "not timed in batch mode"},
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def error_report(V, torch, m, r_gpu, r_or) -> dict:
    """Relative Frobenius error of every result of the mixed factor against
    the oracle's FP64 factorization of the same matrix: each level's W, G, S
    and the last level's L, U (blocks matched by compressed block row), one
    preconditioner application and the FGMRES solution."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import precision_report as pr
    P, Po, c = r_gpu["P"], r_or["P"], r_or["c"]
    rep = pr.factor_errors(P, Po)
    out = {k: float(v) for k, v in pr.summary(rep).items()}
    out["block_rel_median"] = {k: float(v) for k, v in pr.summary(rep, "block_rel_median").items()}
    out["blocks_only_one_side"] = {f"{k}.{n}": [r["blocks_only_gpu"], r["blocks_only_oracle"]]
                                   for k, v in rep.items() for n, r in v.items() if isinstance(r, dict)}
    x = np.random.default_rng(5).standard_normal(m.n)
    y = torch.zeros(m.n, dtype=torch.float64, device="cuda")
    V.vbarms_apply(P, torch.from_numpy(x).cuda(), y)
    yo = np.empty(m.n)
    yo[c.perm] = Po.apply(x[c.perm])
    out["apply"] = pr.rel(y.cpu().numpy(), yo)
    xo = np.empty(m.n)
    xo[c.perm] = r_or["x"]
    out["solution"] = pr.rel(r_gpu["x"].cpu().numpy(), xo)
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    from paper_1508_02219_gb300 import synth as _synth
    if args.workload in _synth.BATCHES:
        return run_batch(args)
    import torch
    from paper_1508_02219_gb300 import build, synth, vbarms as V
    dist, rank, ws = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    m, w = workload(args.workload, args.scale, args.seed)
    prec = "fp32" if w["precision"] == "fp32" else "fp64"
    b = synth.ones_rhs(m)
    dev = torch.device("cuda", local)
    rp = torch.from_numpy(m.rowptr).to(dev)
    ci = torch.from_numpy(m.colind).to(dev)
    vv = torch.from_numpy(m.val).to(dev)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.zeros(m.n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    dd = dd_config(args)

    kf = not args.lean

    def factor(A, precision):
        if dd is None:
            return V.vbarms_factor(A, w["nlev"], w["droptol"], w["lfil"], precision=precision, keep_factors=kf,
                                   group_size=args.group_size)
        if dd[3]:
            return V.vbarms_dd_schur_factor(A, dd[0], dd[3], w["nlev"], w["droptol"], w["lfil"], precision=precision,
                                            keep_factors=kf, group_size=args.group_size)
        return V.vbarms_dd_factor(A, dd[0], dd[1], dd[2], w["nlev"], w["droptol"], w["lfil"], precision=precision,
                                  keep_factors=kf, group_size=args.group_size)

    def step(precision, solve=True, keep=False):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        A = V.vbarms_compress(m.n, rp, ci, vv, w["tau"])
        e[1].record()
        P = factor(A, precision)
        e[2].record()
        its = rr = None
        if solve:
            xd.zero_()
            its, rr, st = V.fgmres_solve(A, P, bd, xd, rtol=1e-8, restart=50, maxit=1000)
        e[3].record()
        torch.cuda.synchronize()
        r = dict(compress_s=e[0].elapsed_time(e[1]) / 1e3, factor_s=e[1].elapsed_time(e[2]) / 1e3,
                 solve_s=e[2].elapsed_time(e[3]) / 1e3, its=its, relres=rr, stats=P.stats(),
                 kstats=P.kernel_stats(0), av_bd=A.query()["av_bd"], av_bs=A.query()["av_bs"],
                 ilut=P.ilut_geometry(), chain=P.ilut_chain())
        if keep:  # the factorization is kept for the error report (after timing)
            r.update(P=P, A=A, x=xd.clone())
        del P, A
        return r

    # the first factorization of the process times the ILUT's candidate
    # workspace shapes (reported below); the later ones reuse the choice
    warm = [step(prec) for _ in range(args.warmup)]
    barrier(dist)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    l0 = V.launch_count()
    t0 = time.perf_counter()
    # the last step's factorization is kept (after its timing) only when the
    # error report against the oracle will use it
    want_report = not args.no_cpu_baseline and dd is None and prec == "fp32" and rank == 0 and kf
    res = [step(prec, keep=(want_report and k == args.steps - 1)) for k in range(args.steps)]
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = V.launch_count() - l0
    clocks = clk.stop()
    barrier(dist)
    setup = statistics.mean(r["compress_s"] + r["factor_s"] for r in res)
    step_s = statistics.mean(r["compress_s"] + r["factor_s"] + r["solve_s"] for r in res)
    setup = max_over_ranks(dist, setup)
    step_s = max_over_ranks(dist, step_s)

    # roofline of the Schur numeric kernel (CUDA events inside the library,
    # on the factorization's stream), averaged over its launches
    kb = sum(r["kstats"]["bytes"] for r in res)
    kms = sum(r["kstats"]["ms"] for r in res)
    kl = sum(r["kstats"]["launches"] for r in res)
    kfl = sum(r["kstats"]["flops"] for r in res)
    peak, peak_kind = peaks()
    achieved = kb / (kms / 1e3) / 1e9 if kms > 0 else 0.0
    roof = {"bound": "hbm", "kernel": "k_schur_numeric", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
            if peak_kind == "measured" else "fallback",
            "traffic": profiled_traffic(), "launches_per_step": kl / max(1, len(res)),
            "algorithmic_bytes_per_launch": kb / max(1, kl), "avg_launch_ms": kms / max(1, kl),
            "flops_per_launch": kfl / max(1, kl),
            "achieved_tflops": kfl / (kms / 1e3) / 1e12 if kms > 0 else 0.0}
    # the step's dominant kernel, the last-level ILUT, is bound by its chain of
    # dependent rows, not by a bandwidth: its longest chain of waits and the
    # time per link of that chain
    chain = res[-1]["chain"]
    ilut_s = statistics.mean(r["stats"]["phase_s"]["last_ilut"] for r in res)
    roof["ilut"] = {"bound": "latency (dependency chain)", "kernel": "k_ilut", "ms": ilut_s * 1e3,
                    "chain_links": chain, "us_per_link": ilut_s * 1e6 / chain if chain else None,
                    "note": "rows on the longest chain of waits (every pending L column, dropped multipliers "
                            "included) and the kernel time per row of that chain; the time-critical path is "
                            "longer (rows also wait for a free warp, and chains join), so the latency of one "
                            "link, from a dependency's publication to the row's own, is below this figure"}

    # FP32 vs FP64: the plain FP64 GPU factor on the same GB300
    fp64 = None
    if not args.no_fp64 and prec == "fp32":
        try:
            r64 = step("fp64")
            fp64 = {"setup_s": r64["compress_s"] + r64["factor_s"], "factor_s": r64["factor_s"],
                    "fgmres_its": r64["its"], "relres": r64["relres"], "phase_s": r64["stats"]["phase_s"],
                    "mem_ratio": r64["stats"]["mem_ratio"], "schur_numeric": r64["kstats"]}
        except V.VbarmsError as e:  # e.g. the FP64 factor does not fit in device memory
            fp64 = {"error": str(e)}
            torch.cuda.synchronize()

    # end to end through the C ABI with host buffers (pinned), copies timed:
    # compress from the host CSR (copied inside the call), factor, upload b,
    # FGMRES, download x -- the same work as a step plus its host copies
    e2e = None
    if not args.no_e2e:
        prp = torch.from_numpy(m.rowptr).pin_memory()
        pci = torch.from_numpy(m.colind).pin_memory()
        pvv = torch.from_numpy(m.val).pin_memory()
        pb = torch.from_numpy(b).pin_memory()
        px = torch.empty(m.n, dtype=torch.float64).pin_memory()
        ets, sets = [], []
        its_e2e = None
        n_e2e = max(1, min(args.steps, 5))
        for i in range(n_e2e):
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            A = V.vbarms_compress(m.n, prp.numpy(), pci.numpy(), pvv.numpy(), w["tau"])
            P = factor(A, prec)
            ev[1].record()
            bdev = pb.to(dev, non_blocking=True)
            xdev = torch.zeros(m.n, dtype=torch.float64, device=dev)
            its_e2e, _, _ = V.fgmres_solve(A, P, bdev, xdev, rtol=1e-8, restart=50, maxit=1000)
            px.copy_(xdev, non_blocking=True)
            ev[2].record()
            torch.cuda.synchronize()
            ets.append(ev[0].elapsed_time(ev[2]) / 1e3)
            sets.append(ev[0].elapsed_time(ev[1]) / 1e3)
            del P, A
        e2e = {"value": max_over_ranks(dist, statistics.mean(ets)), "unit": "s",
               "h2d_bytes_per_step": int(m.rowptr.nbytes + m.colind.nbytes + m.val.nbytes + b.nbytes),
               "d2h_bytes_per_step": int(px.numel() * 8),
               "setup_only_s": max_over_ranks(dist, statistics.mean(sets)), "fgmres_its": its_e2e, "steps": n_e2e,
               "note": "timed per step: compress from pinned host CSR (copied inside the call) + factor + upload of "
                       "b + FGMRES(50) to rtol 1e-8 + download of x; setup_only_s stops after the factor"}

    # the CPU oracle on the whole matrix, once, pinned to one core; its FP64
    # factorization is also the reference of the mixed factor's error report
    cpu = None
    errors = None
    if rank == 0 and not args.no_cpu_baseline:
        with OneCore():
            r = oracle_setup_seconds(m, w, dd=dd, keep=True, gs=args.group_size)
        cpu = {"value": r["compress_s"] + r["factor_s"], "unit": "s", "cores": 1, "kind": "oracle",
               "sample": f"the whole {args.workload} matrix (n = {m.n}), one run of the oracle's compress + factor "
                         f"(FP64, single thread, pinned to one core); its FGMRES took {r['solve_s']:.1f} s and "
                         f"{r['its']} iterations",
               "host_cpus": os.cpu_count(), "cpu_model": cpu_model()}
        if dd is None and prec == "fp32":
            errors = error_report(V, torch, m, res[-1], r)
        del r
    last = res[-1]
    if rank == 0:
        out = {
            "metric": METRIC, "value": setup, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "nodes": m.meta.get("nodes"), "ell": w["ell"], "n": m.n,
                       "nnz": m.nnz, "tau": w["tau"], "nlev": w["nlev"], "droptol": w["droptol"],
                       "lfil": w["lfil"], "factor_precision": prec, "fgmres": "FGMRES(50) rtol 1e-8",
                       "parallelism": "replicas" if ws > 1 else "single",
                       **dd_keys(dd), **({"group_size": args.group_size} if getattr(args, "group_size", 1) > 1 else {}),
                       "l2": "inputs larger than L2 (CSR %.2f GB)" % ((m.nnz * 12 + m.n * 8) / 1e9)},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks,
            "detail": {"compress_s": statistics.mean(r["compress_s"] for r in res),
                       "factor_s": statistics.mean(r["factor_s"] for r in res),
                       "solve_s": statistics.mean(r["solve_s"] for r in res), "fgmres_its": last["its"],
                       "relres": last["relres"], "levels": last["stats"]["levels"],
                       "mem_ratio": last["stats"]["mem_ratio"], "phase_s": last["stats"]["phase_s"],
                       "av_bd": last["av_bd"], "av_bs": last["av_bs"], "wall_timed_s": wall,
                       "fp64_factor": fp64, "error_vs_fp64_oracle": errors,
                       "ilut_geometry": {"first_factorization": (warm or res)[0]["ilut"],
                                         "timed_steps": last["ilut"]}},
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
