#!/usr/bin/env python3
"""Benchmark: per-class 3-center Coulomb integral throughput (FP64) on GB300.

Workload (one step): the per-class sweep of contracted (ab|C) evaluation,
every (la, lb <= 4 | lc <= 6) class with K_ab in {1, 3, 6} (K_a = K_b = K_ab,
K_c = 1), 4096 shell pairs x 512 ket shells per class, all-pure, integral
blocks written to HBM.  Synthetic shells: centres uniform in a 20-bohr cube,
exponents log-uniform in [0.05, 1e4], coefficients uniform in [0.1, 1].

Output: one JSON line (rank 0).  value = integrals computed by all ranks /
max-over-ranks device time of the K timed steps (Gints/s).  Per-class
throughput and the FP64 roofline fraction of the dominant class are included.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--classes la,lb,lc,K ...] [--no-e2e] [--no-cpu] [--no-hints]

The end-to-end leg (e2e) repeats the sweep through the host-buffer call
lx3c_eri3c_host (host shell tables in, page-locked host blocks out).  The
cpu_baseline leg and --impl reference time the CPU oracle on a bounded sample
of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64 roofline denominator: GB300 has 152 SMs issuing 2 DFMA per clock each
# (4 flops/clk/SM) at up to 2070 MHz; the measured DFMA microbenchmark on this
# pool gave 1191.9 GFLOP/s at the clocks it ran at.
FP64_PEAK_GFLOPS = 152 * 4 * 2.070
FP64_PEAK_MEASURED = 1191.9

# DRAM traffic of the (gg|i) K_ab=6 class per pair (512 ket shells, both oriented
# launches), from one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum
# on 64 pairs x 512 ket shells (59,150,592 + 208,663,552 bytes), scaled by pairs;
# the integral blocks written are 4,312,448 bytes per pair, so traffic is 0.97x the
# algorithmic bytes (no re-reads; the B-oriented launch reads back blocks it adds to).
GGI_K6_DRAM_BYTES_PER_PAIR = (59150592 + 208663552) / 64


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--classes", nargs="*", default=None, help="subset la,lb,lc,Kab (default: all 525)")
    ap.add_argument("--npair", type=int, default=4096)
    ap.add_argument("--naux", type=int, default=512)
    ap.add_argument("--product-k", action="store_true", help="read K_ab as (K_a, K_b) = (K_ab, 1)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-hints", action="store_true", help="ignore the package's tuned tile-shape hints")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--per-class-out", default=None, help="write the per-class table to this JSON file")
    return ap.parse_args()


def class_list(args):
    from paper_2210_03192_gb300 import workloads as W
    if args.classes:
        return [tuple(int(x) for x in c.split(",")) for c in args.classes]
    return list(W.SWEEP_CLASSES)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def rank_problem(la, lb, lc, K, npair, naux, rank, product_k=False):
    """The class problem rank `rank` evaluates: rank 0 the sweep recipe itself,
    every other rank the same recipe with its own seed (weak scaling: each
    rank a sweep of its own synthetic shells, no data exchanged)."""
    from paper_2210_03192_gb300 import workloads as W
    if rank == 0:
        return W.sweep_class(la, lb, lc, K, npair, naux, product_reading=product_k)
    return W.class_problem(la, lb, lc, npair, naux, *((K, 1) if product_k else (K, K)), 1,
                           box=20.0, exp_lo=0.05, exp_hi=1.0e4,
                           seed=W.SEED_BASE + 7919 * rank + la * 100 + lb * 10 + lc + 1000 * K)


def max_over_ranks(value, dist, device):
    """The largest `value` over all ranks (the step time of the slowest rank)."""
    if not dist:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def build_plans(classes, args, rank):
    import paper_2210_03192_gb300 as lx
    plans = []
    for (la, lb, lc, K) in classes:
        p = rank_problem(la, lb, lc, K, args.npair, args.naux, rank, args.product_k)
        plan = lx.Eri3cPlan(p.orb, p.aux, p.pairs, p.auxs, bra_pure=True)
        Kab = K * K if not args.product_k else K
        flops = lx.class_flops(la, lb, lc, Kab, 1, True) * plan.npair * plan.naux
        plans.append(dict(cls=(la, lb, lc, K), plan=plan, prob=p, flops=flops, nint=plan.total))
    return plans


def run_ours(args, rank, world, dist):
    import torch
    import paper_2210_03192_gb300 as lx
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    classes = class_list(args)
    t0 = time.time()
    args.hints = 0
    if not args.no_hints and os.path.exists(lx.HINTS_GB300):
        args.hints = lx.load_shape_hints(lx.HINTS_GB300)
    plans = build_plans(classes, args, rank)
    maxtot = max(p["plan"].total for p in plans)
    out = torch.empty(maxtot, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    launches_per_step = sum(p["plan"].launches for p in plans)
    setup_s = time.time() - t0

    def step(events=None):
        for i, p in enumerate(plans):
            if events is not None:
                events[i][0].record(stream)
            p["plan"].execute(out[:p["plan"].total])
            if events is not None:
                events[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    per_class = [[0.0, 0] for _ in plans]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in plans]
    clocks = ClockSampler(dev.index)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for s in range(args.steps):
        step(ev)
        torch.cuda.synchronize()
        for i in range(len(plans)):
            per_class[i][0] += ev[i][0].elapsed_time(ev[i][1])
            per_class[i][1] += 1
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(t_start.elapsed_time(t_end), dist, dev)
    total_int = sum(p["nint"] for p in plans) * args.steps * world
    total_flops = sum(p["flops"] for p in plans) * args.steps
    # per-class table and dominant class
    table = []
    for p, (t, n) in zip(plans, per_class):
        tm = t / max(n, 1)
        table.append(dict(cls=p["cls"], ms=round(tm, 4), gints_s=round(p["nint"] / tm / 1e6, 4),
                          gflops=round(p["flops"] / tm / 1e6, 2),
                          frac=round(p["flops"] / tm / 1e6 / FP64_PEAK_GFLOPS, 4)))
    dom = max(range(len(plans)), key=lambda i: per_class[i][0])
    dms = per_class[dom][0] / max(per_class[dom][1], 1)
    ach = plans[dom]["flops"] / dms / 1e6
    l3 = [r["frac"] for r in table if sum(r["cls"][:3]) >= 3]
    res = dict(ms=ms, total_int=total_int, total_flops=total_flops, table=table, clocks=clk, setup_s=setup_s,
               launches=launches_per_step * args.steps,
               roofline=dict(bound="alu", achieved=round(ach, 2), peak=round(FP64_PEAK_GFLOPS, 1), unit="GFLOP/s",
                             frac=round(ach / FP64_PEAK_GFLOPS, 4),
                             traffic=(round(GGI_K6_DRAM_BYTES_PER_PAIR * args.npair)
                                      if plans[dom]["cls"] == (4, 4, 6, 6) and args.naux == 512 and not args.product_k
                                      else None),
                             traffic_source="ncu dram bytes, both launches, 64 pairs x 512 kets, scaled by pairs",
                             kernel="eri3c_kernel class (%d%d|%d) K_ab=%d" % plans[dom]["cls"],
                             peak_source="152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (recipe unit counts); "
                                         "measured DFMA microbenchmark %.1f" % FP64_PEAK_MEASURED,
                             flops_per_launch=plans[dom]["flops"], launch_ms=round(dms, 3)),
               l3_frac=dict(min=min(l3) if l3 else None, median=statistics.median(l3) if l3 else None))
    # e2e through the host-buffer C-ABI call
    if not args.no_e2e and rank == 0:
        res["e2e"] = run_e2e(plans, args)
    return res


def run_e2e(plans, args):
    """Same sweep through lx3c_eri3c_host: host shell tables in, host blocks out
    (pinned), device allocation, H2D, compute and D2H inside the timed region."""
    import torch
    import paper_2210_03192_gb300 as lx
    maxtot = max(p["plan"].total for p in plans)
    host = torch.empty(maxtot, dtype=torch.float64, pin_memory=True).numpy()
    host[:] = 0.0  # first touch of the page-locked output buffer happens here, outside the timed region
    h2d = d2h = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p in plans:
        pr = p["prob"]
        n = p["plan"].total
        lx.eri3c_host(pr.orb, pr.aux, pr.pairs, pr.auxs, True, out=host[:n])
        h2d += sum(a.nbytes for a in (pr.orb.l, pr.orb.k, pr.orb.xyz, pr.orb.exps, pr.orb.coefs, pr.aux.l,
                                      pr.aux.k, pr.aux.xyz, pr.aux.exps, pr.aux.coefs, pr.pairs, pr.auxs))
        d2h += n * 8
    dt = time.perf_counter() - t0
    tot = sum(p["nint"] for p in plans)
    return dict(value=round(tot / dt / 1e9, 4), unit="Gints/s", h2d_bytes_per_step=int(h2d),
                d2h_bytes_per_step=int(d2h), seconds=round(dt, 3))


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(classes, args, seconds):
    """Time the oracle (as it stands, FP64 mode) on a bounded sample of the
    sweep: the first np pairs against the first 64 ket shells of every class,
    np doubled until the sample takes about `seconds` of host time."""
    import oracle
    from paper_2210_03192_gb300 import workloads as W
    oracle.build()
    probs = [W.sweep_class(la, lb, lc, K, 64, 64, product_reading=args.product_k) for (la, lb, lc, K) in classes]
    npr = 1
    while True:
        t0 = time.perf_counter()
        ints = 0
        for p in probs:
            X = oracle.eri3c(p.orb, p.aux, p.pairs[:npr], p.auxs, bra_pure=True)
            ints += X.size
        dt = time.perf_counter() - t0
        if dt >= seconds / 3 or npr >= 64:
            break
        npr = min(64, max(npr * 2, int(npr * seconds / max(dt, 1e-3))))
    return dict(value=round(ints / dt / 1e9, 6), unit="Gints/s", cores=oracle.num_threads(), kind="oracle",
                sample="%d pairs x 64 ket shells of each of %d classes (%d integrals), McMurchie-Davidson FP64, "
                       "%.1f s" % (npr, len(probs), ints, dt), seconds=dt, ints=ints)


def sweep_config(args, classes, world):
    """The workload both arms report on (the reference arm times a bounded
    sample of it, stated in its cpu_baseline)."""
    nint = sum(args.npair * args.naux * (2 * la + 1) * (2 * lb + 1) * (2 * lc + 1) for (la, lb, lc, _) in classes)
    return dict(workload="per-class sweep: every (la,lb<=4|lc<=6) class, K_ab in {1,3,6} (K_a=K_b=K_ab, K_c=1), "
                         "%d pairs x %d aux shells per class, all-pure, blocks written to HBM" % (args.npair, args.naux),
                classes=len(classes), integrals_per_step=nint,
                l2="each step writes the whole sweep's blocks (TB-scale, far above the 129 MB L2); no flush",
                parallelism="dp%d (independent sweeps per rank)" % world)


def run_reference(args, rank, world):
    classes = class_list(args)
    res = []
    for _ in range(args.warmup):
        oracle_sample(classes[:8], args, 1.0)
    for _ in range(args.steps):
        res.append(oracle_sample(classes, args, max(2.0, args.cpu_seconds / max(args.steps, 1))))
    v = statistics.median(r["value"] for r in res)
    line = dict(metric="3c-ERI Gints/s FP64 per (La,Lb,Lc,K)", value=v, unit="Gints/s", n_gpus=world,
                steps=args.steps, warmup=args.warmup, ms_per_step=round(1000 * res[-1]["seconds"], 2),
                higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic (per-class sweep recipe, seeded)", impl="reference",
                config=sweep_config(args, classes, world),
                cpu_baseline=dict(value=v, unit="Gints/s", cores=res[-1]["cores"], kind="oracle",
                                  sample=res[-1]["sample"]),
                e2e=dict(value=v, unit="Gints/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_
        dist_.init_process_group("nccl" if args.impl == "ours" else "gloo")
        dist = dist_
    if args.impl == "reference":
        if rank == 0:
            run_reference(args, rank, world)
        return
    res = run_ours(args, rank, world, dist)
    if rank != 0:
        return
    classes = class_list(args)
    cpu = None
    if not args.no_cpu:
        c = oracle_sample(classes, args, args.cpu_seconds)
        cpu = {k: c[k] for k in ("value", "unit", "cores", "kind", "sample")}
    value = res["total_int"] / (res["ms"] / 1e3) / 1e9
    top = sorted(res["table"], key=lambda r: -r["ms"])[:12]
    line = dict(
        metric="3c-ERI Gints/s FP64 per (La,Lb,Lc,K)", value=round(value, 4), unit="Gints/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=round(res["ms"] / args.steps, 2),
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
        data="synthetic (per-class sweep recipe, seeded; no public dataset)",
        config=dict(sweep_config(args, classes, world),
                    tile_shapes=("planner default + %d tuned hints (shape_hints_gb300.txt)" % getattr(args, "hints", 0)
                                 if getattr(args, "hints", 0) else "planner default")),
        roofline=res["roofline"], cpu_baseline=cpu, clocks=res["clocks"], gpu_launches=res["launches"],
        fp64_tflops_sweep=round(res["total_flops"] / (res["ms"] / 1e3) / 1e12, 4),
        l3_roofline_frac=res["l3_frac"],
        top_classes=[dict(cls=r["cls"], ms=r["ms"], gints_s=r["gints_s"], frac=r["frac"]) for r in top],
        per_class=[[*r["cls"], r["ms"], r["gints_s"], r["frac"]] for r in res["table"]],
    )
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    if args.per_class_out:
        with open(args.per_class_out, "w") as f:
            json.dump(res["table"], f)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
