#!/usr/bin/env python3
"""Benchmark: per-class 3-center Coulomb integral throughput (FP64) on GB300.

Workload (one step): the per-class sweep of contracted (ab|C) evaluation,
every (la, lb <= 4 | lc <= 6) class with K_ab in {1, 3, 6} (K_a = K_b = K_ab,
K_c = 1), 4096 shell pairs x 512 ket shells per class, all-pure, integral
blocks written to HBM.  Synthetic shells: centres uniform in a 20-bohr cube,
exponents log-uniform in [0.05, 1e4], coefficients uniform in [0.1, 1].

Output: one JSON line (rank 0).  value = integrals computed by all ranks /
max-over-ranks device time of the K timed steps (Gints/s).  The line carries
the FP64 roofline of the dominant class, a short list of the slowest classes
(the full per-class table goes to --per-class-out), and one-off measurements
taken after the timed sweep, each with its own clock record:
  config1  (pp|d), 64 pairs x 32 ket shells: ms per evaluation
  dfj      256-atom DF-J build: fused gamma+J, gamma-only, J-only seconds
  batch    16 molecules in one graph launch vs per-class launches
  grad     64-atom DF-J energy forward, gradient backward, fwd+bwd
  metric   256-atom aux basis: V = (P|Q), Cholesky, solve (c = V^-1 gamma)
  dfj_multi  per-density DF-J time, one density vs eight at once (32 atoms)
  fp64_peak_measured  live FP64 FMA rate (lx3c_fp64_rate)

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--classes la,lb,lc,K ...] [--npair N] [--naux N]
                  [--extras config1,dfj,batch,grad,metric,dfj_multi | --extras none]
                  [--no-e2e] [--no-cpu] [--no-hints] [--per-class-out FILE]

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
# (4 flops/clk/SM) at up to 2070 MHz, 1258.6 GFLOP/s (the nominal 1.25 TFLOP/s
# FP64 figure).  The bench also measures the FMA rate live (lx3c_fp64_rate)
# and reports it beside this figure.
FP64_PEAK_GFLOPS = 152 * 4 * 2.070

# DRAM traffic of the (gg|i) K_ab=6 class per pair (512 ket shells, both oriented
# launches), from one ncu capture of dram__bytes_read.sum + dram__bytes_write.sum
# on 64 pairs x 512 ket shells (1,661,696 + 57,140,224 read, 112,523,008 +
# 96,814,848 written), scaled by pairs; the integral blocks written are 4,312,448
# bytes per pair, so traffic is 0.97x the algorithmic bytes (no re-reads; the
# B-oriented launch reads back the blocks it adds to).
GGI_K6_DRAM_BYTES_PER_PAIR = (1661696 + 57140224 + 112523008 + 96814848) / 64


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
    ap.add_argument("--no-hints", action="store_true", help="ignore the package's tuned tile-shape and HRR hints")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--per-class-out", default=None, help="write the per-class table to this JSON file")
    ap.add_argument("--extras", default="config1,dfj,batch,grad,metric,dfj_multi",
                    help="one-off measurements after the timed sweep (comma list, or 'none')")
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
        flops = plan.flops  # per the orientation each pair runs in
        plans.append(dict(cls=(la, lb, lc, K), plan=plan, prob=p, flops=flops, nint=plan.total))
    return plans


def run_ours(args, rank, world, dist):
    import torch
    import paper_2210_03192_gb300 as lx
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    classes = class_list(args)
    t0 = time.time()
    args.hints = args.hrr_hints = 0
    if not args.no_hints and os.path.exists(lx.HINTS_GB300):
        args.hints = lx.load_shape_hints(lx.HINTS_GB300)
    if not args.no_hints and os.path.exists(lx.HRR_HINTS_GB300):
        args.hrr_hints = lx.load_hrr_hints(lx.HRR_HINTS_GB300)
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
    traffic = None
    if plans[dom]["cls"] == (4, 4, 6, 6) and args.naux == 512 and not args.product_k:
        traffic = round(GGI_K6_DRAM_BYTES_PER_PAIR * args.npair)
    res = dict(ms=ms, total_int=total_int, total_flops=total_flops, table=table, clocks=clk, setup_s=setup_s,
               launches=launches_per_step * args.steps,
               roofline=dict(bound="alu", achieved=round(ach, 2), peak=round(FP64_PEAK_GFLOPS, 1), unit="GFLOP/s",
                             frac=round(ach / FP64_PEAK_GFLOPS, 4), traffic=traffic,
                             kernel="%s, class (%d%d|%d) K_ab=%d" % ((kernel_name(plans[dom]["cls"]),)
                                                                     + tuple(plans[dom]["cls"])),
                             peak_source="derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                             flops_per_launch=plans[dom]["flops"], launch_ms=round(dms, 3)),
               l3_frac=dict(classes=len(l3), min=min(l3) if l3 else None,
                            median=statistics.median(l3) if l3 else None,
                            at_least_half=sum(1 for x in l3 if x >= 0.5)))
    # e2e through the host-buffer C-ABI call
    if not args.no_e2e and rank == 0:
        res["e2e"] = run_e2e(plans, args)
    del out
    for p in plans:
        p["plan"] = None
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def kernel_name(cls):
    """The kernel a sweep class's launches run: the register-resident forms
    for (s s|C) and for (p s|C) / (s p|C) with 1 <= lc <= 4 (or contracted),
    the tile kernel otherwise."""
    la, lb, lc, K = cls
    if la == 0 and lb == 0:
        return "eri3c_ss_kernel"
    if la + lb == 1 and lc <= 4 and (lc > 0 or K > 1):
        return "eri3c_ps_kernel"
    return "eri3c_kernel"


def run_e2e(plans, args):
    """Same sweep through lx3c_eri3c_host: host shell tables in, host blocks out
    (pinned), device allocation, H2D, compute and D2H inside the timed region."""
    import torch
    import paper_2210_03192_gb300 as lx
    maxtot = max(p["plan"].total for p in plans)
    host, host_kind, release = pinned_host_buffer(maxtot)
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
    release()
    tot = sum(p["nint"] for p in plans)
    return dict(value=round(tot / dt / 1e9, 4), unit="Gints/s", h2d_bytes_per_step=int(h2d),
                d2h_bytes_per_step=int(d2h), seconds=round(dt, 3), host_buffer=host_kind)


def pinned_host_buffer(n):
    """n doubles of page-locked host memory, touched before any timing: an
    anonymous mapping advised for transparent huge pages and registered with
    CUDA (cudaHostRegister) where the OS and driver allow, else torch's pinned
    allocator.  The GPU reaches host memory through the CPU's page tables, so
    the page size sets how far its address translation reaches across a
    multi-GB buffer.  Returns (numpy array, kind, release callable)."""
    import mmap
    import torch
    nbytes = int(n) * 8
    try:
        m = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        m.madvise(mmap.MADV_HUGEPAGE)
        arr = np.frombuffer(m, dtype=np.float64)
        arr[:] = 0.0
        torch.cuda.cudart().cudaHostRegister(arr.ctypes.data, nbytes, 0)
        if torch.from_numpy(arr).is_pinned():
            def release():
                torch.cuda.cudart().cudaHostUnregister(arr.ctypes.data)
            return arr, "huge-page mapping, cudaHostRegister", release
    except Exception:
        pass
    host = torch.empty(int(n), dtype=torch.float64, pin_memory=True).numpy()
    host[:] = 0.0
    return host, "torch pinned", lambda: None


# ---------------------------------------------------------------------------
# one-off measurements after the timed sweep (configs 1, 3, 4, 5)
# ---------------------------------------------------------------------------

def event_ms(fn, reps=1):
    """CUDA-event durations (ms) of `reps` calls of fn() on the current stream."""
    import torch
    st = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def with_clocks(dev, fn):
    """fn()'s dict with a compact clock record of its run: [median SM MHz,
    samples, throttle reasons]."""
    clocks = ClockSampler(dev.index)
    clocks.start()
    try:
        res = fn()
    finally:
        clk = clocks.stop()
    res["clocks"] = [clk.get("sm_mhz"), clk.get("samples", 0), clk.get("reasons", [])]
    return res


def extra_config1(dev):
    """(pp|d), K=1, 64 pairs x 32 ket shells: the whole 92,160-integral output."""
    import torch
    import paper_2210_03192_gb300 as lx
    from paper_2210_03192_gb300 import workloads as W
    p = W.ppd_64x32()
    plan = lx.Eri3cPlan(p.orb, p.aux, p.pairs, p.auxs, bra_pure=True)
    out = torch.empty(plan.shape, dtype=torch.float64, device=dev)
    for _ in range(5):
        plan.execute(out)
    # batches of 500 evaluations, about 1.5 s in all, so the clock sampler sees the load
    reps = 500
    ms = statistics.median(t / reps for t in event_ms(lambda: [plan.execute(out) for _ in range(reps)], 40))
    fl = plan.flops
    return dict(workload="(pp|d) 64x32", integrals=int(plan.total),
                ms=round(ms, 4), gints_s=round(plan.total / ms / 1e6, 4),
                frac=round(fl / ms / 1e6 / FP64_PEAK_GFLOPS, 4), launches=plan.launches, reps=40 * reps)


def extra_dfj(dev):
    """256-atom DF-J build: fused gamma+J, gamma-only and J-only, with the
    per-integral digestion and with the (e0|c)-level contraction."""
    import torch
    import paper_2210_03192_gb300 as lx
    from paper_2210_03192_gb300 import workloads as W
    cl = W.cluster256_dfj()
    rng = np.random.default_rng(W.SEED_BASE + 2)
    t0 = time.time()
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12)
    setup = time.time() - t0
    D = torch.tensor(W.density(rng, plan.nao), device=dev)
    c = torch.tensor(rng.standard_normal(plan.naux_ao), device=dev)
    gamma = torch.empty(plan.naux_ao, dtype=torch.float64, device=dev)
    J = torch.empty((plan.nao, plan.nao), dtype=torch.float64, device=dev)

    def times(pl):
        first = event_ms(lambda: pl.execute(D, c, gamma, J))[0]  # loads the kernels and tables
        fused = event_ms(lambda: pl.execute(D, c, gamma, J))[0]
        gonly = event_ms(lambda: pl.execute(D, c, gamma, None, outputs="gamma"))[0]
        jonly = event_ms(lambda: pl.execute(D, c, None, J, outputs="J"))[0]
        return first, fused, gonly, jonly

    _, fused, gonly, jonly = times(plan)
    out = dict(workload="DF-J 256 atoms", nao=plan.nao, naux_ao=plan.naux_ao,
               screened_triples=plan.ntasks, integrals=plan.nint, tile_fill=round(plan.tile_fill, 4),
               setup_s=round(setup, 2), fused_s=round(fused / 1e3, 3),
               gamma_only_s=round(gonly / 1e3, 3), J_only_s=round(jonly / 1e3, 3),
               fused_frac=round(plan.flops / fused / 1e6 / FP64_PEAK_GFLOPS, 4), launches=plan.launches)
    pflops = plan.flops
    del plan
    torch.cuda.empty_cache()
    t0 = time.time()
    cp = lx.DFJPlan(cl.orb, cl.aux, 1e-12, contract=True)
    csetup = time.time() - t0
    _, cfused, cgonly, cjonly = times(cp)
    # the contracted build does fewer flops; its fraction is of its own flops
    out["contracted"] = dict(setup_s=round(csetup, 2), fused_s=round(cfused / 1e3, 3),
                             gamma_only_s=round(cgonly / 1e3, 3), J_only_s=round(cjonly / 1e3, 3),
                             flops_ratio=round(cp.flops / pflops, 4),
                             fused_frac=round(cp.flops / cfused / 1e6 / FP64_PEAK_GFLOPS, 4),
                             speedup=round(fused / cfused, 3), launches=cp.launches)
    return out


def extra_batch(dev):
    """16 molecules (20-400 atoms), every class mixed: one graph launch vs per-class launches."""
    import torch
    import paper_2210_03192_gb300 as lx
    from paper_2210_03192_gb300 import workloads as W
    import oracle
    mols = W.batch16_molecules()
    rng = np.random.default_rng(W.SEED_BASE + 3)
    t0 = time.time()
    b = lx.Batch([(m.orb, m.aux) for m in mols], 1e-12)
    plan_s = time.time() - t0
    Ds = [torch.tensor(W.density(rng, int(oracle.ao_offsets(m.orb)[-1])), device=dev) for m in mols]
    cs = [torch.tensor(rng.standard_normal(int(oracle.ao_offsets(m.aux)[-1])), device=dev) for m in mols]
    t0 = time.time()
    b.bind(Ds, cs)
    bind_s = time.time() - t0
    info = b.info()
    b.execute(2)
    m2 = event_ms(lambda: b.execute(2))[0]
    m0 = event_ms(lambda: b.execute(0))[0]
    m1 = event_ms(lambda: b.execute(1))[0]
    fl = info["flops"]
    return dict(workload="16 molecules, 20-400 atoms",
                screened_triples=info["tasks"], plan_s=round(plan_s, 2), bind_capture_s=round(bind_s, 2),
                graph_branches_s=round(m2 / 1e3, 3), per_class_s=round(m0 / 1e3, 3),
                graph_persistent_s=round(m1 / 1e3, 3),
                frac=dict(graph_branches=round(fl / m2 / 1e6 / FP64_PEAK_GFLOPS, 4),
                          per_class=round(fl / m0 / 1e6 / FP64_PEAK_GFLOPS, 4),
                          graph_persistent=round(fl / m1 / 1e6 / FP64_PEAK_GFLOPS, 4)),
                launches=dict(per_class=int(info["plain_launches"]), graph_branches_kernel_nodes=int(info["branch_kernels"]),
                              graph_persistent_kernel_nodes=int(info["graph_kernels"]),
                              persistent_tiers=int(info["tiers"])),
                speedup_graph_vs_per_class=round(m0 / m2, 4))


def extra_grad(dev):
    """64-atom DF-J energy E = c^T gamma: forward, gradient (backward), fwd+bwd vs plain DF-J."""
    import torch
    import paper_2210_03192_gb300 as lx
    from paper_2210_03192_gb300 import workloads as W
    cl = W.cluster64_grad()
    rng = np.random.default_rng(W.SEED_BASE + 4)
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12, gradient=True)
    D = torch.tensor(W.density(rng, plan.nao), device=dev)
    c = torch.tensor(rng.standard_normal(plan.naux_ao), device=dev)
    gamma = torch.empty(plan.naux_ao, dtype=torch.float64, device=dev)
    J = torch.empty((plan.nao, plan.nao), dtype=torch.float64, device=dev)
    grad = torch.empty((plan.natom, 3), dtype=torch.float64, device=dev)
    plan.energy(D, c)
    plan.gradient(D, c, grad)
    fwd = statistics.median(event_ms(lambda: plan.energy(D, c), 2))
    bwd = statistics.median(event_ms(lambda: plan.gradient(D, c, grad), 2))
    both = statistics.median(event_ms(lambda: (plan.energy(D, c), plan.gradient(D, c, grad)), 2))
    plain = statistics.median(event_ms(lambda: plan.execute(D, c, gamma, J), 2))
    return dict(workload="dE/dR, 64 atoms",
                screened_triples=plan.ntasks, fwd_ms=round(fwd, 2), bwd_ms=round(bwd, 2), fwd_bwd_ms=round(both, 2),
                plain_fwd_gamma_J_ms=round(plain, 2), fwd_bwd_over_fwd=round(both / fwd, 3),
                bwd_frac=round(plan.grad_flops / bwd / 1e6 / FP64_PEAK_GFLOPS, 4),
                launches=dict(fwd=plan.launches, bwd=plan.grad_launches))


def extra_dfj_multi(dev):
    """Per-density DF-J time with one density and with eight at once
    (lx3c_dfj_execute_multi), and the single-density build contracted at the
    (e0|c) level, 32-atom cluster of the 256-atom recipe."""
    import torch
    import paper_2210_03192_gb300 as lx
    from paper_2210_03192_gb300 import workloads as W
    cl = W.cluster((4, 4, 2), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, W.SEED_BASE + 2)
    rng = np.random.default_rng(W.SEED_BASE + 5)
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12)
    cplan = lx.DFJPlan(cl.orb, cl.aux, 1e-12, contract=True)
    D8 = torch.tensor(np.stack([W.density(rng, plan.nao) for _ in range(8)]), device=dev)
    c8 = torch.tensor(rng.standard_normal((8, plan.naux_ao)), device=dev)
    gamma = torch.empty(plan.naux_ao, dtype=torch.float64, device=dev)
    J = torch.empty((plan.nao, plan.nao), dtype=torch.float64, device=dev)
    plan.execute(D8[0], c8[0], gamma, J)
    plan.execute_multi(D8, c8)
    cplan.execute(D8[0], c8[0], gamma, J)
    t1 = statistics.median(event_ms(lambda: plan.execute(D8[0], c8[0], gamma, J), 3))
    t8 = statistics.median(event_ms(lambda: plan.execute_multi(D8, c8), 3))
    tc = statistics.median(event_ms(lambda: cplan.execute(D8[0], c8[0], gamma, J), 3))
    return dict(workload="DF-J 32 atoms", screened_triples=plan.ntasks,
                nd1_ms=round(t1, 2), nd8_ms=round(t8, 2), per_density_ms_nd8=round(t8 / 8, 2),
                per_density_speedup=round(t1 / (t8 / 8), 3), nd1_contracted_ms=round(tc, 2))


def extra_metric(dev):
    """Density-fitting metric of the 256-atom aux basis: V = (P|Q), its Cholesky
    factor and one solve c = V^{-1} gamma."""
    import torch
    import paper_2210_03192_gb300 as lx
    from paper_2210_03192_gb300 import workloads as W
    cl = W.cluster256_dfj()
    mp = lx.MetricPlan(cl.aux)
    n = mp.naux_ao
    A = torch.tensor(W.density(np.random.default_rng(5), 256) + 256 * np.eye(256), device=dev)
    lx.cholesky(A)  # loads the factorization kernels
    V = torch.empty((n, n), dtype=torch.float64, device=dev)
    mp.execute(V)
    tv = statistics.median(event_ms(lambda: mp.execute(V), 3))
    # the basis is numerically singular in FP64 (random diffuse exponents):
    # the drop mode gives functions whose pivot falls to 1e-10 of their
    # diagonal a zero coefficient
    info = []
    tc = event_ms(lambda: info.append(lx.cholesky(V, drop_tol=1e-10)[1]))[0]
    b = torch.tensor(np.random.default_rng(6).standard_normal(n), device=dev)
    ts = statistics.median(event_ms(lambda: lx.cholesky_solve(V, b), 3))
    chol_flops = n ** 3 / 3.0
    return dict(workload="metric, 256-atom aux basis", naux_ao=n,
                metric_ms=round(tv, 2), metric_frac=round(mp.flops / tv / 1e6 / FP64_PEAK_GFLOPS, 4),
                cholesky_ms=round(tc, 2), cholesky_gflops=round(chol_flops / tc / 1e6, 1),
                cholesky_frac=round(chol_flops / tc / 1e6 / FP64_PEAK_GFLOPS, 4), cholesky_dropped=int(info[0]),
                solve_ms=round(ts, 3), metric_launches=mp.launches)


EXTRAS = dict(config1=extra_config1, dfj=extra_dfj, batch=extra_batch, grad=extra_grad, metric=extra_metric,
              dfj_multi=extra_dfj_multi)


def run_extras(args, dev):
    import torch
    import paper_2210_03192_gb300 as lx
    out = {}
    names = [] if args.extras == "none" else [x for x in args.extras.split(",") if x]
    def peak():
        runs = [lx.fp64_rate(1 << 15) for _ in range(3)]
        g, ms = max(runs)
        return dict(gflops=round(g, 1), ms=round(ms, 2), frac_of_derived=round(g / FP64_PEAK_GFLOPS, 4),
                    method="lx3c_fp64_rate")
    out["fp64_peak_measured"] = with_clocks(dev, peak)
    for n in names:
        if n not in EXTRAS:
            raise SystemExit("unknown extra %r (choose from %s)" % (n, ",".join(EXTRAS)))
        out[n] = with_clocks(dev, lambda: EXTRAS[n](dev))
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    return out


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


def make_line(args, res, classes, world, cpu, extras):
    """The bench's one JSON line (kept under 4 KB: the per-class table goes to
    --per-class-out, the line keeps the slowest and the lowest-fraction classes)."""
    value = res["total_int"] / (res["ms"] / 1e3) / 1e9
    top = sorted(res["table"], key=lambda r: -r["ms"])[:4]
    low = sorted((r for r in res["table"] if sum(r["cls"][:3]) >= 3), key=lambda r: r["frac"])[:4]
    line = dict(
        metric="3c-ERI Gints/s FP64 per (La,Lb,Lc,K)", value=round(value, 4), unit="Gints/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=round(res["ms"] / args.steps, 2),
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
        data="synthetic (per-class sweep recipe, seeded)",
        config=dict(sweep_config(args, classes, world),
                    tile_shapes=("planner default + %d tuned hints (shape_hints_gb300.txt)" % getattr(args, "hints", 0)
                                 if getattr(args, "hints", 0) else "planner default"),
                    hrr=("1-q rounds + %d tuned 2-q classes (hrr_hints_gb300.txt)" % getattr(args, "hrr_hints", 0)
                         if getattr(args, "hrr_hints", 0) else "1-q rounds")),
        roofline=res["roofline"], cpu_baseline=cpu, clocks=res["clocks"], gpu_launches=res["launches"],
        fp64_tflops_sweep=round(res["total_flops"] / (res["ms"] / 1e3) / 1e12, 4),
        l3_roofline_frac=res["l3_frac"],
        slowest_classes=[[*r["cls"], r["ms"], r["frac"]] for r in top],
        lowest_frac_l3_classes=[[*r["cls"], r["ms"], r["frac"]] for r in low],
        class_row="[la,lb,lc,K_ab,ms,frac]",
    )
    if "e2e" in res:
        line["e2e"] = res["e2e"]
    line.update(extras)
    return line


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
    import torch
    extras = run_extras(args, torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0))))
    line = make_line(args, res, classes, world, cpu, extras)
    if args.per_class_out:
        with open(args.per_class_out, "w") as f:
            json.dump(res["table"], f)
    print(json.dumps(line, separators=(",", ":")), flush=True)


if __name__ == "__main__":
    main()
