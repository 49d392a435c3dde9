"""Choose the HRR variant per class on the GPU at hand and write a hints
file for load_hrr_hints().

For every class of the per-class sweep recipe with a bra shell of l >= 2
(workloads.sweep_class, reduced to --npair pairs x 512 ket shells, the tuned
tile shapes loaded), the plan is built with one-quantum HRR rounds (Eq. hrr)
and with the two-quantum rounds of Sec. 2.5.5 (both oriented classes hinted
alike) and timed with CUDA events (best of --reps executes after one
warm-up).  A class gets a hint line for each of its two oriented classes when
the 2-q variant beats the 1-q one by more than --margin.

    python -m paper_2210_03192_gb300.tune_hrr [--out FILE] [--npair N]
"""
import argparse
import os
import sys
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None, help="hints file (default: the package's hrr_hints_gb300.txt)")
    ap.add_argument("--npair", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--margin", type=float, default=0.02)
    ap.add_argument("--classes", nargs="*", default=None, help="subset la,lb,lc,Kab")
    args = ap.parse_args(argv)
    import torch
    import paper_2210_03192_gb300 as lx
    from paper_2210_03192_gb300 import workloads as W

    if os.path.exists(lx.HINTS_GB300):
        lx.load_shape_hints(lx.HINTS_GB300)
    classes = [c for c in W.SWEEP_CLASSES if max(c[0], c[1]) >= 2]
    if args.classes:
        classes = [tuple(int(x) for x in c.split(",")) for c in args.classes]
    lines, t0 = [], time.time()
    for (la, lb, lc, K) in classes:
        p = W.sweep_class(la, lb, lc, K, npair=args.npair, naux=512)
        times = {}
        for v in (0, 1):
            lx.hrr_hint(la, lb, lc, v)
            lx.hrr_hint(lb, la, lc, v)
            plan = lx.Eri3cPlan(p.orb, p.aux, p.pairs, p.auxs)
            out = plan.execute()
            best = float("inf")
            for _ in range(args.reps):
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record()
                plan.execute(out)
                e.record()
                torch.cuda.synchronize()
                best = min(best, s.elapsed_time(e))
            times[v] = best
            del plan, out
        lx.hrr_hint(la, lb, lc, -1)
        lx.hrr_hint(lb, la, lc, -1)
        if times[1] < (1.0 - args.margin) * times[0]:
            for (a, b) in {(la, lb), (lb, la)}:
                if b >= 2:
                    lines.append((a, b, lc, times[0], times[1]))
    best_line = {}
    for ln in lines:
        key = ln[:3]
        if key not in best_line or ln[4] / ln[3] < best_line[key][4] / best_line[key][3]:
            best_line[key] = ln
    lines = sorted(best_line.values())
    path = args.out or lx.HRR_HINTS_GB300
    with open(path, "w") as f:
        f.write("# HRR-variant hints for lx3c (load_hrr_hints): la lb lc bra_pure variant (1 = two quanta per round)\n")
        f.write("# written by paper_2210_03192_gb300/tune_hrr.py on %s, %d pairs x 512 ket shells per class;\n"
                % (torch.cuda.get_device_name(0), args.npair))
        f.write("# trailing comment: ms with 1-q rounds -> ms with 2-q rounds\n")
        for (a, b, c, t0_, t1_) in lines:
            f.write("%d %d %d 1 1  # %.3f -> %.3f\n" % (a, b, c, t0_, t1_))
    print("tuned %d classes in %.0f s, %d hint lines -> %s" % (len(classes), time.time() - t0, len(lines), path))
    return 0


if __name__ == "__main__":
    sys.exit(main())
