"""Tune the tile (T triples per tile, chunks of G primitives) of contracted
classes on the GPU at hand and write tile-hint lines for load_shape_hints().

The planner's default tile takes the largest T that fits two CTAs per SM and
then grows G; for highly contracted classes of low angular momentum that
leaves G = 1 (one primitive per chunk, a barrier-separated chunk per
primitive).  This tuner times, for each class, the default and every (T, G)
candidate with T in 1..256 and G among the divisors-like values up to
K = kab (T G between 16 and 2048, two CTAs' shared memory at most), with CUDA
events (best of --reps executes after one warm-up), on --npair pairs x 512
ket shells of the class (workloads.class_problem, exponents and box of the
per-class sweep recipe).  A class gets a tile-hint line (both oriented
classes alike) when its best candidate beats the default by more than
--margin.

Classes: every (la, lb | lc) with (K_a, K_b) pairs of the DF-J and batch
orbital recipes (s K=6, p K=3, d/f/g K=1) and of the sweep (K_a = K_b in
{3, 6}), --lmin-ab <= la + lb <= --lmax-ab (default 0..3), kab >= 3,
heaviest contraction first; tuning stops after --budget seconds.

    python -m paper_2210_03192_gb300.tune_tiles [--out FILE] [--npair N] [--budget S] [--append]
"""
import argparse
import time

TS = (1, 2, 4, 8, 16, 32, 64, 128, 256)
GS = (1, 2, 3, 4, 6, 8, 9, 12, 16, 18, 24, 32, 36)


def class_list(lmax_ab=3, lmin_ab=0):
    ks = {0: 6, 1: 3, 2: 1, 3: 1, 4: 1}
    out = set()
    for la in range(5):
        for lb in range(5):
            if la + lb > lmax_ab or la + lb < lmin_ab:
                continue
            pairs = {(ks[la], ks[lb])}
            pairs |= {(3, 3), (6, 6)}
            for (ka, kb) in pairs:
                if ka * kb < 3:
                    continue
                for lc in range(7):
                    out.add((la, lb, lc, ka, kb))
    return sorted(out, key=lambda c: (-c[3] * c[4], c[0] + c[1], c))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None, help="hints file to write")
    ap.add_argument("--append", action="store_true", help="append to --out instead of overwriting")
    ap.add_argument("--npair", type=int, default=256)
    ap.add_argument("--budget", type=float, default=600.0, help="stop after this many seconds")
    ap.add_argument("--lmax-ab", type=int, default=3)
    ap.add_argument("--lmin-ab", type=int, default=0)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--margin", type=float, default=0.03)
    ap.add_argument("--classes", nargs="*", default=None, help="subset la,lb,lc,Ka,Kb")
    args = ap.parse_args(argv)
    import torch
    import paper_2210_03192_gb300 as lx
    from paper_2210_03192_gb300 import workloads as W

    classes = class_list(args.lmax_ab, args.lmin_ab)
    if args.classes:
        classes = [tuple(int(x) for x in c.split(",")) for c in args.classes]

    def timed(p, orb, aux):
        plan = lx.Eri3cPlan(orb, aux, p.pairs, p.auxs)
        out = plan.execute()
        best = float("inf")
        for _ in range(args.reps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            plan.execute(out)
            e.record()
            torch.cuda.synchronize()
            best = min(best, s.elapsed_time(e))
        used = [sh for sh in plan.shapes if sh["nsub"] > 0]
        shape = (used[0]["T"], used[0]["G"]) if used else (0, 0)
        del plan, out
        return best, shape

    lines, t0 = [], time.time()
    done = 0
    for (la, lb, lc, ka, kb) in classes:
        if time.time() - t0 > args.budget:
            break
        done += 1
        kab = ka * kb
        p = W.class_problem(la, lb, lc, args.npair, 512, Ka=ka, Kb=kb, Kc=1, box=20.0, exp_lo=0.05, exp_hi=1.0e4)
        orb, aux = lx.DeviceBasis(p.orb), lx.DeviceBasis(p.aux)
        t_def, s_def = timed(p, orb, aux)
        best = (t_def, 0, 0)
        for T in TS:
            for G in GS:
                if G > kab or T * G < 16 or T * G > 2048:
                    continue
                lx.tile_hint(la, lb, lc, kab, 1, T, G)
                lx.tile_hint(lb, la, lc, kab, 1, T, G)
                q = lx.shape_query(la, lb, lc, kab, 1, 512)
                if q[0] != T or q[3] > 116 * 1024:
                    continue
                t, _ = timed(p, orb, aux)
                if t < best[0]:
                    best = (t, T, G)
        lx.tile_hint(la, lb, lc, kab, 1, 0, 0)
        lx.tile_hint(lb, la, lc, kab, 1, 0, 0)
        if best[1] and best[0] < (1.0 - args.margin) * t_def:
            for (x, y) in {(la, lb), (lb, la)}:
                lines.append("%d %d %d 1 %d 1 0 %d %d  # default T=%d G=%d %.3f ms -> %.3f ms"
                             % (x, y, lc, kab, best[1], best[2], s_def[0], s_def[1], t_def, best[0]))
        print("(%d %d|%d) Ka=%d Kb=%d: default %.3f ms (T=%d G=%d), best %.3f ms (T=%d G=%d)"
              % (la, lb, lc, ka, kb, t_def, s_def[0], s_def[1], best[0], best[1], best[2]), flush=True)
    dev = torch.cuda.get_device_name()
    head = ["# Tile hints for lx3c (load_shape_hints): la lb lc bra_pure kab kc 0 T G",
            "# written by paper_2210_03192_gb300/tune_tiles.py on %s, %d pairs x 512 ket shells per class"
            % (dev, args.npair)]
    text = "\n".join(([] if args.append else head) + sorted(set(lines))) + "\n"
    if args.out:
        with open(args.out, "a" if args.append else "w") as f:
            f.write(text)
    print("tuned %d of %d classes in %.0f s, %d hint lines" % (done, len(classes), time.time() - t0, len(set(lines))))


if __name__ == "__main__":
    main()
