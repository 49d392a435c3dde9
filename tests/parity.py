"""Element-by-element comparison of GPU integral blocks with the CPU oracle.

Tolerance: every element within 1e-12 relative or 1e-14 absolute of the
oracle, or within 1e-12 of the largest magnitude in its (pair, aux) block
plus 1e-14 (the blockwise form for elements formed by cancellation, whose
own magnitude is far below their block's).  Nothing else is allowed: no
element may miss both forms.  The FP64 oracle is used first; any
(pair, aux) block holding an element outside the per-element form is
recomputed with the oracle's binary128 mode, which decides whether the GPU
or the FP64 oracle lost the digits (projecting a Cartesian bra onto solid
harmonics cancels strongly for compact shells far from their partners).
"""
import numpy as np

import oracle

RTOL, ATOL = 1e-12, 1e-14
BLOCK_RTOL, BLOCK_ATOL = 1e-12, 1e-14


def close(g, o, rtol=RTOL, atol=ATOL):
    return np.abs(g - o) <= np.maximum(rtol * np.abs(o), atol)


def within(g, o):
    """Per-element or blockwise tolerance (blocks are the last three axes)."""
    scale = np.abs(o).max(axis=(-3, -2, -1), keepdims=True)
    return close(g, o) | (np.abs(g - o) <= BLOCK_RTOL * scale + BLOCK_ATOL)


def reference(p, bra_pure, g):
    """Oracle blocks for problem p, binary128 where the FP64 ones disagree with g."""
    o = oracle.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=bra_pure)
    bad = ~close(g, o)
    blocks = np.argwhere(bad.any(axis=(2, 3, 4)))
    if len(blocks):
        q = oracle.eri3c_triples(p.orb, p.aux, p.pairs[blocks[:, 0]], p.auxs[blocks[:, 1]], bra_pure=bra_pure,
                                 mode="quad")
        for (ip, iq), X in zip(blocks, q):
            o[ip, iq] = X
    return o, len(blocks)


def stats(g, o):
    d = np.abs(g - o)
    scale = np.abs(o).max(axis=(2, 3, 4), keepdims=True)
    blk = d / np.where(scale > 0, scale, 1.0)
    return dict(nbad=int((~close(g, o)).sum()), n=int(o.size), max_block_rel=float(blk.max()),
                max_abs=float(d.max()))


def assert_parity(g, p, bra_pure=True):
    o, nq = reference(p, bra_pure, g)
    strict = close(g, o)
    ok = within(g, o)
    if not ok.all():
        bad = np.argwhere(~ok)[:5]
        msg = ["%s gpu=%r oracle=%r" % (tuple(int(x) for x in b), g[tuple(b)], o[tuple(b)]) for b in bad]
        raise AssertionError("%d of %d elements outside tolerance (%d blocks rechecked in binary128):\n%s"
                             % ((~ok).sum(), ok.size, nq, "\n".join(msg)))
    return dict(strict_miss=int((~strict).sum()), n=int(o.size))
