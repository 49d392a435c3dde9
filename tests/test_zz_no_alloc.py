"""The allocation-free entry point lx3c_eri3c_noalloc against the planned path.

lx3c_eri3c_noalloc is for callers that cannot allocate device memory around
the call: code running while a pool allocator owns the device heap (a raw
cudaMalloc there can fail or fragment the pool) and code that must not let
cudaFree synchronise the whole device.  Its scratch lives in one static
device array shared by all calls.

This test calls it through the C ABI three times in a row on one stream,
with no synchronisation between the calls, on three classes (the last with
lb = 0, which has no orientation split), so each call overwrites what the
previous one left in the shared array while the previous kernels may still
be queued.  Each output is then checked against lx3c_eri3c_execute and
against the oracle, with the tolerance the other parity tests use
(tests/parity.py).  It sits in a file of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_2210_03192_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity import assert_parity, within  # noqa: E402  (the tolerance the parity tests use)


def dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a, dt), device="cuda")


def launch_noalloc(lx, p, bra_pure=True):
    """Queue one call on the current stream; returns (output tensor, inputs kept alive)."""
    L = lx._lib.load()
    la, lb, lc = p.la, p.lb, p.lc
    ka, kb, kc = int(p.orb.k[p.pairs[0, 0]]), int(p.orb.k[p.pairs[0, 1]]), int(p.aux.k[p.auxs[0]])
    keep = [dev(p.orb.off, np.int64), dev(p.orb.xyz, np.float64), dev(p.orb.exps, np.float64),
            dev(p.orb.coefs, np.float64), dev(p.aux.off, np.int64), dev(p.aux.xyz, np.float64),
            dev(p.aux.exps, np.float64), dev(p.aux.coefs, np.float64), dev(p.pairs, np.int32),
            dev(p.auxs, np.int32)]
    nA = 2 * la + 1 if bra_pure else (la + 1) * (la + 2) // 2
    nB = 2 * lb + 1 if bra_pure else (lb + 1) * (lb + 2) // 2
    out = torch.full((p.npair, p.naux, nA, nB, 2 * lc + 1), float("nan"), dtype=torch.float64, device="cuda")
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in keep]
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.lx3c_eri3c_noalloc(la, lb, lc, ka, kb, kc, int(bra_pure), *ptrs[:8], ptrs[8], p.npair, ptrs[9], p.naux,
                              ctypes.c_void_p(out.data_ptr()), st)
    assert rc == 0, L.lx3c_last_error()
    return out, keep


def test_noalloc_matches_planned_path_three_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03192_gb300 as lx
    cases = [W.class_problem(2, 3, 4, 7, 45, 3, 2, 1, box=6.0, exp_lo=0.1, exp_hi=50.0, seed=4242),
             W.class_problem(3, 1, 2, 5, 70, 2, 3, 2, box=6.0, exp_lo=0.1, exp_hi=50.0, seed=4343),
             W.class_problem(2, 0, 3, 9, 33, 3, 1, 1, box=6.0, exp_lo=0.1, exp_hi=50.0, seed=4444),
             # register-resident classes: (s s|d), and (s p|f) whose B-oriented
             # list adds onto the A-oriented one
             W.class_problem(0, 0, 2, 11, 50, 3, 2, 1, box=6.0, exp_lo=0.1, exp_hi=50.0, seed=4545),
             W.class_problem(0, 1, 3, 11, 50, 3, 2, 1, box=6.0, exp_lo=0.05, exp_hi=1e4, seed=4646)]
    queued = [launch_noalloc(lx, p) for p in cases]  # back to back, no synchronisation in between
    torch.cuda.synchronize()
    got = [out.cpu().numpy() for out, _ in queued]
    for p, g in zip(cases, got):
        assert np.isfinite(g).all()
        ref = lx.eri3c(p.orb, p.aux, p.pairs, p.auxs).cpu().numpy()
        ok = within(g, ref)
        assert ok.all(), (np.abs(g - ref).max(), (~ok).sum())
        assert_parity(g, p)
