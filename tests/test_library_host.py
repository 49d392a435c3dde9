"""Host-side checks of the C-ABI library (no GPU needed).

The shared library loads, exports every function include/lx3c.h declares,
validates malformed input before touching the device, and its host-built
tables agree with the paper's worked CVRR2 expansions (Sec. 2.5.4) and with
the oracle's independently derived solid harmonics.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.solid import solid_matrix
import paper_2210_03192_gb300 as lx
from paper_2210_03192_gb300 import _lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lx3c.h")
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cvrr2_worked_examples.txt")


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lx3c_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol():
    L = _lib.load()
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(_lib.EXPORTS), set(names) - set(_lib.EXPORTS)


def test_invalid_input_rejected_on_host():
    L = _lib.load()
    h = ctypes.c_void_p()
    l = np.array([1], np.int32)
    k = np.array([1], np.int32)
    xyz = np.zeros(3)
    bad_exp = np.array([-1.0])
    co = np.array([1.0])
    rc = L.lx3c_basis_create(ctypes.byref(h), 1, l.ctypes.data, k.ctypes.data, xyz.ctypes.data, None,
                             bad_exp.ctypes.data, co.ctypes.data, None)
    assert rc == -1 and b"exponent" in L.lx3c_last_error()
    big_l = np.array([9], np.int32)
    rc = L.lx3c_basis_create(ctypes.byref(h), 1, big_l.ctypes.data, k.ctypes.data, xyz.ctypes.data, None,
                             co.ctypes.data, co.ctypes.data, None)
    assert rc == -2
    big_k = np.array([99], np.int32)
    rc = L.lx3c_basis_create(ctypes.byref(h), 1, l.ctypes.data, big_k.ctypes.data, xyz.ctypes.data, None,
                             co.ctypes.data, co.ctypes.data, None)
    assert rc == -2
    rc = L.lx3c_eri3c_plan(ctypes.byref(h), None, None, None, 0, None, 0, 1, None)
    assert rc == -1
    rc = L.lx3c_eri3c_execute(None, None, None)
    assert rc == -1
    f = ctypes.c_double()
    assert L.lx3c_class_flops(-1, 0, 0, 1, 1, 1, ctypes.byref(f)) == -1


@pytest.mark.parametrize("l", range(0, 9))
def test_solid_harmonics_match_oracle(l):
    np.testing.assert_allclose(lx.solid_harmonics(l), solid_matrix(l), rtol=1e-14, atol=1e-14 * 10 ** (l / 2))


def test_cvrr2_worked_examples():
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        a, c, terms = (p.strip() for p in line.split("|"))
        vec = lambda s: tuple(int(x) for x in s.split(","))
        ref = {}
        for t in terms.split():
            coef, e, kk, n = t.split(":")
            ref[(vec(e), int(kk), vec(n))] = float(coef)
        assert lx.cvrr2_expansion(vec(a), vec(c)) == ref


def test_cvrr2_closed_form_all_targets():
    """The library's tabulated n-q expansion equals the closed form for every
    (a, c) up to |a| = 8, |c| = 6."""
    from math import comb, factorial
    from oracle.solid import cart_list
    for la in (0, 3, 8):
        for lc in (0, 2, 6):
            for a in cart_list(la):
                for c in cart_list(lc):
                    ref = {}
                    for ux in range(min(a[0], c[0]) + 1):
                        for uy in range(min(a[1], c[1]) + 1):
                            for uz in range(min(a[2], c[2]) + 1):
                                u = (ux, uy, uz)
                                coef = 1
                                for i in range(3):
                                    coef *= comb(a[i], u[i]) * comb(c[i], u[i]) * factorial(u[i])
                                key = (tuple(a[i] - u[i] for i in range(3)), sum(u),
                                       tuple(c[i] - u[i] for i in range(3)))
                                ref[key] = ref.get(key, 0) + coef
                    assert lx.cvrr2_expansion(a, c) == {k: float(v) for k, v in ref.items()}


def test_class_flops_scale_with_contraction():
    f1 = lx.class_flops(4, 4, 6, 1)
    f2 = lx.class_flops(4, 4, 6, 2)
    f36 = lx.class_flops(4, 4, 6, 36)
    assert f36 - f1 == pytest.approx(35 * (f2 - f1))   # per-primitive work is linear in K
    assert lx.class_flops(0, 0, 0, 1) < lx.class_flops(1, 0, 0, 1) < lx.class_flops(1, 1, 0, 1)


def test_device_calls_fail_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(lx.LibraryError):
        lx.boys(torch.zeros(3, dtype=torch.float64), 4)


def test_shape_query_budgets_and_hints(tmp_path):
    """Planner shapes fit their CTAs-per-SM budget; a hint switches the default
    shape of exactly its class; a hints file applies and removes cleanly."""
    import paper_2210_03192_gb300 as lx
    smem = 233472
    for (la, lb, lc, kab) in [(4, 4, 6, 36), (4, 4, 1, 36), (2, 2, 2, 1), (0, 0, 0, 9), (3, 2, 5, 9)]:
        for ctas in (1, 2, 3):
            T, G, mode, sb = lx.shape_query(la, lb, lc, kab, 1, 512, ctas)
            assert T >= 1 and 1 <= G <= min(kab, 8) and mode == (0 if T >= 32 else 1)
            # fits the budget, or is the fallback of a smaller CTA count
            assert sb <= smem - 1024
            if sb > smem // ctas - 1024:
                assert lx.shape_query(la, lb, lc, kab, 1, 512, ctas) == lx.shape_query(la, lb, lc, kab, 1, 512, ctas - 1)
        default = lx.shape_query(la, lb, lc, kab, 1, 512, 0)
        assert default == lx.shape_query(la, lb, lc, kab, 1, 512, 2)
    three = lx.shape_query(4, 4, 1, 36, 1, 512, 3)
    lx.shape_hint(4, 4, 1, 36, 1, 3)
    try:
        assert lx.shape_query(4, 4, 1, 36, 1, 512, 0) == three
        assert lx.shape_query(4, 4, 1, 9, 1, 512, 0) == lx.shape_query(4, 4, 1, 9, 1, 512, 2)  # other kab untouched
    finally:
        lx.shape_hint(4, 4, 1, 36, 1, 0)
    assert lx.shape_query(4, 4, 1, 36, 1, 512, 0) == lx.shape_query(4, 4, 1, 36, 1, 512, 2)
    f = tmp_path / "hints.txt"
    f.write_text("# la lb lc pure kab kc ctas\n4 4 1 1 36 1 3\n2 2 2 1 1 1 1\n")
    assert lx.load_shape_hints(str(f)) == 2
    try:
        assert lx.shape_query(4, 4, 1, 36, 1, 512, 0) == three
        assert lx.shape_query(2, 2, 2, 1, 1, 512, 0) == lx.shape_query(2, 2, 2, 1, 1, 512, 1)
    finally:
        lx.shape_hint(4, 4, 1, 36, 1, 0)
        lx.shape_hint(2, 2, 2, 1, 1, 0)
    with pytest.raises(lx.LibraryError):
        lx.shape_hint(4, 4, 1, 36, 1, 4)
    with pytest.raises(lx.LibraryError):
        lx.shape_query(9, 4, 1, 36, 1, 512, 2)



def test_tile_hints_fix_the_tile_and_take_precedence(tmp_path):
    """A tile hint fixes (T, G) of exactly its class (G balanced over the
    chunks), wins over a CTAs-per-SM hint, is ignored when the tile cannot fit
    one CTA's shared memory, and rejects arguments out of range."""
    L = _lib.load()
    default = lx.shape_query(0, 0, 6, 36, 1, 512)
    lx.shape_hint(0, 0, 6, 36, 1, 3)
    lx.tile_hint(0, 0, 6, 36, 1, 16, 8)
    try:
        T, G, mode, sb = lx.shape_query(0, 0, 6, 36, 1, 512)
        # 36 primitives in chunks of at most 8: five chunks, balanced to 8 (8+8+8+8+4)
        assert (T, G, mode) == (16, 8, 1) and 0 < sb <= 233472 - 1024
        lx.tile_hint(0, 0, 6, 36, 1, 4, 36)
        assert lx.shape_query(0, 0, 6, 36, 1, 512)[:3] == (4, 36, 1)
        lx.tile_hint(0, 0, 6, 36, 1, 32, 12)  # 36 in chunks of 12: three chunks of 12
        assert lx.shape_query(0, 0, 6, 36, 1, 512)[:3] == (32, 12, 0)
        assert lx.shape_query(0, 0, 6, 9, 1, 512) == lx.shape_query(0, 0, 6, 9, 1, 512, 2)  # other kab untouched
        lx.tile_hint(4, 4, 6, 36, 1, 512, 36)  # far beyond one CTA's shared memory: ignored
        assert lx.shape_query(4, 4, 6, 36, 1, 512) == lx.shape_query(4, 4, 6, 36, 1, 512, 2)
    finally:
        lx.tile_hint(0, 0, 6, 36, 1, 0, 0)
        lx.tile_hint(4, 4, 6, 36, 1, 0, 0)
        lx.shape_hint(0, 0, 6, 36, 1, 0)
    assert lx.shape_query(0, 0, 6, 36, 1, 512) == default
    assert L.lx3c_tile_hint(0, 0, 6, 1, 36, 1, 513, 1) == -1
    assert L.lx3c_tile_hint(0, 0, 6, 1, 36, 1, 16, 37) == -1
    assert L.lx3c_tile_hint(0, 0, 6, 1, 36, 1, 16, 0) == -1
    assert L.lx3c_tile_hint(0, 0, 9, 1, 36, 1, 16, 8) == -1
    f = tmp_path / "tiles.txt"
    f.write_text("# la lb lc pure kab kc 0 T G\n0 0 6 1 36 1 0 8 18\n0 0 5 1 36 1 3\n")
    assert lx.load_shape_hints(str(f)) == 2
    try:
        assert lx.shape_query(0, 0, 6, 36, 1, 512)[:2] == (8, 18)
        assert lx.shape_query(0, 0, 5, 36, 1, 512) == lx.shape_query(0, 0, 5, 36, 1, 512, 3)
    finally:
        lx.tile_hint(0, 0, 6, 36, 1, 0, 0)
        lx.shape_hint(0, 0, 5, 36, 1, 0)

def test_committed_shape_hints_file():
    """The shipped GB300 hints: every line a valid class with a 1-3 CTA target
    or a (T, G) tile, loadable; a tile hint decides its class's shape (G
    balanced over the chunks) and fits one CTA's shared memory; a CTA hint
    decides the others' and fits its target's."""
    import paper_2210_03192_gb300 as lx
    ctas_lines, tile_lines = [], []
    with open(lx.HINTS_GB300) as f:
        for line in f:
            fields = line.split("#", 1)[0].split()
            if not fields:
                continue
            v = tuple(int(x) for x in fields)
            assert len(v) in (7, 9), v
            (tile_lines if len(v) == 9 else ctas_lines).append(v)
    assert ctas_lines and tile_lines
    for (la, lb, lc, pure, kab, kc, ctas) in ctas_lines:
        assert 0 <= la <= 4 and 0 <= lb <= 4 and 0 <= lc <= 6 and pure == 1 and kab in (1, 9, 36) and kc == 1
        assert ctas in (1, 3)
    for (la, lb, lc, pure, kab, kc, zero, T, G) in tile_lines:
        assert 0 <= la <= 4 and 0 <= lb <= 4 and 0 <= lc <= 6 and pure == 1 and kc == 1 and zero == 0
        assert kab in (3, 6, 9, 18, 36) and 1 <= T <= 512 and 1 <= G <= kab
    tiled = {v[:6]: v for v in tile_lines}
    try:
        assert lx.load_shape_hints() == len(ctas_lines) + len(tile_lines)
        for (la, lb, lc, pure, kab, kc, zero, T, G) in tiled.values():
            nch = -(-kab * kc // G)
            Tq, Gq, mode, sb = lx.shape_query(la, lb, lc, kab, kc, 512, 0)
            assert (Tq, Gq) == (T, -(-kab * kc // nch)) and mode == (0 if T >= 32 else 1)
            assert sb <= 233472 - 1024
        for (la, lb, lc, pure, kab, kc, ctas) in ctas_lines:
            if (la, lb, lc, pure, kab, kc) in tiled:
                continue
            T, G, mode, sb = lx.shape_query(la, lb, lc, kab, kc, 512, 0)
            assert (T, G, mode, sb) == lx.shape_query(la, lb, lc, kab, kc, 512, ctas)
            assert sb <= 233472 // ctas - 1024 or ctas == 1
    finally:
        for (la, lb, lc, pure, kab, kc, ctas) in ctas_lines:
            lx.shape_hint(la, lb, lc, kab, kc, 0)
        for v in tile_lines:
            lx.tile_hint(v[0], v[1], v[2], v[4], v[5], 0, 0)


def test_more_entry_points_reject_bad_arguments_on_host():
    """Argument checks that run before any device work: null or empty inputs,
    out-of-range sizes and modes give LX3C_EINVAL (-1) or LX3C_ENOTSUP (-2)
    with an error message, on every family of calls."""
    L = _lib.load()
    h = ctypes.c_void_p()
    # DF-J / gradient
    assert L.lx3c_dfj_plan(ctypes.byref(h), None, None, 1e-12, 0, None) == -1
    assert L.lx3c_dfj_execute(None, None, None, None, None, None) == -1
    assert L.lx3c_dfj_energy(None, None, None, None, None, None) == -1
    assert L.lx3c_dfj_grad(None, None, None, None, None) == -1
    assert L.lx3c_dfj_info(None, None, 0) == -1
    assert L.lx3c_dfj_group(None, 0, None, None, None, None) == -1
    # batch
    assert L.lx3c_batch_plan(ctypes.byref(h), 0, None, None, 1e-12, None, None) == -1
    assert L.lx3c_batch_bind(None, None, None, None, None, None) == -1
    assert L.lx3c_batch_execute(None, 1, None) == -1
    assert L.lx3c_batch_info(None, None, 0) == -1
    # allocation-free class call: limits checked before the device is touched
    nul = [None] * 9
    assert L.lx3c_eri3c_noalloc(7, 0, 0, 1, 1, 1, 1, *nul, 1, None, 1, None, None) == -2   # l beyond 6
    assert L.lx3c_eri3c_noalloc(1, 0, 0, 17, 1, 1, 1, *nul, 1, None, 1, None, None) == -2  # K beyond 16
    assert L.lx3c_eri3c_noalloc(1, 0, 0, 1, 1, 1, 1, *nul, 0, None, 1, None, None) == -1   # empty pair list
    assert L.lx3c_eri3c_noalloc(1, 0, 0, 1, 1, 1, 1, *nul, 1, None, 1, None, None) == -1   # null pointers
    msg = L.lx3c_last_error()
    assert msg and b"null" in msg
    # beyond the static scratch limits: rejected before any device pointer is used
    fake = [ctypes.c_void_p(256)] * 9
    assert L.lx3c_eri3c_noalloc(1, 1, 0, 1, 1, 1, 1, *fake, 65537, ctypes.c_void_p(256), 1, ctypes.c_void_p(256),
                                None) == -2
    assert L.lx3c_eri3c_noalloc(1, 1, 0, 2, 2, 1, 1, *fake, 16385, ctypes.c_void_p(256), 1, ctypes.c_void_p(256),
                                None) == -2  # npair * ka * kb > 65536
    assert L.lx3c_eri3c_noalloc(1, 1, 0, 1, 1, 2, 1, *fake, 1, ctypes.c_void_p(256), 32769, ctypes.c_void_p(256),
                                None) == -2  # naux * kc > 65536
    assert b"scratch limits" in L.lx3c_last_error()
    # accuracy settings, FP64 rate, metric and Cholesky
    assert L.lx3c_set_orientation_threshold(0.5) == -1
    assert L.lx3c_set_orientation_threshold(float("inf")) == -1
    assert L.lx3c_set_orientation_threshold(0.0) == 0
    assert L.lx3c_set_compensation(4) == -1 and L.lx3c_set_compensation(-1) == -1
    assert L.lx3c_set_compensation(0) == 0
    assert L.lx3c_fp64_rate(0, None, None, None) == -1
    assert L.lx3c_metric_plan(ctypes.byref(h), None, None) == -1
    assert L.lx3c_metric_execute(None, None, None) == -1
    assert L.lx3c_metric_info(None, None, 0) == -1
    assert L.lx3c_cholesky(None, 4, 4, 0.0, None, None) == -1
    assert L.lx3c_cholesky(ctypes.c_void_p(256), 4, 3, 0.0, None, None) == -1
    assert L.lx3c_cholesky(ctypes.c_void_p(256), 4, 4, 1.0, None, None) == -1
    assert L.lx3c_cholesky_solve(None, 4, 4, None, 1, None) == -1
    assert L.lx3c_dfj_coulomb(None, None, 0, None, None, None, None, None) == -1
    q = ctypes.c_double()
    assert L.lx3c_schwarz_pair(0, 0, None, None, None, 0, 1, None, None, None, ctypes.byref(q)) == -1
    assert L.lx3c_schwarz_aux(-1, 1, None, None, ctypes.byref(q)) == -1
    # host-buffer path and Boys
    assert L.lx3c_eri3c_host(0, None, None, None, None, None, 0, None, None, None, None, None, None, 0, None, 0,
                             1, None, None) == -1
    assert L.lx3c_boys(None, 4, 3, None, None) == -1
    assert L.lx3c_boys(None, 1, 25, None, None) == -1


def test_class_tables_invariants_every_class():
    """The planner's host tables satisfy their invariants (lx3c_class_tables_check)
    for every integral class (pure bra, la, lb <= 4) and every derivative class
    the gradient uses (Cartesian bra, one shell raised to l <= 5), lc <= 6."""
    L = _lib.load()
    cases = [(la, lb, lc, 1) for la in range(5) for lb in range(5) for lc in range(7)]
    cases += [(la, lb, lc, 0) for la in range(6) for lb in range(6) if la + lb <= 9 for lc in range(7)]
    bad = []
    for (la, lb, lc, pure) in cases:
        if L.lx3c_class_tables_check(la, lb, lc, pure) != 0:
            bad.append((la, lb, lc, pure, L.lx3c_last_error()))
    assert not bad, bad[:5]
    assert L.lx3c_class_tables_check(-1, 0, 0, 1) == -1


@pytest.mark.parametrize("variant", [0, 1])
def test_hrr_tables_exact_on_moment_integrals(variant):
    """Both HRR variants (one or two quanta per round, Eq. hrr / Sec. 2.5.5)
    reproduce moment integrals int (x-A)^a (x-B)^b w dx, for which HRR is
    exact, for every bra class up to (hh|, and pass the table invariants."""
    L = _lib.load()
    AB = np.array([0.7, -1.3, 2.1])
    e = ctypes.c_double()
    for la in range(6):
        for lb in range(6):
            for lc in (0, 4):
                assert L.lx3c_hrr_tables_check(la, lb, lc, 1, variant, AB.ctypes.data, ctypes.byref(e)) == 0, \
                    L.lx3c_last_error()
                assert e.value < 1e-14, (la, lb, lc, e.value)
