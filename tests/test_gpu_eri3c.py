"""GPU parity: (ab|C) from the CUDA path against the CPU oracle, element by element.

Tolerance (stated by the target): each element within 1e-12 relative or
1e-14 absolute of the oracle; blocks the FP64 oracle cannot settle are
recomputed in binary128 (tests/parity.py).
"""
import numpy as np
import pytest

import oracle
from paper_2210_03192_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from parity import assert_parity  # noqa: E402


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03192_gb300 as m
    return m


def run(lx, p, bra_pure=True):
    out = lx.eri3c(p.orb, p.aux, p.pairs, p.auxs, bra_pure=bra_pure)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_ppd_64x32_full(lx):
    """(pp|d), K=1, 64 pairs x 32 aux shells: every integral."""
    p = W.ppd_64x32()
    assert_parity(run(lx, p), p)


SMALL = [(la, lb, lc) for la in range(5) for lb in range(5) for lc in range(7)]


@pytest.mark.parametrize("la,lb,lc", SMALL)
@pytest.mark.parametrize("Kab", [1, 3])
def test_class_small(lx, la, lb, lc, Kab):
    """Every (la, lb <= 4 | lc <= 6) class, 5 pairs x 7 aux shells, K_a = K_b = Kab."""
    p = W.class_problem(la, lb, lc, 5, 7, Kab, Kab, 1, box=6.0, exp_lo=0.1, exp_hi=50.0,
                        seed=1000 + la * 100 + lb * 10 + lc + 7 * Kab)
    assert_parity(run(lx, p), p)


@pytest.mark.parametrize("la,lb,lc", [(1, 1, 1), (2, 1, 3), (3, 3, 2), (4, 2, 5), (2, 4, 6)])
def test_cartesian_bra(lx, la, lb, lc):
    p = W.class_problem(la, lb, lc, 4, 9, 2, 1, 2, box=5.0, exp_lo=0.2, exp_hi=20.0, seed=77 + la + lb + lc)
    assert_parity(run(lx, p, bra_pure=False), p, bra_pure=False)


@pytest.mark.parametrize("la,lb,lc,Ka,Kb,Kc", [(2, 2, 2, 6, 6, 1), (1, 0, 3, 3, 2, 3), (4, 4, 6, 6, 6, 1),
                                                (0, 0, 0, 6, 6, 4), (3, 1, 4, 1, 6, 2), (0, 0, 5, 3, 6, 2)])
def test_high_contraction(lx, la, lb, lc, Ka, Kb, Kc):
    p = W.class_problem(la, lb, lc, 3, 40, Ka, Kb, Kc, box=8.0, exp_lo=0.05, exp_hi=1e4,
                        seed=300 + la + 10 * lb + 100 * lc)
    assert_parity(run(lx, p), p)


@pytest.mark.parametrize("la,lb,lc", [(0, 0, 0), (0, 0, 4), (0, 0, 6), (1, 0, 0), (1, 0, 4), (0, 1, 2), (0, 1, 3)])
def test_register_resident_classes_across_blocks(lx, la, lb, lc):
    """(s s|C), (p s|C) and B-oriented (s p|C) run one thread per triple
    (blocks of 128 and 64 triples): 70 pairs x 37 kets (2,590 triples, the
    last block ragged), contracted on both sides of the bra and in the ket,
    every integral against the oracle."""
    p = W.class_problem(la, lb, lc, 70, 37, 3, 2, 2, box=8.0, exp_lo=0.05, exp_hi=1e4,
                        seed=4200 + 10 * la + 5 * lb + lc)
    assert_parity(run(lx, p), p)
    if la + lb:
        assert_parity(run(lx, p, bra_pure=False), p, bra_pure=False)


def test_ragged_and_single(lx):
    """Aux lists that leave a partial last tile, a single pair, a single aux shell."""
    for (np_, na) in [(1, 1), (1, 33), (2, 129), (3, 257)]:
        p = W.class_problem(1, 2, 1, np_, na, 2, 1, 1, box=6.0, seed=900 + na)
        assert_parity(run(lx, p), p)
        p = W.class_problem(3, 3, 4, np_, na, 1, 1, 1, box=6.0, seed=901 + na)
        assert_parity(run(lx, p), p)


def test_host_path_matches_device(lx):
    p = W.class_problem(2, 1, 2, 6, 17, 3, 3, 1, box=6.0, seed=55)
    g = run(lx, p)
    h = lx.eri3c_host(p.orb, p.aux, p.pairs, p.auxs)
    np.testing.assert_array_equal(g, h)


def test_host_path_chunked(lx):
    """Host path over several ~512 MB output chunks (two device buffers, copies
    overlapped with compute) against the device path, bit for bit; random
    exponents give pairs split between both orientations at chunk edges."""
    p = W.class_problem(4, 4, 6, 300, 512, 1, 1, 1, box=20.0, exp_lo=0.05, exp_hi=1e4, seed=77)
    g = run(lx, p)
    h = torch.empty(g.size, dtype=torch.float64, pin_memory=True).numpy().reshape(g.shape)
    lx.eri3c_host(p.orb, p.aux, p.pairs, p.auxs, out=h)
    assert h.nbytes > 2 * (512 << 20)
    np.testing.assert_array_equal(g, h)


def test_boys_device(lx):
    """Device Boys evaluator against the oracle's extended-precision Boys function."""
    rng = np.random.default_rng(3)
    T = np.concatenate([np.zeros(1), rng.uniform(0, 1, 200), rng.uniform(0, 40, 400), rng.uniform(40, 130, 300),
                        10 ** rng.uniform(2, 6, 200), np.arange(0, 117, 0.125), [116.9999999, 117.0, 117.0000001]])
    mmax = 24
    g = lx.boys(torch.tensor(T, device="cuda"), mmax).cpu().numpy()
    ref = np.array([oracle.boys(mmax, t, mode="quad") for t in T])
    rel = np.abs(g - ref) / np.abs(ref)
    # interpolation region: a few ulp; T >= 117: F_24 = Gamma(24.5)/2 T^-24.5 by
    # 24 multiplications, about one ulp each
    small = T < 117.0
    assert rel[small].max() < 3e-15, (rel[small].max(), T[small][np.unravel_index(rel[small].argmax(), rel[small].shape)[0]])
    assert rel[~small].max() < 6e-15, (rel[~small].max(), T[~small][np.unravel_index(rel[~small].argmax(), rel[~small].shape)[0]])


HRR2 = [(la, lb, lc) for la in range(5) for lb in range(2, 5) for lc in (0, 2, 4, 6)]


@pytest.mark.parametrize("la,lb,lc", HRR2)
def test_class_two_quantum_hrr(lx, la, lb, lc):
    """Classes with lb >= 2 through the two-quantum HRR rounds of Sec. 2.5.5
    (both orientations hinted), against the oracle with the same criterion."""
    p = W.class_problem(la, lb, lc, 5, 7, 2, 2, 1, box=6.0, exp_lo=0.1, exp_hi=50.0,
                        seed=2000 + la * 100 + lb * 10 + lc)
    for (a, b) in {(la, lb), (lb, la)}:
        lx.hrr_hint(a, b, lc, 1)
    try:
        g = run(lx, p)
    finally:
        for (a, b) in {(la, lb), (lb, la)}:
            lx.hrr_hint(a, b, lc, -1)
    assert_parity(g, p)
