"""GPU parity for the density-fitting metric V_PQ = (P|Q), its Cholesky
factor, the solve c = V^{-1} gamma and the one-call DF-J Coulomb build
(Sec. 1 and Sec. 4: density fitting of the Coulomb operator).

V is compared element by element with the binary128 oracle (1e-12 relative
or 1e-14 absolute, else 1e-12 of its shell-pair block's largest element plus
1e-14 of the block's Cauchy-Schwarz scale, see blocks_ok).  The factor and the solve are compared with numpy's on the
same matrices; their forward error is bounded by the condition number, so
those tolerances carry kappa(V) explicitly.
"""
import numpy as np
import pytest

import oracle
from paper_2210_03192_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AUX_METRIC = [(0, 3, 2), (1, 2, 1), (2, 2, 1), (3, 1, 1), (4, 1, 1), (5, 1, 1), (6, 1, 1)]


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03192_gb300 as m
    return m


def blocks_ok(G, O, aux):
    """Per element 1e-12 relative or 1e-14 absolute; else within
    1e-12 max|block| + 1e-14 S_PQ, with S_PQ = sqrt(max (P|P) max (Q|Q)) the
    block's Cauchy-Schwarz scale.  The primitives are not normalised (their
    coefficients are used as given), so an absolute 1e-14 means nothing by
    itself: S_PQ puts it at the scale of the two functions, where it is the
    1e-14 of unit-normalised ones.  It decides blocks that vanish, or nearly,
    by symmetry (same-centre pairs with l_P != l_Q are exactly zero), whose
    computed values are the rounding of intermediates of size S_PQ."""
    aq = oracle.ao_offsets(aux)
    err = np.abs(G - O)
    dg = np.diag(O)
    strict = err <= np.maximum(1e-12 * np.abs(O), 1e-14)
    ok = strict.copy()
    for i in range(aux.nshell):
        for j in range(aux.nshell):
            s = (slice(aq[i], aq[i + 1]), slice(aq[j], aq[j + 1]))
            spq = np.sqrt(dg[aq[i]:aq[i + 1]].max() * dg[aq[j]:aq[j + 1]].max())
            ok[s] |= err[s] <= 1e-12 * np.abs(O[s]).max() + 1e-14 * spq
    return ok


def missed_blocks(G, O, aux, ok):
    """(P, Q, l_P, l_Q, K_P, K_Q, |R_PQ|, max err / block max) of each block
    holding an element outside the criterion."""
    aq = oracle.ao_offsets(aux)
    out = []
    for i in range(aux.nshell):
        for j in range(aux.nshell):
            s = (slice(aq[i], aq[i + 1]), slice(aq[j], aq[j + 1]))
            if not ok[s].all():
                r = float(np.linalg.norm(aux.xyz[i] - aux.xyz[j]))
                e = np.abs(G[s] - O[s]).max() / np.abs(O[s]).max()
                out.append((i, j, int(aux.l[i]), int(aux.l[j]), int(aux.k[i]), int(aux.k[j]), r, e))
    return out


def test_metric_matches_oracle(lx):
    cl = W.cluster((2, 1, 1), W.ORB_RECIPE_DFJ, AUX_METRIC, seed=501, exp_lo=0.05, exp_hi=1e3)
    mp = lx.MetricPlan(cl.aux)
    assert mp.naux_ao == int(oracle.ao_offsets(cl.aux)[-1])
    V = mp.execute().cpu().numpy()
    O = oracle.metric(cl.aux, mode="quad")
    ok = blocks_ok(V, O, cl.aux)
    assert ok.all(), missed_blocks(V, O, cl.aux, ok)
    assert np.abs(V - V.T).max() <= 1e-12 * np.abs(V).max()


def spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return M @ M.T / n + np.eye(n)


@pytest.mark.parametrize("n", [1, 63, 64, 65, 200, 1000])
def test_cholesky_matches_numpy(lx, n):
    A = spd(n, n)
    At = torch.tensor(A, device="cuda")
    _, info = lx.cholesky(At)
    assert info == 0
    L = At.cpu().numpy()
    Lr = np.linalg.cholesky(A)
    np.testing.assert_allclose(np.tril(L), Lr, rtol=0, atol=1e-13 * np.abs(Lr).max())
    # the strictly upper triangle is not written
    iu = np.triu_indices(n, 1)
    assert np.array_equal(L[iu], A[iu])


def test_cholesky_reports_first_nonpositive_pivot(lx):
    A = spd(130, 7)
    A[70, :] = 0.0
    A[:, 70] = 0.0  # row/column 71 (1-based) has a zero pivot after elimination
    _, info = lx.cholesky(torch.tensor(A, device="cuda"))
    assert info == 71


def conditioned_aux():
    """Two atoms 2 bohr apart, each with s(0.3), s(2.0), p(0.7), d(1.1),
    f(1.5), one primitive each, coefficients scaled so that diag(V) = 1:
    kappa(V) is about 5e2, so a solve residual measures the factor's
    accuracy rather than the basis's conditioning."""
    ls, ex, xyz = [], [], []
    for A in ([0.0, 0.0, 0.0], [0.0, 0.0, 2.0]):
        for l, a in ((0, 0.3), (0, 2.0), (1, 0.7), (2, 1.1), (3, 1.5)):
            ls.append(l)
            ex.append(a)
            xyz.append(A)
    ones = W.make_basis(ls, [1] * len(ls), xyz, ex, [1.0] * len(ls))
    d = np.diag(oracle.metric(ones))[oracle.ao_offsets(ones)[:-1]]
    return W.make_basis(ls, [1] * len(ls), xyz, ex, 1.0 / np.sqrt(d))


def test_cholesky_drops_dependent_functions(lx):
    """An aux basis holding one shell twice: the copy's pivots vanish, the
    drop mode removes exactly its 2l+1 functions, and the solve still
    satisfies V c = gamma (the copy's rows equal the original's) to the
    factor's rounding times kappa of the kept functions."""
    aux = conditioned_aux()
    dup = int(np.where(aux.l == 2)[0][0])
    aux2 = aux.subset(list(range(aux.nshell)) + [dup])
    V = lx.MetricPlan(aux2).execute()
    V0 = V.cpu().numpy()
    _, info = lx.cholesky(V, drop_tol=1e-12)
    assert info == 5
    rng = np.random.default_rng(4)
    g = rng.standard_normal(V0.shape[0])
    aq = oracle.ao_offsets(aux2)
    g[aq[-2]:aq[-1]] = g[aq[dup]:aq[dup + 1]]  # a consistent right-hand side
    c = lx.cholesky_solve(V, torch.tensor(g, device="cuda")).cpu().numpy()
    assert np.abs(c[aq[-2]:aq[-1]]).max() == 0.0
    keep = np.arange(aq[-2])
    kappa = np.linalg.cond(V0[np.ix_(keep, keep)])
    assert kappa < 1e4
    assert np.abs(V0 @ c - g).max() <= 20 * kappa * 2.2e-16 * np.abs(g).max()
    co = np.linalg.solve(V0[np.ix_(keep, keep)], g[keep])
    assert np.abs(c[keep] - co).max() <= 20 * kappa * 2.2e-16 * np.abs(co).max()


@pytest.mark.parametrize("n,nrhs", [(1, 1), (100, 1), (257, 3)])
def test_cholesky_solve(lx, n, nrhs):
    A = spd(n, 100 + n)
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, nrhs)) if nrhs > 1 else rng.standard_normal(n)
    At = torch.tensor(A, device="cuda")
    lx.cholesky(At)
    X = lx.cholesky_solve(At, torch.tensor(B, device="cuda")).cpu().numpy()
    Xr = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A)
    assert np.abs(X - Xr).max() <= 20 * kappa * 2.2e-16 * np.abs(Xr).max()


def test_metric_solve_and_dfj_coulomb(lx):
    cl = W.cluster((2, 1, 1), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=502)
    rng = np.random.default_rng(3)
    n = int(oracle.ao_offsets(cl.orb)[-1])
    D = W.density(rng, n)
    mp = lx.MetricPlan(cl.aux)
    V = mp.execute()
    Vo = oracle.metric(cl.aux, mode="quad")
    lx.cholesky(V)
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12)
    g, c, J = plan.coulomb(V, torch.tensor(D, device="cuda"))
    g, c, J = g.cpu().numpy(), c.cpu().numpy(), J.cpu().numpy()
    tasks = plan.tasks()
    go, _ = oracle.dfj(cl.orb, cl.aux, D, np.zeros(len(g)), tasks=tasks, mode="quad")
    assert np.abs(g - go).max() <= 1e-12 * np.abs(go).max()
    co = np.linalg.solve(Vo, go)
    kappa = np.linalg.cond(Vo)
    assert np.abs(c - co).max() <= 20 * kappa * 2.2e-16 * np.abs(co).max(), (np.abs(c - co).max() / np.abs(co).max(), kappa)
    # J from the GPU's own c: the integral contraction, without the solve's conditioning
    _, Jo = oracle.dfj(cl.orb, cl.aux, D, c, tasks=tasks, mode="quad")
    assert np.abs(J - Jo).max() <= 1e-12 * np.abs(Jo).max()
    np.testing.assert_allclose(J, J.T, rtol=0, atol=1e-14 * np.abs(J).max())
