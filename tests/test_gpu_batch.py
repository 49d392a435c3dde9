"""Batched uneven workload (16 molecules of 20-400 atoms, not in the paper): several
molecules' DF-J builds, every class mixed, as one persistent kernel inside one
CUDA graph, checked against the per-class launches and the oracle."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_2210_03192_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from dfj_sampling import sampled_against_oracle  # noqa: E402


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03192_gb300 as m
    return m


def normwise(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_batch_graph_equals_plain_and_oracle(lx):
    mols = [W.molecule(n, 500 + n, aux_fraction=0.5) for n in (2, 3, 5)]
    rng = np.random.default_rng(4)
    Ds, cs = [], []
    for cl in mols:
        n = int(oracle.ao_offsets(cl.orb)[-1])
        naux = int(oracle.ao_offsets(cl.aux)[-1])
        Ds.append(torch.tensor(W.density(rng, n), device="cuda"))
        cs.append(torch.tensor(rng.standard_normal(naux), device="cuda"))
    cache = os.path.join(tempfile.mkdtemp(), "tune.txt")
    b = lx.Batch([(cl.orb, cl.aux) for cl in mols], 1e-12, tune_cache=cache).bind(Ds, cs)
    info = b.info()
    assert info["graph_kernels"] >= 1 and info["work_items"] > 0 and info["branches"] == 4
    assert os.path.exists(cache) and info["tuned"] > 0
    g1, J1 = b.execute(mode=1)
    torch.cuda.synchronize()
    g1 = [g.cpu().numpy().copy() for g in g1]
    J1 = [J.cpu().numpy().copy() for J in J1]
    g2, J2 = b.execute(mode=2)
    torch.cuda.synchronize()
    g2 = [g.cpu().numpy().copy() for g in g2]
    J2 = [J.cpu().numpy().copy() for J in J2]
    g0, J0 = b.execute(mode=0)
    torch.cuda.synchronize()
    for m, cl in enumerate(mols):
        # the class launches on graph branches and the per-class launches run
        # the same kernels into exact fixed-point sums: bit for bit equal; the
        # persistent kernels run the tile body for every class, (s s|C)
        # included, whose products round in another order: equal to rounding
        g0m, J0m = g0[m].cpu().numpy(), J0[m].cpu().numpy()
        assert np.array_equal(g2[m], g0m) and np.array_equal(J2[m], J0m)
        assert np.abs(g1[m] - g0m).max() <= 1e-12 * np.abs(g0m).max()
        assert np.abs(J1[m] - J0m).max() <= 1e-12 * np.abs(J0m).max()
    assert info["branch_kernels"] == info["graph_kernels"] - info["tiers"] + info["class_launches"]
    # oracle on the smallest molecule, same screened tasks
    cl = mols[0]
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12)
    go, Jo = oracle.dfj(cl.orb, cl.aux, Ds[0].cpu().numpy(), cs[0].cpu().numpy(), tasks=plan.tasks(), mode="quad")
    assert normwise(g1[0], go) < 1e-12
    assert normwise(J1[0], Jo) < 1e-12
    # a second plan reads the cache instead of measuring
    b2 = lx.Batch([(cl.orb, cl.aux) for cl in mols], 1e-12, tune_cache=cache)
    assert b2.info()["measured"] == 0


def test_batch_replay_is_stable(lx):
    mols = [W.molecule(n, 600 + n, aux_fraction=0.3) for n in (4, 8)]
    rng = np.random.default_rng(5)
    Ds = [torch.tensor(W.density(rng, int(oracle.ao_offsets(cl.orb)[-1])), device="cuda") for cl in mols]
    cs = [torch.tensor(rng.standard_normal(int(oracle.ao_offsets(cl.aux)[-1])), device="cuda") for cl in mols]
    b = lx.Batch([(cl.orb, cl.aux) for cl in mols]).bind(Ds, cs)
    ga, _ = b.execute(1)
    ga = [g.cpu().numpy().copy() for g in ga]
    gb, _ = b.execute(1)
    for x, y in zip(ga, gb):
        assert np.array_equal(x, y.cpu().numpy())


def test_batch_members_of_the_16_molecule_workload(lx):
    """The two smallest molecules of the 16-molecule workload (20 and 24
    atoms, same recipe and orbital-shell fraction): every graph mode equals
    the per-class launches, and the 20-atom molecule's J blocks and gamma
    entries match the binary128 oracle on sampled entries."""
    mols = W.batch16_molecules()[:2]
    assert mols[0].natom >= 20
    rng = np.random.default_rng(6)
    Ds, cs = [], []
    for cl in mols:
        Ds.append(W.density(rng, int(oracle.ao_offsets(cl.orb)[-1])))
        cs.append(rng.standard_normal(int(oracle.ao_offsets(cl.aux)[-1])))
    b = lx.Batch([(cl.orb, cl.aux) for cl in mols], 1e-12).bind([torch.tensor(D, device="cuda") for D in Ds],
                                                                  [torch.tensor(c, device="cuda") for c in cs])
    res = {}
    for mode in (2, 1, 0):
        g, J = b.execute(mode)
        torch.cuda.synchronize()
        res[mode] = ([x.cpu().numpy().copy() for x in g], [x.cpu().numpy().copy() for x in J])
    for m in range(2):
        assert np.array_equal(res[2][0][m], res[0][0][m]) and np.array_equal(res[2][1][m], res[0][1][m])
        for k in (0, 1):  # the persistent kernels: equal to rounding (see above)
            ref = res[0][k][m]
            assert np.abs(res[1][k][m] - ref).max() <= 1e-12 * np.abs(ref).max()
    cl = mols[0]
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12)  # the same screen, for its task list
    g, J = res[2][0][0], res[2][1][0]
    sampled_against_oracle(cl, plan, Ds[0], cs[0], g, J, 16, 3, 7, "quad", 1e-12)
