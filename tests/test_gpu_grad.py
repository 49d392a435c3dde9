"""GPU gradient of the DF-J energy E = c^T gamma (D, c fixed; not in the paper,
required for differentiation): dE/dR from lx3c_dfj_grad / DFJEnergy.

Checks, following the target's statement:
  - the oracle's analytic gradient (which differentiates all three centres
    independently) on the same screened task list, 1e-11 relative to max|F|,
    in binary128: on a 2-atom cluster in full, and on the full 64-atom
    cluster with D restricted to the shell pairs of two sampled atoms and c
    to sampled ket shells of two others (so only the triples between them
    carry weight; the GPU still runs the whole 64-atom plan);
  - sum of forces = 0 to 1e-10 max|F|;
  - central finite differences of the GPU energy (h = 1e-4 bohr) on the
    64-atom cluster (4x4x4 grid), 12 random coordinates, 1e-7 relative to max|F|;
  - torch.autograd through DFJEnergy returns the same gradient.
"""
import numpy as np
import pytest

import oracle
from paper_2210_03192_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03192_gb300 as m
    return m


def dc(cl, seed):
    rng = np.random.default_rng(seed)
    n = int(oracle.ao_offsets(cl.orb)[-1])
    naux = int(oracle.ao_offsets(cl.aux)[-1])
    return W.density(rng, n), rng.standard_normal(naux)


def test_gradient_vs_oracle_binary128(lx):
    cl = W.cluster((2, 1, 1), W.ORB_RECIPE_SMALL, W.AUX_RECIPE_GRAD, seed=W.SEED_BASE + 40)
    D, c = dc(cl, 5)
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12, gradient=True)
    Dt, ct = torch.tensor(D, device="cuda"), torch.tensor(c, device="cuda")
    G = plan.gradient(Dt, ct).cpu().numpy()
    Go = oracle.dfj_grad(cl.orb, cl.aux, D, c, cl.natom, tasks=plan.tasks(), mode="quad")
    scale = np.abs(Go).max()
    assert np.abs(G - Go).max() <= 1e-11 * scale, (np.abs(G - Go).max() / scale)
    assert np.abs(G.sum(axis=0)).max() <= 1e-10 * np.abs(G).max()
    # the energy of the same plan
    E, g = plan.energy(Dt, ct)
    go, _ = oracle.dfj(cl.orb, cl.aux, D, c, tasks=plan.tasks(), mode="quad")
    assert float(E) == pytest.approx(float(np.dot(c, go)), rel=1e-12)


def test_gradient_64_atoms_sampled_vs_oracle_binary128(lx):
    cl = W.cluster64_grad()
    D, c = dc(cl, 7)
    rng = np.random.default_rng(12)
    atoms = rng.choice(cl.natom, 4, replace=False)
    SA, SC = set(int(x) for x in atoms[:2]), set(int(x) for x in atoms[2:])
    ao, aq = oracle.ao_offsets(cl.orb), oracle.ao_offsets(cl.aux)
    mo = np.zeros(int(ao[-1]), bool)
    for s in range(cl.orb.nshell):
        if int(cl.orb.atom[s]) in SA:
            mo[ao[s]:ao[s + 1]] = True
    kets = [s for s in range(cl.aux.nshell) if int(cl.aux.atom[s]) in SC]
    kets = set(int(x) for x in rng.choice(kets, 20, replace=False))
    mc = np.zeros(int(aq[-1]), bool)
    for s in kets:
        mc[aq[s]:aq[s + 1]] = True
    Dm = np.where(mo[:, None] & mo[None, :], D, 0.0)
    cm = np.where(mc, c, 0.0)
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12, gradient=True)
    G = plan.gradient(torch.tensor(Dm, device="cuda"), torch.tensor(cm, device="cuda")).cpu().numpy()
    t = plan.tasks()
    sel = np.array([int(cl.orb.atom[a]) in SA and int(cl.orb.atom[b]) in SA and int(P) in kets for a, b, P in t])
    Go = oracle.dfj_grad(cl.orb, cl.aux, Dm, cm, cl.natom, tasks=t[sel], mode="quad")
    scale = np.abs(Go).max()
    assert sel.sum() > 1000 and scale > 0
    assert np.abs(G - Go).max() <= 1e-11 * scale, (np.abs(G - Go).max() / scale)


def test_gradient_three_atoms_fp64_oracle(lx):
    cl = W.cluster((3, 1, 1), W.ORB_RECIPE_SMALL, W.AUX_RECIPE_GRAD, seed=W.SEED_BASE + 41)
    D, c = dc(cl, 6)
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12, gradient=True)
    G = plan.gradient(torch.tensor(D, device="cuda"), torch.tensor(c, device="cuda")).cpu().numpy()
    Go = oracle.dfj_grad(cl.orb, cl.aux, D, c, cl.natom, tasks=plan.tasks())
    assert np.abs(G - Go).max() <= 1e-9 * np.abs(Go).max()
    assert np.abs(Go.sum(axis=0)).max() <= 1e-9 * np.abs(Go).max()


def test_gradient_finite_differences_64_atoms(lx):
    cl = W.cluster64_grad()
    D, c = dc(cl, 7)
    Dt, ct = torch.tensor(D, device="cuda"), torch.tensor(c, device="cuda")
    R0 = cl.coords.copy()

    def energy(R):
        plan = lx.DFJPlan(lx._moved(cl.orb, R), lx._moved(cl.aux, R), 1e-12)
        E, _ = plan.energy(Dt, ct)
        return float(E)

    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12, gradient=True)
    G = plan.gradient(Dt, ct).cpu().numpy()
    assert np.abs(G.sum(axis=0)).max() <= 1e-10 * np.abs(G).max()
    rng = np.random.default_rng(11)
    h = 1e-4
    for _ in range(12):
        atom, ax = int(rng.integers(cl.natom)), int(rng.integers(3))
        Rp, Rm = R0.copy(), R0.copy()
        Rp[atom, ax] += h
        Rm[atom, ax] -= h
        fd = (energy(Rp) - energy(Rm)) / (2 * h)
        assert abs(fd - G[atom, ax]) <= 1e-7 * np.abs(G).max(), (atom, ax, fd, G[atom, ax])


def test_autograd_function(lx):
    cl = W.cluster((2, 2, 1), W.ORB_RECIPE_SMALL, W.AUX_RECIPE_GRAD, seed=W.SEED_BASE + 42)
    D, c = dc(cl, 8)
    Dt, ct = torch.tensor(D, device="cuda"), torch.tensor(c, device="cuda")
    R = torch.tensor(cl.coords, dtype=torch.float64, requires_grad=True)
    E = lx.DFJEnergy.apply(R, cl.orb, cl.aux, Dt, ct)
    E.backward()
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12, gradient=True)
    G = plan.gradient(Dt, ct).cpu().numpy()
    E2, _ = plan.energy(Dt, ct)
    assert float(E) == pytest.approx(float(E2), rel=1e-13)
    np.testing.assert_allclose(R.grad.numpy(), G, rtol=0, atol=1e-12 * np.abs(G).max())
