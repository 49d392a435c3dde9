"""Tile-callback DF-J build (lx3c_dfj_execute_tiles, the paper's end-user
DF-J interface of Sec. 3: D tiles in, J tiles out through callables).  The
caller here keeps D as a dictionary of tiles, not as one array, and collects
J tile by tile; gamma and the assembled J must equal the device build of the
same plan, for tiles of one shell, of ~37 AOs and of the whole matrix."""
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


def normwise(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("tile", [1, 37, 100000])
def test_tiles_match_device_build(lx, tile):
    cl = W.cluster((2, 2, 1), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=91)
    rng = np.random.default_rng(tile)
    n = int(oracle.ao_offsets(cl.orb)[-1])
    D = W.density(rng, n)
    c = rng.standard_normal(int(oracle.ao_offsets(cl.aux)[-1]))
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12)
    g0, J0 = plan.execute(torch.tensor(D, device="cuda"), torch.tensor(c, device="cuda"))
    g0, J0 = g0.cpu().numpy(), J0.cpu().numpy()
    asked, got = [], {}

    def get_D(r0, nr, c0, nc):
        asked.append((r0, nr, c0, nc))
        return D[r0:r0 + nr, c0:c0 + nc].copy()

    def put_J(r0, c0, t):
        got[(r0, c0)] = t

    g = plan.execute_tiles(get_D, put_J, c, tile_ao=tile)
    assert all(r0 <= c0 for r0, _, c0, _ in asked)  # upper triangle of tiles only
    J = np.zeros((n, n))
    for (r0, c0), t in got.items():
        J[r0:r0 + t.shape[0], c0:c0 + t.shape[1]] = t
    covered = np.zeros((n, n), bool)
    for (r0, c0), t in got.items():
        covered[r0:r0 + t.shape[0], c0:c0 + t.shape[1]] = True
    assert covered.all()
    assert normwise(g, g0) < 1e-14
    assert normwise(J, J0) < 1e-14


def test_tile_callable_error_stops_the_build(lx):
    cl = W.cluster((2, 1, 1), W.ORB_RECIPE_DFJ, W.AUX_RECIPE_DFJ, seed=92)
    plan = lx.DFJPlan(cl.orb, cl.aux, 1e-12)
    c = np.zeros(int(oracle.ao_offsets(cl.aux)[-1]))

    def bad(r0, nr, c0, nc):
        raise KeyError("tile not stored here")

    with pytest.raises(KeyError):
        plan.execute_tiles(bad, None, c, tile_ao=16)
