"""Seeded synthetic inputs shared by the GPU path's tests, the benchmark and the oracle tests.

This module only draws random numbers and lays out shell tables; it holds none
of the integral arithmetic.  Every generator is deterministic in its seed
(numpy PCG64 via ``default_rng``).

The paper measures on real molecules with def2 basis sets (Sec. 4, Table 6),
which are not available here; the recipes below stand in for them.

Shell table layout (one ``Basis`` per basis set; all arrays C-contiguous):
  l[nsh]    int32   angular momentum of each shell
  k[nsh]    int32   number of primitives
  off[nsh]  int64   index of the shell's first primitive in exps/coefs
  xyz[nsh,3] float64 centre (bohr)
  atom[nsh] int32   owning atom (gradients); -1 if none
  exps, coefs [nprim] float64  primitive exponents and contraction
            coefficients, used as given (non-normalised primitives).
"""
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20221003


@dataclass
class Basis:
    l: np.ndarray
    k: np.ndarray
    off: np.ndarray
    xyz: np.ndarray
    exps: np.ndarray
    coefs: np.ndarray
    atom: np.ndarray = field(default=None)

    def __post_init__(self):
        self.l = np.ascontiguousarray(self.l, np.int32)
        self.k = np.ascontiguousarray(self.k, np.int32)
        self.off = np.ascontiguousarray(self.off, np.int64)
        self.xyz = np.ascontiguousarray(np.asarray(self.xyz, np.float64).reshape(-1, 3))
        self.exps = np.ascontiguousarray(self.exps, np.float64)
        self.coefs = np.ascontiguousarray(self.coefs, np.float64)
        if self.atom is None:
            self.atom = -np.ones(len(self.l), np.int32)
        self.atom = np.ascontiguousarray(self.atom, np.int32)

    @property
    def nshell(self):
        return len(self.l)

    def subset(self, idx):
        """Shells idx (in that order) as a new Basis."""
        idx = np.asarray(idx, np.int64)
        k = self.k[idx]
        off = np.zeros(len(idx), np.int64)
        off[1:] = np.cumsum(k)[:-1]
        sel = np.concatenate([np.arange(self.off[i], self.off[i] + self.k[i]) for i in idx]) \
            if len(idx) else np.zeros(0, np.int64)
        return Basis(self.l[idx], k, off, self.xyz[idx], self.exps[sel], self.coefs[sel], self.atom[idx])


def make_basis(ls, ks, xyz, exps, coefs, atom=None):
    ks = np.asarray(ks, np.int32)
    off = np.zeros(len(ks), np.int64)
    off[1:] = np.cumsum(ks)[:-1]
    return Basis(ls, ks, off, xyz, exps, coefs, atom)


def random_shells(rng, n, l, K, box, exp_lo, exp_hi, coef_lo=0.1, coef_hi=1.0, centres=None):
    """n shells of angular momentum l with K primitives each.

    Centres uniform in [0, box]^3 (unless given), exponents log-uniform in
    [exp_lo, exp_hi], coefficients uniform in [coef_lo, coef_hi]."""
    if centres is None:
        centres = rng.uniform(0.0, box, size=(n, 3))
    exps = np.exp(rng.uniform(np.log(exp_lo), np.log(exp_hi), size=n * K))
    coefs = rng.uniform(coef_lo, coef_hi, size=n * K)
    return make_basis(np.full(n, l), np.full(n, K), centres, exps, coefs)


def concat(*bases):
    ls, ks, xyz, ex, co, at = [], [], [], [], [], []
    for b in bases:
        ls.append(b.l); ks.append(b.k); xyz.append(b.xyz); ex.append(b.exps); co.append(b.coefs); at.append(b.atom)
    return make_basis(np.concatenate(ls), np.concatenate(ks), np.concatenate(xyz),
                      np.concatenate(ex), np.concatenate(co), np.concatenate(at))


@dataclass
class ClassProblem:
    """One (la, lb, lc) class: independent A,B shells per pair and a list of aux shells."""
    la: int
    lb: int
    lc: int
    orb: Basis           # 2*npair shells: shell 2i is a, shell 2i+1 is b of pair i
    aux: Basis           # naux shells of angular momentum lc
    pairs: np.ndarray    # [npair, 2] int32 shell indices into orb
    auxs: np.ndarray     # [naux] int32 shell indices into aux

    @property
    def npair(self):
        return len(self.pairs)

    @property
    def naux(self):
        return len(self.auxs)


def class_problem(la, lb, lc, npair, naux, Ka=1, Kb=1, Kc=1, box=10.0, exp_lo=0.1, exp_hi=100.0,
                  seed=SEED_BASE):
    """Pairs with independent centres A, B and aux shells, all drawn uniformly."""
    rng = np.random.default_rng(seed)
    a = random_shells(rng, npair, la, Ka, box, exp_lo, exp_hi)
    b = random_shells(rng, npair, lb, Kb, box, exp_lo, exp_hi)
    c = random_shells(rng, naux, lc, Kc, box, exp_lo, exp_hi)
    # interleave a and b shells: 2i -> a_i, 2i+1 -> b_i
    order = np.empty(2 * npair, np.int64)
    ab = concat(a, b)
    order[0::2] = np.arange(npair)
    order[1::2] = npair + np.arange(npair)
    orb = ab.subset(order)
    pairs = np.stack([np.arange(0, 2 * npair, 2), np.arange(1, 2 * npair, 2)], axis=1).astype(np.int32)
    return ClassProblem(la, lb, lc, orb, c, pairs, np.arange(naux, dtype=np.int32))


def ppd_64x32():
    """(pp|d), K=1: 64 pairs x 32 aux shells; centres in a 10-bohr cube,
    exponents log-uniform in [0.1, 100], coefficients uniform in [0.1, 1]."""
    return class_problem(1, 1, 2, 64, 32, 1, 1, 1, box=10.0, exp_lo=0.1, exp_hi=100.0, seed=SEED_BASE + 0)


def sweep_class(la, lb, lc, Kab, npair=4096, naux=512, product_reading=False):
    """Per-class sweep member: 4096 pairs x 512 aux shells, centres in a 20-bohr
    cube, exponents log-uniform in [0.05, 1e4], K_c = 1.

    K_ab reading: by default K_a = K_b = K_ab (so K = K_ab^2 primitive triples);
    with product_reading, (K_a, K_b) = (K_ab, 1)."""
    Ka, Kb = (Kab, 1) if product_reading else (Kab, Kab)
    seed = SEED_BASE + 1 + 1000 * (la * 100 + lb * 10 + lc) + Kab
    return class_problem(la, lb, lc, npair, naux, Ka, Kb, 1, box=20.0, exp_lo=0.05, exp_hi=1.0e4, seed=seed)


SWEEP_CLASSES = [(la, lb, lc, K) for la in range(5) for lb in range(5) for lc in range(7) for K in (1, 3, 6)]


# --------------------------------------------------------------------------
# Molecule-like clusters (DF-J, gradients, batched workloads)
# --------------------------------------------------------------------------

@dataclass
class Cluster:
    natom: int
    coords: np.ndarray   # [natom, 3]
    orb: Basis           # orbital shells, atom-major
    aux: Basis           # aux shells, atom-major


def grid_atoms(rng, shape, spacing=1.8, jitter=0.3):
    nx, ny, nz = shape
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), -1).reshape(-1, 3)
    return g * spacing + rng.uniform(-jitter, jitter, size=g.shape)


def _atom_shells(rng, coords, recipe, exp_lo, exp_hi):
    """recipe: list of (l, count, K) per atom.  Shell exponents log-uniform,
    coefficients uniform in [0.1, 1]."""
    ls, ks, xyz, ex, co, at = [], [], [], [], [], []
    for ia, R in enumerate(coords):
        for (l, count, K) in recipe:
            for _ in range(count):
                ls.append(l); ks.append(K); xyz.append(R); at.append(ia)
                ex.append(np.exp(rng.uniform(np.log(exp_lo), np.log(exp_hi), size=K)))
                co.append(rng.uniform(0.1, 1.0, size=K))
    return make_basis(ls, ks, np.array(xyz), np.concatenate(ex), np.concatenate(co), at)


ORB_RECIPE_DFJ = [(0, 4, 6), (1, 3, 3), (2, 2, 1), (3, 1, 1)]                       # 4s3p2d1f, K=6/3/1/1
AUX_RECIPE_DFJ = [(0, 10, 1), (1, 7, 1), (2, 5, 1), (3, 3, 1), (4, 2, 1), (5, 1, 1)]  # 10s7p5d3f2g1h
ORB_RECIPE_SMALL = [(0, 3, 6), (1, 2, 3), (2, 2, 1), (3, 1, 1), (4, 1, 1)]          # 3s2p2d1f1g
AUX_RECIPE_GRAD = [(0, 8, 1), (1, 6, 1), (2, 5, 1), (3, 4, 1), (4, 3, 1), (5, 2, 1)]  # 8s6p5d4f3g2h
AUX_RECIPE_BATCH = AUX_RECIPE_GRAD + [(6, 1, 1)]                                     # + 1i


def cluster(shape, orb_recipe, aux_recipe, seed, spacing=1.8, jitter=0.3, exp_lo=0.05, exp_hi=1.0e4):
    rng = np.random.default_rng(seed)
    coords = grid_atoms(rng, shape, spacing, jitter)
    orb = _atom_shells(rng, coords, orb_recipe, exp_lo, exp_hi)
    aux = _atom_shells(rng, coords, aux_recipe, exp_lo, exp_hi)
    return Cluster(len(coords), coords, orb, aux)


def cluster256_dfj(shape=(8, 8, 4)):
    """256-atom jittered grid (1.8 bohr), orbital 4s3p2d1f (K=6/3/1/1),
    aux 10s7p5d3f2g1h (K=1)."""
    return cluster(shape, ORB_RECIPE_DFJ, AUX_RECIPE_DFJ, SEED_BASE + 2)


def density(rng, n, rank=None):
    """D = C C^T with C an n x (n/5) standard normal matrix."""
    r = max(1, n // 5) if rank is None else rank
    C = rng.standard_normal((n, r))
    return C @ C.T


def cluster64_grad(shape=(4, 4, 4)):
    """64-atom cluster, orbital 3s2p2d1f1g (L<=4), aux 8s6p5d4f3g2h (L<=5)."""
    return cluster(shape, ORB_RECIPE_SMALL, AUX_RECIPE_GRAD, SEED_BASE + 4)


def batch16_sizes():
    """16 molecule sizes n_i = round(20 * 20^(i/15)): 20 ... 400 atoms."""
    return [int(round(20 * 20 ** (i / 15))) for i in range(16)]


def molecule(natom, seed, orb_recipe=None, aux_recipe=None, orb_fraction=1.0, aux_fraction=1.0, spacing=1.8,
             jitter=0.3):
    """A compact jittered-grid molecule of natom atoms (the natom grid points
    nearest the centre of the smallest cube that holds them), orbital / aux
    shells from the recipes.  orb_fraction / aux_fraction < 1 keep that
    fraction of the orbital / aux shells (uniform, seeded)."""
    orb_recipe = ORB_RECIPE_SMALL if orb_recipe is None else orb_recipe
    aux_recipe = AUX_RECIPE_BATCH if aux_recipe is None else aux_recipe
    rng = np.random.default_rng(seed)
    m = 1
    while m ** 3 < natom:
        m += 1
    g = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"), -1).reshape(-1, 3)
    g = g[np.argsort(np.sum((g - (m - 1) / 2.0) ** 2, axis=1), kind="stable")][:natom]
    coords = g * spacing + rng.uniform(-jitter, jitter, size=g.shape)
    orb = _atom_shells(rng, coords, orb_recipe, 0.05, 1.0e4)
    aux = _atom_shells(rng, coords, aux_recipe, 0.05, 1.0e4)
    if orb_fraction < 1.0:
        keep = np.sort(rng.choice(orb.nshell, size=max(1, int(round(orb_fraction * orb.nshell))), replace=False))
        orb = orb.subset(keep)
    if aux_fraction < 1.0:
        keep = np.sort(rng.choice(aux.nshell, size=max(1, int(round(aux_fraction * aux.nshell))), replace=False))
        aux = aux.subset(keep)
    return Cluster(natom, coords, orb, aux)


def batch16_molecules(orb_fraction=0.25):
    """Batched uneven workload: 16 molecules of 20-400 atoms, orbital 3s2p2d1f1g
    (K=6/3/1/1/1), aux 8s6p5d4f3g2h1i (K=1), every class up to (gg|i) mixed.
    A fixed fraction of each molecule's orbital shells is kept (uniform,
    seeded; identical for the batched and the per-class runs), which scales
    the shell pairs by about its square and leaves every pair's ket list, and
    so the tile fill, as in the full molecule."""
    return [molecule(n, SEED_BASE + 3 + 100 * i, orb_fraction=orb_fraction) for i, n in enumerate(batch16_sizes())]
