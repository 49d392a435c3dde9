"""ORACLE — test infrastructure only.

A plain, slow, independent CPU reference for the 3-center Coulomb integrals
(ab|C) and the density-fitting Coulomb quantities built from them.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import or run anything here.
The GPU library never links, imports or calls this package and this package
never imports the GPU library; the two share no code.

Pieces (each cites the passage of the paper it follows):
  md3c.c / md3c_body.h  McMurchie-Davidson contracted Cartesian (ab|c)
                        (definitions: Appendix A; scheme named in Sec. 2.3)
  solid.py              real solid harmonics (Sec. 2.5.1: ket projected to
                        solid harmonics; convention is a documented reading)
  quadrature.py         brute-force quadrature of the defining integral, used
                        only to pin md3c on tiny inputs
  this file             contraction/transform drivers, DF-J gamma and J
                        (Sec. 3: integral digestion into a DF-J build), the
                        density-fitting metric V_PQ = (P|Q) and the fitted
                        density c = V^{-1} gamma (Sec. 1), and the nuclear
                        gradient of E = c^T gamma.

All functions take plain numpy arrays.  A basis is any object with attributes
  l[nsh] int, k[nsh] int (primitives per shell), off[nsh] int (first primitive),
  xyz[nsh,3] float (bohr), exps[nprim], coefs[nprim] float,
  atom[nsh] int (only for gradients)
The primitives are non-normalised (Appendix A); coefficients are used as given.
"""
import ctypes
import os
import platform
import subprocess
import sys

import numpy as np

from .solid import cart_list, ncart, nsph, solid_matrix

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

MODES = {"double": 0, "extended": 1, "quad": 2}
SPH_LMAX = 10


def build(force=False):
    """Compile md3c.c with gcc + OpenMP into oracle/_build/liboracle.so."""
    src = [os.path.join(_HERE, "md3c.c")]
    hdr = [os.path.join(_HERE, "md3c_body.h")]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(f) <= so_t for f in src + hdr):
            return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    libs = ["-lm"]
    if platform.machine() in ("x86_64", "AMD64"):
        libs = ["-lquadmath", "-lm"]
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + src + libs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        L.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, f64p]
        L.oracle_boys.restype = None
        L.oracle_eri3c.argtypes = [i32p, i32p, i64p, f64p, f64p, f64p, ctypes.c_int64, i32p, i64p, f64p,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, f64p, f64p, i64p]
        L.oracle_eri3c.restype = ctypes.c_int
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def num_threads():
    return int(lib().oracle_num_threads())


def _mode(mode, extended=False):
    if extended:
        return 1
    return MODES[mode] if isinstance(mode, str) else int(mode)


def boys(mmax, T, extended=False, mode="double"):
    """[F_0(T), ..., F_mmax(T)] (Appendix A definition of the Boys function)."""
    out = np.zeros(mmax + 1)
    lib().oracle_boys(int(mmax), float(T), _mode(mode, extended), out)
    return out


_SPH = None


def _sph_tables():
    global _SPH
    if _SPH is None:
        from .solid import solid_matrix_hilo
        his, los, off = [], [], [0]
        for l in range(SPH_LMAX + 1):
            h, lo_ = solid_matrix_hilo(l)
            his.append(h.ravel())
            los.append(lo_.ravel())
            off.append(off[-1] + h.size)
        _SPH = (np.ascontiguousarray(np.concatenate(his)), np.ascontiguousarray(np.concatenate(los)),
                np.ascontiguousarray(np.array(off, np.int64)))
    return _SPH


# --------------------------------------------------------------------------
# shell tables
# --------------------------------------------------------------------------

def _combined(*bases):
    """Concatenate shell tables; returns arrays and per-basis shell offsets."""
    l, k, off, xyz, ex, co, base = [], [], [], [], [], [], []
    nsh = 0
    npr = 0
    for b in bases:
        base.append(nsh)
        l.append(np.asarray(b.l, np.int32))
        k.append(np.asarray(b.k, np.int32))
        off.append(np.asarray(b.off, np.int64) + npr)
        xyz.append(np.asarray(b.xyz, np.float64).reshape(-1, 3))
        ex.append(np.asarray(b.exps, np.float64))
        co.append(np.asarray(b.coefs, np.float64))
        nsh += len(b.l)
        npr += len(b.exps)
    cat = lambda xs, dt: np.ascontiguousarray(np.concatenate(xs).astype(dt))
    return (cat(l, np.int32), cat(k, np.int32), cat(off, np.int64),
            np.ascontiguousarray(np.concatenate(xyz).reshape(-1)), cat(ex, np.float64),
            cat(co, np.float64), base)


def _dims(l, pure):
    return nsph(l) if pure else ncart(l)


def blocks(tables, trip, mode="double", bra_pure=False, ket_pure=True, dA=-1, dB=-1, dC=-1):
    """Contracted blocks for shell triples trip[n,3] of a combined table.

    Returns (flat array, offsets, shapes)."""
    l, k, off, xyz, ex, co = tables
    trip = np.ascontiguousarray(np.asarray(trip, np.int32).reshape(-1, 3))
    shapes = [(_dims(int(l[a]), bra_pure), _dims(int(l[b]), bra_pure), _dims(int(l[c]), ket_pure))
              for a, b, c in trip]
    sizes = np.array([x * y * z for x, y, z in shapes], np.int64)
    offs = np.zeros(len(trip), np.int64)
    if len(trip):
        offs[1:] = np.cumsum(sizes)[:-1]
    out = np.zeros(int(sizes.sum()) if len(trip) else 0)
    if len(trip):
        hi, lo, soff = _sph_tables()
        rc = lib().oracle_eri3c(l, k, off, xyz, ex, co, len(trip), trip, offs, out, _mode(mode),
                                int(bool(bra_pure)), int(bool(ket_pure)), int(dA), int(dB), int(dC),
                                SPH_LMAX + 1, hi, lo, soff)
        if rc != 0:
            raise ValueError("oracle_eri3c failed with %d" % rc)
    return out, offs, shapes


def cart_blocks(tables, trip, extended=False):
    """Cartesian bra and Cartesian (true) ket blocks (flat, offsets)."""
    flat, offs, _ = blocks(tables, trip, mode=_mode("double", extended), bra_pure=False, ket_pure=False)
    return flat, offs


def eri3c(orb, aux, pairs, auxs, bra_pure=True, extended=False, mode="double", ket_route="hermite"):
    """(ab|C) blocks for every (pair, aux shell): array [npair, naux, nA, nB, nC].

    The ket is always solid harmonic (Sec. 2.2, first design assumption): with
    ket_route="hermite" it is expanded exactly (Hobson's theorem), with
    ket_route="cartesian" true Cartesian kets are computed and projected (kept
    for cross-checks).  The bra is Cartesian (the paper's target) unless
    bra_pure.  The class must be homogeneous (one (la, lb, lc)).
    """
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    auxs = np.asarray(auxs, np.int64).reshape(-1)
    l, k, off, xyz, ex, co, base = _combined(orb, aux)
    if len(pairs) == 0 or len(auxs) == 0:
        return np.zeros((len(pairs), len(auxs), 0, 0, 0))
    la = {int(orb.l[p]) for p in pairs[:, 0]}
    lb = {int(orb.l[p]) for p in pairs[:, 1]}
    lc = {int(aux.l[q]) for q in auxs}
    if len(la) != 1 or len(lb) != 1 or len(lc) != 1:
        raise ValueError("eri3c needs one (la, lb, lc) class")
    la, lb, lc = la.pop(), lb.pop(), lc.pop()
    trip = np.empty((len(pairs), len(auxs), 3), np.int32)
    trip[:, :, 0] = pairs[:, 0, None]
    trip[:, :, 1] = pairs[:, 1, None]
    trip[:, :, 2] = auxs[None, :] + base[1]
    md = _mode(mode, extended)
    if ket_route == "cartesian":
        flat, _, _ = blocks((l, k, off, xyz, ex, co), trip.reshape(-1, 3), md, bra_pure=False, ket_pure=False)
        X = flat.reshape(len(pairs), len(auxs), ncart(la), ncart(lb), ncart(lc))
        X = np.einsum("Cc,PQabc->PQabC", solid_matrix(lc), X)
        if bra_pure:
            X = np.einsum("Aa,Bb,PQabC->PQABC", solid_matrix(la), solid_matrix(lb), X)
        return X
    flat, _, _ = blocks((l, k, off, xyz, ex, co), trip.reshape(-1, 3), md, bra_pure=bra_pure, ket_pure=True)
    return flat.reshape(len(pairs), len(auxs), _dims(la, bra_pure), _dims(lb, bra_pure), nsph(lc))


def eri3c_triples(orb, aux, trip_pairs, trip_aux, bra_pure=True, extended=False, mode="double"):
    """(ab|C) for explicit triples (pair_i, aux_i), any mix of classes; list of arrays."""
    l, k, off, xyz, ex, co, base = _combined(orb, aux)
    trip_pairs = np.asarray(trip_pairs, np.int64).reshape(-1, 2)
    trip_aux = np.asarray(trip_aux, np.int64).reshape(-1)
    trip = np.empty((len(trip_aux), 3), np.int32)
    trip[:, 0] = trip_pairs[:, 0]
    trip[:, 1] = trip_pairs[:, 1]
    trip[:, 2] = trip_aux + base[1]
    flat, offs, shapes = blocks((l, k, off, xyz, ex, co), trip, _mode(mode, extended), bra_pure=bra_pure,
                                ket_pure=True)
    return [flat[o:o + a * b * c].reshape(a, b, c) for o, (a, b, c) in zip(offs, shapes)]


# --------------------------------------------------------------------------
# DF-J (Sec. 3: gamma_P = sum_ab (ab|P) D_ab, J_ab = sum_P (ab|P) c_P)
# --------------------------------------------------------------------------

def ao_offsets(basis, pure=True):
    n = [nsph(int(l)) if pure else ncart(int(l)) for l in basis.l]
    off = np.zeros(len(n) + 1, np.int64)
    off[1:] = np.cumsum(n)
    return off


def dfj(orb, aux, D, c, tasks=None, extended=False, mode="double"):
    """gamma_P and J_mn over ALL AO pairs (mu, nu) of a pure orbital basis.

    tasks: optional list of (shell_a, shell_b, aux_shell) with shell_a <= shell_b
    (unique pairs) to include; default every unique pair with every aux shell.
    Off-diagonal shell pairs count twice in gamma and fill both J blocks.
    """
    ao = ao_offsets(orb)
    aq = ao_offsets(aux)
    nsh = len(orb.l)
    if tasks is None:
        tasks = [(i, j, P) for i in range(nsh) for j in range(i, nsh) for P in range(len(aux.l))]
    tasks = np.asarray(tasks, np.int64).reshape(-1, 3)
    blocks = eri3c_triples(orb, aux, tasks[:, :2], tasks[:, 2], bra_pure=True, extended=extended, mode=mode)
    gamma = np.zeros(int(aq[-1]))
    J = np.zeros((int(ao[-1]), int(ao[-1])))
    for (i, j, P), X in zip(tasks, blocks):
        si, sj, sp = slice(ao[i], ao[i + 1]), slice(ao[j], ao[j + 1]), slice(aq[P], aq[P + 1])
        w = 1.0 if i == j else 2.0
        gamma[sp] += w * np.einsum("abP,ab->P", X, D[si, sj])
        Jb = np.einsum("abP,P->ab", X, c[sp])
        J[si, sj] += Jb
        if i != j:
            J[sj, si] += Jb.T
    return gamma, J


# --------------------------------------------------------------------------
# Density-fitting metric V_PQ = (P|Q) and the fitted density (Sec. 1, 4)
# --------------------------------------------------------------------------

def unit_shell_basis(aux):
    """aux's shells followed by the constant function 1 = exp(-0 r^2) (an s
    shell with exponent 0 and coefficient 1), so that the 3-centre integral
    (P 1|Q) is the 2-centre Coulomb integral (P|Q)."""
    from types import SimpleNamespace
    k = np.r_[np.asarray(aux.k, np.int32), 1]
    off = np.zeros(len(k), np.int64)
    off[1:] = np.cumsum(k)[:-1]
    return SimpleNamespace(l=np.r_[np.asarray(aux.l, np.int32), 0], k=k, off=off,
                           xyz=np.vstack([np.asarray(aux.xyz, float).reshape(-1, 3), np.zeros((1, 3))]),
                           exps=np.r_[np.asarray(aux.exps, float), 0.0], coefs=np.r_[np.asarray(aux.coefs, float), 1.0])


def metric(aux, mode="double"):
    """V[naux_ao, naux_ao], V_PQ = (P|Q) = int int P(r1) |r1 - r2|^-1 Q(r2),
    all shells solid harmonic, AO order = shell order."""
    bra = unit_shell_basis(aux)
    unit = len(aux.l)
    ns = len(aux.l)
    P, Q = np.meshgrid(np.arange(ns), np.arange(ns), indexing="ij")
    pairs = np.stack([P.ravel(), np.full(P.size, unit)], axis=1)
    blocks = eri3c_triples(bra, aux, pairs, Q.ravel(), bra_pure=True, mode=mode)
    aq = ao_offsets(aux)
    V = np.zeros((int(aq[-1]), int(aq[-1])))
    for (p, q), X in zip(zip(P.ravel(), Q.ravel()), blocks):
        V[aq[p]:aq[p + 1], aq[q]:aq[q + 1]] = X[:, 0, :]
    return V


def fitted_density(V, gamma):
    """c = V^{-1} gamma (a library linear solve on the oracle's metric)."""
    return np.linalg.solve(V, gamma)


# --------------------------------------------------------------------------
# Gradient of E = c^T gamma = sum_{mu nu P} D_{mu nu} c_P (mu nu|P)
# with D and c held fixed.  Each centre is differentiated independently in
# md3c (d/dA_i phi_a = 2 zeta_a phi_{a+1_i} - a_i phi_{a-1_i} from the
# definition in Appendix A; the solid-harmonic ket through its Hermite
# expansion), so that the sum of forces vanishing is a genuine check.
# --------------------------------------------------------------------------

def dfj_grad(orb, aux, D, c, natom, tasks=None, mode="double"):
    """dE/dR[natom, 3] for E = c^T gamma (pure orbital and aux bases)."""
    ao = ao_offsets(orb)
    aq = ao_offsets(aux)
    nsh = len(orb.l)
    if tasks is None:
        tasks = [(i, j, P) for i in range(nsh) for j in range(i, nsh) for P in range(len(aux.l))]
    tasks = np.asarray(tasks, np.int64).reshape(-1, 3)
    l, k, off, xyz, ex, co, base = _combined(orb, aux)
    trip = np.empty((len(tasks), 3), np.int32)
    trip[:, 0] = tasks[:, 0]
    trip[:, 1] = tasks[:, 1]
    trip[:, 2] = tasks[:, 2] + base[1]
    G = np.zeros((natom, 3))
    W = []
    for (i, j, P) in tasks:
        w = 1.0 if i == j else 2.0
        W.append(w * np.einsum("AB,C->ABC", D[ao[i]:ao[i + 1], ao[j]:ao[j + 1]], c[aq[P]:aq[P + 1]]))
    for centre in range(3):
        for axis in range(3):
            d = [-1, -1, -1]
            d[centre] = axis
            flat, offs, shapes = blocks((l, k, off, xyz, ex, co), trip, mode, bra_pure=True, ket_pure=True,
                                        dA=d[0], dB=d[1], dC=d[2])
            for n, (i, j, P) in enumerate(tasks):
                a_, b_, c_ = shapes[n]
                blk = flat[offs[n]:offs[n] + a_ * b_ * c_].reshape(a_, b_, c_)
                atom = (orb.atom[i], orb.atom[j], aux.atom[P])[centre]
                G[int(atom), axis] += float(np.sum(blk * W[n]))
    return G
