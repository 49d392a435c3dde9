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
                        (Sec. 3: integral digestion into a DF-J build), and
                        the nuclear gradient of E = c^T gamma.

All functions take plain numpy arrays.  A basis is any object with attributes
  l[nsh] int, k[nsh] int (primitives per shell), off[nsh] int (first primitive),
  xyz[nsh,3] float (bohr), exps[nprim], coefs[nprim] float,
  atom[nsh] int (only for gradients)
The primitives are non-normalised (Appendix A); coefficients are used as given.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np

from .solid import cart_list, ncart, nsph, solid_matrix

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None


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
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + src + ["-lm"]
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
        L.oracle_eri3c_cart.argtypes = [i32p, i32p, i64p, f64p, f64p, f64p,
                                        ctypes.c_int64, i32p, i64p, f64p, ctypes.c_int]
        L.oracle_eri3c_cart.restype = ctypes.c_int
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def num_threads():
    return int(lib().oracle_num_threads())


def boys(mmax, T, extended=False):
    """[F_0(T), ..., F_mmax(T)] (Appendix A definition of the Boys function)."""
    out = np.zeros(mmax + 1)
    lib().oracle_boys(int(mmax), float(T), int(bool(extended)), out)
    return out


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


def cart_blocks(tables, trip, extended=False):
    """Cartesian contracted blocks for shell triples trip[n,3] of a combined table.

    Returns (flat array, offsets, shapes)."""
    l, k, off, xyz, ex, co = tables
    trip = np.ascontiguousarray(np.asarray(trip, np.int32).reshape(-1, 3))
    sizes = np.array([ncart(l[a]) * ncart(l[b]) * ncart(l[c]) for a, b, c in trip], np.int64)
    offs = np.zeros(len(trip), np.int64)
    if len(trip):
        offs[1:] = np.cumsum(sizes)[:-1]
    out = np.zeros(int(sizes.sum()) if len(trip) else 0)
    if len(trip):
        rc = lib().oracle_eri3c_cart(l, k, off, xyz, ex, co, len(trip), trip, offs, out,
                                     int(bool(extended)))
        if rc != 0:
            raise ValueError("oracle_eri3c_cart failed with %d" % rc)
    return out, offs


def eri3c(orb, aux, pairs, auxs, bra_pure=True, extended=False):
    """(ab|C) blocks for every (pair, aux shell): array [npair, naux, nA, nB, nC].

    The ket is always solid harmonic (Sec. 2.2, first design assumption); the
    bra is Cartesian (the paper's target) unless bra_pure, in which case both
    bra shells are projected with the same solid-harmonic matrices.  The class
    must be homogeneous (one (la, lb, lc)).
    """
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    auxs = np.asarray(auxs, np.int64).reshape(-1)
    l, k, off, xyz, ex, co, base = _combined(orb, aux)
    la = {int(orb.l[p]) for p in pairs[:, 0]}
    lb = {int(orb.l[p]) for p in pairs[:, 1]}
    lc = {int(aux.l[q]) for q in auxs}
    if len(pairs) == 0 or len(auxs) == 0:
        return np.zeros((len(pairs), len(auxs), 0, 0, 0))
    if len(la) != 1 or len(lb) != 1 or len(lc) != 1:
        raise ValueError("eri3c needs one (la, lb, lc) class")
    la, lb, lc = la.pop(), lb.pop(), lc.pop()
    trip = np.empty((len(pairs), len(auxs), 3), np.int32)
    trip[:, :, 0] = pairs[:, 0, None]
    trip[:, :, 1] = pairs[:, 1, None]
    trip[:, :, 2] = auxs[None, :] + base[1]
    flat, _ = cart_blocks((l, k, off, xyz, ex, co), trip.reshape(-1, 3), extended)
    X = flat.reshape(len(pairs), len(auxs), ncart(la), ncart(lb), ncart(lc))
    X = np.einsum("Cc,PQabc->PQabC", solid_matrix(lc), X)
    if bra_pure:
        X = np.einsum("Aa,Bb,PQabC->PQABC", solid_matrix(la), solid_matrix(lb), X)
    return X


def eri3c_triples(orb, aux, trip_pairs, trip_aux, bra_pure=True, extended=False):
    """(ab|C) for explicit triples (pair_i, aux_i), any mix of classes; list of arrays."""
    l, k, off, xyz, ex, co, base = _combined(orb, aux)
    trip_pairs = np.asarray(trip_pairs, np.int64).reshape(-1, 2)
    trip_aux = np.asarray(trip_aux, np.int64).reshape(-1)
    trip = np.empty((len(trip_aux), 3), np.int32)
    trip[:, 0] = trip_pairs[:, 0]
    trip[:, 1] = trip_pairs[:, 1]
    trip[:, 2] = trip_aux + base[1]
    flat, offs = cart_blocks((l, k, off, xyz, ex, co), trip, extended)
    out = []
    for i, (a, b, c) in enumerate(trip):
        la, lb, lc = int(l[a]), int(l[b]), int(l[c])
        n = ncart(la) * ncart(lb) * ncart(lc)
        X = flat[offs[i]:offs[i] + n].reshape(ncart(la), ncart(lb), ncart(lc))
        X = np.einsum("Cc,abc->abC", solid_matrix(lc), X)
        if bra_pure:
            X = np.einsum("Aa,Bb,abC->ABC", solid_matrix(la), solid_matrix(lb), X)
        out.append(X)
    return out


# --------------------------------------------------------------------------
# DF-J (Sec. 3: gamma_P = sum_ab (ab|P) D_ab, J_ab = sum_P (ab|P) c_P)
# --------------------------------------------------------------------------

def ao_offsets(basis, pure=True):
    n = [nsph(int(l)) if pure else ncart(int(l)) for l in basis.l]
    off = np.zeros(len(n) + 1, np.int64)
    off[1:] = np.cumsum(n)
    return off


def dfj(orb, aux, D, c, tasks=None, extended=False):
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
    blocks = eri3c_triples(orb, aux, tasks[:, :2], tasks[:, 2], bra_pure=True, extended=extended)
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
# Gradient of E = c^T gamma = sum_{mu nu P} D_{mu nu} c_P (mu nu|P)
# with D and c held fixed.  Derivatives of a Cartesian primitive:
#   d/dA_i phi_a = 2 zeta_a phi_{a+1_i} - a_i phi_{a-1_i}
# (differentiate the definition in Appendix A), applied to all three centres
# independently, so that sum of forces = 0 is a genuine check.
# --------------------------------------------------------------------------

class _Shifted:
    """Basis whose shells have l+shift and coefficients scaled by (2 zeta)^power."""

    def __init__(self, b, shift, power):
        self.l = np.asarray(b.l) + shift
        self.k = np.asarray(b.k)
        self.off = np.asarray(b.off)
        self.xyz = np.asarray(b.xyz)
        self.exps = np.asarray(b.exps)
        self.coefs = np.asarray(b.coefs) * (2.0 * np.asarray(b.exps)) ** power


def _cart_index(l):
    return {c: i for i, c in enumerate(cart_list(l))}


def _deriv_cart(plus, minus, l):
    """d/dcentre of a Cartesian block along the last axis.

    plus[..., nc(l+1)] holds (.|l+1) with 2zeta-weighted coefficients, minus
    [..., nc(l-1)] the plain (.|l-1) (or None when l = 0).  Returns [3, ..., nc(l)].
    """
    ip = _cart_index(l + 1)
    im = _cart_index(l - 1) if l > 0 else {}
    shape = plus.shape[:-1] + (ncart(l),)
    out = np.zeros((3,) + shape)
    for j, c in enumerate(cart_list(l)):
        for ax in range(3):
            cp = list(c)
            cp[ax] += 1
            out[ax][..., j] += plus[..., ip[tuple(cp)]]
            if c[ax] > 0:
                cm = list(c)
                cm[ax] -= 1
                out[ax][..., j] -= c[ax] * minus[..., im[tuple(cm)]]
    return out


def dfj_grad(orb, aux, D, c, natom, tasks=None):
    """dE/dR[natom, 3] for E = c^T gamma (pure orbital and aux bases)."""
    ao = ao_offsets(orb)
    aq = ao_offsets(aux)
    nsh = len(orb.l)
    if tasks is None:
        tasks = [(i, j, P) for i in range(nsh) for j in range(i, nsh) for P in range(len(aux.l))]
    tasks = np.asarray(tasks, np.int64).reshape(-1, 3)
    G = np.zeros((natom, 3))
    orb_p, orb_m = _Shifted(orb, +1, 1), _Shifted(orb, -1, 0)
    aux_p, aux_m = _Shifted(aux, +1, 1), _Shifted(aux, -1, 0)
    for (i, j, P) in tasks:
        la, lb, lc = int(orb.l[i]), int(orb.l[j]), int(aux.l[P])
        w = 1.0 if i == j else 2.0
        Dab = D[ao[i]:ao[i + 1], ao[j]:ao[j + 1]]
        cP = c[aq[P]:aq[P + 1]]
        W = w * np.einsum("AB,C->ABC", Dab, cP)
        Ta, Tb, Tc = solid_matrix(la), solid_matrix(lb), solid_matrix(lc)

        def cart(bA, sa, bB, sb, bC, sc):
            l_, k_, off_, xyz_, ex_, co_, base = _combined(bA, bB, bC)
            flat, _ = cart_blocks((l_, k_, off_, xyz_, ex_, co_),
                                  np.array([[sa, sb + base[1], sc + base[2]]], np.int32))
            return flat.reshape(ncart(int(l_[sa])), ncart(int(l_[sb + base[1]])),
                                ncart(int(l_[sc + base[2]])))

        # centre A
        plus = cart(orb_p, i, orb, j, aux, P)                   # (a+1 b|c)
        minus = cart(orb_m, i, orb, j, aux, P) if la > 0 else None
        dA = _deriv_cart(np.moveaxis(plus, 0, -1), None if minus is None else np.moveaxis(minus, 0, -1), la)
        dA = np.moveaxis(dA, -1, 1)                             # [3, a, b, c]
        # centre B
        plus = cart(orb, i, orb_p, j, aux, P)
        minus = cart(orb, i, orb_m, j, aux, P) if lb > 0 else None
        dB = _deriv_cart(np.moveaxis(plus, 1, -1), None if minus is None else np.moveaxis(minus, 1, -1), lb)
        dB = np.moveaxis(dB, -1, 2)
        # centre C
        plus = cart(orb, i, orb, j, aux_p, P)
        minus = cart(orb, i, orb, j, aux_m, P) if lc > 0 else None
        dC = _deriv_cart(plus, minus, lc)
        for d, atom in ((dA, orb.atom[i]), (dB, orb.atom[j]), (dC, aux.atom[P])):
            sph = np.einsum("Aa,Bb,Cc,xabc->xABC", Ta, Tb, Tc, d)
            G[int(atom)] += np.einsum("xABC,ABC->x", sph, W)
    return G
