"""GB300-native 3-center Coulomb integrals (ab|C) and density-fitted J.

Python face of the lx3c C-ABI library (include/lx3c.h).  Torch is used only
for device memory and streams; every step of the integral path runs in the
library's CUDA kernels.  Calls fail loudly (LibraryError) when the library or
a GPU is missing: there is no CPU fallback.

Main entry points:
  DeviceBasis(basis)                    upload a shell table (workloads.Basis)
  Eri3cPlan(orb, aux, pairs, auxs, bra_pure)   plan one (la lb|lc) class
      .execute(out=None, stream=None) -> torch.cuda tensor [npair, naux, nA, nB, nC]
  eri3c(orb, aux, pairs, auxs, bra_pure)       one-shot device evaluation
  eri3c_host(orb, aux, pairs, auxs, bra_pure)  host arrays in, numpy out
  boys(T, mmax)                          device Boys function (same evaluator)
  class_flops(la, lb, lc, Kab, Kc, bra_pure)   algorithmic FP64 flops per triple
"""
import ctypes
import os

import numpy as np

from . import _lib
from ._lib import LibraryError, check, ptr
from . import workloads  # noqa: F401  (seeded input generators)

__all__ = ["DeviceBasis", "Eri3cPlan", "DFJPlan", "DFJEnergy", "Batch", "MetricPlan", "cholesky", "cholesky_solve", "eri3c", "eri3c_host", "boys", "class_flops", "solid_harmonics",
           "cvrr2_expansion", "shape_hint", "tile_hint", "hrr_hint", "LibraryError", "workloads"]


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise LibraryError("lx3c needs a CUDA device; none is available")
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class DeviceBasis:
    """A basis uploaded to the current CUDA device (lx3c_basis)."""

    def __init__(self, basis, stream=None):
        L = _lib.load()
        self.basis = basis
        self.handle = ctypes.c_void_p()
        l = np.ascontiguousarray(basis.l, np.int32)
        k = np.ascontiguousarray(basis.k, np.int32)
        xyz = np.ascontiguousarray(basis.xyz, np.float64)
        atom = np.ascontiguousarray(basis.atom, np.int32) if getattr(basis, "atom", None) is not None else None
        ex = np.ascontiguousarray(basis.exps, np.float64)
        co = np.ascontiguousarray(basis.coefs, np.float64)
        check(L.lx3c_basis_create(ctypes.byref(self.handle), len(l), ptr(l), ptr(k), ptr(xyz), ptr(atom), ptr(ex),
                                  ptr(co), _stream_handle(stream)), "lx3c_basis_create")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.lx3c_basis_destroy(h)
            self.handle = None


class Eri3cPlan:
    """Plan for one homogeneous (la lb|lc) class over pair and ket-shell lists."""

    def __init__(self, orb, aux, pairs, auxs, bra_pure=True, stream=None):
        L = _lib.load()
        self.orb = orb if isinstance(orb, DeviceBasis) else DeviceBasis(orb, stream)
        self.aux = aux if isinstance(aux, DeviceBasis) else DeviceBasis(aux, stream)
        pairs = np.ascontiguousarray(np.asarray(pairs).reshape(-1, 2), np.int32)
        auxs = np.ascontiguousarray(np.asarray(auxs).reshape(-1), np.int32)
        self.npair, self.naux = len(pairs), len(auxs)
        self.handle = ctypes.c_void_p()
        check(L.lx3c_eri3c_plan(ctypes.byref(self.handle), self.orb.handle, self.aux.handle, ptr(pairs), len(pairs),
                                ptr(auxs), len(auxs), int(bool(bra_pure)), _stream_handle(stream)),
              "lx3c_eri3c_plan")
        blk, tot = ctypes.c_int64(), ctypes.c_int64()
        check(L.lx3c_plan_sizes(self.handle, ctypes.byref(blk), ctypes.byref(tot)), "lx3c_plan_sizes")
        self.block, self.total = blk.value, tot.value
        b = self.orb.basis
        la, lb = int(b.l[pairs[0, 0]]), int(b.l[pairs[0, 1]])
        lc = int(self.aux.basis.l[auxs[0]])
        nA = (2 * la + 1) if bra_pure else (la + 1) * (la + 2) // 2
        nB = (2 * lb + 1) if bra_pure else (lb + 1) * (lb + 2) // 2
        self.shape = (self.npair, self.naux, nA, nB, 2 * lc + 1)
        self.cls = (la, lb, lc)
        info = np.zeros(14, np.int64)
        check(L.lx3c_plan_info(self.handle, ptr(info), 14), "lx3c_plan_info")
        self.launches = int(info[0])
        self.flops = float(info[13])  # algorithmic flops of one execute, per chosen orientation
        self.shapes = [dict(nsub=int(info[1 + 6 * o]), T=int(info[2 + 6 * o]), G=int(info[3 + 6 * o]),
                            mode=int(info[4 + 6 * o]), smem=int(info[5 + 6 * o]), grid=int(info[6 + 6 * o]))
                       for o in range(2)]

    def execute(self, out=None, stream=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        if out.dtype != torch.float64 or not out.is_cuda or not out.is_contiguous() or out.numel() != self.total:
            raise LibraryError("execute: out must be a contiguous float64 CUDA tensor with %d elements" % self.total)
        check(_lib.load().lx3c_eri3c_execute(self.handle, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
              "lx3c_eri3c_execute")
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.lx3c_plan_destroy(h)
            self.handle = None


def eri3c(orb, aux, pairs, auxs, bra_pure=True, stream=None):
    """(ab|C) for every (pair, ket shell): CUDA tensor [npair, naux, nA, nB, nC]."""
    return Eri3cPlan(orb, aux, pairs, auxs, bra_pure, stream).execute(stream=stream)


def eri3c_host(orb, aux, pairs, auxs, bra_pure=True, out=None, stream=None):
    """Host-buffer path (lx3c_eri3c_host): numpy in, numpy out; copies inside the call."""
    L = _lib.load()
    pairs = np.ascontiguousarray(np.asarray(pairs).reshape(-1, 2), np.int32)
    auxs = np.ascontiguousarray(np.asarray(auxs).reshape(-1), np.int32)
    la, lb = int(orb.l[pairs[0, 0]]), int(orb.l[pairs[0, 1]])
    lc = int(aux.l[auxs[0]])
    nA = (2 * la + 1) if bra_pure else (la + 1) * (la + 2) // 2
    nB = (2 * lb + 1) if bra_pure else (lb + 1) * (lb + 2) // 2
    shape = (len(pairs), len(auxs), nA, nB, 2 * lc + 1)
    if out is None:
        out = np.empty(shape)
    arrs = []

    def a(x, dt):
        x = np.ascontiguousarray(x, dt)
        arrs.append(x)
        return ptr(x)

    st = _stream_handle(stream) if stream is not None else None
    check(L.lx3c_eri3c_host(len(orb.l), a(orb.l, np.int32), a(orb.k, np.int32), a(orb.xyz, np.float64),
                            a(orb.exps, np.float64), a(orb.coefs, np.float64), len(aux.l), a(aux.l, np.int32),
                            a(aux.k, np.int32), a(aux.xyz, np.float64), a(aux.exps, np.float64),
                            a(aux.coefs, np.float64), ptr(pairs), len(pairs), ptr(auxs), len(auxs),
                            int(bool(bra_pure)), ptr(out), st), "lx3c_eri3c_host")
    return out


class DFJPlan:
    """Screened DF-J build (lx3c_dfj): gamma_P and J_mn from D and c, Sec. 3."""

    def __init__(self, orb, aux, schwarz_tol=1e-12, gradient=False, contract=False, stream=None):
        """contract: digest at the (e 0|c) level (LX3C_DFJ_CONTRACT), the DF-J
        analogue of a J-engine: no ket transform, HRR or bra transform per triple."""
        L = _lib.load()
        self.orb = orb if isinstance(orb, DeviceBasis) else DeviceBasis(orb, stream)
        self.aux = aux if isinstance(aux, DeviceBasis) else DeviceBasis(aux, stream)
        self.handle = ctypes.c_void_p()
        flags = (1 if gradient else 0) | (2 if contract else 0)
        check(L.lx3c_dfj_plan(ctypes.byref(self.handle), self.orb.handle, self.aux.handle, float(schwarz_tol),
                              flags, _stream_handle(stream)), "lx3c_dfj_plan")
        info = np.zeros(11)
        check(L.lx3c_dfj_info(self.handle, ptr(info), 11), "lx3c_dfj_info")
        self.ngroups, self.ntasks, self.nint, self.flops, self.launches, self.nao, self.naux_ao = (
            int(info[0]), int(info[1]), float(info[2]), float(info[3]), int(info[4]), int(info[5]), int(info[6]))
        self.natom, self.grad_flops, self.grad_launches = int(info[7]), float(info[8]), int(info[9])
        self.tile_fill = float(info[1]) / max(float(info[10]), 1.0)

    def energy(self, D, c, stream=None):
        """E = c^T gamma (device scalar tensor) and gamma."""
        torch = _torch()
        gamma = torch.empty(self.naux_ao, dtype=torch.float64, device=D.device)
        E = torch.empty((), dtype=torch.float64, device=D.device)
        check(_lib.load().lx3c_dfj_energy(self.handle, ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                          ctypes.c_void_p(gamma.data_ptr()), ctypes.c_void_p(E.data_ptr()),
                                          _stream_handle(stream)), "lx3c_dfj_energy")
        return E, gamma

    def gradient(self, D, c, grad=None, stream=None):
        """dE/dR [natom, 3] for E = c^T gamma (D, c fixed)."""
        torch = _torch()
        if grad is None:
            grad = torch.empty((self.natom, 3), dtype=torch.float64, device=D.device)
        check(_lib.load().lx3c_dfj_grad(self.handle, ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(c.data_ptr()),
                                        ctypes.c_void_p(grad.data_ptr()), _stream_handle(stream)), "lx3c_dfj_grad")
        return grad

    def execute(self, D, c, gamma=None, J=None, stream=None, outputs="both"):
        """gamma and J (outputs="both"), or only one of them ("gamma" / "J"; the
        other is skipped and returned as None)."""
        torch = _torch()
        for name, t, n in (("D", D, self.nao * self.nao), ("c", c, self.naux_ao)):
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise LibraryError("DFJPlan.execute: %s must be a contiguous float64 CUDA tensor of %d" % (name, n))
        if outputs not in ("both", "gamma", "J"):
            raise LibraryError("DFJPlan.execute: outputs must be 'both', 'gamma' or 'J'")
        if outputs == "J":
            gamma = None
        elif gamma is None:
            gamma = torch.empty(self.naux_ao, dtype=torch.float64, device=D.device)
        if outputs == "gamma":
            J = None
        elif J is None:
            J = torch.empty((self.nao, self.nao), dtype=torch.float64, device=D.device)
        vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        check(_lib.load().lx3c_dfj_execute(self.handle, vp(D), vp(c), vp(gamma), vp(J), _stream_handle(stream)),
              "lx3c_dfj_execute")
        return gamma, J

    def execute_tiles(self, get_D, put_J, c, tile_ao=256, stream=None):
        """Tile-callback build (lx3c_dfj_execute_tiles): get_D(row0, nrow, col0, ncol)
        returns that tile of D (array-like [nrow, ncol]); put_J(row0, col0, tile)
        receives each tile of J (None: skip J).  c is host [naux_ao]; returns gamma
        (numpy)."""
        L = _lib.load()
        errors = []

        def g(user, r0, nr, c0, nc, dst, ld):
            try:
                t = np.asarray(get_D(int(r0), int(nr), int(c0), int(nc)), np.float64)
                out = np.ctypeslib.as_array(dst, shape=(int(nr) * int(ld),)).reshape(int(nr), int(ld))
                out[:, :nc] = t
                return 0
            except Exception as e:  # reported through the status
                errors.append(e)
                return 1

        def p(user, r0, nr, c0, nc, src, ld):
            try:
                a = np.ctypeslib.as_array(src, shape=(int(nr) * int(ld),)).reshape(int(nr), int(ld))[:, :nc]
                put_J(int(r0), int(c0), a.copy())
                return 0
            except Exception as e:
                errors.append(e)
                return 1

        gf = _lib.TILE_FN(g)
        pf = _lib.TILE_FN(p) if put_J is not None else ctypes.cast(None, _lib.TILE_FN)
        c = np.ascontiguousarray(c, np.float64)
        gamma = np.empty(self.naux_ao)
        rc = L.lx3c_dfj_execute_tiles(self.handle, int(tile_ao), gf, pf, None, ptr(c), ptr(gamma),
                                      _stream_handle(stream))
        if errors:
            raise errors[0]
        check(rc, "lx3c_dfj_execute_tiles")
        return gamma

    def execute_multi(self, Ds, cs, outputs="both", stream=None):
        """gamma [nd, naux_ao] and J [nd, nao, nao] for nd <= 8 densities Ds
        [nd, nao, nao] and coefficient vectors cs [nd, naux_ao] at once
        (lx3c_dfj_execute_multi); outputs="gamma" or "J" skips the other."""
        torch = _torch()
        nd = Ds.shape[0] if Ds is not None else cs.shape[0]
        for name, t, n in (("Ds", Ds, nd * self.nao * self.nao), ("cs", cs, nd * self.naux_ao)):
            if t is None:
                continue
            if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise LibraryError("DFJPlan.execute_multi: %s must be a contiguous float64 CUDA tensor of %d" % (name, n))
        dev = (Ds if Ds is not None else cs).device
        gamma = None if outputs == "J" else torch.empty((nd, self.naux_ao), dtype=torch.float64, device=dev)
        J = None if outputs == "gamma" else torch.empty((nd, self.nao, self.nao), dtype=torch.float64, device=dev)
        vp = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
        check(_lib.load().lx3c_dfj_execute_multi(self.handle, int(nd), vp(Ds), vp(cs), vp(gamma), vp(J),
                                                 _stream_handle(stream)), "lx3c_dfj_execute_multi")
        return gamma, J

    def coulomb(self, L, D, stream=None):
        """DF-J Coulomb build with the metric's Cholesky factor L:
        gamma, c = V^{-1} gamma and J (lx3c_dfj_coulomb)."""
        torch = _torch()
        gamma = torch.empty(self.naux_ao, dtype=torch.float64, device=D.device)
        c = torch.empty(self.naux_ao, dtype=torch.float64, device=D.device)
        J = torch.empty((self.nao, self.nao), dtype=torch.float64, device=D.device)
        check(_lib.load().lx3c_dfj_coulomb(self.handle, ctypes.c_void_p(L.data_ptr()), L.stride(0),
                                           ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(gamma.data_ptr()),
                                           ctypes.c_void_p(c.data_ptr()), ctypes.c_void_p(J.data_ptr()),
                                           _stream_handle(stream)), "lx3c_dfj_coulomb")
        return gamma, c, J

    def groups(self):
        """Screened task list: list of dicts (class, pairs[n,2], counts[n], auxs[m])."""
        L = _lib.load()
        out = []
        for g in range(self.ngroups):
            info = np.zeros(8, np.int32)
            check(L.lx3c_dfj_group(self.handle, g, ptr(info), None, None, None), "lx3c_dfj_group")
            npair, nket = int(info[6]), int(info[7])
            pairs = np.zeros((npair, 2), np.int32)
            counts = np.zeros(npair, np.int32)
            auxs = np.zeros(nket, np.int32)
            check(L.lx3c_dfj_group(self.handle, g, None, ptr(pairs), ptr(counts), ptr(auxs)), "lx3c_dfj_group")
            out.append(dict(cls=tuple(int(x) for x in info[:6]), pairs=pairs, counts=counts, auxs=auxs))
        return out

    def tasks(self):
        """All screened (a, b, P) triples as an int array [n, 3]."""
        rows = []
        for g in self.groups():
            for (a, b), n in zip(g["pairs"], g["counts"]):
                t = np.empty((n, 3), np.int64)
                t[:, 0], t[:, 1], t[:, 2] = a, b, g["auxs"][:n]
                rows.append(t)
        return np.concatenate(rows) if rows else np.zeros((0, 3), np.int64)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.lx3c_dfj_destroy(h)
            self.handle = None


class MetricPlan:
    """Coulomb metric V_PQ = (P|Q) of an aux basis (lx3c_metric)."""

    def __init__(self, aux, stream=None):
        L = _lib.load()
        self.aux = aux if isinstance(aux, DeviceBasis) else DeviceBasis(aux, stream)
        self.handle = ctypes.c_void_p()
        check(L.lx3c_metric_plan(ctypes.byref(self.handle), self.aux.handle, _stream_handle(stream)),
              "lx3c_metric_plan")
        info = np.zeros(6)
        check(L.lx3c_metric_info(self.handle, ptr(info), 6), "lx3c_metric_info")
        self.naux_ao, self.groups, self.class_launches, self.launches = (int(x) for x in info[:4])
        self.flops = float(info[4])

    def execute(self, V=None, stream=None):
        torch = _torch()
        if V is None:
            V = torch.empty((self.naux_ao, self.naux_ao), dtype=torch.float64, device="cuda")
        if V.dtype != torch.float64 or not V.is_cuda or not V.is_contiguous() or V.numel() != self.naux_ao ** 2:
            raise LibraryError("MetricPlan.execute: V must be a contiguous float64 CUDA tensor [%d, %d]"
                               % (self.naux_ao, self.naux_ao))
        check(_lib.load().lx3c_metric_execute(self.handle, ctypes.c_void_p(V.data_ptr()), _stream_handle(stream)),
              "lx3c_metric_execute")
        return V

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.lx3c_metric_destroy(h)
            self.handle = None


def cholesky(A, drop_tol=0.0, stream=None):
    """In-place lower Cholesky factor of the symmetric positive definite CUDA
    float64 matrix A (lx3c_cholesky); returns (A, info): with drop_tol = 0 the
    1-based first non-positive pivot or 0, else the number of functions
    dropped as linearly dependent (reading info synchronises)."""
    torch = _torch()
    n = A.shape[0]
    if A.dtype != torch.float64 or not A.is_cuda or A.dim() != 2 or A.shape[1] < n or A.stride(1) != 1:
        raise LibraryError("cholesky: A must be a row-major float64 CUDA matrix")
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    check(_lib.load().lx3c_cholesky(ctypes.c_void_p(A.data_ptr()), n, A.stride(0), float(drop_tol),
                                    ctypes.c_void_p(info.data_ptr()), _stream_handle(stream)), "lx3c_cholesky")
    return A, int(info.item())


def cholesky_solve(L, B, stream=None):
    """B <- (L L^T)^{-1} B in place (lx3c_cholesky_solve); B is [n] or [n, nrhs]."""
    torch = _torch()
    n = L.shape[0]
    if B.dtype != torch.float64 or not B.is_cuda or not B.is_contiguous() or B.shape[0] != n:
        raise LibraryError("cholesky_solve: B must be a contiguous float64 CUDA tensor with %d rows" % n)
    nrhs = 1 if B.dim() == 1 else B.shape[1]
    check(_lib.load().lx3c_cholesky_solve(ctypes.c_void_p(L.data_ptr()), n, L.stride(0),
                                          ctypes.c_void_p(B.data_ptr()), nrhs, _stream_handle(stream)),
          "lx3c_cholesky_solve")
    return B


class Batch:
    """Several molecules' DF-J builds as one persistent, graph-captured launch.

    Batch([(orb, aux), ...], schwarz_tol, tune_cache).bind(Ds, cs) then
    .execute(mode) with mode 1 (one graph, one persistent kernel), 2 (one
    graph, class launches on parallel branches) or 0 (per-class launches)."""

    INFO = ["molecules", "tasks", "integrals", "flops", "plain_launches", "graph_kernels", "work_items",
            "class_launches", "smem", "grid", "tuned", "measured", "branch_kernels", "branches", "slots", "tiers"]

    def __init__(self, mols, schwarz_tol=1e-12, tune_cache=None, stream=None):
        L = _lib.load()
        self._bases = [(o if isinstance(o, DeviceBasis) else DeviceBasis(o, stream),
                        a if isinstance(a, DeviceBasis) else DeviceBasis(a, stream)) for o, a in mols]
        orbs = (ctypes.c_void_p * len(mols))(*[o.handle.value for o, _ in self._bases])
        auxs = (ctypes.c_void_p * len(mols))(*[a.handle.value for _, a in self._bases])
        self.handle = ctypes.c_void_p()
        check(L.lx3c_batch_plan(ctypes.byref(self.handle), len(mols), ctypes.cast(orbs, ctypes.c_void_p),
                                ctypes.cast(auxs, ctypes.c_void_p), float(schwarz_tol),
                                tune_cache.encode() if tune_cache else None, _stream_handle(stream)), "lx3c_batch_plan")
        self.nmol = len(mols)

    def info(self):
        out = np.zeros(len(self.INFO))
        check(_lib.load().lx3c_batch_info(self.handle, ptr(out), len(self.INFO)), "lx3c_batch_info")
        return dict(zip(self.INFO, [float(x) for x in out]))

    def bind(self, Ds, cs, stream=None):
        torch = _torch()
        self.D, self.c = list(Ds), list(cs)
        self.gamma = [torch.empty(c.numel(), dtype=torch.float64, device=c.device) for c in cs]
        self.J = [torch.empty_like(D) for D in Ds]
        arr = lambda ts: ctypes.cast((ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts]), ctypes.c_void_p)
        check(_lib.load().lx3c_batch_bind(self.handle, arr(self.D), arr(self.c), arr(self.gamma), arr(self.J),
                                          _stream_handle(stream)), "lx3c_batch_bind")
        return self

    def execute(self, mode=1, stream=None):
        check(_lib.load().lx3c_batch_execute(self.handle, int(mode), _stream_handle(stream)), "lx3c_batch_execute")
        return self.gamma, self.J

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.lx3c_batch_destroy(h)
            self.handle = None


def _moved(basis, R):
    """Copy of a shell table with every shell centred on its atom's row of R."""
    from .workloads import Basis
    b = Basis(basis.l, basis.k, basis.off, np.asarray(R)[np.asarray(basis.atom)], basis.exps, basis.coefs,
              basis.atom)
    return b


class DFJEnergy:
    """E(R) = c^T gamma(R) as a torch.autograd.Function (not in the paper).

    E = DFJEnergy.apply(R, orb, aux, D, c[, tol]) with R [natom, 3] float64
    atom positions (bohr); shells sit on R[atom].  Forward: lx3c_dfj_energy.
    Backward: lx3c_dfj_grad (adjoint derivative integrals contracted with
    D_ab c_P on the fly), dE/dR [natom, 3].  D and c are held fixed.
    """

    @staticmethod
    def _fn():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, R, orb, aux, D, c, tol=1e-12):
                Rn = R.detach().cpu().numpy()
                plan = DFJPlan(_moved(orb, Rn), _moved(aux, Rn), tol, gradient=True)
                E, _ = plan.energy(D, c)
                ctx.plan = plan
                ctx.save_for_backward(D, c)
                ctx.rdev = R.device
                return E.to(R.device)

            @staticmethod
            def backward(ctx, gE):
                D, c = ctx.saved_tensors
                g = ctx.plan.gradient(D, c)
                return (gE.to(g.device) * g).to(ctx.rdev), None, None, None, None, None

        return _F

    _cls = None

    @classmethod
    def apply(cls, *args):
        if cls._cls is None:
            cls._cls = cls._fn()
        return cls._cls.apply(*args)


def boys(T, mmax, stream=None):
    """F_0..F_mmax at the values of the CUDA float64 tensor T: tensor [n, mmax+1]."""
    torch = _torch()
    T = T.contiguous()
    out = torch.empty((T.numel(), mmax + 1), dtype=torch.float64, device=T.device)
    check(_lib.load().lx3c_boys(ctypes.c_void_p(T.data_ptr()), T.numel(), int(mmax), ctypes.c_void_p(out.data_ptr()),
                                _stream_handle(stream)), "lx3c_boys")
    return out


def shape_hint(la, lb, lc, kab, kc=1, ctas_per_sm=2, bra_pure=True):
    """Size later plans of class (la, lb | lc) with kab x kc primitives for
    ctas_per_sm CTAs per SM (lx3c_shape_hint; 0 removes the hint)."""
    check(_lib.load().lx3c_shape_hint(la, lb, lc, int(bool(bra_pure)), kab, kc, ctas_per_sm), "lx3c_shape_hint")


def tile_hint(la, lb, lc, kab, kc, T, G, bra_pure=True):
    """Fix the tile of later plans of class (la, lb | lc) with kab x kc
    primitives: T triples per tile, chunks of G primitives (lx3c_tile_hint;
    T = 0 removes the hint)."""
    check(_lib.load().lx3c_tile_hint(la, lb, lc, int(bool(bra_pure)), kab, kc, int(T), int(G)), "lx3c_tile_hint")


def hrr_hint(la, lb, lc, variant, bra_pure=True):
    """HRR variant of class (la, lb | lc) for later plans: 0 one quantum per
    round, 1 two quanta per round, -1 remove the hint (lx3c_hrr_hint)."""
    check(_lib.load().lx3c_hrr_hint(la, lb, lc, int(bool(bra_pure)), int(variant)), "lx3c_hrr_hint")


def shape_query(la, lb, lc, kab, kc=1, naux=512, ctas_per_sm=0, bra_pure=True):
    """(T, G, mode, smem bytes) the planner gives the class (lx3c_shape_query)."""
    out = np.zeros(4, np.int32)
    check(_lib.load().lx3c_shape_query(la, lb, lc, int(bool(bra_pure)), kab, kc, int(naux), ctas_per_sm, ptr(out)),
          "lx3c_shape_query")
    return tuple(int(x) for x in out)


def set_orientation_threshold(amp_max=0.0):
    """Largest weighted HRR amplification a pair keeps unsplit (0: default 300),
    for later plans (lx3c_set_orientation_threshold)."""
    check(_lib.load().lx3c_set_orientation_threshold(float(amp_max)), "lx3c_set_orientation_threshold")


def set_compensation(bits=0):
    """Compensated summation in later plans' contracted stages: bit 0 gather,
    bit 1 ket transform (lx3c_set_compensation)."""
    check(_lib.load().lx3c_set_compensation(int(bits)), "lx3c_set_compensation")


HINTS_GB300 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "shape_hints_gb300.txt")


def load_shape_hints(path=HINTS_GB300):
    """Apply a tuned hints file, '#' comments; per line either
    "la lb lc bra_pure kab kc ctas_per_sm" (lx3c_shape_hint) or
    "la lb lc bra_pure kab kc 0 T G" (lx3c_tile_hint); returns the number of
    hints applied."""
    n = 0
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            v = [int(x) for x in line]
            la, lb, lc, pure, kab, kc, ctas = v[:7]
            if len(v) == 9:
                tile_hint(la, lb, lc, kab, kc, v[7], v[8], bool(pure))
            else:
                shape_hint(la, lb, lc, kab, kc, ctas, bool(pure))
            n += 1
    return n


def fp64_rate(iters=1 << 16, stream=None):
    """Measured FP64 FMA rate of the current device: (GFLOP/s, ms) (lx3c_fp64_rate)."""
    g, ms = ctypes.c_double(), ctypes.c_double()
    check(_lib.load().lx3c_fp64_rate(int(iters), ctypes.byref(g), ctypes.byref(ms), _stream_handle(stream)),
          "lx3c_fp64_rate")
    return g.value, ms.value


def schwarz_factors(orb, pairs, aux, kets):
    """The DF-J plan's screening factors (host only): Q_ab for each pair of
    orb shells and Q_P for each ket shell (lx3c_schwarz_pair / lx3c_schwarz_aux);
    a triple is kept when Q_ab Q_P >= tol."""
    L = _lib.load()
    f = lambda b, s: (int(b.l[s]), int(b.k[s]), np.ascontiguousarray(b.xyz[s], np.float64),
                      np.ascontiguousarray(b.exps[b.off[s]:b.off[s] + b.k[s]], np.float64),
                      np.ascontiguousarray(b.coefs[b.off[s]:b.off[s] + b.k[s]], np.float64))
    qp, qa = np.zeros(len(pairs)), np.zeros(len(kets))
    q = ctypes.c_double()
    for i, (a, b) in enumerate(pairs):
        la, ka, A, ea, ca = f(orb, a)
        lb, kb, B, eb, cb = f(orb, b)
        check(L.lx3c_schwarz_pair(la, ka, ptr(A), ptr(ea), ptr(ca), lb, kb, ptr(B), ptr(eb), ptr(cb),
                                  ctypes.byref(q)), "lx3c_schwarz_pair")
        qp[i] = q.value
    for i, s in enumerate(kets):
        l, k, _, e, c = f(aux, s)
        check(L.lx3c_schwarz_aux(l, k, ptr(e), ptr(c), ctypes.byref(q)), "lx3c_schwarz_aux")
        qa[i] = q.value
    return qp, qa


HRR_HINTS_GB300 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hrr_hints_gb300.txt")


def load_hrr_hints(path=HRR_HINTS_GB300):
    """Apply an HRR-variant hints file ("la lb lc bra_pure variant" per line,
    '#' comments); returns the number of hints applied."""
    n = 0
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            la, lb, lc, pure, v = (int(x) for x in line)
            hrr_hint(la, lb, lc, v, bool(pure))
            n += 1
    return n


def class_flops(la, lb, lc, Kab, Kc=1, bra_pure=True):
    f = ctypes.c_double()
    check(_lib.load().lx3c_class_flops(la, lb, lc, Kab, Kc, int(bool(bra_pure)), ctypes.byref(f)), "lx3c_class_flops")
    return f.value


def solid_harmonics(l):
    nc = (l + 1) * (l + 2) // 2
    out = np.zeros((2 * l + 1, nc))
    check(_lib.load().lx3c_solid_harmonics(l, ptr(out)), "lx3c_solid_harmonics")
    return out


def cvrr2_expansion(a, c, cap=4096):
    """Library's n-q CVRR2 expansion of (a 0|c): {((ex,ey,ez), k, (nx,ny,nz)): coef}."""
    a = np.ascontiguousarray(a, np.int32)
    c = np.ascontiguousarray(c, np.int32)
    terms = np.zeros((cap, 8))
    n = ctypes.c_int32()
    check(_lib.load().lx3c_cvrr2_expansion(ptr(a), ptr(c), cap, ptr(terms), ctypes.byref(n)), "lx3c_cvrr2_expansion")
    out = {}
    for t in terms[:n.value]:
        out[(tuple(int(x) for x in t[0:3]), int(t[3]), tuple(int(x) for x in t[4:7]))] = float(t[7])
    return out
