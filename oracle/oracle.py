"""FP64 CPU oracle for the two-component plasma TREE method (arXiv 0709.3331).

TEST INFRASTRUCTURE ONLY.  The product path never imports this module; it is
used by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU-baseline leg
of ``bench.py``.  The arithmetic lives in ``ucp_oracle.c`` (plain C, compiled
with ``-ffp-contract=off``); this file only compiles it with gcc and marshals
numpy arrays through ctypes.  It shares no code with the CUDA library.

Every function follows a passage of the paper:
  * :func:`direct`        -- Sec. 2.1 Eq. 1-2, all pair-wise sum (Plummer-softened).
  * :func:`root_cube`, :func:`keys`, :func:`sort_order` -- Sec. 3, the enclosing
    cube and the eight-way boxes, written as integer box coordinates.
  * :class:`Tree`         -- Sec. 3, recursive subdivision, pseudo-particles and
    the particle-tree walk with the opening criterion of Eq. 5.
  * :func:`run`           -- Sec. 2 velocity Verlet with electron substeps.
  * :func:`energy`        -- Sec. 5 kinetic and potential energy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ucp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_d = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_u32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_i8 = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``ucp_oracle.c`` into ``liboracle.so`` beside it (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-std=c11"]
    tmp = _LIB + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.orc_direct.argtypes = [C.c_int64, _d, _i8, _d, C.c_double, C.c_void_p, C.c_int64,
                                     _d, _d, C.c_int]
            L.orc_direct_pe.argtypes = [C.c_int64, _d, _i8, _d, C.c_double]
            L.orc_direct_pe.restype = C.c_double
            L.orc_root_cube.argtypes = [C.c_int64, _d, _d]
            L.orc_int_coords.argtypes = [C.c_int64, _d, _d, _u32]
            L.orc_interleave.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32]
            L.orc_interleave.restype = C.c_uint64
            L.orc_keys.argtypes = [C.c_int64, _d, _d, _u64]
            L.orc_sort_order.argtypes = [C.c_int64, _u64, _i64]
            L.orc_tree_build.argtypes = [C.c_int64, _d, _i8, _d, C.c_int]
            L.orc_tree_build.restype = C.c_void_p
            L.orc_tree_free.argtypes = [C.c_void_p]
            L.orc_tree_nnodes.argtypes = [C.c_void_p]
            L.orc_tree_nnodes.restype = C.c_int64
            L.orc_tree_cube.argtypes = [C.c_void_p, _d]
            L.orc_tree_export.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
            L.orc_tree_force.argtypes = [C.c_void_p, _d, _i8, _d, C.c_double, C.c_double,
                                         C.c_void_p, C.c_int64, _d, _d, C.c_void_p, C.c_void_p,
                                         C.c_int, C.c_int]
            L.orc_run.argtypes = [C.c_int64, _d, _d, _i8, _d, _d, C.c_double, C.c_int, C.c_int64,
                                  C.c_double, C.c_double, C.c_int, C.c_int, _d, C.c_int, C.c_int]
            L.orc_energy.argtypes = [C.c_int64, _d, _d, _i8, _d, _d, C.c_double, C.c_double,
                                     C.c_int, C.c_int, _d, C.c_int]
            L.orc_has_openmp.restype = C.c_int
            L.orc_set_potential.argtypes = [C.c_int, C.c_double]
            L.orc_tree_force_adjoint.argtypes = [C.c_void_p, _d, _i8, _d, _d, C.c_double,
                                                 C.c_double, _d, _d]
            L.orc_direct_force_adjoint.argtypes = [C.c_int64, _d, _i8, _d, _d, C.c_double, _d, _d]
            L.orc_run_adjoint_ke_e.argtypes = [C.c_int64, _d, _d, _i8, _d, _d, C.c_double, C.c_int,
                                               C.c_int64, C.c_double, C.c_double, C.c_int, C.c_int,
                                               _d, _d, C.c_int]
            L.orc_run_adjoint_ke_e.restype = C.c_double
            L.orc_cluster_multipole.argtypes = [C.c_int64, _d, _i8, _d, C.c_double, _d, C.c_int,
                                                _d, _d]
            _lib = L
    return _lib


def _pos(a):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1, 3)


def _sp(a):
    return np.ascontiguousarray(a, dtype=np.int8)


def _qm(v):
    return np.ascontiguousarray(v, dtype=np.float64).reshape(2)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class kelbg:
    """Context manager: direct electron-ion pairs use the Kelbg form (Sec. 2.1
    Eq. 3) with a fixed lambda inside the block; Plummer Coulomb outside."""

    def __init__(self, lam):
        self.lam = float(lam)

    def __enter__(self):
        lib().orc_set_potential(1, self.lam)
        return self

    def __exit__(self, *exc):
        lib().orc_set_potential(0, 1.0)


def has_openmp() -> bool:
    return bool(lib().orc_has_openmp())


def direct(pos, species, q, eps, targets=None, nthreads=1):
    """All pair-wise field E (force per unit target charge) and potential phi
    on ``targets`` (Sec. 2.1 Eq. 1-2, Plummer-softened; no self term)."""
    pos, species, q = _pos(pos), _sp(species), _qm(q)
    n = pos.shape[0]
    tl = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if tl is None else tl.shape[0]
    E = np.zeros((nt, 3))
    phi = np.zeros(nt)
    lib().orc_direct(n, pos, species, q, float(eps), _ptr(tl), nt, E, phi, int(nthreads))
    return E, phi


def direct_pe(pos, species, q, eps):
    pos, species, q = _pos(pos), _sp(species), _qm(q)
    return lib().orc_direct_pe(pos.shape[0], pos, species, q, float(eps))


def root_cube(pos):
    """Enclosing cube {centre x, y, z, side} (Sec. 3)."""
    pos = _pos(pos)
    out = np.zeros(4)
    lib().orc_root_cube(pos.shape[0], pos, out)
    return out


def int_coords(pos, cube):
    pos = _pos(pos)
    k = np.zeros((pos.shape[0], 3), dtype=np.uint32)
    lib().orc_int_coords(pos.shape[0], pos, np.ascontiguousarray(cube, dtype=np.float64), k)
    return k


def interleave(kx, ky, kz) -> int:
    return int(lib().orc_interleave(int(kx), int(ky), int(kz)))


def keys(pos, cube=None):
    pos = _pos(pos)
    cube = root_cube(pos) if cube is None else np.ascontiguousarray(cube, dtype=np.float64)
    out = np.zeros(pos.shape[0], dtype=np.uint64)
    lib().orc_keys(pos.shape[0], pos, cube, out)
    return out


def sort_order(keys_):
    k = np.ascontiguousarray(keys_, dtype=np.uint64)
    out = np.zeros(k.shape[0], dtype=np.int64)
    lib().orc_sort_order(k.shape[0], k, out)
    return out


class Tree:
    """Serial TREE of Sec. 3 over one particle set (owns a C handle)."""

    def __init__(self, pos, species, q, leaf_cap=1):
        self.pos, self.species, self.q = _pos(pos), _sp(species), _qm(q)
        self.n = self.pos.shape[0]
        self.leaf_cap = int(leaf_cap)
        self._h = lib().orc_tree_build(self.n, self.pos, self.species, self.q, self.leaf_cap)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_tree_free(h)
            self._h = None

    @property
    def nnodes(self) -> int:
        return int(lib().orc_tree_nnodes(self._h))

    def cube(self):
        out = np.zeros(4)
        lib().orc_tree_cube(self._h, out)
        return out

    def export(self):
        """Node table: dict of numpy arrays (pre-order).  ``slot`` maps tree
        slot -> original particle index; node ranges index slots."""
        nn = self.nnodes
        topo = np.zeros((nn, 5), dtype=np.int64)
        cell = np.zeros((nn, 3), dtype=np.uint32)
        geom = np.zeros((nn, 20))
        slot = np.zeros(self.n, dtype=np.int64)
        lib().orc_tree_export(self._h, _ptr(topo), _ptr(cell), _ptr(geom), _ptr(slot))
        return {
            "begin": topo[:, 0], "end": topo[:, 1], "next": topo[:, 2], "depth": topo[:, 3],
            "is_leaf": topo[:, 4].astype(bool), "cell": cell, "centre": geom[:, 0:3],
            "side": geom[:, 3], "S0": geom[:, 4], "M": geom[:, 5], "c": geom[:, 6:9],
            "D": geom[:, 9:12], "Q": geom[:, 12:18], "delta": geom[:, 18], "slot": slot,
        }

    def force(self, theta, eps, targets=None, nthreads=1, term_mask=7, counts=False):
        """Tree field E and potential phi on ``targets`` (all when None); with
        ``counts`` also the per-target number of direct pairs and multipoles."""
        tl = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
        nt = self.n if tl is None else tl.shape[0]
        E = np.zeros((nt, 3))
        phi = np.zeros(nt)
        npp = np.zeros(nt, dtype=np.int64) if counts else None
        nmp = np.zeros(nt, dtype=np.int64) if counts else None
        lib().orc_tree_force(self._h, self.pos, self.species, self.q, float(theta), float(eps),
                             _ptr(tl), nt, E, phi, _ptr(npp), _ptr(nmp), int(nthreads),
                             int(term_mask))
        if counts:
            return E, phi, npp, nmp
        return E, phi


def cluster_multipole(pos, species, q, eps, xt, term_mask=7):
    """Field and potential at ``xt`` of the expansion (through quadrupole order)
    of one box holding all the given particles (Sec. 3 pseudo-particle)."""
    pos, species, q = _pos(pos), _sp(species), _qm(q)
    E = np.zeros(3)
    phi = np.zeros(1)
    lib().orc_cluster_multipole(pos.shape[0], pos, species, q, float(eps),
                                np.ascontiguousarray(xt, dtype=np.float64), int(term_mask), E, phi)
    return E, float(phi[0])


def force_adjoint(pos, species, q, m, lam, theta, eps, leaf_cap=1, direct_sum=False):
    """mu = (d a / d x)^T lam for a = q E / m (tree held fixed, or the direct sum)."""
    pos, species, q, m = _pos(pos), _sp(species), _qm(q), _qm(m)
    lam = _pos(lam)
    mu = np.zeros_like(pos)
    if direct_sum:
        lib().orc_direct_force_adjoint(pos.shape[0], pos, species, q, m, float(eps), lam, mu)
    else:
        T = Tree(pos, species, q, leaf_cap)
        lib().orc_tree_force_adjoint(T._h, pos, species, q, m, float(theta), float(eps), lam, mu)
    return mu


def run_adjoint_ke_e(pos, vel, species, q, m, dt_e, k, nblocks, theta, eps, leaf_cap=1,
                     direct_sum=False, nthreads=1):
    """(L, dL/dx0, dL/dv0) for L = electron kinetic energy after ``nblocks`` blocks."""
    pos, vel = _pos(pos), _pos(vel)
    gx = np.zeros_like(pos)
    gv = np.zeros_like(pos)
    L = lib().orc_run_adjoint_ke_e(pos.shape[0], pos, vel, _sp(species), _qm(q), _qm(m),
                                   float(dt_e), int(k), int(nblocks), float(theta), float(eps),
                                   int(leaf_cap), int(bool(direct_sum)), gx, gv, int(nthreads))
    return L, gx, gv


def accel(pos, species, q, m, theta, eps, leaf_cap=1, direct_sum=False, nthreads=1):
    """a_t = q_t E_t / m_t on all particles (tree or direct)."""
    species = _sp(species)
    q, m = _qm(q), _qm(m)
    if direct_sum:
        E, _ = direct(pos, species, q, eps, nthreads=nthreads)
    else:
        E, _ = Tree(pos, species, q, leaf_cap).force(theta, eps, nthreads=nthreads)
    return E * (q[species] / m[species])[:, None]


def run(pos, vel, species, q, m, dt_e, k, nblocks, theta, eps, leaf_cap=1, direct_sum=False,
        acc=None, nthreads=1):
    """Advance ``nblocks`` blocks of ``k`` electron substeps (Sec. 2 velocity
    Verlet, electron/ion split).  Returns (pos, vel, acc) as new arrays."""
    pos = _pos(pos).copy()
    vel = _pos(vel).copy()
    species = _sp(species)
    a = np.zeros_like(pos) if acc is None else _pos(acc).copy()
    lib().orc_run(pos.shape[0], pos, vel, species, _qm(q), _qm(m), float(dt_e), int(k),
                  int(nblocks), float(theta), float(eps), int(leaf_cap), int(bool(direct_sum)),
                  a, int(acc is not None), int(nthreads))
    return pos, vel, a


def energy(pos, vel, species, q, m, theta, eps, leaf_cap=1, direct_sum=False, nthreads=1):
    """[KE_ion, KE_electron, PE, E, |P|] (Sec. 5)."""
    pos, vel = _pos(pos), _pos(vel)
    out = np.zeros(5)
    lib().orc_energy(pos.shape[0], pos, vel, _sp(species), _qm(q), _qm(m), float(theta),
                     float(eps), int(leaf_cap), int(bool(direct_sum)), out, int(nthreads))
    return out
