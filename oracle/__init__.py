"""Plain FP64 CPU oracle for the second-order force scheme (arXiv:2212.07494).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its Python binding) never imports this package, and this
package imports nothing from the product.

The arithmetic lives in ``lbm_oracle.c`` (compiled with gcc, no fast-math, no
FMA contraction so x86 and Arm give identical bits).  This module only
marshals numpy arrays through ctypes and expands force specifications into a
per-node field.

Conventions (shared by the whole library, stated in ``include/lbm.h``):
populations are SoA ``f[i][z][y][x]`` (x fastest), velocity and force fields
``u[a][z][y][x]``, lattice units at the interface.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

D2Q9, D3Q19, D3Q27 = 0, 1, 2
BGK, SMRT, SMRT_FNEQ, MRT_RAW = 0, 1, 2, 3
PACK = 121  # packed Hermite tensor length (1 + 3 + 9 + 27 + 81)
ROUND_NONE, ROUND_F32, ROUND_F16, ROUND_BF16 = 0, 1, 2, 3

LATTICE_DQ = {D2Q9: (2, 9), D3Q19: (3, 19), D3Q27: (3, 27)}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (C99, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("lattice", C.c_int), ("collision", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("periodic", C.c_int * 3), ("tau", C.c_double * 5), ("tau_bulk", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            up = C.POINTER(C.c_ubyte)
            ip = C.POINTER(C.c_int)
            pp = C.POINTER(Params)
            L.or_lattice_tables.argtypes = [C.c_int, ip, ip, ip, dp, ip]
            L.or_hermite_table.argtypes = [C.c_int, dp, up, ip]
            L.or_hermite_at.argtypes = [C.c_int, dp, dp]
            L.or_project.argtypes = [C.c_int, dp, dp]
            L.or_reconstruct.argtypes = [C.c_int, dp, dp]
            L.or_shift.argtypes = [C.c_int, dp, dp, dp]
            L.or_collide_node.argtypes = [pp, dp, dp, dp, dp]
            L.or_initial_node.argtypes = [pp, C.c_double, dp, dp, dp]
            L.or_init.argtypes = [pp, up, dp, dp, dp, dp]
            L.or_step.argtypes = [pp, up, dp, dp, dp]
            L.or_moments.argtypes = [pp, up, dp, dp, dp, dp, dp]
            L.or_round_storage.argtypes = [pp, C.c_int, dp]
            L.or_round_value.argtypes = [C.c_int, dp, dp, C.c_int]
            L.or_run.argtypes = [pp, up, dp, dp, dp, C.c_longlong, C.c_int]
            L.or_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _d(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u8(a):
    if a is None:
        return None
    assert a.dtype == np.uint8 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_ubyte))


def set_threads(n: int) -> int:
    """Set the OpenMP thread count used by ``step``; returns the count in effect."""
    return int(lib().or_set_threads(int(n)))


def make_params(lattice, collision, shape, periodic=(1, 1, 1), tau=(1.0, 1.0, 0.8, 1.0, 1.0), tau_bulk=0.0):
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    p = Params()
    p.lattice, p.collision = int(lattice), int(collision)
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    for k in range(3):
        p.periodic[k] = int(periodic[k])
    t = list(tau) + [1.0] * (5 - len(tau))
    for k in range(5):
        p.tau[k] = float(t[k])
    p.tau_bulk = float(tau_bulk)
    return p


def lattice_tables(lattice):
    D, Q = C.c_int(), C.c_int()
    c = np.zeros((27, 3), np.int32)
    w = np.zeros(27)
    opp = np.zeros(27, np.int32)
    rc = lib().or_lattice_tables(int(lattice), C.byref(D), C.byref(Q),
                                 c.ctypes.data_as(C.POINTER(C.c_int)), _d(w),
                                 opp.ctypes.data_as(C.POINTER(C.c_int)))
    assert rc == 0
    q = Q.value
    return D.value, q, c[:q].copy(), w[:q].copy(), opp[:q].copy()


def hermite_table(lattice):
    """Packed H^(n)(xi_i) (Q x 121), retained mask (121,) and tensor offsets."""
    _, Q = LATTICE_DQ[lattice]
    H = np.zeros((Q, PACK))
    keep = np.zeros(PACK, np.uint8)
    off = np.zeros(6, np.int32)
    rc = lib().or_hermite_table(int(lattice), _d(H), _u8(keep), off.ctypes.data_as(C.POINTER(C.c_int)))
    assert rc == 0
    return H, keep.astype(bool), off


def hermite_at(D, x):
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    H = np.zeros(PACK)
    n = lib().or_hermite_at(int(D), _d(x), _d(H))
    return H[:n]


def project(lattice, f):
    f = np.ascontiguousarray(f, np.float64)
    a = np.zeros(PACK)
    assert lib().or_project(int(lattice), _d(f), _d(a)) == 0
    return a


def reconstruct(lattice, A):
    _, Q = LATTICE_DQ[lattice]
    A = np.ascontiguousarray(np.resize(np.asarray(A, np.float64), PACK))
    f = np.zeros(Q)
    assert lib().or_reconstruct(int(lattice), _d(A), _d(f)) == 0
    return f


def shift(lattice, s, a):
    s = np.zeros(3) + np.pad(np.asarray(s, np.float64), (0, 3 - len(s)))
    a = np.ascontiguousarray(np.resize(np.asarray(a, np.float64), PACK))
    out = np.zeros(PACK)
    assert lib().or_shift(int(lattice), _d(s), _d(a), _d(out)) == 0
    return out


def collide_node(params, fbar, g):
    """One node's collision; returns (fp, dbg) with dbg = 6 x 121 packed
    [a_bar, a_0, a_1, d_1, d_p, a_p] for SMRT (zeros for BGK)."""
    _, Q = LATTICE_DQ[params.lattice]
    fbar = np.ascontiguousarray(fbar, np.float64)
    g = np.zeros(3) + np.pad(np.asarray(g, np.float64), (0, 3 - len(g)))
    fp = np.zeros(Q)
    dbg = np.zeros((6, PACK))
    assert lib().or_collide_node(C.byref(params), _d(fbar), _d(g), _d(fp), _d(dbg)) == 0
    return fp, dbg


def initial_node(params, rho, u, g):
    _, Q = LATTICE_DQ[params.lattice]
    u = np.zeros(3) + np.pad(np.asarray(u, np.float64), (0, 3 - len(u)))
    g = np.zeros(3) + np.pad(np.asarray(g, np.float64), (0, 3 - len(g)))
    f = np.zeros(Q)
    assert lib().or_initial_node(C.byref(params), float(rho), _d(u), _d(g), _d(f)) == 0
    return f


def force_field(params, g, force_kind="uniform"):
    """Expand a force specification into the (D, nz, ny, nx) field the C code takes.

    uniform: g has D values.  rows: g has shape (ny, D), indexed by y.
    field: g already has shape (D, nz, ny, nx) (or (D, ny, nx) in 2-D)."""
    D, _ = LATTICE_DQ[params.lattice]
    nx, ny, nz = params.nx, params.ny, params.nz
    if g is None:
        return None
    g = np.asarray(g, np.float64)
    out = np.zeros((D, nz, ny, nx))
    if force_kind == "uniform":
        for a in range(D):
            out[a] = g[a]
    elif force_kind == "rows":
        g = g.reshape(ny, D)
        for a in range(D):
            out[a] = g[:, a][None, :, None]
    elif force_kind == "field":
        out[:] = g.reshape(D, nz, ny, nx)
    else:
        raise ValueError(force_kind)
    return np.ascontiguousarray(out)


class Sim:
    """Stateful oracle run.  ``d`` holds the stored deviations
    delta_i = fbar_i - w_i of the pre-collision populations fbar(x, t), [Q][N];
    ``populations()`` / ``set_populations()`` speak fbar."""

    def __init__(self, lattice, collision, shape, periodic=(1, 1, 1), tau=(1, 1, 0.8, 1, 1),
                 g=None, force_kind="uniform", solid=None, rho0=None, u0=None, round_mode=0, tau_bulk=0.0):
        self.p = make_params(lattice, collision, shape, periodic, tau, tau_bulk)
        self.D, self.Q = LATTICE_DQ[lattice]
        p = self.p
        self.N = p.nx * p.ny * p.nz
        self.shape = (p.nz, p.ny, p.nx)
        self.solid = None if solid is None else np.ascontiguousarray(
            np.asarray(solid, np.uint8).reshape(self.N))
        self.g = force_field(p, g, force_kind) if g is not None else np.zeros((self.D,) + self.shape)
        self.round_mode = int(round_mode)
        rho0 = None if rho0 is None else np.ascontiguousarray(np.asarray(rho0, np.float64).reshape(self.N))
        u0 = None if u0 is None else np.ascontiguousarray(np.asarray(u0, np.float64).reshape(self.D * self.N))
        self.w = lattice_tables(lattice)[3]
        self.d = np.zeros((self.Q, self.N))
        assert lib().or_init(C.byref(p), _u8(self.solid), _d(rho0), _d(u0), _d(self.g), _d(self.d)) == 0
        if self.round_mode:
            assert lib().or_round_storage(C.byref(p), self.round_mode, _d(self.d)) == 0
        self._work = np.zeros_like(self.d)
        self.t = 0

    def set_force(self, g, force_kind="uniform"):
        self.g = force_field(self.p, g, force_kind)

    def step(self, n=1):
        rc = lib().or_run(C.byref(self.p), _u8(self.solid), _d(self.g), _d(self.d), _d(self._work),
                          int(n), self.round_mode)
        assert rc == 0
        self.t += n

    def moments(self):
        rho = np.zeros(self.N)
        u = np.zeros(self.D * self.N)
        tot = np.zeros(4)
        assert lib().or_moments(C.byref(self.p), _u8(self.solid), _d(self.g), _d(self.d),
                                _d(rho), _d(u), _d(tot)) == 0
        return rho.reshape(self.shape), u.reshape((self.D,) + self.shape), tot

    def populations(self):
        """Pre-collision populations fbar = w + delta, (Q, nz, ny, nx)."""
        return (self.w[:, None] + self.d).reshape((self.Q,) + self.shape)

    def set_populations(self, f, round_mode=None):
        """Replace the state by fbar (deviations taken exactly, then rounded to
        the storage format when round_mode (default: the run's) is set)."""
        d = np.asarray(f, np.float64).reshape(self.Q, self.N) - self.w[:, None]
        self.d = np.ascontiguousarray(d)
        mode = self.round_mode if round_mode is None else int(round_mode)
        if mode:
            assert lib().or_round_storage(C.byref(self.p), mode, _d(self.d)) == 0


def round_values(mode, x):
    x = np.ascontiguousarray(np.asarray(x, np.float64))
    y = np.empty_like(x)
    lib().or_round_value(int(mode), _d(x), _d(y), int(x.size))
    return y
