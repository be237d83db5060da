"""ctypes marshalling for include/lbm.h.  Argument conversion only: every
computation happens in the CUDA library ``lib/liblbm_gb300.so``."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "lib", "liblbm_gb300.so")

LBM_D2Q9, LBM_D3Q19, LBM_D3Q27 = 0, 1, 2
LBM_NOT_CONVERGED = 1
LBM_BGK, LBM_SMRT, LBM_SMRT_FNEQ, LBM_MRT_RAW = 0, 1, 2, 3
LBM_F64, LBM_F32, LBM_F16_SHIFT, LBM_BF16_SHIFT = 0, 1, 2, 3
LBM_G_NONE, LBM_G_UNIFORM, LBM_G_ROWS, LBM_G_FIELD = 0, 1, 2, 3
LBM_LAYOUT_STRIDED, LBM_LAYOUT_VECTOR = 0, 1

_NAMES = {
    "lattice": {"D2Q9": 0, "D3Q19": 1, "D3Q27": 2},
    "collision": {"BGK": 0, "SMRT": 1, "SMRT_FNEQ": 2, "MRT_RAW": 3},
    "storage": {"F64": 0, "F32": 1, "F16": 2, "F16_SHIFT": 2, "BF16": 3, "BF16_SHIFT": 3},
    "force": {"none": 0, "uniform": 1, "rows": 2, "field": 3},
    "layout": {"strided": 0, "vector": 1},
}
_DQ = {0: (2, 9), 1: (3, 19), 2: (3, 27)}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class lbm_desc(C.Structure):
    _fields_ = [("lattice", C.c_int), ("collision", C.c_int), ("storage", C.c_int),
                ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("periodic", C.c_int * 3), ("tau", C.c_double * 5), ("force_kind", C.c_int),
                ("g", C.POINTER(C.c_double)), ("solid", C.POINTER(C.c_uint8)),
                ("rho0", C.POINTER(C.c_double)), ("u0", C.POINTER(C.c_double)),
                ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free_", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("tau_bulk", C.c_double)]


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"lbm status {status}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _LIB_PATH


def library():
    """Load the CUDA library; raise ImportError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is not built: run `python -m paper_2212_07494_gb300.build`")
    L = C.CDLL(_LIB_PATH)
    H = C.c_void_p
    dp = C.POINTER(C.c_double)
    L.lbm_create.argtypes = [C.POINTER(lbm_desc), C.POINTER(H)]
    L.lbm_step.argtypes = [H, C.c_int64]
    L.lbm_moments.argtypes = [H, dp, dp, dp]
    L.lbm_moments_device.argtypes = [H, C.c_void_p, C.c_void_p, C.c_void_p]
    L.lbm_residual.argtypes = [H, C.c_int, dp]
    L.lbm_check_device.argtypes = [H, C.c_void_p]
    L.lbm_set_force.argtypes = [H, dp]
    L.lbm_set_force_schedule.argtypes = [H, dp, C.c_int64]
    L.lbm_set_force_scale_schedule.argtypes = [H, dp, C.c_int64]
    L.lbm_get_populations.argtypes = [H, dp]
    L.lbm_set_populations.argtypes = [H, dp]
    L.lbm_state_bytes.argtypes = [H]
    L.lbm_state_bytes.restype = C.c_size_t
    L.lbm_get_state.argtypes = [H, C.c_void_p, C.c_size_t, C.POINTER(C.c_int64)]
    L.lbm_set_state.argtypes = [H, C.c_void_p, C.c_size_t, C.c_int64]
    L.lbm_info.argtypes = [H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int64),
                           C.POINTER(C.c_size_t)]
    L.lbm_set_launch.argtypes = [H, C.c_int, C.c_int]
    L.lbm_set_launch_layout.argtypes = [H, C.c_int, C.c_int, C.c_int]
    L.lbm_get_launch.argtypes = [H, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.lbm_launch_widths.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.lbm_force_resolution.argtypes = [H, dp]
    L.lbm_alu_peak.argtypes = [C.c_int, C.c_int64, dp, dp]
    L.lbm_autotune.argtypes = [H, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.lbm_check_noalloc.argtypes = [C.POINTER(lbm_desc), C.c_void_p, C.c_void_p, C.c_void_p]
    S = C.c_void_p
    ip = C.POINTER(C.c_int)
    L.lbm_split_schedule.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, ip, ip, C.c_int, ip]
    L.lbm_split_create.argtypes = [C.POINTER(lbm_desc), C.c_int, C.POINTER(S)]
    L.lbm_split_step.argtypes = [S, C.c_int64]
    L.lbm_split_check_device.argtypes = [S, C.c_void_p]
    L.lbm_split_moments.argtypes = [S, dp, dp, dp]
    L.lbm_split_state_bytes.argtypes = [S]
    L.lbm_split_state_bytes.restype = C.c_size_t
    L.lbm_split_get_state.argtypes = [S, C.c_void_p, C.c_size_t, C.POINTER(C.c_int64)]
    L.lbm_split_get_populations.argtypes = [S, dp]
    L.lbm_split_set_launch_layout.argtypes = [S, C.c_int, C.c_int, C.c_int]
    L.lbm_split_last_error.argtypes = [S]
    L.lbm_split_last_error.restype = C.c_char_p
    L.lbm_split_destroy.argtypes = [S]
    L.lbm_split_destroy.restype = None
    B = C.c_void_p
    L.lbm_batch_create.argtypes = [C.POINTER(lbm_desc), C.c_int, C.POINTER(B)]
    L.lbm_batch_run_to_steady.argtypes = [B, C.c_double, C.c_int, C.c_int64, C.POINTER(C.c_int64),
                                          C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.lbm_batch_step.argtypes = [B, C.c_int64]
    L.lbm_batch_reset.argtypes = [B]
    L.lbm_batch_moments.argtypes = [B, C.c_int, dp, dp]
    L.lbm_batch_get_populations.argtypes = [B, C.c_int, dp]
    L.lbm_batch_set_tiles.argtypes = [B, C.c_int, C.c_int]
    L.lbm_batch_autotune.argtypes = [B, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.lbm_batch_set_spin_limit.argtypes = [B, C.c_int64]
    L.lbm_batch_set_handoff.argtypes = [B, C.c_int]
    L.lbm_batch_info.argtypes = [B, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.lbm_batch_last_error.argtypes = [B]
    L.lbm_batch_last_error.restype = C.c_char_p
    L.lbm_batch_destroy.argtypes = [B]
    L.lbm_batch_destroy.restype = None
    L.lbm_destroy.argtypes = [H]
    L.lbm_destroy.restype = None
    L.lbm_last_error.argtypes = [H]
    L.lbm_last_error.restype = C.c_char_p
    for n in ("lbm_create", "lbm_step", "lbm_moments", "lbm_moments_device", "lbm_residual",
              "lbm_check_device",
              "lbm_set_force", "lbm_set_force_schedule", "lbm_set_force_scale_schedule", "lbm_get_populations", "lbm_set_populations", "lbm_get_state",
              "lbm_set_state", "lbm_info", "lbm_set_launch", "lbm_set_launch_layout", "lbm_get_launch",
              "lbm_launch_widths", "lbm_force_resolution", "lbm_alu_peak", "lbm_autotune", "lbm_check_noalloc", "lbm_split_schedule", "lbm_split_create",
              "lbm_split_step", "lbm_split_check_device", "lbm_split_moments", "lbm_split_get_state",
              "lbm_split_get_populations", "lbm_split_set_launch_layout",
              "lbm_batch_create", "lbm_batch_run_to_steady", "lbm_batch_step", "lbm_batch_reset",
              "lbm_batch_moments", "lbm_batch_get_populations", "lbm_batch_set_tiles", "lbm_batch_autotune",
              "lbm_batch_set_spin_limit", "lbm_batch_set_handoff", "lbm_batch_info"):
        getattr(L, n).restype = C.c_int
    _lib = L
    return L


def _check(status, handle=None):
    if status != 0:
        msg = library().lbm_last_error(handle)
        raise LbmError(status, msg.decode() if msg else "")


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).ravel()
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def _enum(kind, v):
    return _NAMES[kind][v] if isinstance(v, str) else int(v)


def make_desc(lattice, collision, shape, tau, storage="F32", periodic=(1, 1, 1), g=None,
              force_kind=None, solid=None, rho0=None, u0=None, stream=None, alloc=None, free=None,
              tau_bulk=0.0):
    """Build an lbm_desc plus the arrays it points to (kept in the returned
    ``keep`` list for as long as the descriptor is used)."""
    lat = _enum("lattice", lattice)
    D, Q = _DQ[lat]
    nx, ny, nz = (list(shape) + [1, 1])[:3]
    N = nx * ny * nz
    if force_kind is None:
        force_kind = "none" if g is None else "uniform"
    fk = _enum("force", force_kind)
    d = lbm_desc()
    d.lattice, d.collision, d.storage = lat, _enum("collision", collision), _enum("storage", storage)
    d.nx, d.ny, d.nz = nx, ny, nz
    for k in range(3):
        d.periodic[k] = int(periodic[k])
    t = list(tau) + [1.0] * (5 - len(tau))
    for k in range(5):
        d.tau[k] = float(t[k])
    d.force_kind = fk
    d.tau_bulk = float(tau_bulk)
    keep = []
    if fk != LBM_G_NONE:
        n = {LBM_G_UNIFORM: D, LBM_G_ROWS: ny * D, LBM_G_FIELD: D * N}[fk]
        ga = _f64(g, n)
        keep.append(ga)
        d.g = _dptr(ga)
    if solid is not None:
        sa = np.ascontiguousarray(np.asarray(solid, np.uint8)).ravel()
        if sa.size != N:
            raise ValueError("solid has the wrong size")
        keep.append(sa)
        d.solid = sa.ctypes.data_as(C.POINTER(C.c_uint8))
    if rho0 is not None:
        r = _f64(rho0, N)
        keep.append(r)
        d.rho0 = _dptr(r)
    if u0 is not None:
        u = _f64(u0, D * N)
        keep.append(u)
        d.u0 = _dptr(u)
    d.stream = stream
    if alloc is not None:
        d.alloc, d.free_ = alloc, free
        keep += [alloc, free]
    return d, keep


# ---------------------------------------------------------------- C ABI names
def lbm_create(desc):
    h = C.c_void_p()
    _check(library().lbm_create(C.byref(desc), C.byref(h)))
    return h


def lbm_destroy(h):
    library().lbm_destroy(h)


def lbm_step(h, n):
    _check(library().lbm_step(h, int(n)), h)


def lbm_moments(h, rho, u, totals):
    _check(library().lbm_moments(h, _dptr(rho), _dptr(u), _dptr(totals)), h)


def lbm_moments_device(h, rho_ptr, u_ptr, totals_ptr):
    _check(library().lbm_moments_device(h, rho_ptr, u_ptr, totals_ptr), h)


def lbm_residual(h, K):
    r = C.c_double()
    _check(library().lbm_residual(h, int(K), C.byref(r)), h)
    return r.value


def lbm_check_device(h, out_ptr):
    _check(library().lbm_check_device(h, out_ptr), h)


def lbm_set_force(h, g):
    _check(library().lbm_set_force(h, _dptr(g)), h)


def lbm_set_force_schedule(h, table, period):
    _check(library().lbm_set_force_schedule(h, _dptr(table) if table is not None else None, int(period)), h)


def lbm_set_force_scale_schedule(h, scale, period):
    _check(library().lbm_set_force_scale_schedule(h, _dptr(scale) if scale is not None else None, int(period)), h)


def lbm_get_populations(h, out):
    _check(library().lbm_get_populations(h, _dptr(out)), h)


def lbm_set_populations(h, f):
    _check(library().lbm_set_populations(h, _dptr(f)), h)


def lbm_state_bytes(h):
    return int(library().lbm_state_bytes(h))


def lbm_get_state(h, buf):
    step = C.c_int64()
    _check(library().lbm_get_state(h, buf.ctypes.data_as(C.c_void_p), buf.nbytes, C.byref(step)), h)
    return step.value


def lbm_set_state(h, buf, step):
    _check(library().lbm_set_state(h, buf.ctypes.data_as(C.c_void_p), buf.nbytes, int(step)), h)


def lbm_info(h):
    D, Q, s, b = C.c_int(), C.c_int(), C.c_int64(), C.c_size_t()
    _check(library().lbm_info(h, C.byref(D), C.byref(Q), C.byref(s), C.byref(b)), h)
    return D.value, Q.value, s.value, b.value


def lbm_set_launch(h, block_x, nodes_per_thread):
    _check(library().lbm_set_launch(h, int(block_x), int(nodes_per_thread)), h)


def lbm_set_launch_layout(h, block_x, nodes_per_thread, layout):
    _check(library().lbm_set_launch_layout(h, int(block_x), int(nodes_per_thread), _enum("layout", layout)), h)


def lbm_get_launch(h):
    """(block_x, nodes_per_thread, layout)"""
    bx, npt, lay = C.c_int(), C.c_int(), C.c_int()
    _check(library().lbm_get_launch(h, C.byref(bx), C.byref(npt), C.byref(lay)), h)
    return bx.value, npt.value, lay.value


def lbm_launch_widths(lattice, storage):
    lo, hi = C.c_int(), C.c_int()
    _check(library().lbm_launch_widths(_enum("lattice", lattice), _enum("storage", storage), C.byref(lo),
                                       C.byref(hi)))
    return lo.value, hi.value


def lbm_force_resolution(h):
    u = C.c_double()
    _check(library().lbm_force_resolution(h, C.byref(u)), h)
    return u.value


def lbm_alu_peak(precision, iters):
    """(TFLOP/s, ms) of the FMA microbenchmark (see lbm_alu_peak)."""
    tf, ms = C.c_double(), C.c_double()
    _check(library().lbm_alu_peak(_enum("storage", precision), int(iters), C.byref(tf), C.byref(ms)))
    return tf.value, ms.value


def lbm_autotune(h, trials=20):
    bx, npt, ms = C.c_int(), C.c_int(), C.c_double()
    _check(library().lbm_autotune(h, int(trials), C.byref(bx), C.byref(npt), C.byref(ms)), h)
    return bx.value, npt.value, ms.value


def lbm_check_noalloc(desc, state_ptr, out_ptr, stream=None):
    """Allocation-free FP64 check of a caller-held state buffer (see lbm.h)."""
    _check(library().lbm_check_noalloc(C.byref(desc), state_ptr, out_ptr, stream))


def lbm_last_error(h=None):
    m = library().lbm_last_error(h)
    return m.decode() if m else ""


class Lattice:
    """One lattice handle.  Arrays are numpy, SoA, x fastest (see lbm.h).

    torch_stream: a ``torch.cuda.Stream`` to run on; with it the handle also
    allocates through PyTorch's caching allocator.  Otherwise the library
    creates its own stream and uses cudaMalloc."""

    def __init__(self, lattice, collision, shape, tau, storage="F32", periodic=(1, 1, 1), g=None,
                 force_kind=None, solid=None, rho0=None, u0=None, torch_stream=None, tau_bulk=0.0):
        self.lattice = _enum("lattice", lattice)
        self.D, self.Q = _DQ[self.lattice]
        nx, ny, nz = (list(shape) + [1, 1])[:3]
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self._cb = []
        stream = None
        alloc = free = None
        if torch_stream is not None:
            import torch
            self._torch_stream = torch_stream
            stream = torch_stream.cuda_stream
            dev = torch_stream.device

            def _alloc(nbytes, ctx):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, torch_stream)

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            alloc, free = ALLOC_FN(_alloc), FREE_FN(_free)
            self._cb = [alloc, free]
        desc, keep = make_desc(lattice, collision, shape, tau, storage, periodic, g, force_kind,
                               solid, rho0, u0, stream, alloc, free, tau_bulk)
        self.signature_fields = (desc.lattice, desc.collision, desc.storage, nx, ny, nz, solid is not None)
        self.force_kind = desc.force_kind
        self.h = lbm_create(desc)
        del keep

    def step(self, n=1):
        lbm_step(self.h, n)

    def moments(self):
        rho = np.empty(self.N)
        u = np.empty(self.D * self.N)
        tot = np.empty(4)
        lbm_moments(self.h, rho, u, tot)
        return rho.reshape(self.shape), u.reshape((self.D,) + self.shape), tot

    def totals(self):
        tot = np.empty(4)
        lbm_moments(self.h, None, None, tot)
        return tot

    def residual(self, K):
        return lbm_residual(self.h, K)

    def check_device(self, out_ptr):
        """Asynchronous FP64 check into 7 doubles at device address out_ptr."""
        lbm_check_device(self.h, out_ptr)

    def set_force(self, g):
        lbm_set_force(self.h, _f64(g))

    def set_force_scale_schedule(self, scale):
        """scale: (period,) factors applied to the force of the next `period`
        steps, repeating; None removes the schedule."""
        if scale is None:
            lbm_set_force_scale_schedule(self.h, None, 0)
            return
        s = np.ascontiguousarray(np.asarray(scale, np.float64).ravel())
        lbm_set_force_scale_schedule(self.h, s, s.size)

    def set_force_schedule(self, table):
        """table: (period, D) accelerations of the next `period` steps, repeating;
        None removes the schedule."""
        if table is None:
            lbm_set_force_schedule(self.h, None, 0)
            return
        t = np.ascontiguousarray(np.asarray(table, np.float64))
        if t.ndim != 2 or t.shape[1] != self.D:
            raise ValueError("schedule must have shape (period, D)")
        lbm_set_force_schedule(self.h, t.ravel(), t.shape[0])

    def populations(self):
        f = np.empty(self.Q * self.N)
        lbm_get_populations(self.h, f)
        return f.reshape((self.Q,) + self.shape)

    def set_populations(self, f):
        lbm_set_populations(self.h, _f64(f, self.Q * self.N))

    def state(self):
        buf = np.empty(lbm_state_bytes(self.h), np.uint8)
        step = lbm_get_state(self.h, buf)
        return buf, step

    def set_state(self, buf, step):
        lbm_set_state(self.h, np.ascontiguousarray(buf), step)

    def info(self):
        return lbm_info(self.h)

    def set_launch(self, block_x, nodes_per_thread, layout=0):
        """layout 0 / "strided" or 1 / "vector" (see lbm_set_launch_layout)."""
        lbm_set_launch_layout(self.h, block_x, nodes_per_thread, layout)

    def launch(self):
        """(block_x, nodes_per_thread, layout) of the step kernel."""
        return lbm_get_launch(self.h)

    def force_resolution(self):
        """Speed above which one step of the force rounds away in the storage
        format (see lbm_force_resolution); inf without a force."""
        return lbm_force_resolution(self.h)

    def note(self):
        """lbm_last_error of the handle (a note lbm_create may leave)."""
        return lbm_last_error(self.h)

    def autotune(self, trials=20, cache=None):
        """Pick the fastest launch shape (see lbm_autotune).  With a cache path,
        reuse a stored choice for the same problem signature or store the new
        one (JSON keyed by lattice, collision, storage, sizes, mask, device)."""
        key = None
        if cache:
            from . import autotune as A
            key = A.signature(self)
            hit = A.lookup(cache, key)
            if hit:
                self.set_launch(*hit["launch"])
                return tuple(hit["launch"]) + (hit["ms"],)
        bx, npt, ms = lbm_autotune(self.h, trials)
        if cache:
            from . import autotune as A
            A.store(cache, key, self.launch(), ms)
        return bx, npt, ms

    def close(self):
        if getattr(self, "h", None) is not None:
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ------------------------------------------------------------- split domains
def _scheck(status, s=None):
    if status != 0:
        msg = library().lbm_split_last_error(s)
        raise LbmError(status, msg.decode() if msg else "")


def lbm_split_schedule(lattice, n_all, parts, periodic):
    """(layers [(g0, n)] per slab, copies [(dst_part, dst_layer, src_part,
    src_layer, pop)]) of one exchange; host only."""
    L = library()
    lat = _enum("lattice", lattice)
    cnt = C.c_int()
    _scheck(L.lbm_split_schedule(lat, int(n_all), int(parts), int(bool(periodic)), None, None, 0, C.byref(cnt)))
    lay = (C.c_int * (2 * parts))()
    cp = (C.c_int * max(1, 5 * cnt.value))()
    _scheck(L.lbm_split_schedule(lat, int(n_all), int(parts), int(bool(periodic)), lay, cp, cnt.value,
                                 C.byref(cnt)))
    layers = [(lay[2 * p], lay[2 * p + 1]) for p in range(parts)]
    copies = [tuple(cp[5 * k:5 * k + 5]) for k in range(cnt.value)]
    return layers, copies


def lbm_split_create(desc, parts):
    s = C.c_void_p()
    _scheck(library().lbm_split_create(C.byref(desc), int(parts), C.byref(s)))
    return s


def lbm_split_step(s, n):
    _scheck(library().lbm_split_step(s, int(n)), s)


def lbm_split_check_device(s, out_ptr):
    _scheck(library().lbm_split_check_device(s, C.c_void_p(out_ptr)), s)


def lbm_split_moments(s, rho, u, totals):
    _scheck(library().lbm_split_moments(s, _dptr(rho), _dptr(u), _dptr(totals)), s)


def lbm_split_state_bytes(s):
    return int(library().lbm_split_state_bytes(s))


def lbm_split_get_state(s, buf):
    step = C.c_int64()
    _scheck(library().lbm_split_get_state(s, buf.ctypes.data_as(C.c_void_p), buf.nbytes, C.byref(step)), s)
    return step.value


def lbm_split_get_populations(s, f):
    _scheck(library().lbm_split_get_populations(s, _dptr(f)), s)


def lbm_split_set_launch_layout(s, block_x, nodes_per_thread, layout):
    _scheck(library().lbm_split_set_launch_layout(s, int(block_x), int(nodes_per_thread),
                                                  _enum("layout", layout)), s)


def lbm_split_last_error(s):
    m = library().lbm_split_last_error(s)
    return m.decode() if m else ""


def lbm_split_destroy(s):
    library().lbm_split_destroy(s)


class Split:
    """A domain split into `parts` slabs along its outermost axis, each slab
    in its own buffers, with the halo exchange after every step (see
    lbm_split_create).  Arguments as Lattice."""

    def __init__(self, parts, lattice, collision, shape, tau, storage="F32", periodic=(1, 1, 1), g=None,
                 force_kind=None, solid=None, rho0=None, u0=None, tau_bulk=0.0):
        self.lattice = _enum("lattice", lattice)
        self.D, self.Q = _DQ[self.lattice]
        nx, ny, nz = (list(shape) + [1, 1])[:3]
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        desc, keep = make_desc(lattice, collision, shape, tau, storage, periodic, g, force_kind, solid, rho0, u0,
                               None, None, None, tau_bulk)
        self.s = lbm_split_create(desc, parts)
        del keep

    def step(self, n=1):
        lbm_split_step(self.s, n)

    def check_device(self, out_ptr):
        lbm_split_check_device(self.s, out_ptr)

    def moments(self):
        rho = np.empty(self.N)
        u = np.empty(self.D * self.N)
        tot = np.empty(4)
        lbm_split_moments(self.s, rho, u, tot)
        return rho.reshape(self.shape), u.reshape((self.D,) + self.shape), tot

    def state(self):
        buf = np.empty(lbm_split_state_bytes(self.s), np.uint8)
        step = lbm_split_get_state(self.s, buf)
        return buf, step

    def populations(self):
        f = np.empty(self.Q * self.N)
        lbm_split_get_populations(self.s, f)
        return f.reshape((self.Q,) + self.shape)

    def set_launch(self, block_x, nodes_per_thread, layout=0):
        lbm_split_set_launch_layout(self.s, block_x, nodes_per_thread, layout)

    def close(self):
        if getattr(self, "s", None) is not None:
            lbm_split_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# -------------------------------------------------------------------- batches
def _bcheck(status, b=None):
    if status != 0:
        msg = library().lbm_batch_last_error(b) if b is not None else library().lbm_last_error(None)
        raise LbmError(status, msg.decode() if msg else "")


def lbm_batch_create(descs):
    arr = (lbm_desc * len(descs))(*descs)
    b = C.c_void_p()
    _bcheck(library().lbm_batch_create(arr, len(descs), C.byref(b)))
    return b


def lbm_batch_run_to_steady(b, n, tol, K, max_steps):
    steps = (C.c_int64 * n)()
    st = (C.c_int * n)()
    r = (C.c_double * n)()
    status = library().lbm_batch_run_to_steady(b, float(tol), int(K), int(max_steps), steps, st, r)
    return status, np.array(steps[:], np.int64), np.array(st[:], np.int32), np.array(r[:])


def lbm_batch_step(b, n):
    _bcheck(library().lbm_batch_step(b, int(n)), b)


def lbm_batch_reset(b):
    _bcheck(library().lbm_batch_reset(b), b)


def lbm_batch_moments(b, i, rho, u):
    _bcheck(library().lbm_batch_moments(b, int(i), _dptr(rho), _dptr(u)), b)


def lbm_batch_get_populations(b, i, f):
    _bcheck(library().lbm_batch_get_populations(b, int(i), _dptr(f)), b)


def lbm_batch_set_tiles(b, block, tile_nodes):
    _bcheck(library().lbm_batch_set_tiles(b, int(block), int(tile_nodes)), b)


def lbm_batch_autotune(b, steps):
    bl, tn, ms = C.c_int(), C.c_int(), C.c_double()
    _bcheck(library().lbm_batch_autotune(b, int(steps), C.byref(bl), C.byref(tn), C.byref(ms)), b)
    return bl.value, tn.value, ms.value


def lbm_batch_set_spin_limit(b, scans):
    _bcheck(library().lbm_batch_set_spin_limit(b, int(scans)), b)


def lbm_batch_set_handoff(b, channels):
    _bcheck(library().lbm_batch_set_handoff(b, int(channels)), b)


def lbm_batch_info(b, i):
    s, t, r = C.c_int64(), C.c_int(), C.c_int()
    _bcheck(library().lbm_batch_info(b, int(i), C.byref(s), C.byref(t), C.byref(r)), b)
    return s.value, t.value, r.value


def lbm_batch_last_error(b):
    m = library().lbm_batch_last_error(b)
    return m.decode() if m else ""


def lbm_batch_destroy(b):
    library().lbm_batch_destroy(b)


class Batch:
    """Independent D2Q9 channels in one persistent launch.  ``channels`` is a
    list of dicts with keys shape, tau, periodic, g (uniform), solid, rho0, u0."""

    def __init__(self, channels, collision="SMRT", storage="F32", stream=None):
        self._keep = []
        descs = []
        for ch in channels:
            d, keep = make_desc("D2Q9", collision, ch["shape"], ch["tau"], storage, ch.get("periodic", (1, 0, 1)),
                                g=ch.get("g"), solid=ch.get("solid"), rho0=ch.get("rho0"), u0=ch.get("u0"),
                                stream=stream)
            descs.append(d)
            self._keep.append(keep)
        self.shapes = [tuple((list(ch["shape"]) + [1, 1])[:3]) for ch in channels]
        self.n = len(descs)
        self.b = lbm_batch_create(descs)

    def run_to_steady(self, tol, K=1000, max_steps=10 ** 7):
        return lbm_batch_run_to_steady(self.b, self.n, tol, K, max_steps)

    def step(self, n):
        lbm_batch_step(self.b, n)

    def reset(self):
        lbm_batch_reset(self.b)

    def moments(self, i):
        nx, ny, _ = self.shapes[i]
        rho = np.empty(nx * ny)
        u = np.empty(2 * nx * ny)
        lbm_batch_moments(self.b, i, rho, u)
        return rho.reshape(1, ny, nx), u.reshape(2, 1, ny, nx)

    def populations(self, i):
        nx, ny, _ = self.shapes[i]
        f = np.empty(9 * nx * ny)
        lbm_batch_get_populations(self.b, i, f)
        return f.reshape(9, 1, ny, nx)

    def set_tiles(self, block, tile_nodes):
        lbm_batch_set_tiles(self.b, block, tile_nodes)

    def autotune(self, steps=200):
        return lbm_batch_autotune(self.b, steps)

    def set_spin_limit(self, scans):
        lbm_batch_set_spin_limit(self.b, scans)

    def set_handoff(self, channels):
        lbm_batch_set_handoff(self.b, channels)

    def info(self, i):
        return lbm_batch_info(self.b, i)

    def close(self):
        if getattr(self, "b", None) is not None:
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ surrogate
def _unet_lib():
    L = library()
    if not getattr(L, "_unet_ready", False):
        U = C.c_void_p
        fp = C.c_void_p
        L.lbm_unet_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(U)]
        L.lbm_unet_num_params.argtypes = [U]
        L.lbm_unet_num_params.restype = C.c_int64
        L.lbm_unet_set_params.argtypes = [U, C.POINTER(C.c_float)]
        L.lbm_unet_get_params.argtypes = [U, C.POINTER(C.c_float)]
        L.lbm_unet_forward.argtypes = [U, fp, fp, C.c_int]
        L.lbm_unet_grad.argtypes = [U, fp, fp, fp, C.c_int, C.c_float, C.POINTER(C.c_double), C.POINTER(C.c_float)]
        L.lbm_unet_adam.argtypes = [U, C.c_float, C.c_float, C.c_float, C.c_float]
        L.lbm_unet_train_step.argtypes = [U, fp, fp, fp, C.c_int, C.c_float, C.c_float, C.c_void_p]
        L.lbm_unet_set_wgrad.argtypes = [U, C.c_int]
        L.lbm_unet_last_error.argtypes = [U]
        L.lbm_unet_last_error.restype = C.c_char_p
        L.lbm_unet_destroy.argtypes = [U]
        L.lbm_unet_destroy.restype = None
        for n in ("lbm_unet_create", "lbm_unet_set_params", "lbm_unet_get_params", "lbm_unet_forward",
                  "lbm_unet_grad", "lbm_unet_adam", "lbm_unet_train_step", "lbm_unet_set_wgrad"):
            getattr(L, n).restype = C.c_int
        L._unet_ready = True
    return L


def _ucheck(status, u=None):
    if status != 0:
        m = _unet_lib().lbm_unet_last_error(u) if u is not None else library().lbm_last_error(None)
        raise LbmError(status, m.decode() if m else "")


def lbm_unet_create(H, W, cin, periodic_x, max_batch, stream=None):
    u = C.c_void_p()
    _ucheck(_unet_lib().lbm_unet_create(int(H), int(W), int(cin), int(bool(periodic_x)), int(max_batch), stream,
                                        C.byref(u)))
    return u


def lbm_unet_num_params(u):
    return int(_unet_lib().lbm_unet_num_params(u))


def lbm_unet_set_params(u, params):
    p = np.ascontiguousarray(np.asarray(params, np.float32))
    _ucheck(_unet_lib().lbm_unet_set_params(u, p.ctypes.data_as(C.POINTER(C.c_float))), u)


def lbm_unet_get_params(u, out):
    _ucheck(_unet_lib().lbm_unet_get_params(u, out.ctypes.data_as(C.POINTER(C.c_float))), u)


def lbm_unet_forward(u, x_ptr, y_ptr, n):
    _ucheck(_unet_lib().lbm_unet_forward(u, x_ptr, y_ptr, int(n)), u)


def lbm_unet_grad(u, x_ptr, t_ptr, m_ptr, n, scale, want_grad=True):
    loss = C.c_double()
    g = np.empty(lbm_unet_num_params(u), np.float32) if want_grad else None
    _ucheck(_unet_lib().lbm_unet_grad(u, x_ptr, t_ptr, m_ptr, int(n), float(scale), C.byref(loss),
                                      g.ctypes.data_as(C.POINTER(C.c_float)) if g is not None else None), u)
    return loss.value, g


def lbm_unet_adam(u, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _ucheck(_unet_lib().lbm_unet_adam(u, float(lr), float(beta1), float(beta2), float(eps)), u)


def lbm_unet_train_step(u, x_ptr, t_ptr, m_ptr, n, scale, lr, loss_ptr=None):
    _ucheck(_unet_lib().lbm_unet_train_step(u, x_ptr, t_ptr, m_ptr, int(n), float(scale), float(lr), loss_ptr), u)


UNET_WGRAD_AUTO, UNET_WGRAD_MMA_SYNC = 0, 1


def lbm_unet_set_wgrad(u, kind):
    _ucheck(_unet_lib().lbm_unet_set_wgrad(u, int(kind)), u)


def lbm_unet_destroy(u):
    _unet_lib().lbm_unet_destroy(u)


class UNet:
    """The surrogate network (see lbm.h).  Device tensors are passed as raw
    pointers (e.g. torch ``data_ptr()``), float32, inputs [n][H][W][cin],
    outputs and targets [n][H][W][3]; periodic_x wraps the convolutions
    around along x."""

    def __init__(self, H, W, max_batch, stream=None, cin=3, periodic_x=False):
        self.H, self.W, self.B, self.cin, self.periodic_x = H, W, max_batch, cin, bool(periodic_x)
        self.u = lbm_unet_create(H, W, cin, periodic_x, max_batch, stream)
        self.n = lbm_unet_num_params(self.u)

    def set_params(self, p):
        lbm_unet_set_params(self.u, p)

    def params(self):
        out = np.empty(self.n, np.float32)
        lbm_unet_get_params(self.u, out)
        return out

    def forward(self, x_ptr, y_ptr, n):
        lbm_unet_forward(self.u, x_ptr, y_ptr, n)

    def grad(self, x_ptr, t_ptr, m_ptr, n, scale, want_grad=True):
        return lbm_unet_grad(self.u, x_ptr, t_ptr, m_ptr, n, scale, want_grad)

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        lbm_unet_adam(self.u, lr, beta1, beta2, eps)

    def train_step(self, x_ptr, t_ptr, m_ptr, n, scale, lr, loss_ptr=None):
        lbm_unet_train_step(self.u, x_ptr, t_ptr, m_ptr, n, scale, lr, loss_ptr)

    def set_wgrad(self, kind):
        """"auto" (tcgen05 where the shape allows) or "mma_sync"."""
        lbm_unet_set_wgrad(self.u, {"auto": UNET_WGRAD_AUTO, "mma_sync": UNET_WGRAD_MMA_SYNC}[kind])

    def close(self):
        if getattr(self, "u", None) is not None:
            lbm_unet_destroy(self.u)
            self.u = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_unet_last_error(u):
    m = _unet_lib().lbm_unet_last_error(u)
    return m.decode() if m else ""
