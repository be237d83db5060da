"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/lbm.h declares (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_07494_gb300 import build as B
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lbm_create", "lbm_step", "lbm_moments", "lbm_destroy", "lbm_residual",
                     "lbm_set_force", "lbm_get_state", "lbm_set_state", "lbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_the_same_names():
    import paper_2212_07494_gb300 as P
    for n in _declared():
        assert hasattr(P, n), n


def test_null_arguments_are_rejected_without_a_gpu(lib):
    """lbm_create validates its description before touching the device."""
    import paper_2212_07494_gb300 as P
    lib.lbm_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.lbm_create(None, ctypes.byref(h)) == -1
    d, keep = P.make_desc("D2Q9", "BGK", (8, 8), (1, 1, 0.5, 1, 1))  # tau = 1/2 is invalid
    assert lib.lbm_create(ctypes.byref(d), ctypes.byref(h)) == -1
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_last_error.argtypes = [ctypes.c_void_p]
    assert b"tau" in lib.lbm_last_error(None)
    d, keep = P.make_desc("D2Q9", "BGK", (8, 8, 2), (1, 1, 0.8, 1, 1))  # nz must be 1 in 2-D
    assert lib.lbm_create(ctypes.byref(d), ctypes.byref(h)) == -1


def test_check_noalloc_rejects_oversized_problems_before_device_work(lib):
    """The allocation-free check refuses problems whose velocity snapshot
    does not fit its static scratch, on the host, before touching a device."""
    import paper_2212_07494_gb300 as P
    desc, keep = P.make_desc("D2Q9", "SMRT", (4096, 4096, 1), (1, 1, 0.6, 1, 1), "F32", (1, 1, 1))
    with pytest.raises(P.LbmError) as e:
        P.lbm_check_noalloc(desc, None, None, None)
    assert e.value.status == -1
    with pytest.raises(P.LbmError) as e:
        P.lbm_check_noalloc(desc, 1, 1, None)
    assert e.value.status == -1 and "static scratch" in str(e.value)
    desc, keep = P.make_desc("D2Q9", "SMRT", (64, 64, 1), (1, 1, 0.6, 1, 1), "F32", (1, 1, 1),
                             solid=np.zeros(64 * 64, np.uint8))
    with pytest.raises(P.LbmError) as e:
        P.lbm_check_noalloc(desc, 1, 1, None)
    assert "solid" in str(e.value)


def test_bulk_tau_arguments_are_checked_without_a_gpu(lib):
    """A bulk relaxation time must exceed 1/2 and applies to the SMRT
    collisions only; both are rejected before any device work."""
    import paper_2212_07494_gb300 as P
    lib.lbm_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_last_error.argtypes = [ctypes.c_void_p]
    h = ctypes.c_void_p()
    for coll, tb in [("SMRT", 0.4), ("BGK", 0.9), ("MRT_RAW", 0.9), ("SMRT_FNEQ", -1.0)]:
        d, keep = P.make_desc("D2Q9", coll, (8, 8), (1, 1, 0.8, 1, 1), tau_bulk=tb)
        assert lib.lbm_create(ctypes.byref(d), ctypes.byref(h)) == -1, coll
        assert b"tau_bulk" in lib.lbm_last_error(None)


def test_unet_wgrad_selector_rejects_a_null_network(lib):
    lib.lbm_unet_set_wgrad.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.lbm_unet_set_wgrad(None, 0) == -1


def _err(lib):
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_last_error.argtypes = [ctypes.c_void_p]
    return lib.lbm_last_error(None).decode()


def test_invalid_descriptions_are_rejected_before_device_work(lib):
    """Every argument check of lbm_create runs on the host before any CUDA
    call: each bad field gives LBM_ERR_ARG and names the problem."""
    import paper_2212_07494_gb300 as P
    lib.lbm_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    h = ctypes.c_void_p()
    cases = [("lattice", 7, "lattice"), ("collision", 9, "collision"), ("storage", 9, "storage"),
             ("force_kind", 9, "force kind"), ("nx", 0, "sizes"), ("ny", 70000, "65535"),
             ("nx", 1 << 20, "too large")]
    for field, value, msg in cases:
        d, keep = P.make_desc("D2Q9", "SMRT", (8, 8), (1, 1, 0.8, 1, 1))
        if field == "nx" and value == 1 << 20:
            d.ny = 60000
        setattr(d, field, value)
        assert lib.lbm_create(ctypes.byref(d), ctypes.byref(h)) == -1, field
        assert msg in _err(lib), (field, _err(lib))
        assert not h.value
    d, keep = P.make_desc("D2Q9", "SMRT", (8, 8), (1, 1, 0.8, 0.5, 1))
    assert lib.lbm_create(ctypes.byref(d), ctypes.byref(h)) == -1 and "tau[2..4]" in _err(lib)
    d, keep = P.make_desc("D2Q9", "SMRT", (8, 8), (1, 1, 0.8, 1, 1))
    d.alloc = ctypes.cast(ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)(lambda n, c: None),
                          type(d.alloc))
    assert lib.lbm_create(ctypes.byref(d), ctypes.byref(h)) == -1 and "together" in _err(lib)


def test_invalid_batches_are_rejected_before_device_work(lib):
    import paper_2212_07494_gb300 as P
    lib.lbm_batch_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    b = ctypes.c_void_p()
    g = [1e-6, 0.0]

    def arr(*descs):
        a = (type(descs[0]) * len(descs))(*descs)
        return a, len(descs)

    ok, k0 = P.make_desc("D2Q9", "SMRT", (16, 8), (1, 1, 0.8, 1, 1), "F32", (1, 0, 1), g=g)
    cases = [
        ([P.make_desc("D3Q27", "SMRT", (8, 8, 8), (1, 1, 0.8, 1, 1), "F32", g=[1e-6, 0, 0])[0]], "D2Q9"),
        ([P.make_desc("D2Q9", "SMRT", (16, 8), (1, 1, 0.8, 1, 1), "F16", (1, 0, 1), g=g)[0]], "F32 or F64"),
        ([P.make_desc("D2Q9", "MRT_RAW", (16, 8), (1, 1, 0.8, 0.5, 1), "F32", (1, 0, 1), g=g)[0]], "tau[2..4]"),
        ([ok, P.make_desc("D2Q9", "BGK", (16, 8), (1, 1, 0.8, 1, 1), "F32", (1, 0, 1), g=g)[0]], "share"),
        ([P.make_desc("D2Q9", "SMRT", (16, 8), (1, 1, 0.8, 1, 1), "F32", (1, 0, 1), g=np.zeros((8, 2)),
                      force_kind="rows")[0]], "uniform force"),
        ([P.make_desc("D2Q9", "SMRT", (16, 8), (1, 1, 0.8, 1, 1), "F32", (1, 0, 1), g=g, tau_bulk=1.1)[0]], "one tau"),
    ]
    for descs, msg in cases:
        a, n = arr(*descs)
        assert lib.lbm_batch_create(a, n, ctypes.byref(b)) == -1, msg
        assert msg in _err(lib), (msg, _err(lib))
        assert not b.value
    a, n = arr(ok)
    assert lib.lbm_batch_create(a, 0, ctypes.byref(b)) == -1 and "at least one" in _err(lib)


def test_invalid_networks_are_rejected_before_device_work(lib):
    lib.lbm_unet_create.argtypes = [ctypes.c_int] * 5 + [ctypes.c_void_p, ctypes.c_void_p]
    u = ctypes.c_void_p()
    for args, msg in [((12, 16, 3, 0, 1), "multiples of 8"), ((16, 16, 0, 0, 1), "cin"),
                      ((16, 16, 17, 0, 1), "cin"), ((256, 16, 3, 0, 300), "65535"),
                      ((16, 16, 3, 2, 1), "periodic_x"), ((16, 16, 3, 0, 0), "max_batch")]:
        assert lib.lbm_unet_create(*args, None, ctypes.byref(u)) == -1, args
        assert msg in _err(lib), (args, _err(lib))
        assert not u.value


def test_null_handles_are_rejected(lib):
    lib.lbm_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    lib.lbm_residual.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    lib.lbm_set_force.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.lbm_step(None, 1) == -1 and "NULL" in _err(lib)
    r = ctypes.c_double()
    assert lib.lbm_residual(None, 10, ctypes.byref(r)) == -1
    assert lib.lbm_set_force(None, None) == -1


def test_vector_widths_without_a_gpu(lib):
    """lbm_launch_widths is host-only: D2Q9 moves 16 bytes per population and
    thread at its wider width in every storage type."""
    import paper_2212_07494_gb300 as P
    for st, size in (("F64", 8), ("F32", 4), ("F16", 2), ("BF16", 2)):
        lo, hi = P.lbm_launch_widths("D2Q9", st)
        assert hi * size == 16 and lo <= hi
        for lat in ("D3Q19", "D3Q27"):
            lo3, hi3 = P.lbm_launch_widths(lat, st)
            assert 4 <= lo3 * size <= hi3 * size <= 8
    with pytest.raises(P.LbmError):
        P.lbm_launch_widths(5, "F32")
