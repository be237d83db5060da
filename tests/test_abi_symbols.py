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
