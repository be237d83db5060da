"""Shared test helpers: run the same seeded problem through the oracle and the
CUDA library and compare.  Tests only (imports both sides)."""
import numpy as np

import oracle as O

LAT = {"D2Q9": O.D2Q9, "D3Q19": O.D3Q19, "D3Q27": O.D3Q27}
COLL = {"BGK": O.BGK, "SMRT": O.SMRT, "SMRT_FNEQ": O.SMRT_FNEQ, "MRT_RAW": O.MRT_RAW}
ROUND = {"F64": O.ROUND_NONE, "F32": O.ROUND_F32, "F16": O.ROUND_F16, "BF16": O.ROUND_BF16}


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (den if den > 0 else 1.0))


def make_pair(lattice, collision, shape, tau, storage="F64", periodic=(1, 1, 1), g=None,
              force_kind="uniform", solid=None, rho0=None, u0=None, emulate_storage=False, tau_bulk=0.0):
    """(gpu Lattice, oracle Sim) built from identical inputs."""
    from paper_2212_07494_gb300 import Lattice
    gl = Lattice(lattice, collision, shape, tau, storage, periodic, g,
                 force_kind if g is not None else "none", solid, rho0, u0, tau_bulk=tau_bulk)
    og = None
    if g is not None:
        og = g
    orc = O.Sim(LAT[lattice], COLL[collision], shape, periodic, tau, g=og, force_kind=force_kind,
                solid=solid, rho0=rho0, u0=u0,
                round_mode=ROUND[storage] if emulate_storage else 0, tau_bulk=tau_bulk)
    return gl, orc
