"""The Python binding's argument marshalling, on the CPU: make_desc lays out
the C descriptor as include/lbm.h defines it and refuses arrays of the wrong
size before anything reaches the library."""

import numpy as np
import pytest


def test_make_desc_fills_the_c_descriptor():
    import paper_2212_07494_gb300 as P
    g = np.arange(2 * 8, dtype=float).reshape(8, 2) * 1e-7
    d, keep = P.make_desc("D2Q9", "SMRT_FNEQ", (16, 8), (1, 1, 0.8, 0.9), "BF16", (1, 0, 1), g=g,
                          force_kind="rows", tau_bulk=1.3)
    assert (d.lattice, d.collision, d.storage) == (P.LBM_D2Q9, P.LBM_SMRT_FNEQ, P.LBM_BF16_SHIFT)
    assert (d.nx, d.ny, d.nz) == (16, 8, 1) and list(d.periodic) == [1, 0, 1]
    assert list(d.tau) == [1.0, 1.0, 0.8, 0.9, 1.0]          # missing orders default to 1
    assert d.tau_bulk == 1.3 and d.force_kind == P.LBM_G_ROWS
    assert np.array_equal(np.ctypeslib.as_array(d.g, (16,)), g.ravel())
    assert not d.solid and not d.rho0 and not d.u0
    d, keep = P.make_desc("D3Q19", "BGK", (4, 5, 6), (1, 1, 0.7), g=[1e-6, 0, 0])
    assert d.force_kind == P.LBM_G_UNIFORM and (d.nx, d.ny, d.nz) == (4, 5, 6)
    d, keep = P.make_desc("D3Q27", "SMRT", (4, 4, 4), (1, 1, 0.7))
    assert d.force_kind == P.LBM_G_NONE and not d.g


@pytest.mark.parametrize("kw", [
    {"g": [1e-6, 0, 0]},                                   # uniform D2Q9 force takes 2 values
    {"g": np.zeros((7, 2)), "force_kind": "rows"},         # one row per y: 8
    {"g": np.zeros(16 * 8), "force_kind": "field"},        # D values per node: 256
    {"solid": np.zeros(16 * 8 + 1, np.uint8)},
    {"rho0": np.ones(16 * 7)},
    {"u0": np.zeros(16 * 8)},
])
def test_make_desc_rejects_wrong_sizes(kw):
    import paper_2212_07494_gb300 as P
    with pytest.raises(ValueError):
        P.make_desc("D2Q9", "SMRT", (16, 8), (1, 1, 0.8), **kw)


def test_make_desc_rejects_unknown_names():
    import paper_2212_07494_gb300 as P
    for kw in ({"lattice": "D2Q7"}, {"collision": "TRT"}, {"storage": "F8"}):
        args = {"lattice": "D2Q9", "collision": "SMRT", "shape": (8, 8), "tau": (1, 1, 0.8)}
        args.update(kw)
        with pytest.raises(KeyError):
            P.make_desc(**args)


def test_descriptor_layout_matches_the_header():
    """Field order and types of lbm_desc as include/lbm.h declares them."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = open(os.path.join(root, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct\s*\{(.*?)\}\s*lbm_desc;", src, re.S).group(1)
    declared = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.search(r"\(\*\s*(\w+)\)", decl)
        if m:
            declared.append(m.group(1))
            continue
        for part in decl.split(","):
            declared.append(re.sub(r"\[.*\]", "", part).split()[-1].lstrip("*"))
    from paper_2212_07494_gb300 import _binding
    bound = [f[0] for f in _binding.lbm_desc._fields_]
    assert bound == declared, (bound, declared)
