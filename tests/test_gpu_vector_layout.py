"""The vector layout of the fused step kernel (k_step_vec: V consecutive nodes
per thread, each population moved as one aligned vector, the pull's one-node
shift taken from the neighbouring lane) against the FP64 oracle and against
the strided layout, through the C ABI.

The shapes put every path of the kernel to work: rows whose pull crosses a
periodic face (wrap at the row band level), rows next to a wall (the
per-node path with halfway bounce-back), walls at the row ends, rows whose
length is not a multiple of V (the ragged last thread), rows too short for
any vector thread, and warps whose first and last lanes load the edge
elements themselves.
"""
import numpy as np
import pytest

import lbm_workloads as W
import oracle as O
from helpers import LAT, make_pair

pytestmark = pytest.mark.gpu

TAU = {"BGK": (1.0, 1.0, 0.71, 1.0, 1.0), "SMRT": (1.0, 1.3, 0.63, 0.87, 1.1),
       "SMRT_TRIM": (1.0, 1.3, 0.63, 1.0, 1.0), "SMRT_FNEQ": (1.0, 1.3, 0.63, 0.87, 1.1),
       "MRT_RAW": (1.0, 1.3, 0.63, 0.87, 1.1)}
COLLS = ["BGK", "SMRT", "SMRT_TRIM", "SMRT_FNEQ", "MRT_RAW"]
# (shape, periodic): walls in y (and z) with a ragged row; walls at the row
# ends with periodic y (z); a row of three warps plus a ragged tail with
# everything periodic; a domain too short for any vector thread; rows that
# every width fills, periodic in x, so the first and last threads of a row
# take their edge elements across the periodic face
CASES = {
    "D2Q9": [((150, 37, 1), (1, 0, 1)), ((136, 20, 1), (0, 1, 1)), ((803, 6, 1), (1, 1, 1)), ((9, 5, 1), (1, 1, 1)),
             ((256, 6, 1), (1, 1, 1))],
    "D3Q19": [((70, 9, 7), (1, 0, 0)), ((64, 6, 5), (0, 1, 1)), ((203, 4, 3), (1, 1, 1)), ((5, 4, 3), (1, 1, 1)),
              ((64, 4, 3), (1, 1, 1))],
    "D3Q27": [((70, 9, 7), (1, 0, 0)), ((64, 6, 5), (0, 1, 1)), ((203, 4, 3), (1, 1, 1)), ((5, 4, 3), (1, 1, 1)),
              ((64, 4, 3), (1, 1, 1))],
}


def _model(coll):
    return "SMRT" if coll == "SMRT_TRIM" else coll


def _g(lat):
    return np.array([2e-5, -1e-5, 4e-6][: 2 if lat == "D2Q9" else 3])


def _widths(lat, st):
    import paper_2212_07494_gb300 as P
    lo, hi = P.lbm_launch_widths(lat, st)
    return sorted({lo, hi})


def _state(lat, shape, seed, amp):
    _, Q, _, w, _ = O.lattice_tables(LAT[lat])
    return W.random_populations(w, shape, seed, amp=amp), w


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("coll", COLLS)
@pytest.mark.parametrize("case", [0, 1, 2, 3, 4])
def test_vector_layout_f64_matches_oracle(lat, coll, case):
    """Three steps from an arbitrary state in FP64 at every vector width and
    two block widths: the oracle's populations to 1e-14."""
    shape, periodic = CASES[lat][case]
    f0, _ = _state(lat, shape, 100 + case, 0.03)
    orc = None
    ref = []
    for V in _widths(lat, "F64"):
        for bx in (32, 128):
            gl, o = make_pair(lat, _model(coll), shape, TAU[coll], "F64", periodic, g=_g(lat))
            gl.set_launch(bx, V, "vector")
            assert gl.launch() == (bx, V, 1)
            gl.set_populations(f0)
            if orc is None:
                orc = o
                orc.set_populations(f0)
                for _ in range(3):
                    orc.step(1)
                    ref.append(orc.populations())
            for s in range(3):
                gl.step(1)
                err = np.abs(gl.populations() - ref[s]).max()
                assert err < 1e-14, (V, bx, s, err)
            gl.close()


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19", "D3Q27"])
@pytest.mark.parametrize("storage", ["F32", "F16", "BF16"])
@pytest.mark.parametrize("coll", ["BGK", "SMRT_TRIM", "MRT_RAW"])
def test_vector_layout_reduced_storage(lat, storage, coll):
    """One step from a state representable in the storage format: against
    the oracle with the same rounding (as the strided kernel's test), and
    against the strided kernel itself, which runs the same per-node
    arithmetic: bit for bit, since a node rounds alike alone or paired."""
    for shape, periodic in CASES[lat][:3] + CASES[lat][4:]:
        f0, w = _state(lat, shape, 200, 0.05)
        gl, orc = make_pair(lat, _model(coll), shape, TAU[coll], storage, periodic, g=_g(lat), emulate_storage=True)
        orc.set_populations(f0)
        fr = orc.populations()
        orc.step(1)
        do = orc.populations() - w[:, None, None, None]
        scale = np.abs(do).max()
        gl.set_launch(64, 1, "strided")
        gl.set_populations(fr)
        gl.step(1)
        strided = gl.populations()
        for V in _widths(lat, storage):
            gl.set_launch(64, V, "vector")
            gl.set_populations(fr)
            gl.step(1)
            fv = gl.populations()
            dg = fv - w[:, None, None, None]
            if storage == "F32":
                assert np.abs(dg - do).max() < 64 * 2.0 ** -24 * scale
            else:
                ulp = 2.0 ** -11 if storage == "F16" else 2.0 ** -8
                assert np.all(np.abs(dg - do) <= 2 * ulp * np.abs(do) + 64 * 2.0 ** -24 * scale + 6e-8)
            # the strided kernel collides its nodes alone (one per thread),
            # the vector one in pairs: FP32 rounds them alike, the same bits
            assert np.array_equal(fv, strided), (V, np.abs(fv - strided).max())
        gl.close()


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q27"])
def test_vector_layout_field_force_and_autotune(lat):
    """A per-node force field (the vector kernel reads it node by node) over
    many steps, then the autotuner over both layouts on the live state: it
    must leave the state unchanged and keep the results."""
    shape, periodic = CASES[lat][0]
    nx, ny, nz = shape
    D = 2 if lat == "D2Q9" else 3
    rng = W.SplitMix64(7)
    g = 1e-5 * rng.normal(D * nx * ny * nz).reshape(D, nz, ny, nx)
    rho0, u0 = W.random_near_equilibrium(lat, shape, seed=8, du=0.02)
    gl, orc = make_pair(lat, "SMRT", shape, TAU["SMRT"], "F64", periodic, g=g, force_kind="field", rho0=rho0, u0=u0)
    assert gl.launch()[2] == 0            # FP64 starts strided
    gl.set_launch(32, _widths(lat, "F64")[-1], "vector")
    gl.step(40)
    orc.step(40)
    before = gl.populations()
    bx, npt, ms = gl.autotune(3)
    assert ms > 0 and gl.launch()[:2] == (bx, npt)
    assert np.array_equal(gl.populations(), before)
    gl.step(20)
    orc.step(20)
    ug, uo = gl.moments()[1], orc.moments()[1]
    assert np.linalg.norm(ug - uo) / np.linalg.norm(uo) < 1e-12
    gl.close()


def test_default_layouts():
    """A new handle starts with the layout measured faster on GB300: the
    vector one for 2-byte storage and D3Q27 in FP32 without a mask, else
    strided."""
    import paper_2212_07494_gb300 as P
    for lat, st, vec in (("D2Q9", "F16", 1), ("D2Q9", "BF16", 1), ("D2Q9", "F32", 0), ("D3Q27", "F16", 1),
                         ("D3Q19", "BF16", 1), ("D3Q27", "F32", 1), ("D3Q19", "F32", 0), ("D2Q9", "F64", 0)):
        shape = (256, 8, 1) if lat == "D2Q9" else (64, 4, 4)
        gl = P.Lattice(lat, "SMRT", shape, TAU["SMRT_TRIM"], st, (1, 1, 1))
        assert gl.launch()[2] == vec, (lat, st, gl.launch())
        gl.close()


def test_vector_layout_rejected_with_a_mask():
    import paper_2212_07494_gb300 as P
    shape = (64, 16, 1)
    solid = W.random_solid(shape, seed=3, frac=0.05)
    gl = P.Lattice("D2Q9", "SMRT", shape, TAU["SMRT"], "F32", (1, 0, 1), g=[1e-6, 0.0], solid=solid)
    assert gl.launch()[2] == 0
    with pytest.raises(P.LbmError):
        gl.set_launch(128, 4, "vector")
    with pytest.raises(P.LbmError):
        gl.set_launch(128, 3, "strided")
    gl.close()
