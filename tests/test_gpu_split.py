"""A domain split into slabs along its outermost axis (separate buffers, one
halo layer per cut, the halo exchange after every step) against the same
domain unsplit: the state must be identical bit for bit after 100 steps,
with walls and obstacles crossing the cuts, in every storage mode and both
kernel layouts; the summed check must equal the whole domain's to rounding.
"""
import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu

TAU = (1.0, 1.0, 0.63, 1.0, 1.0)
TAU_G = (1.0, 1.3, 0.63, 0.87, 1.1)


def _g(D):
    return np.array([2e-5, -1e-5, 4e-6][:D])


def _pair(parts, lat, coll, shape, tau, storage, periodic, **kw):
    import paper_2212_07494_gb300 as P
    whole = P.Lattice(lat, coll, shape, tau, storage, periodic, **kw)
    split = P.Split(parts, lat, coll, shape, tau, storage, periodic, **kw)
    return whole, split


CASES_2D = [
    # shape, periodic, obstacles
    ((150, 37, 1), (1, 0, 1), True),     # walls in y, obstacles across the cuts
    ((96, 40, 1), (1, 1, 1), False),     # periodic y: the exchange wraps
    ((64, 21, 1), (0, 0, 1), True),      # walls on all sides
]


@pytest.mark.parametrize("case", range(len(CASES_2D)))
@pytest.mark.parametrize("parts", [2, 3, 4])
@pytest.mark.parametrize("storage", ["F64", "F32", "F16"])
def test_split_2d_bit_identical(case, parts, storage):
    shape, periodic, obst = CASES_2D[case]
    solid = W.random_solid(shape, seed=7 + case, frac=0.08) if obst else None
    rho0, u0 = W.random_near_equilibrium("D2Q9", shape, seed=11 + case, du=0.02)
    whole, split = _pair(parts, "D2Q9", "SMRT", shape, TAU_G, storage, periodic, g=_g(2), solid=solid,
                         rho0=rho0, u0=u0)
    whole.step(100)
    split.step(100)
    a, sa = whole.state()
    b, sb = split.state()
    assert sa == sb == 100
    assert np.array_equal(a, b), np.mean(a != b)
    ra, ua, ta = whole.moments()
    rb, ub, tb = split.moments()
    assert np.array_equal(ua, ub) and np.array_equal(ra, rb)
    whole.close()
    split.close()


CASES_3D = [
    ((40, 9, 12), (1, 0, 0), True),      # walls in y and z, obstacles
    ((32, 6, 8), (1, 1, 1), False),      # periodic: the exchange wraps in z
]


@pytest.mark.parametrize("lat", ["D3Q19", "D3Q27"])
@pytest.mark.parametrize("case", range(len(CASES_3D)))
@pytest.mark.parametrize("parts", [2, 4])
@pytest.mark.parametrize("storage", ["F64", "F32"])
def test_split_3d_bit_identical(lat, case, parts, storage):
    shape, periodic, obst = CASES_3D[case]
    solid = W.random_solid(shape, seed=17 + case, frac=0.06) if obst else None
    rho0, u0 = W.random_near_equilibrium(lat, shape, seed=19 + case, du=0.02)
    whole, split = _pair(parts, lat, "SMRT", shape, TAU, storage, periodic, g=_g(3), solid=solid,
                         rho0=rho0, u0=u0)
    whole.step(100)
    split.step(100)
    assert np.array_equal(whole.state()[0], split.state()[0])
    whole.close()
    split.close()


@pytest.mark.parametrize("kind", ["rows", "field"])
@pytest.mark.parametrize("layout", ["vector", "strided"])
def test_split_force_kinds_and_layouts(kind, layout):
    """Per-row and per-node forces are sliced with the slabs (halo rows
    included); both kernel layouts."""
    import paper_2212_07494_gb300 as P
    shape = (128, 30, 1)
    nx, ny, _ = shape
    if kind == "rows":
        g = np.zeros((ny, 2))
        g[:, 0] = 1e-5 * np.sin(2 * np.pi * np.arange(ny) / ny)
    else:
        g = 1e-5 * W.SplitMix64(3).normal(2 * nx * ny).reshape(2, 1, ny, nx)
    rho0, u0 = W.random_near_equilibrium("D2Q9", shape, seed=23, du=0.02)
    whole, split = _pair(3, "D2Q9", "MRT_RAW", shape, TAU_G, "F32", (1, 1, 1), g=g, force_kind=kind,
                         rho0=rho0, u0=u0)
    lo, hi = P.lbm_launch_widths("D2Q9", "F32")
    # other shapes on the two sides: a node rounds alike alone or paired
    if layout == "vector":
        whole.set_launch(32, hi, "vector")
        split.set_launch(64, lo, "vector")
    else:
        whole.set_launch(64, 2, "strided")
        split.set_launch(128, 1, "strided")
    whole.step(100)
    split.step(100)
    assert np.array_equal(whole.state()[0], split.state()[0])
    whole.close()
    split.close()


def test_split_check_is_the_sum_of_the_slabs():
    """The all-reduce of the slabs' FP64 checks against the whole domain's
    check: mass, momentum and the residual terms to rounding (the two add
    the same node values in a different order)."""
    import torch
    shape = (150, 37, 1)
    rho0, u0 = W.random_near_equilibrium("D2Q9", shape, seed=29, du=0.02)
    whole, split = _pair(4, "D2Q9", "SMRT", shape, TAU_G, "F64", (1, 0, 1), g=_g(2), rho0=rho0, u0=u0)
    a = torch.zeros(7, dtype=torch.float64, device="cuda")
    b = torch.zeros(7, dtype=torch.float64, device="cuda")
    for _ in range(2):
        whole.step(30)
        split.step(30)
        whole.check_device(a.data_ptr())
        split.check_device(b.data_ptr())
        torch.cuda.synchronize()
        np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=1e-12, atol=1e-18)
    whole.close()
    split.close()
