"""lbm_check_noalloc, the allocation-free FP64 check, against lbm_check_device
on the same states.  It serves callers that may not allocate device memory:
a plug-in that receives device pointers from a host framework, a process
whose device memory a pooling allocator has already reserved, a
fixed-budget loop where cudaMalloc could fail or synchronise the device.
Such a caller holds the state in its own buffer and passes it in.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.  It passes alone in a fresh
process (the first call sets up the device) and after the other tests (only
this file calls lbm_check_noalloc).

All calls on a device share one static snapshot.  A call whose layout
(lattice, storage, sizes) differs from the previous call's clears it first,
so its residual numerator equals its denominator: sum |u - 0|^2 = sum |u|^2.
That is what a fresh handle's lbm_check_device computes on its first call,
so every case below starts with a layout change and needs no ordering.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    ("D2Q9", "SMRT", "F32", (150, 37, 1), (1, 0, 1), [1e-5, -2e-6]),
    ("D3Q27", "BGK", "F64", (70, 9, 7), (1, 1, 0), [2e-6, 1e-6, -3e-6]),
]
TAU = (1.0, 1.0, 0.7, 0.9, 1.0)


def _run_calls(lat, coll, st, shape, periodic, g, calls, seed=5):
    """`calls` pairs of (lbm_check_device on a fresh handle, lbm_check_noalloc
    on a copy of its state), 25 steps apart; returns both sides' outputs."""
    import torch

    import lbm_workloads as W
    import paper_2212_07494_gb300 as P

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    rho0, u0 = W.random_near_equilibrium(lat, shape, seed=seed, du=0.02)
    sim = P.Lattice(lat, coll, shape, TAU, st, periodic, g=g, rho0=rho0, u0=u0, torch_stream=stream)
    desc, keep = P.make_desc(lat, coll, shape, TAU, st, periodic, g=g)
    nbytes = P.lbm_state_bytes(sim.h)
    state = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    ref = torch.zeros(7, dtype=torch.float64, device="cuda")
    new = torch.zeros(7, dtype=torch.float64, device="cuda")
    out = []
    for _ in range(calls):
        sim.step(25)
        buf, _ = sim.state()
        with torch.cuda.stream(stream):
            state.copy_(torch.from_numpy(buf), non_blocking=False)
            sim.check_device(ref.data_ptr())
            P.lbm_check_noalloc(desc, state.data_ptr(), new.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        out.append((ref.cpu().numpy().copy(), new.cpu().numpy().copy()))
    sim.close()
    del keep
    return out


@pytest.mark.parametrize("lat,coll,st,shape,periodic,g", CASES)
def test_check_noalloc_matches_check_device(lat, coll, st, shape, periodic, g):
    """Two calls in a row: the first after a layout change (residual against
    zero), the second against the first's snapshot."""
    out = _run_calls(lat, coll, st, shape, periodic, g, calls=2)
    for k, (r, n) in enumerate(out):
        assert np.all(np.isfinite(n)) and n[6] == 0
        np.testing.assert_allclose(n, r, rtol=1e-12, atol=0)
        assert n[4] > 0 and n[5] > 0
    # first call: the snapshot was cleared, so the numerator is sum |u|^2
    assert out[0][1][4] == out[0][1][5]
    # second call: a real residual against the first call's velocity
    assert out[1][1][4] != out[1][1][5]


def test_layout_change_clears_the_snapshot():
    """F64 then F32 on the same sizes: the F32 call must not read the F64
    call's snapshot bytes as FP32 velocities (halves of doubles, which can be
    huge or NaN); it measures against zero, like a fresh lbm_check_device."""
    shape, periodic, g = (96, 40, 1), (1, 0, 1), [1e-5, 0.0]
    f64 = _run_calls("D2Q9", "SMRT", "F64", shape, periodic, g, calls=2, seed=11)
    f32 = _run_calls("D2Q9", "SMRT", "F32", shape, periodic, g, calls=1, seed=11)
    for r, n in f64 + f32:
        assert np.all(np.isfinite(n)) and n[6] == 0
        np.testing.assert_allclose(n, r, rtol=1e-12, atol=0)
    r, n = f32[0]
    assert n[4] == n[5] and n[4] > 0
