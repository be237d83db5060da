"""lbm_check_noalloc, the allocation-free FP64 check for callers that may not
allocate device memory (a caller holding the state in its own buffer, with
no cudaMalloc allowed), against lbm_check_device on the same states.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.  It passes alone in a fresh
process (the first call sets up the device) and after the other tests (no
other test touches the shared static scratch).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [
    ("D2Q9", "SMRT", "F32", (150, 37, 1), (1, 0, 1), [1e-5, -2e-6]),
    ("D3Q27", "BGK", "F64", (70, 9, 7), (1, 1, 0), [2e-6, 1e-6, -3e-6]),
]


@pytest.mark.parametrize("lat,coll,st,shape,periodic,g", CASES)
def test_check_noalloc_matches_check_device(lat, coll, st, shape, periodic, g):
    import torch

    import lbm_workloads as W
    import paper_2212_07494_gb300 as P

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    tau = (1.0, 1.0, 0.7, 0.9, 1.0)
    rho0, u0 = W.random_near_equilibrium(lat, shape, seed=5, du=0.02)
    sim = P.Lattice(lat, coll, shape, tau, st, periodic, g=g, rho0=rho0, u0=u0, torch_stream=stream)
    desc, keep = P.make_desc(lat, coll, shape, tau, st, periodic, g=g)
    nbytes = P.lbm_state_bytes(sim.h)
    state = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    ref = torch.zeros(7, dtype=torch.float64, device="cuda")
    new = torch.zeros(7, dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row: the second compares against the first's snapshot
        sim.step(25)
        buf, _ = sim.state()
        with torch.cuda.stream(stream):
            state.copy_(torch.from_numpy(buf), non_blocking=False)
            sim.check_device(ref.data_ptr())
            P.lbm_check_noalloc(desc, state.data_ptr(), new.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        r, n = ref.cpu().numpy(), new.cpu().numpy()
        assert np.all(np.isfinite(n)) and n[6] == 0
        np.testing.assert_allclose(n, r, rtol=1e-12, atol=0)
        assert n[4] > 0 and n[5] > 0
    sim.close()
