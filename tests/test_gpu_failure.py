"""Failure detection, injected on the host: a non-finite value in an initial
field is ordinary data to the kernels (nothing faults), and every path that
checks the state must report it.

- a single lattice: lbm_residual and lbm_moments return LBM_ERR_UNSTABLE and
  lbm_check_device counts the non-finite nodes;
- a batch: the poisoned channel ends with LBM_ERR_UNSTABLE while the others
  converge, both when the persistent kernel decides and after the tail
  handoff to plain lattices;
- the learned warm start: a prediction poisoned on the host falls back to a
  cold start, which converges to the cold run's steady state.
"""
import numpy as np
import pytest

import lbm_workloads as W

pytestmark = pytest.mark.gpu

UNSTABLE = -4


@pytest.mark.parametrize("storage", ["F64", "F32", "F16"])
def test_nan_in_initial_velocity_is_reported(storage):
    import torch

    import paper_2212_07494_gb300 as P

    shape = (64, 24, 1)
    rho0, u0 = W.random_near_equilibrium("D2Q9", shape, seed=3, du=0.01)
    u0 = u0.copy()
    u0[0, 0, 7, 11] = np.nan
    # the check before any step sees the poisoned node itself
    lat = P.Lattice("D2Q9", "SMRT", shape, (1, 1, 0.8, 1, 1), storage, (1, 0, 1), g=[1e-6, 0.0],
                    rho0=rho0, u0=u0)
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    lat.check_device(out.data_ptr())
    torch.cuda.synchronize()
    assert out[6].item() >= 1
    with pytest.raises(P.LbmError) as e:
        lat.moments()
    assert e.value.status == UNSTABLE
    # after some steps the NaN has spread; the residual reports it too
    with pytest.raises(P.LbmError) as e:
        lat.residual(20)
    assert e.value.status == UNSTABLE
    lat.close()
    # the same lattice without the NaN is healthy
    ok = P.Lattice("D2Q9", "SMRT", shape, (1, 1, 0.8, 1, 1), storage, (1, 0, 1), g=[1e-6, 0.0],
                   rho0=rho0, u0=np.nan_to_num(u0))
    assert np.isfinite(ok.residual(20))
    ok.close()


@pytest.mark.parametrize("handoff", [0, 8])
def test_batch_channel_with_nan_ends_unstable(handoff):
    import paper_2212_07494_gb300 as P

    spec = []
    for k in range(6):
        nx, ny = 40 + 8 * k, 16 + 2 * k
        ch = {"shape": (nx, ny, 1), "tau": (1.0, 1.0, 0.9, 1.0, 1.0), "periodic": (1, 0, 1), "g": [1e-6, 0.0]}
        if k == 2:
            u0 = np.zeros((2, 1, ny, nx))
            u0[0, 0, ny // 2, nx // 3] = np.nan
            ch["u0"] = u0
        spec.append(ch)
    b = P.Batch(spec, "SMRT", "F32")
    b.set_handoff(handoff)
    status, steps, st, r = b.run_to_steady(1e-7, 200, 400000)
    assert st[2] == UNSTABLE, (status, st)
    assert all(st[k] == 0 for k in range(6) if k != 2), (status, st, r)
    # the poisoned channel stopped at its first check
    assert steps[2] <= 2 * 200 + 1
    for k in range(6):
        if k != 2:
            _, u = b.moments(k)
            assert np.all(np.isfinite(u))
    b.close()


def test_poisoned_prediction_falls_back_to_cold_start():
    import paper_2212_07494_gb300.surrogate as S

    H, Wd = 32, 64
    rng = W.SplitMix64(21)
    cases = []
    for _ in range(4):
        s = int(rng.next_u64(1)[0] & 0x7FFFFFFF)
        cases.append(W.obstacle_channel(s, nx=Wd, ny=H, radius=(3.0, 6.0), ncirc=(1, 1)))

    class Poisoned:
        """A predictor whose outputs are NaN for cases 1 and 3 (a corrupted
        network or input), zero corrections for the others."""
        alpha = (1.0, 1.0)

        def predict(self, X):
            Y = np.zeros(X.shape[:3] + (3,), np.float32)
            Y[1] = np.nan
            Y[3, 5, :, 1] = np.nan   # one row (some of it fluid)
            return Y

    tol, K = 1e-7, 200
    secs, steps, st, out, t_inf, fallbacks = S.warm_start(Poisoned(), cases, tol, K, 400000)
    assert fallbacks == 2
    assert np.all(st == 0)
    cs, csteps, cst, cr, bc = S.solve(cases, tol, K, 400000)
    cold = S.final_fields(bc, len(cases))
    bc.close()
    for k in (1, 3):
        # the fallback is a cold run, after the failed warm attempt: it ends
        # at the cold run's steady state (the two batches tile differently,
        # so agreement is to rounding, not bitwise)
        scale = np.abs(cold[k][1]).max()
        np.testing.assert_allclose(out[k][1], cold[k][1], rtol=0, atol=1e-4 * scale)
        assert steps[k] > csteps[k] - 2 * K
    for k in range(4):
        assert np.all(np.isfinite(out[k][1]))
