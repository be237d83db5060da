"""Batched persistent launch: every channel must evolve exactly as it does on
its own (same kernels' arithmetic), match the FP64 oracle in FP64, stop on
the same residual check as the plain run-to-steady loop, and report a
bounded-wait timeout as an error status without harming the context."""
import numpy as np
import pytest

import lbm_workloads as W
import oracle as O
from helpers import rel_l2

pytestmark = pytest.mark.gpu


def _channels(n, seed, nx=(5, 90), ny=(3, 40)):
    rng = W.SplitMix64(seed)
    out = []
    for _ in range(n):
        cx, cy = rng.randint(*nx), rng.randint(*ny)
        t2 = 0.55 + 0.9 * rng.uniform(1)[0]
        gx = 10 ** (-7 + 2 * rng.uniform(1)[0])
        out.append({"shape": (cx, cy, 1), "tau": (1.0, 1.0, t2, 1.0, 1.0), "periodic": (1, 0, 1), "g": [gx, 0.0]})
    return out


@pytest.mark.parametrize("coll,storage", [("SMRT", "F32"), ("BGK", "F32"), ("SMRT", "F64"), ("SMRT_FNEQ", "F32"),
                                          ("SMRT_FNEQ", "F64"), ("MRT_RAW", "F32"), ("MRT_RAW", "F64")])
def test_batch_matches_single_lattices(coll, storage):
    import paper_2212_07494_gb300 as P
    chans = _channels(12, 7)
    # a channel with initial velocity, to exercise rho0/u0 upload
    rho0, u0 = W.random_near_equilibrium("D2Q9", (33, 17, 1), seed=4, du=0.01)
    chans.append({"shape": (33, 17, 1), "tau": (1, 1, 0.7, 0.9, 1.1), "periodic": (1, 1, 1), "g": [1e-5, -2e-6],
                  "rho0": rho0, "u0": u0})
    b = P.Batch(chans, coll, storage)
    b.set_tiles(128, 256)   # several tiles per step for the larger channels
    b.step(37)
    for i, ch in enumerate(chans):
        s = P.Lattice("D2Q9", coll, ch["shape"], ch["tau"], storage, ch["periodic"], g=ch["g"],
                      rho0=ch.get("rho0"), u0=ch.get("u0"))
        s.step(37)
        fb, fs = b.populations(i), s.populations()
        if storage == "F32":
            # FP32 nodes round alike alone and paired: the same bits
            assert np.array_equal(fb, fs), (i, np.abs(fb - fs).max())
        else:
            assert np.abs(fb - fs).max() <= 1e-15, (i, np.abs(fb - fs).max())
        assert b.info(i)[0] == 37
        s.close()
    b.close()


@pytest.mark.parametrize("storage", ["F32", "F64"])
def test_batch_channels_with_obstacles(storage):
    """Seeded obstacle channels (as the surrogate's data) match single masked
    lattices, and in FP64 the oracle."""
    import paper_2212_07494_gb300 as P
    chans = []
    for k in range(5):
        solid, t2, g = W.obstacle_channel(100 + k, nx=96, ny=48, radius=(3, 8))
        chans.append({"shape": (96, 48, 1), "tau": (1, 1, t2, 1, 1), "periodic": (1, 0, 1), "g": [g, 0.0],
                      "solid": solid})
    chans.append(_channels(1, 1)[0])  # and one without a mask
    b = P.Batch(chans, "SMRT", storage)
    b.set_tiles(128, 512)
    b.step(60)
    for i, ch in enumerate(chans):
        s = P.Lattice("D2Q9", "SMRT", ch["shape"], ch["tau"], storage, ch["periodic"], g=ch["g"],
                      solid=ch.get("solid"))
        s.step(60)
        fb, fs = b.populations(i), s.populations()
        if storage == "F32":
            assert np.array_equal(fb, fs), (i, np.abs(fb - fs).max())
        else:
            assert np.abs(fb - fs).max() <= 1e-15, (i, np.abs(fb - fs).max())
        if storage == "F64" and ch.get("solid") is not None:
            orc = O.Sim(O.D2Q9, O.SMRT, ch["shape"], ch["periodic"], ch["tau"], g=ch["g"], solid=ch["solid"])
            orc.step(60)
            assert rel_l2(b.moments(i)[1], orc.moments()[1]) < 1e-12
        s.close()
    b.close()


def test_batch_channel_matches_oracle_f64():
    import paper_2212_07494_gb300 as P
    chans = _channels(6, 11)
    b = P.Batch(chans, "SMRT", "F64")
    b.step(150)
    for i, ch in enumerate(chans):
        orc = O.Sim(O.D2Q9, O.SMRT, ch["shape"], ch["periodic"], ch["tau"], g=ch["g"])
        orc.step(150)
        _, ub = b.moments(i)
        _, uo, _ = orc.moments()
        assert rel_l2(ub, uo) < 1e-12
    b.close()


def test_run_to_steady_agrees_with_plain_loop():
    """Fast-converging channels (large viscosity, narrow): the batch stops one
    step after the check that meets tol, at the same residual as a plain
    lbm_residual loop on the same channel."""
    import paper_2212_07494_gb300 as P
    chans = [{"shape": (nx, ny, 1), "tau": (1, 1, t, 1, 1), "periodic": (1, 0, 1), "g": [g, 0.0]}
             for nx, ny, t, g in [(40, 12, 1.4, 1e-5), (17, 9, 1.2, 3e-6), (64, 16, 1.5, 1e-6), (8, 5, 0.9, 1e-5)]]
    tol, K = 1e-6, 100
    b = P.Batch(chans, "SMRT", "F32")
    status, steps, st, r = b.run_to_steady(tol, K, max_steps=200000)
    assert status == 0
    assert np.all(st == 0), st
    for i, ch in enumerate(chans):
        s = P.Lattice("D2Q9", "SMRT", ch["shape"], ch["tau"], "F32", ch["periodic"], g=ch["g"])
        n = 0
        while True:
            rr = s.residual(K)
            n += K
            if rr <= tol:
                break
        assert steps[i] == n + 1, (i, steps[i], n)
        assert abs(r[i] - rr) <= 1e-6 * rr, (r[i], rr)
        s.close()
    b.close()


@pytest.mark.parametrize("storage", ["F32", "F64"])
def test_tail_handoff_matches_the_kernel_alone(storage):
    """The tail handed to plain lattices ends where the persistent kernel
    alone ends: the same status and step count for every channel, the
    residual to its summation order, and the final fields: bit for bit in
    FP32 (the batch and a plain lattice round every node alike), to FP64
    rounding in FP64 (the two kernels may contract differently).  Handoff
    1000 hands every channel over after its first step, 8 only the last
    eight, 0 never."""
    import paper_2212_07494_gb300 as P
    chans = _channels(24, 13, nx=(24, 96), ny=(8, 40))
    chans[5]["solid"] = W.random_solid((chans[5]["shape"][0], chans[5]["shape"][1], 1), 3, frac=0.05)
    tol, K = 1e-7, 200
    res = {}
    for ho in (0, 8, 1000):
        b = P.Batch(chans, "SMRT", storage)
        b.set_handoff(ho)
        status, steps, st, r = b.run_to_steady(tol, K, max_steps=400000)
        assert status == 0
        res[ho] = (steps.copy(), st.copy(), r.copy(), [b.moments(i)[1] for i in range(len(chans))])
        b.close()
    assert np.all(res[0][1] == 0), res[0][1]
    for ho in (8, 1000):
        assert np.array_equal(res[ho][1], res[0][1]), (ho, res[ho][1])
        assert np.array_equal(res[ho][0], res[0][0]), (ho, res[ho][0] - res[0][0])
        assert np.allclose(res[ho][2], res[0][2], rtol=1e-6), ho
        for i in range(len(chans)):
            if storage == "F32":
                assert np.array_equal(res[ho][3][i], res[0][3][i]), (ho, i)
            else:
                assert rel_l2(res[ho][3][i], res[0][3][i]) < 1e-10, (ho, i)


def test_run_to_steady_reports_not_converged():
    import paper_2212_07494_gb300 as P
    chans = _channels(5, 3)
    b = P.Batch(chans, "SMRT", "F32")
    status, steps, st, r = b.run_to_steady(1e-30, 50, max_steps=400)
    assert status == 0
    assert np.all(st == P.LBM_NOT_CONVERGED) and np.all(steps == 400)
    b.close()


def test_bounded_scan_times_out_cleanly():
    """With a scan limit of one, CTAs that find no tile to claim give up at
    once: the run returns LBM_ERR_TIMEOUT (no hang, no fault) and the batch
    stays usable."""
    import paper_2212_07494_gb300 as P
    chans = _channels(2, 5, nx=(40, 60), ny=(8, 12))
    b = P.Batch(chans, "SMRT", "F32")
    b.set_handoff(0)   # the kernel alone: the test is about its bounded scan
    b.set_spin_limit(1)
    status, steps, st, r = b.run_to_steady(0.0, 10, max_steps=100000)
    assert status == -5, status
    b.set_spin_limit(1 << 26)
    b.reset()
    b.step(10)
    assert all(b.info(i)[0] == 10 for i in range(len(chans)))
    b.close()


def test_batch_autotune_and_reset():
    import paper_2212_07494_gb300 as P
    chans = _channels(20, 9)
    b = P.Batch(chans, "SMRT", "F32")
    bl, tn, ms = b.autotune(20)
    assert bl in (64, 128, 256) and tn in (1024, 2048, 4096, 8192) and ms > 0
    assert all(b.info(i)[0] == 0 for i in range(len(chans)))
    b.close()
