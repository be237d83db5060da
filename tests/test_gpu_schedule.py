"""The device-side force schedule (lbm_set_force_schedule): a time-dependent
uniform force that runs inside the captured step graphs.  The oracle is
driven the way the paper's Womersley case is stated, with the force of step
t set before step t (Sec. III.B)."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from helpers import make_pair, rel_l2

pytestmark = pytest.mark.gpu

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_cases.json")))


def _table(A, T):
    t = np.arange(T)
    return np.stack([-A * np.cos(2 * np.pi * t / T), np.zeros(T)], axis=1)


@pytest.mark.parametrize("coll", ["SMRT", "BGK"])
@pytest.mark.parametrize("steps", [1, 63, 200])
def test_schedule_matches_per_step_forcing(coll, steps):
    """200 steps = three 64-step graphs + 8 single launches; 63 = single
    launches only.  Populations to FP64 rounding, then the velocity, which
    uses the force of the current step (Eq. half_F)."""
    A, T, shape = 2e-4, 96, (8, 40, 1)
    tau = (1, 1, 0.8, 1, 1)
    tab = _table(A, T)
    gl, orc = make_pair("D2Q9", coll, shape, tau, "F64", (1, 0, 1), g=[0.0, 0.0])
    gl.set_force_schedule(tab)
    gl.step(steps)
    for t in range(steps):
        orc.set_force(tab[t % T])
        orc.step(1)
    assert np.abs(gl.populations() - orc.populations()).max() < 1e-14
    orc.set_force(tab[steps % T])
    assert rel_l2(gl.moments()[1], orc.moments()[1]) < 1e-12
    gl.close()


def test_schedule_of_period_one_is_the_constant_force():
    shape, tau = (8, 40, 1), (1, 1, 0.8, 1, 1)
    g = np.array([3e-5, -1e-5])
    a, _ = make_pair("D2Q9", "SMRT", shape, tau, "F32", (1, 0, 1), g=g)
    b, _ = make_pair("D2Q9", "SMRT", shape, tau, "F32", (1, 0, 1), g=g)
    b.set_force_schedule(g[None, :])
    a.step(150)
    b.step(150)
    assert np.array_equal(a.populations(), b.populations())


def test_set_force_and_empty_schedule_remove_it():
    shape, tau = (8, 40, 1), (1, 1, 0.8, 1, 1)
    g = np.array([3e-5, 0.0])
    tab = _table(1e-4, 32)
    a, orc = make_pair("D2Q9", "SMRT", shape, tau, "F64", (1, 0, 1), g=g)
    a.set_force_schedule(tab)
    a.step(70)
    for t in range(70):
        orc.set_force(tab[t % 32])
        orc.step(1)
    a.set_force(g)                       # constant force again
    orc.set_force(g)
    a.step(70)
    orc.step(70)
    a.set_force_schedule(tab)
    a.set_force_schedule(None)           # removed: the constant force applies
    a.step(10)
    orc.step(10)
    assert np.abs(a.populations() - orc.populations()).max() < 1e-14


def test_schedule_needs_a_uniform_force():
    import paper_2212_07494_gb300 as P
    shape = (8, 40, 1)
    rows = np.zeros((40, 2))
    gl = P.Lattice("D2Q9", "SMRT", shape, (1, 1, 0.8, 1, 1), "F32", (1, 0, 1), g=rows, force_kind="rows")
    with pytest.raises(P.LbmError) as e:
        gl.set_force_schedule(np.zeros((4, 2)))
    assert e.value.status == -6          # LBM_ERR_STATE
    gl.close()


def test_womersley_on_the_gpu_with_a_schedule():
    """Sec. III.B on the paper's 50 x 200 channel for 20 periods, the force
    from the schedule inside the step graphs.  Against the analytic profile
    (with the start-up transient) at t = 20T + nT/16, as the oracle's own
    test does, and against the oracle's strip run at the end."""
    from test_oracle_flows import _womersley_periodic, _womersley_transient
    import paper_2212_07494_gb300 as P
    cfg = GOLD["womersley"]
    nx, ny, T, nu, A = cfg["nx"], cfg["ny"], cfg["T"], cfg["nu"], cfg["Ap"]
    tau = 3 * nu + 0.5
    om = 2 * math.pi / T
    Lh = ny / 2
    y = np.arange(ny) + 0.5 - Lh
    tab = _table(A, T)
    gl = P.Lattice("D2Q9", "SMRT", (nx, ny, 1), (1, 1, tau, 1, 1), "F64", (1, 0, 1), g=tab[0])
    gl.set_force_schedule(tab)
    t = 0
    worst = 0.0
    for n in range(cfg["periods"] * 16 + 15):
        tgt = n * T // 16
        gl.step(tgt - t)
        t = tgt
        if n >= cfg["periods"] * 16 and (n - cfg["periods"] * 16) in cfg["sample_n"]:
            u = gl.moments()[1]
            assert np.abs(u[0] - u[0][:, :, :1]).max() < 1e-15          # uniform in x
            ua = _womersley_periodic(y, t, A, om, nu, Lh) + _womersley_transient(y, t, A, om, nu, Lh)
            worst = max(worst, np.abs(u[0, 0, :, 0] - ua).max() / (A / om))
    assert worst < 3e-3, worst
    orc = O.Sim(O.D2Q9, O.SMRT, (1, ny, 1), (1, 0, 1), (1, 1, tau, 1, 1), g=[-A, 0.0])
    for s in range(t):
        orc.set_force([-A * math.cos(om * s), 0.0])
        orc.step(1)
    orc.set_force([-A * math.cos(om * t), 0.0])
    assert rel_l2(gl.moments()[1][0, 0, :, 0], orc.moments()[1][0, 0, :, 0]) < 1e-12
    gl.close()


def test_forced_taylor_green_second_order_on_the_gpu():
    """Sec. III.A on the GPU: L = 16, 32, 64, FP64 storage.  The force field
    decays as exp(-2 (k1^2 + k2^2) nu t) (reading C-9); the scale schedule
    applies that factor inside the step graphs.  The E2 error at t = T falls
    at second order, and at L = 16 the run equals the oracle's, whose force
    is set before every step."""
    import lbm_workloads as W
    import paper_2212_07494_gb300 as P
    cfg = GOLD["taylor_green_2d"]
    errs = []
    for L in cfg["L"]:
        tau, T, uinit, force = W.taylor_green_2d(L, cfg["u0"], cfg["Re"])
        k, nu = 2 * np.pi / L, cfg["u0"] * L / cfg["Re"]
        scale = np.exp(-2.0 * (2.0 * k * k) * nu * np.arange(T + 1))
        gl = P.Lattice("D2Q9", "SMRT", (L, L, 1), (1, 1, tau, 1, 1), "F64", (1, 1, 1), g=force(0),
                       force_kind="field", u0=uinit)
        gl.set_force_scale_schedule(scale)
        gl.step(T)
        u = gl.moments()[1]
        gl.close()
        ua = uinit * math.exp(-2 * k * k * nu * T)
        errs.append(math.sqrt(((u - ua) ** 2).sum() / (ua ** 2).sum()))
        if L == cfg["L"][0]:
            orc = O.Sim(O.D2Q9, O.SMRT, (L, L, 1), (1, 1, 1), (1, 1, tau, 1, 1), g=force(0),
                        force_kind="field", u0=uinit)
            for t in range(T):
                orc.set_force(force(t), "field")
                orc.step(1)
            orc.set_force(force(T), "field")
            assert rel_l2(u, orc.moments()[1]) < 1e-12
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    lo, hi = cfg["slope_range"]
    assert all(lo <= s <= hi for s in slopes), (errs, slopes)
