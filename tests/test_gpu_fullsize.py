"""Parity at the benchmark sizes, in the launch configuration the bench runs,
on sampled outputs.

A node's state after s steps depends only on the nodes within s cells of it
(pull streaming moves one cell per step).  So the FP64 oracle can compute a
sampled node of a 4096^2 or 256^3 run by itself. It runs a periodic patch of
radius R > s + 1 around the node, built from the same seeded inputs, and its
wrap-around only corrupts cells more than s steps away from the centre.  The
GPU run is the full domain. The samples include the domain's edges and
corners, where the GPU's periodic wrap acts.

Tolerance: FP32 arithmetic and storage against FP64 over three steps. The
per-step rounding is a few units of 2^-24 of the deviations, so 1e-5 of the
sample's deviation scale bounds it with a wide margin. A wrong neighbour,
force row or sign is off by the size of the deviations themselves."""
import numpy as np
import pytest

import lbm_workloads as W
import oracle as O

pytestmark = pytest.mark.gpu

STEPS, R = 3, 5


def _samples(n, k, seed, D):
    rng = np.random.default_rng(seed)
    pts = [tuple([0] * D), tuple([n - 1] * D), tuple([0] + [n - 1] * (D - 1))]
    pts += [tuple(int(v) for v in rng.integers(0, n, size=D)) for _ in range(k - len(pts))]
    return pts


@pytest.mark.parametrize("coll", ["SMRT", "SMRT_FNEQ", "MRT_RAW"])
def test_kolmogorov_4096_sampled_nodes(coll):
    """D2Q9 SMRT FP32, 4096 x 4096, per-row force: the bench's workload, also
    with the force's non-equilibrium terms and with the raw-moment MRT."""
    import paper_2212_07494_gb300 as P
    wl = W.kolmogorov(n=4096)
    n = 4096
    lat = P.Lattice("D2Q9", coll, wl.shape, wl.tau, "F32", wl.periodic, g=wl.g, force_kind="rows", u0=wl.u0)
    lat.step(STEPS)
    f = lat.populations()                       # (9, 1, n, n)
    lat.close()
    _, Q, _, w, _ = O.lattice_tables(O.D2Q9)
    worst, scale = 0.0, 0.0
    for x, y in _samples(n, 24, 1, 2):
        rows = np.arange(y - R, y + R + 1) % n
        cols = np.arange(x - R, x + R + 1) % n
        u0 = wl.u0[:, :, rows][:, :, :, cols]
        orc = O.Sim(O.D2Q9, getattr(O, coll), (2 * R + 1, 2 * R + 1, 1), (1, 1, 1), wl.tau, g=wl.g[rows],
                    force_kind="rows", u0=np.ascontiguousarray(u0))
        orc.step(STEPS)
        fo = orc.populations()[:, 0, R, R]
        fg = f[:, 0, y, x]
        worst = max(worst, float(np.abs(fg - fo).max()))
        scale = max(scale, float(np.abs(fo - w).max()))
    print(f"4096^2: max |f_gpu - f_oracle| = {worst:.3e}, deviation scale {scale:.3e}")
    assert worst <= 1e-5 * scale + 1e-12, (worst, scale)


@pytest.mark.parametrize("lattice", ["D3Q27", "D3Q19"])
def test_taylor_green_256_cubed_sampled_nodes(lattice):
    """D3Q27 and D3Q19 SMRT FP32, 256^3 Taylor-Green vortex at Re 1600 plus
    g_x: the precision workload's 3-D cases; rho and u of sampled nodes."""
    import paper_2212_07494_gb300 as P
    wl = W.taylor_green_3d(n=256)
    n = 256
    lat = P.Lattice(lattice, "SMRT", wl.shape, wl.tau, "F32", wl.periodic, g=wl.g, rho0=wl.rho0, u0=wl.u0)
    lat.step(STEPS)
    rho, u, _ = lat.moments()                   # (n, n, n), (3, n, n, n)
    lat.close()
    worst_u = worst_r = 0.0
    for x, y, z in _samples(n, 12, 2, 3):
        idx = [np.arange(c - R, c + R + 1) % n for c in (z, y, x)]
        sl = np.ix_(*idx)
        r0 = wl.rho0[sl]
        u0 = np.stack([wl.u0[a][sl] for a in range(3)])
        orc = O.Sim(getattr(O, lattice), O.SMRT, (2 * R + 1,) * 3, (1, 1, 1), wl.tau, g=wl.g, rho0=r0, u0=u0)
        orc.step(STEPS)
        ro, uo, _ = orc.moments()
        worst_r = max(worst_r, abs(float(rho[z, y, x] - ro[R, R, R])))
        worst_u = max(worst_u, float(np.abs(u[:, z, y, x] - uo[:, R, R, R]).max()))
    print(f"256^3: max |u_gpu - u_oracle| = {worst_u:.3e}, max |rho_gpu - rho_oracle| = {worst_r:.3e}")
    U0 = 0.05
    assert worst_u <= 1e-5 * U0, worst_u
    assert worst_r <= 1e-5 * 3 * U0 * U0, worst_r


@pytest.mark.parametrize("storage", ["F16", "BF16"])
def test_kolmogorov_4096_sampled_nodes_2byte_storage(storage):
    """The bench's --storage F16 / BF16 lines: 4096 x 4096 with 2-byte
    deviations (FP32 arithmetic), sampled nodes against oracle patches that
    round the stored deviations the same way (round to nearest even) after
    each step.  The two sides may round a value differently where FP32 and
    FP64 arithmetic straddle a rounding boundary, so the bar is a few units
    in the last place of the stored deviation (F16 keeps subnormals below
    6.1e-5, where its unit is 2^-24 absolute), and most values equal."""
    import paper_2212_07494_gb300 as P
    wl = W.kolmogorov(n=4096)
    n = 4096
    lat = P.Lattice("D2Q9", "SMRT", wl.shape, wl.tau, storage, wl.periodic, g=wl.g, force_kind="rows", u0=wl.u0)
    lat.step(STEPS)
    f = lat.populations()
    lat.close()
    _, Q, _, w, _ = O.lattice_tables(O.D2Q9)
    mode = O.ROUND_F16 if storage == "F16" else O.ROUND_BF16
    ulp = 2.0 ** -11 if storage == "F16" else 2.0 ** -8
    sub = 2.0 ** -24 if storage == "F16" else 0.0
    dg_all, do_all = [], []
    for x, y in _samples(n, 24, 3, 2):
        rows = np.arange(y - R, y + R + 1) % n
        cols = np.arange(x - R, x + R + 1) % n
        u0 = wl.u0[:, :, rows][:, :, :, cols]
        orc = O.Sim(O.D2Q9, O.SMRT, (2 * R + 1, 2 * R + 1, 1), (1, 1, 1), wl.tau, g=wl.g[rows],
                    force_kind="rows", u0=np.ascontiguousarray(u0), round_mode=mode)
        orc.step(STEPS)
        do_all.append(orc.populations()[:, 0, R, R] - w)
        dg_all.append(f[:, 0, y, x] - w)
    dg, do = np.array(dg_all), np.array(do_all)
    scale = np.abs(do).max()
    bound = 4 * ulp * np.abs(do) + 4 * sub + 64 * 2.0 ** -24 * scale
    assert np.all(np.abs(dg - do) <= bound), np.abs(dg - do).max()
    assert np.mean(dg == do) > 0.9, np.mean(dg == do)


def test_batch_512_channels_sampled():
    """The batched workload at its benchmark size: 512 seeded channels
    (U[32,512] x U[16,256], redrawn under the stability bound) in one
    persistent launch, with the tiles the autotuner picks as the bench does.
    100 steps from rest.  Sampled channels, the three largest, the two
    smallest and three others, against the FP64 oracle run of each channel
    alone."""
    import paper_2212_07494_gb300 as P
    chans = W.batch_channels(n=512)
    spec = [{"shape": (c.nx, c.ny, 1), "tau": (1.0, 1.0, c.tau2, 1.0, 1.0), "periodic": (1, 0, 1),
             "g": [c.gx, 0.0]} for c in chans]
    b = P.Batch(spec, "SMRT", "F32")
    b.autotune(50)                        # leaves every channel at step 0
    steps = 100
    b.step(steps)
    sizes = np.array([c.nx * c.ny for c in chans])
    order = np.argsort(sizes)
    rng = np.random.default_rng(4)
    pick = list(order[-3:]) + list(order[:2]) + [int(i) for i in rng.choice(len(chans), 3, replace=False)]
    _, Q, _, w, _ = O.lattice_tables(O.D2Q9)
    for i in pick:
        c = chans[i]
        fg = b.populations(int(i))
        orc = O.Sim(O.D2Q9, O.SMRT, (c.nx, c.ny, 1), (1, 0, 1), (1.0, 1.0, c.tau2, 1.0, 1.0), g=[c.gx, 0.0])
        orc.step(steps)
        fo = orc.populations()
        scale = np.abs(fo - w[:, None, None, None]).max()
        err = np.abs(fg - fo).max()
        assert scale > 0 and err <= 1e-5 * scale + 1e-12, (i, c.nx, c.ny, err, scale)
    b.close()
