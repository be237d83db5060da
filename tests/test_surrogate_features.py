"""Host-side inputs of the learned warm start (paper_2212_07494_gb300.surrogate):
the lubrication estimate of a periodic channel with obstacles, the feature
and target encodings, and the mirror augmentation.  No GPU."""
import numpy as np

import lbm_workloads as W
import paper_2212_07494_gb300.surrogate as S


def test_empty_channel_gives_the_parabola():
    H, Wd = 16, 24
    u, p = S.lubrication(np.zeros((1, H, Wd), np.uint8))
    y = np.arange(H) + 0.5
    assert np.allclose(u, (4.0 * y * (H - y) / H ** 2)[:, None], atol=1e-15)
    assert np.all(p == 0.0)


def test_column_flux_is_constant_and_pressure_periodic():
    solid, t2, g = W.obstacle_channel(7, nx=64, ny=32, radius=(3.0, 8.0), ncirc=(2, 3))
    s = solid[0] != 0
    u, p = S.lubrication(solid)
    assert np.all(u[s] == 0.0) and np.all(u[~s] > 0.0)
    q = u.sum(axis=0)                      # flux of every column
    assert np.ptp(q) < 1e-12 * q.max()
    assert abs(p.mean()) < 1e-15
    # the pressure falls along the flow where the channel narrows: the
    # drop over a column is 1 - G/g, negative where C is below its harmonic mean
    assert p.max() > 0 and p.min() < 0


def test_features_targets_fields_round_trip():
    solid, t2, g = W.obstacle_channel(3, nx=64, ny=32, radius=(3.0, 8.0), ncirc=(1, 2))
    H, Wd = solid.shape[-2:]
    Sv, P = S.poiseuille_scale(t2, g, H), S.density_scale(g, Wd)
    rng = np.random.default_rng(0)
    fl = solid[0] == 0
    # fields within the prediction bounds
    rho = (1.0 + P * np.clip(0.3 * rng.normal(size=(1, H, Wd)), -1.5, 1.5)) * fl + (~fl)
    u = np.stack([Sv * np.clip(0.3 * rng.normal(size=(1, H, Wd)), -0.4, 1.4),
                  Sv * np.clip(0.3 * rng.normal(size=(1, H, Wd)), -0.9, 0.9)]) * fl
    x = S.features(solid, t2, g)
    assert x.shape == (H, Wd, S.NF) and x.dtype == np.float32
    alpha = (0.6, 1.3)
    t = S.targets(rho, u, t2, g, solid, alpha)
    r0, u0 = S.fields(t.astype(np.float64), solid, t2, g, alpha=alpha)
    # targets are float32 in units of S (velocity) and P (density)
    assert np.abs(u0[:, 0][:, fl] - u[:, 0][:, fl]).max() < 8 * 2.0 ** -24 * Sv
    assert np.abs(r0[0][fl] - rho[0][fl]).max() < 8 * 2.0 ** -24 * P
    # a zero correction is the scaled lubrication estimate itself (bounded)
    r1, u1 = S.fields(np.zeros((H, Wd, 3)), solid, t2, g, alpha=alpha)
    uL, pL = S.lubrication(solid)
    assert np.allclose(u1[0, 0], Sv * np.clip(alpha[0] * uL, *S.U_BOUNDS) * fl)
    # wild predictions are bounded
    r2, u2 = S.fields(np.full((H, Wd, 3), 50.0), solid, t2, g)
    assert u2[0].max() <= S.U_BOUNDS[1] * Sv * (1 + 1e-12) and np.abs(u2[1]).max() <= S.V_BOUND * Sv * (1 + 1e-12)


def test_global_channels_and_prior_scale():
    H, Wd = 16, 32
    empty = np.zeros((1, H, Wd), np.uint8)
    x = S.features(empty, 0.8, 1e-6)
    assert np.all(x[..., 5] == 0) and np.all(x[..., 6] == 0)
    assert np.allclose(x[..., 7], 1.0)            # lubrication flux of the empty channel
    solid, t2, g = W.obstacle_channel(9, nx=Wd, ny=H, radius=(2.0, 4.0), ncirc=(1, 2))
    x = S.features(solid, t2, g)
    for c in (5, 6, 7):
        assert np.ptp(x[..., c]) == 0             # constants over the channel
    assert abs(x[0, 0, 5] - 4 * solid.mean()) < 1e-6 and 0 < x[0, 0, 7] < 1
    # prior_scale recovers the factors of fields built from the estimate
    cases, steady = [], []
    for k, (a_u, a_p) in enumerate([(0.6, 1.3)] * 3):
        solid, t2, g = W.obstacle_channel(20 + k, nx=Wd, ny=H, radius=(2.0, 4.0), ncirc=(1, 2))
        uL, pL = S.lubrication(solid)
        fl = solid[0] == 0
        u = np.zeros((2, 1, H, Wd))
        u[0, 0] = a_u * S.poiseuille_scale(t2, g, H) * uL
        rho = (1.0 + a_p * S.density_scale(g, Wd) * pL[None, :] * fl)[None]
        cases.append((solid, t2, g))
        steady.append((rho, u))
    a_u, a_p = S.prior_scale(cases, steady)
    assert abs(a_u - 0.6) < 1e-12 and abs(a_p - 1.3) < 1e-9


def test_mirror_reflects_geometry_and_flips_uy():
    solid, t2, g = W.obstacle_channel(11, nx=32, ny=16, radius=(2.0, 4.0), ncirc=(1, 1))
    X = S.features(solid, t2, g)[None]
    Xm = S.features(solid[:, ::-1], t2, g)[None]
    Y = np.random.default_rng(1).normal(size=(1, 16, 32, 3)).astype(np.float32)
    M = (1.0 - solid[0])[None].astype(np.float32)
    Xf, Yf, Mf = S.mirror(X, Y, M)
    assert np.allclose(Xf, Xm, atol=1e-7)
    assert np.array_equal(Yf[0, :, :, 1], Y[0, ::-1, :, 1])
    assert np.array_equal(Yf[0, :, :, 2], -Y[0, ::-1, :, 2])
    assert np.array_equal(Mf[0], M[0, ::-1])
