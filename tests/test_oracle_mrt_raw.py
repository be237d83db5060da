"""Pins of the oracle's raw-moment MRT (the appendix's collision model).

The appendix relaxes the raw (not co-moving) non-equilibrium moments order by
order, takes the fourth-order one from a recursion, and keeps the force's
equilibrium part only.  The test restates it without any of the oracle's
formulas:
  * the recursion says that the fourth-order central moment of fbar's
    non-equilibrium part is zero, so the test zeroes the central moments of
    order >= 4 of fbar (central moments as the matrix M_u of
    He_m(xi_i - u));
  * the step is then the trapezoidal rule (Eq. newf with Eq. evolution) with
    the collision diagonal per order in the raw moments M_0 f, the
    equilibrium f_eq = M_u^-1 (rho e_0), and the force's Hermite coefficients
    those of -g . grad_xi f_eq (lowering operator on the raw equilibrium
    moments);
  * f is recovered from fbar by one linear solve.
A wrong sign in the recursion, a missing placement, the force built on the
wrong moments or a tau of the wrong order breaks the equality.  D2Q9 has a
complete basis; on D3Q27 the result is projected onto the raw orders <= 4,
as the scheme keeps.
"""
import math

import numpy as np
import pytest

import oracle as O
from test_oracle_force_noneq import SQ3, _moment_matrix, _multi, _span_state


def _raw_mrt_reference(lat, fbar, gL, tau_hat):
    D, Q, c, w, _ = O.lattice_tables(lat)
    xi = SQ3 * c[:, :D].astype(float)
    g = SQ3 * np.asarray(gL, float)
    mult = _multi(D)
    order = np.array([sum(m) for m in mult])
    index = {m: r for r, m in enumerate(mult)}
    rho = fbar.sum()
    u = (fbar @ xi + 0.5 * rho * g) / rho
    Mu = _moment_matrix(xi, u, mult)
    M0 = _moment_matrix(xi, np.zeros(D), mult)
    e0 = np.zeros(len(mult))
    e0[index[(0,) * D]] = 1.0
    # the recursion: central moments of order >= 4 of fbar set to zero
    d = Mu @ fbar
    d[order >= 4] = 0.0
    fbar_r = np.linalg.solve(Mu, d)
    a0 = M0 @ np.linalg.solve(Mu, rho * e0)        # raw moments of f_eq
    G = np.zeros((len(mult), len(mult)))            # Hermite coefficients of -g . grad_xi
    for r, m in enumerate(mult):
        for a, ma in enumerate(m):
            if ma:
                G[r, index[tuple(mb - (b == a) for b, mb in enumerate(m))]] += ma * g[a]
    aF = G @ a0
    T = np.diag([0.0 if n < 2 else 1.0 / (tau_hat[min(n, 4)] - 0.5) for n in order])
    abar = M0 @ fbar_r
    # abar = a + T (a - a0)/2 - aF/2  ->  a (raw moments of f)
    a = np.linalg.solve(np.eye(len(mult)) + 0.5 * T, abar + 0.5 * T @ a0 + 0.5 * aF)
    ap = abar - T @ (a - a0) + aF
    if D == 3:
        ap[order > 4] = 0.0
    return np.linalg.solve(M0, ap)


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q27])
def test_raw_mrt_is_the_regularised_trapezoidal_rule(lat):
    D = O.LATTICE_DQ[lat][0]
    rng = np.random.default_rng(60 + lat)
    for taus in [(0.57, 0.83, 1.31), (0.9, 1.0, 1.0), (1.7, 0.61, 0.74)]:
        tau_hat = (1.0, 1.0) + taus
        p = O.make_params(lat, O.MRT_RAW, (2, 2, 2 if D == 3 else 1), tau=tau_hat)
        f = _span_state(lat, rng)
        gL = rng.normal(size=D) * 3e-3
        fp, _ = O.collide_node(p, f, gL)
        ref = _raw_mrt_reference(lat, f, gL, tau_hat)
        assert np.abs(fp - ref).max() < 5e-15, (taus, np.abs(fp - ref).max())


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_raw_mrt_equals_smrt_when_its_relaxation_commutes_with_the_shift(lat):
    """With one tau for orders 2 to 4, relaxing raw or central moments is the
    same.  The recursion makes the fourth central moment vanish before the
    collision, and the equilibrium-only force has no fourth central moment, so
    the result is SMRT with that tau for orders 2 and 3 and tau_4 = 1."""
    D, Q, c, w, _ = O.lattice_tables(lat)
    rng = np.random.default_rng(61)
    shape = (2, 2, 2 if D == 3 else 1)
    for tau in (0.58, 0.9, 1.45):
        f = w * (1 + 0.05 * rng.normal(size=Q))
        gL = rng.normal(size=D) * 3e-3
        fa, _ = O.collide_node(O.make_params(lat, O.MRT_RAW, shape, tau=(1, 1, tau, tau, tau)), f, gL)
        fb, _ = O.collide_node(O.make_params(lat, O.SMRT, shape, tau=(1, 1, tau, tau, 1.0)), f, gL)
        assert np.abs(fa - fb).max() < 2e-15


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_raw_mrt_differs_from_smrt_with_split_taus(lat):
    D, Q, c, w, _ = O.lattice_tables(lat)
    rng = np.random.default_rng(62)
    shape = (2, 2, 2 if D == 3 else 1)
    tau = (1, 1, 0.6, 0.8, 1.3)
    f = w * (1 + 0.05 * rng.normal(size=Q))
    gL = rng.normal(size=D) * 3e-3
    fa, _ = O.collide_node(O.make_params(lat, O.MRT_RAW, shape, tau=tau), f, gL)
    fb, _ = O.collide_node(O.make_params(lat, O.SMRT, shape, tau=tau), f, gL)
    assert np.abs(fa - fb).max() > 1e-6
