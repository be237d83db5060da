"""Pins of the oracle's SMRT collision, with and without the force's
non-equilibrium contributions (Eq. Frc, third and fourth terms).

The explicit update is the trapezoidal rule in disguise.  With the stored
variable fbar = f - Omega(f)/2 - F(f)/2 (Eq. newf) and the update
fbar_p = fbar + Omega(f) + F(f) (Eq. evolution), the step is
f(t+1) - f(t) = [Omega + F](t)/2 + [Omega + F](t+1)/2.  The test writes that
statement out in population space on its own:
  * central moments d_m = sum_i f_i He_m(xi_i - u) over the product
    multi-indices m, as one matrix M_u;
  * Omega(f) = -M_u^-1 T (M_u f - rho e_0), with T the per-order 1/tau
    (tau = tau_hat - 1/2, the time of the continuous collision);
  * F(f) = M_u^-1 G M_u f, with (G d)_m = sum_a m_a g_a d_{m - e_a}, the
    Hermite coefficients of -g . grad_xi f (Eq. af, in the co-moving frame).
    Without the non-equilibrium contributions G keeps only its first-order
    rows;
  * f is recovered from fbar by one linear solve, since rho and u follow from
    fbar alone (Eq. half_F).
None of the oracle's explicit relations are used: no
(1 - 1/tau) d_1 + (1 - 1/2tau) d_F form, no recovery factor, no symmetric
products or frame-shift code.  A wrong recovery factor, a tau of the wrong
order, a missing fourth-order force term or a mean taken where the paper sums
over placements breaks the equality.  D2Q9 has a complete basis of nine
multi-indices.  On D3Q27 the scheme keeps Hermite orders <= 4, so the result
is projected onto the raw orders <= 4 and the input is drawn from that span.
D3Q19's retained set is not a complete basis; test_oracle_d3q19 pins it at one
relaxation time for every order, the shear-wave test of test_oracle_flows at
unequal ones (its decay rate is the shear viscosity's), and the invariants
below and GPU-vs-oracle parity cover the rest.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O

SQ3 = math.sqrt(3.0)


def _he(k, x):
    return [np.ones_like(x), x, x * x - 1.0, x ** 3 - 3 * x][k]


def _multi(D):
    return list(itertools.product(range(3), repeat=D))


def _moment_matrix(xi, u, mult):
    """rows: He_m(xi_i - u) = prod_a He_{m_a}(xi_ia - u_a)"""
    M = np.ones((len(mult), len(xi)))
    for r, m in enumerate(mult):
        for a, ma in enumerate(m):
            M[r] *= _he(ma, xi[:, a] - u[a])
    return M


def _trapezoidal_step(lat, fbar, gL, tau_hat, fneq, tau_bulk=None):
    D, Q, c, w, _ = O.lattice_tables(lat)
    xi = SQ3 * c[:, :D].astype(float)
    g = SQ3 * np.asarray(gL, float)
    mult = _multi(D)
    order = np.array([sum(m) for m in mult])
    rho = fbar.sum()
    u = (fbar @ xi + 0.5 * rho * g) / rho          # Eq. (half_F), Hermite units
    M = _moment_matrix(xi, u, mult)
    Minv = np.linalg.inv(M)
    T = np.diag([0.0 if n < 2 else 1.0 / (tau_hat[min(n, 4)] - 0.5) for n in order])
    if tau_bulk is not None:
        # second order: traceless part at 1/tau_2, trace part at 1/tau_bulk
        # (Eq. domg with tau_{2,2}, tau_{2,0}); P projects onto the trace part
        diag = [r for r, m in enumerate(mult) if sorted(m)[-1] == 2 and sum(m) == 2]
        P = np.zeros_like(T)
        for r in diag:
            P[r, diag] = 1.0 / D
        two = np.diag((order == 2).astype(float))
        T = T - two / (tau_hat[2] - 0.5) + (two - P) / (tau_hat[2] - 0.5) + P / (tau_bulk - 0.5)
    G = np.zeros((len(mult), len(mult)))
    index = {m: r for r, m in enumerate(mult)}
    for r, m in enumerate(mult):
        if not fneq and order[r] != 1:
            continue
        for a, ma in enumerate(m):
            if ma:
                lower = tuple(mb - (b == a) for b, mb in enumerate(m))
                G[r, index[lower]] += ma * g[a]
    e0 = np.zeros(len(mult))
    e0[index[(0,) * D]] = 1.0
    # fbar = f + T(d - rho e0)/2 - G d/2 in central moments d = M f
    d = np.linalg.solve(np.eye(len(mult)) + 0.5 * T - 0.5 * G, M @ fbar + 0.5 * T @ (rho * e0))
    omega = -Minv @ (T @ (d - rho * e0))
    force = Minv @ (G @ d)
    out = fbar + omega + force
    if D == 3:                                      # keep raw orders <= 4
        R = _moment_matrix(xi, np.zeros(D), mult)
        keep = np.diag([1.0 if n <= 4 else 0.0 for n in order])
        out = np.linalg.inv(R) @ keep @ R @ out
    return out


def _span_state(lat, rng, amp=0.03):
    """fbar = w sum_m a_m He_m(xi)/m! with random a_m on the orders <= 4."""
    D, Q, c, w, _ = O.lattice_tables(lat)
    xi = SQ3 * c[:, :D].astype(float)
    f = np.zeros(Q)
    for m in _multi(D):
        if sum(m) > 4:
            continue
        a = 1.0 if sum(m) == 0 else amp * rng.normal()
        f += a * w * np.prod([_he(ma, xi[:, k]) / math.factorial(ma) for k, ma in enumerate(m)], axis=0)
    return f


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q27])
@pytest.mark.parametrize("coll", [O.SMRT, O.SMRT_FNEQ])
def test_smrt_is_the_trapezoidal_rule(lat, coll):
    D = O.LATTICE_DQ[lat][0]
    rng = np.random.default_rng(40 + lat)
    for taus in [(0.57, 0.83, 1.31), (0.9, 1.0, 1.0), (1.7, 0.61, 0.74)]:
        tau_hat = (1.0, 1.0) + taus
        p = O.make_params(lat, coll, (2, 2, 2 if D == 3 else 1), tau=tau_hat)
        f = _span_state(lat, rng)
        gL = rng.normal(size=D) * 3e-3
        fp, _ = O.collide_node(p, f, gL)
        ref = _trapezoidal_step(lat, f, gL, tau_hat, coll == O.SMRT_FNEQ)
        assert np.abs(fp - ref).max() < 5e-15, (taus, np.abs(fp - ref).max())


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q27])
@pytest.mark.parametrize("coll", [O.SMRT, O.SMRT_FNEQ])
def test_split_bulk_tau_is_the_trapezoidal_rule(lat, coll):
    """Eq. (domg) with the second order split into its traceless (shear,
    tau_2) and trace (bulk, tau_bulk) parts, as the same trapezoidal
    statement with a non-diagonal second-order block."""
    D = O.LATTICE_DQ[lat][0]
    rng = np.random.default_rng(45 + lat)
    for taus, tb in [((0.57, 0.83, 1.31), 1.7), ((0.9, 1.0, 1.0), 0.52), ((1.7, 0.61, 0.74), 0.8)]:
        tau_hat = (1.0, 1.0) + taus
        p = O.make_params(lat, coll, (2, 2, 2 if D == 3 else 1), tau=tau_hat, tau_bulk=tb)
        f = _span_state(lat, rng)
        gL = rng.normal(size=D) * 3e-3
        fp, _ = O.collide_node(p, f, gL)
        ref = _trapezoidal_step(lat, f, gL, tau_hat, coll == O.SMRT_FNEQ, tau_bulk=tb)
        assert np.abs(fp - ref).max() < 5e-15, (taus, tb, np.abs(fp - ref).max())
        plain = _trapezoidal_step(lat, f, gL, tau_hat, coll == O.SMRT_FNEQ)
        assert np.abs(ref - plain).max() > 1e-5


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q27])
def test_noneq_force_terms_are_visible(lat):
    """The two modes differ by the size the extra force terms have (g times a
    non-equilibrium moment), so the previous test tells them apart."""
    D = O.LATTICE_DQ[lat][0]
    rng = np.random.default_rng(50)
    tau_hat = (1.0, 1.0, 0.6, 0.9, 1.2)
    f = _span_state(lat, rng)
    gL = rng.normal(size=D) * 3e-3
    a = _trapezoidal_step(lat, f, gL, tau_hat, True)
    b = _trapezoidal_step(lat, f, gL, tau_hat, False)
    assert np.abs(a - b).max() > 1e-6


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_noneq_force_leaves_orders_up_to_two(lat):
    """d_F^(2) = 2 g d^(1) = 0 and the extra terms start at order three, so
    the post-collision mass, momentum and second moments equal plain SMRT's."""
    D, Q, c, w, _ = O.lattice_tables(lat)
    c = c[:, :D].astype(float)
    rng = np.random.default_rng(51)
    for _ in range(4):
        tau = (1.0, 1.0) + tuple(rng.uniform(0.55, 1.6, size=3))
        f = w * (1 + 0.05 * rng.normal(size=Q))
        gL = rng.normal(size=D) * 3e-3
        shape = (2, 2, 2 if D == 3 else 1)
        fa, _ = O.collide_node(O.make_params(lat, O.SMRT_FNEQ, shape, tau=tau), f, gL)
        fb, _ = O.collide_node(O.make_params(lat, O.SMRT, shape, tau=tau), f, gL)
        assert abs(fa.sum() - fb.sum()) < 1e-15
        assert np.abs(fa @ c - fb @ c).max() < 1e-15
        assert np.abs(np.einsum("i,ia,ib->ab", fa - fb, c, c)).max() < 1e-15
        assert np.abs(fa - fb).max() > 1e-9
