"""Pins of the oracle's collision and force term.

* Force term (Sec. II.A, Eq. af and the second-order F(xi)): zeroth moment 0,
  first moment rho g, second moment the symmetrised 2 rho g u.
* BGK (Eq. explict_eq) against Guo's textbook update written out here in
  lattice units, independently of the oracle (Sec. II.B: the scheme reduces to
  Guo et al. at second order).
* SMRT with equal relaxation times equals population BGK with the retained
  equilibrium and force, written here in product form on the tensor-product
  lattices.
* The explicit RCM -> RM relations of Eq. (bbd1): a_p^(1) = F/2 for any tau_1,
  the second- and third-order forms, and the fourth-order recursion that holds
  when d_p^(4) is trimmed (tau_4 = 1).
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O

SQ3 = math.sqrt(3.0)
LATTICES = [O.D2Q9, O.D3Q19, O.D3Q27]


def _force_populations(p, rho, u, g):
    """F_i recovered from the initial state fbar = f_eq - F/2."""
    f_g = O.initial_node(p, rho, u, g)
    f_0 = O.initial_node(p, rho, u, np.zeros_like(g))
    return -2.0 * (f_g - f_0)


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("coll", [O.BGK, O.SMRT])
def test_force_moments(lat, coll):
    D, Q, c, w, _ = O.lattice_tables(lat)
    c = c[:, :D].astype(float)
    p = O.make_params(lat, coll, (4, 4, 4 if D == 3 else 1))
    rng = np.random.default_rng(10)
    for _ in range(5):
        rho = 1.0 + 0.1 * rng.normal()
        u = rng.normal(size=D) * 0.05
        g = rng.normal(size=D) * 1e-3
        F = _force_populations(p, rho, u, g)
        assert abs(F.sum()) < 2e-15                                 # mass
        assert np.abs(F @ c - rho * g).max() < 2e-15                # momentum: rho g dt
        second = np.einsum("i,ia,ib->ab", F, c, c)
        assert np.abs(second - rho * (np.outer(g, u) + np.outer(u, g))).max() < 2e-15


def _guo_bgk(c, w, tau, f, g):
    """Guo, Zheng & Shi (2002) in lattice units, c_s^2 = 1/3."""
    rho = f.sum()
    u = (f @ c + 0.5 * rho * g) / rho
    cu = c @ u
    feq = rho * w * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * u @ u)
    Fi = w * (1 - 0.5 / tau) * ((3 * (c - u) + 9 * cu[:, None] * c) @ (rho * g))
    return f - (f - feq) / tau + Fi


@pytest.mark.parametrize("lat", LATTICES)
def test_bgk_equals_guo(lat):
    D, Q, c, w, _ = O.lattice_tables(lat)
    c = c[:, :D].astype(float)
    rng = np.random.default_rng(11)
    for tau in (0.55, 0.8, 1.7):
        p = O.make_params(lat, O.BGK, (2, 2, 2 if D == 3 else 1), tau=(1, 1, tau, 1, 1))
        f = w * (1 + 0.05 * rng.normal(size=Q))
        g = rng.normal(size=D) * 1e-3
        fp, _ = O.collide_node(p, f, g)
        assert np.abs(fp - _guo_bgk(c, w, tau, f, g)).max() < 2e-15


def _he1(m, x):
    return [np.ones_like(x), x, x * x - 1.0][m]


def _multi(D):
    """Multi-indices m (per-axis order <= 2, total order <= 4)."""
    return [m for m in itertools.product(range(3), repeat=D) if sum(m) <= 4]


def _basis(c):
    """phi_m(xi_i) / prod m_a! for the retained multi-indices, xi = sqrt3 c."""
    xi = SQ3 * c
    out = {}
    for m in _multi(c.shape[1]):
        v = np.ones(len(c))
        for a, ma in enumerate(m):
            v = v * _he1(ma, xi[:, a]) / math.factorial(ma)
        out[m] = v
    return out


def _retained_feq(c, w, rho, u):
    """w_i sum_{|m|<=4, m_a<=2} rho prod_a u_a^{m_a} He_{m_a}(xi_a)/m_a!  (Hermite u)."""
    B = _basis(c)
    uh = SQ3 * u
    return w * sum(rho * np.prod([uh[a] ** ma for a, ma in enumerate(m)]) * B[m] for m in B)


def _retained_force(c, w, rho, u, g):
    """Same expansion with the coefficients rho d/de prod (u + e g)^m at e = 0."""
    B = _basis(c)
    uh, gh = SQ3 * u, SQ3 * g
    out = 0.0
    for m in B:
        coef = 0.0
        for a, ma in enumerate(m):
            if ma:
                coef += ma * uh[a] ** (ma - 1) * gh[a] * np.prod(
                    [uh[b] ** mb for b, mb in enumerate(m) if b != a])
        out = out + rho * coef * B[m]
    return w * out


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q27])
def test_smrt_equal_tau_is_regularised_bgk(lat):
    """With tau_2 = tau_3 = tau_4 = tau the order-by-order relaxation commutes
    with the frame shift, so SMRT is f_eq + (1 - 1/tau)(f - f_eq) + (1 - 1/2tau) F
    with the equilibrium and force expanded on the retained components (here
    written as a sum over multi-indices of products of 1-D Hermite polynomials)."""
    D, Q, c, w, _ = O.lattice_tables(lat)
    c = c[:, :D].astype(float)
    B = _basis(c)
    rng = np.random.default_rng(12)
    for tau in (0.6, 0.9, 1.4):
        p = O.make_params(lat, O.SMRT, (2, 2, 2 if D == 3 else 1), tau=(1, 1, tau, tau, tau))
        # populations inside the retained span: random coefficients per multi-index
        coef = {m: (1.0 if sum(m) == 0 else 0.02 * rng.normal()) for m in B}
        f = w * sum(coef[m] * B[m] for m in B)
        g = rng.normal(size=D) * 1e-3
        rho = f.sum()
        u = (f @ c) / rho + 0.5 * g
        feq = _retained_feq(c, w, rho, u)
        F = _retained_force(c, w, rho, u, g)
        ref = feq + (1 - 1 / tau) * (f - feq) + (1 - 0.5 / tau) * F
        fp, _ = O.collide_node(p, f, g)
        assert np.abs(fp - ref).max() < 2e-15


def _comps(D, n):
    return list(itertools.product(range(D), repeat=n))


def _unpack(v, D, n):
    off = sum(D ** k for k in range(n))
    T = np.zeros([D] * n) if n else np.array(0.0)
    for idx in range(D ** n):
        a = tuple((idx // D ** j) % D for j in range(n))
        if n:
            T[a] = v[off + idx]
        else:
            T = np.array(v[off])
    return T


def _place(vecs, X, n):
    """Sum over the distinct placements of the vectors' product and X in an
    order-n symmetric tensor: positions of the vectors chosen without order."""
    D = len(vecs[0]) if vecs else X.shape[0]
    k = len(vecs)
    out = np.zeros([D] * n)
    for a in itertools.product(range(D), repeat=n):
        s = 0.0
        for S in itertools.combinations(range(n), k):
            rest = tuple(a[j] for j in range(n) if j not in S)
            pv = np.prod([vecs[0][a[j]] for j in S]) if k else 1.0
            s += pv * (X[rest] if rest else float(X))
        out[a] = s
    return out


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q27, O.D3Q19])
def test_bbd1_explicit_relations(lat):
    D, Q, c, w, _ = O.lattice_tables(lat)
    rng = np.random.default_rng(13)
    t1 = rng.uniform(0.6, 2.0)
    t2, t3 = 0.63, 0.91
    p = O.make_params(lat, O.SMRT, (2, 2, 2 if D == 3 else 1), tau=(1, t1, t2, t3, 1.0))
    f = w * (1 + 0.05 * rng.normal(size=Q))
    gL = rng.normal(size=D) * 1e-3
    fp, dbg = O.collide_node(p, f, gL)
    abar, a0, a1, d1, dp, ap = dbg
    rho = f.sum()
    u = (f @ (SQ3 * c[:, :D])) / rho + 0.5 * SQ3 * gL     # Hermite units
    F = rho * SQ3 * gL
    w2, w3 = 1 / t2, 1 / t3
    # first order: a_p^(1) = d_p^(1) = F/2 whatever tau_1 is
    assert np.abs(_unpack(ap, D, 1) - F / 2).max() < 2e-15
    assert np.abs(_unpack(a1, D, 1) + F / 2).max() < 2e-15      # Eq. (half_F)
    # second order: (1 - w2) a_1^(2) + (1 - w2/2) a_F^(2), a_F^(2) = 2 sym(F u)
    A1_2 = _unpack(a1, D, 2)
    aF2 = np.outer(F, u) + np.outer(u, F)
    ref2 = (1 - w2) * A1_2 + (1 - w2 / 2) * aF2
    assert np.abs(_unpack(ap, D, 2) - ref2).max() < 1e-15
    # third order, second line of Eq. (bbd1) at theta = 1 (u_1 = u u):
    #   (1 - w3)(a_1^(3) - 3u a_1^(2) + 3uu a_1^(1)) + 3u a_p^(2) - 3uu a_p^(1)
    A1_1 = _unpack(a1, D, 1)
    A1_3 = _unpack(a1, D, 3)
    Ap1 = _unpack(ap, D, 1)
    Ap2 = _unpack(ap, D, 2)
    d13 = A1_3 - _place([u], A1_2, 3) + _place([u, u], A1_1, 3)
    ref3 = (1 - w3) * d13 + _place([u], Ap2, 3) - _place([u, u], Ap1, 3)
    assert np.abs(_unpack(ap, D, 3) - ref3).max() < 1e-15
    # fourth order with d_p^(4) trimmed (tau_4 = 1):
    #   a_p^(4) = 4u a_p^(3) - 6 u_1 a_p^(2) + 4 (u u_2) a_p^(1)
    Ap3 = _unpack(ap, D, 3)
    ref4 = _place([u], Ap3, 4) - _place([u, u], Ap2, 4) + _place([u, u, u], Ap1, 4)
    assert np.abs(_unpack(ap, D, 4) - ref4).max() < 1e-15
    assert np.abs(_unpack(dp, D, 4)).max() == 0.0


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q19, O.D3Q27])
def test_collision_conserves_mass_and_adds_momentum(lat):
    D, Q, c, w, _ = O.lattice_tables(lat)
    c = c[:, :D].astype(float)
    rng = np.random.default_rng(14)
    for coll, tau in [(O.BGK, (1, 1, 0.7, 1, 1)), (O.SMRT, (1, 1.3, 0.57, 0.8, 1.2)),
                      (O.SMRT_FNEQ, (1, 1.3, 0.57, 0.8, 1.2)), (O.MRT_RAW, (1, 1.3, 0.57, 0.8, 1.2))]:
        p = O.make_params(lat, coll, (2, 2, 2 if D == 3 else 1), tau=tau)
        f = w * (1 + 0.05 * rng.normal(size=Q))
        g = rng.normal(size=D) * 1e-3
        fp, _ = O.collide_node(p, f, g)
        rho = f.sum()
        assert abs(fp.sum() - rho) < 1e-15
        assert np.abs(fp @ c - f @ c - rho * g).max() < 2e-15
