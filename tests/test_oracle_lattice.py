"""Pins of the oracle's lattice tables, Hermite polynomials, discrete transform
and frame shifts against facts independent of the oracle's code.

Sec. II.A of the paper: Gauss-Hermite quadrature (w_i, xi_i), the tensor
Hermite polynomials from the Rodrigues formula and the discrete transform of
Eq. (dft).  Sec. II.C / Eq. (bbd1): moments in the frame moving with the fluid.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O

LATTICES = [O.D2Q9, O.D3Q19, O.D3Q27]
SQ3 = math.sqrt(3.0)


def _iso(D, order):
    """Isotropic tensor of the lattice-unit quadrature moments (c_s^2 = 1/3)."""
    idx = list(itertools.product(range(D), repeat=order))
    T = np.zeros([D] * order)
    for a in idx:
        if order == 2:
            T[a] = (a[0] == a[1]) / 3.0
        elif order == 4:
            d = lambda i, j: float(a[i] == a[j])
            T[a] = (d(0, 1) * d(2, 3) + d(0, 2) * d(1, 3) + d(0, 3) * d(1, 2)) / 9.0
    return T


@pytest.mark.parametrize("lat", LATTICES)
def test_quadrature_moments(lat):
    D, Q, c, w, opp = O.lattice_tables(lat)
    c = c[:, :D].astype(float)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.all(w > 0)
    for order in range(1, 6):
        M = np.zeros([D] * order)
        for i in range(Q):
            t = w[i]
            for _ in range(order):
                t = np.multiply.outer(t, c[i])
            M = M + t
        if order % 2:
            assert np.abs(M).max() < 1e-16, order
        else:
            assert np.abs(M - _iso(D, order)).max() < 1e-15 if order in (2, 4) else True
    # opposite directions
    for i in range(Q):
        assert np.all(c[opp[i]] == -c[i])
    assert c[0].tolist() == [0.0] * D


def _he(m, x):
    """Probabilists' Hermite polynomials He_0..He_4 (one dimension)."""
    return [1.0, x, x * x - 1.0, x ** 3 - 3 * x, x ** 4 - 6 * x * x + 3.0][m]


@pytest.mark.parametrize("D", [2, 3])
def test_hermite_tensor_equals_product_of_1d(D):
    """Each component of H^(n) with axis multiplicities (m_x, m_y, m_z) equals
    prod_a He_{m_a}(x_a) (the weight factorises, so the Rodrigues formula does)."""
    rng = np.random.default_rng(1)
    for _ in range(5):
        x = rng.normal(size=D) * 1.7
        H = O.hermite_at(D, x)
        o = 0
        for n in range(5):
            for idx in range(D ** n):
                a = [(idx // D ** j) % D for j in range(n)]
                m = [a.count(k) for k in range(D)]
                ref = np.prod([_he(m[k], x[k]) for k in range(D)])
                assert abs(H[o] - ref) < 1e-12 * max(1.0, abs(ref)), (n, a)
                o += 1


@pytest.mark.parametrize("lat", [O.D2Q9, O.D3Q27, O.D3Q19])
def test_hermite_orthogonality_on_lattice(lat):
    """sum_i w_i H_m(xi_i) H_m'(xi_i) = delta_mm' prod m_a! for the retained
    components whose product has degree <= 5 (exact quadrature); on D2Q9 and
    D3Q27 (tensor-product rules) every retained pair is orthogonal."""
    D, Q, c, w, _ = O.lattice_tables(lat)
    H, keep, off = O.hermite_table(lat)
    comps = []
    for n in range(5):
        for idx in range(D ** n):
            k = off[n] + idx
            a = tuple(sorted((idx // D ** j) % D for j in range(n)))
            if keep[k] and a not in [x[1] for x in comps]:
                comps.append((k, a, n))
    for (k1, a1, n1), (k2, a2, n2) in itertools.product(comps, comps):
        g = float(np.sum(w * H[:, k1] * H[:, k2]))
        if lat == O.D3Q19 and n1 + n2 > 5:
            continue
        if a1 == a2:
            m = [a1.count(k) for k in range(D)]
            assert abs(g - np.prod([math.factorial(x) for x in m])) < 1e-13
        else:
            assert abs(g) < 1e-13, (a1, a2, g)
    # the retained set has exactly Q independent components on D2Q9, Q minus
    # the 4 components of orders 5, 6 on D3Q27, and orders <= 2 plus the six
    # (2,1,0) third-order components (16) on D3Q19
    expect = {O.D2Q9: 9, O.D3Q19: 16, O.D3Q27: 23}[lat]
    assert len(comps) == expect


def test_transform_round_trip_d2q9():
    """On D2Q9 the nine retained components span the population space, so
    reconstruct(project(f)) = f for any f (Eq. dft)."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        f = rng.normal(size=9)
        a = O.project(O.D2Q9, f)
        assert np.abs(O.reconstruct(O.D2Q9, a) - f).max() < 1e-14


@pytest.mark.parametrize("lat", [O.D3Q27])
def test_transform_idempotent(lat):
    """On D3Q27 the truncation to order <= 4 is an orthogonal projection."""
    rng = np.random.default_rng(3)
    f = rng.normal(size=27)
    p1 = O.reconstruct(lat, O.project(lat, f))
    p2 = O.reconstruct(lat, O.project(lat, p1))
    assert np.abs(p1 - p2).max() < 1e-14
    assert np.abs(p1 - f).max() > 1e-3  # orders 5, 6 really are removed


@pytest.mark.parametrize("lat", LATTICES)
def test_shift_is_projection_in_moving_frame(lat):
    """Shifting the raw moments by -u equals projecting directly onto Hermite
    polynomials of xi - u (the co-moving-frame moments of Sec. II.C at theta 1)."""
    D, Q, c, w, _ = O.lattice_tables(lat)
    rng = np.random.default_rng(4)
    f = rng.normal(size=Q)
    u = rng.normal(size=D) * 0.3
    a = O.project(lat, f)
    d = O.shift(lat, -u, a)
    direct = np.zeros_like(d)
    for i in range(Q):
        h = O.hermite_at(D, SQ3 * c[i, :D] - u)
        direct[: len(h)] += f[i] * h
    n = sum(D ** k for k in range(5))
    assert np.abs(d[:n] - direct[:n]).max() < 1e-12


@pytest.mark.parametrize("lat", LATTICES)
def test_shift_inverse_and_binomial(lat):
    """shift(+u) o shift(-u) = identity; and shift(s, a)^(n) equals the
    symmetrised binomial sum  sum_k C(n,k) sym(s^k (x) a^(n-k))  computed here
    by averaging over all index permutations."""
    D = 2 if lat == O.D2Q9 else 3
    rng = np.random.default_rng(5)
    # random symmetric tensors of orders 0..4, packed
    a = np.zeros(O.PACK)
    full = []
    o = 0
    for n in range(5):
        T = rng.normal(size=[D] * n) if n else np.array(rng.normal())
        if n:
            T = sum(np.transpose(T, p) for p in itertools.permutations(range(n))) / math.factorial(n)
        full.append(T)
        for idx in range(D ** n):
            ai = tuple((idx // D ** j) % D for j in range(n))
            a[o] = T[ai] if n else T
            o += 1
    s = rng.normal(size=D) * 0.4
    out = O.shift(lat, s, a)
    back = O.shift(lat, -s, out)
    assert np.abs(back[:o] - a[:o]).max() < 1e-12
    o = 0
    for n in range(5):
        ref = np.zeros([D] * n) if n else 0.0
        for k in range(n + 1):
            sk = np.array(1.0)
            for _ in range(k):
                sk = np.multiply.outer(sk, s)
            outer = np.multiply.outer(sk, full[n - k])
            if n:
                sym = sum(np.transpose(outer, p) for p in itertools.permutations(range(n))) / math.factorial(n)
            else:
                sym = outer
            ref = ref + math.comb(n, k) * sym
        for idx in range(D ** n):
            ai = tuple((idx // D ** j) % D for j in range(n))
            r = ref[ai] if n else ref
            assert abs(out[o] - r) < 1e-12, (n, ai)
            o += 1
