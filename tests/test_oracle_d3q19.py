"""A pin of the oracle's SMRT collision on D3Q19, whose retained set (orders
<= 2 and the six (2,1,0)-type third-order components) is not a complete
basis, so the trapezoidal restatement of test_oracle_force_noneq does not
apply there.

With one relaxation time for every order (tau_1 = tau_2 = tau_3 = tau_4 = tau)
the co-moving relaxation commutes with the frame shift: shifting the
non-equilibrium moments to the co-moving frame, scaling them and shifting
back is the same as scaling the raw ones (the shift is linear and its
inverse is exact on the orders the oracle keeps).  The force's co-moving
coefficient d_F^(1) = rho g shifts to the raw a_F^(n) = n F u^(n-1).  So
  fbar_p = R[ a_0 + (1 - 1/tau) (P(fbar) - a_0) + (1 - 1/(2 tau)) a_F ]
with P the Hermite projection (Eq. dft) and R the reconstruction on the
retained components.  The test writes P, R, a_0 and a_F with its own full
Hermite tensors (Rodrigues' formula, every index tuple) in numpy, and none
of the oracle's code; the retained set is the reading stated above.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O

SQ3 = math.sqrt(3.0)


def _hermite(n, xi):
    """H^(n)(xi) for all index tuples, shape (Q,) + (3,) * n, at theta = 1
    (n <= 3: D3Q19 keeps nothing of order 4)."""
    Q = xi.shape[0]
    d = np.eye(3)
    if n == 0:
        return np.ones(Q)
    if n == 1:
        return xi.copy()
    if n == 2:
        return np.einsum("ia,ib->iab", xi, xi) - d[None]
    if n == 3:
        t = np.einsum("ia,ib,ic->iabc", xi, xi, xi)
        s = (np.einsum("ia,bc->iabc", xi, d) + np.einsum("ib,ac->iabc", xi, d) + np.einsum("ic,ab->iabc", xi, d))
        return t - s
    raise ValueError(n)


def _retained(n, idx):
    """D3Q19: orders <= 2, and order 3 where one axis appears twice and
    another once (the (2,1,0) type)."""
    if n <= 2:
        return True
    if n == 3:
        counts = sorted(np.bincount(np.array(idx), minlength=3))
        return counts == [0, 1, 2]
    return False


def _sym(vecs):
    """Symmetrised outer product of the vectors (mean over placements)."""
    n = len(vecs)
    out = 0.0
    perms = list(itertools.permutations(range(n)))
    for p in perms:
        t = vecs[p[0]]
        for j in p[1:]:
            t = np.multiply.outer(t, vecs[j])
        out = out + t
    return out / len(perms)


def _reference(fbar, gL, tau, c, w):
    xi = SQ3 * c
    g = SQ3 * gL
    rho = fbar.sum()
    u = (fbar @ xi + 0.5 * rho * g) / rho
    F = rho * g
    H = [_hermite(n, xi) for n in range(4)]
    om = 1.0 / tau
    out = np.zeros_like(fbar)
    for n in range(4):
        P = np.tensordot(fbar, H[n], axes=(0, 0))                 # a_bar^(n)
        a0 = rho * (_sym([u] * n) if n else 1.0)                  # rho u^(n)
        aF = 0.0 if n == 0 else n * _sym([F] + [u] * (n - 1))     # n F u^(n-1), symmetrised
        A = a0 + (1 - om) * (P - a0) + (1 - 0.5 * om) * aF
        if n == 0:
            out += w * A
            continue
        for idx in itertools.product(range(3), repeat=n):
            if _retained(n, idx):
                out += w * A[idx] * H[n][(slice(None),) + idx] / math.factorial(n)
    return out


@pytest.mark.parametrize("tau", [0.56, 0.9, 1.6])
def test_d3q19_smrt_equal_tau_is_raw_moment_relaxation(tau):
    D, Q, c, w, _ = O.lattice_tables(O.D3Q19)
    c = c[:, :3].astype(float)
    rng = np.random.default_rng(70)
    p = O.make_params(O.D3Q19, O.SMRT, (2, 2, 2), tau=(tau, tau, tau, tau, tau))
    for _ in range(4):
        f = w * (1 + 0.05 * rng.normal(size=Q))
        gL = rng.normal(size=3) * 3e-3
        fp, _ = O.collide_node(p, f, gL)
        ref = _reference(f, gL, tau, c, w)
        assert np.abs(fp - ref).max() < 5e-15, np.abs(fp - ref).max()

