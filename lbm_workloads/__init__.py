"""Seeded synthetic inputs for the lattice Boltzmann workloads.

This module is the ONLY code shared by the FP64 oracle side and the CUDA side.
It holds no arithmetic of the method: it draws random numbers (SplitMix64 ->
53-bit uniforms -> Box-Muller normals) and lays out initial fields, force
specifications, obstacle masks and channel parameters for the flows the paper
and its workloads use.  Both sides consume the same arrays.

Units are lattice units throughout (c_s^2 = 1/3, dt = dx = 1).  A "tau" is the
relaxation time tau-hat = tau + 1/2 that appears in the explicit update
(Eq. explict_eq of the paper); the kinematic viscosity is nu = (tau - 1/2)/3.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

D2Q9, D3Q19, D3Q27 = "D2Q9", "D3Q19", "D3Q27"
BGK, SMRT = "BGK", "SMRT"

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), vectorised with numpy."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(1, n + 1, dtype=np.uint64)
            z = self.state + k * _GOLDEN
            self.state = self.state + np.uint64(n) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            return z ^ (z >> np.uint64(31))

    def uniform(self, n: int) -> np.ndarray:
        """n doubles uniform on [0, 1) with 53 random bits each."""
        return (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller on pairs of uniforms."""
        m = (n + 1) // 2
        u = self.uniform(2 * m)
        r = np.sqrt(-2.0 * np.log1p(-u[0::2]))
        t = 2.0 * np.pi * u[1::2]
        out = np.empty(2 * m)
        out[0::2] = r * np.cos(t)
        out[1::2] = r * np.sin(t)
        return out[:n]

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + int(self.uniform(1)[0] * (hi - lo + 1))


@dataclass
class Workload:
    """A flow problem in the layout the C ABI takes (SoA, x fastest)."""
    name: str
    lattice: str
    collision: str
    shape: tuple                       # (nx, ny, nz)
    periodic: tuple                    # per axis, 0 => bounce-back walls
    tau: tuple                         # tau-hat per Hermite order n = 0..4
    force_kind: str = "uniform"        # uniform | rows | field
    g: np.ndarray | None = None        # (D,) | (ny, D) | (D, nz, ny, nx)
    solid: np.ndarray | None = None    # uint8 (nz, ny, nx)
    rho0: np.ndarray | None = None     # (nz, ny, nx)
    u0: np.ndarray | None = None       # (D, nz, ny, nx)
    steps: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def D(self):
        return 2 if self.lattice == D2Q9 else 3

    @property
    def Q(self):
        return {D2Q9: 9, D3Q19: 19, D3Q27: 27}[self.lattice]

    @property
    def nodes(self):
        nx, ny, nz = self.shape
        return nx * ny * nz


def tau_from_nu(nu: float) -> float:
    return 3.0 * nu + 0.5


def poiseuille_channel(nx=64, ny=32, tau=0.8, gx=1e-6, steps=20000) -> Workload:
    """Force-driven channel: periodic in x, halfway bounce-back walls in y,
    rho0 = 1, u0 = 0, uniform g_x (the 64 x 32, tau 0.8, g 1e-6 FP64 case)."""
    return Workload("poiseuille_d2q9_bgk", D2Q9, BGK, (nx, ny, 1), (1, 0, 1),
                    (1.0, 1.0, tau, 1.0, 1.0), "uniform", np.array([gx, 0.0]), steps=steps)


def kolmogorov(n=4096, seed=2212074940, amp=1e-5, noise=1e-4, tau2=0.6, steps=10000,
               collision=SMRT) -> Workload:
    """Fully periodic Kolmogorov flow: g_x(y) = amp sin(2 pi y / n) as a per-row
    table; initial u_x = amp sin(2 pi y / n) plus iid N(0, noise^2) in u_x and
    u_y at every node, rho0 = 1."""
    rng = SplitMix64(seed)
    y = np.arange(n, dtype=np.float64)
    prof = amp * np.sin(2.0 * np.pi * y / n)
    g = np.zeros((n, 2))
    g[:, 0] = prof
    u0 = rng.normal(2 * n * n).reshape(2, 1, n, n) * noise
    u0[0, 0] += prof[:, None]
    return Workload(f"kolmogorov_d2q9_{n}", D2Q9, collision, (n, n, 1), (1, 1, 1),
                    (1.0, 1.0, tau2, 1.0, 1.0), "rows", g, rho0=None, u0=u0, steps=steps,
                    meta={"seed": seed})


def taylor_green_3d(n=256, U0=0.05, Re=1600.0, gx=1e-6, steps=5000, lattice=D3Q27,
                    length="N/2pi") -> Workload:
    """Periodic 3-D Taylor-Green vortex on x = 2 pi i / n with velocity scale U0
    and viscosity from Re on the length n/(2 pi):
      u = U0 sin x cos y cos z,  v = -U0 cos x sin y cos z,  w = 0,
      p = (U0^2/16)(cos 2x + cos 2y)(cos 2z + 2),  rho = 1 + 3 p,
    plus a uniform body force g_x."""
    Lref = n / (2.0 * np.pi) if length == "N/2pi" else float(n)
    nu = U0 * Lref / Re
    s = 2.0 * np.pi * np.arange(n) / n
    z, y, x = np.meshgrid(s, s, s, indexing="ij")
    u = U0 * np.sin(x) * np.cos(y) * np.cos(z)
    v = -U0 * np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p = (U0 * U0 / 16.0) * (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0)
    rho = 1.0 + 3.0 * p
    return Workload(f"tgv3d_{lattice.lower()}_{n}", lattice, SMRT, (n, n, n), (1, 1, 1),
                    (1.0, 1.0, tau_from_nu(nu), 1.0, 1.0), "uniform", np.array([gx, 0.0, 0.0]),
                    rho0=rho, u0=np.stack([u, v, w]), steps=steps, meta={"nu": nu, "U0": U0})


def taylor_green_2d(L: int, u0=0.005, Re=50.0):
    """The paper's forced 2-D Taylor-Green case on an L x L periodic grid with
    nodes at integer positions: returns (tau, T, u_init (2,1,L,L), force(t)),
    force(t) giving the per-node acceleration field (2,1,L,L) at step t.
    The force is rho (u.grad)u of the decaying solution, so it carries the
    factor exp(-2 (k1^2 + k2^2) nu t)."""
    k = 2.0 * np.pi / L
    nu = u0 * L / Re
    x = np.arange(L, dtype=np.float64)[None, :] * np.ones((L, 1))
    y = np.arange(L, dtype=np.float64)[:, None] * np.ones((1, L))
    T = int(round(math.log(2.0) / (2.0 * nu * k * k)))
    uinit = np.stack([-u0 * np.cos(k * x) * np.sin(k * y), u0 * np.sin(k * x) * np.cos(k * y)])[:, None]

    def force(t):
        e = math.exp(-2.0 * (2.0 * k * k) * nu * t)
        return np.stack([-(u0 * u0 / 2.0) * k * np.sin(2 * k * x) * e,
                         -(u0 * u0 / 2.0) * k * np.sin(2 * k * y) * e])[:, None]

    return tau_from_nu(nu), T, uinit, force


@dataclass
class Channel:
    nx: int
    ny: int
    tau2: float
    gx: float
    redraws: int = 0


def batch_channels(n=512, seed=2212074941, nx=(32, 512), ny=(16, 256), tau2=(0.55, 1.5),
                   gx=(1e-7, 1e-5), umax=0.1) -> list:
    """Independent force-driven channels (periodic x, walls in y) with seeded
    uniform sizes and tau_2 and log-uniform g_x.  A draw whose Poiseuille peak
    g H^2 / (8 nu) exceeds umax is redrawn from the same stream."""
    rng = SplitMix64(seed)
    out = []
    lg0, lg1 = math.log(gx[0]), math.log(gx[1])
    for _ in range(n):
        red = 0
        while True:
            cx = rng.randint(*nx)
            cy = rng.randint(*ny)
            t2 = tau2[0] + (tau2[1] - tau2[0]) * rng.uniform(1)[0]
            g = math.exp(lg0 + (lg1 - lg0) * rng.uniform(1)[0])
            nu = (t2 - 0.5) / 3.0
            if g * cy * cy / (8.0 * nu) <= umax:
                break
            red += 1
        out.append(Channel(cx, cy, t2, g, red))
    return out


def obstacle_channel(seed: int, nx=256, ny=128, tau2=(0.55, 1.2), gx=(1e-7, 1e-5),
                     radius=(6.0, 20.0), ncirc=(1, 4), clearance=2.0, umax=0.1, re_max=60.0):
    """256 x 128 channel (periodic x, walls in y) with 1-4 circular obstacles of
    radius U[6, 20], centres uniform with >= clearance cells from the walls and
    from each other (rejection), tau_2 uniform, g_x log-uniform, redrawn while
    the plain-channel Poiseuille peak U = g H^2 / (8 nu) exceeds umax.  Then,
    so that the flow has a steady state (cylinder wakes shed vortices above a
    diameter Reynolds number of about 50), g_x alone is redrawn while
    U (2 r_max) / nu exceeds re_max (re_max=None: no such bound); U
    overestimates the approach velocity past any obstacle.  Returns
    (solid (1,ny,nx) uint8, tau2, gx)."""
    rng = SplitMix64(seed)
    while True:
        t2 = tau2[0] + (tau2[1] - tau2[0]) * rng.uniform(1)[0]
        g = math.exp(math.log(gx[0]) + (math.log(gx[1]) - math.log(gx[0])) * rng.uniform(1)[0])
        if g * ny * ny / (8.0 * (t2 - 0.5) / 3.0) <= umax:
            break
    k = rng.randint(*ncirc)
    circles = []
    tries = 0
    while len(circles) < k and tries < 10000:
        tries += 1
        r = radius[0] + (radius[1] - radius[0]) * rng.uniform(1)[0]
        cx = nx * rng.uniform(1)[0]
        cy = ny * rng.uniform(1)[0]
        if cy - r < clearance - 0.5 or cy + r > ny - 0.5 - clearance:
            continue
        if any(math.hypot(cx - a, cy - b) < r + rb + clearance for a, b, rb in circles):
            continue
        circles.append((cx, cy, r))
    nu = (t2 - 0.5) / 3.0
    rmax = max((c[2] for c in circles), default=0.0)
    while re_max is not None and g * ny * ny / (8.0 * nu) * 2.0 * rmax / nu > re_max:
        g = math.exp(math.log(gx[0]) + (math.log(gx[1]) - math.log(gx[0])) * rng.uniform(1)[0])
        if gx[0] * ny * ny / (8.0 * nu) * 2.0 * rmax / nu > re_max:
            raise ValueError("no g_x in range keeps the flow below re_max")
    yy, xx = np.mgrid[0:ny, 0:nx].astype(np.float64)
    solid = np.zeros((ny, nx), np.uint8)
    for cx, cy, r in circles:
        dx = np.minimum(np.abs(xx - cx), nx - np.abs(xx - cx))  # periodic in x
        solid |= ((dx * dx + (yy - cy) ** 2) <= r * r).astype(np.uint8)
    return solid[None], t2, g


def random_near_equilibrium(lattice: str, shape, seed: int, du=0.02, drho=0.01):
    """Random smooth-free macroscopic fields for parity tests: rho0 = 1 + drho N,
    u0 = du N per component."""
    rng = SplitMix64(seed)
    nx, ny, nz = shape
    D = 2 if lattice == D2Q9 else 3
    rho0 = 1.0 + drho * rng.normal(nx * ny * nz).reshape(nz, ny, nx)
    u0 = du * rng.normal(D * nx * ny * nz).reshape(D, nz, ny, nx)
    return rho0, u0


def random_populations(weights: np.ndarray, shape, seed: int, amp=0.01):
    """Arbitrary populations f_i = w_i (1 + amp N) (non-equilibrium included),
    SoA (Q, nz, ny, nx).  weights: the lattice weights w_i of the population
    order documented in include/lbm.h."""
    rng = SplitMix64(seed)
    nx, ny, nz = shape
    Q = len(weights)
    noise = rng.normal(Q * nx * ny * nz).reshape(Q, nz, ny, nx)
    return np.asarray(weights)[:, None, None, None] * (1.0 + amp * noise)


def random_solid(shape, seed: int, frac=0.1):
    rng = SplitMix64(seed)
    nx, ny, nz = shape
    return (rng.uniform(nx * ny * nz).reshape(nz, ny, nx) < frac).astype(np.uint8)
