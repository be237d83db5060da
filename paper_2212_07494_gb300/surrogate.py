"""Warm start of steady force-driven channel flows from a learned surrogate.

The channel is periodic in x with walls in y (height H = ny) and solid
obstacles; it is driven by a uniform body force g_x.  The network (the
library's U-Net, see include/lbm.h; its convolutions wrap around along x like
the channel) sees per-node inputs
  x = [solid mask, (tau_2 - 0.875) / 0.325, log10(g_x) + 6, u_L / S, p_L,
       4 phi, beta, q_L],
where (u_L, p_L) is a lubrication estimate of the steady flow (below) and the
last three are constants over the channel, global quantities a 3x3
convolution stack cannot gather from a 256-wide domain: the solid fraction
phi, the largest blocked fraction of a column beta, and the lubrication flux
relative to the empty channel q_L.  It predicts the steady fields as
corrections to the estimate scaled by factors (a_u, a_p) fitted to the
training fields by least squares (lubrication misjudges round obstacles by a
systematic factor):
  y = [(rho - 1) / P - a_p p_L, u_x / S - a_u u_L / S, u_y / S],
with S = g_x H^2 / (8 nu) the Poiseuille peak of the empty channel
(nu = (tau_2 - 1/2) / 3) and P = 3 g_x W the density scale of a pressure
drop g_x over the channel length W.  Training data are steady fields
computed by the batched solver; the prediction initialises a run (rho0, u0),
which then relaxes to the same residual tolerance as a cold start (rho = 1,
u = 0).  The cold start is the fallback: a warm run that fails (non-finite,
or not converged within its step budget) is rerun cold.

Lubrication estimate: every column x is a set of fluid gaps (runs of fluid
nodes between solid nodes or walls, halfway bounce-back places the wall half
a node beyond the last fluid node).  A gap of height h carries plane
Poiseuille flow under the local driving G(x) = g - dp/dx; summed over its
nodes (midpoints y - a + 1/2 of the cells) the parabola carries the flux
G (2 h^3 + h) / (24 nu).  Mass conservation makes the column flux
Q = G(x) C(x) / (24 nu), C(x) = sum_gaps (2 h^3 + h), the same in every
column, and periodicity makes the mean of dp/dx vanish, so
G(x) / g = (1 / C(x)) / mean_x(1 / C(x)), and
p(x) = g sum_{x' < x} (1 - G(x') / g) up to a constant (zero mean).  This is
exact for the empty channel (G = g, the parabola, no pressure drop).

torch supplies device memory only; every operation of the network runs in the
library's kernels; the features are plain host arithmetic on the inputs.
"""
from __future__ import annotations

import math
import time

import numpy as np

from ._binding import Batch, UNet

TAU_MID, TAU_HALF = 0.875, 0.325
NF = 8   # input channels
# bounds of a prediction in units of S (u) and P (rho - 1): a run never starts
# from a wild extrapolation
U_BOUNDS, V_BOUND, P_BOUND = (-0.5, 1.5), 1.0, 2.0


def poiseuille_scale(tau2: float, gx: float, H: int) -> float:
    nu = (tau2 - 0.5) / 3.0
    return gx * H * H / (8.0 * nu)


def density_scale(gx: float, W: int) -> float:
    return 3.0 * gx * W


def lubrication(solid: np.ndarray, with_flux=False):
    """(u_L / S (H, W), p_L (W,)) of the lubrication estimate for a solid
    mask (H, W) or (1, H, W); p_L = p / (g_x W) with zero mean.  with_flux
    also returns q_L, its flux relative to the empty channel's."""
    s = np.asarray(solid).reshape(np.asarray(solid).shape[-2:]) != 0
    H, W = s.shape
    f = ~s
    start = f & ~np.vstack([np.zeros((1, W), bool), f[:-1]])
    lab = np.cumsum(start, axis=0) * f                       # gap number within the column, 0 on solid
    gid = lab + np.arange(W)[None, :] * (H + 1)               # one id per (column, gap)
    n = W * (H + 1)
    y = np.broadcast_to(np.arange(H)[:, None], (H, W))
    h = np.bincount(gid[f], minlength=n).astype(np.float64)   # gap heights
    a = np.full(n, H, np.int64)
    np.minimum.at(a, gid[f], y[f])                            # first fluid node of each gap
    C = (2.0 * h ** 3 + h).reshape(W, H + 1).sum(axis=1)
    if np.any(C == 0):
        raise ValueError("a column is blocked: the channel carries no flow")
    Gg = (1.0 / C) / np.mean(1.0 / C)
    ag, hg = a[gid], h[gid]
    prof = np.where(f, (y - ag + 0.5) * (ag + hg - 0.5 - y), 0.0)
    u = Gg[None, :] * prof * (4.0 / (H * H))
    dp = 1.0 - Gg
    p = np.cumsum(dp) - 0.5 * dp
    p = (p - p.mean()) / W
    if with_flux:
        return u, p, (1.0 / (2.0 * H ** 3 + H)) / np.mean(1.0 / C)
    return u, p


def features(solid: np.ndarray, tau2: float, gx: float) -> np.ndarray:
    """(H, W, NF) float32 network input for one channel (solid: (H, W) or (1, H, W))."""
    s = np.asarray(solid, np.float32).reshape(np.asarray(solid).shape[-2:])
    u, p, q = lubrication(solid, with_flux=True)
    x = np.empty(s.shape + (NF,), np.float32)
    x[..., 0] = s
    x[..., 1] = (tau2 - TAU_MID) / TAU_HALF
    x[..., 2] = math.log10(gx) + 6.0
    x[..., 3] = u
    x[..., 4] = p[None, :] * (1.0 - s)
    x[..., 5] = 4.0 * s.mean()
    x[..., 6] = s.mean(axis=0).max()
    x[..., 7] = q
    return x


def prior_scale(cases, steady):
    """Least-squares factors (a_u, a_p) with u_x ~ a_u S u_L and
    rho - 1 ~ a_p P p_L over solved cases: cases [(solid, tau2, gx)],
    steady [(rho (1, H, W), u (2, 1, H, W))]."""
    nu = du = np_ = dp = 0.0
    for (solid, t2, g), (rho, u) in zip(cases, steady):
        H, W = rho.shape[-2:]
        S, P = poiseuille_scale(t2, g, H), density_scale(g, W)
        uL, pL = lubrication(solid)
        fl = np.asarray(solid).reshape(H, W) == 0
        a, b = u[0].reshape(H, W)[fl] / S, uL[fl]
        nu += float(a @ b)
        du += float(b @ b)
        c, d = (rho.reshape(H, W) - 1.0)[fl] / P, np.broadcast_to(pL[None, :], (H, W))[fl]
        np_ += float(c @ d)
        dp += float(d @ d)
    return (nu / du if du > 0 else 1.0, np_ / dp if dp > 0 else 1.0)


def targets(rho: np.ndarray, u: np.ndarray, tau2: float, gx: float, solid: np.ndarray,
            alpha=(1.0, 1.0)) -> np.ndarray:
    """(H, W, 3) float32 training target from steady rho (1, H, W) and u
    (2, 1, H, W), relative to the lubrication estimate scaled by alpha =
    (a_u, a_p)."""
    H, W = rho.shape[-2:]
    S, P = poiseuille_scale(tau2, gx, H), density_scale(gx, W)
    uL, pL = lubrication(solid)
    fl = 1.0 - (np.asarray(solid).reshape(H, W) != 0)
    t = np.empty((H, W, 3), np.float32)
    t[..., 0] = ((rho.reshape(H, W) - 1.0) / P - alpha[1] * pL[None, :]) * fl
    t[..., 1] = (u[0].reshape(H, W) / S - alpha[0] * uL) * fl
    t[..., 2] = u[1].reshape(H, W) / S * fl
    return t


def fields(y: np.ndarray, solid: np.ndarray, tau2: float, gx: float, use_rho=True, alpha=(1.0, 1.0)):
    """(rho0 (1, H, W), u0 (2, 1, H, W)) from a prediction y (H, W, 3), the
    inverse of targets (within U_BOUNDS, V_BOUND, P_BOUND); y = 0 gives the
    scaled lubrication estimate itself; use_rho=False keeps rho0 = 1 and
    takes only the velocity."""
    H, W = y.shape[:2]
    S, P = poiseuille_scale(tau2, gx, H), density_scale(gx, W)
    uL, pL = lubrication(solid)
    fl = 1.0 - (np.asarray(solid).reshape(H, W) != 0)
    rho0 = np.ones((1, H, W))
    if use_rho:
        rho0[0] += P * np.clip(y[..., 0] + alpha[1] * pL[None, :], -P_BOUND, P_BOUND) * fl
    ux = np.clip(y[..., 1] + alpha[0] * uL, *U_BOUNDS)
    uy = np.clip(y[..., 2], -V_BOUND, V_BOUND)
    u0 = np.stack([S * ux * fl, S * uy * fl])[:, None]
    return rho0, u0


def mirror(X: np.ndarray, Y: np.ndarray, M: np.ndarray):
    """The channel reflected about its mid-plane y -> H - 1 - y: the inputs
    and the lubrication estimate reflect, u_y changes sign."""
    Yf = Y[:, ::-1].copy()
    Yf[..., 2] *= -1.0
    return X[:, ::-1].copy(), Yf, M[:, ::-1].copy()


def solve(cases, tol, K, max_steps, storage="F32", init=None, stream=None):
    """Run channel cases to steady state in one batched launch.
    cases: list of (solid (1, H, W), tau2, gx); init: optional list of
    (rho0, u0).  Returns (seconds, steps, status, residuals, batch)."""
    spec = []
    for k, (solid, t2, g) in enumerate(cases):
        H, W = solid.shape[-2:]
        ch = {"shape": (W, H, 1), "tau": (1.0, 1.0, t2, 1.0, 1.0), "periodic": (1, 0, 1), "g": [g, 0.0],
              "solid": solid}
        if init is not None:
            ch["rho0"], ch["u0"] = init[k]
        spec.append(ch)
    b = Batch(spec, "SMRT", storage, stream)
    t0 = time.perf_counter()
    status, steps, st, r = b.run_to_steady(tol, K, max_steps)
    return time.perf_counter() - t0, steps, st, r, b


def init_params(n_layers_spec, seed: int) -> np.ndarray:
    """He-normal weights (std sqrt(2 / (9 cin)); sqrt(1 / (9 cin)) for the
    linear head) and zero biases in the canonical layout, from the seeded
    generator of lbm_workloads."""
    import lbm_workloads as W
    rng = W.SplitMix64(seed)
    out = []
    for cin, cout, relu in n_layers_spec:
        std = math.sqrt((2.0 if relu else 1.0) / (9 * cin))
        out.append(rng.normal(9 * cin * cout) * std)
        out.append(np.zeros(cout))
    return np.concatenate(out).astype(np.float32)


# (cin, cout, relu) of the library's layers, in the canonical order
ARCH = [(NF, 32, 1), (32, 32, 1), (32, 64, 1), (64, 64, 1), (64, 128, 1), (128, 128, 1), (128, 256, 1),
        (256, 256, 1), (256, 128, 1), (256, 128, 1), (128, 128, 1), (128, 64, 1), (128, 64, 1), (64, 64, 1),
        (64, 32, 1), (64, 32, 1), (32, 32, 1), (32, 3, 0)]


def train_flops_per_sample(H: int, W: int) -> float:
    """Multiply-adds x 2 of one forward + backward (input and weight
    gradients) pass of one sample (the first layer has no input gradient)."""
    res = [1, 1, 2, 2, 4, 4, 8, 8, 4, 4, 4, 2, 2, 2, 1, 1, 1, 1]  # resolution divisor per layer
    f = 0.0
    for (cin, cout, _), d in zip(ARCH, res):
        px = (H // d) * (W // d)
        f += 2.0 * px * 9 * cin * cout
    return 3.0 * f - 2.0 * H * W * 9 * NF * 32


class Surrogate:
    """Train and apply the network on device-resident data."""

    def __init__(self, H, W, batch=8, seed=2212074944, alpha=(1.0, 1.0)):
        import torch
        self.torch = torch
        self.H, self.W, self.batch = H, W, batch
        self.alpha = tuple(alpha)   # scale of the lubrication estimate the targets are relative to
        # the network runs on torch's current stream, so the batches torch
        # gathers (and the memory it recycles) are ordered with its kernels
        self.net = UNet(H, W, batch, torch.cuda.current_stream().cuda_stream, cin=NF, periodic_x=True)
        self.net.set_params(init_params(ARCH, seed))

    def _dev(self, a):
        return self.torch.as_tensor(np.ascontiguousarray(a), dtype=self.torch.float32, device="cuda")

    def train(self, X, Y, M, epochs=10, lr=1e-3, seconds=None, seed=0, lr_final=0.05):
        """X: (n, H, W, NF), Y: (n, H, W, 3); M: (n, H, W) loss weights (1 on
        fluid nodes).  The learning rate decays from lr to lr * lr_final on a
        cosine over the run (its wall time when seconds is given, else its
        epochs).  Returns per-epoch mean losses, the training wall time and
        the number of steps."""
        torch = self.torch
        Xd, Yd, Md = self._dev(X), self._dev(Y), self._dev(M)
        n = X.shape[0]
        rng = np.random.default_rng(seed)
        losses = []
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        steps = 0
        for ep in range(epochs):
            perm = rng.permutation(n)
            acc = torch.zeros(1, dtype=torch.float64, device="cuda")
            nb = 0
            for s in range(0, n - self.batch + 1, self.batch):
                idx = torch.as_tensor(perm[s:s + self.batch], device="cuda")
                xb, yb, mb = Xd[idx].contiguous(), Yd[idx].contiguous(), Md[idx].contiguous()
                scale = 1.0 / (3.0 * float(M[perm[s:s + self.batch]].sum()))
                frac = ((time.perf_counter() - t0) / seconds if seconds is not None
                        else (ep + s / n) / max(1, epochs))
                lr_t = lr * (lr_final + (1.0 - lr_final) * 0.5 * (1.0 + math.cos(math.pi * min(1.0, frac))))
                self.net.train_step(xb.data_ptr(), yb.data_ptr(), mb.data_ptr(), self.batch, scale, lr_t,
                                    ld.data_ptr())
                acc += ld
                nb += 1
                steps += 1
            torch.cuda.synchronize()
            losses.append(float(acc.item()) / max(1, nb))
            if seconds is not None and time.perf_counter() - t0 > seconds:
                break
        torch.cuda.synchronize()
        return losses, time.perf_counter() - t0, steps

    def predict(self, X):
        torch = self.torch
        n = X.shape[0]
        Y = np.empty(X.shape[:3] + (3,), np.float32)
        out = torch.empty((self.batch, self.H, self.W, 3), dtype=torch.float32, device="cuda")
        for s in range(0, n, self.batch):
            k = min(self.batch, n - s)
            xb = self._dev(X[s:s + k])
            self.net.forward(xb.data_ptr(), out.data_ptr(), k)
            torch.cuda.synchronize()
            Y[s:s + k] = out[:k].cpu().numpy()
        return Y

    def loss(self, X, Y, M):
        torch = self.torch
        tot, cnt = 0.0, 0
        for s in range(0, X.shape[0] - self.batch + 1, self.batch):
            xb, yb, mb = (self._dev(a[s:s + self.batch]) for a in (X, Y, M))
            scale = 1.0 / (3.0 * float(M[s:s + self.batch].sum()))
            l, _ = self.net.grad(xb.data_ptr(), yb.data_ptr(), mb.data_ptr(), self.batch, scale, want_grad=False)
            tot += l
            cnt += 1
        return tot / max(1, cnt)

    def close(self):
        self.net.close()


def final_fields(b, n):
    """(rho, u) of every channel of a finished batch."""
    return [b.moments(k) for k in range(n)]


def warm_start(sur, cases, tol, K, max_steps, use_rho=True, alpha=None):
    """Predict, initialise and run to steady state; cases that fail warm
    (non-finite or not converged) are rerun cold.  sur=None starts from the
    lubrication estimate alone (a zero correction) scaled by alpha (default
    the surrogate's, else 1).  Returns (seconds incl. inference, steps,
    status, final fields [(rho, u)], inference seconds, number of
    fallbacks)."""
    t0 = time.perf_counter()
    if alpha is None:
        alpha = sur.alpha if sur is not None else (1.0, 1.0)
    X = np.stack([features(s, t2, g) for s, t2, g in cases])
    Y = sur.predict(X) if sur is not None else np.zeros(X.shape[:3] + (3,), np.float32)
    init = [fields(Y[k], s, t2, g, use_rho, alpha) for k, (s, t2, g) in enumerate(cases)]
    t_inf = time.perf_counter() - t0
    secs, steps, st, r, b = solve(cases, tol, K, max_steps, init=init)
    out = final_fields(b, len(cases))
    b.close()
    bad = [k for k in range(len(cases)) if st[k] != 0]
    if bad:
        secs2, steps2, st2, r2, b2 = solve([cases[k] for k in bad], tol, K, max_steps)
        for j, k in enumerate(bad):
            steps[k] += steps2[j]
            st[k] = st2[j]
            out[k] = b2.moments(j)
        b2.close()
    return time.perf_counter() - t0, steps, st, out, t_inf, len(bad)
