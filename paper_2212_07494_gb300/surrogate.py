"""Warm start of steady force-driven channel flows from a learned surrogate.

The network (the library's U-Net, see include/lbm.h) maps per-node inputs
  x = [solid mask, (tau_2 - 0.875) / 0.325, log10(g_x) + 6]
to the steady fields in units of the plain-channel Poiseuille peak
S = g_x H^2 / (8 nu) (nu = (tau_2 - 1/2) / 3, H = ny):
  y = [(rho - 1) / S, u_x / S, u_y / S].
Training data are steady fields computed by the batched solver; the trained
network's prediction initialises a run (rho0, u0), which then relaxes to the
same residual tolerance as a cold start (rho = 1, u = 0).  The cold start is
the fallback: a warm run that fails (non-finite, or not converged within its
step budget) is rerun cold.

torch supplies device memory only; every operation of the network runs in the
library's kernels.
"""
from __future__ import annotations

import math
import time

import numpy as np

from ._binding import Batch, UNet

TAU_MID, TAU_HALF = 0.875, 0.325


def poiseuille_scale(tau2: float, gx: float, H: int) -> float:
    nu = (tau2 - 0.5) / 3.0
    return gx * H * H / (8.0 * nu)


def features(solid: np.ndarray, tau2: float, gx: float) -> np.ndarray:
    """(H, W, 3) float32 network input for one channel (solid: (H, W) or (1, H, W))."""
    s = np.asarray(solid, np.float32).reshape(solid.shape[-2:])
    x = np.empty(s.shape + (3,), np.float32)
    x[..., 0] = s
    x[..., 1] = (tau2 - TAU_MID) / TAU_HALF
    x[..., 2] = math.log10(gx) + 6.0
    return x


def targets(rho: np.ndarray, u: np.ndarray, tau2: float, gx: float) -> np.ndarray:
    """(H, W, 3) float32 training target from steady rho (1, H, W) and u (2, 1, H, W)."""
    H = rho.shape[-2]
    S = poiseuille_scale(tau2, gx, H)
    t = np.empty(rho.shape[-2:] + (3,), np.float32)
    t[..., 0] = (rho.reshape(rho.shape[-2:]) - 1.0) / S
    t[..., 1] = u[0].reshape(rho.shape[-2:]) / S
    t[..., 2] = u[1].reshape(rho.shape[-2:]) / S
    return t


def fields(y: np.ndarray, solid: np.ndarray, tau2: float, gx: float, use_rho=True):
    """(rho0 (1, H, W), u0 (2, 1, H, W)) from a prediction y (H, W, 3);
    use_rho=False keeps rho0 = 1 and takes only the velocity."""
    H, W = y.shape[:2]
    S = poiseuille_scale(tau2, gx, H)
    fl = 1.0 - np.asarray(solid, np.float64).reshape(H, W)
    rho0 = np.ones((1, H, W))
    if use_rho:
        rho0[0] += S * y[..., 0] * fl
    u0 = np.stack([S * y[..., 1] * fl, S * y[..., 2] * fl])[:, None]
    return rho0, u0


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
ARCH = [(3, 32, 1), (32, 32, 1), (32, 64, 1), (64, 64, 1), (64, 128, 1), (128, 128, 1), (128, 256, 1),
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
    return 3.0 * f - 2.0 * H * W * 9 * 3 * 32


class Surrogate:
    """Train and apply the network on device-resident data."""

    def __init__(self, H, W, batch=8, seed=2212074944):
        import torch
        self.torch = torch
        self.H, self.W, self.batch = H, W, batch
        # the network runs on torch's current stream, so the batches torch
        # gathers (and the memory it recycles) are ordered with its kernels
        self.net = UNet(H, W, batch, torch.cuda.current_stream().cuda_stream)
        self.net.set_params(init_params(ARCH, seed))

    def _dev(self, a):
        return self.torch.as_tensor(np.ascontiguousarray(a), dtype=self.torch.float32, device="cuda")

    def train(self, X, Y, M, epochs=10, lr=1e-3, seconds=None, seed=0):
        """X, Y: (n, H, W, 3); M: (n, H, W) loss weights (1 on fluid nodes).
        Returns per-epoch mean losses and the training wall time."""
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
                self.net.train_step(xb.data_ptr(), yb.data_ptr(), mb.data_ptr(), self.batch, scale, lr, ld.data_ptr())
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
        Y = np.empty(X.shape, np.float32)
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


def warm_start(sur: Surrogate, cases, tol, K, max_steps, use_rho=True):
    """Predict, initialise and run to steady state; cases that fail warm
    (non-finite or not converged) are rerun cold.  Returns (seconds incl.
    inference, steps, status, final fields [(rho, u)], inference seconds,
    number of fallbacks)."""
    t0 = time.perf_counter()
    X = np.stack([features(s, t2, g) for s, t2, g in cases])
    Y = sur.predict(X)
    init = [fields(Y[k], s, t2, g, use_rho) for k, (s, t2, g) in enumerate(cases)]
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
