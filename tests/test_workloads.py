"""The seeded input generators (lbm_workloads), which feed both the GPU path
and the oracle and hold none of the method's arithmetic.

* SplitMix64 reproduces the generator's published reference outputs.
* The 512 force-driven channels of the batch workload keep the stability
  rule of their reading (Poiseuille peak g H^2 / (8 nu) <= 0.1, unstable draws
  redrawn from the same stream), stay in their ranges and are reproducible;
  the redraw count is the one the benchmark line records.
* The Kolmogorov inputs have the profile and noise they state.
* The forced Taylor-Green case (Sec. III.A): its force is the convective term
  (u . grad) u of the decaying solution, checked against spectral derivatives
  of the initial field, with the decay factor exp(-2 (k1^2 + k2^2) nu t).
"""
import math

import numpy as np

import lbm_workloads as W


def test_splitmix64_reference_outputs():
    assert [int(v) for v in W.SplitMix64(1234567).next_u64(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431, 16408922859458223821]
    assert int(W.SplitMix64(0).next_u64(1)[0]) == 0xE220A8397B1DCDAF
    # drawing in pieces continues the same stream
    a = W.SplitMix64(99).next_u64(7)
    r = W.SplitMix64(99)
    b = np.concatenate([r.next_u64(3), r.next_u64(4)])
    assert np.array_equal(a, b)
    u = W.SplitMix64(5).uniform(100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 5e-3


def test_batch_channels_keep_the_stability_rule_and_ranges():
    chans = W.batch_channels(512)
    assert len(chans) == 512
    for c in chans:
        nu = (c.tau2 - 0.5) / 3.0
        assert c.gx * c.ny * c.ny / (8.0 * nu) <= 0.1
        assert 32 <= c.nx <= 512 and 16 <= c.ny <= 256
        assert 0.55 <= c.tau2 < 1.5 and 1e-7 <= c.gx < 1e-5
    assert sum(c.redraws for c in chans) == 89
    again = W.batch_channels(512)
    assert all((a.nx, a.ny, a.tau2, a.gx) == (b.nx, b.ny, b.tau2, b.gx) for a, b in zip(chans, again))


def test_kolmogorov_inputs():
    n = 128
    wl = W.kolmogorov(n=n)
    prof = 1e-5 * np.sin(2 * np.pi * np.arange(n) / n)
    assert np.array_equal(wl.g[:, 0], prof) and not wl.g[:, 1].any()
    noise = wl.u0.copy()
    noise[0, 0] -= prof[:, None]
    assert abs(noise.std() / 1e-4 - 1) < 0.02 and abs(noise.mean()) < 3e-6
    assert np.array_equal(W.kolmogorov(n=n).u0, wl.u0)


def test_forced_taylor_green_force_is_the_convective_term():
    L = 32
    tau, T, uinit, force = W.taylor_green_2d(L)
    u, v = uinit[0, 0], uinit[1, 0]
    k = 2 * np.pi / L
    kk = np.fft.fftfreq(L, d=1.0) * 2 * np.pi

    def ddx(f):
        return np.real(np.fft.ifft(1j * kk[None, :] * np.fft.fft(f, axis=1), axis=1))

    def ddy(f):
        return np.real(np.fft.ifft(1j * kk[:, None] * np.fft.fft(f, axis=0), axis=0))

    conv = np.stack([u * ddx(u) + v * ddy(u), u * ddx(v) + v * ddy(v)])
    f0 = force(0)[:, 0]
    assert np.abs(f0 - conv).max() < 1e-15 * L
    assert np.abs(f0).max() > 0
    nu = (tau - 0.5) / 3.0
    t = 17
    assert np.allclose(force(t)[:, 0], f0 * math.exp(-2 * (2 * k * k) * nu * t), rtol=1e-13, atol=0)
    assert T == round(math.log(2) / (2 * nu * k * k))
