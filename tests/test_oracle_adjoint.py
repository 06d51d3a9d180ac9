"""The oracle's discrete adjoint (torch autograd through the unchanged oracle
step, the reference the GPU adjoint is compared with) pinned on CPU against
central differences of the same oracle step, in u and in the bathymetry b:
<w, (S(u + e v) - S(u - e v)) / 2e> = <v, S'^T w>, along smooth seeded
directions (the step is only piecewise smooth: white noise flips the
wave-speed maximum at nearly tied faces)."""
import numpy as np
import pytest
import torch

from oracle.basis import Basis
from oracle.crkfr import Scheme2D
from oracle.systems import ShallowWater2D

G = 9.81


def positions(N, Ex, Ey, L):
    bs = Basis(N)
    dx, dy = L / Ex, L / Ey
    x = (np.arange(Ex)[None, :, None, None] + bs.xi[None, None, None, :]) * dx
    y = (np.arange(Ey)[:, None, None, None] + bs.xi[None, None, :, None]) * dy
    x, y = np.broadcast_arrays(x, y)
    return x, y, dx, dy


def smooth(rng, x, y, L, k=3):
    d = np.zeros(x.shape)
    for _ in range(k):
        cx, cy = rng.uniform(0, L, 2)
        w = rng.uniform(0.15, 0.3) * L
        ddx = np.minimum(np.abs(x - cx) % L, L - np.abs(x - cx) % L)
        ddy = np.minimum(np.abs(y - cy) % L, L - np.abs(y - cy) % L)
        d += rng.standard_normal() * np.exp(-(ddx ** 2 + ddy ** 2) / (2 * w * w))
    return d


@pytest.mark.parametrize("N", [1, 2, 3])
def test_oracle_vjp_against_central_differences(N):
    L, Ex, Ey = 1.0, 4, 3
    x, y, dx, dy = positions(N, Ex, Ey, L)
    b = 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    u = np.stack([1.0 - b + 0.05 * np.sin(2 * np.pi * (x + y)),
                  0.1 * np.cos(2 * np.pi * y), 0.1 * np.sin(2 * np.pi * x)])
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy)
    dt = 0.5 * sch.compute_dt(u, b, 0.1, 0.5)
    rng = np.random.default_rng(N)
    w = np.stack([smooth(rng, x, y, L) for _ in range(3)])
    ut = torch.tensor(u, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)
    (sch.step(ut, bt, dt) * torch.tensor(w)).sum().backward()
    gu, gb = ut.grad.numpy(), bt.grad.numpy()
    eps = 1e-6
    v = np.stack([smooth(rng, x, y, L) for _ in range(3)])
    fd = np.sum(w * (sch.step(u + eps * v, b, dt) - sch.step(u - eps * v, b, dt))) / (2 * eps)
    assert fd == pytest.approx(np.sum(v * gu), rel=1e-7)
    vb = smooth(rng, x, y, L)
    fdb = np.sum(w * (sch.step(u, b + eps * vb, dt) - sch.step(u, b - eps * vb, dt))) / (2 * eps)
    assert fdb == pytest.approx(np.sum(vb * gb), rel=1e-7)
