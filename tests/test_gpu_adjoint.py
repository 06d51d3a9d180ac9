"""The hand-written adjoint of the 2D step (crkfr_step_adjoint): against the
oracle's exact discrete adjoint (torch autograd through the oracle step),
the dot-product identity with central differences of the GPU step, and the
full checkpointed gradient of a final-time surface misfit against central
finite differences in seeded random directions."""
import numpy as np
import pytest
import torch

from gpu_common import G, golden_cfl, load, positions_2d, rel_l2, to_dev, to_host
from oracle.basis import Basis
from oracle.crkfr import Scheme2D
from oracle.systems import ShallowWater2D
from paper_2512_08611_gb300.workloads import SWE2DInput, accept_seed

pytestmark = pytest.mark.gpu


def case(N, Ex, Ey, L=100.0, flow=0.05, seed=0):
    bs = Basis(N)
    x, y, dx, dy = positions_2d(bs, Ex, Ey, L)
    inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=L, n_gauss=8), (x, y), seed)
    u, b = inp.state(x, y)
    u[1] = flow * u[0] * np.sin(2 * np.pi * y / L)
    u[2] = flow * u[0] * np.cos(2 * np.pi * x / L)
    return u, b, dx, dy


def smooth_direction(rng, x, y, L=100.0, k=4):
    """A seeded smooth field (sum of k periodic Gaussians of width 5..15).
    White-noise perturbations flip the wave-speed maximum at many nearly
    tied faces of a smooth flow, where the step is only piecewise smooth, so
    central differences along them lose several digits."""
    d = np.zeros(np.broadcast(x, y).shape)
    for _ in range(k):
        cx, cy = rng.uniform(0, L, 2)
        w = rng.uniform(5.0, 15.0)
        ddx = np.minimum(np.abs(x - cx) % L, L - np.abs(x - cx) % L)
        ddy = np.minimum(np.abs(y - cy) % L, L - np.abs(y - cy) % L)
        d += rng.standard_normal() * np.exp(-(ddx ** 2 + ddy ** 2) / (2 * w * w))
    return d


def solver(crk, N, Ex, Ey, b, L=100.0):
    s = crk.Solver("swe2d", N, gravity=G, cfl_number=golden_cfl(N, "gl"))
    s.set_mesh([Ex, Ey], [0.0, 0.0], [L, L])
    s.set_coefficients(to_dev(b))
    return s


@pytest.mark.parametrize("N", [1, 2, 3])
def test_adjoint_step_matches_oracle_vjp(N):
    crk = load()
    Ex, Ey = 5, 4
    u, b, dx, dy = case(N, Ex, Ey)
    rng = np.random.default_rng(1)
    w = rng.standard_normal(u.shape)
    dt = 0.4 * Scheme2D(ShallowWater2D(G), N, dx, dy).compute_dt(u, b, golden_cfl(N, "gl"), 0.5)
    # oracle: autograd of its own step
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy)
    ut = torch.tensor(u, requires_grad=True)
    bt = torch.tensor(b, requires_grad=True)
    out = sch.step(ut, bt, dt)
    (out * torch.tensor(w)).sum().backward()
    s = solver(crk, N, Ex, Ey, b)
    ub0, bb = s.step_adjoint(to_dev(u), to_dev(w), dt)
    assert rel_l2(to_host(ub0), ut.grad.numpy()) < 1e-11
    assert rel_l2(to_host(bb), bt.grad.numpy()) < 1e-10


def test_adjoint_dot_product_identity_with_gpu_step():
    """<(S(u + e v) - S(u - e v)) / 2e, w> = <v, S'^T w> and the same in b."""
    crk = load()
    N, Ex, Ey = 3, 6, 5
    u, b, dx, dy = case(N, Ex, Ey)
    x, y, _, _ = positions_2d(Basis(N), Ex, Ey, 100.0)
    rng = np.random.default_rng(2)
    w = rng.standard_normal(u.shape)
    v = np.stack([0.01 * smooth_direction(rng, x, y), smooth_direction(rng, x, y),
                  smooth_direction(rng, x, y)])
    vb = 0.01 * smooth_direction(rng, x, y)
    s = solver(crk, N, Ex, Ey, b)
    dt = 0.4 * s.compute_dt(to_dev(u))

    def S(uu, bb):
        s.set_coefficients(to_dev(bb))
        x = to_dev(uu)
        s.step(x, dt, 1)
        return to_host(x)
    eps = 1e-4
    lhs_u = np.sum((S(u + eps * v, b) - S(u - eps * v, b)) / (2 * eps) * w)
    lhs_b = np.sum((S(u, b + eps * vb) - S(u, b - eps * vb)) / (2 * eps) * w)
    s.set_coefficients(to_dev(b))
    ub0, bb = s.step_adjoint(to_dev(u), to_dev(w), dt)
    assert np.sum(v * to_host(ub0)) == pytest.approx(lhs_u, rel=1e-7)
    assert np.sum(vb * to_host(bb)) == pytest.approx(lhs_b, rel=1e-7)


def _gradient_check(crk, N, E, nsteps, every, ndir, L=100.0):
    from paper_2512_08611_gb300.adjoint import (BathymetryToState, quadrature_weights,
                                                surface_misfit)
    _, b, dx, dy = case(N, E, E, L, flow=0.0)
    bs = Basis(N)
    x, y, _, _ = positions_2d(bs, E, E, L)
    eta0 = 1.0 + 0.01 * SWE2DInput(seed=0, L=L).bump(x, y)
    # target: the final surface of a run from a second seeded surface over a
    # second seeded bathymetry
    _, b2, _, _ = case(N, E, E, L, flow=0.0, seed=7)
    eta2 = 1.0 + 0.01 * SWE2DInput(seed=7, L=L).bump(x, y)
    s = solver(crk, N, E, E, b2, L)
    dt = 0.5 * s.compute_dt(to_dev(np.stack([eta2 - b2, 0 * b2, 0 * b2])))
    eta0_d = to_dev(eta0)
    W = quadrature_weights(s)
    with torch.no_grad():
        uT2 = BathymetryToState.apply(to_dev(b2), s, to_dev(eta2), dt, nsteps, every)
        target = uT2[0] + to_dev(b2)

    def J(bb):
        with torch.no_grad():
            uT = BathymetryToState.apply(bb, s, eta0_d, dt, nsteps, every)
            return float(surface_misfit(uT, bb, target, W))
    bt = to_dev(b).requires_grad_(True)
    uT = BathymetryToState.apply(bt, s, eta0_d, dt, nsteps, every)
    surface_misfit(uT, bt, target, W).backward()
    grad = to_host(bt.grad)
    # Directions: a seeded smooth field plus the gradient direction, both of
    # unit norm, scaled to a maximum of 0.01.  A random direction alone is
    # nearly orthogonal to the gradient of a mesh-sized parameter (|cos| about
    # 0.01 here), which leaves the directional derivative at the level of the
    # difference quotient's own error; with the gradient part it is about
    # 0.7 |grad| |d| and the relative comparison means something.
    rng = np.random.default_rng(3)
    gunit = grad / np.linalg.norm(grad)
    worst = 0.0
    for _ in range(ndir):
        sm = smooth_direction(rng, x, y, L)
        d = sm / np.linalg.norm(sm) + gunit
        d = 0.01 * d / np.abs(d).max()
        eps = 1e-5
        fd = (J(to_dev(b + eps * d)) - J(to_dev(b - eps * d))) / (2 * eps)
        ad = float(np.sum(grad * d))
        worst = max(worst, abs(fd - ad) / abs(fd))
    return worst


def test_gradient_small_mesh_against_finite_differences():
    crk = load()
    assert _gradient_check(crk, 3, 12, 20, 5, 6) < 1e-6


def test_gradient_config5_against_finite_differences():
    """256 x 256 quads, N = 3, 200 steps with checkpoints every 20, J the L2
    misfit of the final surface against a seeded target run, 32 seeded
    directions."""
    crk = load()
    assert _gradient_check(crk, 3, 256, 200, 20, 32) < 1e-6
