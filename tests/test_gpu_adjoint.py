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
    rng = np.random.default_rng(2)
    v, w, vb = rng.standard_normal(u.shape), rng.standard_normal(u.shape), rng.standard_normal(b.shape)
    v[0] *= 1e-2
    s = solver(crk, N, Ex, Ey, b)
    dt = 0.4 * s.compute_dt(to_dev(u))

    def S(uu, bb):
        s.set_coefficients(to_dev(bb))
        x = to_dev(uu)
        s.step(x, dt, 1)
        return to_host(x)
    eps = 1e-6
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
    # target: the final surface of a run over a second seeded bathymetry
    _, b2, _, _ = case(N, E, E, L, flow=0.0, seed=7)
    s = solver(crk, N, E, E, b2, L)
    dt = 0.5 * s.compute_dt(to_dev(np.stack([eta0 - b2, 0 * b2, 0 * b2])))
    eta0_d = to_dev(eta0)
    W = quadrature_weights(s)
    with torch.no_grad():
        uT2 = BathymetryToState.apply(to_dev(b2), s, eta0_d, dt, nsteps, every)
        target = uT2[0] + to_dev(b2)

    def J(bb):
        with torch.no_grad():
            uT = BathymetryToState.apply(bb, s, eta0_d, dt, nsteps, every)
            return float(surface_misfit(uT, bb, target, W))
    bt = to_dev(b).requires_grad_(True)
    uT = BathymetryToState.apply(bt, s, eta0_d, dt, nsteps, every)
    surface_misfit(uT, bt, target, W).backward()
    grad = to_host(bt.grad)
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(ndir):
        d = rng.standard_normal(b.shape) * 0.01
        eps = 1e-4
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
    random directions."""
    crk = load()
    assert _gradient_check(crk, 3, 256, 200, 20, 32) < 1e-6
