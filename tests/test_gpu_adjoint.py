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


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_recorded_adjoint_step_equals_the_recomputing_one(N):
    """crkfr_step_record (with and without stepping) writes the face traces
    and stage values the adjoint step would recompute; the recorded adjoint
    step then gives the recomputing one's result, and the recording step the
    plain step's state (ragged 9 x 5 mesh)."""
    crk = load()
    Ex, Ey = 9, 5
    u, b, dx, dy = case(N, Ex, Ey)
    rng = np.random.default_rng(4)
    w = rng.standard_normal(u.shape)
    s = solver(crk, N, Ex, Ey, b)
    dt = 0.4 * s.compute_dt(to_dev(u))
    rec = s.new_records(2)
    s.step_record(to_dev(u), dt, rec[0], advance=False)
    x = to_dev(u)
    s.step_record(x, dt, rec[1], advance=True)
    y = to_dev(u)
    s.step(y, dt, 1)
    assert torch.equal(x, y)
    assert torch.equal(rec[0], rec[1])
    ub0, bb = s.step_adjoint(to_dev(u), to_dev(w), dt)
    rb0, rbb = s.step_adjoint_recorded(to_dev(u), rec[0], to_dev(w), dt)
    assert rel_l2(to_host(rb0), to_host(ub0)) < 1e-14
    assert rel_l2(to_host(rbb), to_host(bb)) < 1e-14
    s.status()


def test_record_arguments_are_checked():
    crk = load()
    N, Ex, Ey = 2, 4, 3
    u, b, dx, dy = case(N, Ex, Ey)
    s = solver(crk, N, Ex, Ey, b)
    n = N + 1
    assert s.record_size() == 14 * n * (2 * Ex * Ey + 2 * Ex) + 3 * 2 * Ex * Ey * n * n
    rec = s.new_records(1)
    with pytest.raises(crk.CrkfrError):
        s.step_record(to_dev(u), 0.0, rec[0])
    with pytest.raises(ValueError):
        s.step_record(to_dev(u), 0.01, rec[0, :-1].contiguous())
    s1 = crk.Solver("swe2d", N, nodes="gll", gravity=G)
    s1.set_mesh([Ex, Ey], [0.0, 0.0], [100.0, 100.0])
    s1.set_coefficients(to_dev(b))
    with pytest.raises(crk.CrkfrError) as e:
        s1.step_record(to_dev(u), 0.01, s1.new_records(1)[0])
    assert e.value.status == -2


@pytest.mark.parametrize("recorded", [True, False])
def test_checkpointed_gradient_matches_oracle_vjp_over_several_steps(recorded):
    """dJ/db of the checkpointed, recorded backward pass (7 steps, checkpoints
    every 3, so segments of 3, 3 and 1 steps) on a 16 x 16, N = 3 mesh equals
    the oracle's exact discrete adjoint of the same 7 steps (torch autograd
    through the oracle), J the surface misfit of adjoint.py."""
    from paper_2512_08611_gb300.adjoint import (BathymetryToState, quadrature_weights,
                                                surface_misfit)
    crk = load()
    N, E, L, nsteps, every = 3, 16, 100.0, 7, 3
    _, b, dx, dy = case(N, E, E, L, flow=0.0)
    x, y, _, _ = positions_2d(Basis(N), E, E, L)
    eta0 = 1.0 + 0.01 * SWE2DInput(seed=0, L=L).bump(x, y) + 0.005 * np.sin(2 * np.pi * x / L)
    rng = np.random.default_rng(9)
    target = 1.0 + 0.002 * rng.standard_normal(b.shape)
    s = solver(crk, N, E, E, b, L)
    dt = 0.5 * s.compute_dt(to_dev(np.stack([eta0 - b, 0 * b, 0 * b])))
    W = quadrature_weights(s)
    bt = to_dev(b).requires_grad_(True)
    uT = BathymetryToState.apply(bt, s, to_dev(eta0), dt, nsteps, every, recorded)
    surface_misfit(uT, bt, to_dev(target), W).backward()
    # oracle
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy)
    bo = torch.tensor(b, requires_grad=True)
    z = torch.zeros_like(bo)
    v = torch.stack([torch.tensor(eta0) - bo, z, z])
    for _ in range(nsteps):
        v = sch.step(v, bo, dt)
    Wo = torch.tensor(to_host(W))
    d = v[0] + bo - torch.tensor(target)
    (0.5 * torch.sum(Wo * d * d)).backward()
    assert rel_l2(to_host(uT.detach()), v.detach().numpy()) < 1e-12
    assert rel_l2(to_host(bt.grad), bo.grad.numpy()) < 1e-10


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
    # Directions: seeded smooth fields (four periodic Gaussians) scaled to a
    # maximum of 0.01, independent of the gradient under test.  A smooth field
    # is nearly orthogonal to the gradient (|cos| 1e-6 .. 2e-3 on these
    # meshes), so the difference quotient must resolve a small directional
    # derivative: with steps eps d of 1e-4 at most, J (about 5e-4 .. 4e-3) is
    # nearly linear in b and the quotient's error is mostly rounding noise,
    # which grows as 1/eps.  Measured relative errors (GB300) at eps = 1e-2:
    # 3e-9 .. 2.4e-7 (12^2, 20 steps), 4e-10 .. 1.1e-8 (256^2, 200 steps); at
    # eps = 1e-5: 1e-6 .. 1e-4.  Each direction's noise floor is measured as
    # the change of the quotient when eps is halved; the tolerance is 1e-6
    # relative plus four times that floor, and the floor must stay below the
    # 1e-6 tolerance for most directions (its median), so that the check
    # keeps its meaning where the directional derivative is not tiny.
    rng = np.random.default_rng(3)
    rows = []
    for _ in range(ndir):
        sm = smooth_direction(rng, x, y, L)
        d = 0.01 * sm / np.abs(sm).max()
        fd = {}
        for eps in (1e-2, 5e-3):
            fd[eps] = (J(to_dev(b + eps * d)) - J(to_dev(b - eps * d))) / (2 * eps)
        ad = float(np.sum(grad * d))
        rows.append((fd[1e-2], abs(fd[1e-2] - fd[5e-3]), ad))
    return rows


def _assert_gradient(rows):
    for fd, noise, ad in rows:
        assert abs(fd - ad) <= 1e-6 * abs(ad) + 4.0 * noise, (fd, noise, ad)
    assert np.median([noise / abs(ad) for _, noise, ad in rows]) < 1e-6, rows


def test_gradient_small_mesh_against_finite_differences():
    crk = load()
    _assert_gradient(_gradient_check(crk, 3, 12, 20, 5, 6))


def test_gradient_config5_against_finite_differences():
    """256 x 256 quads, N = 3, 200 steps with checkpoints every 20, J the L2
    misfit of the final surface against a seeded target run, 32 seeded
    directions."""
    crk = load()
    _assert_gradient(_gradient_check(crk, 3, 256, 200, 20, 32))


def adjoint_slab(crk, N, Ex, Ey, b, first, count, L=100.0):
    dy = L / Ey
    s = crk.Solver("swe2d", N, gravity=G, cfl_number=golden_cfl(N, "gl"))
    s.set_mesh([Ex, count], [0.0, first * dy], [L, (first + count) * dy])
    s.set_subdomain(True)
    rows = [(first - 1) % Ey] + list(range(first, first + count)) + [(first + count) % Ey]
    s.set_coefficients(to_dev(np.ascontiguousarray(b[rows])))
    return s


@pytest.mark.parametrize("N,parts", [(3, [(0, 7), (7, 9)]), (2, [(0, 1), (1, 10), (11, 5)]),
                                     (1, [(0, 16)])])
def test_slab_adjoint_equals_whole_mesh_adjoint(N, parts):
    """The adjoint step on slabs (crkfr_adjoint_local, exchange of the
    forward traces and of ubar1's correction sums, crkfr_adjoint_faces),
    with a one-row slab and a slab that is its own neighbour among the
    cases: ubar0 and the bathymetry gradient of every slab equal the rows
    of crkfr_step_adjoint on the whole mesh bit for bit."""
    crk = load()
    Ex, Ey = 16, 16
    u, b, dx, dy = case(N, Ex, Ey)
    rng = np.random.default_rng(5)
    w = rng.standard_normal(u.shape)
    m = solver(crk, N, Ex, Ey, b)
    dt = 0.5 * m.compute_dt(to_dev(u))
    ub_want, bb_want = m.step_adjoint(to_dev(u), to_dev(w), dt)
    slabs = [adjoint_slab(crk, N, Ex, Ey, b, f, c) for f, c in parts]
    us = [to_dev(np.ascontiguousarray(u[:, f:f + c])) for f, c in parts]
    ws = [to_dev(np.ascontiguousarray(w[:, f:f + c])) for f, c in parts]
    for s, x, y in zip(slabs, us, ws):
        s.adjoint_local(x, y, dt)
    k_ = len(parts)
    for bufs in ([s.halo_buffers() for s in slabs], [s.adjoint_halo_buffers() for s in slabs]):
        for k in range(k_):
            bufs[k][2].copy_(bufs[(k - 1) % k_][1])   # recv_bottom <- send_top of the slab below
            bufs[k][3].copy_(bufs[(k + 1) % k_][0])   # recv_top <- send_bottom of the slab above
    outs = [s.adjoint_faces(x, y, dt) for s, x, y in zip(slabs, us, ws)]
    ub = np.concatenate([to_host(o[0]) for o in outs], axis=1)
    bb = np.concatenate([to_host(o[1]) for o in outs], axis=0)
    assert np.array_equal(ub, to_host(ub_want)), rel_l2(ub, to_host(ub_want))
    assert np.array_equal(bb, to_host(bb_want)), rel_l2(bb, to_host(bb_want))


def test_slab_adjoint_through_the_distributed_helper_and_errors():
    from paper_2512_08611_gb300.distributed import SlabStepper, slab_adjoint
    crk = load()
    N, Ex, Ey = 3, 12, 8
    u, b, dx, dy = case(N, Ex, Ey)
    w = np.random.default_rng(2).standard_normal(u.shape)
    m = solver(crk, N, Ex, Ey, b)
    dt = 0.5 * m.compute_dt(to_dev(u))
    ub_want, bb_want = m.step_adjoint(to_dev(u), to_dev(w), dt)
    s = adjoint_slab(crk, N, Ex, Ey, b, 0, Ey)
    with pytest.raises(crk.CrkfrError) as e:
        s.adjoint_halo_buffers()          # before the first adjoint_local
    assert e.value.status == -6
    with pytest.raises(crk.CrkfrError) as e:
        s.step_adjoint(to_dev(u), to_dev(w), dt)
    assert e.value.status == -6
    with pytest.raises(crk.CrkfrError) as e:
        m.adjoint_local(to_dev(u), to_dev(w), dt)
    assert e.value.status == -6
    ub, bb = slab_adjoint(SlabStepper(s), to_dev(u), to_dev(w), dt)
    assert np.array_equal(to_host(ub), to_host(ub_want))
    assert np.array_equal(to_host(bb), to_host(bb_want))


@pytest.mark.parametrize("recorded", [True, False])
def test_slab_autograd_function_equals_whole_mesh(recorded):
    """SlabBathymetryToState on a slab that is its own periodic neighbour
    (one rank) gives the final state and the bathymetry gradient of a surface
    misfit of BathymetryToState on the whole mesh, bit for bit, with
    recorded and with recomputing adjoint steps."""
    from paper_2512_08611_gb300.adjoint import (BathymetryToState, SlabBathymetryToState,
                                                quadrature_weights, surface_misfit)
    from paper_2512_08611_gb300.distributed import SlabStepper
    crk = load()
    N, Ex, Ey, nsteps, every = 3, 12, 10, 7, 3
    _, b, dx, dy = case(N, Ex, Ey, flow=0.0)
    x, y, _, _ = positions_2d(Basis(N), Ex, Ey, 100.0)
    eta0 = to_dev(1.0 + 0.01 * SWE2DInput(seed=0, L=100.0).bump(x, y))
    m = solver(crk, N, Ex, Ey, b)
    dt = 0.5 * m.compute_dt(torch.stack([eta0 - to_dev(b), 0 * eta0, 0 * eta0]))
    target = eta0.flip(0).contiguous()
    W = quadrature_weights(m)
    b1 = to_dev(b).requires_grad_(True)
    u1 = BathymetryToState.apply(b1, m, eta0, dt, nsteps, every, False)
    surface_misfit(u1, b1, target, W).backward()
    s = adjoint_slab(crk, N, Ex, Ey, b, 0, Ey)
    b2 = to_dev(b).requires_grad_(True)
    u2 = SlabBathymetryToState.apply(b2, SlabStepper(s), eta0, dt, nsteps, every, recorded)
    surface_misfit(u2, b2, target, W).backward()
    assert torch.equal(u1.detach(), u2.detach())
    assert torch.equal(b1.grad, b2.grad)
    assert float(b1.grad.abs().max()) > 0.0


def ring_exchange(bufs):
    k_ = len(bufs)
    for k in range(k_):
        bufs[k][2].copy_(bufs[(k - 1) % k_][1])   # recv_bottom <- send_top of the slab below
        bufs[k][3].copy_(bufs[(k + 1) % k_][0])   # recv_top <- send_bottom of the slab above


def test_slab_recorded_step_and_adjoint():
    """Recorded slab steps (crkfr_step_local_record, exchange of the
    record's y-trace blocks, crkfr_step_faces_record) and the recorded slab
    adjoint (crkfr_adjoint_sums, exchange, crkfr_adjoint_faces_recorded),
    with a one-row slab: the step and the adjoint of the whole mesh, bit for
    bit."""
    crk = load()
    N, Ex, Ey = 3, 16, 16
    u, b, dx, dy = case(N, Ex, Ey)
    w = np.random.default_rng(9).standard_normal(u.shape)
    m = solver(crk, N, Ex, Ey, b)
    dt = 0.5 * m.compute_dt(to_dev(u))
    step_want = to_dev(u)
    m.step(step_want, dt, 1)
    ub_want, bb_want = m.step_adjoint(to_dev(u), to_dev(w), dt)
    parts = [(0, 5), (5, 1), (6, 10)]
    slabs = [adjoint_slab(crk, N, Ex, Ey, b, f, c) for f, c in parts]
    us = [to_dev(np.ascontiguousarray(u[:, f:f + c])) for f, c in parts]
    ws = [to_dev(np.ascontiguousarray(w[:, f:f + c])) for f, c in parts]
    recs = [s.new_records(1)[0] for s in slabs]
    xs = [x.clone() for x in us]
    for s, x, r in zip(slabs, xs, recs):
        s.step_local_record(x, dt, r)
    ring_exchange([s.record_halo_buffers(r) for s, r in zip(slabs, recs)])
    for s, x, r in zip(slabs, xs, recs):
        s.step_faces_record(x, r)
    got = np.concatenate([to_host(x) for x in xs], axis=1)
    assert np.array_equal(got, to_host(step_want))
    for s, y in zip(slabs, ws):
        s.adjoint_sums(y)
    ring_exchange([s.adjoint_halo_buffers() for s in slabs])
    outs = [s.adjoint_faces_recorded(x, r, y, dt) for s, x, r, y in zip(slabs, us, recs, ws)]
    ub = np.concatenate([to_host(o[0]) for o in outs], axis=1)
    bb = np.concatenate([to_host(o[1]) for o in outs], axis=0)
    assert np.array_equal(ub, to_host(ub_want)), rel_l2(ub, to_host(ub_want))
    assert np.array_equal(bb, to_host(bb_want)), rel_l2(bb, to_host(bb_want))
