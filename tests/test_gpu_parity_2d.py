"""GPU parity of the 2D shallow-water cRK-FR path (C ABI, sm_103a) against
the oracle: small meshes over several warps/blocks with ragged tails, and
the full 1024 x 1024, N = 3 workload on sampled elements."""
import numpy as np
import pytest

from gpu_common import G, golden_cfl, load, positions_2d, rel_l2, residual_close, to_dev, to_host
from oracle.basis import Basis
from oracle.crkfr import Scheme1D, Scheme2D
from oracle.systems import ShallowWater1D, ShallowWater2D
from paper_2512_08611_gb300.workloads import SWE2DInput, accept_seed

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-12


@pytest.fixture(scope="module")
def crk():
    return load()


def swe2d_case(N, family, Ex, Ey, seed=0, L=100.0, flow=True):
    bs = Basis(N, family)
    x, y, dx, dy = positions_2d(bs, Ex, Ey, L)
    inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=L), (x, y), seed)
    u, b = inp.state(x, y)
    if flow:   # add a smooth velocity so every flux term is exercised
        u[1] = 0.05 * np.sin(2 * np.pi * y / L) * u[0]
        u[2] = 0.05 * np.cos(2 * np.pi * x / L) * u[0]
    return u, b, dx, dy


def solver(crk, N, family, Ex, Ey, b, L=100.0, cs=0.5):
    s = crk.Solver("swe2d", N, nodes=family, gravity=G, cfl_safety=cs,
                   cfl_number=golden_cfl(N, family))
    s.set_mesh([Ex, Ey], [0.0, 0.0], [L, L])
    s.set_coefficients(to_dev(b))
    return s


CASES = [(N, fam) for N in (1, 2, 3, 4) for fam in ("gl", "gll")]


@pytest.mark.parametrize("N,family", CASES)
@pytest.mark.parametrize("Ex,Ey", [(1, 1), (3, 2), (9, 5), (17, 4)])
def test_one_step_and_residual(crk, N, family, Ex, Ey):
    u, b, dx, dy = swe2d_case(N, family, Ex, Ey)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family=family)
    dt = sch.compute_dt(u, b, golden_cfl(N, family), 0.5)
    want = sch.step(u, b, dt)
    s = solver(crk, N, family, Ex, Ey, b)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP
    r = to_host(s.residual(to_dev(u), dt))
    assert residual_close(r, -sch.residual(u, b, dt), u, dt)
    s.status()


@pytest.mark.parametrize("N,family", [(1, "gl"), (3, "gl"), (3, "gll"), (4, "gl")])
def test_cfl_steps(crk, N, family):
    Ex, Ey, nsteps = 12, 7, 20
    u, b, dx, dy = swe2d_case(N, family, Ex, Ey, seed=4)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family=family)
    cfl = golden_cfl(N, family)
    s = solver(crk, N, family, Ex, Ey, b)
    du = to_dev(u)
    assert s.compute_dt(du) == pytest.approx(sch.compute_dt(u, b, cfl, 0.5), rel=1e-14)
    v = u
    for _ in range(nsteps):
        v = sch.step(v, b, sch.compute_dt(v, b, cfl, 0.5))
    s.step(du, 0.0, nsteps)
    assert rel_l2(to_host(du), v) < 1e-11


def test_y_invariant_2d_matches_1d_gpu(crk):
    """Property at any size: y-invariant data with zero y-momentum advances
    like the 1D scheme on every row (GPU 2D vs GPU 1D)."""
    N, Ex, Ey, L = 3, 40, 3, 100.0
    bs = Basis(N)
    dx = L / Ex
    x = (np.arange(Ex)[:, None] + bs.xi[None, :]) * dx
    b1 = 0.2 * np.exp(-((x - 40) ** 2) / 20)
    u1 = np.stack([1.0 - b1 + 0.01 * np.sin(2 * np.pi * x / L), 0.1 * np.cos(2 * np.pi * x / L)])
    n = N + 1
    tile = lambda a: np.ascontiguousarray(np.broadcast_to(a[None, :, None, :], (Ey, Ex, n, n)))
    u2 = np.stack([tile(u1[0]), tile(u1[1]), np.zeros((Ey, Ex, n, n))])
    s2 = solver(crk, N, "gl", Ex, Ey, tile(b1))
    d2 = to_dev(u2)
    s2.step(d2, 0.01, 10)
    s1 = crk.Solver("swe1d", N, gravity=G, cfl_safety=0.5)
    s1.set_mesh([Ex], [0.0], [L])
    s1.set_coefficients(to_dev(b1))
    d1 = to_dev(u1)
    s1.step(d1, 0.01, 10)
    g2, g1 = to_host(d2), to_host(d1)
    for v in range(2):
        assert np.max(np.abs(g2[v] - g1[v][None, :, None, :])) < 1e-12
    assert np.max(np.abs(g2[2])) < 1e-12


@pytest.fixture(scope="module")
def config3(crk):
    N, E = 3, 1024
    u, b, dx, dy = swe2d_case(N, "gl", E, E, seed=0, flow=False)
    return N, E, u, b, dx, dy


def test_config3_sampled_step(crk, config3):
    """Full 1024^2, N = 3 workload, one CFL step in the launch configuration
    the benchmark uses; the oracle recomputes 256 sampled elements (incl.
    the four corners) from their stencils."""
    N, E, u, b, dx, dy = config3
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy)
    cfl = golden_cfl(N, "gl")
    dt = sch.compute_dt(u, b, cfl, 0.5)
    s = solver(crk, N, "gl", E, E, b)
    du = to_dev(u)
    assert s.compute_dt(du) == pytest.approx(dt, rel=1e-14)
    s.step(du, 0.0, 1)
    got = to_host(du)
    rng = np.random.default_rng(11)
    ey = np.concatenate([[0, 0, E - 1, E - 1], rng.integers(0, E, 252)])
    ex = np.concatenate([[0, E - 1, 0, E - 1], rng.integers(0, E, 252)])
    want = sch.step_elements(u, b, dt, ey, ex)
    assert rel_l2(got[:, ey, ex], want) < TOL_STEP
    # the bump moves: the sampled update is not the identity
    assert np.max(np.abs(want - u[:, ey, ex])) > 0
    s.status()


def test_config3_mass_conservation(crk, config3):
    N, E, u, b, dx, dy = config3
    w = Basis(N).w
    W = dx * dy * w[:, None] * w[None, :]
    s = solver(crk, N, "gl", E, E, b)
    du = to_dev(u)
    s.step(du, 0.0, 10)
    got = to_host(du)
    m0, m1 = np.sum(W * u[0]), np.sum(W * got[0])
    assert abs(m1 - m0) < 1e-13 * abs(m0)


def test_checkpoint_resume_repeats_the_run():
    """state_dict after 10 CFL steps, then 5 more; a second context loaded
    from the checkpoint and stepped 5 times gives the same bits and time."""
    crk = load()
    N, Ex, Ey = 3, 12, 10
    u, b, dx, dy = swe2d_case(N, "gl", Ex, Ey)
    s1 = solver(crk, N, "gl", Ex, Ey, b)
    d1 = to_dev(u)
    s1.step(d1, 0.0, 10)
    sd = s1.state_dict(d1)
    s1.step(d1, 0.0, 5)
    s2 = solver(crk, N, "gl", Ex, Ey, b)
    d2 = to_dev(np.zeros_like(u))
    s2.load_state_dict(sd, d2)
    s2.step(d2, 0.0, 5)
    assert np.array_equal(to_host(d1), to_host(d2))
    assert s1.time()[0] == s2.time()[0]


@pytest.mark.parametrize("Ex,Ey", [(5, 3), (7, 8), (6, 37), (3, 70)])
@pytest.mark.parametrize("limited", [False, True])
def test_host_step_reads_rows_back_in_chunks(crk, Ex, Ey, limited):
    """crkfr_step_host uploads the state in parts of element rows while the
    rate and the first stage's local operator of the parts already there are
    computed, runs the last face kernel in chunks of rows and copies each
    chunk back while the next one computes: the result is the device step's,
    bit for bit (CFL steps, one and three per call, with and without the
    limiter, and fixed steps in place), from pinned and from ordinary host
    memory."""
    import torch
    N = 3
    u, b, dx, dy = swe2d_case(N, "gl", Ex, Ey)
    for nsteps in (1, 3):
        s1 = solver(crk, N, "gl", Ex, Ey, b)
        s2 = solver(crk, N, "gl", Ex, Ey, b)
        if limited:
            s1.set_limiter("blend")
            s2.set_limiter("blend")
        du = to_dev(u)
        s1.step(du, 0.0, nsteps)
        pinned = torch.tensor(u).pin_memory().numpy()
        out = s2.step_host(pinned, dt=0.0, nsteps=nsteps)
        assert np.array_equal(out, to_host(du))
        plain = s2.step_host(np.ascontiguousarray(u), dt=0.0, nsteps=nsteps)
        assert np.array_equal(plain, to_host(du))
        # two host calls from the same state: twice the simulated time
        assert s2.time()[0] == pytest.approx(2 * s1.time()[0], rel=1e-15)
    # a fixed step (no rate in the upload) and a second call in place
    s1 = solver(crk, N, "gl", Ex, Ey, b)
    s2 = solver(crk, N, "gl", Ex, Ey, b)
    dt = 0.5 * s1.compute_dt(to_dev(u))
    du = to_dev(u)
    s1.step(du, dt, 2)
    h = torch.tensor(u).pin_memory().numpy()
    s2.step_host(h, h, dt=dt, nsteps=1)
    s2.step_host(h, h, dt=dt, nsteps=1)
    assert np.array_equal(h, to_host(du))


def test_thousand_steps_2d(crk):
    """1000 CFL steps of the 2D workload's recipe (32 Gaussians of bathymetry,
    a surface bump, a smooth current) on a 12 x 10, N = 3 mesh: 1e-10
    relative L2 after 1000 steps."""
    N, Ex, Ey = 3, 12, 10
    u, b, dx, dy = swe2d_case(N, "gl", Ex, Ey, seed=7)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy)
    cfl = golden_cfl(N, "gl")
    v = u
    for _ in range(1000):
        v = sch.step(v, b, sch.compute_dt(v, b, cfl, 0.5))
    s = solver(crk, N, "gl", Ex, Ey, b)
    du = to_dev(u)
    s.step(du, 0.0, 1000)
    s.status()
    assert rel_l2(to_host(du), v) < 1e-10
    # the flow has moved
    assert rel_l2(v, u) > 1e-4
