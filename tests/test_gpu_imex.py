"""GPU parity of the source-term (IMEX) path against the oracle.

With a source the inner stages follow SSP3-IMEX(4,3,3) (Sec. 2, Eqs.
crkfr.inner, crkfr, avg.source; App. C): the kernels solve each stage's
point-implicit equation in closed form, the oracle by Newton's method.
Tolerance 1e-12 relative L2 per step, as for the source-free path (the two
sides differ in FP64 rounding order and in how the stage equation is
solved to rounding)."""
import numpy as np
import pytest

from gpu_common import (G, golden_cfl_imex, load, positions_1d, positions_2d, rel_l2,
                        residual_close, to_dev, to_host)
from oracle.basis import Basis
from oracle.crkfr import Scheme1D, Scheme2D
from oracle.sources import ChezyFriction, LinearDamping
from oracle.systems import ShallowWater1D, ShallowWater2D, VarCoeffAdvection
from oracle.tableau import ssp3_imex433
from paper_2512_08611_gb300.workloads import SWE1DInput, SWE2DInput, VarAdvInput, accept_seed

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-12
CASES_1D = [(N, f) for N in range(5) for f in ("gl", "gll") if not (f == "gll" and N == 0)]
CASES_2D = [(N, f) for N in range(1, 5) for f in ("gl", "gll")]


@pytest.fixture(scope="module")
def crk():
    return load()


def swe1d_case(N, family, E, L=100.0, seed=1):
    bs = Basis(N, family)
    x, dx = positions_1d(bs, E, 0.0, L)
    inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=L), (x,), seed)
    u, b = inp.state(x)
    u[1] = u[0] * (0.6 + 0.3 * np.sin(2 * np.pi * x / L))     # a current
    return u, b, dx


def swe2d_case(N, family, Ex, Ey, L=100.0, seed=0):
    bs = Basis(N, family)
    x, y, dx, dy = positions_2d(bs, Ex, Ey, L)
    inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=L, n_gauss=8), (x, y), seed)
    u, b = inp.state(x, y)
    u[1] = u[0] * (0.5 + 0.2 * np.sin(2 * np.pi * y / L))
    u[2] = u[0] * (-0.3 + 0.2 * np.cos(2 * np.pi * x / L))
    return u, b, dx, dy


def solver(crk, system, N, family, n_elem, hi, c, source, coef, cs=0.5):
    s = crk.Solver(system, N, nodes=family, gravity=G, cfl_safety=cs,
                   cfl_number=golden_cfl_imex(N, family), source=source, source_coef=coef)
    s.set_mesh(list(n_elem), [0.0] * len(n_elem), [hi] * len(n_elem))
    s.set_coefficients(to_dev(c))
    return s


@pytest.mark.parametrize("N,family", CASES_1D)
@pytest.mark.parametrize("Cf", [0.05, 200.0])
@pytest.mark.parametrize("E", [3, 127, 300])
def test_swe1d_chezy_step_and_residual(crk, N, family, Cf, E):
    """Chezy friction, mild (C_f dt |v| / h << 1) and stiff (>> 1)."""
    u, b, dx = swe1d_case(N, family, E)
    sch = Scheme1D(ShallowWater1D(G), N, dx, family=family, source=ChezyFriction(Cf))
    dt = sch.compute_dt(u, b, golden_cfl_imex(N, family), 0.5)
    want = sch.step(u, b, dt)
    s = solver(crk, "swe1d", N, family, [E], 100.0, b, "chezy", Cf)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP
    r = to_host(s.residual(to_dev(u), dt))
    assert residual_close(r, -sch.residual(u, b, dt), u, dt)
    s.status()


@pytest.mark.parametrize("N,family", CASES_1D)
@pytest.mark.parametrize("K", [2.0, 1e6])
def test_varadv_linear_damping_step(crk, N, family, K):
    E = 130
    bs = Basis(N, family)
    x, dx = positions_1d(bs, E, 0.0, 1.0)
    inp = VarAdvInput()
    v, a = inp.v0(x)[None], inp.a(x)
    sch = Scheme1D(VarCoeffAdvection(), N, dx, family=family, source=LinearDamping(K))
    dt = sch.compute_dt(v, a, golden_cfl_imex(N, family), 0.5)
    want = sch.step(v, a, dt)
    s = solver(crk, "varadv1d", N, family, [E], 1.0, a, "linear", K)
    dv = to_dev(v)
    s.step(dv, dt, 1)
    got = to_host(dv)
    # with K dt ~ 1e3 the result is ~1e-4 of the data: compare against it
    assert np.linalg.norm(got - want) <= TOL_STEP * max(np.linalg.norm(want), 1e-3 * np.linalg.norm(v))


@pytest.mark.parametrize("N,family", CASES_2D)
@pytest.mark.parametrize("Cf", [0.05, 200.0])
def test_swe2d_chezy_step_and_residual(crk, N, family, Cf):
    Ex, Ey = 9, 7
    u, b, dx, dy = swe2d_case(N, family, Ex, Ey)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family=family, source=ChezyFriction(Cf))
    dt = sch.compute_dt(u, b, golden_cfl_imex(N, family), 0.5)
    want = sch.step(u, b, dt)
    s = solver(crk, "swe2d", N, family, [Ex, Ey], 100.0, b, "chezy", Cf)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP
    r = to_host(s.residual(to_dev(u), dt))
    assert residual_close(r, -sch.residual(u, b, dt), u, dt)
    s.status()


@pytest.mark.parametrize("N", [2, 3])
def test_swe1d_chezy_many_steps(crk, N):
    """100 CFL steps (the device recomputes dt from each state) against the
    oracle's loop with its own time step: 1e-10 relative L2."""
    E = 200
    u, b, dx = swe1d_case(N, "gl", E)
    Cf = 0.5
    sch = Scheme1D(ShallowWater1D(G), N, dx, source=ChezyFriction(Cf))
    cfl = golden_cfl_imex(N, "gl")
    want = u.copy()
    for _ in range(100):
        want = sch.step(want, b, sch.compute_dt(want, b, cfl, 0.5))
    s = solver(crk, "swe1d", N, "gl", [E], 100.0, b, "chezy", Cf)
    du = to_dev(u)
    s.step(du, 0.0, 100)
    assert rel_l2(to_host(du), want) < 1e-10


def test_swe2d_chezy_many_steps(crk):
    N, Ex, Ey = 3, 12, 10
    u, b, dx, dy = swe2d_case(N, "gl", Ex, Ey)
    Cf = 0.5
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, source=ChezyFriction(Cf))
    cfl = golden_cfl_imex(N, "gl")
    want = u.copy()
    for _ in range(40):
        want = sch.step(want, b, sch.compute_dt(want, b, cfl, 0.5))
    s = solver(crk, "swe2d", N, "gl", [Ex, Ey], 100.0, b, "chezy", Cf)
    du = to_dev(u)
    s.step(du, 0.0, 40)
    assert rel_l2(to_host(du), want) < 1e-10


@pytest.mark.parametrize("N", [1, 3])
def test_uniform_damping_is_the_stability_function(crk, N):
    """A uniform state under s = -K v: the step is R(-K dt) times the state,
    R the stability function of the implicit tableau, from moderate to very
    stiff K dt (L-stability: R(-inf) = 0)."""
    E = 64
    t = ssp3_imex433()
    for K in (1.0, 1e3, 1e9):
        s = solver(crk, "varadv1d", N, "gl", [E], 1.0, np.ones((E, N + 1)), "linear", K)
        v = np.full((1, E, N + 1), 0.75)
        dv = to_dev(v)
        dt = 1e-3
        s.step(dv, dt, 1)
        z = -K * dt
        R = 1.0 + z * t.bi @ np.linalg.solve(np.eye(4) - z * t.Ai, np.ones(4))
        assert np.max(np.abs(to_host(dv) - 0.75 * R)) < 1e-14 * max(1.0, -z)


def test_batch_with_source_equals_single_runs(crk):
    """Ragged ensemble with Chezy friction: each instance equals its own
    crkfr_step run bitwise."""
    import torch
    members = [(2, 150, 0.0, 100.0), (3, 333, 0.0, 80.0), (4, 97, 0.0, 120.0), (3, 1, 0.0, 50.0)]
    Cf = 0.3
    batch = crk.Batch("swe1d", members, gravity=G, source="chezy", source_coef=Cf)
    us, cs, singles = [], [], []
    for i, (N, E, lo, hi) in enumerate(members):
        u, b, dx = swe1d_case(N, "gl", E, L=hi, seed=10 + i)
        us.append(u)
        cs.append(b)
        s = crk.Solver("swe1d", N, gravity=G, source="chezy", source_coef=Cf)
        s.set_mesh([E], [lo], [hi])
        s.set_coefficients(to_dev(b))
        du = to_dev(u)
        s.step(du, 0.0, 7)
        singles.append(to_host(du))
    u = torch.cat([to_dev(x).reshape(-1) for x in us])
    c = torch.cat([to_dev(x).reshape(-1) for x in cs])
    batch.set_coefficients(c)
    batch.step(u, 0.0, 7, graph=True)
    batch.status()
    for i in range(len(members)):
        assert np.array_equal(to_host(batch.state_view(u, i)), singles[i]), i


def test_noalloc_with_source_equals_step(crk):
    N, E = 3, 500
    u, b, dx = swe1d_case(N, "gl", E)
    s = crk.Solver("swe1d", N, gravity=G, source="chezy", source_coef=1.0)
    s.set_mesh([E], [0.0], [100.0])
    s.set_coefficients(to_dev(b))
    d1 = to_dev(u)
    s.step(d1, 0.0, 5)
    import torch
    d2 = to_dev(u)
    out = torch.empty_like(d2)
    crk.step_1d_noalloc("swe1d", N, E, 0.0, 100.0, to_dev(b), d2, out, dt=0.0, nsteps=5,
                        gravity=G, source="chezy", source_coef=1.0)
    torch.cuda.synchronize()
    assert torch.equal(out, d1)


def test_adjoint_with_source_is_refused(crk):
    N, Ex, Ey = 2, 4, 4
    u, b, dx, dy = swe2d_case(N, "gl", Ex, Ey)
    s = solver(crk, "swe2d", N, "gl", [Ex, Ey], 100.0, b, "chezy", 0.1)
    with pytest.raises(crk.CrkfrError) as e:
        s.step_adjoint(to_dev(u), to_dev(np.ones_like(u)), 1e-3)
    assert e.value.status == -2


def test_swe2d_chezy_thousand_steps(crk):
    """1000 CFL steps of the friction workload's recipe (bathymetry, bump and
    current; C_f = 0.0025 as in the bench) on a 12 x 10, N = 3 mesh: 1e-10
    relative L2 after 1000 steps."""
    N, Ex, Ey = 3, 12, 10
    bs = Basis(N)
    x, y, dx, dy = positions_2d(bs, Ex, Ey, 100.0)
    inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=100.0, current=(0.3, 0.2)), (x, y), 3)
    u, b = inp.state(x, y)
    Cf = 0.0025
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, source=ChezyFriction(Cf))
    cfl = golden_cfl_imex(N, "gl")
    want = u.copy()
    for _ in range(1000):
        want = sch.step(want, b, sch.compute_dt(want, b, cfl, 0.5))
    s = solver(crk, "swe2d", N, "gl", [Ex, Ey], 100.0, b, "chezy", Cf)
    du = to_dev(u)
    s.step(du, 0.0, 1000)
    s.status()
    assert rel_l2(to_host(du), want) < 1e-10
    assert rel_l2(want, u) > 1e-4


def test_full_size_friction_workload_sampled(crk):
    """The friction bench workload as the benchmark launches it (1024^2,
    N = 3, GL, C_f = 0.0025, current (0.3, 0.2), seed 0): one CFL step; the
    oracle recomputes 128 sampled elements (incl. the corners)."""
    N, E = 3, 1024
    bs = Basis(N)
    x, y, dx, dy = positions_2d(bs, E, E, 100.0)
    inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=100.0, current=(0.3, 0.2)), (x, y), 0)
    u, b = inp.state(x, y)
    del x, y
    Cf = 0.0025
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, source=ChezyFriction(Cf))
    dt = sch.compute_dt(u, b, golden_cfl_imex(N, "gl"), 0.5)
    s = solver(crk, "swe2d", N, "gl", [E, E], 100.0, b, "chezy", Cf)
    du = to_dev(u)
    assert s.compute_dt(du) == pytest.approx(dt, rel=1e-14)
    s.step(du, 0.0, 1)
    got = to_host(du)
    rng = np.random.default_rng(21)
    ey = np.concatenate([[0, 0, E - 1, E - 1], rng.integers(0, E, 124)])
    ex = np.concatenate([[0, E - 1, 0, E - 1], rng.integers(0, E, 124)])
    want = sch.step_elements(u, b, dt, ey, ex)
    assert rel_l2(got[:, ey, ex], want) < 1e-12
    s.status()
