"""GPU parity of the well-balanced shallow-water forms (CRKFR_SYS_SWE_1D_WB,
CRKFR_SYS_SWE_2D_WB) against the oracle, and the lake at rest kept to
round-off on the GPU (the standard form moves it by its truncation error).
Tolerance 1e-12 relative L2 per step, as for the other forms."""
import numpy as np
import pytest

from gpu_common import (G, golden_cfl, golden_cfl_imex, load, positions_1d, positions_2d, rel_l2,
                        residual_close, to_dev, to_host)
from oracle.basis import Basis
from oracle.crkfr import Scheme1D, Scheme2D
from oracle.sources import ChezyFriction
from oracle.systems import ShallowWater1DWB, ShallowWater2DWB
from paper_2512_08611_gb300.workloads import SWE1DInput, SWE2DInput, accept_seed

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-12
CASES_1D = [(N, f) for N in range(5) for f in ("gl", "gll") if not (f == "gll" and N == 0)]
CASES_2D = [(N, f) for N in range(1, 5) for f in ("gl", "gll")]


@pytest.fixture(scope="module")
def crk():
    return load()


def case_1d(N, family, E, L=100.0, seed=1, still=False):
    bs = Basis(N, family)
    x, dx = positions_1d(bs, E, 0.0, L)
    inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=L, still=still), (x,), seed)
    u, b = inp.state(x)
    if not still:
        u[1] = u[0] * (0.4 + 0.3 * np.sin(2 * np.pi * x / L))
    return u, b, dx


def case_2d(N, family, Ex, Ey, L=100.0, seed=0, still=False):
    bs = Basis(N, family)
    x, y, dx, dy = positions_2d(bs, Ex, Ey, L)
    cur = (0.0, 0.0) if still else (0.3, -0.2)
    inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=L, n_gauss=8, current=cur), (x, y), seed)
    u, b = inp.state(x, y)
    if still:
        u[0] = 1.0 - b
    return u, b, dx, dy


def solver(crk, system, N, family, n_elem, hi, c, source=None, coef=0.0):
    cfl = golden_cfl_imex(N, family) if source else golden_cfl(N, family)
    s = crk.Solver(system, N, nodes=family, gravity=G, cfl_safety=0.5, cfl_number=cfl,
                   source=source, source_coef=coef)
    s.set_mesh(list(n_elem), [0.0] * len(n_elem), [hi] * len(n_elem))
    s.set_coefficients(to_dev(c))
    return s


@pytest.mark.parametrize("N,family", CASES_1D)
@pytest.mark.parametrize("E", [3, 127, 300])
@pytest.mark.parametrize("Cf", [None, 2.0])
def test_wb1d_step_and_residual(crk, N, family, E, Cf):
    u, b, dx = case_1d(N, family, E)
    src = ChezyFriction(Cf) if Cf else None
    sch = Scheme1D(ShallowWater1DWB(G), N, dx, family=family, source=src)
    cfl = golden_cfl_imex(N, family) if Cf else golden_cfl(N, family)
    dt = sch.compute_dt(u, b, cfl, 0.5)
    want = sch.step(u, b, dt)
    s = solver(crk, "swe1d_wb", N, family, [E], 100.0, b, "chezy" if Cf else None, Cf or 0.0)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP
    r = to_host(s.residual(to_dev(u), dt))
    assert residual_close(r, -sch.residual(u, b, dt), u, dt)
    s.status()


@pytest.mark.parametrize("N,family", CASES_2D)
@pytest.mark.parametrize("Cf", [None, 2.0])
def test_wb2d_step_and_residual(crk, N, family, Cf):
    Ex, Ey = 9, 7
    u, b, dx, dy = case_2d(N, family, Ex, Ey)
    src = ChezyFriction(Cf) if Cf else None
    sch = Scheme2D(ShallowWater2DWB(G), N, dx, dy, family=family, source=src)
    cfl = golden_cfl_imex(N, family) if Cf else golden_cfl(N, family)
    dt = sch.compute_dt(u, b, cfl, 0.5)
    want = sch.step(u, b, dt)
    s = solver(crk, "swe2d_wb", N, family, [Ex, Ey], 100.0, b, "chezy" if Cf else None, Cf or 0.0)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP
    r = to_host(s.residual(to_dev(u), dt))
    assert residual_close(r, -sch.residual(u, b, dt), u, dt)
    s.status()


def test_wb1d_many_steps(crk):
    N, E = 3, 200
    u, b, dx = case_1d(N, "gl", E)
    sch = Scheme1D(ShallowWater1DWB(G), N, dx)
    want = u.copy()
    for _ in range(100):
        want = sch.step(want, b, sch.compute_dt(want, b, golden_cfl(N, "gl"), 0.5))
    s = solver(crk, "swe1d_wb", N, "gl", [E], 100.0, b)
    du = to_dev(u)
    s.step(du, 0.0, 100)
    assert rel_l2(to_host(du), want) < 1e-10


@pytest.mark.parametrize("N,family", [(2, "gl"), (3, "gl"), (4, "gll")])
def test_lake_at_rest_1d_on_gpu(crk, N, family):
    """200 CFL steps of a lake at rest over the seeded bathymetry: the
    well-balanced form keeps it to round-off, the standard form does not."""
    E = 1000
    u, b, dx = case_1d(N, family, E, still=True)
    u[0] = 1.0 - b
    wb = solver(crk, "swe1d_wb", N, family, [E], 100.0, b)
    du = to_dev(u)
    wb.step(du, 0.0, 200)
    assert np.max(np.abs(to_host(du) - u)) < 1e-13
    st = solver(crk, "swe1d", N, family, [E], 100.0, b)
    dv = to_dev(u)
    st.step(dv, 0.0, 200)
    # (the standard form's defect is its truncation error: about 1e-9 at
    # N = 4 on this resolved bathymetry, larger at lower degree)
    assert np.max(np.abs(to_host(dv) - u)) > 1e-11


@pytest.mark.parametrize("Cf", [None, 5.0])
def test_lake_at_rest_2d_on_gpu(crk, Cf):
    N, E = 3, 64
    u, b, dx, dy = case_2d(N, "gl", E, E, still=True)
    s = solver(crk, "swe2d_wb", N, "gl", [E, E], 100.0, b, "chezy" if Cf else None, Cf or 0.0)
    du = to_dev(u)
    s.step(du, 0.0, 50)
    assert np.max(np.abs(to_host(du) - u)) < 1e-13
    st = solver(crk, "swe2d", N, "gl", [E, E], 100.0, b)
    dv = to_dev(u)
    st.step(dv, 0.0, 50)
    assert np.max(np.abs(to_host(dv) - u)) > 1e-11


def test_wb_batch_equals_single_runs(crk):
    import torch
    members = [(2, 150, 0.0, 100.0), (3, 333, 0.0, 80.0), (4, 97, 0.0, 120.0)]
    batch = crk.Batch("swe1d_wb", members, gravity=G)
    us, cs, singles = [], [], []
    for i, (N, E, lo, hi) in enumerate(members):
        u, b, dx = case_1d(N, "gl", E, L=hi, seed=20 + i)
        us.append(u)
        cs.append(b)
        s = crk.Solver("swe1d_wb", N, gravity=G)
        s.set_mesh([E], [lo], [hi])
        s.set_coefficients(to_dev(b))
        du = to_dev(u)
        s.step(du, 0.0, 6)
        singles.append(to_host(du))
    u = torch.cat([to_dev(x).reshape(-1) for x in us])
    c = torch.cat([to_dev(x).reshape(-1) for x in cs])
    batch.set_coefficients(c)
    batch.step(u, 0.0, 6, graph=True)
    batch.status()
    for i in range(len(members)):
        assert np.array_equal(to_host(batch.state_view(u, i)), singles[i]), i


def test_adjoint_of_wb_is_refused(crk):
    N, E = 2, 4
    u, b, dx, dy = case_2d(N, "gl", E, E)
    s = solver(crk, "swe2d_wb", N, "gl", [E, E], 100.0, b)
    with pytest.raises(crk.CrkfrError) as e:
        s.step_adjoint(to_dev(u), to_dev(np.ones_like(u)), 1e-3)
    assert e.value.status == -2


def test_full_size_sampled_step_wb_and_friction(crk):
    """The 1024^2, N = 3 workload in its well-balanced form with Chezy
    friction and a current, one CFL step as the benchmark launches it; the
    oracle recomputes 128 sampled elements (incl. the corners)."""
    N, E = 3, 1024
    u, b, dx, dy = case_2d(N, "gl", E, E)
    Cf = 0.0025
    sch = Scheme2D(ShallowWater2DWB(G), N, dx, dy, source=ChezyFriction(Cf))
    dt = sch.compute_dt(u, b, golden_cfl_imex(N, "gl"), 0.5)
    s = solver(crk, "swe2d_wb", N, "gl", [E, E], 100.0, b, "chezy", Cf)
    du = to_dev(u)
    s.step(du, 0.0, 1)
    got = to_host(du)
    rng = np.random.default_rng(12)
    ey = np.concatenate([[0, 0, E - 1, E - 1], rng.integers(0, E, 124)])
    ex = np.concatenate([[0, E - 1, 0, E - 1], rng.integers(0, E, 124)])
    want = sch.step_elements(u, b, dt, ey, ex)
    assert rel_l2(got[:, ey, ex], want) < TOL_STEP
    s.status()


def test_thousand_steps_wb_with_friction(crk):
    """1000 CFL steps of the well-balanced 1D form with friction: 1e-10
    relative L2 against the oracle's loop."""
    N, E = 3, 256
    u, b, dx = case_1d(N, "gl", E)
    sch = Scheme1D(ShallowWater1DWB(G), N, dx, source=ChezyFriction(0.2))
    cfl = golden_cfl_imex(N, "gl")
    v = u
    for _ in range(1000):
        v = sch.step(v, b, sch.compute_dt(v, b, cfl, 0.5))
    s = solver(crk, "swe1d_wb", N, "gl", [E], 100.0, b, "chezy", 0.2)
    du = to_dev(u)
    s.step(du, 0.0, 1000)
    assert rel_l2(to_host(du), v) < 1e-10
    s.status()


def test_wb2d_thousand_steps(crk):
    """1000 CFL steps of the well-balanced 2D form on a moving flow over
    bathymetry (12 x 10, N = 3): 1e-10 relative L2 after 1000 steps."""
    N, Ex, Ey = 3, 12, 10
    u, b, dx, dy = case_2d(N, "gl", Ex, Ey, seed=2)
    sch = Scheme2D(ShallowWater2DWB(G), N, dx, dy)
    want = u.copy()
    for _ in range(1000):
        want = sch.step(want, b, sch.compute_dt(want, b, golden_cfl(N, "gl"), 0.5))
    s = solver(crk, "swe2d_wb", N, "gl", [Ex, Ey], 100.0, b)
    du = to_dev(u)
    s.step(du, 0.0, 1000)
    s.status()
    assert rel_l2(to_host(du), want) < 1e-10
    assert rel_l2(want, u) > 1e-4


def test_full_size_wb_workload_sampled(crk):
    """The well-balanced bench workload as the benchmark launches it (1024^2,
    N = 3, GL, 32 Gaussians, bump, at rest otherwise, seed 0): one CFL step;
    the oracle recomputes 128 sampled elements (incl. the corners)."""
    N, E = 3, 1024
    bs = Basis(N)
    x, y, dx, dy = positions_2d(bs, E, E, 100.0)
    inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=100.0), (x, y), 0)
    u, b = inp.state(x, y)
    del x, y
    sch = Scheme2D(ShallowWater2DWB(G), N, dx, dy)
    dt = sch.compute_dt(u, b, golden_cfl(N, "gl"), 0.5)
    s = solver(crk, "swe2d_wb", N, "gl", [E, E], 100.0, b)
    du = to_dev(u)
    assert s.compute_dt(du) == pytest.approx(dt, rel=1e-14)
    s.step(du, 0.0, 1)
    got = to_host(du)
    rng = np.random.default_rng(22)
    ey = np.concatenate([[0, 0, E - 1, E - 1], rng.integers(0, E, 124)])
    ex = np.concatenate([[0, E - 1, 0, E - 1], rng.integers(0, E, 124)])
    want = sch.step_elements(u, b, dt, ey, ex)
    assert rel_l2(got[:, ey, ex], want) < TOL_STEP
    assert np.max(np.abs(want - u[:, ey, ex])) > 0
    s.status()
