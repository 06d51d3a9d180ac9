"""GPU parity of the 1D subcell blending limiter (crkfr_set_limiter; Sec. 4,
Eqs. blended.scheme, low.order.update, Fblend, Algorithms 1 and 2) against
the oracle's Blending1D: fixed blending coefficients from 0 to 1, the
smoothness indicator, positivity and mass on a dam break onto a thin layer,
a source term, and the well-balanced lake at rest.  1e-12 relative L2 per
step (the indicator's logistic function goes through CUDA's exp, the
oracle's through numpy's: both within an ulp)."""
import numpy as np
import pytest

from gpu_common import G, golden_cfl, golden_cfl_imex, load, positions_1d, rel_l2, to_dev, to_host
from oracle.basis import Basis
from oracle.crkfr import Scheme1D
from oracle.limiter import Blending1D, hennemann_alpha
from oracle.sources import ChezyFriction
from oracle.systems import ShallowWater1D, ShallowWater1DWB, VarCoeffAdvection

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-12
SYSTEMS = {"swe1d": ShallowWater1D, "swe1d_wb": ShallowWater1DWB}
CASES = [(N, f) for N in range(1, 5) for f in ("gl", "gll")]


@pytest.fixture(scope="module")
def crk():
    return load()


def flow(N, family, E, L=1.0):
    bs = Basis(N, family)
    x, dx = positions_1d(bs, E, 0.0, L)
    b = 0.1 * np.sin(2 * np.pi * x) ** 2
    u = np.stack([1.0 + 0.1 * np.cos(2 * np.pi * x) - b, 0.3 * np.sin(2 * np.pi * x)])
    return u, b, dx


def dam(N, family, E, hR=1e-3):
    bs = Basis(N, family)
    x, dx = positions_1d(bs, E, 0.0, 1.0)
    h = np.where((x > 0.2537) & (x < 0.7537), 1.0, hR)   # jumps inside elements
    return np.stack([h, np.zeros_like(h)]), np.zeros_like(h), dx


def solver(crk, system, N, family, E, c, cs=0.5, source=None, coef=0.0):
    cfl = golden_cfl_imex(N, family) if source else golden_cfl(N, family)
    s = crk.Solver(system, N, nodes=family, gravity=G, cfl_safety=cs, cfl_number=cfl,
                   source=source, source_coef=coef)
    s.set_mesh([E], [0.0], [1.0])
    s.set_coefficients(to_dev(c))
    return s


@pytest.mark.parametrize("N,family", CASES)
@pytest.mark.parametrize("system", ["swe1d", "swe1d_wb"])
@pytest.mark.parametrize("alpha", [0.0, 0.4, 1.0])
def test_fixed_alpha_step(crk, N, family, system, alpha):
    E = 130
    u, b, dx = flow(N, family, E)
    sch = Scheme1D(SYSTEMS[system](G), N, dx, family=family)
    dt = sch.compute_dt(u, b, golden_cfl(N, family), 0.5)
    want = Blending1D(sch, alpha=alpha).step(u, b, dt)
    s = solver(crk, system, N, family, E, b)
    s.set_limiter("fixed", alpha)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP
    assert np.all(to_host(s.limiter_alpha()) == alpha)


@pytest.mark.parametrize("N,family", CASES)
def test_fixed_alpha_advection(crk, N, family):
    E = 130
    bs = Basis(N, family)
    x, dx = positions_1d(bs, E, 0.0, 1.0)
    a = 1.0 + 0.5 * np.sin(2 * np.pi * x)
    v = np.where((x > 0.215) & (x < 0.515), 1.0, 0.0)[None]
    sch = Scheme1D(VarCoeffAdvection(), N, dx, family=family)
    dt = sch.compute_dt(v, a, golden_cfl(N, family), 0.5)
    want = Blending1D(sch, alpha=0.7).step(v, a, dt)
    s = solver(crk, "varadv1d", N, family, E, a)
    s.set_limiter("fixed", 0.7)
    dv = to_dev(v)
    s.step(dv, dt, 1)
    assert rel_l2(to_host(dv), want) < TOL_STEP


@pytest.mark.parametrize("N", [2, 3, 4])
def test_indicator_and_step_on_a_dam_break(crk, N):
    """GLL nodes, C_s 0.2: the indicator's alpha per element and the limited
    step (Algorithms 1 and 2 active at the thin layer) against the oracle."""
    E = 64
    u, b, dx = dam(N, "gll", E)
    sch = Scheme1D(ShallowWater1D(G), N, dx, family="gll")
    lim = Blending1D(sch)
    dt = sch.compute_dt(u, b, golden_cfl(N, "gll"), 0.2)
    want = lim.step(u, b, dt)
    s = solver(crk, "swe1d", N, "gll", E, b, cs=0.2)
    s.set_limiter("blend")
    du = to_dev(u)
    s.step(du, dt, 1)
    got_alpha = to_host(s.limiter_alpha())
    assert np.max(np.abs(got_alpha - lim.last_alpha)) < 1e-12
    assert np.max(got_alpha) > 0.5
    assert rel_l2(to_host(du), want) < TOL_STEP


def test_dam_break_positive_conservative_and_close_to_oracle(crk):
    N, E, steps = 3, 200, 200
    u, b, dx = dam(N, "gll", E)
    s = solver(crk, "swe1d", N, "gll", E, b, cs=0.2)
    s.set_limiter("blend")
    du = to_dev(u)
    bs = Basis(N, "gll")
    mass0 = np.sum(bs.w * u[0])
    for _ in range(steps // 20):
        s.step(du, 0.0, 20)
        h = to_host(du)[0]
        assert np.min(h) > 0.0
    s.status()
    assert abs(np.sum(bs.w * to_host(du)[0]) - mass0) < 1e-12 * mass0
    # the first 20 CFL steps against the oracle
    sch = Scheme1D(ShallowWater1D(G), N, dx, family="gll")
    lim = Blending1D(sch)
    v = u.copy()
    for _ in range(20):
        v = lim.step(v, b, sch.compute_dt(v, b, golden_cfl(N, "gll"), 0.2))
    s2 = solver(crk, "swe1d", N, "gll", E, b, cs=0.2)
    s2.set_limiter("blend")
    dv = to_dev(u)
    s2.step(dv, 0.0, 20)
    assert rel_l2(to_host(dv), v) < 1e-10


@pytest.mark.parametrize("N", [1, 3])
def test_limiter_with_chezy_friction(crk, N):
    E = 130
    u, b, dx = flow(N, "gl", E)
    sch = Scheme1D(ShallowWater1D(G), N, dx, source=ChezyFriction(3.0))
    dt = sch.compute_dt(u, b, golden_cfl_imex(N, "gl"), 0.5)
    want = Blending1D(sch, alpha=0.5).step(u, b, dt)
    s = solver(crk, "swe1d", N, "gl", E, b, source="chezy", coef=3.0)
    s.set_limiter("fixed", 0.5)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP


def test_well_balanced_lake_at_rest_with_limiter(crk):
    N, E = 3, 100
    bs = Basis(N, "gll")
    x, dx = positions_1d(bs, E, 0.0, 1.0)
    b = 0.3 * np.exp(-((x - 0.4) ** 2) / (2 * 0.05 ** 2)) + np.where(x > 0.7, 0.2, 0.0)
    u0 = np.stack([1.0 - b, np.zeros_like(b)])
    s = solver(crk, "swe1d_wb", N, "gll", E, b)
    s.set_limiter("blend")
    du = to_dev(u0)
    s.step(du, 0.0, 100)
    assert np.max(np.abs(to_host(du) - u0)) < 1e-13
    assert np.max(to_host(s.limiter_alpha())) > 0.5


def test_limiter_configuration_errors(crk):
    s0 = crk.Solver("swe1d", 0, gravity=G)
    s0.set_mesh([8], [0.0], [1.0])
    with pytest.raises(crk.CrkfrError) as e:
        s0.set_limiter("blend")
    assert e.value.status == -2
    s1 = crk.Solver("swe1d", 2, gravity=G)
    s1.set_mesh([8], [0.0], [1.0])
    with pytest.raises(crk.CrkfrError) as e:
        s1.set_limiter("fixed", 1.5)
    assert e.value.status == -1


def test_config2_size_with_limiter(crk):
    """The 1D workload's size (1e5 elements, N = 4, GL, [0, 100]) with the
    indicator-driven limiter: one CFL step against the oracle on the whole
    mesh (smooth data: the indicator stays off almost everywhere, the step
    is then the plain cRK-FR step)."""
    from paper_2512_08611_gb300.workloads import SWE1DInput, accept_seed
    N, E = 4, 100000
    bs = Basis(N)
    x, dx = positions_1d(bs, E, 0.0, 100.0)
    inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=100.0), (x,), 0)
    u, b = inp.state(x)
    sch = Scheme1D(ShallowWater1D(G), N, dx)
    lim = Blending1D(sch)
    dt = sch.compute_dt(u, b, golden_cfl(N, "gl"), 0.5)
    want = lim.step(u, b, dt)
    s = crk.Solver("swe1d", N, gravity=G, cfl_safety=0.5, cfl_number=golden_cfl(N, "gl"))
    s.set_mesh([E], [0.0], [100.0])
    s.set_coefficients(to_dev(b))
    s.set_limiter("blend")
    du = to_dev(u)
    s.step(du, 0.0, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP
    assert np.max(np.abs(to_host(s.limiter_alpha()) - lim.last_alpha)) < 1e-12
