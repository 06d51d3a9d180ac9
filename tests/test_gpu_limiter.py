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


def dam_on(N, E, L, hR=1e-3):
    """The dam break on [0, L] (GLL nodes), jumps inside elements 101 and 301
    of 400."""
    bs = Basis(N, "gll")
    x, dx = positions_1d(bs, E, 0.0, L)
    h = np.where((x > 0.2537 * L) & (x < 0.7537 * L), 1.0, 1e-3)
    return np.stack([h, np.zeros_like(h)]), np.zeros_like(h), dx


def smooth_on(N, E, L):
    bs = Basis(N, "gll")
    x, dx = positions_1d(bs, E, 0.0, L)
    b = 0.1 * np.sin(2 * np.pi * x / L) ** 2
    u = np.stack([1.0 + 0.1 * np.cos(2 * np.pi * x / L) - b, 0.3 * np.sin(2 * np.pi * x / L)])
    return u, b, dx


# (the dam break needs the indicator: with a fixed alpha, or at N = 2, the
# blended step's depth goes negative within a few CFL steps of C_s = 0.1, in
# the oracle as on the GPU)
@pytest.mark.parametrize("system,N,mode,alpha,source,data", [
    ("swe1d", 3, "blend", 0.0, None, "dam"), ("swe1d", 4, "blend", 0.0, None, "dam"),
    ("swe1d", 2, "fixed", 0.4, None, "smooth"), ("swe1d_wb", 3, "blend", 0.0, None, "dam"),
    ("swe1d", 3, "blend", 0.0, "chezy", "dam")])
def test_limited_ranges_equal_single_domain(crk, system, N, mode, alpha, source, data):
    """Four ranges of a 400-element mesh (100, 2, 199 and 99 elements; the
    dam's jumps lie in elements 101 and 301, at the range ends 101 | 102 and
    300 | 301), each exchanging its end elements' states and raw indicator
    with its neighbours: the ranges' states and blending coefficients equal
    the single-domain limited step bit for bit."""
    E, L, steps = 400, 100.0, 5        # dx = 1/4: every range's 1/dx is the mesh's
    u, b, dx = dam_on(N, E, L) if data == "dam" else smooth_on(N, E, L)
    cfl = golden_cfl_imex(N, "gll") if source else golden_cfl(N, "gll")
    coef = 2.0 if source else 0.0

    def make(first, count):
        s = crk.Solver(system, N, nodes="gll", gravity=G, cfl_safety=0.1, cfl_number=cfl,
                       source=source, source_coef=coef)
        s.set_mesh([count], [first * dx], [(first + count) * dx])
        return s
    m = make(0, E)
    m.set_coefficients(to_dev(b))
    m.set_limiter(mode, alpha)
    want = to_dev(u)
    parts = [(0, 100), (100, 2), (102, 199), (301, 99)]
    ranges = []
    for f, c in parts:
        s = make(f, c)
        s.set_subdomain(True)
        el = [(f - 1) % E] + list(range(f, f + c)) + [(f + c) % E]
        s.set_coefficients(to_dev(np.ascontiguousarray(b[el])))
        s.set_limiter(mode, alpha)
        ranges.append(s)
    states = [to_dev(np.ascontiguousarray(u[:, f:f + c])) for f, c in parts]
    bufs = [s.halo_buffers() for s in ranges]
    k_ = len(parts)
    for _ in range(steps):
        # the CFL step of the state (the dam's speeds grow as it breaks)
        dt = m.compute_dt(want)
        m.step(want, dt, 1)
        for s, x in zip(ranges, states):
            s.step_local(x, dt)
        for k in range(k_):
            bufs[k][2].copy_(bufs[(k - 1) % k_][1])    # left ghost <- right end of the left range
            bufs[k][3].copy_(bufs[(k + 1) % k_][0])    # right ghost <- left end of the right range
        for s, x in zip(ranges, states):
            s.step_faces(x)
    got = np.concatenate([to_host(x) for x in states], axis=1)
    assert np.all(np.isfinite(got)) and np.min(got[0]) > 0.0
    assert np.array_equal(got, to_host(want)), rel_l2(got, to_host(want))
    a = np.concatenate([to_host(s.limiter_alpha()) for s in ranges])
    a_want = to_host(m.limiter_alpha())
    assert np.array_equal(a, a_want)
    if data == "dam":
        assert np.max(a_want[[99, 100, 101, 102, 299, 300, 301, 302]]) > 0.5
        assert np.min(a_want) == 0.0


def test_limited_range_configuration(crk):
    """A limited range needs two elements; the stepper runs a limited range
    that is its own periodic neighbour, in CFL steps."""
    from paper_2512_08611_gb300.distributed import SlabStepper
    r = crk.Solver("swe1d", 2, gravity=G)
    r.set_mesh([1], [0.0], [1.0])
    r.set_subdomain(True)
    with pytest.raises(crk.CrkfrError) as e:
        r.set_limiter("blend")
    assert e.value.status == -2
    N, E, L = 3, 40, 100.0
    u, b, dx = dam_on(N, E, L)
    m = crk.Solver("swe1d", N, nodes="gll", gravity=G, cfl_safety=0.1,
                   cfl_number=golden_cfl(N, "gll"))
    m.set_mesh([E], [0.0], [L])
    m.set_coefficients(to_dev(b))
    m.set_limiter("blend")
    s = crk.Solver("swe1d", N, nodes="gll", gravity=G, cfl_safety=0.1,
                   cfl_number=golden_cfl(N, "gll"))
    s.set_mesh([E], [0.0], [L])
    s.set_subdomain(True)
    s.set_coefficients(to_dev(np.ascontiguousarray(b[[E - 1] + list(range(E)) + [0]])))
    s.set_limiter("blend")
    x, want = to_dev(u), to_dev(u)
    st = SlabStepper(s)
    for _ in range(3):
        dt = m.compute_dt(want)
        m.step(want, dt, 1)
        st.step(x, 0.0, 1)
        assert st.last_dt == dt
    assert np.array_equal(to_host(x), to_host(want))
