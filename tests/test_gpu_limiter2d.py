"""GPU parity of the 2D subcell blending limiter (crkfr_set_limiter on a 2D
mesh; the tensor-product extension of Sec. 4, Eqs. blended.scheme,
low.order.update, Fblend, Algorithms 1 and 2) against the oracle's
Blending2D: fixed blending coefficients from 0 to 1 for the standard and the
well-balanced forms, the 2D smoothness indicator, positivity and mass on a
circular dam break onto a thin layer, Chezy friction, the well-balanced lake
at rest, and the full 1024 x 1024, N = 3 mesh on sampled elements.  1e-12
relative L2 per step (the indicator's logistic function goes through CUDA's
exp, the oracle's through numpy's)."""
import numpy as np
import pytest

from gpu_common import G, golden_cfl, golden_cfl_imex, load, positions_2d, rel_l2, to_dev, to_host
from oracle.basis import Basis
from oracle.crkfr import Scheme2D
from oracle.limiter import Blending2D
from oracle.sources import ChezyFriction
from oracle.systems import ShallowWater2D, ShallowWater2DWB

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-12
SYSTEMS = {"swe2d": ShallowWater2D, "swe2d_wb": ShallowWater2DWB}
CASES = [(N, f) for N in range(1, 5) for f in ("gl", "gll")]


@pytest.fixture(scope="module")
def crk():
    return load()


def flow(N, family, Ex, Ey):
    bs = Basis(N, family)
    x, y, dx, dy = positions_2d(bs, Ex, Ey, 1.0)
    b = 0.1 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    u = np.stack([1.2 - b + 0.05 * np.sin(2 * np.pi * (x + y)), 0.2 * np.cos(2 * np.pi * y),
                  0.1 * np.sin(2 * np.pi * x)])
    return u, b, dx, dy


def dam(N, Ex, Ey, hR=1e-3, r=0.2):
    """Circular dam break onto a thin layer (GLL nodes: GL traces of the
    jump can be negative)."""
    bs = Basis(N, "gll")
    x, y, dx, dy = positions_2d(bs, Ex, Ey, 1.0)
    h = np.where((x - 0.5037) ** 2 + (y - 0.4963) ** 2 < r * r, 1.0, hR)
    z = np.zeros_like(h)
    return np.stack([h, z, z.copy()]), z.copy(), dx, dy


def solver(crk, system, N, family, Ex, Ey, c, cs=0.5, source=None, coef=0.0):
    cfl = golden_cfl_imex(N, family) if source else golden_cfl(N, family)
    s = crk.Solver(system, N, nodes=family, gravity=G, cfl_safety=cs, cfl_number=cfl,
                   source=source, source_coef=coef)
    s.set_mesh([Ex, Ey], [0.0, 0.0], [1.0, 1.0])
    s.set_coefficients(to_dev(c))
    return s


@pytest.mark.parametrize("N,family", CASES)
@pytest.mark.parametrize("system", ["swe2d", "swe2d_wb"])
@pytest.mark.parametrize("alpha", [0.0, 0.4, 1.0])
def test_fixed_alpha_step(crk, N, family, system, alpha):
    Ex, Ey = 9, 5    # several tiles of both kernels, ragged in x and y
    u, b, dx, dy = flow(N, family, Ex, Ey)
    sch = Scheme2D(SYSTEMS[system](G), N, dx, dy, family=family)
    dt = sch.compute_dt(u, b, golden_cfl(N, family), 0.5)
    want = Blending2D(sch, alpha=alpha).step(u, b, dt)
    s = solver(crk, system, N, family, Ex, Ey, b)
    s.set_limiter("fixed", alpha)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP
    a = to_host(s.limiter_alpha())
    assert a.shape == (Ey, Ex) and np.all(a == alpha)


@pytest.mark.parametrize("Ex,Ey", [(1, 1), (2, 7), (17, 4), (33, 9)])
def test_fixed_alpha_mesh_shapes(crk, Ex, Ey):
    N, family = 3, "gl"
    u, b, dx, dy = flow(N, family, Ex, Ey)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family=family)
    dt = sch.compute_dt(u, b, golden_cfl(N, family), 0.5)
    want = Blending2D(sch, alpha=0.6).step(u, b, dt)
    s = solver(crk, "swe2d", N, family, Ex, Ey, b)
    s.set_limiter("fixed", 0.6)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP


@pytest.mark.parametrize("N", [2, 3, 4])
def test_indicator_and_step_on_a_dam_break(crk, N):
    """C_s 0.1: the indicator's alpha per element and the limited step
    (Algorithms 1 and 2 active at the thin layer) against the oracle."""
    Ex, Ey = 14, 11
    u, b, dx, dy = dam(N, Ex, Ey)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family="gll")
    lim = Blending2D(sch)
    dt = sch.compute_dt(u, b, golden_cfl(N, "gll"), 0.1)
    want = lim.step(u, b, dt)
    s = solver(crk, "swe2d", N, "gll", Ex, Ey, b, cs=0.1)
    s.set_limiter("blend")
    du = to_dev(u)
    s.step(du, dt, 1)
    got_alpha = to_host(s.limiter_alpha())
    assert np.max(np.abs(got_alpha - lim.last_alpha)) < 1e-12
    assert np.max(got_alpha) > 0.5 and np.min(got_alpha) == 0.0
    assert rel_l2(to_host(du), want) < TOL_STEP


def test_dam_break_positive_conservative_and_close_to_oracle(crk):
    N, E, steps = 3, 24, 60
    u, b, dx, dy = dam(N, E, E)
    bs = Basis(N, "gll")
    W = dx * dy * bs.w[:, None] * bs.w[None, :]
    s = solver(crk, "swe2d", N, "gll", E, E, b, cs=0.1)
    s.set_limiter("blend")
    du = to_dev(u)
    m0 = np.sum(W * u[0])
    for _ in range(steps // 10):
        s.step(du, 0.0, 10)
        assert np.min(to_host(du)[0]) > 0.0
    s.status()
    assert abs(np.sum(W * to_host(du)[0]) - m0) < 1e-12 * m0
    # the first 10 CFL steps against the oracle
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family="gll")
    lim = Blending2D(sch)
    v = u.copy()
    for _ in range(10):
        v = lim.step(v, b, sch.compute_dt(v, b, golden_cfl(N, "gll"), 0.1))
    s2 = solver(crk, "swe2d", N, "gll", E, E, b, cs=0.1)
    s2.set_limiter("blend")
    dv = to_dev(u)
    s2.step(dv, 0.0, 10)
    assert rel_l2(to_host(dv), v) < 1e-10


@pytest.mark.parametrize("N,family", [(1, "gl"), (3, "gl"), (2, "gll")])
@pytest.mark.parametrize("system", ["swe2d", "swe2d_wb"])
def test_limiter_with_chezy_friction(crk, N, family, system):
    Ex, Ey = 9, 5
    u, b, dx, dy = flow(N, family, Ex, Ey)
    sch = Scheme2D(SYSTEMS[system](G), N, dx, dy, family=family, source=ChezyFriction(3.0))
    dt = sch.compute_dt(u, b, golden_cfl_imex(N, family), 0.5)
    want = Blending2D(sch, alpha=0.5).step(u, b, dt)
    s = solver(crk, system, N, family, Ex, Ey, b, source="chezy", coef=3.0)
    s.set_limiter("fixed", 0.5)
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP


def test_dam_break_with_friction_and_indicator(crk):
    N, E = 3, 12
    u, b, dx, dy = dam(N, E, E)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family="gll", source=ChezyFriction(2.0))
    lim = Blending2D(sch)
    dt = sch.compute_dt(u, b, golden_cfl_imex(N, "gll"), 0.1)
    want = lim.step(u, b, dt)
    s = solver(crk, "swe2d", N, "gll", E, E, b, cs=0.1, source="chezy", coef=2.0)
    s.set_limiter("blend")
    du = to_dev(u)
    s.step(du, dt, 1)
    assert rel_l2(to_host(du), want) < TOL_STEP


def test_well_balanced_lake_at_rest_with_limiter(crk):
    N, Ex, Ey = 3, 20, 16
    bs = Basis(N, "gll")
    x, y, dx, dy = positions_2d(bs, Ex, Ey, 1.0)
    b = 0.3 * np.exp(-((x - 0.4) ** 2 + (y - 0.5) ** 2) / (2 * 0.08 ** 2)) + np.where(x > 0.7, 0.2, 0.0)
    u0 = np.stack([1.0 - b, np.zeros_like(b), np.zeros_like(b)])
    s = solver(crk, "swe2d_wb", N, "gll", Ex, Ey, b)
    s.set_limiter("blend")
    du = to_dev(u0)
    s.step(du, 0.0, 50)
    assert np.max(np.abs(to_host(du) - u0)) < 1e-13
    assert np.max(to_host(s.limiter_alpha())) > 0.5


def test_well_balanced_dam_break_against_oracle(crk):
    """Dam break over bathymetry in the well-balanced form, indicator on."""
    N, E = 2, 13
    u, _, dx, dy = dam(N, E, E, hR=0.05)
    bs = Basis(N, "gll")
    x, y, _, _ = positions_2d(bs, E, E, 1.0)
    b = 0.04 * np.sin(2 * np.pi * x) ** 2
    sch = Scheme2D(ShallowWater2DWB(G), N, dx, dy, family="gll")
    lim = Blending2D(sch)
    v = u.copy()
    for _ in range(5):
        v = lim.step(v, b, sch.compute_dt(v, b, golden_cfl(N, "gll"), 0.1))
    s = solver(crk, "swe2d_wb", N, "gll", E, E, b, cs=0.1)
    s.set_limiter("blend")
    du = to_dev(u)
    s.step(du, 0.0, 5)
    assert rel_l2(to_host(du), v) < 1e-11


def test_limiter_configuration_errors_2d(crk):
    s = crk.Solver("swe2d", 2, gravity=G)
    s.set_mesh([4, 4], [0.0, 0.0], [1.0, 1.0])
    s.set_limiter("blend")
    # a limited slab of at least two rows, in either order of the calls
    s.set_subdomain(True)
    s.set_limiter(None)
    s.set_limiter("fixed", 0.5)
    s.set_subdomain(False)
    with pytest.raises(crk.CrkfrError) as e:
        s.set_limiter("fixed", -0.1)
    assert e.value.status == -1
    # a one-row slab cannot send the two indicator rows its neighbours need
    t = crk.Solver("swe2d", 2, gravity=G)
    t.set_mesh([4, 1], [0.0, 0.0], [1.0, 0.25])
    t.set_subdomain(True)
    with pytest.raises(crk.CrkfrError) as e:
        t.set_limiter("blend")
    assert e.value.status == -2
    t.set_subdomain(False)
    t.set_limiter("blend")
    with pytest.raises(crk.CrkfrError) as e:
        t.set_subdomain(True)
    assert e.value.status == -2
    # whole meshes and 1D ranges have no limiter halo blocks (a range's
    # exchange carries the indicator with the end elements' states)
    with pytest.raises(crk.CrkfrError) as e:
        s.limiter_halo_buffers(0)
    assert e.value.status == -6
    r = crk.Solver("swe1d", 2, gravity=G)
    r.set_mesh([8], [0.0], [1.0])
    r.set_subdomain(True)
    r.set_limiter("blend")
    with pytest.raises(crk.CrkfrError) as e:
        r.limiter_halo_buffers(1)
    assert e.value.status == -6


def limited_slab(crk, system, N, Ex, Ey, c, first, count, mode, alpha, source=None, coef=0.0,
                 family="gll", cs=0.1):
    cfl = golden_cfl_imex(N, family) if source else golden_cfl(N, family)
    s = crk.Solver(system, N, nodes=family, gravity=G, cfl_safety=cs, cfl_number=cfl,
                   source=source, source_coef=coef)
    dy = 1.0 / Ey
    s.set_mesh([Ex, count], [0.0, first * dy], [1.0, (first + count) * dy])
    s.set_subdomain(True)
    rows = [(first - 1) % Ey] + list(range(first, first + count)) + [(first + count) % Ey]
    s.set_coefficients(to_dev(np.ascontiguousarray(c[rows])))
    s.set_limiter(mode, alpha)
    return s


def ring(bufs):
    """In-process exchange of one kind of halo block between slabs stacked
    in order on a periodic ring."""
    k_ = len(bufs)
    for k in range(k_):
        bufs[k][2].copy_(bufs[(k - 1) % k_][1])    # recv_bottom <- send_top of the slab below
        bufs[k][3].copy_(bufs[(k + 1) % k_][0])    # recv_top <- send_bottom of the slab above


@pytest.mark.parametrize("system,N,mode,alpha,source", [
    ("swe2d", 3, "blend", 0.0, None), ("swe2d", 2, "fixed", 0.4, None),
    ("swe2d_wb", 2, "blend", 0.0, None), ("swe2d", 3, "blend", 0.0, "chezy")])
def test_limited_slabs_equal_single_domain(crk, system, N, mode, alpha, source):
    """A circular dam break across three slabs (of 5, 2 and 9 rows, the
    second only as tall as the two indicator rows a slab sends): raw
    indicator, exchange of its boundary rows, local phase, exchange of the
    traces and the limiter's face data, face phase.  The slabs' states and
    blending coefficients equal the single-domain limited step bit for bit."""
    Ex, Ey, steps = 16, 16, 4
    u, b, dx, dy = dam(N, Ex, Ey)
    coef = 2.0 if source else 0.0
    m = solver(crk, system, N, "gll", Ex, Ey, b, cs=0.1, source=source, coef=coef)
    m.set_limiter(mode, alpha)
    want = to_dev(u)
    parts = [(0, 5), (5, 2), (7, 9)]
    slabs = [limited_slab(crk, system, N, Ex, Ey, b, f, c, mode, alpha, source, coef)
             for f, c in parts]
    states = [to_dev(np.ascontiguousarray(u[:, f:f + c])) for f, c in parts]
    traces = [s.halo_buffers() for s in slabs]
    raw = [s.limiter_halo_buffers(0) for s in slabs]
    face = [s.limiter_halo_buffers(1) for s in slabs]
    for _ in range(steps):
        # the CFL step of the state (the dam's speeds grow as it breaks)
        dt = m.compute_dt(want)
        m.step(want, dt, 1)
        for s, x in zip(slabs, states):
            s.step_indicator(x)
        ring(raw)
        for s, x in zip(slabs, states):
            s.step_local(x, dt)
        ring(traces)
        ring(face)
        for s, x in zip(slabs, states):
            s.step_faces(x)
    got = np.concatenate([to_host(x) for x in states], axis=1)
    assert np.all(np.isfinite(got)) and np.min(got[0]) > 0.0
    assert np.array_equal(got, to_host(want)), rel_l2(got, to_host(want))
    a = np.concatenate([to_host(s.limiter_alpha()) for s in slabs], axis=0)
    a_want = to_host(m.limiter_alpha())
    assert np.array_equal(a, a_want)
    if mode == "blend":
        # the dam (y in 0.30 .. 0.70) spans the slab boundaries at y = 5/16, 7/16
        assert np.max(a_want) > 0.5 and np.min(a_want) == 0.0


@pytest.mark.parametrize("system,N,mode,alpha", [("swe2d", 3, "fixed", 0.4),
                                                ("swe2d_wb", 2, "blend", 0.0),
                                                ("swe2d", 4, "blend", 0.0)])
def test_limited_slabs_gl_nodes(crk, system, N, mode, alpha):
    """GL nodes (traces through l(0), l(1), Radau corrections at every node)
    on the smooth flow over a varying bottom, split into slabs of 3 and 5
    rows through SlabStepper-like phases: bit for bit the single domain
    (dy = 1/8, so that every slab's bounds and 1/dy are exact)."""
    Ex, Ey, steps = 9, 8, 3
    u, b, dx, dy = flow(N, "gl", Ex, Ey)
    m = solver(crk, system, N, "gl", Ex, Ey, b)
    m.set_limiter(mode, alpha)
    want = to_dev(u)
    parts = [(0, 3), (3, 5)]
    slabs = [limited_slab(crk, system, N, Ex, Ey, b, f, c, mode, alpha, family="gl", cs=0.5)
             for f, c in parts]
    states = [to_dev(np.ascontiguousarray(u[:, f:f + c])) for f, c in parts]
    traces = [s.halo_buffers() for s in slabs]
    raw = [s.limiter_halo_buffers(0) for s in slabs]
    face = [s.limiter_halo_buffers(1) for s in slabs]
    for _ in range(steps):
        dt = m.compute_dt(want)
        m.step(want, dt, 1)
        for s, x in zip(slabs, states):
            s.step_indicator(x)
        ring(raw)
        for s, x in zip(slabs, states):
            s.step_local(x, dt)
        ring(traces)
        ring(face)
        for s, x in zip(slabs, states):
            s.step_faces(x)
    got = np.concatenate([to_host(x) for x in states], axis=1)
    assert np.all(np.isfinite(got))
    assert np.array_equal(got, to_host(want)), rel_l2(got, to_host(want))


def test_single_limited_slab_through_the_stepper(crk):
    """One limited slab, its own periodic neighbour, stepped by SlabStepper
    (which adds the limiter's exchanges), in CFL steps."""
    from paper_2512_08611_gb300.distributed import SlabStepper
    N, Ex, Ey = 3, 12, 10
    u, b, dx, dy = dam(N, Ex, Ey)
    m = solver(crk, "swe2d", N, "gll", Ex, Ey, b, cs=0.1)
    m.set_limiter("blend")
    s = limited_slab(crk, "swe2d", N, Ex, Ey, b, 0, Ey, "blend", 0.0)
    x, want = to_dev(u), to_dev(u)
    st = SlabStepper(s)
    for _ in range(3):
        dt = m.compute_dt(want)
        m.step(want, dt, 1)
        st.step(x, 0.0, 1)
        assert st.last_dt == dt
    assert np.array_equal(to_host(x), to_host(want))


def test_phased_and_adjoint_steps_refuse_the_limiter(crk):
    N, E = 2, 6
    u, b, dx, dy = flow(N, "gl", E, E)
    s = solver(crk, "swe2d", N, "gl", E, E, b)
    s.set_limiter("fixed", 0.3)
    du = to_dev(u)
    with pytest.raises(crk.CrkfrError) as e:
        s.step_local(du, 1e-4)
    assert e.value.status == -2
    ub = to_dev(np.ones_like(u))
    with pytest.raises(crk.CrkfrError) as e:
        s.step_adjoint(du, ub, 1e-4)
    assert e.value.status == -2


def _patch(a, ey, ex, r=2):
    """The (2r+1)^2 elements around (ey, ex) of a periodic mesh, as a periodic
    mesh of their own (axes -4, -3 of a are (Ey, Ex))."""
    Ey, Ex = a.shape[-4], a.shape[-3]
    iy = (ey + np.arange(-r, r + 1)) % Ey
    ix = (ex + np.arange(-r, r + 1)) % Ex
    return a[..., iy[:, None], ix[None, :], :, :]


def test_full_size_dam_break_sampled(crk):
    """The 1024 x 1024, N = 3 mesh (GLL) with a circular dam break, one CFL
    step with the indicator: the limited step of an element reads the
    indicator of elements up to two faces away and the face data of its four
    neighbours, so the oracle's step of the 5 x 5 patch around a sampled
    element (periodic on its own) gives that element's result.  96 samples,
    most of them on the front, plus the corners."""
    N, E = 3, 1024
    u, b, dx, dy = dam(N, E, E, r=0.3)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family="gll")
    cfl = golden_cfl(N, "gll")
    s = solver(crk, "swe2d", N, "gll", E, E, b, cs=0.1)
    s.set_limiter("blend")
    du = to_dev(u)
    dt = s.compute_dt(du)
    s.step(du, dt, 1)
    got = to_host(du)
    alpha = to_host(s.limiter_alpha())
    rng = np.random.default_rng(5)
    front = np.argwhere(alpha > 0.0)
    pick = front[rng.choice(len(front), 80, replace=False)]
    ey = np.concatenate([[0, 0, E - 1, E - 1], pick[:, 0], rng.integers(0, E, 12)])
    ex = np.concatenate([[0, E - 1, 0, E - 1], pick[:, 1], rng.integers(0, E, 12)])
    sch5 = Scheme2D(ShallowWater2D(G), N, dx, dy, family="gll")
    for y, x in zip(ey, ex):
        lim = Blending2D(sch5)
        out = lim.step(_patch(u, y, x), _patch(b[None], y, x)[0], dt)
        assert rel_l2(got[:, y, x], out[:, 2, 2]) < TOL_STEP, (y, x)
        assert abs(alpha[y, x] - lim.last_alpha[2, 2]) < 1e-12
    assert np.max(alpha) > 0.5
    assert dt == pytest.approx(sch.compute_dt(u, b, cfl, 0.1), rel=1e-14)


def test_thousand_limited_steps_2d(crk):
    """1000 CFL steps of the limited 2D step with the indicator on a circular
    dam break onto a thin layer (8 x 8, N = 3, GLL, C_s 0.1): positive, and
    1e-10 relative L2 from the oracle after 1000 steps."""
    N, E = 3, 8
    u, b, dx, dy = dam(N, E, E)
    sch = Scheme2D(ShallowWater2D(G), N, dx, dy, family="gll")
    lim = Blending2D(sch)
    cfl = golden_cfl(N, "gll")
    v = u.copy()
    for _ in range(1000):
        v = lim.step(v, b, sch.compute_dt(v, b, cfl, 0.1))
    s = solver(crk, "swe2d", N, "gll", E, E, b, cs=0.1)
    s.set_limiter("blend")
    du = to_dev(u)
    s.step(du, 0.0, 1000)
    s.status()
    got = to_host(du)
    assert np.min(got[0]) > 0.0
    assert rel_l2(got, v) < 1e-10


def test_full_size_limited_workload_sampled(crk):
    """The limited bench workload as the benchmark launches it (1024^2, N = 3,
    GL, the default workload's inputs, indicator on): one CFL step; 64
    sampled elements (incl. the corners) against the oracle's step of the
    5 x 5 patch around each."""
    from paper_2512_08611_gb300.workloads import SWE2DInput, accept_seed
    N, E = 3, 1024
    bs = Basis(N)
    x, y, dx, dy = positions_2d(bs, E, E, 100.0)
    inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=100.0), (x, y), 0)
    u, b = inp.state(x, y)
    del x, y
    s = crk.Solver("swe2d", N, gravity=G, cfl_safety=0.5, cfl_number=golden_cfl(N, "gl"))
    s.set_mesh([E, E], [0.0, 0.0], [100.0, 100.0])
    s.set_coefficients(to_dev(b))
    s.set_limiter("blend")
    du = to_dev(u)
    dt = s.compute_dt(du)
    s.step(du, 0.0, 1)
    got = to_host(du)
    alpha = to_host(s.limiter_alpha())
    rng = np.random.default_rng(9)
    ey = np.concatenate([[0, 0, E - 1, E - 1], rng.integers(0, E, 60)])
    ex = np.concatenate([[0, E - 1, 0, E - 1], rng.integers(0, E, 60)])
    sch5 = Scheme2D(ShallowWater2D(G), N, dx, dy)
    for yy, xx in zip(ey, ex):
        lim = Blending2D(sch5)
        out = lim.step(_patch(u, yy, xx), _patch(b[None], yy, xx)[0], dt)
        assert rel_l2(got[:, yy, xx], out[:, 2, 2]) < TOL_STEP, (yy, xx)
        assert abs(alpha[yy, xx] - lim.last_alpha[2, 2]) < 1e-12


def test_checkpoint_resume_with_the_limiter(crk):
    """state_dict of a limited run carries the limiter setting: a fresh
    context loaded from it (limiter not set by hand) repeats the run bitwise."""
    N, E = 3, 10
    u, b, dx, dy = dam(N, E, E)
    s1 = solver(crk, "swe2d", N, "gll", E, E, b, cs=0.1)
    s1.set_limiter("blend")
    d1 = to_dev(u)
    s1.step(d1, 0.0, 5)
    sd = s1.state_dict(d1)
    s1.step(d1, 0.0, 5)
    s2 = solver(crk, "swe2d", N, "gll", E, E, b, cs=0.1)
    d2 = to_dev(np.zeros_like(u))
    s2.load_state_dict(sd, d2)
    assert s2.limiter == ("blend", 0.0)
    s2.step(d2, 0.0, 5)
    assert np.array_equal(to_host(d1), to_host(d2))
