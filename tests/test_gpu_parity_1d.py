"""GPU parity of the 1D cRK-FR path (C ABI, sm_103a) against the oracle.

Tolerances: 1e-12 relative L2 per step, 1e-10 after 1000 steps (the CUDA
path and the oracle differ only in FP64 rounding order: FMA chains, the
reciprocal by Newton iteration, the order of the time-average sums)."""
import numpy as np
import pytest

from gpu_common import G, golden_cfl, load, positions_1d, rel_l2, residual_close, to_dev, to_host
from oracle.basis import Basis
from oracle.crkfr import Scheme1D
from oracle.exact import SineCoefficient, l2_error_1d
from oracle.systems import ShallowWater1D, VarCoeffAdvection
from paper_2512_08611_gb300.workloads import SWE1DInput, VarAdvInput, accept_seed

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-12


@pytest.fixture(scope="module")
def crk():
    return load()


def swe_case(N, family, E, seed=1, L=100.0, still=False):
    bs = Basis(N, family)
    x, dx = positions_1d(bs, E, 0.0, L)
    inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=L, still=still), (x,), seed)
    u, b = inp.state(x)
    return u, b, dx


def varadv_case(N, family, E):
    bs = Basis(N, family)
    x, dx = positions_1d(bs, E, 0.0, 1.0)
    inp = VarAdvInput()
    return inp.v0(x)[None], inp.a(x), dx


def solver(crk, system, N, family, E, lo, hi, c, cfl=None, cs=0.5):
    s = crk.Solver(system, N, nodes=family, gravity=G, cfl_safety=cs,
                   cfl_number=golden_cfl(N, family) if cfl is None else cfl)
    s.set_mesh([E], [lo], [hi])
    s.set_coefficients(to_dev(c))
    return s


CASES = [(N, fam) for N in range(5) for fam in ("gl", "gll") if not (fam == "gll" and N == 0)]


@pytest.mark.parametrize("N,family", CASES)
@pytest.mark.parametrize("E", [1, 3, 126, 127, 300])
def test_swe_one_step_and_residual(crk, N, family, E):
    u, b, dx = swe_case(N, family, E)
    sch = Scheme1D(ShallowWater1D(G), N, dx, family=family)
    dt = sch.compute_dt(u, b, golden_cfl(N, family), 0.5)
    want = sch.step(u, b, dt)
    s = solver(crk, "swe1d", N, family, E, 0.0, 100.0, b)
    du = to_dev(u)
    s.step(du, dt, 1)
    got = to_host(du)
    assert rel_l2(got, want) < TOL_STEP
    # residual r = (u^{n+1} - u^n)/dt, evaluated directly
    r = to_host(s.residual(to_dev(u), dt))
    r_want = -sch.residual(u, b, dt)
    assert residual_close(r, r_want, u, dt)
    s.status()


@pytest.mark.parametrize("N,family", CASES)
@pytest.mark.parametrize("E", [1, 5, 130])
def test_varadv_one_step_and_residual(crk, N, family, E):
    v, a, dx = varadv_case(N, family, E)
    sch = Scheme1D(VarCoeffAdvection(), N, dx, family=family)
    dt = sch.compute_dt(v, a, golden_cfl(N, family), 0.5)
    want = sch.step(v, a, dt)
    s = solver(crk, "varadv1d", N, family, E, 0.0, 1.0, a)
    dv = to_dev(v)
    s.step(dv, dt, 1)
    assert rel_l2(to_host(dv), want) < TOL_STEP
    r = to_host(s.residual(to_dev(v), dt))
    assert residual_close(r, -sch.residual(v, a, dt), v, dt)


@pytest.mark.parametrize("N,family", [(1, "gl"), (2, "gll"), (3, "gl"), (4, "gl"), (4, "gll")])
def test_swe_cfl_steps(crk, N, family):
    """Steps with the device-side time step of Eq. time.step.2d."""
    E, nsteps = 257, 40
    u, b, dx = swe_case(N, family, E, seed=3)
    sch = Scheme1D(ShallowWater1D(G), N, dx, family=family)
    cfl = golden_cfl(N, family)
    s = solver(crk, "swe1d", N, family, E, 0.0, 100.0, b)
    du = to_dev(u)
    assert s.compute_dt(du) == pytest.approx(sch.compute_dt(u, b, cfl, 0.5), rel=1e-14)
    t = 0.0
    v = u
    for _ in range(nsteps):
        dt = sch.compute_dt(v, b, cfl, 0.5)
        v = sch.step(v, b, dt)
        t += dt
    s.step(du, 0.0, nsteps)
    assert rel_l2(to_host(du), v) < 1e-11
    tg, _ = s.time()
    assert tg == pytest.approx(t, rel=1e-13)
    s.status()


def test_config1_to_final_time(crk):
    """Variable-coefficient advection, N = 3, E = 100, CFL 0.5, T = 1, last
    step shortened to land on T; GPU vs oracle and vs characteristics."""
    N, E, T = 3, 100, 1.0
    v, a, dx = varadv_case(N, "gl", E)
    sch = Scheme1D(VarCoeffAdvection(), N, dx)
    cfl = golden_cfl(N, "gl")
    w, t, k = v, 0.0, 0
    while t < T:
        dt = min(sch.compute_dt(w, a, cfl, 0.5), T - t)
        w = sch.step(w, a, dt)
        t += dt
        k += 1
    s = solver(crk, "varadv1d", N, "gl", E, 0.0, 1.0, a)
    dv = to_dev(v)
    steps = s.advance(dv, T)
    got = to_host(dv)
    assert steps == k
    assert s.time()[0] == T
    assert rel_l2(got, w) < 1e-10
    sc = SineCoefficient(0.5)
    err = l2_error_1d(got[0], lambda x: np.sin(2 * np.pi * sc.foot(x, T)), 0.0, dx, Basis(N).xi)
    assert err < 1e-6


@pytest.mark.parametrize("N", [2, 3])
def test_config1_design_order_on_gpu(crk, N):
    """The first configuration's convergence study on the GPU: E = 25, 50,
    100, 200, CFL 0.5, T = 1, L2 error against the characteristics solution;
    the observed order on the finest pair is at least N + 1 - 0.3."""
    sc = SineCoefficient(0.5)
    errs = []
    for E in (25, 50, 100, 200):
        v, a, dx = varadv_case(N, "gl", E)
        s = solver(crk, "varadv1d", N, "gl", E, 0.0, 1.0, a)
        dv = to_dev(v)
        s.advance(dv, 1.0)
        errs.append(l2_error_1d(to_host(dv)[0], lambda x: np.sin(2 * np.pi * sc.foot(x, 1.0)),
                                0.0, dx, Basis(N).xi))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > N + 1 - 0.3, (errs, rates)


def test_swe_self_convergence_on_gpu(crk):
    """Shallow water over a Gaussian bump, a smooth moving wave to T = 0.05
    on E = 10, 20, 40, 80 and a 320-element reference, N = 3, all on the GPU:
    the differences to the reference, interpolated at 37 fixed points, fall
    at order about N + 1 (> 3.7 on the finest pair)."""
    N, T = 3, 0.05
    pts = np.linspace(0.013, 0.987, 37)
    vals = []
    for E in (10, 20, 40, 80, 320):
        bs = Basis(N)
        x, dx = positions_1d(bs, E, 0.0, 1.0)
        b = 0.2 * np.exp(-((x - 0.5) ** 2) / (2 * 0.08 ** 2))
        u = np.stack([1.0 + 0.1 * np.sin(2 * np.pi * x) - b, 0.3 * np.cos(2 * np.pi * x)])
        s = solver(crk, "swe1d", N, "gl", E, 0.0, 1.0, b)
        du = to_dev(u)
        s.advance(du, T)
        got = to_host(du)
        e = np.floor(pts / dx).astype(int)
        xi = pts / dx - e
        Lm = np.ones((len(pts), N + 1))
        for j in range(N + 1):
            for k in range(N + 1):
                if k != j:
                    Lm[:, j] *= (xi - bs.xi[k]) / (bs.xi[j] - bs.xi[k])
        vals.append(np.array([got[:, e[i], :] @ Lm[i] for i in range(len(pts))]))
    errs = np.array([np.max(np.abs(v - vals[-1])) for v in vals[:-1]])
    rates = np.log2(errs[:-1] / errs[1:])
    assert rates[-1] > 3.7, (errs, rates)


@pytest.fixture(scope="module")
def config2(crk):
    N, E = 4, 100000
    u, b, dx = swe_case(N, "gl", E, seed=0)
    return N, E, u, b, dx


def test_config2_one_step(crk, config2):
    N, E, u, b, dx = config2
    sch = Scheme1D(ShallowWater1D(G), N, dx)
    cfl = golden_cfl(N, "gl")
    dt = sch.compute_dt(u, b, cfl, 0.5)
    want = sch.step(u, b, dt)
    s = solver(crk, "swe1d", N, "gl", E, 0.0, 100.0, b)
    du = to_dev(u)
    s.step(du, 0.0, 1)
    assert s.time()[1] == pytest.approx(dt, rel=1e-14)
    assert rel_l2(to_host(du), want) < TOL_STEP


def test_config2_ten_steps(crk, config2):
    N, E, u, b, dx = config2
    sch = Scheme1D(ShallowWater1D(G), N, dx)
    cfl = golden_cfl(N, "gl")
    v = u
    for _ in range(10):
        v = sch.step(v, b, sch.compute_dt(v, b, cfl, 0.5))
    s = solver(crk, "swe1d", N, "gl", E, 0.0, 100.0, b)
    du = to_dev(u)
    s.step(du, 0.0, 10)
    assert rel_l2(to_host(du), v) < 1e-11
    s.status()


def test_thousand_steps(crk):
    """1000 CFL steps of the 1D workload's recipe on 4096 elements (N = 4):
    1e-10 relative L2 after 1000 steps."""
    N, E = 4, 4096
    u, b, dx = swe_case(N, "gl", E, seed=0)
    sch = Scheme1D(ShallowWater1D(G), N, dx)
    cfl = golden_cfl(N, "gl")
    v = u
    for _ in range(1000):
        v = sch.step(v, b, sch.compute_dt(v, b, cfl, 0.5))
    s = solver(crk, "swe1d", N, "gl", E, 0.0, 100.0, b)
    du = to_dev(u)
    s.step(du, 0.0, 1000)
    got = to_host(du)
    assert rel_l2(got, v) < 1e-10
    s.status()


def test_config2_lake_at_rest(crk):
    """Lake at rest (perturbation 0): not well balanced by construction
    (Sec. 6 lists that as open); GPU and oracle agree on the defect."""
    N, E = 4, 100000
    u, b, dx = swe_case(N, "gl", E, seed=0, still=True)
    sch = Scheme1D(ShallowWater1D(G), N, dx)
    cfl = golden_cfl(N, "gl")
    v = u
    for _ in range(20):
        v = sch.step(v, b, sch.compute_dt(v, b, cfl, 0.5))
    s = solver(crk, "swe1d", N, "gl", E, 0.0, 100.0, b)
    du = to_dev(u)
    s.step(du, 0.0, 20)
    got = to_host(du)
    defect_gpu = np.max(np.abs(got - u))
    defect_oracle = np.max(np.abs(v - u))
    assert defect_gpu == pytest.approx(defect_oracle, rel=1e-3, abs=1e-14)
    assert np.max(np.abs(got - v)) < 1e-13


def test_mass_conservation_gpu(crk):
    N, E = 3, 5000
    u, b, dx = swe_case(N, "gl", E, seed=2)
    w = Basis(N).w
    s = solver(crk, "swe1d", N, "gl", E, 0.0, 100.0, b)
    du = to_dev(u)
    s.step(du, 0.0, 200)
    got = to_host(du)
    m0, m1 = np.sum(dx * w * u[0]), np.sum(dx * w * got[0])
    assert abs(m1 - m0) < 1e-13 * abs(m0)


def test_host_entry_point_matches_device(crk):
    N, E = 3, 300
    u, b, dx = swe_case(N, "gl", E)
    s = solver(crk, "swe1d", N, "gl", E, 0.0, 100.0, b)
    du = to_dev(u)
    s.step(du, 0.01, 3)
    s2 = solver(crk, "swe1d", N, "gl", E, 0.0, 100.0, b)
    out = s2.step_host(np.ascontiguousarray(u), dt=0.01, nsteps=3)
    assert np.array_equal(out, to_host(du))


def test_nonphysical_state_is_reported(crk):
    N, E = 2, 40
    u, b, dx = swe_case(N, "gl", E)
    u[0, 7, 1] = -0.5
    s = solver(crk, "swe1d", N, "gl", E, 0.0, 100.0, b)
    du = to_dev(u)
    s.step(du, 1e-3, 1)
    with pytest.raises(crk.CrkfrError) as e:
        s.status()
    assert e.value.status == -4
    s.status()   # cleared


def test_even_and_odd_step_counts(crk):
    """The 1D step alternates between the caller's buffer and a work buffer;
    any step count must end in the caller's buffer."""
    N, E = 2, 200
    u, b, dx = swe_case(N, "gl", E)
    sch = Scheme1D(ShallowWater1D(G), N, dx)
    for k in (1, 2, 3):
        v = u
        for _ in range(k):
            v = sch.step(v, b, 0.02)
        s = solver(crk, "swe1d", N, "gl", E, 0.0, 100.0, b)
        du = to_dev(u)
        s.step(du, 0.02, k)
        assert rel_l2(to_host(du), v) < 1e-12
