"""The 2D step split into horizontal slabs (local phase, one exchange of face
traces, face phase) equals the single-domain step bitwise on the GPU: two
subdomain contexts exchanging their halo blocks in one process, and a single
slab that is its own periodic neighbour."""
import numpy as np
import pytest

from gpu_common import G, golden_cfl, load, rel_l2, to_dev, to_host
from oracle.basis import Basis
from paper_2512_08611_gb300.workloads import SWE2DInput, accept_seed

pytestmark = pytest.mark.gpu


def case(N, Ex, Ey, L):
    bs = Basis(N)
    dx, dy = L / Ex, L / Ey
    x = (np.arange(Ex)[None, :, None, None] + bs.xi[None, None, None, :]) * dx
    y = (np.arange(Ey)[:, None, None, None] + bs.xi[None, None, :, None]) * dy
    x, y = np.broadcast_arrays(x, y)
    inp, _ = accept_seed(lambda s: SWE2DInput(seed=s, L=L, n_gauss=6), (x, y), 0)
    u, b = inp.state(x, y)
    u[1] = 0.05 * u[0] * np.sin(2 * np.pi * y / L)
    u[2] = 0.05 * u[0] * np.cos(2 * np.pi * x / L)
    return u, b


def mono(crk, N, Ex, Ey, L, u, b, dt, steps, system="swe2d", source=None):
    s = crk.Solver(system, N, gravity=G, cfl_number=golden_cfl(N, "gl"), source=source,
                   source_coef=0.5 if source else 0.0)
    s.set_mesh([Ex, Ey], [0.0, 0.0], [L, L])
    s.set_coefficients(to_dev(b))
    du = to_dev(u)
    s.step(du, dt, steps)
    return to_host(du)


def slab(crk, N, Ex, Ey, L, b, first, count, system="swe2d", source=None):
    dy = L / Ey
    s = crk.Solver(system, N, gravity=G, cfl_number=golden_cfl(N, "gl"), source=source,
                   source_coef=0.5 if source else 0.0)
    s.set_mesh([Ex, count], [0.0, first * dy], [L, (first + count) * dy])
    s.set_subdomain(True)
    rows = [(first - 1) % Ey] + list(range(first, first + count)) + [(first + count) % Ey]
    s.set_coefficients(to_dev(np.ascontiguousarray(b[rows])))
    return s


@pytest.mark.parametrize("N,system,source", [(1, "swe2d", None), (3, "swe2d", None),
                                             (3, "swe2d_wb", None), (2, "swe2d", "chezy"),
                                             (3, "swe2d_wb", "chezy")])
def test_two_slabs_equal_single_domain(N, system, source):
    """Also for the well-balanced form and with Chezy friction: the slab
    kernels are the same instantiations as the single-domain ones."""
    crk = load()
    Ex, Ey, L, dt, steps = 16, 16, 64.0, 0.02, 5      # dx = dy = 4: exact slab bounds
    u, b = case(N, Ex, Ey, L)
    want = mono(crk, N, Ex, Ey, L, u, b, dt, steps, system, source)
    parts = [(0, 7), (7, 9)]
    solvers = [slab(crk, N, Ex, Ey, L, b, f, c, system, source) for f, c in parts]
    states = [to_dev(np.ascontiguousarray(u[:, f:f + c])) for f, c in parts]
    bufs = [s.halo_buffers() for s in solvers]       # (send_bottom, send_top, recv_bottom, recv_top)
    for _ in range(steps):
        for s, x in zip(solvers, states):
            s.step_local(x, dt)
        for k in range(2):
            below, above = (k - 1) % 2, (k + 1) % 2
            bufs[k][2].copy_(bufs[below][1])           # recv_bottom <- send_top of the slab below
            bufs[k][3].copy_(bufs[above][0])           # recv_top <- send_bottom of the slab above
        for s, x in zip(solvers, states):
            s.step_faces(x)
    got = np.concatenate([to_host(x) for x in states], axis=1)
    assert np.array_equal(got, want), rel_l2(got, want)


def exchange_2d(bufs):
    for k in range(len(bufs)):
        below, above = (k - 1) % len(bufs), (k + 1) % len(bufs)
        bufs[k][2].copy_(bufs[below][1])
        bufs[k][3].copy_(bufs[above][0])


@pytest.mark.parametrize("N,system", [(3, "swe2d"), (2, "swe2d_wb")])
def test_two_slabs_cfl_steps_take_the_whole_mesh_step(N, system):
    """CFL steps of a split mesh: the step is the minimum of the slabs' own
    steps (crkfr_compute_dt), which equals the whole mesh's crkfr_compute_dt
    bit for bit; the slabs then equal the single domain stepped with those
    steps bitwise, and its own CFL run (whose later steps come from the face
    kernel's rates) to round-off."""
    crk = load()
    Ex, Ey, L, steps = 16, 16, 64.0, 5
    u, b = case(N, Ex, Ey, L)
    m = crk.Solver(system, N, gravity=G, cfl_number=golden_cfl(N, "gl"))
    m.set_mesh([Ex, Ey], [0.0, 0.0], [L, L])
    m.set_coefficients(to_dev(b))
    want = to_dev(u)
    parts = [(0, 5), (5, 11)]
    solvers = [slab(crk, N, Ex, Ey, L, b, f, c, system) for f, c in parts]
    states = [to_dev(np.ascontiguousarray(u[:, f:f + c])) for f, c in parts]
    bufs = [s.halo_buffers() for s in solvers]
    for _ in range(steps):
        dt = min(s.compute_dt(x) for s, x in zip(solvers, states))
        assert dt == m.compute_dt(want)
        m.step(want, dt, 1)
        for s, x in zip(solvers, states):
            s.step_local(x, dt)
        exchange_2d(bufs)
        for s, x in zip(solvers, states):
            s.step_faces(x)
    got = np.concatenate([to_host(x) for x in states], axis=1)
    assert np.array_equal(got, to_host(want)), rel_l2(got, to_host(want))
    cfl = mono(crk, N, Ex, Ey, L, u, b, 0.0, steps, system)
    assert rel_l2(got, cfl) < 1e-12


def test_single_slab_is_its_own_neighbour():
    from paper_2512_08611_gb300.distributed import SlabStepper
    crk = load()
    N, Ex, Ey, L, dt, steps = 3, 24, 8, 64.0, 0.02, 4
    u, b = case(N, Ex, Ey, L)
    want = mono(crk, N, Ex, Ey, L, u, b, dt, steps)
    s = slab(crk, N, Ex, Ey, L, b, 0, Ey)
    x = to_dev(u)
    SlabStepper(s).step(x, dt, steps)
    assert np.array_equal(to_host(x), want)
    # CFL steps through the stepper: one rank, so its own step is the mesh's
    m = crk.Solver("swe2d", N, gravity=G, cfl_number=golden_cfl(N, "gl"))
    m.set_mesh([Ex, Ey], [0.0, 0.0], [L, L])
    m.set_coefficients(to_dev(b))
    y, z = to_dev(u), to_dev(u)
    st = SlabStepper(s)
    for _ in range(3):
        dt = m.compute_dt(z)
        m.step(z, dt, 1)
        st.step(y, 0.0, 1)
        assert st.last_dt == dt
    assert np.array_equal(to_host(y), to_host(z))


def test_monolithic_step_refused_in_subdomain_mode():
    crk = load()
    u, b = case(2, 8, 8, 64.0)
    s = slab(crk, 2, 8, 8, 64.0, b, 0, 8)
    with pytest.raises(crk.CrkfrError) as e:
        s.step(to_dev(u), 0.01, 1)
    assert e.value.status == -6


# ---------------------------------------------------------------------------
# 1D subdomains: contiguous element ranges; a step is the packing of the two
# end elements, one exchange with each ring neighbour, and the fused step
# with the neighbours' end elements as ghosts
# ---------------------------------------------------------------------------
def case_1d(N, E, L, system):
    from paper_2512_08611_gb300.workloads import SWE1DInput
    bs = Basis(N)
    x = (np.arange(E)[:, None] + bs.xi[None, :]) * (L / E)
    if system == "varadv1d":
        from paper_2512_08611_gb300.workloads import VarAdvInput
        inp = VarAdvInput(L=L)
        return inp.v0(x)[None], inp.a(x)
    inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=L), (x,), 3)
    u, b = inp.state(x)
    u[1] = 0.1 * u[0] * np.sin(2 * np.pi * x / L)
    return u, b


def mono_1d(crk, N, E, L, u, b, dt, steps, system, source=None):
    s = crk.Solver(system, N, gravity=G, cfl_number=golden_cfl(N, "gl"), source=source,
                   source_coef=0.5 if source else 0.0)
    s.set_mesh([E], [0.0], [L])
    s.set_coefficients(to_dev(b))
    du = to_dev(u)
    s.step(du, dt, steps)
    return to_host(du)


def slab_1d(crk, N, E, L, b, first, count, system, source=None):
    dx = L / E
    s = crk.Solver(system, N, gravity=G, cfl_number=golden_cfl(N, "gl"), source=source,
                   source_coef=0.5 if source else 0.0)
    s.set_mesh([count], [first * dx], [(first + count) * dx])
    s.set_subdomain(True)
    elems = [(first - 1) % E] + list(range(first, first + count)) + [(first + count) % E]
    s.set_coefficients(to_dev(np.ascontiguousarray(b[elems])))
    return s


@pytest.mark.parametrize("N,system,source", [(1, "swe1d", None), (4, "swe1d", None),
                                             (3, "swe1d_wb", None), (2, "varadv1d", None),
                                             (2, "swe1d", "chezy")])
def test_three_1d_subdomains_equal_single_domain(N, system, source):
    """Three ranges of a periodic 1D mesh (one shorter than a tile, one
    spanning several), exchanging their end elements in one process, give
    the single-domain step bitwise."""
    crk = load()
    # dx = 1/4 exactly, so that each range's 1/dx equals the whole mesh's
    E, L, steps = 400, 100.0, 6
    u, b = case_1d(N, E, L, system)
    dt = 0.2 * (L / E) / 4.0 * golden_cfl(N, "gl")
    want = mono_1d(crk, N, E, L, u, b, dt, steps, system, source)
    parts = [(0, 37), (37, 300), (337, 63)]
    solvers = [slab_1d(crk, N, E, L, b, f, c, system, source) for f, c in parts]
    states = [to_dev(np.ascontiguousarray(u[:, f:f + c])) for f, c in parts]
    bufs = [s.halo_buffers() for s in solvers]       # (send_left, send_right, ghost_left, ghost_right)
    k_ = len(parts)
    for _ in range(steps):
        for s, x in zip(solvers, states):
            s.step_local(x, dt)
        for k in range(k_):
            left, right = (k - 1) % k_, (k + 1) % k_
            bufs[k][2].copy_(bufs[left][1])            # ghost left <- right end of the left range
            bufs[k][3].copy_(bufs[right][0])           # ghost right <- left end of the right range
        for s, x in zip(solvers, states):
            s.step_faces(x)
    got = np.concatenate([to_host(x) for x in states], axis=1)
    assert np.array_equal(got, want), rel_l2(got, want)


@pytest.mark.parametrize("N,system", [(4, "swe1d"), (2, "varadv1d")])
def test_three_1d_subdomains_cfl_steps_take_the_whole_mesh_step(N, system):
    crk = load()
    E, L, steps = 400, 100.0, 6
    u, b = case_1d(N, E, L, system)
    m = crk.Solver(system, N, gravity=G, cfl_number=golden_cfl(N, "gl"))
    m.set_mesh([E], [0.0], [L])
    m.set_coefficients(to_dev(b))
    want = to_dev(u)
    parts = [(0, 37), (37, 300), (337, 63)]
    solvers = [slab_1d(crk, N, E, L, b, f, c, system) for f, c in parts]
    states = [to_dev(np.ascontiguousarray(u[:, f:f + c])) for f, c in parts]
    bufs = [s.halo_buffers() for s in solvers]
    k_ = len(parts)
    for _ in range(steps):
        dt = min(s.compute_dt(x) for s, x in zip(solvers, states))
        assert dt == m.compute_dt(want)
        m.step(want, dt, 1)
        for s, x in zip(solvers, states):
            s.step_local(x, dt)
        for k in range(k_):
            bufs[k][2].copy_(bufs[(k - 1) % k_][1])
            bufs[k][3].copy_(bufs[(k + 1) % k_][0])
        for s, x in zip(solvers, states):
            s.step_faces(x)
    got = np.concatenate([to_host(x) for x in states], axis=1)
    assert np.array_equal(got, to_host(want)), rel_l2(got, to_host(want))


def test_single_1d_subdomain_is_its_own_neighbour():
    from paper_2512_08611_gb300.distributed import SlabStepper
    crk = load()
    N, E, L, steps = 3, 300, 100.0, 5
    u, b = case_1d(N, E, L, "swe1d")
    dt = 0.05 * (L / E) * golden_cfl(N, "gl")
    want = mono_1d(crk, N, E, L, u, b, dt, steps, "swe1d")
    s = slab_1d(crk, N, E, L, b, 0, E, "swe1d")
    x = to_dev(u)
    SlabStepper(s).step(x, dt, steps)
    assert np.array_equal(to_host(x), want)
    with pytest.raises(crk.CrkfrError) as e:
        s.step(x, dt, 1)
    assert e.value.status == -6
