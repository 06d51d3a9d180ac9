"""crkfr_step_1d_noalloc, the 1D step for callers that cannot allocate
device memory (their application owns every device allocation, or their
loop cannot afford the synchronisation an allocation may cause): its
buffers live in a static device array instead.  It launches the same
kernels on the same inputs as the context-based crkfr_step, so its results
must equal those bit for bit, on two calls in a row (the second call reuses
the array the first one left behind), and a second call must leave the
device's free memory unchanged.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from gpu_common import G, golden_cfl, load, positions_1d, to_dev, to_host
from oracle.basis import Basis
from paper_2512_08611_gb300.workloads import SWE1DInput, VarAdvInput, accept_seed

pytestmark = pytest.mark.gpu


def case(system, N, family, E, seed):
    if system == "varadv1d":
        x, _ = positions_1d(Basis(N, family), E, 0.0, 1.0)
        inp = VarAdvInput()
        return inp.v0(x)[None], inp.a(x), 1.0
    x, _ = positions_1d(Basis(N, family), E, 0.0, 100.0)
    inp, _ = accept_seed(lambda s: SWE1DInput(seed=s), (x,), seed)
    u, b = inp.state(x)
    return u, b, 100.0


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("system,N,family", [("swe1d", 4, "gl"), ("varadv1d", 3, "gl"),
                                             ("swe1d_wb", 2, "gll"), ("swe1d", 3, "gll")])
@pytest.mark.parametrize("mode,nsteps", [("cfl", 7), ("fixed", 4)])
def test_noalloc_step_matches_context_step_twice(system, N, family, mode, nsteps):
    crk = load()
    cfl = golden_cfl(N, family)
    free_after = []
    for call, (E, seed) in enumerate([(3001, 1), (20000, 2)]):
        u, b, L = case(system, N, family, E, seed)
        # fixed step: a quarter of the CFL step for wave speeds up to 4
        dt = 0.0 if mode == "cfl" else 0.25 * cfl * (L / E) / 4.0
        s = crk.Solver(system, N, nodes=family, gravity=G, cfl_safety=0.5, cfl_number=cfl)
        s.set_mesh([E], [0.0], [L])
        db = to_dev(b)
        s.set_coefficients(db)
        want = to_dev(u)
        s.step(want, dt, nsteps)
        got = to_dev(np.zeros_like(u))
        inplace = to_dev(u)
        src = to_dev(u)
        # every tensor exists before the calls: only the library could allocate
        fb = free_bytes()
        crk.step_1d_noalloc(system, N, E, 0.0, L, db, src, got, nodes=family, dt=dt,
                            nsteps=nsteps, gravity=G, cfl_safety=0.5, cfl_number=cfl)
        crk.step_1d_noalloc(system, N, E, 0.0, L, db, inplace, inplace, nodes=family, dt=dt,
                            nsteps=nsteps, gravity=G, cfl_safety=0.5, cfl_number=cfl)
        free_after.append((fb, free_bytes()))
        w = to_host(want)
        assert np.all(np.isfinite(w))
        assert np.array_equal(to_host(got), w), call
        assert np.array_equal(to_host(inplace), w), call
    # the first call may load the module; the second allocates nothing
    fb, fa = free_after[1]
    assert fa == fb, (fb, fa)


def test_noalloc_rejects_meshes_beyond_its_array():
    crk = load()
    N, E = 4, 200000
    c = torch.zeros((E, N + 1), dtype=torch.float64, device="cuda")
    u = torch.ones((2, E, N + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(crk.CrkfrError) as e:
        crk.step_1d_noalloc("swe1d", N, E, 0.0, 100.0, c, u, u, dt=0.01, nsteps=1)
    assert e.value.status == -1


def test_noalloc_rejects_bad_dt_and_tensors_on_the_host():
    """A NaN or +inf dt is refused by the library; tensors of the wrong
    shape, type, layout or device are refused by the binding before the
    library sees their pointers."""
    crk = load()
    N, E = 2, 50
    c = torch.zeros((E, N + 1), dtype=torch.float64, device="cuda")
    u = torch.ones((2, E, N + 1), dtype=torch.float64, device="cuda")
    for dt in (float("nan"), float("inf")):
        with pytest.raises(crk.CrkfrError) as e:
            crk.step_1d_noalloc("swe1d", N, E, 0.0, 100.0, c, u, u, dt=dt, nsteps=1)
        assert e.value.status == -1
    bad = [(c[:-1], u, u), (c, u[:, :-1], u), (c, u, u.float()), (c, u, u.cpu()),
           (c.t(), u, u), (c, u, u.transpose(1, 2))]
    for cc, ui, uo in bad:
        with pytest.raises((TypeError, ValueError)):
            crk.step_1d_noalloc("swe1d", N, E, 0.0, 100.0, cc, ui, uo, dt=0.01, nsteps=1)
    with pytest.raises(ValueError):
        crk.step_1d_noalloc("swe2d", N, E, 0.0, 100.0, c, u, u, dt=0.01, nsteps=1)
