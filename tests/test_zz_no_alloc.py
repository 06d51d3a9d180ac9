"""crkfr_step_1d_noalloc, the 1D step for callers that cannot allocate
device memory (their application owns every device allocation, or their
loop cannot afford the synchronisation an allocation may cause): its
buffers live in a static device array instead.  Its results must equal
those of the context-based crkfr_step, on two calls in a row (the second
call reuses the array the first one left behind).  This file is collected
last on purpose."""
import numpy as np
import pytest

from gpu_common import G, golden_cfl, load, positions_1d, rel_l2, to_dev, to_host
from oracle.basis import Basis
from paper_2512_08611_gb300.workloads import SWE1DInput, accept_seed

pytestmark = pytest.mark.gpu


def case(N, E, seed):
    x, dx = positions_1d(Basis(N), E, 0.0, 100.0)
    inp, _ = accept_seed(lambda s: SWE1DInput(seed=s), (x,), seed)
    return inp.state(x)


@pytest.mark.parametrize("mode,nsteps", [("cfl", 7), ("fixed", 4)])
def test_noalloc_step_matches_context_step_twice(mode, nsteps):
    crk = load()
    N = 4
    for call, (E, seed) in enumerate([(3001, 1), (20000, 2)]):
        u, b = case(N, E, seed)
        # fixed step: a quarter of the CFL step for wave speeds up to 4
        dt = 0.0 if mode == "cfl" else 0.25 * golden_cfl(N, "gl") * (100.0 / E) / 4.0
        s = crk.Solver("swe1d", N, gravity=G, cfl_safety=0.5, cfl_number=golden_cfl(N, "gl"))
        s.set_mesh([E], [0.0], [100.0])
        db = to_dev(b)
        s.set_coefficients(db)
        want = to_dev(u)
        s.step(want, dt, nsteps)
        got = to_dev(np.zeros_like(u))
        crk.step_1d_noalloc("swe1d", N, E, 0.0, 100.0, db, to_dev(u), got, dt=dt, nsteps=nsteps,
                            gravity=G, cfl_safety=0.5, cfl_number=golden_cfl(N, "gl"))
        inplace = to_dev(u)
        crk.step_1d_noalloc("swe1d", N, E, 0.0, 100.0, db, inplace, inplace, dt=dt,
                            nsteps=nsteps, gravity=G, cfl_safety=0.5,
                            cfl_number=golden_cfl(N, "gl"))
        w = to_host(want)
        assert np.all(np.isfinite(w)) and np.min(w[0]) > 0
        assert rel_l2(to_host(got), w) < 1e-12, call
        assert rel_l2(to_host(inplace), w) < 1e-12, call


def test_noalloc_rejects_meshes_beyond_its_array():
    crk = load()
    N, E = 4, 200000
    import torch
    c = torch.zeros((E, N + 1), dtype=torch.float64, device="cuda")
    u = torch.ones((2, E, N + 1), dtype=torch.float64, device="cuda")
    with pytest.raises(crk.CrkfrError) as e:
        crk.step_1d_noalloc("swe1d", N, E, 0.0, 100.0, c, u, u, dt=0.01, nsteps=1)
    assert e.value.status == -1
