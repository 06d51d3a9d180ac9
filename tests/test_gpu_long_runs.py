"""Long runs at the workloads' full size against the oracle's stored runs
(tests/golden/long_*.json, written by tests/golden/make_long_runs.py, which
calls only oracle/): the 1e5-element N = 4 shallow-water mesh over 1000 CFL
steps, the 1024^2 N = 3 mesh over 500 CFL steps, and eight instances of the
256-instance ragged ensemble over 1000 CFL steps in one graph.  Each run is
stepped as the benchmark steps it; the final state is compared with the
stored final time, quadrature norms and totals per variable, block means of
the element means and every value of the stored sample of elements.

Tolerance: 1e-10 relative L2 after the run (the CUDA path and the oracle
differ only in FP64 rounding order; the time step is recomputed from the
state every step on both sides, so the two runs also take their own, nearly
equal, step sizes)."""
import json
import os

import numpy as np
import pytest

from gpu_common import G, ROOT, golden_cfl, load, positions_1d, positions_2d, rel_l2, to_dev, to_host
from oracle.basis import Basis
from paper_2512_08611_gb300.workloads import SWE1DInput, SWE2DInput, accept_seed

pytestmark = pytest.mark.gpu

TOL = 1e-10


def golden(name):
    path = os.path.join(ROOT, "tests", "golden", f"long_{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written")
    with open(path) as fh:
        return json.load(fh)


def check_1d(got, t, ref, N, dx, nblocks):
    """Compare a 1D final state with a stored summary."""
    w = Basis(N).w
    assert t == pytest.approx(ref["t_final"], rel=1e-12)
    elems = np.asarray(ref["sample_elements"])
    assert rel_l2(got[:, elems, :], np.asarray(ref["sample"])) < TOL
    E = got.shape[1]
    means = np.einsum("p,vep->ve", w, got)
    edges = (np.arange(nblocks + 1) * E) // nblocks
    blocks = np.stack([means[:, a:b].mean(axis=1) for a, b in zip(edges[:-1], edges[1:])], axis=1)
    assert rel_l2(blocks, np.asarray(ref["block_means"])) < TOL
    for v in range(got.shape[0]):
        assert np.sqrt(np.sum(dx * w * got[v] ** 2)) == pytest.approx(ref["l2"][v], rel=1e-12)
    # mass: conserved by both to round-off
    assert np.sum(dx * w * got[0]) == pytest.approx(ref["total"][0], rel=1e-13)


def test_swe1d_full_size_thousand_steps():
    """1e5 elements, N = 4, 1000 CFL steps (the 1D workload's recipe and
    launch configuration)."""
    ref = golden("swe1d")
    crk = load()
    N, E, L = ref["N"], ref["E"], ref["L"]
    x, dx = positions_1d(Basis(N), E, 0.0, L)
    inp, seed = accept_seed(lambda s: SWE1DInput(seed=s, L=L), (x,), 0)
    assert seed == ref["input_seed"]
    u, b = inp.state(x)
    s = crk.Solver("swe1d", N, gravity=G, cfl_safety=ref["cfl_safety"],
                   cfl_number=golden_cfl(N, "gl"))
    s.set_mesh([E], [0.0], [L])
    s.set_coefficients(to_dev(b))
    du = to_dev(u)
    s.step(du, 0.0, ref["steps"])
    s.status()
    got = to_host(du)
    check_1d(got, s.time()[0], ref, N, dx, 100)
    # the run moved the state
    assert rel_l2(got, u) > 1e-6


def test_swe2d_full_size_five_hundred_steps():
    """1024 x 1024 quads, N = 3, 500 CFL steps, stepped as the benchmark
    steps the default workload."""
    ref = golden("swe2d")
    crk = load()
    N, (Ex, Ey), L = ref["N"], ref["E"], ref["L"]
    bs = Basis(N)
    x, y, dx, dy = positions_2d(bs, Ex, Ey, L)
    inp, seed = accept_seed(lambda s: SWE2DInput(seed=s, L=L), (x, y), 0)
    assert seed == ref["input_seed"]
    u, b = inp.state(x, y)
    s = crk.Solver("swe2d", N, gravity=G, cfl_safety=ref["cfl_safety"],
                   cfl_number=golden_cfl(N, "gl"))
    s.set_mesh([Ex, Ey], [0.0, 0.0], [L, L])
    s.set_coefficients(to_dev(b))
    du = to_dev(u)
    s.step(du, 0.0, ref["steps"])
    s.status()
    assert s.time()[0] == pytest.approx(ref["t_final"], rel=1e-12)
    ey, ex = np.asarray(ref["sample_ey"]), np.asarray(ref["sample_ex"])
    got_s = to_host(du[:, ey, ex])
    assert rel_l2(got_s, np.asarray(ref["sample"])) < TOL
    w = bs.w
    means = to_host(torch_means(du, w))
    nb = len(ref["block_means"][0])
    blocks = means.reshape(3, nb, Ey // nb, nb, Ex // nb).mean(axis=(2, 4))
    assert rel_l2(blocks, np.asarray(ref["block_means"])) < TOL
    W = dx * dy * w[:, None] * w[None, :]
    got = to_host(du)
    for v in range(3):
        assert np.sqrt(np.sum(W * got[v] ** 2)) == pytest.approx(ref["l2"][v], rel=1e-12)
    assert np.sum(W * got[0]) == pytest.approx(ref["total"][0], rel=1e-13)
    assert rel_l2(got, u) > 1e-6


def torch_means(du, w):
    import torch
    wt = torch.tensor(w, dtype=torch.float64, device=du.device)
    return torch.einsum("q,p,vyxqp->vyx", wt, wt, du)


def test_ensemble_full_size_thousand_steps():
    """The 256-instance ensemble (element counts log-uniform in [2^10, 2^16],
    N in {2, 3, 4}), autotuned and stepped 1000 CFL steps in one CUDA graph
    as the benchmark does; eight instances (the largest, the smallest and six
    seeded others) against the oracle's runs."""
    from paper_2512_08611_gb300.workloads import ensemble_members
    ref = golden("ensemble")
    crk = load()
    L = ref["L"]
    mem = ensemble_members(256, seed=0)
    members, us, cs = [], [], []
    for m in mem:
        N, E = m["N"], m["E"]
        x, _ = positions_1d(Basis(N), E, 0.0, L)
        inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=L), (x,), m["seed"])
        u, b = inp.state(x)
        members.append((N, E, 0.0, L))
        us.append(u)
        cs.append(b)
    import torch
    batch = crk.Batch("swe1d", members, gravity=G, cfl_safety=ref["cfl_safety"])
    u = torch.cat([to_dev(x).reshape(-1) for x in us])
    c = torch.cat([to_dev(x).reshape(-1) for x in cs])
    batch.set_coefficients(c)
    batch.autotune(u, steps=3)
    batch.step(u, 0.0, ref["steps"], graph=True)
    batch.status()
    times = batch.times()
    for inst in ref["instances"]:
        i = inst["index"]
        N, E = members[i][0], members[i][1]
        assert (N, E) == (inst["N"], inst["E"])
        got = to_host(batch.state_view(u, i))
        check_1d(got, times[i], inst, N, L / E, 16)
