"""Ragged ensemble (crkfr_batch_*): every instance of a batch advanced
together equals the same mesh advanced alone by crkfr_step (the same tile
body runs on the same data), with and without CUDA-graph capture, and one
instance matches the oracle."""
import numpy as np
import pytest
import torch

from gpu_common import G, golden_cfl, load, positions_1d, rel_l2, to_dev, to_host
from oracle.basis import Basis
from oracle.crkfr import Scheme1D
from oracle.systems import ShallowWater1D
from paper_2512_08611_gb300.workloads import SWE1DInput, accept_seed

pytestmark = pytest.mark.gpu

MEMBERS = [(2, 1, 0.0, 100.0), (3, 5, 0.0, 40.0), (4, 130, 0.0, 100.0), (2, 127, 10.0, 90.0),
           (4, 300, 0.0, 100.0), (3, 2000, 0.0, 100.0), (1, 7, 0.0, 100.0), (0, 4, 0.0, 100.0),
           (4, 126, 0.0, 100.0), (3, 253, 0.0, 60.0)]


def inputs(members):
    us, cs = [], []
    for i, (N, E, lo, hi) in enumerate(members):
        x, _ = positions_1d(Basis(N), E, lo, hi)
        inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=hi - lo), (x - lo,), 100 + i)
        u, b = inp.state(x - lo)
        us.append(u)
        cs.append(b)
    return us, cs


def packed(batch, us, cs):
    u = torch.cat([to_dev(x).reshape(-1) for x in us])
    c = torch.cat([to_dev(x).reshape(-1) for x in cs])
    assert u.numel() == batch.state_offsets[-1] and c.numel() == batch.coef_offsets[-1]
    return u, c


def alone(crk, N, E, lo, hi, u, b, dt, nsteps):
    s = crk.Solver("swe1d", N, gravity=G, cfl_safety=0.5)
    s.set_mesh([E], [lo], [hi])
    s.set_coefficients(to_dev(b))
    du = to_dev(u)
    s.step(du, dt, nsteps)
    return to_host(du), s.time()[0]


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("dt", [0.0, 2e-4])
def test_batch_equals_instances_alone(graph, dt):
    crk = load()
    us, cs = inputs(MEMBERS)
    batch = crk.Batch("swe1d", MEMBERS, gravity=G, cfl_safety=0.5)
    u, c = packed(batch, us, cs)
    batch.set_coefficients(c)
    batch.step(u, dt, 9, graph=graph)
    batch.step(u, dt, 9, graph=graph)       # a second call (graph replay)
    times = batch.times()
    batch.status()
    for i, (N, E, lo, hi) in enumerate(MEMBERS):
        want, t = alone(crk, N, E, lo, hi, us[i], cs[i], dt, 18)
        got = to_host(batch.state_view(u, i))
        assert np.array_equal(got, want), (i, rel_l2(got, want))
        assert times[i] == t


def test_batch_instance_matches_oracle():
    crk = load()
    us, cs = inputs(MEMBERS)
    batch = crk.Batch("swe1d", MEMBERS, gravity=G, cfl_safety=0.5)
    u, c = packed(batch, us, cs)
    batch.set_coefficients(c)
    batch.step(u, 0.0, 5)
    i = 5
    N, E, lo, hi = MEMBERS[i]
    sch = Scheme1D(ShallowWater1D(G), N, (hi - lo) / E)
    v = us[i]
    for _ in range(5):
        v = sch.step(v, cs[i], sch.compute_dt(v, cs[i], golden_cfl(N, "gl"), 0.5))
    assert rel_l2(to_host(batch.state_view(u, i)), v) < 1e-11


@pytest.mark.parametrize("tpb,order,parallel", [(1, 1, False), (3, 0, True), (8, 1, True),
                                                (2, 0, False)])
@pytest.mark.parametrize("graph", [False, True])
def test_launch_shapes_give_the_same_bits(tpb, order, parallel, graph):
    """Tiles per block, work-list order and concurrent degree classes change
    only the schedule: every instance still equals its standalone run."""
    crk = load()
    us, cs = inputs(MEMBERS)
    batch = crk.Batch("swe1d", MEMBERS, gravity=G, cfl_safety=0.5)
    batch.set_tuning(tpb, order, parallel)
    assert batch.tuning()[:3] == (tpb, order, parallel)
    u, c = packed(batch, us, cs)
    batch.set_coefficients(c)
    batch.step(u, 0.0, 7, graph=graph)
    batch.step(u, 0.0, 7, graph=graph)
    times = batch.times()
    for i, (N, E, lo, hi) in enumerate(MEMBERS):
        want, t = alone(crk, N, E, lo, hi, us[i], cs[i], 0.0, 14)
        assert np.array_equal(to_host(batch.state_view(u, i)), want), i
        assert times[i] == t


@pytest.mark.parametrize("N,family", [(4, "gl"), (3, "gll")])
@pytest.mark.parametrize("system", ["swe1d", "swe1d_wb"])
def test_single_mesh_tile_sizes_give_the_same_bits(system, N, family):
    """The single-mesh step picks its block size per mesh (on 152 SMs: 64
    threads for 3001 elements, 128 for 19152 = 152 x 126, 96 for 1e5) unless
    crkfr_set_tile_1d fixes it; the ensemble always runs 128-thread tiles.
    Each element's arithmetic is the same in every tile size, so the mesh
    stepped alone with any tile size equals a one-instance batch, bit for
    bit, in CFL and fixed steps."""
    crk = load()
    for E in (3001, 19152, 100000):
        x, dx = positions_1d(Basis(N, family), E, 0.0, 100.0)
        inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=100.0), (x,), 7)
        u, b = inp.state(x)
        for dt in (0.0, 0.1 * dx):
            batch = crk.Batch(system, [(N, E, 0.0, 100.0)], nodes=family, gravity=G,
                              cfl_safety=0.5)
            got, c = packed(batch, [u], [b])
            batch.set_coefficients(c)
            batch.step(got, dt, 5)
            batch.status()
            ref = to_host(batch.state_view(got, 0))
            for tile in (0, 64, 96, 128):
                s = crk.Solver(system, N, nodes=family, gravity=G, cfl_safety=0.5)
                s.set_tile_1d(tile)
                s.set_mesh([E], [0.0], [100.0])
                s.set_coefficients(to_dev(b))
                want = to_dev(u)
                s.step(want, dt, 5)
                s.status()
                assert np.array_equal(to_host(want), ref), (E, dt, tile)
                assert batch.times()[0] == s.time()[0]


def test_autotune_leaves_state_and_times_and_keeps_the_bits():
    crk = load()
    us, cs = inputs(MEMBERS)
    batch = crk.Batch("swe1d", MEMBERS, gravity=G, cfl_safety=0.5)
    u, c = packed(batch, us, cs)
    batch.set_coefficients(c)
    batch.step(u, 0.0, 3)
    u_before = u.clone()
    t_before = batch.times()
    tpb, order, parallel, ms = batch.autotune(u, steps=3)
    assert tpb in (1, 2, 4, 8) and order in (0, 1) and ms > 0.0
    assert torch.equal(u, u_before)
    assert np.array_equal(batch.times(), t_before)
    batch.step(u, 0.0, 4)
    for i, (N, E, lo, hi) in enumerate(MEMBERS):
        want, _ = alone(crk, N, E, lo, hi, us[i], cs[i], 0.0, 7)
        assert np.array_equal(to_host(batch.state_view(u, i)), want), i


def test_full_size_ensemble_sampled():
    """The 256-instance ensemble of the benchmark (element counts
    log-uniform in [2^10, 2^16], N in {2, 3, 4}), autotuned as the benchmark
    does, 3 CFL steps in a graph: 8 sampled instances equal their standalone
    runs bitwise and one matches the oracle."""
    from paper_2512_08611_gb300.workloads import ensemble_members
    crk = load()
    L = 100.0
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
    batch = crk.Batch("swe1d", members, gravity=G, cfl_safety=0.5)
    u, c = packed(batch, us, cs)
    batch.set_coefficients(c)
    batch.autotune(u, steps=3)
    batch.step(u, 0.0, 3, graph=True)
    batch.status()
    rng = np.random.default_rng(5)
    for i in rng.choice(len(members), 8, replace=False):
        N, E, lo, hi = members[i]
        want, _ = alone(crk, N, E, lo, hi, us[i], cs[i], 0.0, 3)
        assert np.array_equal(to_host(batch.state_view(u, i)), want), i
    i = int(np.argmin([m[1] for m in members]))
    N, E, lo, hi = members[i]
    sch = Scheme1D(ShallowWater1D(G), N, (hi - lo) / E)
    v = us[i]
    for _ in range(3):
        v = sch.step(v, cs[i], sch.compute_dt(v, cs[i], golden_cfl(N, "gl"), 0.5))
    assert rel_l2(to_host(batch.state_view(u, i)), v) < 1e-12


def test_batch_kernel_timing_counts_the_step_kernels():
    """crkfr_batch_profile_*: every step kernel of a call without a graph is
    timed (classes x steps launches, positive summed time); calls with a
    graph are not; enabling again clears the sums."""
    crk = load()
    us, cs = inputs(MEMBERS)
    batch = crk.Batch("swe1d", MEMBERS, gravity=G, cfl_safety=0.5)
    u, c = packed(batch, us, cs)
    batch.set_coefficients(c)
    classes = len({m[0] for m in MEMBERS})
    batch.profile(True)
    batch.step(u, 0.0, 4, graph=False)
    n, ms = batch.profile_read()
    assert n == 4 * classes and ms > 0.0
    batch.step(u, 0.0, 3, graph=True)
    assert batch.profile_read()[0] == 4 * classes
    batch.profile(True)
    assert batch.profile_read() == (0, 0.0)
    batch.profile(False)
    batch.step(u, 0.0, 2, graph=False)
    assert batch.profile_read() == (0, 0.0)
    batch.status()
