"""Writes the stored results of the oracle's long runs at full workload size
(this script calls nothing but ``oracle/`` and the seeded input recipes of
``paper_2512_08611_gb300.workloads``, which hold none of the method's
arithmetic).

    python tests/golden/make_long_runs.py swe1d    # 1e5 elements, N = 4, 1000 CFL steps
    python tests/golden/make_long_runs.py swe2d    # 1024^2 quads, N = 3, 500 CFL steps
    python tests/golden/make_long_runs.py ensemble # 8 of the 256 ragged instances, 1000 CFL steps

Each run is the oracle's cRK-FR step (Sec. 3, Eq. crkfr.non.cons.final) with
the time step of Sec. 5, Eq. time.step.2d at C_s = 0.5 and the stored
CFL(N) of ``oracle_cfl.json``, repeated on the same seeded inputs the GPU
tests and the benchmark use.  A run stores what a GPU run of the same
workload can be compared with: the final time, quadrature L2 norms and
totals per variable, element means averaged over blocks of elements, and
every value of a seeded sample of elements.

The 2D run takes about an hour on eight cores: the mesh is split into
horizontal slabs, one process per slab (spawned), and each process steps its
rows from the previous state with one halo row on either side (the step of a
row reads only its own and its two neighbour rows' local parts, so the
slab's rows equal the full step's).  The time step is the maximum of the
slabs' wave-speed rates, which is the whole mesh's maximum exactly.
"""
import argparse
import json
import multiprocessing
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.basis import Basis  # noqa: E402
from oracle.crkfr import Scheme1D, Scheme2D  # noqa: E402
from oracle.systems import ShallowWater1D, ShallowWater2D  # noqa: E402
from paper_2512_08611_gb300.workloads import (SWE1DInput, SWE2DInput, accept_seed,  # noqa: E402
                                             ensemble_members)

G = 9.81
CS = 0.5
L = 100.0


def golden_cfl(N):
    with open(os.path.join(HERE, "oracle_cfl.json")) as fh:
        return json.load(fh)["cfl"][f"{N}_gl"]


def positions_1d(N, E):
    bs = Basis(N)
    dx = L / E
    return (np.arange(E)[:, None] + bs.xi[None, :]) * dx, dx


def positions_2d(N, E):
    bs = Basis(N)
    d = L / E
    x = (np.arange(E)[None, :, None, None] + bs.xi[None, None, None, :]) * d
    y = (np.arange(E)[:, None, None, None] + bs.xi[None, None, :, None]) * d
    x, y = np.broadcast_arrays(x, y)
    return x, y, d


def block_means(means, nblocks):
    """Means over nblocks contiguous element ranges (edges at
    floor(k E / nblocks)) of per-element values means[var, elem]."""
    E = means.shape[-1]
    edges = (np.arange(nblocks + 1) * E) // nblocks
    return np.stack([means[:, a:b].mean(axis=1) for a, b in zip(edges[:-1], edges[1:])], axis=1)


def summary_1d(u, N, dx, nblocks, nsample, seed):
    """Norms, totals, block means of the element means, sampled elements."""
    w = Basis(N).w
    E = u.shape[1]
    means = np.einsum("p,vep->ve", w, u)
    blocks = block_means(means, nblocks)
    rng = np.random.default_rng(seed)
    elems = np.unique(np.concatenate([[0, E - 1], rng.integers(0, E, nsample - 2)]))
    return {
        "l2": [float(np.sqrt(np.sum(dx * w * v * v))) for v in u],
        "total": [float(np.sum(dx * w * v)) for v in u],
        "block_means": blocks.tolist(),
        "sample_elements": elems.tolist(),
        "sample": u[:, elems, :].tolist(),
    }


# ---------------------------------------------------------------------------
def run_swe1d():
    N, E, steps = 4, 100000, 1000
    x, dx = positions_1d(N, E)
    inp, seed = accept_seed(lambda s: SWE1DInput(seed=s, L=L), (x,), 0)
    u, b = inp.state(x)
    sch = Scheme1D(ShallowWater1D(G), N, dx)
    cfl = golden_cfl(N)
    t = 0.0
    for _ in range(steps):
        dt = sch.compute_dt(u, b, cfl, CS)
        u = sch.step(u, b, dt)
        t += dt
    out = {"workload": "swe1d", "N": N, "E": E, "L": L, "input_seed": seed, "steps": steps,
           "cfl_safety": CS, "cfl": cfl, "t_final": t}
    out.update(summary_1d(u, N, dx, 100, 512, 1))
    return out


# ---------------------------------------------------------------------------
_W = {}


def _attach(names, shape, N, d):
    from multiprocessing import shared_memory
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    shms = [shared_memory.SharedMemory(name=n) for n in names]
    _W["shm"] = shms
    _W["u"] = [np.ndarray(shape, dtype=np.float64, buffer=s.buf) for s in shms[:2]]
    _W["b"] = np.ndarray(shape[1:], dtype=np.float64, buffer=shms[2].buf)
    _W["sch"] = Scheme2D(ShallowWater2D(G), N, d, d)


def _slab_step(job):
    """Rows [r0, r1) of the step from buffer ``src`` into buffer ``1 - src``;
    returns the maximum wave-speed rate of the new rows."""
    src, r0, r1, dt = job
    u, out, b, sch = _W["u"][src], _W["u"][1 - src], _W["b"], _W["sch"]
    Ey = u.shape[1]
    rows = np.array([(r0 - 1) % Ey] + list(range(r0, r1)) + [r1 % Ey])
    sub, bsub = u[:, rows], b[rows]
    R = sch.residual(sub, bsub, dt)
    new = sub[:, 1:-1] - dt * R[:, 1:-1]
    out[:, r0:r1] = new
    return float(sch.max_rate(new, bsub[1:-1]))


def _slab_rate(job):
    src, r0, r1 = job
    return float(_W["sch"].max_rate(_W["u"][src][:, r0:r1], _W["b"][r0:r1]))


def run_swe2d(procs, E=1024, steps=500):
    from multiprocessing import shared_memory
    N = 3
    x, y, d = positions_2d(N, E)
    inp, seed = accept_seed(lambda s: SWE2DInput(seed=s, L=L), (x, y), 0)
    u0, b0 = inp.state(x, y)
    shape = u0.shape
    shms = [shared_memory.SharedMemory(create=True, size=u0.nbytes) for _ in range(2)]
    shms.append(shared_memory.SharedMemory(create=True, size=b0.nbytes))
    try:
        np.ndarray(shape, dtype=np.float64, buffer=shms[0].buf)[...] = u0
        np.ndarray(shape[1:], dtype=np.float64, buffer=shms[2].buf)[...] = b0
        cfl = golden_cfl(N)
        nslab = max(procs, 1)
        cuts = np.linspace(0, E, nslab + 1).astype(int)
        slabs = list(zip(cuts[:-1], cuts[1:]))
        ctx = multiprocessing.get_context("spawn")
        t, src = 0.0, 0
        t0 = time.time()
        with ctx.Pool(procs, initializer=_attach,
                      initargs=([s.name for s in shms], shape, N, d)) as pool:
            rate = max(pool.map(_slab_rate, [(0, r0, r1) for r0, r1 in slabs]))
            for k in range(steps):
                dt = CS * cfl / rate
                rate = max(pool.map(_slab_step, [(src, r0, r1, dt) for r0, r1 in slabs]))
                src = 1 - src
                t += dt
                if k % 25 == 0 and E >= 256:
                    print(f"step {k + 1}/{steps}  t = {t:.6g}  {time.time() - t0:.0f} s",
                          flush=True)
        u = np.array(np.ndarray(shape, dtype=np.float64, buffer=shms[src].buf))
    finally:
        for s in shms:
            s.close()
            s.unlink()
    w = Basis(N).w
    W = d * d * w[:, None] * w[None, :]
    means = np.einsum("q,p,vyxqp->vyx", w, w, u)
    nb = 32
    blocks = means.reshape(3, nb, E // nb, nb, E // nb).mean(axis=(2, 4))
    rng = np.random.default_rng(2)
    ey = np.concatenate([[0, 0, E - 1, E - 1], rng.integers(0, E, 124)])
    ex = np.concatenate([[0, E - 1, 0, E - 1], rng.integers(0, E, 124)])
    return {"workload": "swe2d", "N": N, "E": [E, E], "L": L, "input_seed": seed,
            "steps": steps, "cfl_safety": CS, "cfl": cfl, "t_final": t,
            "l2": [float(np.sqrt(np.sum(W * v * v))) for v in u],
            "total": [float(np.sum(W * v)) for v in u],
            "block_means": blocks.tolist(),
            "sample_ey": ey.tolist(), "sample_ex": ex.tolist(),
            "sample": u[:, ey, ex].tolist()}


# ---------------------------------------------------------------------------
def _instance(job):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    i, N, E, seed, steps = job
    x, dx = positions_1d(N, E)
    inp, _ = accept_seed(lambda s: SWE1DInput(seed=s, L=L), (x,), seed)
    u, b = inp.state(x)
    sch = Scheme1D(ShallowWater1D(G), N, dx)
    cfl = golden_cfl(N)
    t = 0.0
    for _ in range(steps):
        dt = sch.compute_dt(u, b, cfl, CS)
        u = sch.step(u, b, dt)
        t += dt
    out = {"index": i, "N": N, "E": E, "seed": seed, "t_final": t}
    out.update(summary_1d(u, N, dx, 16, 64, 100 + i))
    return out


def ensemble_indices(mem):
    """The largest and the smallest instance and six seeded others."""
    E = np.array([m["E"] for m in mem])
    rng = np.random.default_rng(7)
    rest = [int(i) for i in rng.permutation(len(mem)) if i not in (E.argmax(), E.argmin())]
    return [int(E.argmax()), int(E.argmin())] + rest[:6]


def run_ensemble(procs):
    steps = 1000
    mem = ensemble_members(256, seed=0)
    idx = ensemble_indices(mem)
    jobs = [(i, mem[i]["N"], mem[i]["E"], mem[i]["seed"], steps) for i in idx]
    with multiprocessing.get_context("spawn").Pool(min(procs, len(jobs))) as pool:
        res = pool.map(_instance, jobs)
    return {"workload": "ensemble", "members": "ensemble_members(256, seed=0)", "L": L,
            "steps": steps, "cfl_safety": CS, "instances": res}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("run", choices=["swe1d", "swe2d", "ensemble"])
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    t0 = time.time()
    if a.run == "swe1d":
        out = run_swe1d()
    elif a.run == "swe2d":
        out = run_swe2d(a.procs)
    else:
        out = run_ensemble(a.procs)
    out["source"] = ("oracle.crkfr (Sec. 3, Eq. crkfr.non.cons.final; Sec. 5, Eq. time.step.2d) "
                     "on the seeded inputs of paper_2512_08611_gb300.workloads; written by "
                     "tests/golden/make_long_runs.py")
    out["host_seconds"] = round(time.time() - t0, 1)
    with open(os.path.join(HERE, f"long_{a.run}.json"), "w") as fh:
        json.dump(out, fh, separators=(",", ":"))
        fh.write("\n")


if __name__ == "__main__":
    main()
