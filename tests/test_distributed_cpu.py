"""The domain-decomposed step on CPU ranks (gloo, world sizes 2 and 3).

1. halo_exchange sends each slab's bottom/top boundary traces to the right
   ring neighbours, pairing messages by issue order as NCCL does.
2. A 2D step split over ranks — element-local phase per slab, one halo
   exchange, face phase per slab — reproduces the single-domain step
   bitwise; so do 1D ranges, CFL steps whose size is the minimum over ranks,
   and the limited 2D step with two rows exchanged.  The arithmetic here is
   the oracle's (CPU); the exchange and the reduction are the product's
   (paper_2512_08611_gb300.distributed)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _worker_exchange(rank, world, port, out):
    from paper_2512_08611_gb300.distributed import halo_exchange, neighbours
    _init(rank, world, port)
    sb = torch.full((5,), 10.0 * rank + 1, dtype=torch.float64)
    st = torch.full((5,), 10.0 * rank + 2, dtype=torch.float64)
    rb, rt = torch.zeros(5, dtype=torch.float64), torch.zeros(5, dtype=torch.float64)
    halo_exchange(sb, st, rb, rt)
    below, above = neighbours(rank, world)
    ok = bool(torch.all(rt == 10.0 * above + 1)) and bool(torch.all(rb == 10.0 * below + 2))
    out[rank] = ok
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_ring(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = free_port()
    procs = [ctx.Process(target=_worker_exchange, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert all(out[r] for r in range(world))


@pytest.mark.parametrize("world", [2, 3, 4])
def test_exchange_pairs_by_issue_order_without_tags(world):
    """Pair every rank's sends with its peers' receives the way NCCL does,
    by issue order per (sender, receiver) pair and ignoring tags: each halo
    still receives the right neighbour's traces (with two ranks the rank
    below is also the rank above, so only the order can tell the two
    messages apart)."""
    from paper_2512_08611_gb300.distributed import exchange_plan, neighbours
    sends, recvs = {}, {}
    for r in range(world):
        for kind, name, peer, _tag in exchange_plan(r, world):
            (sends if kind == "send" else recvs).setdefault((r, peer) if kind == "send"
                                                            else (peer, r), []).append(name)
    got = {}
    for (src, dst), names in sends.items():
        assert len(names) == len(recvs[(src, dst)])
        for sent, into in zip(names, recvs[(src, dst)]):
            got[(dst, into)] = (src, sent)
    for r in range(world):
        below, above = neighbours(r, world)
        assert got[(r, "recv_top")] == (above, "send_bottom")
        assert got[(r, "recv_bottom")] == (below, "send_top")


def _case(Ey, Ex, N, seed=3):
    from oracle.basis import Basis
    rng = np.random.default_rng(seed)
    bs = Basis(N)
    L = 10.0
    dx, dy = L / Ex, L / Ey
    x = (np.arange(Ex)[None, :, None, None] + bs.xi[None, None, None, :]) * dx
    y = (np.arange(Ey)[:, None, None, None] + bs.xi[None, None, :, None]) * dy
    x, y = np.broadcast_arrays(x, y)
    b = 0.2 * np.exp(-((x - 4) ** 2 + (y - 6) ** 2) / 3.0)
    u = np.stack([1.0 - b + 0.01 * rng.standard_normal(x.shape),
                  0.1 * np.sin(2 * np.pi * y / L), 0.1 * np.cos(2 * np.pi * x / L)])
    return u, b, dx, dy


def _split_step(sch, u_slab, c_slab, dt):
    """One step of a slab: local phase, halo exchange of the y-boundary face
    traces, face phase (oracle arithmetic, product exchange)."""
    from paper_2512_08611_gb300.distributed import halo_exchange
    loc = sch.local(u_slab, c_slab, dt)
    ax_y, ax_x = -3, -2
    bot_keys = ("G_b", "U_b", "un_b", "c_b")
    top_keys = ("G_t", "U_t", "un_t", "c_t")
    pack = lambda keys, row: torch.from_numpy(np.concatenate(
        [np.ascontiguousarray(np.take(loc[k], row, axis=ax_y)).ravel() for k in keys]))
    Ey = u_slab.shape[1]
    send_bottom, send_top = pack(bot_keys, 0), pack(top_keys, Ey - 1)
    recv_bottom, recv_top = torch.empty_like(send_top), torch.empty_like(send_bottom)
    halo_exchange(send_bottom, send_top, recv_bottom, recv_top)

    def unpack(buf, keys):
        out, off = {}, 0
        for k in keys:
            shape = np.take(loc[k], 0, axis=ax_y).shape
            size = int(np.prod(shape))
            out[k] = buf[off:off + size].numpy().reshape(shape)
            off += size
        return out
    halo_below = unpack(recv_bottom, top_keys)   # top-side traces of the row below
    halo_above = unpack(recv_top, bot_keys)      # bottom-side traces of the row above

    xm = {k: np.roll(loc[k], 1, axis=ax_x) for k in ("F_r", "U_r", "un_r", "c_r")}
    xp = {k: loc[k] for k in ("F_l", "U_l", "un_l", "c_l")}
    Txm, Txp, _ = sch._xface(xm, xp)
    # y faces: face k between row k-1 and row k, k = 0..Ey (0 and Ey use halos)
    ym = {k: np.concatenate([np.expand_dims(halo_below[k], ax_y), loc[k]], axis=ax_y)
          for k in top_keys}
    yp = {k: np.concatenate([loc[k], np.expand_dims(halo_above[k], ax_y)], axis=ax_y)
          for k in bot_keys}
    Tym, Typ, _ = sch._yface(ym, yp)
    Tr = np.roll(Txm, -1, axis=ax_x)
    Tt = np.take(Tym, np.arange(1, Ey + 1), axis=ax_y)
    Tb = np.take(Typ, np.arange(0, Ey), axis=ax_y)
    return u_slab - dt * (loc["vol"] + sch._corrections(Tr, Txp, Tt, Tb))


def _worker_step(rank, world, port, out):
    from oracle.crkfr import Scheme2D
    from oracle.systems import ShallowWater2D
    from paper_2512_08611_gb300.distributed import slab_rows
    _init(rank, world, port)
    N, Ey, Ex = 2, 7, 5
    u, b, dx, dy = _case(Ey, Ex, N)
    sch = Scheme2D(ShallowWater2D(9.81), N, dx, dy)
    first, count = slab_rows(Ey, rank, world)
    rows = slice(first, first + count)
    got = _split_step(sch, u[:, rows], b[rows], 0.004)
    want = sch.step(u, b, 0.004)[:, rows]
    out[rank] = (bool(np.array_equal(got, want)), float(np.max(np.abs(got - want))))
    dist.destroy_process_group()


def _worker_step_cfl(rank, world, port, out):
    """CFL steps: each rank's own step from its slab (the oracle's
    compute_dt), the minimum over ranks (the product's reduction), then the
    split step; the single-domain run takes the step of the whole mesh."""
    from oracle.crkfr import Scheme2D
    from oracle.systems import ShallowWater2D
    from paper_2512_08611_gb300.distributed import min_over_ranks, slab_rows
    _init(rank, world, port)
    N, Ey, Ex = 2, 7, 5
    u, b, dx, dy = _case(Ey, Ex, N)
    sch = Scheme2D(ShallowWater2D(9.81), N, dx, dy)
    first, count = slab_rows(Ey, rank, world)
    rows = slice(first, first + count)
    v, want = u[:, rows].copy(), u.copy()
    ok = True
    for _ in range(3):
        dt = min_over_ranks(sch.compute_dt(v, b[rows], 0.2, 0.5))
        dt_all = sch.compute_dt(want, b, 0.2, 0.5)
        ok &= dt == dt_all
        v = _split_step(sch, v, b[rows], dt)
        want = sch.step(want, b, dt_all)
        ok &= bool(np.array_equal(v, want[:, rows]))
    out[rank] = (ok, float(np.max(np.abs(v - want[:, rows]))))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_cfl_step_takes_the_single_domain_step(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = free_port()
    procs = [ctx.Process(target=_worker_step_cfl, args=(r, world, port, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r][0], out[r]


@pytest.mark.parametrize("world", [2, 3])
def test_split_step_equals_single_domain(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = free_port()
    procs = [ctx.Process(target=_worker_step, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r][0], out[r]


def _worker_limited(rank, world, port, out):
    """The limited 2D step (Sec. 4, tensor-product reading) of a slab depends
    on two element rows beyond each of its boundaries (the neighbours' raw
    indicator for the smoothing of the row next to the slab, that row's face
    data): each rank exchanges its two boundary rows of u with the product's
    exchange and runs the oracle's limited step on its slab extended by
    them (whose own results are dropped); the slab equals the single-domain
    oracle step bitwise."""
    from oracle.basis import Basis
    from oracle.crkfr import Scheme2D
    from oracle.limiter import Blending2D
    from oracle.systems import ShallowWater2D
    from paper_2512_08611_gb300.distributed import halo_exchange, slab_rows
    _init(rank, world, port)
    N, Ey, Ex, L = 2, 8, 5, 1.0
    bs = Basis(N, "gll")
    dx, dy = L / Ex, L / Ey
    x = (np.arange(Ex)[None, :, None, None] + bs.xi[None, None, None, :]) * dx
    y = (np.arange(Ey)[:, None, None, None] + bs.xi[None, None, :, None]) * dy
    x, y = np.broadcast_arrays(x, y)
    h = np.where((x - 0.45) ** 2 + (y - 0.52) ** 2 < 0.09, 1.0, 1e-3)
    b = np.zeros_like(h)
    u = np.stack([h, 0.0 * h, 0.0 * h])
    sch = Scheme2D(ShallowWater2D(9.81), N, dx, dy, family="gll")
    lim = Blending2D(sch)
    dt = 0.2 * sch.compute_dt(u, b, 0.1, 1.0)
    first, count = slab_rows(Ey, rank, world)
    v, want = u[:, first:first + count].copy(), u.copy()
    ok = True
    for _ in range(3):
        send_bottom = torch.from_numpy(np.ascontiguousarray(v[:, :2]).ravel())
        send_top = torch.from_numpy(np.ascontiguousarray(v[:, -2:]).ravel())
        recv_bottom, recv_top = torch.empty_like(send_top), torch.empty_like(send_bottom)
        halo_exchange(send_bottom, send_top, recv_bottom, recv_top)
        shape = (3, 2) + v.shape[2:]
        ext = np.concatenate([recv_bottom.numpy().reshape(shape), v,
                              recv_top.numpy().reshape(shape)], axis=1)
        rows = [(first + k) % Ey for k in range(-2, count + 2)]
        v = lim.step(ext, b[rows], dt)[:, 2:-2]
        want = lim.step(want, b, dt)
        ok &= bool(np.array_equal(v, want[:, first:first + count]))
    out[rank] = (ok, float(np.max(np.abs(v - want[:, first:first + count]))),
                 float(np.max(lim.last_alpha)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_limited_step_equals_single_domain(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = free_port()
    procs = [ctx.Process(target=_worker_limited, args=(r, world, port, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r][0], out[r]
    # the indicator is active on the mesh
    assert max(out[r][2] for r in range(world)) > 0.1


def _worker_limited_1d(rank, world, port, out):
    """The limited 1D step of a range depends on two elements beyond each
    end: ranks exchange their two end elements and run the oracle's limited
    step on the extended range, dropping the ends' results."""
    from oracle.basis import Basis
    from oracle.crkfr import Scheme1D
    from oracle.limiter import Blending1D
    from oracle.systems import ShallowWater1D
    from paper_2512_08611_gb300.distributed import halo_exchange, slab_rows
    _init(rank, world, port)
    N, E, L = 3, 30, 10.0
    bs = Basis(N, "gll")
    x = (np.arange(E)[:, None] + bs.xi[None, :]) * (L / E)
    h = np.where((x > 2.61) & (x < 6.37), 1.0, 1e-3)
    b = np.zeros_like(h)
    u = np.stack([h, 0.0 * h])
    sch = Scheme1D(ShallowWater1D(9.81), N, L / E, family="gll")
    lim = Blending1D(sch)
    dt = 0.2 * sch.compute_dt(u, b, 0.1, 1.0)
    first, count = slab_rows(E, rank, world)
    v, want = u[:, first:first + count].copy(), u.copy()
    ok = True
    for _ in range(3):
        send_left = torch.from_numpy(np.ascontiguousarray(v[:, :2]).ravel())
        send_right = torch.from_numpy(np.ascontiguousarray(v[:, -2:]).ravel())
        ghost_left, ghost_right = torch.empty_like(send_right), torch.empty_like(send_left)
        halo_exchange(send_left, send_right, ghost_left, ghost_right)
        ext = np.concatenate([ghost_left.numpy().reshape(2, 2, N + 1), v,
                              ghost_right.numpy().reshape(2, 2, N + 1)], axis=1)
        el = [(first + k) % E for k in range(-2, count + 2)]
        v = lim.step(ext, b[el], dt)[:, 2:-2]
        want = lim.step(want, b, dt)
        ok &= bool(np.array_equal(v, want[:, first:first + count]))
    out[rank] = (ok, float(np.max(np.abs(v - want[:, first:first + count]))),
                 float(np.max(lim.last_alpha)))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_limited_1d_step_equals_single_domain(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = free_port()
    procs = [ctx.Process(target=_worker_limited_1d, args=(r, world, port, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r][0], out[r]
    assert max(out[r][2] for r in range(world)) > 0.1


def _worker_adjoint(rank, world, port, out):
    """The adjoint of a slab step (the oracle's exact discrete adjoint:
    autograd through its step) needs one element row beyond the slab, of u
    and of ubar1: the outputs next to the slab depend on the slab's rows only
    through the face between them, which the two rows fix.  Ranks exchange
    one boundary row of u and of ubar1, differentiate the oracle step of their
    slab extended by those rows, and keep their own rows of ubar0 and of the
    bathymetry gradient, which equal the whole mesh's (the library exchanges
    the same: the forward traces and the correction sums of that row)."""
    from oracle.crkfr import Scheme2D
    from oracle.systems import ShallowWater2D
    from paper_2512_08611_gb300.distributed import halo_exchange, slab_rows
    _init(rank, world, port)
    N, Ey, Ex = 2, 9, 5
    u, b, dx, dy = _case(Ey, Ex, N)
    sch = Scheme2D(ShallowWater2D(9.81), N, dx, dy)
    dt = 0.5 * sch.compute_dt(u, b, 0.2, 0.5)
    w = np.random.default_rng(11).standard_normal(u.shape)
    first, count = slab_rows(Ey, rank, world)
    own = slice(first, first + count)

    def swap(a, depth):
        sb = torch.from_numpy(np.ascontiguousarray(a[:, :depth]).ravel())
        st = torch.from_numpy(np.ascontiguousarray(a[:, -depth:]).ravel())
        rb, rt = torch.empty_like(st), torch.empty_like(sb)
        halo_exchange(sb, st, rb, rt)
        shape = (a.shape[0], depth) + a.shape[2:]
        return rb.numpy().reshape(shape), rt.numpy().reshape(shape)
    ub_, ut_ = swap(u[:, own], 1)
    wb_, wt_ = swap(w[:, own], 1)
    u_ext = np.concatenate([ub_, u[:, own], ut_], axis=1)
    w_ext = np.concatenate([wb_, w[:, own], wt_], axis=1)
    b_ext = b[[(first + k) % Ey for k in range(-1, count + 1)]]
    uu = torch.tensor(u_ext, requires_grad=True)
    bb = torch.tensor(b_ext, requires_grad=True)
    (sch.step(uu, bb, dt) * torch.tensor(w_ext)).sum().backward()
    ug = torch.tensor(u, requires_grad=True)
    bg = torch.tensor(b, requires_grad=True)
    (sch.step(ug, bg, dt) * torch.tensor(w)).sum().backward()
    du = np.abs(uu.grad.numpy()[:, 1:-1] - ug.grad.numpy()[:, own]).max()
    db = np.abs(bb.grad.numpy()[1:-1] - bg.grad.numpy()[own]).max()
    scale = max(np.abs(ug.grad.numpy()).max(), np.abs(bg.grad.numpy()).max())
    out[rank] = (bool(du <= 1e-14 * scale and db <= 1e-14 * scale), float(du), float(db))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_adjoint_equals_single_domain(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = free_port()
    procs = [ctx.Process(target=_worker_adjoint, args=(r, world, port, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r][0], out[r]


def test_slab_rows_cover_the_mesh():
    from paper_2512_08611_gb300.distributed import slab_rows
    for G in (1, 7, 1024):
        for W in (1, 2, 3, 8):
            parts = [slab_rows(G, r, W) for r in range(W)]
            assert sum(c for _, c in parts) == G
            assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(W - 1))


def _worker_drop(rank, world, port, out):
    """Rank 1 leaves between steps (it raises before its exchange); rank 0's
    exchange must end with an error (peer gone, or the short process-group
    timeout), not wait forever."""
    import datetime
    import time
    from paper_2512_08611_gb300.distributed import halo_exchange
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    bufs = [torch.zeros(4, dtype=torch.float64) for _ in range(4)]
    halo_exchange(*bufs)                       # step 1: both ranks present
    if rank == 1:
        out[rank] = "left"
        raise SystemExit(3)                    # leaves before step 2
    t0 = time.time()
    try:
        halo_exchange(*bufs)                   # step 2: the peer is gone
        out[rank] = "no error"
    except Exception as e:                     # noqa: BLE001
        out[rank] = "error after %.1f s: %s" % (time.time() - t0, type(e).__name__)


def test_rank_drop_is_detected():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = free_port()
    procs = [ctx.Process(target=_worker_drop, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert procs[1].exitcode == 3
    assert out[1] == "left"
    assert str(out[0]).startswith("error after"), out[0]


def _worker_build(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    from paper_2512_08611_gb300 import build
    _init(rank, world, port)
    bench.build_once(world, dist)
    out[rank] = build.up_to_date()
    dist.destroy_process_group()


def test_benchmark_ranks_build_the_library_once():
    """Under torchrun every rank of bench.py needs the library: rank 0 builds
    it while the others wait at a barrier, then all find it up to date."""
    from paper_2512_08611_gb300 import build
    build.build_library()
    world, port = 2, free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker_build, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert all(out[r] for r in range(world))


def _worker_step_1d(rank, world, port, out):
    """1D ranges: each rank exchanges its two end elements with its ring
    neighbours (the product's exchange) and steps its range with the
    neighbours' end elements as ghosts (the oracle's arithmetic on the range
    extended by one element on either side, whose own results are dropped)."""
    from oracle.basis import Basis
    from oracle.crkfr import Scheme1D
    from oracle.systems import ShallowWater1D
    from paper_2512_08611_gb300.distributed import halo_exchange, slab_rows
    _init(rank, world, port)
    N, E, L = 3, 23, 10.0
    rng = np.random.default_rng(5)
    bs = Basis(N)
    x = (np.arange(E)[:, None] + bs.xi[None, :]) * (L / E)
    b = 0.2 * np.exp(-((x - 4.0) ** 2))
    u = np.stack([1.0 - b + 0.02 * np.sin(2 * np.pi * x / L) + 0.01 * rng.standard_normal(x.shape),
                  0.1 * np.cos(2 * np.pi * x / L)])
    sch = Scheme1D(ShallowWater1D(9.81), N, L / E)
    first, count = slab_rows(E, rank, world)
    mine = slice(first, first + count)
    c_ext = b[[(first - 1) % E] + list(range(first, first + count)) + [(first + count) % E]]
    v, want = u[:, mine].copy(), u.copy()
    ok, err = True, 0.0
    for _ in range(4):
        send_left = torch.from_numpy(np.ascontiguousarray(v[:, 0, :]).ravel())
        send_right = torch.from_numpy(np.ascontiguousarray(v[:, -1, :]).ravel())
        ghost_left, ghost_right = torch.empty_like(send_right), torch.empty_like(send_left)
        halo_exchange(send_left, send_right, ghost_left, ghost_right)
        ext = np.concatenate([ghost_left.numpy().reshape(2, 1, N + 1), v,
                              ghost_right.numpy().reshape(2, 1, N + 1)], axis=1)
        v = sch.step(ext, c_ext, 0.01)[:, 1:-1]
        want = sch.step(want, b, 0.01)
        ok &= bool(np.array_equal(v, want[:, mine]))
        err = max(err, float(np.max(np.abs(v - want[:, mine]))))
    out[rank] = (ok, err)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_split_1d_step_equals_single_domain(world):
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = free_port()
    procs = [ctx.Process(target=_worker_step_1d, args=(r, world, port, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r][0], out[r]
