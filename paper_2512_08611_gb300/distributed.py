"""Domain decomposition of the 2D step across ranks (torch.distributed).

The mesh is split into horizontal slabs of element rows, one per rank, on a
periodic ring: rank r's slab lies between rank r-1 (below) and rank r+1
(above).  The only inter-element coupling of a cRK-FR step is one Riemann
problem per face after the element-local stages (Sec. 3), so a step needs one
exchange: after the local phase each rank sends the face traces of its bottom
element row (their bottom side) to the rank below, which stores them as its
top halo, and those of its top row (their top side) to the rank above, which
stores them as its bottom halo.  The face phase then runs on every rank with
no further communication.  A 1D mesh splits the same way into contiguous
element ranges, whose exchange carries the two end elements.  A CFL step
needs the largest wave-speed rate of the whole mesh: each rank computes its
slab's own step and the ranks take the minimum (one all-reduce per step).
This module holds only that exchange and that reduction; the arithmetic
stays in the library.
"""
import torch
import torch.distributed as dist

TAG_UP, TAG_DOWN = 7101, 7102


def neighbours(rank, world):
    """(below, above) ranks on the periodic ring."""
    return (rank - 1) % world, (rank + 1) % world


def exchange_plan(rank, world):
    """The point-to-point operations of one halo exchange in issue order:
    (kind, buffer, peer, tag) with kind 'send' or 'recv'.

    NCCL ignores tags: between two ranks it pairs the k-th send of one with
    the k-th receive of the other.  Every rank therefore issues its two sends
    in the order (top traces up, bottom traces down) and its two receives in
    the order (bottom halo from below, top halo from above).  With two ranks,
    where the rank below is also the rank above, the peer's first send (its
    top traces) meets this rank's first receive (the bottom halo) and its
    second send (its bottom traces) the second receive (the top halo), as the
    ring requires; with more ranks each pair of ranks exchanges one message
    per direction.  The tags agree with this pairing, for backends that
    honour them (gloo)."""
    below, above = neighbours(rank, world)
    return [("send", "send_top", above, TAG_UP),
            ("send", "send_bottom", below, TAG_DOWN),
            ("recv", "recv_bottom", below, TAG_UP),
            ("recv", "recv_top", above, TAG_DOWN)]


def halo_exchange(send_bottom, send_top, recv_bottom, recv_top, group=None):
    """Exchange the slab-boundary traces with the two ring neighbours.

    send_bottom: traces of this slab's bottom row (bottom side), goes to the
                 rank below and becomes its ``recv_top``;
    send_top:    traces of this slab's top row (top side), goes to the rank
                 above and becomes its ``recv_bottom``.
    With one rank the slab is its own neighbour (periodic).  The operations
    are issued in the order of ``exchange_plan``, which pairs them without
    relying on tags."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        recv_top.copy_(send_bottom)
        recv_bottom.copy_(send_top)
        return
    rank = dist.get_rank(group)
    bufs = {"send_bottom": send_bottom, "send_top": send_top, "recv_bottom": recv_bottom,
            "recv_top": recv_top}
    ops = [dist.P2POp(dist.isend if kind == "send" else dist.irecv, bufs[name], peer, group, tag)
           for kind, name, peer, tag in exchange_plan(rank, world)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


class SlabStepper:
    """Steps one rank's slab of a 2D mesh (or range of a 1D mesh): local
    phase, halo exchange, face phase.  ``solver`` is a crkfr.Solver in
    subdomain mode.  With a single process (no process group) the slab is its
    own periodic neighbour."""

    def __init__(self, solver, group=None):
        self.s = solver
        self.group = group
        self.send_bottom, self.send_top, self.recv_bottom, self.recv_top = solver.halo_buffers()
        self.last_dt = None
        self._lim = None

    def _limiter_buffers(self):
        """The limiter's halo blocks of a limited 2D slab (None without the
        limiter): the raw indicator rows and the y-face data."""
        if self.s.limiter[0] is None or len(self.s.n_elem) == 1:
            return None   # (a 1D range's exchange carries the indicator itself)
        if self._lim is None:
            self._lim = (self.s.limiter_halo_buffers(0), self.s.limiter_halo_buffers(1))
        return self._lim

    def step(self, u, dt=0.0, nsteps=1):
        """nsteps steps of u in place (with the limiter of a 2D slab when the
        solver has one: two more exchanges per step).  dt > 0: that step; dt <= 0: the CFL
        step of the whole mesh (Sec. 5, Eq. time.step.2d), the minimum over
        ranks of each slab's own step (crkfr_compute_dt), one all-reduce and
        one host synchronisation per step.  The minimum of C / rate_r over
        slabs is C / max_r rate_r to the last bit (IEEE division is monotone),
        so the ranks take the single-domain step exactly."""
        lim = self._limiter_buffers()
        for _ in range(nsteps):
            h = dt if dt > 0.0 else min_over_ranks(self.s.compute_dt(u), self.group)
            if lim is not None:
                # the limiter: the raw indicator's boundary rows before the
                # local phase, its face data with the traces after it
                self.s.step_indicator(u)
                halo_exchange(*lim[0], self.group)
            self.s.step_local(u, h)
            halo_exchange(self.send_bottom, self.send_top, self.recv_bottom, self.recv_top,
                          self.group)
            if lim is not None:
                halo_exchange(*lim[1], self.group)
            self.s.step_faces(u)
            self.last_dt = h
        return u


def slab_step_record(stepper, u, dt, record, advance=True):
    """One recorded step of a 2D slab (advance) or the record of its state
    only: local phase into the record, exchange of the record's boundary
    blocks of y traces, face phase from the record."""
    s = stepper.s
    s.step_local_record(u, dt, record, advance)
    halo_exchange(*s.record_halo_buffers(record), stepper.group)
    if advance:
        s.step_faces_record(u, record)
    return u


def slab_adjoint(stepper, u, ubar1, dt, ubar0=None, bbar=None, record=None):
    """Adjoint of one step of a 2D slab: ubar0 of the slab's elements and
    their bathymetry gradient added to bbar.  Without a record:
    crkfr_adjoint_local, the exchange of the forward traces and of ubar1's
    correction sums, crkfr_adjoint_faces; with the record of the step
    (slab_step_record): the sums and their exchange, then
    crkfr_adjoint_faces_recorded.  ``stepper`` is the slab's SlabStepper
    (its trace buffers and group)."""
    s = stepper.s
    if record is None:
        s.adjoint_local(u, ubar1, dt)
        halo_exchange(stepper.send_bottom, stepper.send_top, stepper.recv_bottom,
                      stepper.recv_top, stepper.group)
    else:
        s.adjoint_sums(ubar1)
    if getattr(stepper, "_adj", None) is None:
        stepper._adj = s.adjoint_halo_buffers()
    halo_exchange(*stepper._adj, stepper.group)
    if record is None:
        return s.adjoint_faces(u, ubar1, dt, ubar0, bbar)
    return s.adjoint_faces_recorded(u, record, ubar1, dt, ubar0, bbar)


def slab_rows(global_rows, rank, world):
    """(first row, row count) of a rank's slab: contiguous, sizes differ by at
    most one."""
    base, extra = divmod(global_rows, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def min_over_ranks(x, group=None):
    """Min of a float over the ranks of ``group`` (the time step of the whole
    mesh from the slabs' own steps)."""
    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend(group) == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return float(t.item())


def max_over_ranks(x):
    """Max of a float over ranks (for the time step of Eq. time.step.2d the
    ranks need the global maximum wave-speed rate)."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
