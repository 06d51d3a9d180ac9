"""Gradient of a final-time misfit with respect to the bathymetry, through the
library's hand-written adjoint step (crkfr_step_adjoint), with step-level
checkpointing.

Forward: the initial state is u0 = (eta0 - b, 0, 0) (a given free surface at
rest over the bathymetry b), the 2D shallow-water cRK-FR step S(.; b) with a
fixed dt is applied nsteps times, and the state u_T is returned.  Backward:
the states are recomputed segment by segment from checkpoints stored every
``every`` steps, and the adjoint steps run in reverse, accumulating
dJ/db through the static terms of the step (g b_x, g b_y, the face jumps of
b) and, at the end, through the initial condition (h0 = eta0 - b).  With
``recorded`` (the default) the recomputation records each step's face traces
and inner stage values (crkfr_step_record, one record per step of a segment
held at a time) and the adjoint steps read them back
(crkfr_step_adjoint_recorded) instead of recomputing them.

``BathymetryToState`` is a torch.autograd.Function, so any differentiable
torch expression of u_T and b can serve as J; ``surface_misfit`` is the
L2 misfit of the free surface h + b at the final time.
``SlabBathymetryToState`` is the same for one rank's slab of a mesh split
over ranks (the slab adjoint step, recorded or recomputing).
"""
import torch


def quadrature_weights(solver):
    """w_p w_q dx dy per node, shaped like one variable of the state."""
    _, w = solver.nodes()
    Ex, Ey = solver.n_elem
    dx = (solver.hi[0] - solver.lo[0]) / Ex
    dy = (solver.hi[1] - solver.lo[1]) / Ey
    W = torch.tensor(w[:, None] * w[None, :] * dx * dy, dtype=torch.float64, device="cuda")
    return W.expand(Ey, Ex, solver.n, solver.n)


def initial_state(eta0, b):
    z = torch.zeros_like(b)
    return torch.stack([eta0 - b, z, z])


class BathymetryToState(torch.autograd.Function):
    """u_T(b) for a 2D swe Solver (GL nodes) with fixed dt."""

    @staticmethod
    def forward(ctx, b, solver, eta0, dt, nsteps, every, recorded=True):
        solver.set_coefficients(b.detach().contiguous())
        u = initial_state(eta0, b.detach()).contiguous()
        checkpoints = [u.clone()]
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            solver.step(u, dt, k)
            done += k
            if done < nsteps:
                checkpoints.append(u.clone())
        ctx.solver, ctx.dt, ctx.nsteps, ctx.every = solver, dt, nsteps, every
        ctx.recorded = recorded
        ctx.checkpoints = checkpoints
        ctx.b = b.detach().contiguous()
        return u

    @staticmethod
    def backward(ctx, ubar):
        s, dt, nsteps, every = ctx.solver, ctx.dt, ctx.nsteps, ctx.every
        s.set_coefficients(ctx.b)
        ubar = ubar.contiguous().clone()
        bbar = torch.zeros_like(ctx.b)
        other = torch.empty_like(ubar)
        starts = list(range(0, nsteps, every))
        records = s.new_records(min(every, nsteps)) if ctx.recorded else None
        for seg, start in reversed(list(enumerate(starts))):
            k = min(every, nsteps - start)
            states = [ctx.checkpoints[seg].clone()]
            for j in range(k - 1):
                x = states[-1].clone()
                if records is None:
                    s.step(x, dt, 1)
                else:
                    s.step_record(x, dt, records[j])
                states.append(x)
            if records is None:
                for x in reversed(states):
                    s.step_adjoint(x, ubar, dt, ubar0=other, bbar=bbar)
                    ubar, other = other, ubar
            else:
                # the recomputation recorded the steps from states 0..k-2;
                # record the last one without stepping
                s.step_record(states[-1], dt, records[k - 1], advance=False)
                for j in reversed(range(k)):
                    s.step_adjoint_recorded(states[j], records[j], ubar, dt, ubar0=other,
                                            bbar=bbar)
                    ubar, other = other, ubar
        # initial condition h0 = eta0 - b
        bbar -= ubar[0]
        return bbar, None, None, None, None, None, None


class SlabBathymetryToState(torch.autograd.Function):
    """u_T(b) of one rank's slab of a 2D mesh split into slabs (a
    distributed.SlabStepper over a Solver in subdomain mode, fixed dt): b and
    eta0 are the slab's own rows, [Ey_local][Ex][n][n].  Every rank calls
    forward and backward together (both exchange with the neighbouring
    slabs).  The forward pass gets the element rows of b next to the slab
    from the neighbours; the backward pass runs the slab adjoint step
    (distributed.slab_adjoint) over states recomputed from checkpoints, with
    recorded steps (distributed.slab_step_record) unless ``recorded`` is
    false, and
    the gradient it returns is complete for the slab's own rows: the
    gradient of a neighbour's bathymetry at a shared face is formed by that
    neighbour."""

    @staticmethod
    def forward(ctx, b, stepper, eta0, dt, nsteps, every, recorded=True):
        from .distributed import halo_exchange
        bd = b.detach().contiguous()
        below, above = torch.empty_like(bd[-1:]), torch.empty_like(bd[:1])
        halo_exchange(bd[:1].contiguous(), bd[-1:].contiguous(), below, above, stepper.group)
        coef = torch.cat([below, bd, above]).contiguous()
        stepper.s.set_coefficients(coef)
        u = initial_state(eta0, bd).contiguous()
        checkpoints = [u.clone()]
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            stepper.step(u, dt, k)
            done += k
            if done < nsteps:
                checkpoints.append(u.clone())
        ctx.stepper, ctx.dt, ctx.nsteps, ctx.every = stepper, dt, nsteps, every
        ctx.checkpoints, ctx.coef, ctx.b = checkpoints, coef, bd
        ctx.recorded = recorded
        return u

    @staticmethod
    def backward(ctx, ubar):
        from .distributed import slab_adjoint, slab_step_record
        st, dt, nsteps, every = ctx.stepper, ctx.dt, ctx.nsteps, ctx.every
        st.s.set_coefficients(ctx.coef)
        ubar = ubar.contiguous().clone()
        bbar = torch.zeros_like(ctx.b)
        other = torch.empty_like(ubar)
        records = st.s.new_records(min(every, nsteps)) if ctx.recorded else None
        for seg, start in reversed(list(enumerate(range(0, nsteps, every)))):
            k = min(every, nsteps - start)
            states = [ctx.checkpoints[seg].clone()]
            for j in range(k - 1):
                x = states[-1].clone()
                if records is None:
                    st.step(x, dt, 1)
                else:
                    slab_step_record(st, x, dt, records[j])
                states.append(x)
            if records is not None:
                slab_step_record(st, states[-1], dt, records[k - 1], advance=False)
            for j in reversed(range(k)):
                slab_adjoint(st, states[j], ubar, dt, ubar0=other, bbar=bbar,
                             record=None if records is None else records[j])
                ubar, other = other, ubar
        bbar -= ubar[0]
        return bbar, None, None, None, None, None, None


def surface_misfit(u, b, target, weights):
    """J = 1/2 sum_nodes w (h + b - target)^2."""
    d = u[0] + b - target
    return 0.5 * torch.sum(weights * d * d)
