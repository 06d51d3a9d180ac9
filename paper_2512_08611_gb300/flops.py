"""FP64 operation counts of the kernels, per element, from the formulation
they implement (an FMA counts as 2 flops, a multiply or add as 1).

Element-local 2D kernel (per node, per stage i of an s-stage tableau with
nnz_i nonzero entries a_ij in row i):
  stage value      3 nnz_i FMA
  fluxes           5 FMA + 5 MUL   (1/h: 3 FMA; u, v, h^2, g h^2/2, hu v: MUL;
                                    (hu)^2/h + p, (hv)^2/h + p: FMA)
  local operator   3 MUL + (6n - 1) FMA  (D_x and D_y chains of the three
                                          variables, g h b_x and g h b_y)
  time averages    9 FMA if b_i != 0 (a copy at the first stage, the
                   weights being b_i / b_0): V (3), U (3), two x-fluxes and
                   one y-flux of the momenta
and per node W = u - dt V: 3 FMA; per element row and face side, for each of
7 trace fields: 1 MUL + (n - 1) FMA, in x and in y (GL nodes).

Fused 1D kernel (shallow water, per node and stage): stage value 2 nnz_i FMA,
flux 4 FMA + 2 MUL, local operator 2 MUL + (2n - 1) FMA, time averages
5 FMA if b_i != 0 (a copy at the first stage; V 2, U 2, F 1).  Per element:
traces 5 fields x 2 sides x (1 MUL + (n - 1) FMA); one face (its right face):
two wave speeds (1/h 3 FMA, |m/h| + sqrt(g h) with the 5-instruction square
root: 6 FMA + 4 MUL + 1 ADD each), 5 ADD + 1 MUL of differences, 6 FMA of
face terms; corrections and update 3 FMA per variable and node; the next
time step's rate: element means 2 (n - 1) FMA + 2 MUL, one wave speed, 1 MUL.

With Chezy friction (imex=True, SSP3-IMEX(4,3,3), 2D) per node and stage:
stage value nnz~_i FMA per variable plus nnz_i FMA per momentum; the
closed-form implicit solve 14 FMA + 11 MUL + 1 ADD (1/h, |r| through the
5-instruction square root, sqrt(1 + 4 k |r|), 1/(1 + q), m = r f); the
source -C_f |m| m / h^2 4 MUL; the fluxes and local operator only on stages
whose operator is used (their 1/h shared with the solve: 2 FMA + 5 MUL);
time averages 11 FMA (with the two source averages) on weighted stages
after the first; W 5 FMA per node.

First-order part of the 2D subcell blending limiter in the element-local
kernel (limited=True; per element, GL nodes): per node the parts of both
directions (1/h 3 FMA; sqrt(g h): 1 MUL + the 5-instruction root, 3 FMA +
2 MUL; v_x, v_y 2 MUL; the two spectral radii 2 ADD; the normal fluxes
with pressure 3 MUL + 2 FMA (well-balanced: 2 MUL); the tangential fluxes
2 MUL); per inner subface (2 N n of them) the Rusanov flux from those parts
(3 FMA + 4 MUL + 6 ADD; well-balanced: the jump and mean of eta, 3 ADD
more) and the two fluctuations (4 MUL + 3 ADD); per node and variable the
first-order update without the face terms (2 ADD + 2 FMA) plus 1 MUL per
node; the traces of c at the four faces (4 n (1 MUL + (n - 1) FMA)).

Well-balanced 2D form (system swe2d_wb): the fluxes lose the pressure
(3 FMA + 5 MUL: 1/h, u, v, and the three products), the local operator gains
D_x h and D_y h (2 MUL + 2 (n - 1) FMA) and g h_x + g b_x, g h_y + g b_y
(2 FMA).
"""
import numpy as np


def _tableau(N):
    from .tableau_py import stages_nnz_b
    return stages_nnz_b(N)


def _imex_swe2d(N):
    from .tableau_py import imex_structure
    t = imex_structure()
    n = N + 1
    fma = mul = add = 0
    first = t["b"].index(True)
    for i in range(4):
        fma += 3 * t["nnz_e"][i] + 2 * t["nnz_i"][i]
        fma += 14
        mul += 11
        add += 1
        mul += 4
        if t["need_L"][i]:
            fma += 2 + (6 * n - 1)
            mul += 5 + 3
        if t["b"][i] and i > first:
            fma += 11
    fma += 5
    per_node = 2 * fma + mul + add
    traces = 2 * n * 7 * 2 * (1 + 2 * (n - 1))
    return per_node * n * n + traces


def _swe2d_wb(N):
    n = N + 1
    nnz, bnz = _tableau(N)
    fma = mul = 0
    for i, (k, bz) in enumerate(zip(nnz, bnz)):
        fma += 3 * k + 3 + (6 * n - 1) + 2 * (n - 1) + 2
        mul += 5 + 3 + 2
        if bz and i > 0:
            fma += 9
    fma += 3
    per_node = 2 * fma + mul
    traces = 2 * n * 7 * 2 * (1 + 2 * (n - 1))
    return per_node * n * n + traces


def limiter_local_flops_per_element(system, N, gll=False):
    """Flops the first-order part of the 2D limiter adds to the element-local
    kernel (counts in the module docstring)."""
    if system not in ("swe2d", "swe2d_wb"):
        raise ValueError("the limiter's local count is written out for 2D shallow water")
    n = N + 1
    wb = system == "swe2d_wb"
    node = 2 * (3 + 3 + (0 if wb else 2)) + (1 + 2 + 2 + (2 if wb else 3) + 2) + 2
    sub = 2 * 3 + 4 + 6 + (3 if wb else 0) + 4 + 3
    update = 3 * (2 + 2 * 2) + 1
    ctr = 0 if gll else 4 * n * (1 + 2 * (n - 1))
    return n * n * (node + update) + 2 * N * n * sub + ctr


def local_flops_per_element(system, N, imex=False):
    n = N + 1
    if system == "swe2d_wb" and not imex:
        return _swe2d_wb(N)
    if imex:
        if system != "swe2d":
            raise ValueError("the IMEX operation count is written out for swe2d")
        return _imex_swe2d(N)
    nnz, bnz = _tableau(N)
    fma = mul = 0
    if system == "swe2d":
        for i, (k, bz) in enumerate(zip(nnz, bnz)):
            fma += 3 * k + 5 + (6 * n - 1)
            mul += 5 + 3
            if bz and i > 0:
                fma += 9
        fma += 3
        per_node = 2 * fma + mul
        traces = 2 * n * 7 * 2 * (1 + 2 * (n - 1))   # x and y, n rows, 7 fields, 2 sides
        return per_node * n * n + traces
    if system == "swe1d":
        for i, (k, bz) in enumerate(zip(nnz, bnz)):
            fma += 2 * k + 4 + (2 * n - 1)
            mul += 2 + 2
            if bz and i > 0:
                fma += 5
        per_node = 2 * fma + mul
        traces = 5 * 2 * (1 + 2 * (n - 1))
        speed = 2 * 6 + 4 + 1
        face = 2 * speed + 5 + 1 + 2 * 6
        update = 2 * 3 * 2 * n
        rate = 2 * 2 * (n - 1) + 2 + speed + 1
        return per_node * n + traces + face + update + rate
    raise ValueError(system)
