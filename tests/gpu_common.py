"""Shared helpers of the GPU parity tests: build/load the library, seeded
inputs at the oracle's solution points, comparison norms."""
import json
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
G = 9.81


def golden_cfl(N, family):
    with open(os.path.join(ROOT, "tests", "golden", "oracle_cfl.json")) as fh:
        return json.load(fh)["cfl"][f"{N}_{family}"]


def golden_cfl_imex(N, family):
    """CFL(N) of the explicit part of the IMEX tableau (used with a source)."""
    with open(os.path.join(ROOT, "tests", "golden", "oracle_cfl.json")) as fh:
        return json.load(fh)["cfl_imex"][f"{N}_{family}"]


def load():
    from paper_2512_08611_gb300 import build
    build.build_library()
    from paper_2512_08611_gb300 import crkfr
    crkfr.lib()
    return crkfr


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def residual_close(r, r_want, u, dt, rtol=1e-11, utol=1e-13):
    """A residual r = (u^{n+1} - u^n)/dt matches if its error, as an error of
    the update dt r, is below utol of the state, or below rtol of r itself
    (a zero residual, e.g. of a constant state, is checked the first way)."""
    err = np.linalg.norm((np.asarray(r) - r_want).ravel())
    return err <= rtol * np.linalg.norm(np.ravel(r_want)) + utol * np.linalg.norm(np.ravel(u)) / dt


def positions_1d(basis, E, lo, hi):
    dx = (hi - lo) / E
    return lo + (np.arange(E)[:, None] + basis.xi[None, :]) * dx, dx


def positions_2d(basis, Ex, Ey, L):
    dx, dy = L / Ex, L / Ey
    x = (np.arange(Ex)[None, :, None, None] + basis.xi[None, None, None, :]) * dx
    y = (np.arange(Ey)[:, None, None, None] + basis.xi[None, None, :, None]) * dy
    x, y = np.broadcast_arrays(x, y)
    return x, y, dx, dy


def to_dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def to_host(t):
    return t.detach().cpu().numpy()
