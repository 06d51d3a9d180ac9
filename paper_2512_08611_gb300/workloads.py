"""Seeded synthetic inputs for the cRK-FR workloads.

This module only draws random parameters and evaluates the initial fields
at positions the caller supplies; it holds none of the scheme's arithmetic,
so both the CUDA path and the CPU oracle can take their inputs from it.

Workloads (all periodic, FP64):

* ``varadv``: v_t + a(x) v_x = 0 on [0, 1], a = 1 + 0.5 sin(2 pi x),
  v0 = sin(2 pi x)  (the variable-coefficient test of Sec. 5.1.3 with a
  periodic coefficient).
* ``swe1d``: shallow water with bathymetry on [0, 100]: b is a sum of 8
  Gaussians (amplitude U[0.05, 0.3], width U[1, 5], centre U[0, L)), the
  free surface is h + b = 1 + 0.01 p(x) with
  p(x) = sum_{k=1..4} sin(2 pi k x / L + phi_k) / 4, phi_k ~ U[0, 2 pi), and
  the velocity is zero.  ``still=True`` gives the lake at rest (p = 0).
* ``swe2d``: 2D shallow water on [0, 100]^2: b is a sum of 32 Gaussians
  (same ranges), h + b = 1 + 0.01 G(x, y) with G one unit Gaussian bump of
  width U[1, 5] at a random centre, zero velocity.
* ``swe2d-friction``: the same fields with a uniform current, velocity
  (0.3, 0.2), under Chezy friction C_f = 0.0025 (g / C^2 with a Chezy
  constant C of about 63 m^(1/2)/s).

Distances are periodic (d = min(|x - c|, L - |x - c|) per coordinate).  A
seed whose minimum depth h = 1 + 0.01 p - b falls below 0.1 on the sampled
positions is rejected and the next seed is drawn from the same stream.
"""
import numpy as np

GRAVITY = 9.81


def periodic_distance(x, centre, L):
    d = np.abs(np.asarray(x) - centre) % L
    return np.minimum(d, L - d)


class VarAdvInput:
    """Coefficient a(x) = 1 + eps sin(2 pi x / L) and v0 = sin(2 pi x / L)."""

    def __init__(self, eps=0.5, L=1.0):
        self.eps, self.L = eps, L

    def a(self, x):
        return 1.0 + self.eps * np.sin(2 * np.pi * np.asarray(x) / self.L)

    def v0(self, x):
        return np.sin(2 * np.pi * np.asarray(x) / self.L)


class SWE1DInput:
    """Seeded 1D bathymetry / free-surface recipe."""

    def __init__(self, seed=0, L=100.0, n_gauss=8, amp=(0.05, 0.3), width=(1.0, 5.0),
                 still=False):
        self.L = L
        self.still = still
        rng = np.random.default_rng(seed)
        self.amp = rng.uniform(amp[0], amp[1], n_gauss)
        self.width = rng.uniform(width[0], width[1], n_gauss)
        self.centre = rng.uniform(0.0, L, n_gauss)
        self.phase = rng.uniform(0.0, 2 * np.pi, 4)

    def b(self, x):
        x = np.asarray(x, dtype=float)
        out = np.zeros_like(x)
        for A, w, c in zip(self.amp, self.width, self.centre):
            d = periodic_distance(x, c, self.L)
            out += A * np.exp(-d * d / (2 * w * w))
        return out

    def p(self, x):
        x = np.asarray(x, dtype=float)
        if self.still:
            return np.zeros_like(x)
        return sum(np.sin(2 * np.pi * k * x / self.L + ph) for k, ph in
                   zip(range(1, 5), self.phase)) / 4.0

    def eta(self, x):
        return 1.0 + 0.01 * self.p(x)

    def state(self, x):
        """(h, m) at positions x and the bathymetry b."""
        b = self.b(x)
        h = self.eta(x) - b
        return np.stack([h, np.zeros_like(h)]), b


class SWE2DInput:
    """Seeded 2D bathymetry / free-surface recipe on [0, L]^2."""

    def __init__(self, seed=0, L=100.0, n_gauss=32, amp=(0.05, 0.3), width=(1.0, 5.0),
                 current=(0.0, 0.0)):
        self.L = L
        self.current = tuple(float(c) for c in current)
        rng = np.random.default_rng(seed)
        self.amp = rng.uniform(amp[0], amp[1], n_gauss)
        self.width = rng.uniform(width[0], width[1], n_gauss)
        self.cx = rng.uniform(0.0, L, n_gauss)
        self.cy = rng.uniform(0.0, L, n_gauss)
        self.bump_w = rng.uniform(width[0], width[1])
        self.bump_c = rng.uniform(0.0, L, 2)

    def b(self, x, y):
        x, y = np.asarray(x, dtype=float), np.asarray(y, dtype=float)
        out = np.zeros(np.broadcast(x, y).shape)
        for A, w, cx, cy in zip(self.amp, self.width, self.cx, self.cy):
            dx = periodic_distance(x, cx, self.L)
            dy = periodic_distance(y, cy, self.L)
            out += A * np.exp(-(dx * dx + dy * dy) / (2 * w * w))
        return out

    def bump(self, x, y):
        dx = periodic_distance(x, self.bump_c[0], self.L)
        dy = periodic_distance(y, self.bump_c[1], self.L)
        return np.exp(-(dx * dx + dy * dy) / (2 * self.bump_w ** 2))

    def eta(self, x, y):
        return 1.0 + 0.01 * self.bump(x, y)

    def state(self, x, y):
        """(h, hu, hv) at positions (x, y) and the bathymetry b."""
        b = self.b(x, y)
        h = self.eta(x, y) - b
        return np.stack([h, self.current[0] * h, self.current[1] * h]), b


def accept_seed(make, positions, seed, min_depth=0.1, tries=64):
    """First seed >= ``seed`` whose input has min depth >= ``min_depth`` at
    ``positions`` (a tuple of coordinate arrays)."""
    for s in range(seed, seed + tries):
        inp = make(s)
        u, _ = inp.state(*positions)
        if np.min(u[0]) >= min_depth:
            return inp, s
    raise RuntimeError("no admissible seed found")


def ensemble_members(n=256, seed=0, log2_range=(10, 16), degrees=(2, 3, 4)):
    """Instance list of the ragged ensemble: element count
    floor(2^U[10, 16]), degree uniform over ``degrees`` and an own seed."""
    rng = np.random.default_rng(seed)
    E = np.floor(2.0 ** rng.uniform(log2_range[0], log2_range[1], n)).astype(np.int64)
    N = rng.choice(np.asarray(degrees), n)
    seeds = rng.integers(0, 2 ** 31 - 1, n)
    return [dict(E=int(e), N=int(k), seed=int(s)) for e, k, s in zip(E, N, seeds)]
