"""Seeded synthetic inputs shared by the tests, the bench and the oracle legs.

Only random draws live here (numpy PCG64): refinement windows and levels,
Stokeslet positions and strengths, interior target points, and the named wall
configurations.  No arithmetic of the method (kernels, quadrature, solves) is
in this module; each side computes boundary data and everything else itself.

Workload recipes (the paper's geometries are not available, Sec. 5):

* ``star``: r(t) = 1 + a cos(k t); 3 Stokeslets at radius 2 with angles
  U[0, 2 pi) and strengths N(0, I2); targets at radius U[0, 0.5].
* ``channel``: the constricted 20 x 1 channel; 5 exterior Stokeslets per
  right-hand side (Sec. 5.2 uses 5), x ~ U[-10, 10], y = +-U[1, 3];
  targets x ~ U[-8, 8], |y| <= 0.1 (inside the 0.4-wide constriction).
* time stepping: an 8-panel window starting at a seeded j0 that advances one
  panel per step (modulo P), levels ~ U{2..5} per step.
"""
import numpy as np

WALLS = {
    # name: (curve kind, params, panels, leaf points, ID tolerance)
    "star64": ("star", dict(a=0.3, k=5), 64, 64, 1e-12),
    "channel1024": ("channel", dict(), 1024, 64, 1e-12),
    "channel2048": ("channel", dict(), 2048, 64, 1e-12),
}


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def refinement_window(seed, n_panels, m, level_lo, level_hi):
    """Contiguous window of m panels at a seeded start (modulo P) and one
    seeded level in [level_lo, level_hi] applied to every panel."""
    g = rng(seed)
    j0 = int(g.integers(0, n_panels))
    L = int(g.integers(level_lo, level_hi + 1))
    return [(j0 + i) % n_panels for i in range(m)], [L] * m


def time_schedule(seed, n_panels, steps, m=8, level_lo=2, level_hi=5):
    """Moving-window schedule: list of (panels, levels) per step."""
    g = rng(seed)
    j0 = int(g.integers(0, n_panels))
    out = []
    for s in range(steps):
        L = int(g.integers(level_lo, level_hi + 1))
        out.append(([(j0 + s + i) % n_panels for i in range(m)], [L] * m))
    return out


def stokeslets_star(seed, nrhs=1, n=3, radius=2.0):
    """Point forces outside the star wall: positions (n,), (n,) and
    strengths (n, 2, nrhs)."""
    g = rng(seed)
    th = g.uniform(0.0, 2.0 * np.pi, size=n)
    f = g.standard_normal(size=(n, 2, nrhs))
    return radius * np.cos(th), radius * np.sin(th), f


def stokeslets_channel(seed, nrhs=1, n=5):
    """Point forces outside the channel (above and below it)."""
    g = rng(seed)
    sx = g.uniform(-10.0, 10.0, size=n)
    sy = g.uniform(1.0, 3.0, size=n) * np.where(g.uniform(size=n) < 0.5, -1.0, 1.0)
    f = g.standard_normal(size=(n, 2, nrhs))
    return sx, sy, f


def stokeslet_pairs_channel(seed, nrhs):
    """One pair of exterior point forces per right-hand side (positions and
    strengths drawn per pair): positions (2 nrhs,), (2 nrhs,) and strengths
    (2 nrhs, 2, nrhs) with right-hand side r driven only by its own pair."""
    g = rng(seed)
    sx = g.uniform(-10.0, 10.0, size=2 * nrhs)
    sy = g.uniform(1.0, 3.0, size=2 * nrhs) * np.where(g.uniform(size=2 * nrhs) < 0.5, -1.0, 1.0)
    f = np.zeros((2 * nrhs, 2, nrhs))
    for r in range(nrhs):
        f[2 * r:2 * r + 2, :, r] = g.standard_normal(size=(2, 2))
    return sx, sy, f


def targets_star(seed, n=16):
    g = rng(seed)
    r = g.uniform(0.0, 0.5, size=n)
    th = g.uniform(0.0, 2.0 * np.pi, size=n)
    return r * np.cos(th), r * np.sin(th)


def targets_channel(seed, n=16):
    g = rng(seed)
    return g.uniform(-8.0, 8.0, size=n), g.uniform(-0.1, 0.1, size=n)
