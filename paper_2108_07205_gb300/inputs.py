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
* added holes (App. B, Sec. 5.2: three circles of 10 panels in the channel,
  two below the centre line and one above; data from 5 exterior Stokeslets
  plus 2, 2 and 1 Stokeslets inside the holes): circles of radius 0.12 at
  (-7.5, -0.15), (6.5, -0.15), (8, 0.15), each x jittered by U[-0.3, 0.3];
  in the star wall, circles of radius 0.1 at distance 0.35 from the centre,
  angles 2 pi i / 3 + U[0, 0.4].  Stokeslets inside a hole sit within 0.4 R
  of its centre; fluid targets are the wall's targets with those closer
  than 2 R to a hole centre redrawn.
* exterior star (Sec. 2.2, Fig. demo_figs (b): the fluid outside the star
  wall): 3 Stokeslets inside the curve at radius U[0, 0.4] with angles
  U[0, 2 pi) and strengths N(0, I2); targets in the fluid at radius
  U[2, 3].  Outside the channel: 3 Stokeslets inside it at x ~ U[-8, 8],
  y ~ U[-0.1, 0.1]; targets at x ~ U[-12, 12], |y| ~ U[1.5, 3].
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


def stokeslets_inside_star(seed, nrhs=1, n=3, rmax=0.4):
    """Point forces inside the star wall (the exterior problem's data):
    positions (n,), (n,) and strengths (n, 2, nrhs)."""
    g = rng(seed)
    r = g.uniform(0.0, rmax, size=n)
    th = g.uniform(0.0, 2.0 * np.pi, size=n)
    f = g.standard_normal(size=(n, 2, nrhs))
    return r * np.cos(th), r * np.sin(th), f


def targets_outside_star(seed, n=16, r_lo=2.0, r_hi=3.0):
    """Targets in the fluid outside the star wall."""
    g = rng(seed)
    r = g.uniform(r_lo, r_hi, size=n)
    th = g.uniform(0.0, 2.0 * np.pi, size=n)
    return r * np.cos(th), r * np.sin(th)


def stokeslets_inside_channel(seed, nrhs=1, n=3):
    """Point forces inside the channel, the exterior problem's data (within
    the constriction's half-height 0.2): positions (n,), (n,) and strengths
    (n, 2, nrhs)."""
    g = rng(seed)
    sx = g.uniform(-8.0, 8.0, size=n)
    sy = g.uniform(-0.1, 0.1, size=n)
    f = g.standard_normal(size=(n, 2, nrhs))
    return sx, sy, f


def targets_outside_channel(seed, n=16):
    """Targets in the fluid outside the channel, above and below it."""
    g = rng(seed)
    tx = g.uniform(-12.0, 12.0, size=n)
    ty = g.uniform(1.5, 3.0, size=n) * np.where(g.uniform(size=n) < 0.5, -1.0, 1.0)
    return tx, ty


def targets_channel(seed, n=16):
    g = rng(seed)
    return g.uniform(-8.0, 8.0, size=n), g.uniform(-0.1, 0.1, size=n)


def holes_channel(seed, n_panels=10, radius=0.12):
    """Three circular holes in the constricted channel: list of dicts
    (cx, cy, R, a, k, P)."""
    g = rng(seed)
    base = [(-7.5, -0.15), (6.5, -0.15), (8.0, 0.15)]
    return [dict(cx=x + float(g.uniform(-0.3, 0.3)), cy=y, R=radius, a=0.0, k=1, P=n_panels) for x, y in base]


def holes_star(seed, n_panels=10, radius=0.1, n=3, a=0.0, k=1):
    """n holes inside the star wall at distance 0.35 from its centre."""
    g = rng(seed)
    out = []
    for i in range(n):
        th = 2.0 * np.pi * i / n + float(g.uniform(0.0, 0.4))
        out.append(dict(cx=0.35 * np.cos(th), cy=0.35 * np.sin(th), R=radius, a=a, k=k, P=n_panels))
    return out


def stokeslets_in_holes(seed, holes, counts, nrhs=1):
    """Point forces inside the holes (counts[i] in hole i, within 0.4 R of its
    centre): positions (n,), (n,) and strengths (n, 2, nrhs)."""
    g = rng(seed)
    sx, sy = [], []
    for h, c in zip(holes, counts):
        for _ in range(c):
            rad = 0.4 * h["R"] * np.sqrt(g.uniform())
            th = g.uniform(0.0, 2.0 * np.pi)
            sx.append(h["cx"] + rad * np.cos(th))
            sy.append(h["cy"] + rad * np.sin(th))
    f = g.standard_normal(size=(len(sx), 2, nrhs))
    return np.asarray(sx), np.asarray(sy), f


def targets_fluid(seed, holes, kind="channel", n=16):
    """Targets of the wall's recipe, redrawn while closer than 2 R to a hole
    centre."""
    draw = targets_channel if kind == "channel" else targets_star
    tx, ty = [], []
    s = seed
    while len(tx) < n:
        x, y = draw(s, n)
        s += 7919
        for a, b in zip(x, y):
            if all((a - h["cx"]) ** 2 + (b - h["cy"]) ** 2 >= (2.0 * h["R"]) ** 2 for h in holes) and len(tx) < n:
                tx.append(a)
                ty.append(b)
    return np.asarray(tx), np.asarray(ty)
