"""Pins for oracle/holes.py: the wall with added holes (App. B) and the
combined-field operator of Eq. exterior_BIE on the holes.

* logarithmic potential on a circle of radius R, at its own nodes:
  int log|x - y| cos(m theta_y) ds_y = 2 pi R log R (m = 0) and
  -(pi R / m) cos(m theta_x) (m >= 1), for every Fourier mode the panels
  resolve; the plain panel rule misses by O(0.1);
* single layer of a constant density c on a circle: (R / 4)(1 - 2 log R) c
  (the log part from the first pin, and int r r^T / |r|^2 ds = pi R I);
* closed form: in the fluid between the wall and the holes, the velocity of
  the solved density equals the field of the Stokeslets that made the data
  (outside the wall and inside every hole), with spectral decay under panel
  refinement, on the star wall (with circular and star-shaped holes) and the
  channel; planted mistakes -- the interior jump -1/2 on the holes, no
  single layer on the holes, the plain rule on the log singularity -- each
  break it (the N term extended over the holes does not: it is an
  equivalent reading for consistent data);
* the pressure of the same representation equals the Stokeslet pressure up to
  one constant;
* the row-at-a-time residual equals the dense system's.
"""
import numpy as np
import pytest

from oracle import holes as H, discretize as D, stokes as S
from paper_2108_07205_gb300 import inputs as I

STAR = dict(a=0.3, k=5)


def _circle(P=16, R=0.7):
    hl = [dict(cx=0.3, cy=-0.2, R=R, a=0.0, k=1, P=P)]
    return hl, H.hole_nodes(hl)


@pytest.mark.parametrize("m", list(range(0, 9)))
def test_log_potential_fourier_modes(m):
    R = 0.7
    hl, hn = _circle(16, R)
    Lw = H.log_matrix(hn, hl)
    th = hn["t"]
    for f, ex in ((np.cos(m * th), -(np.pi * R / max(m, 1)) * np.cos(m * th)),
                  (np.sin(m * th), -(np.pi * R / max(m, 1)) * np.sin(m * th))):
        if m == 0:
            if not f.any():
                continue
            ex = 2.0 * np.pi * R * np.log(R) * np.ones_like(th)
        assert np.abs(Lw @ f - ex).max() < 2e-14


def test_plain_rule_misses_the_log_singularity():
    R = 0.7
    hl, hn = _circle(16, R)
    rx = hn["x"][:, None] - hn["x"][None, :]
    ry = hn["y"][:, None] - hn["y"][None, :]
    r2 = rx * rx + ry * ry
    np.fill_diagonal(r2, 1.0)
    plain = 0.5 * np.log(r2) * hn["w"][None, :]
    assert np.abs(plain.sum(1) - 2.0 * np.pi * R * np.log(R)).max() > 1e-2


@pytest.mark.parametrize("R", [0.7, 1.3])
def test_single_layer_constant_density_circle(R):
    hl, hn = _circle(12, R)
    Sm = H.single_layer_matrix(hn, hl)
    c = np.tile([0.3, -0.7], hn["x"].size)
    assert np.abs(Sm @ c - 0.25 * R * (1.0 - 2.0 * np.log(R)) * c).max() < 1e-14


def _setup(kind, P, PH, hole_a=0.0, hole_k=1, nrhs=2):
    if kind == "star":
        wall = D.wall_nodes("star", STAR, P)
        hl = I.holes_star(3, n_panels=PH, a=hole_a, k=hole_k)
        sx, sy, f = I.stokeslets_star(0, nrhs=nrhs)
    else:
        wall = D.wall_nodes("channel", {}, P)
        hl = I.holes_channel(3, n_panels=PH)
        sx, sy, f = I.stokeslets_channel(0, nrhs=nrhs)
    hx, hy, hf = I.stokeslets_in_holes(1, hl, [2, 2, 1], nrhs=nrhs)
    sx, sy, f = np.concatenate([sx, hx]), np.concatenate([sy, hy]), np.concatenate([f, hf])
    hn = H.hole_nodes(hl)
    tx, ty = I.targets_fluid(2, hl, kind, 16)
    return wall, hl, hn, (sx, sy, f), (tx, ty)


def _error(wall, hl, hn, src, tg, A=None):
    sx, sy, f = src
    g = H.boundary_data(wall, hn, sx, sy, f)
    A = H.system(wall, hn, hl) if A is None else A
    tau = np.linalg.solve(A, g)
    u = H.velocity(wall, hn, tau, *tg)
    ue = S.stokeslet_velocity(*tg, sx, sy, f)
    return np.abs(u - ue).max() / np.abs(ue).max(), tau, g, A


def test_closed_form_star_with_holes_and_spectral_decay():
    errs = [_error(*_setup("star", P, PH))[0] for P, PH in ((8, 3), (12, 4), (16, 5), (32, 6))]
    assert errs[-1] < 1e-13
    assert errs[0] > errs[1] > errs[2]


def test_closed_form_star_shaped_holes():
    errs = [_error(*_setup("star", 32, PH, hole_a=0.2, hole_k=3))[0] for PH in (6, 8, 12)]
    assert errs[-1] < 1e-13
    assert errs[0] > errs[1] > errs[2]


def test_closed_form_channel_with_holes():
    err = _error(*_setup("channel", 256, 10))[0]
    assert err < 1e-11


def test_planted_mistakes_break_the_closed_form(monkeypatch):
    wall, hl, hn, src, tg = _setup("star", 32, 6)
    base = _error(wall, hl, hn, src, tg)[0]
    assert base < 1e-13
    # interior jump on the holes
    assert _error(wall, hl, hn, src, tg, H.system(wall, hn, hl, jump=-0.5))[0] > 1e-3
    # no single layer on the holes (double layer alone cannot carry a net force)
    nk = 2 * wall["x"].size
    A = H.system(wall, hn, hl)
    A[:, nk:] -= np.vstack([H.cross_single(wall, hn), H.single_layer_matrix(hn, hl)])
    assert _error(wall, hl, hn, src, tg, A)[0] > 1e-3
    # plain rule on the logarithmic singularity
    monkeypatch.setattr(H, "NEAR_PANELS", -1)
    A = H.system(wall, hn, hl)
    monkeypatch.undo()
    assert _error(wall, hl, hn, src, tg, A)[0] > 1e-3


def test_n_term_over_the_holes_is_equivalent():
    # Extending N to every point adds n_i times the total flux of tau, which
    # vanishes for consistent data: the same velocity (a reading, not a pin).
    wall, hl, hn, src, tg = _setup("star", 32, 6)
    nk = 2 * wall["x"].size
    allpts = {k: np.concatenate([wall[k], hn[k]]) for k in ("nx", "ny", "w")}
    nvec = np.ravel(np.stack([allpts["nx"], allpts["ny"]], 1))
    wn = np.ravel(np.stack([allpts["w"] * allpts["nx"], allpts["w"] * allpts["ny"]], 1))
    A = H.system(wall, hn, hl)
    A_full = A + np.outer(nvec, wn)
    A_full[:nk, :nk] -= np.outer(nvec[:nk], wn[:nk])
    e0, tau0, _, _ = _error(wall, hl, hn, src, tg, A)
    e1, tau1, _, _ = _error(wall, hl, hn, src, tg, A_full)
    assert e0 < 1e-13 and e1 < 1e-13
    assert np.abs(wn @ tau0).max() < 1e-12


def test_pressure_up_to_a_constant():
    wall, hl, hn, src, tg = _setup("star", 32, 6)
    _, tau, _, _ = _error(wall, hl, hn, src, tg)
    p = H.pressure(wall, hn, tau, *tg)
    pe = S.stokeslet_pressure(*tg, *src)
    d = p - pe
    assert np.abs(d - d.mean(axis=0)).max() < 1e-11 * np.abs(pe).max()


def test_apply_rows_matches_dense_system():
    wall, hl, hn, src, tg = _setup("star", 16, 4)
    A = H.system(wall, hn, hl)
    x = I.rng(5).standard_normal((A.shape[0], 3))
    rows = np.concatenate([I.rng(6).choice(2 * wall["x"].size, 7, replace=False),
                           2 * wall["x"].size + I.rng(7).choice(2 * hn["x"].size, 7, replace=False)])
    got = H.apply_rows(wall, hn, hl, x, rows)
    assert np.abs(got - (A @ x)[rows]).max() < 1e-13 * np.abs(A @ x).max()


@pytest.mark.parametrize("kind", ["channel", "star"])
def test_seeded_hole_layouts_are_valid(kind):
    # every seeded layout keeps its holes inside the wall, at least one hole
    # radius away from it, and apart from one another (the input recipe)
    from oracle.curves import evaluate
    t = np.linspace(0.0, 2.0 * np.pi, 20001)
    wall = evaluate("channel", t) if kind == "channel" else evaluate("star", t, a=0.3, k=5)
    for seed in range(20):
        hl = I.holes_channel(seed) if kind == "channel" else I.holes_star(seed)
        for i, h in enumerate(hl):
            d = np.hypot(wall["x"] - h["cx"], wall["y"] - h["cy"]).min()
            assert d >= 2.0 * h["R"], (seed, i, d)
            # inside: a ray to the right from the centre crosses the wall an odd number of times
            ys = wall["y"] - h["cy"]
            cross = (np.sign(ys[:-1]) != np.sign(ys[1:])) & (wall["x"][:-1] > h["cx"])
            assert cross.sum() % 2 == 1, (seed, i)
            for j in range(i):
                g = hl[j]
                assert np.hypot(h["cx"] - g["cx"], h["cy"] - g["cy"]) > 3.0 * max(h["R"], g["R"])
