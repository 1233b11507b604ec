"""Planted mistakes in the oracle's matrix are caught by its pins.

Each plant is a plausible error in assembling A = -1/2 I + D + N (Sec. 2,
Eq. interior_BIE_discretized2), made on the CPU by wrapping the oracle's own
matrix() for the duration of one test:
  * jump sign: +1/2 I instead of -1/2 I (the exterior limit);
  * diagonal sign: the curvature limit of D taken as +(kappa w / 2 pi) t t^T;
  * N weight index: w_i n_i n_j^T instead of w_j n_i n_j^T (Remark 2.1);
  * r sign: r = y - x in the off-diagonal double-layer entries.
The pins of tests/test_oracle_stokes.py (unit circle, left null vector,
closed-form interior velocity on the star, the channel and a refined star)
then run against the planted matrix; every plant must fail at least two of
them, so a mistake of this kind anywhere in the assembly cannot pass
unnoticed."""
import numpy as np
import pytest

import oracle.dense as DN
import oracle.stokes as S
import test_oracle_stokes as T

REAL_MATRIX = S.matrix


def _parts(n):
    """The correct matrix split into its terms (interleaved DOFs)."""
    A = REAL_MATRIX(n)
    N = n["x"].size
    nv = np.empty(2 * N)
    nv[0::2], nv[1::2] = n["nx"], n["ny"]
    wn = nv * np.repeat(n["w"], 2)
    Nterm = np.outer(nv, wn)                       # w_j n_i n_j^T
    d = -n["kappa"] * n["w"] / (2.0 * np.pi)
    curv = np.zeros_like(A)
    i = np.arange(N)
    curv[2 * i, 2 * i] = d * n["ny"] ** 2
    curv[2 * i, 2 * i + 1] = -d * n["nx"] * n["ny"]
    curv[2 * i + 1, 2 * i] = -d * n["nx"] * n["ny"]
    curv[2 * i + 1, 2 * i + 1] = d * n["nx"] ** 2
    return A, nv, Nterm, curv


def _jump(n):
    A = REAL_MATRIX(n)
    return A + np.eye(A.shape[0])


def _diag_sign(n):
    A, _, _, curv = _parts(n)
    return A - 2.0 * curv


def _n_index(n):
    A, nv, Nterm, _ = _parts(n)
    wi = np.repeat(n["w"], 2)
    return A - Nterm + np.outer(nv * wi, nv)       # w_i n_i n_j^T


def _r_sign(n):
    A, _, Nterm, curv = _parts(n)
    D_off = A - Nterm - curv + 0.5 * np.eye(A.shape[0])
    for i in range(n["x"].size):                   # the off-diagonal blocks only
        D_off[2 * i:2 * i + 2, 2 * i:2 * i + 2] = 0.0
    return A - 2.0 * D_off


PLANTS = {"jump sign": _jump, "diagonal sign": _diag_sign, "N weight index": _n_index, "r sign": _r_sign}

PINS = [
    ("unit circle", lambda: T.test_circle_constant_density(8)),
    ("left null vector (star)", lambda: T.test_left_null_vector_and_N("star", T.STAR, 32)),
    ("closed form (star)", T.test_closed_form_and_spectral_convergence_star),
    ("closed form (channel)", T.test_closed_form_channel),
    ("closed form (refined star)", T.test_closed_form_refined_star),
]


def test_unplanted_matrix_passes_every_pin():
    for _, pin in PINS:
        pin()


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_planted_mistake_is_caught(plant, monkeypatch):
    bad = PLANTS[plant]
    monkeypatch.setattr(S, "matrix", bad)
    monkeypatch.setattr(DN, "matrix", bad)
    caught = []
    for name, pin in PINS:
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError):
            caught.append(name)
    assert len(caught) >= 2, (plant, caught)
