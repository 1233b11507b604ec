"""Closed wall curves x(t), t in [0, 2*pi), counter-clockwise, with exact first
and second derivatives.

The paper's geometries (spline channel, fish, Fallopian tube, star lattice) are
not available, so the walls are synthetic stand-ins with the same character:

* star: x(t) = r(t) (cos t, sin t), r(t) = 1 + a cos(k t).
* channel: a 20 x 1 rounded rectangle (superellipse |x/A|^p + |y/B|^p = 1,
  p = 8, A = 10, B = 0.5) whose y coordinate is scaled by
  c(x) = 1 - delta (1 + cos(pi x / A)) / 2 with delta = 0.6, i.e. a smooth
  constriction of absolute amplitude 0.3 = delta * B at x = 0 on both walls.

Derivatives come from second-order Taylor jets (forward-mode differentiation
written out below), so the normal and curvature are exact to rounding; the
tests pin them by the total curvature (2 pi), the enclosed area (closed form for
the star, shoelace on a fine polygon for the channel) and finite differences.
"""
import numpy as np


class Jet:
    """Value with first and second derivative in one variable: (f, f', f'')."""

    __slots__ = ("v", "d1", "d2")

    def __init__(self, v, d1=0.0, d2=0.0):
        self.v, self.d1, self.d2 = v, d1, d2

    @staticmethod
    def lift(o):
        return o if isinstance(o, Jet) else Jet(o, 0.0, 0.0)

    def __add__(self, o):
        o = Jet.lift(o)
        return Jet(self.v + o.v, self.d1 + o.d1, self.d2 + o.d2)

    __radd__ = __add__

    def __neg__(self):
        return Jet(-self.v, -self.d1, -self.d2)

    def __sub__(self, o):
        return self + (-Jet.lift(o))

    def __rsub__(self, o):
        return Jet.lift(o) + (-self)

    def __mul__(self, o):
        o = Jet.lift(o)
        return Jet(self.v * o.v,
                   self.d1 * o.v + self.v * o.d1,
                   self.d2 * o.v + 2.0 * self.d1 * o.d1 + self.v * o.d2)

    __rmul__ = __mul__

    def pow(self, a):
        """self**a for real a (self.v > 0 unless a is a positive integer)."""
        f0 = self.v ** a
        f1 = a * self.v ** (a - 1.0)
        f2 = a * (a - 1.0) * self.v ** (a - 2.0)
        return Jet(f0, f1 * self.d1, f2 * self.d1 ** 2 + f1 * self.d2)


def jcos(j):
    c, s = np.cos(j.v), np.sin(j.v)
    return Jet(c, -s * j.d1, -c * j.d1 ** 2 - s * j.d2)


def jsin(j):
    c, s = np.cos(j.v), np.sin(j.v)
    return Jet(s, c * j.d1, -s * j.d1 ** 2 + c * j.d2)


def star(t, a=0.3, k=5, scale=1.0):
    """Star wall r(t) = scale * (1 + a cos(k t)); returns (x, y) jets."""
    T = Jet(np.asarray(t, dtype=np.float64), 1.0, 0.0)
    r = scale * (1.0 + a * jcos(k * T))
    return r * jcos(T), r * jsin(T)


def channel(t, A=10.0, B=0.5, p=8, delta=0.6):
    """Constricted-channel wall; returns (x, y) jets."""
    T = Jet(np.asarray(t, dtype=np.float64), 1.0, 0.0)
    c, s = jcos(T), jsin(T)
    h = c.pow(p) + s.pow(p)          # cos^p + sin^p > 0 (p even)
    sc = h.pow(-1.0 / p)
    X = A * c * sc
    Yb = B * s * sc
    squeeze = 1.0 - 0.5 * delta * (1.0 + jcos((np.pi / A) * X))
    return X, Yb * squeeze


CURVES = {"star": star, "channel": channel}


def evaluate(kind, t, **params):
    """Position, first and second derivative of a named curve at t.

    Returns dict with x, y, dx, dy, ddx, ddy (arrays)."""
    X, Y = CURVES[kind](t, **params)
    return dict(x=X.v, y=Y.v, dx=X.d1, dy=Y.d1, ddx=X.d2, ddy=Y.d2)
