"""Panel discretisation, local refinement and the index sets of Sec. 3.1.

* Panels are equal in the parameter t (Sec. 5 preamble; Fig. PerturbedBoundary:
  "uniformly distributed in parameterization space").  Panel j covers
  [2 pi j / P, 2 pi (j+1) / P].
* On each panel the 16 Gauss-Legendre nodes; the smooth quadrature weight is
  w = omega_q * h * |x'(t)| with h the half-width of the panel in t.
* Outward normal n = (y', -x') / |x'| (counter-clockwise curve), unit tangent
  t = x' / |x'|, signed curvature kappa = (x' y'' - y' x'') / |x'|^3.
* Local refinement (Sec. 3.1, Fig. PerturbedBoundary): each cut panel is
  replaced by 2^L sub-panels of equal t-width (reading of "split dyadically L
  levels"), each again carrying 16 Gauss-Legendre nodes.  The cut panels are a
  contiguous run j0, j0+1, ... taken modulo P (a run may wrap past t = 2 pi).

Index sets (Sec. 3.1): I_o = original points (panel order), I_c = points of
the cut panels, I_k = I_o minus I_c, I_p = the new points, I_n = I_k union I_p.
The refined ("n") order walks the original panels 0..P-1 and emits, for a cut
panel, its sub-panels in increasing t.  The added points are also numbered in
window order (j0 first), which is the order the extended system uses for I_p.
"""
import numpy as np

from .quadrature import gauss_legendre, NQ
from .curves import evaluate


def _nodes_on_intervals(kind, params, ta, tb):
    """Gauss-Legendre nodes on the t-intervals [ta_i, tb_i] (arrays)."""
    xi, om = gauss_legendre(NQ)
    ta = np.asarray(ta, dtype=np.float64)
    tb = np.asarray(tb, dtype=np.float64)
    half = 0.5 * (tb - ta)
    mid = 0.5 * (tb + ta)
    t = (mid[:, None] + half[:, None] * xi[None, :]).ravel()
    wq = (half[:, None] * om[None, :]).ravel()
    g = evaluate(kind, t, **params)
    speed = np.hypot(g["dx"], g["dy"])
    nx = g["dy"] / speed
    ny = -g["dx"] / speed
    kappa = (g["dx"] * g["ddy"] - g["dy"] * g["ddx"]) / speed ** 3
    return dict(t=t, x=g["x"], y=g["y"], nx=nx, ny=ny, w=wq * speed, kappa=kappa)


def wall_nodes(kind, params, n_panels):
    """Nodes of the original (reference) discretisation with P equal panels."""
    j = np.arange(n_panels, dtype=np.float64)
    h = 2.0 * np.pi / n_panels
    return _nodes_on_intervals(kind, params, j * h, (j + 1.0) * h)


def window(j0, m, n_panels):
    """Cut panels j0, j0+1, ..., j0+m-1 modulo P (window order)."""
    return [(j0 + i) % n_panels for i in range(m)]


def refined_panel_nodes(kind, params, n_panels, panel, level):
    """Nodes of the 2^level equal sub-panels of one original panel."""
    h = 2.0 * np.pi / n_panels
    ns = 2 ** level
    s = np.arange(ns, dtype=np.float64)
    ta = panel * h + s * (h / ns)
    tb = panel * h + (s + 1.0) * (h / ns)
    return _nodes_on_intervals(kind, params, ta, tb)


def _cat(parts):
    return {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}


def refine(kind, params, n_panels, panels, levels):
    """Locally refined discretisation.

    panels: cut panel ids in window order; levels: refinement level per panel.
    Returns dict with
      o      : original nodes (dict of arrays, panel order)
      p      : added nodes (window order)
      n      : refined nodes (refined order)
      I_k, I_c : indices into o
      n_src  : for each refined point, ('o', i) encoded as i >= 0 for a kept
               point and -(1 + q) for added point q (index into p).
    """
    o = wall_nodes(kind, params, n_panels)
    panels = [int(j) for j in panels]
    levels = [int(L) for L in levels]
    if len(set(panels)) != len(panels):
        raise ValueError("cut panels must be distinct")
    lev = dict(zip(panels, levels))
    p_parts, p_start = [], {}
    count = 0
    for j in panels:
        part = refined_panel_nodes(kind, params, n_panels, j, lev[j])
        p_start[j] = count
        count += part["x"].size
        p_parts.append(part)
    p = _cat(p_parts)
    cut = np.zeros(n_panels, dtype=bool)
    cut[panels] = True
    I_c = np.concatenate([np.arange(NQ * j, NQ * (j + 1)) for j in sorted(panels)])
    I_k = np.concatenate([np.arange(NQ * j, NQ * (j + 1))
                          for j in range(n_panels) if not cut[j]])
    n_src = []
    for j in range(n_panels):
        if cut[j]:
            npts = NQ * 2 ** lev[j]
            n_src.extend(-(1 + p_start[j] + q) for q in range(npts))
        else:
            n_src.extend(range(NQ * j, NQ * (j + 1)))
    n_src = np.asarray(n_src, dtype=np.int64)
    n = {}
    for key in o:
        vals = np.empty(n_src.size)
        kept = n_src >= 0
        vals[kept] = o[key][n_src[kept]]
        vals[~kept] = p[key][-(n_src[~kept] + 1)]
        n[key] = vals
    return dict(o=o, p=p, n=n, I_k=I_k, I_c=np.sort(I_c), n_src=n_src)


def dof(idx):
    """Interleaved degrees of freedom (2i, 2i+1) of point indices idx."""
    idx = np.asarray(idx, dtype=np.int64)
    return np.stack([2 * idx, 2 * idx + 1], axis=1).ravel()
