"""Stokes kernels and the Nystrom matrix of the interior double-layer BIE.

Sec. 2, with mu = 1 and r = x - y, n_y the outward normal at the source:

* Stokeslet (Eq. stokeslet):  S(x, y) = 1/(4 pi) (-log|r| I + r r^T / |r|^2).
* Double layer:               D(x, y) = 1/pi (r r^T / |r|^2) (r . n_y) / |r|^2.
* Interior BIE (Eq. interior_BIE): -1/2 tau + D tau = g; the rank-one
  nullspace is removed by N tau = n_x int tau . n_y ds_y (Remark 2.1,
  Eq. null), giving A = -1/2 I + D + N (Eq. interior_BIE_discretized2).

Nystrom discretisation (readings where the paper is silent):
* off-diagonal 2x2 block (i != j):  w_j D(x_i, x_j) + w_j n_i n_j^T;
* diagonal block: -1/2 I - (kappa_i w_i / (2 pi)) t_i t_i^T + w_i n_i n_i^T,
  the smooth limit of the double-layer kernel on the curve (the 2D Stokes
  double layer is smooth on a smooth curve, so no singular quadrature).
* degrees of freedom interleaved: (x-component, y-component) per point.

Interior velocity (Sec. 2.1): u(x) = sum_j w_j D(x, y_j) tau_j (no N term).
Pressure (Sec. 2): the double-layer velocity's pressure
p(x) = sum_j w_j P(x, y_j) . tau_j, P_j = (1/pi)(-n_j / r^2 + 2 r_j (r . n) / r^4);
the Stokeslet's pressure kernel is Q_j = r_j / (2 pi r^2).
"""
import numpy as np


def stokeslet_velocity(tx, ty, sx, sy, f):
    """u at targets (tx, ty) from point forces f (ns x 2 or ns x 2 x nrhs) at
    (sx, sy).  Returns array (nt, 2) or (nt, 2, nrhs)."""
    f = np.asarray(f, dtype=np.float64)
    squeeze = f.ndim == 2
    if squeeze:
        f = f[:, :, None]
    rx = np.asarray(tx)[:, None] - np.asarray(sx)[None, :]
    ry = np.asarray(ty)[:, None] - np.asarray(sy)[None, :]
    r2 = rx * rx + ry * ry
    lg = -0.5 * np.log(r2)
    c = 1.0 / (4.0 * np.pi)
    # u_a = sum_s c * ( -log r f_a + r_a (r . f) / r^2 )
    fx, fy = f[:, 0, :], f[:, 1, :]                       # (ns, nrhs)
    rdotf = rx[:, :, None] * fx[None] + ry[:, :, None] * fy[None]
    ux = c * np.sum(lg[:, :, None] * fx[None] + rx[:, :, None] * rdotf / r2[:, :, None], axis=1)
    uy = c * np.sum(lg[:, :, None] * fy[None] + ry[:, :, None] * rdotf / r2[:, :, None], axis=1)
    u = np.stack([ux, uy], axis=1)
    return u[:, :, 0] if squeeze else u


def stokeslet_pressure(tx, ty, sx, sy, f):
    """Pressure at targets of the point forces of stokeslet_velocity: the
    single-layer pressure kernel Q_j(x, y) = r_j / (2 pi r^2) of Sec. 2
    applied to the forces.  Returns (nt,) or (nt, nrhs)."""
    f = np.asarray(f, dtype=np.float64)
    squeeze = f.ndim == 2
    if squeeze:
        f = f[:, :, None]
    rx = np.asarray(tx)[:, None] - np.asarray(sx)[None, :]
    ry = np.asarray(ty)[:, None] - np.asarray(sy)[None, :]
    r2 = rx * rx + ry * ry
    fx, fy = f[:, 0, :], f[:, 1, :]
    rdotf = rx[:, :, None] * fx[None] + ry[:, :, None] * fy[None]
    p = np.sum(rdotf / r2[:, :, None], axis=1) / (2.0 * np.pi)
    return p[:, 0] if squeeze else p


def boundary_data(nodes, sx, sy, f):
    """g at the nodes (interleaved, length 2N, or 2N x nrhs)."""
    u = stokeslet_velocity(nodes["x"], nodes["y"], sx, sy, f)
    if u.ndim == 2:
        return u.reshape(-1)
    return u.reshape(-1, u.shape[2])


def matrix(nodes):
    """Dense A = -1/2 I + D + N on a node set (2N x 2N, interleaved)."""
    x, y = nodes["x"], nodes["y"]
    nx, ny, w, kap = nodes["nx"], nodes["ny"], nodes["w"], nodes["kappa"]
    N = x.size
    rx = x[:, None] - x[None, :]
    ry = y[:, None] - y[None, :]
    r2 = rx * rx + ry * ry
    np.fill_diagonal(r2, 1.0)
    rdn = rx * nx[None, :] + ry * ny[None, :]
    fac = w[None, :] * rdn / (np.pi * r2 * r2)
    Dxx, Dxy, Dyy = fac * rx * rx, fac * rx * ry, fac * ry * ry
    # diagonal: smooth limit -(kappa w / 2 pi) t t^T with t = (-ny, nx)
    d = -kap * w / (2.0 * np.pi)
    ii = np.arange(N)
    Dxx[ii, ii] = d * ny * ny
    Dxy[ii, ii] = -d * nx * ny
    Dyy[ii, ii] = d * nx * nx
    A = np.empty((2 * N, 2 * N))
    A[0::2, 0::2] = Dxx + nx[:, None] * nx[None, :] * w[None, :]
    A[0::2, 1::2] = Dxy + nx[:, None] * ny[None, :] * w[None, :]
    A[1::2, 0::2] = Dxy + ny[:, None] * nx[None, :] * w[None, :]
    A[1::2, 1::2] = Dyy + ny[:, None] * ny[None, :] * w[None, :]
    A[np.arange(2 * N), np.arange(2 * N)] -= 0.5
    return A


def velocity(nodes, tau, tx, ty):
    """Interior velocity u(x) = sum_j w_j D(x, y_j) tau_j at targets.

    tau: interleaved density (2N) or (2N x nrhs).  Returns (nt, 2[, nrhs])."""
    tau = np.asarray(tau, dtype=np.float64)
    squeeze = tau.ndim == 1
    if squeeze:
        tau = tau[:, None]
    rx = np.asarray(tx)[:, None] - nodes["x"][None, :]
    ry = np.asarray(ty)[:, None] - nodes["y"][None, :]
    r2 = rx * rx + ry * ry
    rdn = rx * nodes["nx"][None, :] + ry * nodes["ny"][None, :]
    fac = nodes["w"][None, :] * rdn / (np.pi * r2 * r2)
    tx_, ty_ = tau[0::2, :], tau[1::2, :]
    rdt = rx[:, :, None] * tx_[None] + ry[:, :, None] * ty_[None]
    ux = np.einsum("ij,ijr->ir", fac * rx, rdt)
    uy = np.einsum("ij,ijr->ir", fac * ry, rdt)
    u = np.stack([ux, uy], axis=1)
    return u[:, :, 0] if squeeze else u


def pressure(nodes, tau, tx, ty):
    """Interior pressure matching the double-layer velocity (Sec. 2):
    p(x) = sum_j w_j P(x, y_j) . tau_j with
    P_j(x, y) = (mu / pi) (-n_j(y) / r^2 + 2 r_j (r . n(y)) / r^4), mu = 1.
    tau: interleaved (2N) or (2N x nrhs).  Returns (nt,) or (nt, nrhs)."""
    tau = np.asarray(tau, dtype=np.float64)
    squeeze = tau.ndim == 1
    if squeeze:
        tau = tau[:, None]
    rx = np.asarray(tx)[:, None] - nodes["x"][None, :]
    ry = np.asarray(ty)[:, None] - nodes["y"][None, :]
    r2 = rx * rx + ry * ry
    nx, ny = nodes["nx"][None, :], nodes["ny"][None, :]
    rdn = rx * nx + ry * ny
    tx_, ty_ = tau[0::2, :], tau[1::2, :]
    # P . tau = (1/pi) ( -(n . tau) / r^2 + 2 (r . tau)(r . n) / r^4 )
    ndt = nx[:, :, None] * tx_[None] + ny[:, :, None] * ty_[None]
    rdt = rx[:, :, None] * tx_[None] + ry[:, :, None] * ty_[None]
    w = nodes["w"][None, :, None]
    term = w * (-ndt / r2[:, :, None] + 2.0 * rdt * rdn[:, :, None] / (r2 * r2)[:, :, None]) / np.pi
    p = np.sum(term, axis=1)
    return p[:, 0] if squeeze else p


def apply_rows(nodes, tau, rows):
    """(A tau)[rows] for selected interleaved DOFs, one row at a time.

    Used to check full-size results on sampled rows.  tau is 2N (or 2N x nrhs);
    rows are DOF indices.  Each row is the definition of A written out."""
    tau = np.asarray(tau, dtype=np.float64)
    squeeze = tau.ndim == 1
    if squeeze:
        tau = tau[:, None]
    out = np.empty((len(rows), tau.shape[1]))
    x, y = nodes["x"], nodes["y"]
    nx, ny, w, kap = nodes["nx"], nodes["ny"], nodes["w"], nodes["kappa"]
    flux = (w * nx) @ tau[0::2, :] + (w * ny) @ tau[1::2, :]   # int tau . n ds
    for r, dof in enumerate(rows):
        i, a = divmod(int(dof), 2)
        rx = x[i] - x
        ry = y[i] - y
        r2 = rx * rx + ry * ry
        r2[i] = 1.0
        rdn = rx * nx + ry * ny
        fac = w * rdn / (np.pi * r2 * r2)
        ra = rx if a == 0 else ry
        row_x = fac * ra * rx
        row_y = fac * ra * ry
        t = (-ny[i], nx[i])
        dk = -kap[i] * w[i] / (2.0 * np.pi)
        row_x[i] = dk * t[a] * t[0]
        row_y[i] = dk * t[a] * t[1]
        na = nx[i] if a == 0 else ny[i]
        out[r] = row_x @ tau[0::2, :] + row_y @ tau[1::2, :] + na * flux - 0.5 * tau[dof, :]
    return out[:, 0] if squeeze else out
