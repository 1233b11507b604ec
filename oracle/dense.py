"""Dense reference solves: the refined system and the extended linear system.

* ``solve_refined``: tau_n = A_nn^{-1} g_n by LAPACK LU with partial pivoting
  (Eq. perturbedlLinearSystem).  The method of Sec. 3 reaches this result up
  to its compression tolerance, so this is the parity reference.
* ``extended_system``: A_ext = A~ + Q in the ordering [o ; p] (original points
  in panel order, then added points), Eq. extendedlLinearSystem with
  A~ = blkdiag(A_oo, A_pp) and the three nonzero blocks of Q (-A_kc, A_kp,
  A_pk).  The paper orders [k ; c ; p]; the permutation is immaterial.
* ``svd_factors``: truncated-SVD blockwise factors L_block, R_block
  (Eq. uniform_concat) and the recompressed L_optimal, R_optimal (Sec. 3.4).
* ``woodbury``: tau_ext by Eq. wood with dense A~^{-1}.
"""
import numpy as np
import scipy.linalg as sla

from .discretize import dof
from .stokes import matrix


def solve_refined(ref, g_n):
    """Dense LU solve of A_nn tau = g on the refined nodes."""
    A = matrix(ref["n"])
    lu = sla.lu_factor(A)
    return sla.lu_solve(lu, g_n)


def extended_system(ref):
    """Return dict with A_ext, At (= A~), Q, and index arrays (DOF level) of
    the blocks k, c (inside o) and p (offset by 2 N_o) in [o ; p] order."""
    o, p = ref["o"], ref["p"]
    No, Np = o["x"].size, p["x"].size
    allpts = {key: np.concatenate([o[key], p[key]]) for key in o}
    Abig = matrix(allpts)
    dk, dc = dof(ref["I_k"]), dof(ref["I_c"])
    dp = 2 * No + np.arange(2 * Np)
    Aext = Abig.copy()
    Aext[np.ix_(dk, dc)] = 0.0        # k rows, c columns
    Aext[np.ix_(dc, dp)] = 0.0        # c rows, p columns
    Aext[np.ix_(dp, dc)] = 0.0        # p rows, c columns
    At = np.zeros_like(Abig)
    At[:2 * No, :2 * No] = Abig[:2 * No, :2 * No]
    At[2 * No:, 2 * No:] = Abig[2 * No:, 2 * No:]
    Q = Aext - At
    return dict(A_ext=Aext, At=At, Q=Q, dk=dk, dc=dc, dp=dp, No=No, Np=Np)


def g_ext(ref, g_n):
    """Right-hand side of the extended system: (g_k, 0, g_p) in [o ; p]."""
    No, Np = ref["o"]["x"].size, ref["p"]["x"].size
    g = np.zeros((2 * (No + Np),) + np.shape(g_n)[1:])
    src = ref["n_src"]
    for i_n, s in enumerate(src):
        tgt = s if s >= 0 else No + (-(s + 1))
        g[2 * tgt:2 * tgt + 2] = g_n[2 * i_n:2 * i_n + 2]
    return g


def ext_to_n(ref, tau_ext):
    """Pick tau_n = (tau_k, tau_p) in refined order from tau_ext."""
    No = ref["o"]["x"].size
    src = ref["n_src"]
    idx = np.where(src >= 0, src, No + (-(src + 1)))
    return tau_ext[dof(idx)]


def _tsvd(M, tol):
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return U[:, :0], s[:0], Vt[:0]
    k = int(np.sum(s > tol * s[0]))
    return U[:, :k], s[:k], Vt[:k]


def svd_factors(ext, tol, recompress=True):
    """Blockwise truncated-SVD factors of Q (Eq. uniform_concat) and, if
    recompress, L_opt = U_block, R_opt = Sigma_block V_block^T R_block.

    Returns (L, R) with Q ~= L R."""
    Q = ext["Q"]
    n = Q.shape[0]
    dk, dc, dp = ext["dk"], ext["dc"], ext["dp"]
    blocks = [(dp, dk), (dk, dc), (dk, dp)]         # pk, kc, kp (column order of L_1)
    Ls, Rs = [], []
    for rows, cols in blocks:
        U, s, Vt = _tsvd(Q[np.ix_(rows, cols)], tol)
        Lb = np.zeros((n, U.shape[1]))
        Lb[rows] = U
        Rb = np.zeros((U.shape[1], n))
        Rb[:, cols] = s[:, None] * Vt
        Ls.append(Lb)
        Rs.append(Rb)
    Lblk, Rblk = np.hstack(Ls), np.vstack(Rs)
    if not recompress:
        return Lblk, Rblk
    U, s, Vt = _tsvd(Lblk, tol)
    return U, (s[:, None] * Vt) @ Rblk


def woodbury(ext, L, R, g):
    """tau_ext = A~^{-1} g - A~^{-1} L (I + R A~^{-1} L)^{-1} R A~^{-1} g
    (Eq. wood), dense.  Returns (tau_ext, W)."""
    lu = sla.lu_factor(ext["At"])
    y = sla.lu_solve(lu, g)
    X = sla.lu_solve(lu, L)
    W = np.eye(L.shape[1]) + R @ X
    z = np.linalg.solve(W, R @ y)
    return y - X @ z, W


def pinv_cond(M):
    """Condition number ||M^+|| ||M|| of a full-rank rectangular matrix
    (Lemma 3.1's kappa-hat), from its singular values."""
    s = np.linalg.svd(M, compute_uv=False)
    return s[0] / s[-1]
