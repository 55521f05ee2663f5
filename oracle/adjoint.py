"""Adjoint of the random walker solve — oracle (TEST INFRASTRUCTURE ONLY).

The paper defines the forward solve (Sec. III-B); the gradient is not in the
paper.  For A(w) x_U = b(w) and a loss l(x) the adjoint gives

    dl/dtheta = lambda^T (db/dtheta - dA/dtheta x_U),   A lambda = dl/dx_U.

``dense_adjoint`` assembles A, b and every dA/dtheta, db/dtheta densely
(tiny volumes, <= 12^3) and applies that formula literally;
``matfree_adjoint`` solves A lambda = dl/dx_U with the FP64 PCG and sums the
per-edge terms in C.  Both are checked against central finite differences.
"""
from __future__ import annotations

import numpy as np

from . import FREE, SEED, W_MIN, adjoint_grad, rw_solve


def _edges(shape):
    nz, ny, nx = shape
    idx = np.arange(nx * ny * nz).reshape(shape)
    out = []
    out.append((idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()))
    out.append((idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()))
    out.append((idx[:-1, :, :].ravel(), idx[1:, :, :].ravel()))
    return np.concatenate([a for a, _ in out]), np.concatenate([b for _, b in out])


def dense_system(g, code, value, beta, w_min=W_MIN):
    """Dense Laplacian L = D - W of the 6-connected graph (Sec. III-B) with
    w = max(exp(-beta d^2), w_min); returns (L, free index, seed index)."""
    g = np.asarray(g, dtype=np.float64).ravel()
    code = np.asarray(code).ravel()
    n = g.size
    i, j = _edges(np.asarray(value).shape)
    keep = (code[i] != 2) & (code[j] != 2)
    i, j = i[keep], j[keep]
    d = g[i] - g[j]
    w = np.maximum(np.exp(-beta * d * d), w_min)
    L = np.zeros((n, n))
    np.add.at(L, (i, j), -w)
    np.add.at(L, (j, i), -w)
    np.add.at(L, (i, i), w)
    np.add.at(L, (j, j), w)
    U = np.flatnonzero(code == FREE)
    M = np.flatnonzero(code == SEED)
    return L, U, M, (i, j, d, w)


def dense_solve(g, code, value, beta, w_min=W_MIN):
    """x from L_UU x_U = -L_UM x_M by Cholesky (tiny volumes only)."""
    L, U, M, _ = dense_system(g, code, value, beta, w_min)
    xm = np.asarray(value, dtype=np.float64).ravel()[M]
    A = L[np.ix_(U, U)]
    b = -L[np.ix_(U, M)] @ xm
    c = np.linalg.cholesky(A)
    xu = np.linalg.solve(c.T, np.linalg.solve(c, b))
    x = np.asarray(value, dtype=np.float64).ravel().copy()
    x[U] = xu
    x[code.ravel() == 2] = 0.0
    return x.reshape(np.asarray(value).shape)


def dense_adjoint(g, code, value, beta, dl_dx, w_min=W_MIN):
    """(dl/dg, dl/dbeta) by the dense adjoint formula, one parameter at a time."""
    shape = np.asarray(value).shape
    L, U, M, (ei, ej, d, w) = dense_system(g, code, value, beta, w_min)
    n = L.shape[0]
    xm = np.asarray(value, dtype=np.float64).ravel()[M]
    A = L[np.ix_(U, U)]
    b = -L[np.ix_(U, M)] @ xm
    xu = np.linalg.solve(A, b)
    x = np.asarray(value, dtype=np.float64).ravel().copy()
    x[U] = xu
    lam = np.linalg.solve(A, np.asarray(dl_dx, dtype=np.float64).ravel()[U])
    active = np.exp(-beta * d * d) > w_min
    dw_dbeta = np.where(active, -d * d * w, 0.0)
    dw_dgi = np.where(active, -2.0 * beta * d * w, 0.0)

    def dL_of(dw):
        dL = np.zeros((n, n))
        np.add.at(dL, (ei, ej), -dw)
        np.add.at(dL, (ej, ei), -dw)
        np.add.at(dL, (ei, ei), dw)
        np.add.at(dL, (ej, ej), dw)
        return dL

    def grad_from(dL):
        dA = dL[np.ix_(U, U)]
        db = -dL[np.ix_(U, M)] @ xm
        return float(lam @ (db - dA @ xu))

    dbeta = grad_from(dL_of(dw_dbeta))
    dg = np.zeros(n)
    for v in range(n):
        dw = np.where(ei == v, dw_dgi, 0.0) + np.where(ej == v, -dw_dgi, 0.0)
        if not np.any(dw):
            continue
        dg[v] = grad_from(dL_of(dw))
    return dg.reshape(shape), dbeta, x.reshape(shape)


def soft_dice(x, y, eps=1e-6):
    """Soft-Dice loss 1 - (2 sum xy + eps) / (sum x + sum y + eps) and dl/dx."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = 2.0 * np.sum(x * y) + eps
    S = np.sum(x) + np.sum(y) + eps
    return 1.0 - N / S, (N - 2.0 * y * S) / (S * S)


def matfree_adjoint(g, code, value, beta, dl_dx, x=None, w_min=W_MIN, tol=1e-13):
    """(dl/dg, dl/dbeta, x): lambda by FP64 PCG on the same SPD system (zero
    on seeds), then the per-edge sums in C."""
    code = np.asarray(code, dtype=np.uint8)
    if x is None:
        xin = np.where(code == SEED, value, 0.0)
        x, _, _, _ = rw_solve(g, code, xin, beta, w_min=w_min, tol=tol)
    zero = np.zeros(code.shape, dtype=np.float64)
    rhs = np.where(code == FREE, dl_dx, 0.0)
    lam, _, _, st = rw_solve(g, code, zero, beta, w_min=w_min, tol=tol, rhs=rhs)
    dg, db = adjoint_grad(g, code, x, lam, beta, w_min)
    return dg, db, x
