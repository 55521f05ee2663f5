"""Pins of the oracle's adjoint gradient: central finite differences of the
forward solve (independent of any adjoint code) and dense vs matrix-free."""
import numpy as np

import oracle as O
import phantoms as P
from oracle import adjoint as A


def _loss(g, code, value, beta, mask):
    x, _, _, st = O.rw_solve(g, code, np.where(code == 1, value, 0.0), beta, tol=1e-14)
    assert st in (0, 3)
    return A.soft_dice(x, mask)[0]


def test_dense_adjoint_matches_finite_differences():
    c = P.ball_case(n=6, seed=4, radius=1.8, sigma=0.05)
    g = c["volume"].astype(np.float64)
    beta = 20.0
    x = A.dense_solve(g, c["code"], c["value"], beta)
    _, dl_dx = A.soft_dice(x, c["mask"])
    dg, db, _ = A.dense_adjoint(g, c["code"], c["value"], beta, dl_dx)
    h = 1e-3
    fd_b = (_loss(g, c["code"], c["value"], beta + h, c["mask"]) -
            _loss(g, c["code"], c["value"], beta - h, c["mask"])) / (2 * h)
    assert abs(fd_b - db) <= 1e-4 * max(abs(db), 1e-8)
    scale = np.max(np.abs(dg))
    assert scale > 1e-6 and abs(db) > 1e-8
    free = np.flatnonzero(c["code"].ravel() == 0)
    for v in list(free[:: max(1, len(free) // 12)]) + [int(np.argmax(np.abs(dg)))]:
        gp = g.copy().ravel(); gp[v] += h
        gm = g.copy().ravel(); gm[v] -= h
        fd = (_loss(gp.reshape(g.shape), c["code"], c["value"], beta, c["mask"]) -
              _loss(gm.reshape(g.shape), c["code"], c["value"], beta, c["mask"])) / (2 * h)
        assert abs(fd - dg.ravel()[v]) <= 1e-3 * scale


def test_matfree_adjoint_matches_dense():
    c = P.ball_case(n=7, seed=5, radius=2.2, sigma=0.05)
    g = c["volume"].astype(np.float64)
    beta = 40.0
    x = A.dense_solve(g, c["code"], c["value"], beta)
    _, dl_dx = A.soft_dice(x, c["mask"])
    dg, db, _ = A.dense_adjoint(g, c["code"], c["value"], beta, dl_dx)
    dg2, db2, x2 = A.matfree_adjoint(g, c["code"], c["value"], beta, dl_dx)
    assert np.max(np.abs(x2 - x)) < 1e-11
    assert abs(db2 - db) <= 1e-9 * max(1.0, abs(db))
    assert np.max(np.abs(dg2 - dg)) <= 1e-9 * max(1.0, np.max(np.abs(dg)))
