"""Parity of the CUDA adjoint (rw_solve_adjoint, RWSolveFn) with the oracle's
adjoint and with central finite differences."""
import numpy as np
import pytest

import oracle as O
import phantoms as P
from oracle import adjoint as OA

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rw():
    import torch
    assert torch.cuda.is_available()
    import paper_2103_09564_gb300 as m
    m.load()
    return m


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,seed,beta", [(12, 0, 130.0), (24, 1, 130.0), (17, 2, 60.0)])
def test_adjoint_matches_oracle(rw, n, seed, beta):
    c = P.ball_case(n=n, seed=seed, radius=0.3 * n, ellipsoid=(seed % 2 == 1))
    g = c["volume"].astype(np.float64)
    xo, _, _, _ = O.rw_solve(g, c["code"], np.where(c["code"] == 1, c["value"], 0.0), beta)
    _, dl = OA.soft_dice(xo, c["mask"])
    dgo, dbo, _ = OA.matfree_adjoint(g, c["code"], c["value"], beta, dl, x=xo)
    opts = rw.Opts(beta=beta, tol=1e-10)
    x, _ = rw.rw_solve(_cuda(c["volume"]), _cuda(c["code"]), _cuda(c["value"]), opts, storage=rw.RW_STORE_F32)
    dg, db, st = rw.rw_solve_adjoint(_cuda(c["volume"]), _cuda(c["code"]), x, _cuda(dl.astype(np.float32)), opts)
    assert abs(db[0] - dbo) <= 1e-4 * abs(dbo)
    assert np.max(np.abs(dg.cpu().numpy() - dgo)) <= 1e-3 * np.max(np.abs(dgo))


def test_dense_adjoint_on_12_cubed_crop(rw):
    # a 12^3 crop straddling the ball surface; seeds = crop border valued by the mask
    c = P.ball_case(n=48, seed=4, radius=14.0)
    sl = (slice(18, 30), slice(18, 30), slice(3, 15))
    vol = np.ascontiguousarray(c["volume"][sl])
    mask = c["mask"][sl]
    code = np.zeros(vol.shape, np.uint8)
    code[P.border_faces(vol.shape)] = 1
    val = np.where(code == 1, mask.astype(np.float32), 0.0).astype(np.float32)
    beta = 130.0
    g = vol.astype(np.float64)
    xo = OA.dense_solve(g, code, val, beta)
    _, dl = OA.soft_dice(xo, mask)
    dgo, dbo, _ = OA.dense_adjoint(g, code, val, beta, dl)
    opts = rw.Opts(beta=beta, tol=1e-11)
    x, _ = rw.rw_solve(_cuda(vol), _cuda(code), _cuda(val), opts, storage=rw.RW_STORE_F32)
    dg, db, _ = rw.rw_solve_adjoint(_cuda(vol), _cuda(code), x, _cuda(dl.astype(np.float32)), opts)
    assert abs(db[0] - dbo) <= 1e-4 * abs(dbo)
    assert np.max(np.abs(dg.cpu().numpy() - dgo)) <= 1e-3 * np.max(np.abs(dgo))


def _oracle_loss(g, code, value, beta, mask):
    x, _, _, st = O.rw_solve(g, code, np.where(code == 1, value, 0.0), beta, tol=1e-14)
    assert st in (0, 3)
    return OA.soft_dice(x, mask)[0]


@pytest.mark.parametrize("n,seed", [(16, 0), (20, 3)])
def test_adjoint_matches_oracle_finite_differences(rw, n, seed):
    # central differences of the FP64 oracle's forward solve (step 1e-3): the
    # GPU adjoint's dl/dbeta within 1e-4 relative, dl/dg within 1e-3 of
    # max |dl/dg| at a spread of free voxels and at the largest one
    c = P.ball_case(n=n, seed=seed, radius=0.3 * n, ellipsoid=(seed % 2 == 1))
    beta, h = 130.0, 1e-3
    g = c["volume"].astype(np.float64)
    xo, _, _, _ = O.rw_solve(g, c["code"], np.where(c["code"] == 1, c["value"], 0.0), beta, tol=1e-14)
    _, dl = OA.soft_dice(xo, c["mask"])
    opts = rw.Opts(beta=beta, tol=1e-10)
    x, _ = rw.rw_solve(_cuda(c["volume"]), _cuda(c["code"]), _cuda(c["value"]), opts, storage=rw.RW_STORE_F32)
    dg, db, _ = rw.rw_solve_adjoint(_cuda(c["volume"]), _cuda(c["code"]), x, _cuda(dl.astype(np.float32)), opts)
    dg = dg.cpu().numpy().astype(np.float64)
    fd_b = (_oracle_loss(g, c["code"], c["value"], beta + h, c["mask"]) -
            _oracle_loss(g, c["code"], c["value"], beta - h, c["mask"])) / (2 * h)
    assert abs(db[0] - fd_b) <= 1e-4 * abs(fd_b)
    scale = np.max(np.abs(dg))
    free = np.flatnonzero(c["code"].ravel() == 0)
    for v in list(free[:: max(1, len(free) // 10)]) + [int(np.argmax(np.abs(dg)))]:
        gp = g.copy().ravel(); gp[v] += h
        gm = g.copy().ravel(); gm[v] -= h
        fd = (_oracle_loss(gp.reshape(g.shape), c["code"], c["value"], beta, c["mask"]) -
              _oracle_loss(gm.reshape(g.shape), c["code"], c["value"], beta, c["mask"])) / (2 * h)
        assert abs(fd - dg.ravel()[v]) <= 1e-3 * scale


def _autograd_fd_check(rw, n, batch):
    """Soft-Dice loss over a batch through RWSolveFn: the adjoint's gradients
    with respect to beta and to the three largest-gradient intensities agree
    with central finite differences of the GPU forward solve.  Its FP32
    output limits these differences (a one-voxel step of 2^-10 moves the loss
    by little more than the output's rounding), hence the looser bounds; the
    FP64 differences of the oracle pin the adjoint to 1e-4 / 1e-3 above."""
    import torch
    from paper_2103_09564_gb300.autograd import RWSolveFn
    b = P.adjoint_batch(n=n, batch=batch)
    g = _cuda(b["volume"]).requires_grad_(True)
    beta = torch.tensor(130.0, device="cuda", requires_grad=True)
    code, val = _cuda(b["code"]), _cuda(b["value"])
    y = _cuda(b["mask"].astype(np.float32))
    kw = {"tol": 1e-10}

    def loss_of(gv, bv):
        # the loss is evaluated in FP64: an FP32 sum cannot resolve the
        # finite-difference change of the loss
        x = RWSolveFn.apply(gv, bv, code, val, kw).double()
        yd = y.double()
        inter = (x * yd).sum(dim=(1, 2, 3))
        den = x.sum(dim=(1, 2, 3)) + yd.sum(dim=(1, 2, 3))
        return (1 - (2 * inter + 1e-6) / (den + 1e-6)).mean()

    L = loss_of(g, beta)
    L.backward()
    h = 0.0625          # exactly representable, so beta +- h is exact in FP32
    with torch.no_grad():
        fd = (loss_of(g, beta + h) - loss_of(g, beta - h)).item() / (2 * h)
    assert abs(beta.grad.item() - fd) <= 1e-3 * abs(fd) + 1e-9
    gg = g.grad.cpu().numpy()
    idx = np.unravel_index(np.argsort(-np.abs(gg).ravel())[:3], gg.shape)
    h = 2.0 ** -10
    for k in range(3):
        i = tuple(int(v[k]) for v in idx)
        gp = g.detach().clone(); gp[i] += h
        gm = g.detach().clone(); gm[i] -= h
        with torch.no_grad():
            fdg = (loss_of(gp, beta) - loss_of(gm, beta)).item() / (2 * h)
        assert abs(gg[i] - fdg) <= 2e-2 * abs(gg).max()


def test_autograd_function_batch_and_fd(rw):
    _autograd_fd_check(rw, 16, 4)


def test_autograd_full_size_batch_fd(rw):
    # the differentiable workload at full size: 32 volumes of 96^3, as the
    # benchmark solves them
    _autograd_fd_check(rw, 96, 32)
