"""Pins of the FP64 oracle's plain random walker (Sec. III-B) against facts that
do not come from the oracle: hand-derived closed forms, a dense direct solve of
the defining linear system, the discrete maximum principle, multi-class
sum-to-one, symmetry and special cases."""
import math

import numpy as np
import pytest

import oracle as O
import phantoms as P
from conftest import load_golden


def _dense_reference(g, code, value, beta, w_min=1e-30):
    """Dense Dirichlet problem written independently of the oracle: energy
    D(x) = 1/2 sum w (x_p - x_q)^2 (Sec. III-B); its stationarity conditions
    on the free vertices are solved by Cholesky."""
    shape = g.shape
    n = g.size
    gf = g.ravel()
    L = np.zeros((n, n))
    idx = np.arange(n).reshape(shape)
    for axis in range(3):
        a = np.moveaxis(idx, axis, 0)[:-1].ravel()
        b = np.moveaxis(idx, axis, 0)[1:].ravel()
        for p, q in zip(a, b):
            if code.ravel()[p] == 2 or code.ravel()[q] == 2:
                continue
            w = max(np.exp(-beta * (gf[p] - gf[q]) ** 2), w_min)
            L[p, p] += w; L[q, q] += w; L[p, q] -= w; L[q, p] -= w
    U = np.flatnonzero(code.ravel() == 0)
    M = np.flatnonzero(code.ravel() == 1)
    xm = value.ravel()[M].astype(np.float64)
    A = L[np.ix_(U, U)]
    rhs = -L[np.ix_(U, M)] @ xm
    c = np.linalg.cholesky(A)
    xu = np.linalg.solve(c.T, np.linalg.solve(c, rhs))
    x = np.zeros(n)
    x[M] = xm
    x[U] = xu
    return x.reshape(shape)


@pytest.mark.parametrize("case", load_golden("voltage_divider.txt"), ids=lambda c: c["name"])
def test_golden_voltage_divider(case):
    nx, ny, nz = (int(v) for v in case["dims"])
    g = np.array(case["g"]).reshape(nz, ny, nx)
    code = np.array(case["code"], dtype=np.uint8).reshape(nz, ny, nx)
    value = np.array(case["value"]).reshape(nz, ny, nx)
    x, it, rr, st = O.rw_solve(g, code, value, case["beta"][0], w_min=0.0)
    assert st == 0
    np.testing.assert_allclose(x.ravel(), case["expect"], rtol=0, atol=1e-13)


@pytest.mark.parametrize("shape,beta,seed", [((3, 4, 5), 5.0, 1), ((8, 8, 8), 30.0, 2), ((2, 7, 3), 20.0, 3),
                                             ((6, 5, 8), 25.0, 4), ((1, 1, 9), 10.0, 5), ("ball", 130.0, 6)])
def test_cg_matches_dense_cholesky(shape, beta, seed):
    # uniform random intensities make beta = 130 numerically singular (weights
    # down to 1e-30); the phantom-like ball keeps Cholesky meaningful there
    if shape == "ball":
        c = P.ball_case(n=8, seed=seed, radius=2.5)
    else:
        c = P.random_case(shape, seed=seed, seed_frac=0.15)
    g = O.dequantize(O.quantize(c["volume"]))
    x, it, rr, st = O.rw_solve(g, c["code"], c["value"], beta)
    assert st == 0
    ref = _dense_reference(g, c["code"], c["value"].astype(np.float64), beta)
    assert np.max(np.abs(x - ref)) <= 1e-12


def test_absent_vertices_match_dense():
    c = P.random_case((6, 6, 6), seed=9, seed_frac=0.1)
    code = c["code"].copy()
    code[:, :, 4:] = 2          # a block of absent vertices: no edges
    g = O.dequantize(O.quantize(c["volume"]))
    x, _, _, st = O.rw_solve(g, code, c["value"], 20.0)
    assert st == 0
    keep = code != 2
    sub = (slice(None), slice(None), slice(0, 4))
    ref = _dense_reference(g[sub], code[sub], c["value"][sub].astype(np.float64), 20.0)
    assert np.max(np.abs(x[sub] - ref)) <= 1e-12
    assert np.all(x[~keep] == 0.0)


def test_linear_ramp_closed_form():
    # constant volume: every weight is 1; seed planes x = 0 (value 1) and
    # x = nx-1 (value 0); free voxels solve the 1-D discrete Laplace equation
    # with Neumann borders in y and z -> x_i = 1 - i/(nx-1).
    nz, ny, nx = 4, 5, 17
    g = np.full((nz, ny, nx), 0.5)
    code = np.zeros((nz, ny, nx), np.uint8)
    val = np.zeros((nz, ny, nx))
    code[:, :, 0] = 1; val[:, :, 0] = 1.0
    code[:, :, -1] = 1
    x, it, rr, st = O.rw_solve(g, code, val, 130.0)
    assert st == 0
    expect = 1.0 - np.arange(nx) / (nx - 1.0)
    assert np.max(np.abs(x - expect[None, None, :])) <= 1e-12


def test_maximum_principle_and_harmonic():
    c = P.random_case((10, 9, 11), seed=7, seed_frac=0.05)
    g = O.dequantize(O.quantize(c["volume"]))
    val = c["value"].astype(np.float64)
    x, it, rr, st = O.rw_solve(g, c["code"], val, 40.0)
    assert st == 0
    seeds = c["code"] == 1
    assert np.all(x[seeds] == val[seeds])
    lo, hi = val[seeds].min(), val[seeds].max()
    assert x.min() >= lo - 1e-12 and x.max() <= hi + 1e-12
    # each free voxel is the weighted mean of its neighbours
    nz, ny, nx = g.shape
    num = np.zeros_like(x); den = np.zeros_like(x)
    for axis in range(3):
        for sh in (1, -1):
            gn = np.roll(g, sh, axis=axis); xn = np.roll(x, sh, axis=axis)
            w = np.maximum(np.exp(-40.0 * (g - gn) ** 2), 1e-30)
            valid = np.ones_like(x, dtype=bool)
            sl = [slice(None)] * 3
            sl[axis] = 0 if sh == 1 else -1
            valid[tuple(sl)] = False
            num += np.where(valid, w * xn, 0.0); den += np.where(valid, w, 0.0)
    free = ~seeds
    assert np.max(np.abs(x[free] - num[free] / den[free])) < 1e-10


def test_multiclass_sums_to_one():
    # Sec. III-B: m runs, class i foreground, all other seeds background; the
    # exact probabilities of the m runs sum to 1 at every voxel.
    c = P.random_case((9, 8, 7), seed=11, seed_frac=0.08, levels=[0, 1, 2])
    g = O.dequantize(O.quantize(c["volume"]))
    cls = np.rint(c["value"]).astype(int)
    xs = []
    for k in range(3):
        val = np.where(c["code"] == 1, (cls == k).astype(np.float64), 0.0)
        x, _, _, st = O.rw_solve(g, c["code"], val, 60.0)
        assert st == 0
        xs.append(x)
    assert np.max(np.abs(sum(xs) - 1.0)) < 1e-10
    lab = np.argmax(np.stack(xs), axis=0)
    assert np.all(lab[c["code"] == 1] == cls[c["code"] == 1])


def test_mirror_symmetry():
    c = P.random_case((7, 8, 9), seed=12, seed_frac=0.1)
    g = O.dequantize(O.quantize(c["volume"]))
    x, _, _, _ = O.rw_solve(g, c["code"], c["value"], 50.0)
    xm, _, _, _ = O.rw_solve(g[:, :, ::-1].copy(), c["code"][:, :, ::-1].copy(), c["value"][:, :, ::-1].copy(), 50.0)
    assert np.max(np.abs(xm[:, :, ::-1] - x)) < 1e-11
    xt, _, _, _ = O.rw_solve(np.ascontiguousarray(g.transpose(2, 1, 0)), np.ascontiguousarray(c["code"].transpose(2, 1, 0)),
                             np.ascontiguousarray(c["value"].transpose(2, 1, 0)), 50.0)
    assert np.max(np.abs(xt.transpose(2, 1, 0) - x)) < 1e-11


def test_special_cases():
    c = P.random_case((6, 6, 6), seed=13, seed_frac=0.2)
    g = O.dequantize(O.quantize(c["volume"]))
    val = np.where(c["code"] == 1, 0.37, 0.0)
    x, _, _, st = O.rw_solve(g, c["code"], val, 20.0)
    assert st == 0 and np.max(np.abs(x - 0.37)) < 1e-11          # all seeds equal
    zero = np.zeros_like(val)
    x, it, _, st = O.rw_solve(g, c["code"], zero, 80.0)
    assert st == 0 and it == 0 and np.all(x == 0.0)               # b = 0 -> x_U = 0
    code0 = np.zeros_like(c["code"])
    _, _, _, st = O.rw_solve(g, code0, zero, 80.0)
    assert st == 2                                                # no seeds


def test_quantize_pins():
    v = np.array([-1.0, 0.0, 0.25, 0.5, 1.0, 2.0, np.nan, 1.0 / 65535.0 * 0.5], dtype=np.float32)
    q = O.quantize(v)
    assert q[0] == 0 and q[1] == 0 and q[4] == 65535 and q[5] == 65535 and q[6] == 0
    assert q[2] == 16384 and q[3] == 32768      # 0.25*65535 = 16383.75 -> 16384; 32767.5 -> 32768 (even)
    raw = np.array([0, 1000, 2500, 5000, 6000], dtype=np.uint16)
    q = O.quantize(raw, 0.0, 5000.0, True)
    assert list(q) == [0, 13107, 32768, 65535, 65535]   # 0.2*65535 = 13107; 0.5*65535 = 32767.5 -> 32768


def test_weight_formula():
    assert O.weight(0.3, 0.7, 130.0) == pytest.approx(np.exp(-130.0 * 0.16), rel=1e-15)
    assert O.weight(0.0, 1.0, 130.0) == 1e-30       # exp(-130) = 3.5e-57 is clamped at w_min
    assert O.weight(0.5, 0.5, 130.0) == 1.0


def test_config1_plain_ball_solution_properties():
    c = P.plain_ball()
    x, it, rr, st = O.solve_volume(c["volume"], c["code"], c["value"], 130.0)
    assert st == 0 and rr < 1e-12 and 100 < it < 5000
    assert x.min() >= -1e-12 and x.max() <= 1.0 + 1e-12
    seeds = c["code"] == 1
    assert np.all(x[seeds] == c["value"][seeds])
    # with sigma = 0.1 and beta = 130 the ball leaks through noisy boundary
    # edges, so only the neighbourhood of the seed line exceeds 0.5; the ball
    # still carries far more foreground probability than the background
    m = c["mask"]
    assert x[m].mean() > 5 * x[~m].mean()
    assert x[32, 32, 27] > 0.5 and x[32, 32, 37] > 0.5


def test_weakly_attached_pairs():
    # Each bright pair is joined internally by a weight-1 edge and to the rest
    # only through a ~2e-9 edge to its bridge voxel (other exits ~1e-28): its
    # two voxels share one value, the weighted mean of its exits, i.e. the
    # bridge voxel's value (Sec. III-B: every free voxel is the weighted mean
    # of its neighbours).  The pair's common mode has eigenvalue ~1e-9, so
    # the residual test resolves it only to ~1e-5.
    from conftest import determined_mask
    c = P.pocket_case()
    x, it, rr, st = O.solve_volume(c["volume"], c["code"], c["value"], 130.0, tol=1e-13)
    assert st == 0
    for (z, y, xx) in c["pairs"]:
        assert abs(x[z, y, xx] - x[z, y + 1, xx]) <= 1e-9
        assert abs(x[z, y, xx] - x[z, y, xx + 1]) <= 5e-5
    g = O.dequantize(O.quantize(c["volume"]))
    assert determined_mask(g, 130.0, seeds=c["code"] == 1).all()
    # without the seed information the seeded background cluster looks trapped
    assert not determined_mask(g, 130.0).all()


def test_poisson_weight_is_the_count_formula():
    # Sec. III-C case study: w = exp(-(sqrt(n_p) - sqrt(n_q))^2 / 2) on raw
    # counts; the oracle takes g = n / S with beta = S
    S = 255.0
    for na, nb in [(100, 100), (100, 81), (49, 64), (0, 9), (250, 30), (255, 0)]:
        want = max(math.exp(-0.5 * (math.sqrt(na) - math.sqrt(nb)) ** 2), O.W_MIN)
        got = O.weight(na / S, nb / S, S, kind="poisson")
        assert abs(got - want) <= 1e-12 * want


def test_poisson_voltage_divider():
    # seed 0 -- free -- seed 1 on a 1 x 1 x 3 chain: x = w2 / (w1 + w2)
    S = 255.0
    n = np.array([16.0, 25.0, 49.0])
    g = (n / S).reshape(1, 1, 3)
    code = np.array([O.SEED, O.FREE, O.SEED], np.uint8).reshape(1, 1, 3)
    xin = np.array([0.0, 0.0, 1.0]).reshape(1, 1, 3)
    x, it, rr, st = O.rw_solve(g, code, xin, S, kind="poisson")
    w1, w2 = math.exp(-0.5 * (4 - 5) ** 2), math.exp(-0.5 * (5 - 7) ** 2)
    assert st == 0 and abs(x[0, 0, 1] - w2 / (w1 + w2)) <= 1e-12


def _dense_laplacian(g, code, beta, w_min=1e-30):
    """Graph Laplacian of the 6-connected grid (Sec. III-B) without absent vertices, dense."""
    n = g.size
    L = np.zeros((n, n))
    idx = np.arange(n).reshape(g.shape)
    cf, gf = code.ravel(), g.ravel()
    for axis in range(3):
        a = np.moveaxis(idx, axis, 0)[:-1].ravel()
        b = np.moveaxis(idx, axis, 0)[1:].ravel()
        keep = (cf[a] != 2) & (cf[b] != 2)
        a, b = a[keep], b[keep]
        w = np.maximum(np.exp(-beta * (gf[a] - gf[b]) ** 2), w_min)
        np.add.at(L, (a, a), w)
        np.add.at(L, (b, b), w)
        np.add.at(L, (a, b), -w)
        np.add.at(L, (b, a), -w)
    return L


def test_residual_matches_dense_operator():
    # r = b - A x on the free vertices with b = -B^T x_M (+ an extra
    # right-hand side), A = L_U: written out with the dense Laplacian
    c = P.random_case((5, 6, 7), seed=14, seed_frac=0.15)
    code = c["code"].copy()
    code[1:3, 2:4, 4:6] = 2
    g = O.dequantize(O.quantize(c["volume"]))
    beta = 25.0
    x = P.uniform(14, 70, np.arange(g.size, dtype=np.uint64)).reshape(g.shape)
    x = np.where(code == 1, c["value"], x)
    extra = P.uniform(14, 71, np.arange(g.size, dtype=np.uint64)).reshape(g.shape) - 0.5
    L = _dense_laplacian(g, code, beta)
    U = np.flatnonzero(code.ravel() == 0)
    M = np.flatnonzero(code.ravel() == 1)
    xf = x.ravel()
    for rhs in (None, extra):
        b = -L[np.ix_(U, M)] @ xf[M] + (0.0 if rhs is None else rhs.ravel()[U])
        want = np.zeros(g.size)
        want[U] = b - L[np.ix_(U, U)] @ xf[U]
        r, bn = O.residual(g, code, x, beta, rhs=rhs)
        assert np.max(np.abs(r.ravel() - want)) <= 1e-13
        assert bn == pytest.approx(np.linalg.norm(b), rel=1e-14)
    # at the dense solution the residual vanishes
    xs = _dense_reference(g, code, np.where(code == 1, c["value"], 0.0), beta)
    r, bn = O.residual(g, code, xs, beta)
    assert np.max(np.abs(r)) <= 1e-13 * bn
