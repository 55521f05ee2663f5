"""Parity of the plain CUDA solve (rw_solve through the C ABI) with the FP64
oracle, element by element; edge cases; host/device pointer paths."""
import numpy as np
import pytest

import oracle as O
import phantoms as P

pytestmark = pytest.mark.gpu

TOL = 1e-4          # max abs probability error vs the FP64 oracle


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


def _solve(rw, c, **kw):
    storage = kw.pop("storage", rw.RW_STORE_UNORM16)
    x, st = rw.rw_solve(_cuda(c["volume"]), _cuda(c["code"]), _cuda(c["value"]), rw.Opts(**kw), storage=storage)
    return x.cpu().numpy().astype(np.float64), st


def _oracle(c, beta, storage_f32=False, tol=1e-13):
    if storage_f32:
        g = np.clip(c["volume"], 0, 1).astype(np.float64)
        xin = np.where(c["code"] == 1, c["value"], 0.0)
        x, it, rr, st = O.rw_solve(g, c["code"], xin, beta, tol=tol)
    else:
        x, it, rr, st = O.solve_volume(c["volume"], c["code"], c["value"], beta, tol=tol)
    assert st == 0
    return x


def _labels_agree(x, xo):
    far = np.abs(xo - 0.5) > 1e-3
    return np.array_equal(x[far] > 0.5, xo[far] > 0.5)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_plain_ball_64_parity(rw, precision):
    c = P.plain_ball()
    xo = _oracle(c, 130.0)
    x, st = _solve(rw, c, beta=130.0, tol=1e-8, precision=precision)
    assert np.max(np.abs(x - xo)) <= TOL
    assert _labels_agree(x, xo)
    assert st["rel_resid"] <= 1e-8 and st["iters"] > 100
    assert st["free_voxels"] == 238319


RAGGED = [((37, 23, 19), 1), ((5, 70, 33), 2), ((1, 1, 50), 3), ((2, 3, 1), 4), ((64, 17, 130), 5), ((9, 40, 41), 6)]


@pytest.mark.parametrize("shape,seed", RAGGED)
@pytest.mark.parametrize("beta,bound,tol", [(10.0, 1e-6, 1e-10), (25.0, TOL, 1e-13)])
def test_ragged_random_parity(rw, shape, seed, beta, bound, tol):
    # uniform noise: with beta = 10 every weight is >= exp(-10), so both FP64
    # references are accurate far below 1e-6.  With beta = 25 weights reach
    # exp(-25) ~ 1e-11: a segment attached only through such an edge moves the
    # residual by ~1e-11 x its error, so it is resolved only at a tolerance
    # that shows it (the 1 x 1 x 50 chain at 1e-13, where its FP32 rounds
    # stagnate and FP64 sweeps finish it); the configs' 1e-4 bound applies
    c = P.random_case(shape, seed=seed, seed_frac=0.05, beta=beta)
    xo = _oracle(c, beta, tol=1e-14)
    x, st = _solve(rw, c, beta=beta, tol=tol)
    assert np.max(np.abs(x - xo)) <= bound
    assert _labels_agree(x, xo)


@pytest.mark.parametrize("shape,seed", [((37, 23, 45), 1), ((21, 70, 33), 2), ((64, 17, 130), 5), ((9, 40, 41), 6),
                                        ((3, 30, 50), 7)])
def test_ragged_ball_beta130_parity(rw, shape, seed):
    # the configs' beta = 130 on ragged boxes: a noisy ball (sigma 0.1) centred
    # in the box, background border faces, a foreground line through the centre
    c = P.ball_case(seed=seed, radius=0.3 * sorted(shape)[1], shape=shape)
    xo = _oracle(c, 130.0)
    x, st = _solve(rw, c, beta=130.0, tol=1e-8)
    assert st["rel_resid"] <= 1e-8
    assert np.max(np.abs(x - xo)) <= TOL
    assert _labels_agree(x, xo)


def test_ill_conditioned_chain_falls_back_to_fp64(rw):
    # a 1-D chain with one seed and weights down to 1e-11: its far segment
    # hangs on a ~1e-11 edge (Jacobi-scaled eigenvalue ~1e-11, far below FP32
    # resolution).  An error e there adds only ~1e-11 e to the residual, so
    # the segment is resolved only by a tolerance at which that shows: at
    # 1e-13 the FP32 rounds stagnate and the solve finishes with FP64 sweeps.
    c = P.random_case((1, 1, 50), seed=3, seed_frac=0.05, beta=25.0)
    xo = _oracle(c, 25.0, tol=1e-14)
    x, st = _solve(rw, c, beta=25.0, tol=1e-13)
    assert st["rel_resid"] <= 1e-13
    assert st["fp64_fallbacks"] == 1
    assert np.max(np.abs(x - xo)) <= TOL
    # at 1e-10 only the residual bound is guaranteed for that segment
    x2, st2 = _solve(rw, c, beta=25.0, tol=1e-10)
    assert st2["rel_resid"] <= 1e-10


# every FP32 sweep tile (the autotuner's candidates and 32x8, the narrow-box tile)
STRIP_TILES = ["s64x11", "s32x22", "s32x20", "s64x8", "s40x20", "s40x8", "s32x20_d3", "s64x8_d3", "s32x22_d1",
               "s64x8_d1", "s64x14_d1", "r64x14_d2", "r64x14_d1", "r64x11_d2", "r64x11_d3", "r32x22_d2",
               "r32x20_d3", "r64x13_d3", "r64x12_d3", "r40x20_d2", "r40x20_d3", "r40x8_d2"]
F32_TILES = ["32x8"] + STRIP_TILES


@pytest.mark.parametrize("tile", F32_TILES)
def test_every_u16_tile_matches_oracle(rw, tile):
    c = P.plain_ball(n=48, seed=3)
    xo = _oracle(c, 130.0)
    x, st = _solve(rw, c, beta=130.0, tol=1e-9, tile=tile)
    assert np.max(np.abs(x - xo)) <= TOL
    assert st["tile"] == rw._abi.RW_TILE[tile]


@pytest.mark.parametrize("tile", F32_TILES)
@pytest.mark.parametrize("beta,bound", [(10.0, 1e-6), (30.0, TOL)])
def test_every_f32_tile_matches_oracle(rw, tile, beta, bound):
    # FP32 intensity storage (the gradient path) on a ragged box; beta = 30
    # lets uniform-noise weights reach exp(-30)
    c = P.random_case((45, 43, 85), seed=8, seed_frac=0.03, beta=beta)
    xo = _oracle(c, beta, storage_f32=True)
    x, st = _solve(rw, c, beta=beta, tol=1e-10, tile=tile, storage=rw.RW_STORE_F32)
    assert st["tile"] == rw._abi.RW_TILE[tile]
    assert np.max(np.abs(x - xo)) <= bound


def test_every_strip_tile_takes_the_same_iterations(rw):
    # the tiles differ only in how the sweep is cut into work items: the six
    # sums of every sweep must be the same up to rounding, so that each exact
    # line step leaves (D u', p_k) at rounding level and every tile needs the
    # same iterations (a tile whose per-item sums lost a term took 60 % more)
    c = P.random_case((9, 40, 41), seed=6, seed_frac=0.05, beta=25.0)
    its = {}
    for tile in STRIP_TILES:
        x, st = _solve(rw, c, beta=25.0, tol=1e-10, tile=tile)
        assert st["fp64_fallbacks"] == 0 and st["rel_resid"] <= 1e-10, tile
        its[tile] = st["iters"]
    ref = its["s40x20"]
    assert all(abs(v - ref) <= 0.05 * ref for v in its.values()), its


@pytest.mark.parametrize("tile", ["32x8", "40x8"])
def test_fp64_tiles(rw, tile):
    c = P.random_case((21, 45, 50), seed=9, seed_frac=0.05, beta=40.0)
    xo = _oracle(c, 40.0)
    x, st = _solve(rw, c, beta=40.0, tol=1e-11, precision="fp64", tile=tile)
    assert np.max(np.abs(x - xo)) <= 1e-7


def test_absent_voxels(rw):
    c = P.random_case((20, 22, 24), seed=10, seed_frac=0.05, beta=20.0)
    c["code"][:, 5:9, 3:20] = 2
    xo = _oracle(c, 20.0)
    x, st = _solve(rw, c, beta=20.0, tol=1e-10)
    assert np.max(np.abs(x - xo)) <= 1e-6
    assert np.all(x[c["code"] == 2] == 0.0)


def test_batch_of_volumes(rw):
    cs = [P.ball_case(n=32, seed=s, radius=9.0, ellipsoid=(s % 2 == 1)) for s in range(3)]
    vol = np.stack([c["volume"] for c in cs])
    code = np.stack([c["code"] for c in cs])
    val = np.stack([c["value"] for c in cs])
    x, st = rw.rw_solve(_cuda(vol), _cuda(code), _cuda(val), rw.Opts(beta=130.0, tol=1e-9))
    x = x.cpu().numpy()
    for b, c in enumerate(cs):
        assert np.max(np.abs(x[b] - _oracle(c, 130.0))) <= TOL


@pytest.mark.parametrize("variant", range(4))
def test_cluster_resident_rounds_continue_from_the_fp64_residual(rw, monkeypatch, variant):
    # 12 systems of 32^3, more than the resident 16-CTA clusters: each round
    # starts in the batched strip sweeps (which alternate the buffer parity
    # every sweep) and finishes in the cluster-resident solver (which goes on
    # from the system's own parity).  Six systems start near their solution
    # and finish in the first refinement round, so the second round of the six
    # cold ones runs in the cluster-resident solver from its first sweep.  The
    # FP64 residual between rounds moves every system to buffer 0; a round
    # that read the buffer of the last sweep instead would iterate on an old
    # residual, end short of the tolerance and fall back to FP64 sweeps.  The
    # warm starts' distance varies the parity at which the six cold systems
    # enter the cluster-resident solver.  Both modes must converge in FP32
    # rounds alone, in about the same number of iterations, to the oracle.
    n = 12
    cs = [P.ball_case(n=32, seed=60 + n * variant + s, radius=8.0 + (s % 4), ellipsoid=(s % 2 == 1))
          for s in range(n)]
    vol, code, val = (_cuda(np.stack([c[k] for c in cs])) for k in ("volume", "code", "value"))
    monkeypatch.setenv("RW_CLUSTER", "0")
    xr, _ = rw.rw_solve(vol, code, val, rw.Opts(beta=130.0, tol=1e-10, tile="s40x20"))
    x0 = xr.cpu().numpy()
    warm = np.arange(n) % 2 == 0
    rs = np.random.default_rng(variant)
    x0[warm] += np.float32(10.0 ** (-7 + 0.5 * variant)) * rs.standard_normal(x0[warm].shape).astype(np.float32)
    x0[~warm] = 0.0
    out = {}
    for mode in ("0", "1"):
        monkeypatch.setenv("RW_CLUSTER", mode)
        x, st = rw.rw_solve(vol, code, val, rw.Opts(beta=130.0, tol=1e-10, tile="s40x20"), x0=_cuda(x0))
        assert st["fp64_fallbacks"] == 0, (mode, st)
        assert st["refine_rounds"] >= 2 and st["rel_resid"] <= 1e-10
        out[mode] = (x.cpu().numpy().astype(np.float64), st)
    (xs, ss), (xc, sc) = out["0"], out["1"]
    assert not np.array_equal(xs, xc)           # the cluster-resident solver ran
    assert abs(sc["iters"] - ss["iters"]) <= 0.15 * ss["iters"]
    assert np.max(np.abs(xs - xc)) <= 1e-6
    for b in (1, 6):
        assert np.max(np.abs(xc[b] - _oracle(cs[b], 130.0))) <= TOL


def test_host_pointers_equal_device_pointers(rw):
    # one fixed tile: an autotuning call runs its tuning sweeps as real
    # iterations and rounds differently from a call with a cached choice
    c = P.plain_ball(n=40, seed=4)
    xd, _ = _solve(rw, c, beta=130.0, tol=1e-9, tile="s40x20")
    xh, st = rw.rw_solve(c["volume"], c["code"], c["value"], rw.Opts(beta=130.0, tol=1e-9, tile="s40x20"))
    assert isinstance(xh, np.ndarray)
    assert np.array_equal(xh.astype(np.float64), xd)


def test_deterministic(rw):
    c = P.plain_ball(n=40, seed=5)
    a, _ = _solve(rw, c, beta=130.0, tol=1e-9, tile="r64x14_d2")
    b, _ = _solve(rw, c, beta=130.0, tol=1e-9, tile="r64x14_d2")
    assert np.array_equal(a, b)


def test_edge_cases(rw):
    c = P.random_case((6, 7, 8), seed=11, seed_frac=0.1, beta=20.0)
    # no seeds at all: error
    c0 = dict(c, code=np.zeros_like(c["code"]))
    with pytest.raises(rw.RWError) as ei:
        _solve(rw, c0, beta=20.0)
    assert ei.value.status == 2
    # zero right-hand side: x_U = 0 exactly, even from a non-zero initial guess
    cz = dict(c, value=np.zeros_like(c["value"]))
    x0 = np.full(c["volume"].shape, 0.3, np.float32)
    x, st = rw.rw_solve(_cuda(cz["volume"]), _cuda(cz["code"]), _cuda(cz["value"]), rw.Opts(beta=20.0),
                        x0=_cuda(x0))
    assert np.all(x.cpu().numpy() == 0.0)
    # every voxel a seed: x = seeds
    ca = dict(c, code=np.ones_like(c["code"]))
    x, st = _solve(rw, ca, beta=20.0)
    assert np.array_equal(x, c["value"].astype(np.float32).astype(np.float64))
    # a single voxel volume with a seed
    c1 = {"volume": np.zeros((1, 1, 1), np.float32), "code": np.ones((1, 1, 1), np.uint8),
          "value": np.full((1, 1, 1), 0.25, np.float32)}
    x, st = _solve(rw, c1, beta=20.0)
    assert x[0, 0, 0] == 0.25


def test_warm_start_reaches_same_solution(rw):
    c = P.plain_ball(n=40, seed=6)
    xo = _oracle(c, 130.0)
    x0 = np.clip(xo + 0.05, 0, 1).astype(np.float32)
    x, st = rw.rw_solve(_cuda(c["volume"]), _cuda(c["code"]), _cuda(c["value"]), rw.Opts(beta=130.0, tol=1e-9),
                        x0=_cuda(x0))
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= TOL


def test_normalisation_window_u16_input(rw):
    ph = P.vessel_tree(n=48, seed=1, n_segments=12)
    vol = ph["volume"]
    code = np.zeros(vol.shape, np.uint8)
    val = np.zeros(vol.shape, np.float32)
    code[P.border_faces(vol.shape)] = 1
    z, y, x = (np.floor(ph["labels_xyz"][ph["labels_value"] == 1][:, ::-1])).astype(int).T
    code[z, y, x] = 1
    val[z, y, x] = 1.0
    q = O.quantize(vol, 0.0, 5000.0, True)
    xo, it, rr, st = O.rw_solve(O.dequantize(q), code, np.where(code == 1, val, 0.0), 130.0)
    # uint16 host array: staged by the library, normalised with the window
    xg, stg = rw.rw_solve(vol, code, val, rw.Opts(beta=130.0, tol=1e-9), lo=0.0, hi=5000.0, normalize=True)
    assert np.max(np.abs(xg - xo)) <= TOL


def test_ellipsoids_scaled_parity(rw):
    c = P.plain_ellipsoids(n=96, seed=0)
    xo = _oracle(c, 130.0, tol=1e-12)
    x, st = _solve(rw, c, beta=130.0, tol=1e-8)
    assert np.max(np.abs(x - xo)) <= TOL
    assert _labels_agree(x, xo)


def _residual_numpy(g, code, x, beta, w_min=1e-30):
    """FP64 residual of the Sec. III-B system computed in the test (property check)."""
    free = code == 0
    num = np.zeros_like(x)
    den = np.zeros_like(x)
    for axis in range(3):
        n = g.shape[axis]
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[axis] = slice(0, n - 1)
        b[axis] = slice(1, n)
        a, b = tuple(a), tuple(b)
        w = np.maximum(np.exp(-beta * (g[a] - g[b]) ** 2), w_min)
        num[a] += w * x[b]
        den[a] += w
        num[b] += w * x[a]
        den[b] += w
    r = np.where(free, num - den * x, 0.0)
    return r


def test_ellipsoids_256_full_size_properties(rw):
    """The 256^3 workload in the benchmark's launch configuration: properties
    that hold at any size (FP64 residual, maximum principle, seeds exact)."""
    c = P.plain_ellipsoids(n=256, seed=0)
    x, st = _solve(rw, c, beta=130.0, tol=1e-8)
    assert st["status"] == 0 and st["rel_resid"] <= 1e-8
    g = O.dequantize(O.quantize(c["volume"]))
    r = _residual_numpy(g, c["code"], x, 130.0)
    # b = sum over seeded neighbours of w m: recompute ||b|| with x = seeds only
    xs = np.where(c["code"] == 1, c["value"].astype(np.float64), 0.0)
    b = _residual_numpy(g, c["code"], xs, 130.0)
    # (output is rounded to FP32, so the residual of the stored x is ~1e-7 relative)
    assert np.linalg.norm(r) <= 1e-5 * np.linalg.norm(b)
    assert x.min() >= -1e-6 and x.max() <= 1 + 1e-6
    seeds = c["code"] == 1
    assert np.all(x[seeds] == c["value"][seeds])


def test_ellipsoids_256_full_size_parity(rw):
    """The benchmark's exact call on the 256^3 three-ellipsoid workload
    (tol 1e-8, autotuned tile, FP32 sweeps with FP64 refinement) against the
    FP64 oracle solved to 1e-13, element by element, with the thresholded
    labels bit-exact wherever the oracle is more than 1e-3 from 0.5.  (Every
    voxel of this system is numerically determined: no cluster hangs on
    w_min edges.)"""
    c = P.plain_ellipsoids(n=256, seed=0)
    x, st = _solve(rw, c, beta=130.0, tol=1e-8)
    assert st["status"] == 0 and st["rel_resid"] <= 1e-8
    xo = _oracle(c, 130.0)
    err = float(np.max(np.abs(x - xo)))
    assert err <= TOL, err
    assert _labels_agree(x, xo)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_weakly_attached_pairs_parity(rw, precision):
    # salt pairs whose common mode has eigenvalue ~1e-9: the FP32 sweep must
    # keep each weak edge's contribution (difference-form stencil); with the
    # d*p - sum(w p_j) form the FP32 operator loses it, is no longer positive
    # definite there, and the refinement rounds diverge
    c = P.pocket_case()
    xo = _oracle(c, 130.0)
    x, st = _solve(rw, c, beta=130.0, tol=1e-10, precision=precision)
    assert st["rel_resid"] <= 1e-10
    assert st["fp64_fallbacks"] == 0
    assert np.max(np.abs(x - xo)) <= TOL
    for (z, y, xx) in c["pairs"]:
        assert abs(x[z, y, xx] - x[z, y + 1, xx]) <= 1e-5


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_poisson_weights_parity(rw, precision):
    # counts normalised by S = 255 (window [0, 255]); beta = S makes the
    # weights exp(-(sqrt(n_p) - sqrt(n_q))^2 / 2) on the counts
    S = 255.0
    c = P.poisson_ball(n=48, seed=2)
    x, st = rw.rw_solve(_cuda(c["volume"]), _cuda(c["code"]), _cuda(c["value"]),
                        rw.Opts(beta=S, tol=1e-10, precision=precision, weight="poisson"),
                        lo=0.0, hi=S, normalize=True)
    xo, it, rr, so = O.solve_volume(c["volume"], c["code"], c["value"], S, lo=0.0, hi=S, normalize=True,
                                    kind="poisson")
    assert so == 0
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= TOL
    with pytest.raises(rw.RWError):
        rw.rw_solve_adjoint(_cuda(c["volume"].astype(np.float32) / S), _cuda(c["code"]), x,
                            torch_ones_like(x), rw.Opts(beta=S, weight="poisson"))


def torch_ones_like(x):
    import torch
    return torch.ones_like(x)
