"""rw_solve_noalloc: the plain solve for callers that cannot allocate device
memory (its scratch is a fixed device array inside the library).  Collected
last on purpose, so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process as well.  Results are
compared with the FP64 oracle and with rw_solve, the entry point it stands in
for, on consecutive calls."""
import ctypes

import numpy as np
import pytest

import oracle as O
import phantoms as P

pytestmark = pytest.mark.gpu
TOL = 1e-4        # the parity tolerance of the plain-solve tests


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


def test_noalloc_matches_oracle_and_rw_solve_on_two_calls(rw):
    # 64^3 = RW_NOALLOC_MAX_VOXELS, the largest input the fixed scratch takes
    c = P.plain_ball()
    vol, code, val = _cuda(c["volume"]), _cuda(c["code"]), _cuda(c["value"])
    opts = rw.Opts(beta=130.0, tol=1e-8)
    ref, st_ref = rw.rw_solve(vol, code, val, opts)
    ref = ref.cpu().numpy()
    xo, _, _, so = O.solve_volume(c["volume"], c["code"], c["value"], 130.0)
    assert so == 0
    seeds = c["code"] == 1
    for call in range(2):
        x, st = rw.rw_solve_noalloc(vol, code, val, opts)
        x = x.cpu().numpy()
        assert st["status"] == 0 and st["rel_resid"] <= 1e-8, (call, st)
        assert np.max(np.abs(x - xo)) <= TOL, call
        assert np.max(np.abs(x - ref)) <= TOL, call
        assert np.all(x[seeds] == c["value"][seeds])
        far = np.abs(xo - 0.5) > 1e-3
        assert np.array_equal(x[far] > 0.5, xo[far] > 0.5)


def test_noalloc_batch_with_initial_guess_on_a_side_stream(rw):
    # 8 volumes of 32^3 (balls and ellipsoids), one started from an initial
    # guess, on a non-default stream: every volume matches the oracle and
    # rw_solve (same x0) on two consecutive calls
    import torch
    cs = [P.ball_case(n=32, seed=s, radius=9.0, ellipsoid=(s % 2 == 1)) for s in range(8)]
    vol = _cuda(np.stack([c["volume"] for c in cs]))
    code = _cuda(np.stack([c["code"] for c in cs]))
    val = _cuda(np.stack([c["value"] for c in cs]))
    x0 = np.zeros((8, 32, 32, 32), np.float32)
    x0[3] = 0.5
    x0 = _cuda(x0)
    opts = rw.Opts(beta=130.0, tol=1e-9)
    ref, _ = rw.rw_solve(vol, code, val, opts, x0=x0)
    ref = ref.cpu().numpy()
    xo = [O.solve_volume(c["volume"], c["code"], c["value"], 130.0)[0] for c in cs]
    side = torch.cuda.Stream()
    out = torch.empty_like(vol)
    side.wait_stream(torch.cuda.current_stream())
    for call in range(2):
        with torch.cuda.stream(side):
            x, st = rw.rw_solve_noalloc(vol, code, val, opts, x0=x0, out=out, stream=side)
        assert st["status"] == 0 and st["rel_resid"] <= 1e-9, (call, st)
        xh = x.cpu().numpy()
        for b in range(8):
            assert np.max(np.abs(xh[b] - xo[b])) <= TOL, (call, b)
            assert np.max(np.abs(xh[b] - ref[b])) <= TOL, (call, b)


def test_noalloc_rejects_inputs_beyond_its_scratch(rw):
    import torch
    from paper_2103_09564_gb300 import _abi
    big = torch.zeros((65, 64, 64), dtype=torch.float32, device="cuda")
    code = torch.ones((65, 64, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(rw.RWError) as ei:
        rw.rw_solve_noalloc(big, code, None, rw.Opts())
    assert ei.value.status == _abi.RW_ERR_INVALID_ARG
    assert b"exceed" in rw.load().rw_last_error()
    # host memory is refused as well (the entry point stages nothing)
    v = _abi.rw_volume()
    h = np.zeros((4, 4, 4), np.float32)
    v.data = h.ctypes.data
    v.dims[0] = v.dims[1] = v.dims[2] = 4
    hc = np.ones((4, 4, 4), np.uint8)
    sm = _abi.rw_seed_mask(hc.ctypes.data, None)
    out = np.zeros((4, 4, 4), np.float32)
    st = _abi.rw_stats()
    rc = rw.load().rw_solve_noalloc(ctypes.byref(v), ctypes.byref(sm), None, None, out.ctypes.data,
                                    ctypes.byref(st), None)
    assert rc == _abi.RW_ERR_INVALID_ARG
