"""Failure detection without a GPU fault: a bounded wait inside a sweep
kernel that runs out is reported as RW_ERR_TIMEOUT, and the context stays
usable.  The failure is injected on the host (RW_FAULT=grid_barrier makes the
looped sweep's grid barrier expect one arrival more than the grid has, so no
CTA is the last one and every CTA's bounded spin ends); no copy is in flight
at that barrier, so every CTA returns cleanly."""
import numpy as np
import pytest

import oracle as O
import phantoms as P

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


def test_grid_barrier_wait_runs_out_and_the_context_survives(rw, monkeypatch):
    # a 40^3 system with the brick tile fits one wave: it runs looped from the
    # start (the cluster-resident mode, which would take it otherwise, is off)
    c = P.plain_ball(n=40, seed=4)
    args = (_cuda(c["volume"]), _cuda(c["code"]), _cuda(c["value"]), rw.Opts(beta=130.0, tol=1e-9, tile="s40x20"))
    monkeypatch.setenv("RW_CLUSTER", "0")
    monkeypatch.setenv("RW_FAULT", "grid_barrier")
    with pytest.raises(rw.RWError) as ei:
        rw.rw_solve(*args)
    assert ei.value.status == rw._abi.RW_ERR_TIMEOUT
    assert b"ran out" in rw.load().rw_last_error()
    monkeypatch.delenv("RW_FAULT")
    x, st = rw.rw_solve(*args)
    xo, _, _, so = O.solve_volume(c["volume"], c["code"], c["value"], 130.0)
    assert so == 0 and st["status"] == 0
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-4
