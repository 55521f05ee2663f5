"""The synthetic inputs are drawn from a counter-based generator: a value is a
function of (seed, stream, index) only, so it does not depend on the order or
the slab in which it is drawn, and the numpy (host) and torch (device) paths
that generate the phantoms agree."""
import numpy as np
import pytest

import phantoms as P


def test_values_do_not_depend_on_order():
    idx = np.arange(100000, dtype=np.uint64)
    perm = np.random.default_rng(0).permutation(len(idx))
    u = P.uniform(7, 3, idx)
    assert np.array_equal(P.uniform(7, 3, idx[perm]), u[perm])
    # slabs drawn separately equal one draw
    assert np.array_equal(np.concatenate([P.uniform(7, 3, idx[:40000]), P.uniform(7, 3, idx[40000:])]), u)
    # streams and seeds are independent draws
    assert not np.array_equal(P.uniform(7, 4, idx), u)
    assert not np.array_equal(P.uniform(8, 3, idx), u)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_numpy_and_torch_generators_agree():
    torch = pytest.importorskip("torch")
    idx = np.arange(0, 1 << 20, 37, dtype=np.uint64)
    t = torch.from_numpy(idx.astype(np.int64))
    assert np.array_equal(P.uniform_torch(5, 2, t).numpy(), P.uniform(5, 2, idx))
    assert np.allclose(P.normal_torch(5, 2, t).numpy(), P.normal(5, 2, idx), rtol=0, atol=1e-12)


def test_vessel_phantom_same_on_both_paths():
    torch = pytest.importorskip("torch")
    a = P.vessel_tree(n=48, seed=2, n_segments=12)
    b = P.vessel_tree(n=48, seed=2, n_segments=12, device=torch.device("cpu"))
    va = np.asarray(a["volume"]).astype(np.int64)
    vb = b["volume"].to(torch.int32).numpy().astype(np.int64)
    # values round to uint16 the same way except where the two paths' last-bit
    # differences fall on a rounding boundary
    assert np.mean(va != vb) < 1e-4 and np.max(np.abs(va - vb)) <= 1
    assert np.array_equal(a["labels_xyz"], b["labels_xyz"])
    assert np.array_equal(a["labels_value"], b["labels_value"])
