import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture of 'case ... end' blocks."""
    path = os.path.join(ROOT, "tests", "golden", name)
    cases, cur = [], None
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "case":
                cur = {"name": vals[0]}
            elif key == "end":
                cases.append(cur)
                cur = None
            else:
                cur[key] = [float(v) for v in vals]
    return cases


def determined_mask(g, beta, w_min=1e-30, strong=1e-6, ratio=1e-12, seeds=None):
    """Voxels whose random-walker value is numerically determined.

    Excludes clusters of two or more voxels joined by strong edges
    (w > `strong`) whose total conductance to the rest of the volume is below
    `ratio` times their internal conductance — e.g. adjacent salt-noise
    voxels, linked to their surroundings only through w_min edges.  Their
    Jacobi-scaled eigenvalue is ~w_min, far below what any iterative solve
    (FP64 included) resolves, so their value depends on the solver's path.
    Computed from the intensities alone; a cluster holding a voxel of the
    optional boolean `seeds` mask is determined."""
    import numpy as np
    from scipy import sparse
    from scipy.sparse.csgraph import connected_components
    g = np.asarray(g, dtype=np.float64)
    n = g.size
    idx = np.arange(n).reshape(g.shape)
    gf = g.ravel()
    a_l, b_l, w_l = [], [], []
    for ax in range(3):
        a = np.moveaxis(idx, ax, 0)[:-1].ravel()
        b = np.moveaxis(idx, ax, 0)[1:].ravel()
        a_l.append(a)
        b_l.append(b)
        w_l.append(np.maximum(np.exp(-beta * (gf[a] - gf[b]) ** 2), w_min))
    a, b, w = np.concatenate(a_l), np.concatenate(b_l), np.concatenate(w_l)
    s = w > strong
    G = sparse.coo_matrix((np.ones(int(s.sum())), (a[s], b[s])), shape=(n, n))
    nc, lab = connected_components(G, directed=False)
    size = np.bincount(lab, minlength=nc)
    cross = lab[a] != lab[b]
    exitw = (np.bincount(lab[a[cross]], weights=w[cross], minlength=nc) +
             np.bincount(lab[b[cross]], weights=w[cross], minlength=nc))
    intw = np.bincount(lab[a[~cross]], weights=w[~cross], minlength=nc)
    trapped = (size >= 2) & (exitw < ratio * np.maximum(intw, 1e-300))
    if seeds is not None:
        trapped[np.unique(lab[np.asarray(seeds, bool).ravel()])] = False
    return ~trapped[lab].reshape(g.shape)
