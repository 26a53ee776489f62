"""Several small cells cut together in one shared-memory tile.

A team stages consecutive cells of its ticket chunk side by side in its tile
and cuts all their sets in the same rounds (Sec. 3, Steps 2-6 per cell; the
cells stay independent).  These cases check, against the oracle, that the
batching changes nothing: membership, output order, per-cell near-tie flags
and the copy of cells with N <= N_min between batched cells.
"""
import numpy as np
import pytest

import oracle
from paper_1504_00636_gb300 import binding, synth

from parity import compare, conservation, run_gpu

pytestmark = pytest.mark.gpu


def small_cells(sizes, seed, dtype=np.float64, tol=(0.05, 0.05)):
    """Cells of the given sizes (dx = 2, dp = 3): positions uniform in the
    cell, momenta a drifting thermal spread, log-normal weights."""
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes, np.int64)
    n = int(sizes.sum())
    cell = np.repeat(np.arange(sizes.size, dtype=np.int32), sizes)
    nx = 64
    pos = rng.random((2, n))
    pos[0] += cell % nx
    pos[1] += cell // nx
    mom = rng.normal(0.0, 0.05, size=(3, n))
    mom[0] += 0.3
    w = rng.lognormal(0.0, 1.0, size=n)
    return synth.Particles("small_cells", 2, 3, int(sizes.size), (1.0, 1.0, 1.0), tol[0],
                           tol[1], 0, cell, pos.astype(dtype), mom.astype(dtype),
                           w.astype(dtype))


def _check(p, precision, n_min=0, classes=None):
    import torch
    m = binding.Merger(p.dx, p.dp, p.n_cells, max(p.n, 1), p.cell_size, n_min, precision)
    if classes is not None:
        m.set_classes(classes)
    g = run_gpu(p, precision, n_min=n_min, merger=m)
    m.close()
    torch.cuda.synchronize()
    r = oracle.merge_particles(p, threads=8, n_min=n_min)
    rep = compare(p, g, r, mixed=precision == "mixed")
    assert rep["unexplained"] == 0
    conservation(p, g)
    return g, r, rep


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("classes", [(256, 1024, 2048), (512, 1024, 2048), (64, 1024, 2048)],
                         ids=["tiny256", "tiny512", "small1024"])
def test_small_cells_share_a_tile(precision, classes):
    # sizes 0..300 with many cells of 0-3 particles (pass-through under
    # n_min = 3) between the merged ones; the tiny and small classes both
    # pack several cells per tile
    rng = np.random.default_rng(11)
    sizes = rng.integers(4, 300, size=700)
    sizes[::7] = rng.integers(0, 4, size=sizes[::7].size)
    dtype = np.float32 if precision == "mixed" else np.float64
    p = small_cells(sizes, seed=5, dtype=dtype)
    g, r, rep = _check(p, precision, n_min=3, classes=classes)
    # cells at or under n_min come out verbatim, in input order
    keep = np.flatnonzero(sizes <= 3)
    for c in keep[:20]:
        sel = g["cell"] == c
        assert sel.sum() == sizes[c]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_many_tiny_cells_take_long_chunks(precision):
    # enough one-warp cells for the longer ticket chunk (Poisson(12) cells,
    # 160,000 of them)
    rng = np.random.default_rng(12)
    sizes = rng.poisson(12, size=160_000)
    dtype = np.float32 if precision == "mixed" else np.float64
    p = small_cells(sizes, seed=6, dtype=dtype)
    g, r, rep = _check(p, precision, classes=(256, 1024, 2048))
    assert g["count"] == r.count or rep["flagged"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_near_tie_flags_stay_with_their_cell(precision):
    # forty cells of eight particles; cell 17 instead holds two particles
    # whose position spread is exactly the tolerance (Delta_x = 0.25 = T_X),
    # a stop-test tie.  Only that cell of its batch may carry the flag.
    sizes = np.full(40, 8)
    sizes[17] = 2
    dtype = np.float32 if precision == "mixed" else np.float64
    p = small_cells(sizes, seed=7, dtype=dtype, tol=(0.25, 10.0))
    b = int(np.sum(sizes[:17]))
    p.pos[0, b:b + 2] = np.array([0.25, 0.75], dtype) + (17 % 64)
    p.pos[1, b:b + 2] = 0.5
    p.mom[:, b:b + 2] = np.array([[0.3], [0.0], [0.0]], dtype)
    p.w[b:b + 2] = 1.0
    g, r, rep = _check(p, precision, classes=(256, 1024, 2048))
    assert r.flags[17] & oracle.NEAR_STOP
    assert g["flags"][17] & binding.PMA_NEAR_STOP
    others = np.delete(np.arange(40), 17)
    assert not np.any(g["flags"][others] & binding.PMA_NEAR_ANY)
    assert not np.any(r.flags[others])
    assert g["stats"]["cells_flagged"] == int(np.count_nonzero(g["flags"]))
