"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare it with the CPU oracle on the same seeded inputs.

Comparison rules:
* membership: per cell, the local output index of every particle and the
  number of outputs must be identical, except in cells where the oracle
  flagged a near-tie (a decision within 1e-9 relative of a threshold, of the
  runner-up axis, or a particle within rounding of the cut value);
* coordinates (FP64 path): |gpu - oracle| <= 1e-10 * scale, scale the mean
  |q| of the cell on that axis (weights: 1e-10 relative);
* conservation: per cell, |sum_out w - sum_in w| <= 1e-12 sum_in w and
  |sum_out w p - sum_in w p| <= 1e-12 sum_in w |p| on every momentum axis.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_1504_00636_gb300 import binding


def run_gpu(p, precision="fp64", tol_x=None, tol_p=None, n_min=None, capacity=None,
            shuffle_seed=None, merger=None, flags=0):
    import torch
    dev = torch.device("cuda", 0)
    dt = torch.float32 if precision == "mixed" else torch.float64
    n = p.n
    m = merger or binding.Merger(p.dx, p.dp, p.n_cells, capacity or max(n, 1), p.cell_size,
                                 p.n_min if n_min is None else n_min, precision, flags)
    cells = torch.from_numpy(p.cell).to(dev)
    pos = [torch.from_numpy(np.ascontiguousarray(p.pos[a])).to(dev, dt) for a in range(p.dx)]
    mom = [torch.from_numpy(np.ascontiguousarray(p.mom[a])).to(dev, dt) for a in range(p.dp)]
    w = torch.from_numpy(np.ascontiguousarray(p.w)).to(dev, dt)
    M, out = m.merge(cells, pos, mom, w, p.tol_x if tol_x is None else tol_x,
                     p.tol_p if tol_p is None else tol_p)
    res = dict(count=M,
               cell=out.cell[:M].cpu().numpy(),
               pos=np.stack([t[:M].cpu().double().numpy() for t in out.pos]) if M else np.zeros((p.dx, 0)),
               mom=np.stack([t[:M].cpu().numpy() for t in out.mom]) if M else np.zeros((p.dp, 0)),
               w=out.w[:M].cpu().numpy(),
               index=out.index[:n].cpu().numpy(),
               count_dev=int(out.count_dev.item()),
               stats=m.stats())
    if merger is None:
        m.close()
    return res


def local_index(index, cell_of_input, out_cell, n_cells):
    """Per particle: output slot relative to the first output of its cell
    (outputs are ordered by cell, so the first slot comes from a search)."""
    first = np.searchsorted(out_cell, np.arange(n_cells, dtype=out_cell.dtype), side="left")
    return index.astype(np.int64) - first[cell_of_input]


def compare(p, g, r, coord_rtol=1e-10, check_coords=True, allow_flagged=True):
    """Assert GPU result g (dict) equals oracle result r; returns a report."""
    n_cells = p.n_cells
    flagged = r.flags != 0 if allow_flagged else np.zeros(n_cells, bool)
    gi = local_index(g["index"], p.cell, g["cell"], n_cells)
    oi = local_index(r.index, p.cell, r.cell, n_cells)
    g_cnt = np.bincount(g["cell"], minlength=n_cells)
    o_cnt = np.bincount(r.cell, minlength=n_cells)
    bad_cells = np.zeros(n_cells, bool)
    bad_cells |= g_cnt != o_cnt
    mism = gi != oi
    if mism.any():
        bad_cells[np.unique(p.cell[mism])] = True
    unexplained = bad_cells & ~flagged
    report = dict(cells=n_cells, flagged=int(flagged.sum()), differing=int(bad_cells.sum()),
                  unexplained=int(unexplained.sum()), M_gpu=g["count"], M_oracle=r.count)
    assert not unexplained.any(), "membership differs in unflagged cells: %s" % (
        np.flatnonzero(unexplained)[:10],)
    if not flagged.any():
        assert g["count"] == r.count
        np.testing.assert_array_equal(g["index"], r.index)
        np.testing.assert_array_equal(g["cell"], r.cell)
    if check_coords:
        ok_out = ~np.isin(g["cell"], np.flatnonzero(bad_cells))
        ok_ref = ~np.isin(r.cell, np.flatnonzero(bad_cells))
        assert ok_out.sum() == ok_ref.sum()
        np.testing.assert_allclose(g["w"][ok_out], r.w[ok_ref], rtol=coord_rtol, atol=0)
        for arr, ref, q in ((g["pos"], r.pos, p.pos), (g["mom"], r.mom, p.mom)):
            for a in range(arr.shape[0]):
                scale = float(np.mean(np.abs(q[a]))) if q.shape[1] else 1.0
                np.testing.assert_allclose(arr[a][ok_out], ref[a][ok_ref], rtol=0,
                                           atol=coord_rtol * max(scale, 1e-300))
    return report


def conservation(p, g, rtol=1e-12):
    """Per-cell conservation of W and of W P on every momentum axis."""
    n_cells = p.n_cells
    w_in = p.w.astype(np.float64)
    W_in = np.bincount(p.cell, weights=w_in, minlength=n_cells)
    W_out = np.bincount(g["cell"], weights=g["w"], minlength=n_cells)
    assert np.all(np.abs(W_out - W_in) <= rtol * W_in)
    worst = 0.0
    for a in range(p.dp):
        q = p.mom[a].astype(np.float64)
        S_in = np.bincount(p.cell, weights=w_in * q, minlength=n_cells)
        A_in = np.bincount(p.cell, weights=w_in * np.abs(q), minlength=n_cells)
        S_out = np.bincount(g["cell"], weights=g["w"] * g["mom"][a], minlength=n_cells)
        err = np.abs(S_out - S_in)
        assert np.all(err <= rtol * A_in + 1e-300), "momentum axis %d not conserved" % a
        nz = A_in > 0
        if nz.any():
            worst = max(worst, float(np.max(err[nz] / A_in[nz])))
    return worst
