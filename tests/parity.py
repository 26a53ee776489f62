"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and compare it with the CPU oracle on the same seeded inputs.

Comparison rules:
* membership: per cell, the local output index of every particle and the
  number of outputs must be identical, except in cells where the oracle or
  the CUDA path flagged a near-tie (a decision within about 1e-9 relative of
  a threshold or of the runner-up axis, or a particle within rounding of the
  cut value).  This holds for both precisions: the mixed path certifies each
  FP32 decision against its error bound and retakes the close ones in FP64;
* coordinates (FP64 path): |gpu - oracle| <= 1e-10 * scale, scale the mean
  |q| of that axis (weights: 1e-10 relative);
* coordinates (mixed path, FP32 positions out, FP64 W and P): the position
  within one float ulp of the oracle's FP64 centroid (plus 1e-12 * scale);
  W within 1e-12 relative and P within 1e-12 * scale: both are FP64 sums of
  exact products of the stored float values;
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
               flags=out.cell_flags.cpu().numpy().astype(np.uint32),
               stats=m.stats())
    if merger is None:
        m.close()
    return res


def local_index(index, cell_of_input, out_cell, n_cells):
    """Per particle: output slot relative to the first output of its cell
    (outputs are ordered by cell, so the first slot comes from a search)."""
    first = np.searchsorted(out_cell, np.arange(n_cells, dtype=out_cell.dtype), side="left")
    return index.astype(np.int64) - first[cell_of_input]


def flagged_cells(g, r, n_cells):
    """Cells with a near-tie flag from the oracle or from the CUDA path."""
    f = r.flags != 0
    if g.get("flags") is not None:
        f = f | ((g["flags"][:n_cells] & binding.PMA_NEAR_ANY) != 0)
    return f


def compare(p, g, r, coord_rtol=1e-10, check_coords=True, allow_flagged=True, mixed=False):
    """Assert GPU result g (dict) equals oracle result r; returns a report."""
    n_cells = p.n_cells
    flagged = flagged_cells(g, r, n_cells) if allow_flagged else np.zeros(n_cells, bool)
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
    if not bad_cells.any():
        assert g["count"] == r.count
        np.testing.assert_array_equal(g["index"], r.index)
        np.testing.assert_array_equal(g["cell"], r.cell)
    if check_coords:
        ok_out = ~np.isin(g["cell"], np.flatnonzero(bad_cells))
        ok_ref = ~np.isin(r.cell, np.flatnonzero(bad_cells))
        assert ok_out.sum() == ok_ref.sum()
        w_rtol = 1e-12 if mixed else coord_rtol
        np.testing.assert_allclose(g["w"][ok_out], r.w[ok_ref], rtol=w_rtol, atol=0)
        for a in range(g["pos"].shape[0]):
            scale = float(np.mean(np.abs(p.pos[a]))) if p.pos.shape[1] else 1.0
            got, ref = g["pos"][a][ok_out], r.pos[a][ok_ref]
            if mixed:
                # float output: the FP64 centroid rounded to nearest float
                tol = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) \
                    + 1e-12 * max(scale, 1e-300)
                bad = np.abs(got - ref) > tol
                assert not bad.any(), ("position axis", a, got[bad][:5], ref[bad][:5])
            else:
                np.testing.assert_allclose(got, ref, rtol=0, atol=coord_rtol * max(scale, 1e-300))
        for a in range(g["mom"].shape[0]):
            scale = float(np.mean(np.abs(p.mom[a]))) if p.mom.shape[1] else 1.0
            got, ref = g["mom"][a][ok_out], r.mom[a][ok_ref]
            if mixed:
                # an FP64 mean of exact products: 1e-12 of the larger of the
                # axis scale and the value itself
                tol = 1e-12 * np.maximum(max(scale, 1e-300), np.abs(ref))
                bad = np.abs(got - ref) > tol
                assert not bad.any(), ("momentum axis", a, got[bad][:5], ref[bad][:5])
            else:
                np.testing.assert_allclose(got, ref, rtol=0, atol=coord_rtol * max(scale, 1e-300))
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
