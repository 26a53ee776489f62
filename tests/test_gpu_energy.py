"""The energy-conserving replacement (PMA_FLAG_CONSERVE_ENERGY) on the CUDA
path against the oracle's VAR_CONSERVE_ENERGY, and the conservation of W,
W P and the total energy per cell."""
import numpy as np
import pytest

import oracle
from paper_1504_00636_gb300 import binding, scan, synth

from parity import compare, conservation, run_gpu

pytestmark = pytest.mark.gpu

EC = binding.PMA_FLAG_CONSERVE_ENERGY
WORKLOADS = [lambda: synth.counter_beams(),
             lambda: synth.two_stream(cells=64),
             lambda: synth.shower(grid=(20, 20), cap=9000),
             lambda: synth.random_cell(np.random.default_rng(3), 3000, 2, 1, drift=(0.4,),
                                       spread=0.2, weights="lognormal")]
WIDS = ["counter_beams", "two_stream_64", "shower_20x20", "one_axis_cell"]


def total_energy_per_cell(cell, w, mom, n_cells):
    g = np.sqrt(1.0 + np.sum(np.asarray(mom, np.float64) ** 2, axis=0))
    return np.bincount(cell, weights=np.asarray(w, np.float64) * g, minlength=n_cells)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("make", WORKLOADS, ids=WIDS)
def test_energy_mode_matches_oracle_and_conserves(make, precision):
    p = make()
    if precision == "mixed":
        p = p.astype(np.float32)
    g = run_gpu(p, precision, flags=EC)
    r = oracle.merge_particles(p, threads=8, variant=oracle.VAR_CONSERVE_ENERGY)
    compare(p, g, r, check_coords=False)
    ok = ~np.isin(g["cell"], np.flatnonzero(r.flags))
    okr = ~np.isin(r.cell, np.flatnonzero(r.flags))
    np.testing.assert_allclose(g["w"][ok], r.w[okr], rtol=1e-12)
    # d comes from g^2 - 1 - |P|^2, which cancels when a set's momenta are
    # close: compare momenta against the set's momentum scale
    scale = np.maximum(np.sqrt(np.sum(r.mom[:, okr] ** 2, axis=0)), 1.0)
    assert np.all(np.abs(g["mom"][:, ok] - r.mom[:, okr]) <= 1e-8 * scale)
    np.testing.assert_allclose(g["pos"][:, ok], r.pos[:, okr],
                               rtol=1e-6 if precision == "mixed" else 1e-12, atol=1e-12)
    conservation(p, g)
    e_in = total_energy_per_cell(p.cell, p.w, p.mom, p.n_cells)
    e_out = total_energy_per_cell(g["cell"], g["w"], g["mom"], p.n_cells)
    assert np.all(np.abs(e_out - e_in) <= 1e-12 * e_in + 1e-300)


def test_energy_mode_keeps_the_partition():
    # Step 7 is the only change: the same sets, two outputs per merged set
    p = synth.two_stream(cells=32)
    lit = run_gpu(p, "fp64")
    ec = run_gpu(p, "fp64", flags=EC)
    assert ec["stats"]["splits"] == lit["stats"]["splits"]
    assert ec["stats"]["leaves"] == lit["stats"]["leaves"]
    sizes = np.bincount(lit["index"], minlength=lit["count"])
    assert ec["count"] == int(np.sum(np.where(sizes >= 2, 2, 1)))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_energy_stats_match_the_oracle_and_the_outputs(precision):
    # PMA_FLAG_ENERGY_STATS: FP64 kinetic energy of the input and of the
    # output (the paper's delta E, Sec. 3 remark on energy), summed in a
    # fixed order (identical on every call)
    p = synth.shower(grid=(24, 24))
    if precision == "mixed":
        p = p.astype(np.float32)
    flags = binding.PMA_FLAG_ENERGY_STATS
    g = run_gpu(p, precision, flags=flags)
    st = g["stats"]
    r = oracle.merge_particles(p, threads=8)
    assert st["energy_in"] == pytest.approx(r.stats["energy_in"], rel=1e-12)
    assert st["energy_in"] == pytest.approx(scan.energy(p.w, p.mom), rel=1e-12)
    assert st["energy_out"] == pytest.approx(scan.energy(g["w"], g["mom"]), rel=1e-12)
    if not (r.flags.any() or (g["flags"] & binding.PMA_NEAR_ANY).any()):
        assert st["energy_out"] == pytest.approx(r.stats["energy_out"], rel=1e-12)
    assert st["energy_out"] <= st["energy_in"] * (1 + 1e-12)  # centroids lose energy
    g2 = run_gpu(p, precision, flags=flags)
    assert g2["stats"]["energy_in"] == st["energy_in"]
    assert g2["stats"]["energy_out"] == st["energy_out"]
    # with the energy-conserving replacement, out equals in
    ge = run_gpu(p, precision, flags=flags | EC)
    assert ge["stats"]["energy_out"] == pytest.approx(ge["stats"]["energy_in"], rel=1e-12)
