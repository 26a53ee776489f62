"""The tolerance scan on the CUDA path (a synthetic counterpart of the
paper's Sec. 4.3 study): identities and monotonicity that the method fixes."""
import numpy as np
import pytest

import oracle
from paper_1504_00636_gb300 import scan, synth

pytestmark = pytest.mark.gpu


def test_scan_identities_and_monotonicity():
    p = synth.shower(grid=(32, 32), cap=6000)
    tps = [0.01, 0.02, 0.05, 0.2]
    rows = scan.tolerance_scan(p, [0.25, 0.5, 1.0], tps, precision="fp64")
    by = {(r["tol_x"], r["tol_p"]): r for r in rows}
    for tp in tps:
        # in-cell positions have Delta_x <= 1/2: T_X = 0.5 and 1.0 coincide
        assert by[(0.5, tp)]["M"] == by[(1.0, tp)]["M"]
        assert by[(0.5, tp)]["dE"] == by[(1.0, tp)]["dE"]  # same partition, same sums
    for tx in (0.25, 0.5, 1.0):
        Ms = [by[(tx, tp)]["M"] for tp in tps]
        dEs = [by[(tx, tp)]["dE"] for tp in tps]
        assert all(a >= b for a, b in zip(Ms, Ms[1:])), Ms
        assert all(b >= a - 1e-12 for a, b in zip(dEs, dEs[1:])), dEs
        assert min(dEs) >= -1e-12  # a centroid never gains energy
    for tp in tps:
        assert by[(0.25, tp)]["M"] >= by[(0.5, tp)]["M"]


def test_scan_point_matches_oracle():
    p = synth.shower(grid=(24, 24))
    rows = scan.tolerance_scan(p, [0.1], [0.05], precision="fp64")
    r = oracle.merge_particles(p, threads=8, tol_x=0.1, tol_p=0.05)
    assert rows[0]["M"] == r.count or r.flags.any()
    dE = (r.stats["energy_in"] - r.stats["energy_out"]) / r.stats["energy_in"]
    assert rows[0]["dE"] == pytest.approx(dE, rel=1e-6, abs=1e-12)
