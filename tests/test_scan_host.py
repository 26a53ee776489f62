"""Host logic of the tolerance scan: its energy definition matches the
oracle's energy bookkeeping (Sec. 3, remark on energy; E = sum w (gamma - 1))."""
import numpy as np
import pytest

import oracle
from paper_1504_00636_gb300 import scan, synth


@pytest.mark.parametrize("make", [lambda: synth.counter_beams(cells=6),
                                  lambda: synth.shower(grid=(8, 8))],
                         ids=["counter_beams", "shower_8x8"])
def test_energy_matches_oracle_bookkeeping(make):
    p = make()
    r = oracle.merge_particles(p)
    assert scan.energy(p.w, p.mom) == pytest.approx(r.stats["energy_in"], rel=1e-12)
    assert scan.energy(r.w, r.mom) == pytest.approx(r.stats["energy_out"], rel=1e-12)


def test_energy_of_a_known_particle():
    # |p| = 3/4: gamma = 5/4, kinetic energy 1/4 per unit weight
    assert scan.energy(np.array([2.0]), np.array([[0.6], [0.0], [0.45]])) == pytest.approx(0.5, rel=1e-15)
