"""Parity cases run in a child process against the bounds-checked build of
the library (PMA_LIBRARY names it): every check must pass, and the results
must still match the oracle.  Prints one line per case; exits non-zero on a
failure.  Used by test_gpu_checked.py."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1504_00636_gb300 import binding, synth  # noqa: E402
from parity import compare, conservation, run_gpu  # noqa: E402


def with_big_cells():
    p = synth.shower(grid=(24, 24), cap=3000)
    cell = p.cell.copy()
    cell[:9000] = 5
    cell[9000:17000] = 7
    import dataclasses
    return dataclasses.replace(p, name="shower_big_cells", cell=cell)


def case(name, p, precision, flags=0, variant=0, check_oracle=True):
    if precision == "mixed":
        p = p.astype(np.float32)
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, p.n_min, precision, flags)
    g = run_gpu(p, precision, merger=m, flags=flags)
    first = binding.pma_check_first(m.handle)
    m.close()
    assert first is None, "%s: bounds check failed at site %d, index %d" % (name, *first)
    if check_oracle:
        r = oracle.merge_particles(p, threads=8, variant=variant)
        compare(p, g, r, mixed=precision == "mixed")
        conservation(p, g)
    print("ok", name, precision, g["count"], g["stats"]["big_cells"], flush=True)


def main():
    assert binding.pma_checked_build(), "PMA_LIBRARY is not the checked build"
    for prec in ("fp64", "mixed"):
        case("two_stream_64", synth.two_stream(cells=64), prec)
        case("big_cells_shuffled", with_big_cells().shuffled(8), prec)
        case("shower_small_cells", synth.shower(grid=(16, 16)), prec)
    case("momentum_norm", synth.shower(grid=(16, 16)), "mixed",
         flags=binding.PMA_FLAG_MOMENTUM_NORM, variant=oracle.VAR_PNORM)
    case("conserve_energy", synth.counter_beams(), "mixed",
         flags=binding.PMA_FLAG_CONSERVE_ENERGY, check_oracle=False)


if __name__ == "__main__":
    main()
