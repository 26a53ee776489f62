"""The autotuner on the GPU: it picks valid population classes, class base
and group widening, the result of a merge depends on none of them (every
decision is exact up to flagged near-ties, so cells give the same sets on
every path, in every size class and with any number of lanes per set), and
its choice is cached under PMA_TUNE_CACHE."""
import json

import numpy as np
import pytest

from paper_1504_00636_gb300 import binding, synth

from parity import local_index, run_gpu

pytestmark = pytest.mark.gpu


def _inputs(p, mixed):
    import torch
    dev = torch.device("cuda", 0)
    dt = torch.float32 if mixed else torch.float64
    return (torch.from_numpy(p.cell).to(dev),
            [torch.from_numpy(np.ascontiguousarray(p.pos[a])).to(dev, dt) for a in range(p.dx)],
            [torch.from_numpy(np.ascontiguousarray(p.mom[a])).to(dev, dt) for a in range(p.dp)],
            torch.from_numpy(np.ascontiguousarray(p.w)).to(dev, dt))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_classes_do_not_change_the_result(precision):
    # uneven cells (lognormal populations up to 9000) cross every path under
    # each setting of the classes
    p = synth.shower(grid=(48, 48), cap=9000)
    if precision == "mixed":
        p = p.astype(np.float32)
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, 0, precision)
    base = run_gpu(p, precision, merger=m)
    default = m.classes()
    for caps in [(128, 512, 2048, 12, 0), (512, 1024, 4096, 16, 1), (64, 256, 1024, 24, 0),
                 (256, 1024, 8191, 32, 1), (256, 1024, 8191, 12, 1)]:
        caps = (caps[0], caps[1], min(caps[2], default[2]), caps[3], caps[4])
        m.set_classes(caps)
        assert m.classes() == caps
        g = run_gpu(p, precision, merger=m)
        flagged = (base["flags"] | g["flags"]) & binding.PMA_NEAR_ANY
        if not flagged.any():
            for key in ("cell", "index", "w", "pos", "mom"):
                np.testing.assert_array_equal(g[key], base[key])
        else:
            # outside the flagged cells, the same sets in the same order
            li_b = local_index(base["index"], p.cell, base["cell"], p.n_cells)
            li_g = local_index(g["index"], p.cell, g["cell"], p.n_cells)
            keep = flagged[p.cell] == 0
            np.testing.assert_array_equal(li_g[keep], li_b[keep])
    with pytest.raises(binding.PmaError):
        m.set_classes((512, 256, 4096))  # cap_t above cap_w
    with pytest.raises(binding.PmaError):
        m.set_classes((256, 1024, 100000))
    for bad_base in (11, 33):
        with pytest.raises(binding.PmaError):
            m.set_classes((256, 1024, 2048, bad_base, 0))
    with pytest.raises(binding.PmaError):
        m.set_classes((256, 1024, 2048, 12, 2))
    m.set_classes(default)
    assert m.classes() == default
    m.close()


def test_tune_picks_valid_classes_and_caches_them(tmp_path, monkeypatch):
    import torch
    path = tmp_path / "tune.json"
    monkeypatch.setenv("PMA_TUNE_CACHE", str(path))
    p = synth.shower(grid=(64, 64), cap=9000).astype(np.float32)
    cells, pos, mom, w = _inputs(p, True)
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, 0, "mixed")
    caps = m.tune(cells, pos, mom, w, p.tol_x, p.tol_p)
    assert caps[0] <= caps[1] <= caps[2] <= 8191 and 12 <= caps[3] <= 32 and caps[4] in (0, 1)
    d = json.load(open(path))
    assert len(d) == 1
    key, val = next(iter(d.items()))
    assert key.startswith("D=5 mixed flags=0") and tuple(val[:5]) == caps
    # a second handle finds the entry and takes it
    m2 = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, 0, "mixed")
    m2.set_classes((64, 256, 1024, 20, 1))
    assert m2.tune(cells, pos, mom, w, p.tol_x, p.tol_p) == caps
    # the tuned handle gives the untuned handle's result
    g = run_gpu(p, "mixed", merger=m)
    ref = run_gpu(p, "mixed")
    if not ((g["flags"] | ref["flags"]) & binding.PMA_NEAR_ANY).any():
        for key in ("cell", "index", "w", "pos", "mom"):
            np.testing.assert_array_equal(g[key], ref[key])
    torch.cuda.synchronize()
    m.close()
    m2.close()
