"""Failure detection without a GPU fault.

Every wait of a CTA for another CTA's status word (the single-pass prefix
scans of Step 1 and Step 7) is bounded in time: when it runs out, the kernel
sets an error bit and returns, the kernels after it return at once, and the
call reports PMA_ERR_TIMEOUT.  The GPU test makes a wait run out on purpose
with a test hook that withholds one scan tile's status word (a flag that
nothing sets), with a short limit, and checks that the handle still works
afterwards.  The CPU test checks how device error bits map to status codes.
"""
import numpy as np
import pytest

import oracle
from paper_1504_00636_gb300 import binding, synth

from parity import compare, run_gpu


def test_device_error_bits_map_to_status_codes():
    lib = binding.load()
    assert lib.pma_test_status_of_bits(0) == binding.PMA_OK
    assert lib.pma_test_status_of_bits(1) == binding.PMA_ERR_INPUT
    assert lib.pma_test_status_of_bits(2) == binding.PMA_ERR_INTERNAL
    assert lib.pma_test_status_of_bits(4) == binding.PMA_ERR_TIMEOUT
    # precedence: bad data, then a wait that gave up, then an internal bound
    assert lib.pma_test_status_of_bits(1 | 4) == binding.PMA_ERR_INPUT
    assert lib.pma_test_status_of_bits(2 | 4) == binding.PMA_ERR_TIMEOUT
    assert lib.pma_test_status_of_bits(7) == binding.PMA_ERR_INPUT


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_withheld_status_word_times_out_and_the_handle_recovers(precision):
    import torch
    # 3000 cells: two scan tiles of 2048 cells, so tile 1 waits for tile 0
    p = synth.two_stream(cells=3000)
    if precision == "mixed":
        p = p.astype(np.float32)
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, 0, precision)
    dev = torch.device("cuda", 0)
    dt = torch.float32 if precision == "mixed" else torch.float64
    cells = torch.from_numpy(p.cell).to(dev)
    pos = [torch.from_numpy(np.ascontiguousarray(p.pos[0])).to(dev, dt)]
    mom = [torch.from_numpy(np.ascontiguousarray(p.mom[a])).to(dev, dt) for a in range(3)]
    w = torch.from_numpy(np.ascontiguousarray(p.w)).to(dev, dt)
    with pytest.raises(binding.PmaError):
        binding.pma_set_wait_limit(m.handle, 10)  # below 1 us: rejected
    binding.pma_set_wait_limit(m.handle, 200_000)  # 0.2 ms
    binding.pma_test_withhold_status(m.handle, 0)
    with pytest.raises(binding.PmaError) as ei:
        m.merge(cells, pos, mom, w, p.tol_x, p.tol_p)
    assert ei.value.code == binding.PMA_ERR_TIMEOUT
    # the context is intact and the next call starts afresh
    binding.pma_test_withhold_status(m.handle, -1)
    binding.pma_set_wait_limit(m.handle, 0)
    g = run_gpu(p, precision, merger=m)
    torch.cuda.synchronize()
    m.close()
    compare(p, g, oracle.merge_particles(p, threads=8), mixed=precision == "mixed")
