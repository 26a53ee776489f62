"""The allocation-free entry point, pma_merge_noalloc, against pma_merge.

Some callers cannot allocate device memory while they merge: a PIC code whose
device memory is owned by its own pool allocator, or a time step that must not
pay the implicit device synchronisation that cudaMalloc and cudaFree can
cause.  pma_merge_noalloc serves them without a handle: its scratch is a fixed
array inside the library, and the caller passes only inputs and outputs
(allocated here by the test, before the calls).  Two calls in a row, on
different inputs, must each give the result of pma_merge on the same inputs:
the same output count and membership, the same merged particles (to the 1e-10
tolerance of the other parity tests), and the same per-cell conservation.
"""
import dataclasses

import numpy as np
import pytest

from paper_1504_00636_gb300 import binding, synth

from parity import conservation, run_gpu

pytestmark = pytest.mark.gpu


def _device_inputs(p, dt):
    import torch
    dev = torch.device("cuda", 0)
    return (torch.from_numpy(p.cell).to(dev),
            [torch.from_numpy(np.ascontiguousarray(p.pos[a])).to(dev, dt) for a in range(p.dx)],
            [torch.from_numpy(np.ascontiguousarray(p.mom[a])).to(dev, dt) for a in range(p.dp)],
            torch.from_numpy(np.ascontiguousarray(p.w)).to(dev, dt))


def _noalloc(p, precision, flags=0):
    import torch
    dt = torch.float32 if precision == "mixed" else torch.float64
    cells, pos, mom, w = _device_inputs(p, dt)
    dev = cells.device
    N = p.n
    out = binding.Output(torch.empty(N, dtype=torch.int32, device=dev),
                         [torch.empty(N, dtype=dt, device=dev) for _ in range(p.dx)],
                         [torch.empty(N, dtype=torch.float64, device=dev) for _ in range(p.dp)],
                         torch.empty(N, dtype=torch.float64, device=dev),
                         torch.empty(N, dtype=torch.int32, device=dev),
                         torch.zeros(1, dtype=torch.int64, device=dev))
    cfg = binding.pma_config()
    cfg.dx, cfg.dp = p.dx, p.dp
    for a in range(3):
        cfg.cell_size[a] = p.cell_size[a]
    cfg.n_cells = p.n_cells
    cfg.n_min = p.n_min
    cfg.precision = binding.PMA_MIXED if precision == "mixed" else binding.PMA_FP64
    cfg.flags = flags
    stream = torch.cuda.current_stream(dev).cuda_stream
    M = binding.pma_merge_noalloc(cfg, N, cells.data_ptr(), [t.data_ptr() for t in pos],
                                  [t.data_ptr() for t in mom], w.data_ptr(), p.tol_x, p.tol_p,
                                  out.struct(), stream=stream)
    return dict(count=M, cell=out.cell[:M].cpu().numpy(),
                pos=np.stack([t[:M].cpu().double().numpy() for t in out.pos]),
                mom=np.stack([t[:M].cpu().numpy() for t in out.mom]),
                w=out.w[:M].cpu().numpy(), index=out.index[:N].cpu().numpy(),
                count_dev=int(out.count_dev.item()))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_matches_pma_merge_on_two_calls(precision):
    inputs = [synth.two_stream(cells=48), synth.counter_beams()]
    if precision == "mixed":
        inputs = [q.astype(np.float32) for q in inputs]
    for p in inputs:  # two calls in a row, different inputs
        assert p.n <= binding.PMA_NOALLOC_MAX_N
        ref = run_gpu(p, precision)
        got = _noalloc(p, precision)
        assert got["count"] == ref["count"] == got["count_dev"]
        np.testing.assert_array_equal(got["index"], ref["index"])
        np.testing.assert_array_equal(got["cell"], ref["cell"])
        np.testing.assert_allclose(got["w"], ref["w"], rtol=1e-10, atol=0)
        for a in range(p.dx):
            np.testing.assert_allclose(got["pos"][a], ref["pos"][a], rtol=1e-10, atol=1e-12)
        for a in range(p.dp):
            np.testing.assert_allclose(got["mom"][a], ref["mom"][a], rtol=1e-10, atol=1e-12)
        conservation(p, got)


def test_noalloc_rejects_sizes_beyond_its_limit():
    cfg = binding.pma_config()
    cfg.dx, cfg.dp, cfg.n_cells, cfg.precision = 1, 3, 4, binding.PMA_FP64
    cfg.cell_size[0] = 1.0
    o = binding.pma_output()
    with pytest.raises(binding.PmaError) as ei:
        binding.pma_merge_noalloc(cfg, binding.PMA_NOALLOC_MAX_N + 1, 1, [1], [1, 1, 1], 1,
                                  0.1, 0.1, o)
    assert ei.value.code == binding.PMA_ERR_CAPACITY
    cfg.n_cells = binding.PMA_NOALLOC_MAX_CELLS + 1
    with pytest.raises(binding.PmaError) as ei:
        binding.pma_merge_noalloc(cfg, 10, 1, [1], [1, 1, 1], 1, 0.1, 0.1, o)
    assert ei.value.code == binding.PMA_ERR_CAPACITY


def _grouped_cells(sizes, seed, dx=1, dp=3):
    rng = np.random.default_rng(seed)
    parts = []
    for c, m in enumerate(sizes):
        q = synth.random_cell(rng, m, dx, dp, weights="lognormal")
        q.cell[:] = c
        parts.append(q)
    return synth.Particles("cells", dx, dp, len(sizes), (1.0, 1.0, 1.0), 0.05, 0.05, 0,
                           np.concatenate([q.cell for q in parts]),
                           np.concatenate([q.pos for q in parts], axis=1),
                           np.concatenate([q.mom for q in parts], axis=1),
                           np.concatenate([q.w for q in parts]))


def test_noalloc_reports_bad_input_on_the_device():
    # ids out of order, an id out of range, and a non-finite momentum in a
    # one-particle cell (copied as it is) each return PMA_ERR_INPUT
    base = _grouped_cells([30, 1, 40], 5)
    for bad in ("descending", "range", "nan_single"):
        p = dataclasses.replace(base, cell=base.cell.copy(), mom=base.mom.copy())
        if bad == "descending":
            p.cell[[0, 35]] = p.cell[[35, 0]]
        elif bad == "range":
            p.cell[-1] = 7
        else:
            p.mom[1, 30] = np.nan  # the one-particle cell
        with pytest.raises(binding.PmaError) as ei:
            _noalloc(p, "fp64")
        assert ei.value.code == binding.PMA_ERR_INPUT, bad


def test_noalloc_refuses_a_cell_above_its_tile_and_variant_flags():
    p = _grouped_cells([100, 9000, 50], 6)
    with pytest.raises(binding.PmaError) as ei:
        _noalloc(p, "fp64")
    assert ei.value.code == binding.PMA_ERR_CAPACITY
    q = _grouped_cells([100, 50], 7)
    for flags in (binding.PMA_FLAG_MOMENTUM_NORM, binding.PMA_FLAG_SPLIT_NORMALIZED,
                  binding.PMA_FLAG_CONSERVE_ENERGY):
        with pytest.raises(binding.PmaError) as ei:
            _noalloc(q, "fp64", flags=flags)
        assert ei.value.code == binding.PMA_ERR_INVALID_ARG


def test_noalloc_passes_small_cells_through_like_pma_merge():
    # n_min > 0: cells of at most n_min particles are copied as they are
    p = dataclasses.replace(_grouped_cells([12, 40, 3, 25, 1, 60], 8), n_min=25)
    ref = run_gpu(p, "fp64")
    got = _noalloc(p, "fp64")
    assert got["count"] == ref["count"]
    np.testing.assert_array_equal(got["index"], ref["index"])
    np.testing.assert_array_equal(got["w"], ref["w"])
    np.testing.assert_array_equal(got["mom"], ref["mom"])


def test_noalloc_allocates_no_device_memory():
    # after a first call (which looks up the scratch array's address), a
    # call leaves the device's free memory and torch's allocation unchanged
    import torch
    p = synth.two_stream(cells=40)
    _noalloc(p, "fp64")
    torch.cuda.synchronize()
    dt = torch.float64
    cells, pos, mom, w = _device_inputs(p, dt)
    dev = cells.device
    N = p.n
    out = binding.Output(torch.empty(N, dtype=torch.int32, device=dev),
                         [torch.empty(N, dtype=dt, device=dev)],
                         [torch.empty(N, dtype=torch.float64, device=dev) for _ in range(3)],
                         torch.empty(N, dtype=torch.float64, device=dev),
                         torch.empty(N, dtype=torch.int32, device=dev),
                         torch.zeros(1, dtype=torch.int64, device=dev))
    cfg = binding.pma_config()
    cfg.dx, cfg.dp, cfg.n_cells, cfg.precision = 1, 3, p.n_cells, binding.PMA_FP64
    cfg.cell_size[0] = 1.0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    M = binding.pma_merge_noalloc(cfg, N, cells.data_ptr(), [t.data_ptr() for t in pos],
                                  [t.data_ptr() for t in mom], w.data_ptr(), p.tol_x, p.tol_p,
                                  out.struct(), stream=torch.cuda.current_stream(dev).cuda_stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert M > 0
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
