"""CUDA path vs the CPU oracle, element by element, through the C ABI."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1504_00636_gb300 import binding, synth

from parity import compare, conservation, run_gpu

pytestmark = pytest.mark.gpu


def _oracle(p, **kw):
    return oracle.merge_particles(p, threads=8, **kw)


# ------------------------------------------------------------ FP64 parity

@pytest.mark.parametrize("make", [
    lambda: synth.counter_beams(),
    lambda: synth.two_stream(cells=96),
    lambda: synth.shower(grid=(24, 24)),
    lambda: synth.random_cell(np.random.default_rng(1), 777, 2, 3, weights="lognormal"),
], ids=["counter_beams", "two_stream_96", "shower_24x24", "one_cell_777"])
def test_fp64_matches_oracle(make):
    p = make()
    g = run_gpu(p, "fp64")
    r = _oracle(p)
    rep = compare(p, g, r)
    assert g["count_dev"] == g["count"]
    conservation(p, g)
    st = g["stats"]
    assert st["n_out"] == g["count"]
    assert st["depth_sum"] == r.stats["depth_sum"] or rep["flagged"]


def test_fp64_two_stream_full_size():
    # the full 4096-cell two-stream workload (4.1M particles)
    p = synth.two_stream()
    g = run_gpu(p, "fp64")
    r = _oracle(p)
    rep = compare(p, g, r)
    conservation(p, g)
    assert rep["differing"] <= rep["flagged"]


@pytest.mark.parametrize("sizes", [[32], [33], [1, 2, 3], [31, 32, 33, 64, 65, 129]])
def test_fp64_subset_size_boundaries(sizes):
    # unit sizes at the warp / thread hand-over and single particles
    rng = np.random.default_rng(sum(sizes))
    parts = []
    for c, m in enumerate(sizes):
        q = synth.random_cell(rng, m, 1, 3, weights="lognormal")
        q.cell[:] = c
        q.pos[0] += c
        parts.append(q)
    p = synth.Particles("sizes", 1, 3, len(sizes), (1.0, 1.0, 1.0), 0.05, 0.05, 0,
                        np.concatenate([q.cell for q in parts]),
                        np.concatenate([q.pos for q in parts], axis=1),
                        np.concatenate([q.mom for q in parts], axis=1),
                        np.concatenate([q.w for q in parts]))
    g = run_gpu(p, "fp64")
    compare(p, g, _oracle(p))
    conservation(p, g)


def test_fp64_big_cells_take_the_global_path():
    # cells above the shared-memory capacity are cut in global memory first
    rng = np.random.default_rng(9)
    sizes = [6000, 40, 9000, 2500, 1]
    parts = []
    for c, m in enumerate(sizes):
        q = synth.random_cell(rng, m, 2, 3, weights="lognormal", drift=(0.5, 0.1, -0.2))
        q.cell[:] = c
        parts.append(q)
    p = synth.Particles("big", 2, 3, len(sizes), (1.0, 1.0, 1.0), 0.2, 0.1, 0,
                        np.concatenate([q.cell for q in parts]),
                        np.concatenate([q.pos for q in parts], axis=1),
                        np.concatenate([q.mom for q in parts], axis=1),
                        np.concatenate([q.w for q in parts]))
    g = run_gpu(p, "fp64")
    assert g["stats"]["big_cells"] >= 2
    compare(p, g, _oracle(p))
    conservation(p, g)
    # the same cells, ungrouped: sorted stably, so the result is unchanged
    x = p.shuffled(4)
    y, order = _grouped(x)
    gx, gy = run_gpu(x, "fp64"), run_gpu(y, "fp64")
    assert gx["stats"]["sorted_input"] == 0 and gx["stats"]["big_cells"] >= 2
    for key in ("cell", "pos", "mom", "w"):
        np.testing.assert_array_equal(gx[key], gy[key])
    np.testing.assert_array_equal(gx["index"][order], gy["index"])


def test_fp64_shuffled_input():
    p = synth.two_stream(cells=40).shuffled(3)
    g = run_gpu(p, "fp64")
    assert g["stats"]["sorted_input"] == 0
    compare(p, g, _oracle(p))
    conservation(p, g)


def _grouped(x):
    """The same particles grouped by cell, keeping input order inside a cell
    (Step 1's order), and the permutation used."""
    order = np.argsort(x.cell, kind="stable")
    y = dataclasses.replace(x, name=x.name + "_grouped", cell=x.cell[order],
                            pos=np.ascontiguousarray(x.pos[:, order]),
                            mom=np.ascontiguousarray(x.mom[:, order]),
                            w=np.ascontiguousarray(x.w[order]))
    return y, order


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("make", [
    lambda: synth.two_stream(cells=64).shuffled(5),
    lambda: synth.shower(grid=(40, 40), cap=3000).shuffled(6),
], ids=["two_stream_64", "shower_40x40"])
def test_ungrouped_input_sorts_stably(make, precision):
    # ungrouped input is sorted by (cell, input index): the result equals the
    # run on the grouped copy bit for bit, and repeats exactly
    x = make()
    if precision == "mixed":
        x = x.astype(np.float32)
    y, order = _grouped(x)
    gx, gx2, gy = run_gpu(x, precision), run_gpu(x, precision), run_gpu(y, precision)
    assert gx["stats"]["sorted_input"] == 0 and gy["stats"]["sorted_input"] == 1
    for key in ("cell", "pos", "mom", "w"):
        np.testing.assert_array_equal(gx[key], gy[key])
        np.testing.assert_array_equal(gx[key], gx2[key])
    np.testing.assert_array_equal(gx["index"][order], gy["index"])
    if precision == "fp64":
        compare(x, gx, _oracle(x))


def _with_big_cells():
    """A shower-shaped set in which two cells hold 9000 and 8000 particles:
    above every large tile (7551 in float32 and 4223 in FP64 for D = 5), so
    they are cut in global memory first and their pieces read the inputs
    through the permutation, while the other cells read the sorted copy."""
    p = synth.shower(grid=(24, 24), cap=3000)
    cell = p.cell.copy()
    cell[:9000] = 5
    cell[9000:17000] = 7
    return dataclasses.replace(p, name="shower_big_cells", cell=cell)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ungrouped_input_with_big_cells(precision):
    x = _with_big_cells().shuffled(8)
    if precision == "mixed":
        x = x.astype(np.float32)
    y, order = _grouped(x)
    gx, gy = run_gpu(x, precision), run_gpu(y, precision)
    assert gx["stats"]["sorted_input"] == 0 and gx["stats"]["big_cells"] == 2
    for key in ("cell", "pos", "mom", "w"):
        np.testing.assert_array_equal(gx[key], gy[key])
    np.testing.assert_array_equal(gx["index"][order], gy["index"])
    if precision == "fp64":
        compare(x, gx, _oracle(x))
        conservation(x, gx)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_work_after_an_empty_call_gets_done(precision):
    # a handle sizes the launches of work sources that were empty in its last
    # call small; when such a source has work in the next call (here: tiny
    # cells, big cells and ungrouped input after a call with none of them)
    # the result must still equal a fresh handle's
    first = synth.two_stream(cells=64)
    second = _with_big_cells().shuffled(9)
    if precision == "mixed":
        first, second = first.astype(np.float32), second.astype(np.float32)
    # one handle sized for both (same cell count and dimensions for both runs)
    n_cells = max(first.n_cells, second.n_cells)
    a = dataclasses.replace(first, n_cells=n_cells, dx=second.dx,
                            pos=np.concatenate([first.pos, first.pos[:1]])
                            if first.dx < second.dx else first.pos,
                            cell_size=second.cell_size)
    m = binding.Merger(second.dx, second.dp, n_cells, max(a.n, second.n), second.cell_size, 0,
                       precision)
    ga = run_gpu(a, precision, merger=m)
    assert ga["stats"]["cells_tiny"] == 0 and ga["stats"]["big_cells"] == 0
    assert ga["stats"]["sorted_input"] == 1
    g = run_gpu(second, precision, merger=m)
    fresh = run_gpu(second, precision)
    assert g["stats"]["big_cells"] == 2 and g["stats"]["cells_tiny"] > 0
    for key in ("cell", "pos", "mom", "w", "index"):
        np.testing.assert_array_equal(g[key], fresh[key])
    m.close()


def test_ungrouped_input_many_cells():
    # 2^18 + 3 cells need three 7-bit radix passes; most cells hold 0-3
    # particles; a few ids repeat far apart in the input
    rng = np.random.default_rng(11)
    n_cells, n = (1 << 18) + 3, 400_000
    cell = rng.integers(0, n_cells, n).astype(np.int32)
    cell[rng.integers(0, n, 2000)] = n_cells - 1
    pos = (rng.random((2, n)) + 0.0)
    mom = rng.normal(0.2, 0.05, size=(3, n))
    w = rng.lognormal(0.0, 0.5, size=n)
    x = synth.Particles("many_cells", 2, 3, n_cells, (1.0, 1.0, 1.0), 0.05, 0.05, 0,
                        cell, pos, mom, w)
    y, order = _grouped(x)
    gx, gy = run_gpu(x, "fp64"), run_gpu(y, "fp64")
    assert gx["stats"]["sorted_input"] == 0
    for key in ("cell", "pos", "mom", "w"):
        np.testing.assert_array_equal(gx[key], gy[key])
    np.testing.assert_array_equal(gx["index"][order], gy["index"])
    compare(x, gx, _oracle(x))
    conservation(x, gx)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_one_cell_holding_the_whole_box(precision):
    # Sec. 3, remark 2: the first set may hold every particle of the box; a
    # 120,000-particle set is cut in global memory over many levels first
    p = synth.two_stream(cells=120)
    p = dataclasses.replace(p, name="whole_box", cell=np.zeros(p.n, np.int32), n_cells=1,
                            cell_size=(120.0, 1.0, 1.0))
    if precision == "mixed":
        p = p.astype(np.float32)
    g = run_gpu(p, precision)
    r = _oracle(p)
    assert g["stats"]["big_cells"] == 1
    compare(p, g, r, mixed=precision == "mixed")
    conservation(p, g)


def test_fp64_n_min_passthrough():
    p = synth.counter_beams(cells=8)
    g = run_gpu(p, "fp64", n_min=200)
    assert g["count"] == p.n
    r = _oracle(p, n_min=200)
    compare(p, g, r)
    np.testing.assert_array_equal(g["w"], r.w)
    np.testing.assert_array_equal(g["mom"], r.mom)


def test_fp64_identical_particles_and_zero_tolerance():
    m = 50
    p = synth.Particles("same", 1, 3, 2, (1.0, 1.0, 1.0), 0.0, 0.0, 0,
                        np.repeat(np.arange(2, dtype=np.int32), m),
                        np.full((1, 2 * m), 0.25), np.full((3, 2 * m), 0.5),
                        np.linspace(0.5, 1.5, 2 * m))
    p.pos[0, m:] += 1.0
    g = run_gpu(p, "fp64")
    # identical values never split; rounding of the centroid may leave a
    # degenerate cut, which ends the recursion as well
    assert g["count"] == 2
    conservation(p, g)


def test_empty_input():
    p = synth.counter_beams(cells=4)
    e = synth.Particles("empty", 1, 3, 4, (1.0, 1.0, 1.0), 0.1, 0.1, 0,
                        p.cell[:0], p.pos[:, :0], p.mom[:, :0], p.w[:0])
    g = run_gpu(e, "fp64", capacity=16)
    assert g["count"] == 0 and g["count_dev"] == 0


# ----------------------------------------------------------- mixed path

@pytest.mark.parametrize("make", [
    lambda: synth.two_stream_f32(cells=128),
    lambda: synth.shower(grid=(24, 24)).astype(np.float32),
    lambda: synth.hot_6d(grid=(10, 10, 10), hot_count=3000, hot_frac=0.005),
], ids=["two_stream_f32", "shower_f32", "hot_6d_small"])
def test_mixed_against_oracle_on_rounded_inputs(make):
    # every FP32 decision is certified against its error bound (close ones are
    # retaken in FP64), so membership equals the FP64 oracle's on the same
    # float32 values except in cells flagged as near-ties by either side
    p = make()
    g = run_gpu(p, "mixed")
    r = _oracle(p)  # oracle on the float32 values, upcast exactly
    rep = compare(p, g, r, mixed=True)
    assert rep["unexplained"] == 0
    # near-ties are rare on continuous data
    assert rep["flagged"] <= max(2, np.unique(p.cell).size // 100), rep
    conservation(p, g)
    st = g["stats"]
    assert st["cells_flagged"] == int(np.count_nonzero(g["flags"]))
    assert st["near_stop"] + st["near_argmax"] + st["near_cut"] >= int(
        np.count_nonzero(g["flags"] & binding.PMA_NEAR_ANY))


def test_mixed_rechecks_close_decisions_in_fp64():
    # a cell whose particles sit exactly on a tolerance edge: two particles at
    # momenta a, b with |a - b| / |a + b| = T_P exactly in binary (a = 3, b = 5,
    # T_P = 1/4) make the FP32 stop test too close to call; the FP64 recheck
    # takes the paper's <= (a leaf), as the oracle does
    a, b = np.float32(3.0), np.float32(5.0)
    p = synth.Particles("edge", 1, 1, 1, (1.0, 1.0, 1.0), 0.5, 0.25, 0,
                        np.zeros(2, np.int32), np.array([[0.25, 0.25]], np.float32),
                        np.array([[a, b]], np.float32), np.ones(2, np.float32))
    g = run_gpu(p, "mixed")
    r = _oracle(p)
    assert g["count"] == r.count == 1
    assert g["stats"]["fp64_rechecks"] >= 1
    assert g["flags"][0] & binding.PMA_RECHECKED
    assert g["flags"][0] & binding.PMA_NEAR_STOP and r.flags[0] & oracle.NEAR_STOP


# --------------------------------------------------------- API behaviour

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_shorter_call_ignores_the_longer_calls_head_bytes(precision):
    # the same handle merges 96 two-stream cells, then the first 41 cells
    # minus 7 particles (a length that is not a multiple of 16): Step 7 must
    # count only the positions of the second call, although the workspace
    # still holds the first call's head bytes after them
    p = synth.two_stream(cells=96)
    if precision == "mixed":
        p = p.astype(np.float32)
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, 0, precision)
    run_gpu(p, precision, merger=m)
    n2 = int(np.searchsorted(p.cell, 41)) - 7
    q = dataclasses.replace(p, cell=p.cell[:n2].copy(), pos=p.pos[:, :n2].copy(),
                            mom=p.mom[:, :n2].copy(), w=p.w[:n2].copy())
    assert n2 % 16 != 0
    g = run_gpu(q, precision, merger=m)
    m.close()
    r = _oracle(q)
    rep = compare(q, g, r, mixed=precision == "mixed")
    assert rep["unexplained"] == 0
    assert g["count_dev"] == g["count"]
    conservation(q, g)


def test_async_merge_then_sync_and_host_variant():
    import torch
    p = synth.two_stream(cells=16)
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, 0, "fp64")
    dev = torch.device("cuda", 0)
    cells = torch.from_numpy(p.cell).to(dev)
    pos = [torch.from_numpy(p.pos[0].copy()).to(dev)]
    mom = [torch.from_numpy(p.mom[a].copy()).to(dev) for a in range(3)]
    w = torch.from_numpy(p.w).to(dev)
    M0, out0 = m.merge(cells, pos, mom, w, p.tol_x, p.tol_p)
    _, out1 = m.merge(cells, pos, mom, w, p.tol_x, p.tol_p, sync=False)
    m.sync()
    assert int(out1.count_dev.item()) == M0
    assert torch.equal(out0.index, out1.index)
    # host-buffer variant
    N = p.n
    hc = np.empty(N, np.int32)
    hp = [np.empty(N) for _ in range(1)]
    hm = [np.empty(N) for _ in range(3)]
    hw = np.empty(N)
    hi = np.empty(N, np.int32)
    o = binding.pma_output()
    o.cell = hc.ctypes.data
    o.pos[0] = hp[0].ctypes.data
    for a in range(3):
        o.mom[a] = hm[a].ctypes.data
    o.w = hw.ctypes.data
    o.index = hi.ctypes.data
    pc = [np.ascontiguousarray(p.pos[0])]
    mc = [np.ascontiguousarray(p.mom[a]) for a in range(3)]
    M = binding.pma_merge_host(m.handle, N, p.cell.ctypes.data, [x.ctypes.data for x in pc],
                               [x.ctypes.data for x in mc], p.w.ctypes.data, p.tol_x, p.tol_p, o)
    assert M == M0
    np.testing.assert_array_equal(hi, out0.index.cpu().numpy())
    np.testing.assert_array_equal(hw[:M], out0.w[:M].cpu().numpy())
    m.close()


def _host_call(p, precision):
    """pma_merge_host on numpy arrays: returns M, outputs, counters."""
    mixed = precision == "mixed"
    ft = np.float32 if mixed else np.float64
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, p.n_min, precision)
    N = p.n
    hc, hw, hi = np.empty(N, np.int32), np.empty(N), np.empty(N, np.int32)
    hp = [np.empty(N, ft) for _ in range(p.dx)]
    hm = [np.empty(N) for _ in range(p.dp)]
    o = binding.pma_output()
    o.cell, o.w, o.index = hc.ctypes.data, hw.ctypes.data, hi.ctypes.data
    for a in range(p.dx):
        o.pos[a] = hp[a].ctypes.data
    for a in range(p.dp):
        o.mom[a] = hm[a].ctypes.data
    pc = [np.ascontiguousarray(p.pos[a], ft) for a in range(p.dx)]
    mc = [np.ascontiguousarray(p.mom[a], ft) for a in range(p.dp)]
    wc = np.ascontiguousarray(p.w, ft)
    M = binding.pma_merge_host(m.handle, N, p.cell.ctypes.data, [x.ctypes.data for x in pc],
                               [x.ctypes.data for x in mc], wc.ctypes.data, p.tol_x, p.tol_p, o)
    st = m.stats()
    m.close()
    return M, dict(cell=hc[:M], pos=np.stack([x[:M] for x in hp]), mom=np.stack([x[:M] for x in hm]),
                   w=hw[:M], index=hi), st


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shuffle", [False, True], ids=["grouped", "shuffled"])
def test_host_call_equals_device_call(precision, shuffle):
    # the host-buffer call on 2.6M particles (grouped or not) gives the
    # device call's result bit for bit
    p = synth.two_stream(cells=2600)
    if shuffle:
        p = p.shuffled(9)
    if precision == "mixed":
        p = p.astype(np.float32)
    g = run_gpu(p, precision)
    M, h, st = _host_call(p, precision)
    assert M == g["count"]
    for key in ("cell", "w", "index"):
        np.testing.assert_array_equal(h[key], g[key])
    np.testing.assert_array_equal(h["mom"], g["mom"])
    np.testing.assert_array_equal(h["pos"].astype(np.float64), g["pos"])
    for key in ("splits", "leaves", "depth_sum", "cells_merged"):
        assert st[key] == g["stats"][key]
    assert st["n_out"] == M and st["sorted_input"] == (0 if shuffle else 1)


@pytest.mark.parametrize("bad", ["cell", "weight", "nan"])
def test_bad_particle_data_is_reported(bad):
    p = synth.counter_beams(cells=4)
    if bad == "cell":
        p.cell[5] = 99
    elif bad == "weight":
        p.w[7] = -1.0
    else:
        p.mom[1, 9] = np.nan
    with pytest.raises(binding.PmaError) as ei:
        run_gpu(p, "fp64")
    assert ei.value.code == binding.PMA_ERR_INPUT


def test_capacity_and_tolerance_checks():
    import torch
    p = synth.counter_beams(cells=2)
    m = binding.Merger(1, 3, 2, 100, precision="fp64")
    dev = torch.device("cuda", 0)
    cells = torch.from_numpy(p.cell).to(dev)
    pos = [torch.from_numpy(p.pos[0].copy()).to(dev)]
    mom = [torch.from_numpy(p.mom[a].copy()).to(dev) for a in range(3)]
    w = torch.from_numpy(p.w).to(dev)
    with pytest.raises(binding.PmaError) as ei:
        m.merge(cells, pos, mom, w, 0.1, 0.1)
    assert ei.value.code == binding.PMA_ERR_CAPACITY
    m.close()
    m = binding.Merger(1, 3, 2, p.n, precision="fp64")
    with pytest.raises(binding.PmaError) as ei:
        m.merge(cells, pos, mom, w, -0.1, 0.1)
    assert ei.value.code == binding.PMA_ERR_INVALID_ARG
    m.close()


def test_mixed_verbatim_copies_are_exact_for_special_values():
    # one-particle sets and pass-through cells are copied verbatim: the float32
    # -> float64 widening must be exact for zeros, subnormals and extremes
    vals = np.array([0.0, -0.0, 1e-40, -3e-39, 1.4e-45, 3.3e38, -2.5e-38, 1.17549435e-38],
                    dtype=np.float32)
    n = vals.size
    p = synth.Particles("special", 1, 3, n, (1.0, 1.0, 1.0), 0.1, 0.1, 0,
                        np.arange(n, dtype=np.int32), (np.arange(n) + 0.5)[None, :].astype(np.float32),
                        np.stack([vals, vals[::-1], vals]).astype(np.float32),
                        np.linspace(0.5, 2.0, n).astype(np.float32))
    g = run_gpu(p, "mixed")
    assert g["count"] == n
    np.testing.assert_array_equal(g["mom"], p.mom.astype(np.float64))
    assert np.array_equal(np.signbit(g["mom"]), np.signbit(p.mom))
    np.testing.assert_array_equal(g["w"], p.w.astype(np.float64))


def test_merge_step_replays_from_a_cuda_graph():
    # the whole call (binning, partition, emit, status copy) is stream-ordered
    # with no host synchronisation, so it can be captured once and replayed
    import torch
    p = synth.two_stream(cells=64).astype(np.float32)
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, 0, "mixed")
    dev = torch.device("cuda", 0)
    cells = torch.from_numpy(p.cell).to(dev)
    pos = [torch.from_numpy(p.pos[0].copy()).to(dev)]
    mom = [torch.from_numpy(p.mom[a].copy()).to(dev) for a in range(3)]
    w = torch.from_numpy(p.w).to(dev)
    ref_M, ref = m.merge(cells, pos, mom, w, p.tol_x, p.tol_p)
    out = m.alloc_output(dev)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        m.merge(cells, pos, mom, w, p.tol_x, p.tol_p, out=out, sync=False, stream=s)  # warm-up
    s.synchronize()
    m.sync()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        m.merge(cells, pos, mom, w, p.tol_x, p.tol_p, out=out, sync=False, stream=s)
    for _ in range(3):
        out.index.fill_(-1)
        out.count_dev.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert int(out.count_dev.item()) == ref_M
        assert torch.equal(out.index, ref.index)
        assert torch.equal(out.w[:ref_M], ref.w[:ref_M])
    m.close()


def test_host_call_reports_bad_data():
    # a bad weight near the end of a 2.6M-particle host call is reported
    p = synth.two_stream(cells=2600)
    p.w[p.n - 10] = -1.0
    with pytest.raises(binding.PmaError) as ei:
        _host_call(p, "fp64")
    assert ei.value.code == binding.PMA_ERR_INPUT
