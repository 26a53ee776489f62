"""Throughput of the Voronoi merge step (Sec. 3, Steps 1-7) on one GB300.

One step = one pma_merge call over the whole workload: binning, recursive
partition of every cell, centroid emission (every row of the hot path).
Default workload: the two-stream-shaped set, 1D grid of 4096 cells x ~1000
particles (4.1M particles, 1D position + 3D momentum), tol 0.05, seed 1.
The headline `value` is the mixed-precision path (float32 storage,
compensated float32 moments, FP64-certain decisions, FP64 merged W and P);
the plain FP64 path on the same particles is reported beside it.

Timing: inputs resident on the device; W untimed warm-up steps; the step is
captured once into a CUDA graph, and K replays are timed, each bracketed by
CUDA events on the capture stream, with a 256 MB L2 flush before each step
(outside the events).  Per-kernel durations come from K eager steps timed
right after with the library's per-stage events on the same stream.  Under torchrun (N > 1) every rank runs its own
replica; the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Mparticles/s merged and % of HBM roofline, FP32-mixed vs FP64 plain at equal "
          "conservation error")
UNIT = "Mparticles/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}


def kernels_per_step(n_cells):
    """Library kernels one merge call launches: the clearing kernel, hist,
    scan, radix prep, one radix pass per 8-bit digit of the cell id and the
    sorted-order copy (these return at once on grouped input), big-cell
    cuts, four team launches (tiny, small, large cells, pieces), count,
    tiles, emit."""
    bits = max(1, int(n_cells).bit_length())
    return 1 + 2 + 1 + (bits + 7) // 8 + 1 + 1 + 4 + 3


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return PEAKS_FALLBACK, "fallback"


def workload(name):
    from paper_1504_00636_gb300 import synth
    if name == "two_stream":
        return synth.two_stream()
    if name == "two_stream_small":
        return synth.two_stream(cells=1024)
    if name == "two_stream_8k":
        # 8192 cells (8.2M particles, 196 MB in float32): inputs larger than
        # L2, for profiling captures
        return synth.two_stream(cells=8192)
    if name == "two_stream_shuffled":
        return synth.two_stream().shuffled(3)
    if name == "shower":
        return synth.shower()
    if name == "hot_6d":
        return synth.hot_6d()
    if name == "hot_6d_small":
        # 48^3 cells (about 1.3e7 particles, 350 MB in float32): the 6D
        # hot-spot shape at a size for profiling captures
        return synth.hot_6d(grid=(48, 48, 48))
    if name == "counter_beams":
        return synth.counter_beams()
    raise SystemExit("unknown workload " + name)


# --------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.lines = []
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(2)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- roofline

def bytes_per_particle(p, mixed):
    """Algorithmic bytes: read every input particle once, write every merged
    particle once (cell id, position, FP64 momentum and weight) and the
    4-byte input->output index."""
    s_in = 4 if mixed else 8
    b_in = 4 + (p.dx + p.dp + 1) * s_in
    b_out = 4 + p.dx * s_in + (p.dp + 1) * 8
    return b_in, b_out


def source_hash():
    h = hashlib.sha256()
    for f in ("team.cuh", "warp.cu", "split_common.cuh", "pma_device.cuh"):
        with open(os.path.join(ROOT, "paper_1504_00636_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload_name, precision):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel][workload_name][precision]
        if e.get("source") != source_hash():
            return None
        return e["bytes_per_launch"]
    except Exception:
        return None


# ----------------------------------------------------------- multi-rank

def max_over_ranks(t_ms, world, device=None):
    """This rank's timed milliseconds, or their maximum over the ranks of the
    job (one process per GPU, each merging its own replica)."""
    t = float(t_ms)
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    x = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def job_throughput(n_per_rank, steps, world, t_ms):
    """Whole-job Mparticles/s: every rank merges n_per_rank particles per step
    (weak scaling), and the job takes the slowest rank's time."""
    return world * n_per_rank * steps / (t_ms * 1e-3) / 1e6


# ----------------------------------------------------------------- runs

def to_device(p, mixed, dev):
    import torch
    dt = torch.float32 if mixed else torch.float64
    return (torch.from_numpy(p.cell).to(dev),
            [torch.from_numpy(np.ascontiguousarray(p.pos[a])).to(dev, dt) for a in range(p.dx)],
            [torch.from_numpy(np.ascontiguousarray(p.mom[a])).to(dev, dt) for a in range(p.dp)],
            torch.from_numpy(np.ascontiguousarray(p.w)).to(dev, dt))


def alu_peaks():
    """Measured FMA rates (independent FMAs per second, every SM) in FP32 and
    FP64, from the library's probe, and the SM count read from the device."""
    from paper_1504_00636_gb300 import binding
    f32, sms = binding.pma_probe_fma("mixed")
    f64, _ = binding.pma_probe_fma("fp64")
    return {"fp32_fma_per_s": f32, "fp64_fma_per_s": f64, "sms": sms,
            "source": "pma_probe_fma: 8 independent FMA chains per thread, 8 CTAs x 256 "
                      "threads per SM, best of 5 launches (CUDA events)"}


def time_device(p, mixed, steps, warmup, dev, flush, flags=0, tune=True):
    """K steps of one pma_merge each, inputs resident.  With `tune`, the
    library's autotuner (pma_tune) first picks the population classes and the
    class base on these particles, untimed, as a user would once per
    workload shape.  The step is captured once into a CUDA graph and
    replayed; each replay is bracketed by CUDA events on the capture stream
    (if capture fails, the same loop runs eagerly).  Then K eager steps on
    the same stream are timed with the library's per-stage events, which
    give the kernel durations."""
    import torch
    from paper_1504_00636_gb300 import binding
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, p.n_min,
                       "mixed" if mixed else "fp64", flags)
    cells, pos, mom, w = to_device(p, mixed, dev)
    out = m.alloc_output(dev)
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    default_classes = m.classes()
    tune_s = None
    if tune:
        t0 = time.perf_counter()
        m.tune(cells, pos, mom, w, p.tol_x, p.tol_p, out=out, stream=stream)
        tune_s = round(time.perf_counter() - t0, 3)
    classes = m.classes()
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.fill_(1.0)
            m.merge(cells, pos, mom, w, p.tol_x, p.tol_p, out=out, sync=False, stream=stream)
    stream.synchronize()
    m.sync()
    M = int(out.count_dev.item())

    def run(step, stages=False):
        ms = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        stream.synchronize()
        with torch.cuda.stream(stream):
            for k in range(steps):
                flush.fill_(1.0)
                ev[k][0].record(stream)
                step()
                ev[k][1].record(stream)
        stream.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms, (m.timing() if stages else None)

    def eager():
        m.merge(cells, pos, mom, w, p.tol_x, p.tol_p, out=out, sync=False, stream=stream)

    graph_ok = False
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            eager()
        g.replay()
        stream.synchronize()
        graph_ok = int(out.count_dev.item()) == M
    except Exception as exc:  # fall back to eager launches
        print("graph capture failed: %r" % (exc,), file=sys.stderr)
    ms, _ = run(g.replay if graph_ok else eager)
    # per-kernel durations: the library's stage events around the same
    # kernels, launched eagerly on the same stream right after
    m.set_timing(True)
    eager_ms, stage = run(eager, stages=True)
    m.set_timing(False)
    m.sync()
    st = m.stats()
    m.close()
    del cells, pos, mom, w, out
    torch.cuda.empty_cache()
    return dict(ms=ms, stage=stage, stats=st, M=M, graph=graph_ok, eager_ms=eager_ms,
                classes=classes, default_classes=default_classes, tune_s=tune_s)


def classes_report(res):
    """The team classes a run used: (cap_t, cap_w, cap, class base), whether
    the tuner chose them, and how long tuning took."""
    return {"used": list(res["classes"]), "default": list(res["default_classes"]),
            "tuned": res["tune_s"] is not None, "tune_s": res["tune_s"]}


def time_e2e(p, mixed, steps, warmup, classes=None):
    """Same metric through pma_merge_host: host->device copies of the inputs,
    the merge, and device->host copies of the result inside the timed step
    (with the classes the device run used)."""
    import torch
    from paper_1504_00636_gb300 import binding
    dt = np.float32 if mixed else np.float64
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, p.n_min,
                       "mixed" if mixed else "fp64")
    if classes is not None:
        m.set_classes(classes)

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        return t

    cells = pinned(p.cell)
    pos = [pinned(p.pos[a].astype(dt)) for a in range(p.dx)]
    mom = [pinned(p.mom[a].astype(dt)) for a in range(p.dp)]
    w = pinned(p.w.astype(dt))
    N = p.n
    oc = torch.empty(N, dtype=torch.int32).pin_memory()
    op = [torch.empty(N, dtype=torch.float32 if mixed else torch.float64).pin_memory()
          for _ in range(p.dx)]
    om = [torch.empty(N, dtype=torch.float64).pin_memory() for _ in range(p.dp)]
    ow = torch.empty(N, dtype=torch.float64).pin_memory()
    oi = torch.empty(N, dtype=torch.int32).pin_memory()
    o = binding.pma_output()
    o.cell = oc.data_ptr()
    for a in range(p.dx):
        o.pos[a] = op[a].data_ptr()
    for a in range(p.dp):
        o.mom[a] = om[a].data_ptr()
    o.w = ow.data_ptr()
    o.index = oi.data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    args = (m.handle, N, cells.data_ptr(), [t.data_ptr() for t in pos],
            [t.data_ptr() for t in mom], w.data_ptr(), p.tol_x, p.tol_p, o)
    for _ in range(warmup):
        M = binding.pma_merge_host(*args, stream=stream)
    ts = []
    for _ in range(steps):
        t0 = time.perf_counter()
        M = binding.pma_merge_host(*args, stream=stream)
        ts.append(time.perf_counter() - t0)
    m.close()
    s_in = 4 if mixed else 8
    h2d = N * (4 + (p.dx + p.dp + 1) * s_in)
    d2h = M * (4 + p.dx * s_in + (p.dp + 1) * 8) + 4 * N
    return dict(s=ts, h2d=h2d, d2h=d2h, M=M)


def decisions_differing(tr, labels):
    """Split decisions of one cell at which a result departs from the oracle's
    recursion tree: walk the tree (V1-first preorder) and count the nodes
    whose set the result does not treat alike (a leaf that is not one final
    set of the result; a split with a final set of the result across it, or
    whose halves come out in the other order, i.e. another axis or side);
    nodes below a departure are not counted again.  labels[i] is the
    result's output slot of the cell's i-th particle."""
    import numpy as np
    nodes = list(zip(tr.begin.tolist(), tr.end.tolist(), tr.depth.tolist(), tr.axis.tolist()))
    by_begin = {}
    for k, (b, e, d, ax) in enumerate(nodes):
        by_begin.setdefault((b, d), k)
    lab = labels[tr.perm]

    def walk(k):
        b, e, d, ax = nodes[k]
        seg = lab[b:e]
        if ax < 0:
            whole = np.count_nonzero(labels == seg[0])
            return 0 if (np.all(seg == seg[0]) and whole == e - b) else 1
        c1 = by_begin.get((b, d + 1))
        if c1 is None:
            return 1
        b1, e1 = nodes[c1][0], nodes[c1][1]
        if np.intersect1d(lab[b1:e1], lab[e1:e]).size or (np.all(seg == seg[0])):
            return 1
        if e1 < e and lab[b1:e1].max() > lab[e1:e].min():
            return 1  # the same halves, in the other order
        c2 = by_begin.get((e1, d + 1))
        return walk(c1) + (walk(c2) if c2 is not None else 1)

    return walk(0) if nodes else 0


def accuracy_report(p, dev, sample_cells=256, seed=0, flags=0, variant=0):
    """Mixed path vs the FP64 oracle on sampled cells (outside any timed
    region).  Membership: cells differing, of which explained by a near-tie
    flag of either side (unexplained must be 0), and the split decisions that
    differ (walk of the oracle's recursion tree).  Coordinates: worst error
    of the merged particles relative to each axis' mean |q|.  Per-cell
    conservation of W and W P relative to sum w and sum w |p|, and the
    relative kinetic-energy loss of both sides.  The oracle runs on (a) the
    float32-rounded inputs the mixed path stores and (b) the original FP64
    inputs, separating input rounding from the path's own arithmetic."""
    import torch
    import oracle
    from paper_1504_00636_gb300 import binding
    q = p.astype(np.float32)
    m = binding.Merger(q.dx, q.dp, q.n_cells, q.n, q.cell_size, q.n_min, "mixed",
                       flags | binding.PMA_FLAG_ENERGY_STATS)
    cells, pos, mom, w = to_device(q, True, dev)
    M, out = m.merge(cells, pos, mom, w, q.tol_x, q.tol_p)
    st = m.stats()
    g_cell = out.cell[:M].cpu().numpy()
    g_index = out.index[:q.n].cpu().numpy().astype(np.int64)
    g_flags = out.cell_flags.cpu().numpy().astype(np.uint32)
    g_w = out.w[:M].cpu().numpy()
    g_c = np.concatenate([np.stack([t[:M].cpu().double().numpy() for t in out.pos]),
                          np.stack([t[:M].cpu().numpy() for t in out.mom])])
    m.close()
    del cells, pos, mom, w, out
    rng = np.random.default_rng(seed)
    present = np.unique(q.cell)
    sample = np.sort(rng.choice(present, min(sample_cells, present.size), replace=False))
    first_g = np.searchsorted(g_cell, np.arange(q.n_cells))
    rep = {"sample_cells": int(sample.size),
           "gpu": {"fp64_rechecks": st["fp64_rechecks"], "cells_flagged": st["cells_flagged"],
                   "near_stop": st["near_stop"], "near_argmax": st["near_argmax"],
                   "near_cut": st["near_cut"],
                   "energy_loss_rel": (st["energy_in"] - st["energy_out"]) / st["energy_in"]}}
    g_near = (g_flags & binding.PMA_NEAR_ANY) != 0
    for tag, src in (("vs_oracle_on_f32_inputs", q), ("vs_oracle_on_f64_inputs", p)):
        sub = src.select_cells(sample)
        r = oracle.merge_particles(sub, threads=os.cpu_count() or 1, variant=variant)
        mask = np.isin(q.cell, sample)
        gi = g_index[mask] - first_g[q.cell[mask]]
        first_o = np.searchsorted(r.cell, np.arange(q.n_cells))
        oi = r.index.astype(np.int64) - first_o[sub.cell]
        cnt_g = np.bincount(g_cell, minlength=q.n_cells)[sample]
        cnt_o = np.bincount(r.cell, minlength=q.n_cells)[sample]
        diff = np.union1d(np.unique(sub.cell[gi != oi]), sample[cnt_g != cnt_o])
        explained = (r.flags[diff] != 0) | g_near[diff]
        # split decisions that differ, from the oracle's recursion tree
        ndec = 0
        for c in diff:
            sel = sub.cell == c
            tr = oracle.trace(sub.pos[:, sel], sub.mom[:, sel], sub.w[sel], sub.cell_size,
                              sub.tol_x, sub.tol_p, variant=variant)
            ndec += decisions_differing(tr, gi[sel])
        same = np.setdiff1d(sample, diff)
        go = np.isin(g_cell, same)
        oo = np.isin(r.cell, same)
        worst = 0.0
        if go.sum() == oo.sum() and go.any():
            ref = np.concatenate([r.pos, r.mom])[:, oo]
            got = g_c[:, go]
            scale = np.mean(np.abs(np.concatenate([sub.pos, sub.mom]).astype(np.float64)), axis=1)
            worst = float(np.max(np.abs(got - ref) / scale[:, None]))
        e_in, e_out = r.stats["energy_in"], r.stats["energy_out"]
        rep[tag] = {"cells_differing": int(diff.size),
                    "cells_differing_unexplained": int(np.count_nonzero(~explained)),
                    "decisions_differing": int(ndec),
                    "oracle_flagged_cells": int((r.flags[sample] != 0).sum()),
                    "gpu_flagged_cells": int(g_near[sample].sum()),
                    "max_coord_err_rel": worst,
                    "oracle_energy_loss_rel": (e_in - e_out) / e_in if e_in else 0.0}
    # conservation against the stored (float32) inputs, every sampled cell
    mask_o = np.isin(g_cell, sample)
    wq = q.w.astype(np.float64)
    Win = np.bincount(q.cell, weights=wq, minlength=q.n_cells)[sample]
    Wout = np.bincount(g_cell[mask_o], weights=g_w[mask_o], minlength=q.n_cells)[sample]
    worst = float(np.max(np.abs(Wout - Win) / Win))
    for a in range(q.dp):
        qa = q.mom[a].astype(np.float64)
        Sin = np.bincount(q.cell, weights=wq * qa, minlength=q.n_cells)[sample]
        Ain = np.bincount(q.cell, weights=wq * np.abs(qa), minlength=q.n_cells)[sample]
        Sout = np.bincount(g_cell[mask_o], weights=g_w[mask_o] * g_c[q.dx + a][mask_o],
                           minlength=q.n_cells)[sample]
        worst = max(worst, float(np.max(np.abs(Sout - Sin) / np.maximum(Ain, 1e-300))))
    rep["conservation_err_rel"] = worst
    return rep


def time_oracle(p, threads, reps):
    import oracle
    oracle.build()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        r = oracle.merge_particles(p, threads=threads)
        ts.append(time.perf_counter() - t0)
    return ts, r


def roofline(p, mixed, stats, stage_ms, peaks, peak_kind, M, workload_name, alu):
    """Roofline of the dominant kernel: the per-cell partition of the small-cell
    class (team_kernel, 4 warps per cell), from its live event timing.
    Bytes: it reads every particle of the cells it owns once and writes the
    4-byte final permutation and the head byte of every particle.  Ops: one
    multiply-add per moment accumulator (1 + 2D) and one compare per particle
    and tree level, F = depth_sum (2D + 2), against the measured FMA rate of
    the path's arithmetic (FP32 for mixed, FP64 for plain).  The larger of
    the two times is the bound that is reported."""
    b_in, _ = bytes_per_particle(p, mixed)
    t = stage_ms["warp_cells"] * 1e-3
    n = p.n
    bytes_alg = n * (b_in - 4 + 4 + 1)
    D = p.dx + p.dp
    ops_alg = stats["depth_sum"] * (2 * D + 2)
    hbm = peaks["hbm_gbs"] * 1e9
    alu_peak = alu["fp32_fma_per_s"] if mixed else alu["fp64_fma_per_s"]
    t_hbm, t_alu = bytes_alg / hbm, ops_alg / alu_peak
    traffic = ncu_traffic("team_kernel", workload_name, "mixed" if mixed else "fp64")
    other = {"t_hbm_us": round(t_hbm * 1e6, 2), "t_alu_us": round(t_alu * 1e6, 2),
             "bytes_alg": int(bytes_alg), "ops_alg": int(ops_alg)}
    if t_hbm >= t_alu:
        ach = bytes_alg / t / 1e9
        return {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                "traffic": traffic, "kernel": "team_kernel",
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind, **other}
    ach = ops_alg / t / 1e12
    return {"bound": "alu", "achieved": round(ach, 4), "peak": round(alu_peak / 1e12, 3),
            "unit": "Tops/s", "frac": round(ach / (alu_peak / 1e12), 4), "traffic": traffic,
            "kernel": "team_kernel",
            "peak_source": "measured %s FMA rate (%s)" % ("FP32" if mixed else "FP64",
                                                          alu["source"]), **other}


def extra_line(name, p, mixed, steps, warmup, dev, flush, peaks, flags=0, tune=True):
    """One more configuration, timed like the headline (tuned classes, graph
    replays, L2 flushed between steps): Mparticles/s, ms per call, step HBM
    fraction of the algorithmic bytes, M and the per-stage times."""
    res = time_device(p, mixed, steps, warmup, dev, flush, flags, tune)
    t_ms = float(np.mean(res["ms"]))
    b_in, b_out = bytes_per_particle(p, mixed)
    step_bytes = p.n * (b_in + 4) + res["M"] * b_out
    return {"workload": name, "precision": "mixed" if mixed else "fp64", "flags": flags,
            "n": p.n, "cells": p.n_cells, "value": round(p.n / (t_ms * 1e-3) / 1e6, 2),
            "unit": UNIT, "ms_per_step": round(t_ms, 4), "steps": steps,
            "hbm_frac_step": round(step_bytes / (t_ms * 1e-3) / (peaks["hbm_gbs"] * 1e9), 4),
            "M": res["M"], "stage_ms": {k: round(x, 4) for k, x in res["stage"].items()},
            "fp64_rechecks": res["stats"]["fp64_rechecks"],
            "cells_flagged": res["stats"]["cells_flagged"],
            "cells_per_path": {k: res["stats"][k] for k in
                               ("cells_tiny", "cells_small", "cells_large", "big_cells")},
            "classes": classes_report(res)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="two_stream")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--precision", default="both", choices=["both", "mixed", "fp64"])
    ap.add_argument("--classes", default="tuned", choices=["tuned", "default"],
                    help="team classes: chosen by pma_tune on the workload (untimed), "
                         "or the library's defaults")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations (counter beams, shuffled and "
                         "momentum-norm two-stream, shower, 6D hot spots)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    p = workload(args.workload)
    cfg = {"workload": "%s: %d cells, %d particles, dx=%d dp=%d, tol_x=%g tol_p=%g"
                       % (args.workload, p.n_cells, p.n, p.dx, p.dp, p.tol_x, p.tol_p),
           "l2": "256 MB buffer written between timed steps", "n_min": p.n_min}

    if args.impl == "reference":
        if rank != 0:
            return
        threads = os.cpu_count() or 1
        for _ in range(args.warmup):
            time_oracle(p, threads, 1)
        ts, r = time_oracle(p, threads, args.steps)
        v = p.n / float(np.mean(ts)) / 1e6
        line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": round(1e3 * float(np.mean(ts)), 3), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": cfg,
                "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": threads,
                                 "kind": "oracle",
                                 "sample": "whole workload per step (%d particles)" % p.n},
                "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    peaks, peak_kind = load_peaks()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    alu = alu_peaks()
    results = {}
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    precs = {"both": [True, False], "mixed": [True], "fp64": [False]}[args.precision]
    for mixed in precs:
        q = p.astype(np.float32) if mixed else p
        results[mixed] = time_device(q, mixed, args.steps, args.warmup, dev, flush,
                                     tune=args.classes == "tuned")
    barrier()
    clk = clocks.stop()

    def agg(ms_list):
        return max_over_ranks(np.sum(ms_list), world, dev)

    lines = {}
    for mixed, res in results.items():
        q = p.astype(np.float32) if mixed else p
        t_ms = agg(res["ms"])
        v = job_throughput(p.n, args.steps, world, t_ms)
        b_in, b_out = bytes_per_particle(q, mixed)
        step_bytes = p.n * (b_in + 4) + res["M"] * b_out
        lines[mixed] = dict(
            value=round(v, 2), ms_per_step=round(t_ms / args.steps, 4),
            hbm_frac_step=round(step_bytes / (t_ms / args.steps * 1e-3) / (peaks["hbm_gbs"] * 1e9), 4),
            M=res["M"], stage_ms={k: round(x, 4) for k, x in res["stage"].items()},
            roofline=roofline(q, mixed, res["stats"], res["stage"], peaks, peak_kind,
                              res["M"], args.workload, alu),
            depth_sum=res["stats"]["depth_sum"], splits=res["stats"]["splits"],
            fp64_rechecks=res["stats"]["fp64_rechecks"],
            cells_flagged=res["stats"]["cells_flagged"],
            graph=res["graph"], classes=classes_report(res),
            eager_ms_per_step=round(float(np.mean(res["eager_ms"])), 4))
    head = lines[True] if True in lines else lines[False]
    mixed_head = True in lines
    e2e = None
    if not args.no_e2e:
        # every rank copies its own replica in and out; the job takes the
        # slowest rank's time
        q = p.astype(np.float32) if mixed_head else p
        e = time_e2e(q, mixed_head, max(3, args.steps // 4), 2,
                     classes=results[mixed_head]["classes"])
        t_e2e = max_over_ranks(1e3 * float(np.mean(e["s"])), world, dev)
        e2e = {"value": round(job_throughput(p.n, 1, world, t_e2e), 2), "unit": UNIT,
               "h2d_bytes_per_step": e["h2d"] * world, "d2h_bytes_per_step": e["d2h"] * world}
    if rank != 0:
        return
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64" if mixed_head else "f64", "data": "synthetic", "config": cfg,
            "roofline": head["roofline"], "hbm_frac_step": head["hbm_frac_step"],
            "stage_ms": head["stage_ms"], "M": head["M"],
            "cuda_graph": head["graph"], "eager_ms_per_step": head["eager_ms_per_step"],
            "gpu_launches": kernels_per_step(p.n_cells) * args.steps * len(lines),
            "clocks": clk, "alu_peaks": alu,
            "fp64_rechecks": head["fp64_rechecks"], "cells_flagged": head["cells_flagged"],
            "classes": head["classes"]}
    if mixed_head and False in lines:
        f = lines[False]
        line["fp64_plain"] = {"value": f["value"], "ms_per_step": f["ms_per_step"],
                              "cuda_graph": f["graph"], "eager_ms_per_step": f["eager_ms_per_step"],
                              "roofline": f["roofline"], "stage_ms": f["stage_ms"], "M": f["M"],
                              "classes": f["classes"],
                              "speedup_mixed_over_fp64": round(head["value"] / f["value"], 3)}
    if e2e is not None:
        line["e2e"] = e2e
    if not args.no_extras and world == 1:
        # the other configurations of the benchmark, each timed like the
        # headline on its own inputs (fewer steps); not part of `value`
        from paper_1504_00636_gb300 import binding, synth
        ex = []
        K = max(3, min(args.steps, 10))
        tune = args.classes == "tuned"
        cb = synth.counter_beams()
        for mx in (True, False):
            q = cb.astype(np.float32) if mx else cb
            ex.append(extra_line("counter_beams (latency)", q, mx, K, 3, dev, flush, peaks,
                                 tune=tune))
        ts = synth.two_stream()
        sh = ts.shuffled(3).astype(np.float32)
        ex.append(extra_line("two_stream shuffled", sh, True, K, 3, dev, flush, peaks,
                             tune=tune))
        ex.append(extra_line("two_stream momentum-norm CV", ts.astype(np.float32), True, K, 3,
                             dev, flush, peaks, binding.PMA_FLAG_MOMENTUM_NORM, tune=tune))
        del sh, ts
        shw = synth.shower()
        for mx in (True, False):
            q = shw.astype(np.float32) if mx else shw
            ex.append(extra_line("shower", q, mx, K, 3, dev, flush, peaks, tune=tune))
        del shw, q
        h6 = synth.hot_6d()
        ex.append(extra_line("hot_6d", h6, True, K, 3, dev, flush, peaks, tune=tune))
        del h6
        line["other_configs"] = ex
    if mixed_head and not args.no_accuracy:
        line["accuracy_mixed"] = accuracy_report(p, dev)
    if not args.no_cpu:
        threads = os.cpu_count() or 1
        ts, _ = time_oracle(p, threads, 3)
        line["cpu_baseline"] = {"value": round(p.n / float(np.mean(ts)) / 1e6, 3), "unit": UNIT,
                                "cores": threads, "kind": "oracle",
                                "sample": "whole workload, FP64 oracle, 3 runs with %d threads"
                                          % threads}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
