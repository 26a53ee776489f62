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
FP32_OPS_PEAK = 152 * 128 * 2.07e9  # FP32 lanes x SMs x max clock (instr/s)
FP64_OPS_PEAK = 1.25e12 / 2.0       # nominal GB300 FP64 FMA rate (ops/s)


def kernels_per_step(n_cells):
    """Library kernels one merge call launches: the clearing kernel, hist,
    scan, radix prep, one radix pass per 8-bit digit of the cell id (these
    return at once on grouped input), big-cell cuts, four team launches
    (tiny, small, large cells, pieces), count, tiles, emit."""
    bits = max(1, int(n_cells).bit_length())
    return 1 + 2 + 1 + (bits + 7) // 8 + 1 + 4 + 3


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
    if name == "two_stream_shuffled":
        return synth.two_stream().shuffled(3)
    if name == "shower":
        return synth.shower()
    if name == "hot_6d":
        return synth.hot_6d()
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


def time_device(p, mixed, steps, warmup, dev, flush):
    """K steps of one pma_merge each, inputs resident.  The step is captured
    once into a CUDA graph and replayed; each replay is bracketed by CUDA
    events on the capture stream (if capture fails, the same loop runs
    eagerly).  Then K eager steps on the same stream are timed with the
    library's per-stage events, which give the kernel durations."""
    import torch
    from paper_1504_00636_gb300 import binding
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, p.n_min,
                       "mixed" if mixed else "fp64")
    cells, pos, mom, w = to_device(p, mixed, dev)
    out = m.alloc_output(dev)
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
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
    return dict(ms=ms, stage=stage, stats=st, M=M, graph=graph_ok, eager_ms=eager_ms)


def time_e2e(p, mixed, steps, warmup):
    """Same metric through pma_merge_host: host->device copies of the inputs,
    the merge, and device->host copies of the result inside the timed step."""
    import torch
    from paper_1504_00636_gb300 import binding
    dt = np.float32 if mixed else np.float64
    m = binding.Merger(p.dx, p.dp, p.n_cells, p.n, p.cell_size, p.n_min,
                       "mixed" if mixed else "fp64")

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


def accuracy_report(p, dev, sample_cells=256, seed=0):
    """Mixed path vs the FP64 oracle on sampled cells (outside any timed
    region): cells whose membership differs, worst coordinate error of the
    merged particles (relative to each axis' mean |q|), worst per-cell
    conservation error of W and W P (relative to sum w and sum w |p|).
    The oracle runs on (a) the float32-rounded inputs the mixed path stores
    and (b) the original FP64 inputs, separating input rounding from
    accumulation."""
    import torch
    import oracle
    from paper_1504_00636_gb300 import binding
    q = p.astype(np.float32)
    m = binding.Merger(q.dx, q.dp, q.n_cells, q.n, q.cell_size, q.n_min, "mixed")
    cells, pos, mom, w = to_device(q, True, dev)
    M, out = m.merge(cells, pos, mom, w, q.tol_x, q.tol_p)
    g_cell = out.cell[:M].cpu().numpy()
    g_index = out.index[:q.n].cpu().numpy().astype(np.int64)
    g_w = out.w[:M].cpu().numpy()
    g_c = np.concatenate([np.stack([t[:M].cpu().double().numpy() for t in out.pos]),
                          np.stack([t[:M].cpu().numpy() for t in out.mom])])
    m.close()
    rng = np.random.default_rng(seed)
    present = np.unique(q.cell)
    sample = np.sort(rng.choice(present, min(sample_cells, present.size), replace=False))
    first_g = np.searchsorted(g_cell, np.arange(q.n_cells))
    rep = {"sample_cells": int(sample.size)}
    for tag, src in (("vs_oracle_on_f32_inputs", q), ("vs_oracle_on_f64_inputs", p)):
        sub = src.select_cells(sample)
        r = oracle.merge_particles(sub, threads=os.cpu_count() or 1)
        mask = np.isin(q.cell, sample)
        gi = g_index[mask] - first_g[q.cell[mask]]
        first_o = np.searchsorted(r.cell, np.arange(q.n_cells))
        oi = r.index.astype(np.int64) - first_o[sub.cell]
        diff = np.unique(sub.cell[gi != oi])
        same = np.setdiff1d(sample, diff)
        go = np.isin(g_cell, same)
        oo = np.isin(r.cell, same)
        worst = 0.0
        if go.sum() == oo.sum() and go.any():
            ref = np.concatenate([r.pos, r.mom])[:, oo]
            got = g_c[:, go]
            scale = np.mean(np.abs(np.concatenate([sub.pos, sub.mom]).astype(np.float64)), axis=1)
            worst = float(np.max(np.abs(got - ref) / scale[:, None]))
        rep[tag] = {"cells_differing": int(diff.size), "flagged_near_ties": int((r.flags != 0).sum()),
                    "max_coord_err_rel": worst}
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


def roofline(p, mixed, stats, stage_ms, peaks, peak_kind, M, workload_name):
    """Roofline of the dominant kernel: the per-cell partition of the small-cell
    class (team_kernel, 4 warps per cell), from its live event timing."""
    b_in, _ = bytes_per_particle(p, mixed)
    t = stage_ms["warp_cells"] * 1e-3
    n = p.n
    # per launch it reads every particle of the cells it owns once and writes
    # the 4-byte final permutation and the head byte of every particle
    bytes_alg = n * (b_in - 4 + 4 + 1)
    D = p.dx + p.dp
    ops_alg = stats["depth_sum"] * (2 * D + 2)
    hbm = peaks["hbm_gbs"] * 1e9
    alu_peak = FP32_OPS_PEAK if mixed else FP64_OPS_PEAK
    t_hbm, t_alu = bytes_alg / hbm, ops_alg / alu_peak
    traffic = ncu_traffic("team_kernel", workload_name, "mixed" if mixed else "fp64")
    if t_hbm >= t_alu:
        ach = bytes_alg / t / 1e9
        return {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(ach / peaks["hbm_gbs"], 4),
                "traffic": traffic, "kernel": "team_kernel",
                "peak_source": peak_kind}
    ach = ops_alg / t / 1e12
    return {"bound": "alu", "achieved": round(ach, 4), "peak": round(alu_peak / 1e12, 3),
            "unit": "Tops/s", "frac": round(ach / (alu_peak / 1e12), 4), "traffic": traffic,
            "kernel": "team_kernel",
            "peak_source": "FP32 lanes x SMs x max clock" if mixed else
            "nominal GB300 FP64 1.25 TFLOP/s / 2"}


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

    results = {}
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    precs = {"both": [True, False], "mixed": [True], "fp64": [False]}[args.precision]
    for mixed in precs:
        q = p.astype(np.float32) if mixed else p
        results[mixed] = time_device(q, mixed, args.steps, args.warmup, dev, flush)
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
                              res["M"], args.workload),
            depth_sum=res["stats"]["depth_sum"], splits=res["stats"]["splits"],
            graph=res["graph"],
            eager_ms_per_step=round(float(np.mean(res["eager_ms"])), 4))
    head = lines[True] if True in lines else lines[False]
    mixed_head = True in lines
    e2e = None
    if not args.no_e2e:
        # every rank copies its own replica in and out; the job takes the
        # slowest rank's time
        q = p.astype(np.float32) if mixed_head else p
        e = time_e2e(q, mixed_head, max(3, args.steps // 4), 2)
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
            "clocks": clk}
    if mixed_head and False in lines:
        f = lines[False]
        line["fp64_plain"] = {"value": f["value"], "ms_per_step": f["ms_per_step"],
                              "cuda_graph": f["graph"], "eager_ms_per_step": f["eager_ms_per_step"],
                              "roofline": f["roofline"], "stage_ms": f["stage_ms"], "M": f["M"],
                              "speedup_mixed_over_fp64": round(head["value"] / f["value"], 3)}
    if e2e is not None:
        line["e2e"] = e2e
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
