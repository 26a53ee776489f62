"""Tolerance scan: merge ratio and energy change against (T_X, T_P).

A synthetic counterpart of the paper's tolerance study (Sec. 4.3): the same
particles are merged for every pair of tolerances, and each run reports the
merge ratio M/N and the relative change of the kinetic energy.  Merging
conserves W and W P (Step 7) but not energy (Sec. 3, remark on energy): a
centroid's energy is at most the weighted mean of its members' energies
(sqrt(1 + |p|^2) is convex), so the energy can only drop.

Readings used here: energy E = sum w (sqrt(1 + |p|^2) - 1), momenta in units
of m c (unit mass).  In exact arithmetic a larger tolerance stops every
branch of the recursion no later (Step 3) and, with the paper's split rule,
cuts on the same axis (Step 4 does not involve T), so M/N never rises and the
energy loss never falls as (T_X, T_P) grow.  Position CVs of in-cell
positions are at most 1/2, so T_X = 0.5 and T_X = 1.0 give the same result.

Usage (one GPU):  python -m paper_1504_00636_gb300.scan --workload shower_256
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import binding, synth


def energy(w, mom):
    """Kinetic energy sum w (sqrt(1 + |p|^2) - 1) of host arrays (mom of
    shape [dp, M]), for checks on the host.  Computed as
    w |p|^2 / (sqrt(1 + |p|^2) + 1), which has no cancellation for small |p|."""
    p2 = np.sum(np.asarray(mom, dtype=np.float64) ** 2, axis=0)
    return float(np.sum(np.asarray(w, dtype=np.float64) * p2 / (np.sqrt(1.0 + p2) + 1.0)))


def tolerance_scan(p, tol_x, tol_p, precision="mixed", flags=0, device="cuda"):
    """Merge the particles ``p`` (a ``synth.Particles``) for every (T_X, T_P)
    pair; returns a list of dicts with tol_x, tol_p, M, ratio = M/N,
    dE = (E_in - E_out) / E_in (the library's FP64 energy accounting,
    PMA_FLAG_ENERGY_STATS) and the call time in ms."""
    import torch
    dev = torch.device(device)
    q = p.astype(np.float32) if precision == "mixed" else p
    dt = torch.float32 if precision == "mixed" else torch.float64
    m = binding.Merger(q.dx, q.dp, q.n_cells, q.n, q.cell_size, q.n_min, precision,
                       flags | binding.PMA_FLAG_ENERGY_STATS)
    try:
        cells = torch.from_numpy(q.cell).to(dev)
        pos = [torch.from_numpy(np.ascontiguousarray(q.pos[a])).to(dev, dt) for a in range(q.dx)]
        mom = [torch.from_numpy(np.ascontiguousarray(q.mom[a])).to(dev, dt) for a in range(q.dp)]
        w = torch.from_numpy(np.ascontiguousarray(q.w)).to(dev, dt)
        out = m.alloc_output(dev, index=False)
        rows = []
        for tx in tol_x:
            for tp in tol_p:
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                M, out = m.merge(cells, pos, mom, w, float(tx), float(tp), out=out)
                t1 = time.perf_counter()
                st = m.stats()
                e_in, e_out = st["energy_in"], st["energy_out"]
                rows.append(dict(tol_x=float(tx), tol_p=float(tp), M=int(M),
                                 ratio=M / max(q.n, 1), dE=(e_in - e_out) / e_in,
                                 ms=1e3 * (t1 - t0)))
        return rows
    finally:
        m.close()


WORKLOADS = {
    "shower_256": lambda: synth.shower(grid=(256, 256)),
    "shower": lambda: synth.shower(),
    "two_stream": lambda: synth.two_stream(),
}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="shower_256", choices=sorted(WORKLOADS))
    ap.add_argument("--tx", default="0.05,0.1,0.25,0.5,1.0")
    ap.add_argument("--tp", default="0.01,0.02,0.05,0.1,0.2")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--flags", type=int, default=0)
    a = ap.parse_args(argv)
    p = WORKLOADS[a.workload]()
    rows = tolerance_scan(p, [float(x) for x in a.tx.split(",")],
                          [float(x) for x in a.tp.split(",")], a.precision, a.flags)
    print(json.dumps({"workload": a.workload, "n": p.n, "precision": a.precision,
                      "flags": a.flags, "rows": rows}))


if __name__ == "__main__":
    main()
