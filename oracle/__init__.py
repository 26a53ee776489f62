"""CPU oracle of the Voronoi particle-merging algorithm (Sec. 3, Steps 1-7).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / reference leg are the only users.  Nothing in
the CUDA library imports, links or executes anything here, and nothing here
uses the CUDA library.

Two independent implementations:

* ``merge`` / ``trace`` / ``subset_moments``: ctypes wrappers around the plain
  FP64 C code in ``pma_oracle.c`` (compiled on first use with gcc).
* ``exact`` (module ``oracle.exact``): the same steps in exact rational
  arithmetic (``fractions.Fraction``) for cells of a few dozen particles.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pma_oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

NEAR_STOP = 1
NEAR_ARGMAX = 2
NEAR_CUT = 4

# decision variants (bit flags), off by default:
# VAR_NORMALIZED  Step 4 maximises Delta_l / T_l instead of the raw Delta_l
# VAR_PNORM       momentum CVs use |P| (length of the mean momentum vector)
VAR_NORMALIZED = 2
VAR_PNORM = 4
# Step 7 variant: sets of m >= 3 become two particles that also conserve the
# total energy sum w sqrt(1 + |p|^2) (see pma_oracle.c)
VAR_CONSERVE_ENERGY = 8

_ERRORS = {1: "invalid argument", 2: "invalid input", 3: "out of memory"}


class _Stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "n_in", "n_out", "cells_merged", "cells_passthrough", "splits", "leaves",
        "depth_sum", "max_depth", "near_stop", "near_argmax", "near_cut",
        "degenerate_cuts")] + [("energy_in", ctypes.c_double),
                               ("energy_out", ctypes.c_double)]


def compile_source(src: str, out: str) -> str:
    """gcc -O2 a C source of the oracle into a shared object."""
    tmp = out + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           "-ffp-contract=off", "-o", tmp, src, "-lm", "-lpthread"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_liboracle.so``."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


def load_library(path):
    """Bind the oracle's C entry points from a compiled shared object."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.pma_oracle_merge.argtypes = [i64, P, ctypes.c_int, ctypes.c_int, P, P, P,
                                     i64, P, i32, dbl, dbl, ctypes.c_int,
                                     P, P, P, P, P, P, P, ctypes.POINTER(_Stats),
                                     ctypes.c_uint]
    lib.pma_oracle_merge.restype = ctypes.c_int
    lib.pma_oracle_trace.argtypes = [i64, ctypes.c_int, ctypes.c_int, P, P, P, P,
                                     dbl, dbl, P, P, P, P, P, P, P, P, ctypes.c_uint]
    lib.pma_oracle_trace.restype = ctypes.c_int
    lib.pma_oracle_subset_moments.argtypes = [i64, ctypes.c_int, ctypes.c_int, P, P,
                                              i64, P, P, P, P, P, P, P, ctypes.c_uint]
    lib.pma_oracle_subset_moments.restype = ctypes.c_int
    return lib


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    with _lock:
        if _lib is None:
            build()
            _lib = load_library(_LIB)
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclasses.dataclass
class MergeResult:
    count: int
    cell: np.ndarray  # int32 [M]
    pos: np.ndarray  # float64 [dx, M]
    mom: np.ndarray  # float64 [dp, M]
    w: np.ndarray  # float64 [M]
    index: np.ndarray  # int32 [n]: output slot of every input particle
    flags: np.ndarray  # uint8 [n_cells]: near-tie bits per cell
    stats: dict


def merge(cell, pos, mom, w, n_cells, cell_size=(1.0, 1.0, 1.0), n_min=0,
          tol_x=0.1, tol_p=0.1, threads=1, lib=None, variant=0) -> MergeResult:
    """Merge every cell (Steps 1-7); inputs are upcast to float64."""
    lib = _load(lib)
    cell = np.ascontiguousarray(cell, dtype=np.int32)
    pos = _f64(pos)
    mom = _f64(mom)
    w = _f64(w)
    n = cell.shape[0]
    dx, dp = pos.shape[0], mom.shape[0]
    cap = max(n, 1)
    cs = _f64(list(cell_size)[:3] + [1.0] * (3 - len(cell_size)))
    out_cell = np.empty(cap, np.int32)
    out_pos = np.empty((dx, cap))
    out_mom = np.empty((dp, cap))
    out_w = np.empty(cap)
    out_index = np.empty(cap, np.int32)
    flags = np.zeros(int(n_cells), np.uint8)
    count = ctypes.c_int64(0)
    st = _Stats()
    rc = lib.pma_oracle_merge(n, _ptr(cell), dx, dp, _ptr(pos), _ptr(mom), _ptr(w),
                              int(n_cells), _ptr(cs), int(n_min), float(tol_x), float(tol_p),
                              int(threads), _ptr(out_cell), _ptr(out_pos), _ptr(out_mom),
                              _ptr(out_w), _ptr(out_index), _ptr(flags),
                              ctypes.byref(count), ctypes.byref(st), int(variant))
    if rc != 0:
        raise ValueError("oracle merge failed: %s" % _ERRORS.get(rc, rc))
    m = count.value
    stats = {k: getattr(st, k) for k, _ in _Stats._fields_}
    return MergeResult(m, out_cell[:m].copy(), out_pos[:, :m].copy(),
                       out_mom[:, :m].copy(), out_w[:m].copy(), out_index[:n].copy(),
                       flags, stats)


def merge_particles(p, threads=1, tol_x=None, tol_p=None, n_min=None, lib=None,
                    variant=0) -> MergeResult:
    """``merge`` on a ``synth.Particles`` set."""
    return merge(p.cell, p.pos, p.mom, p.w, p.n_cells, p.cell_size,
                 p.n_min if n_min is None else n_min,
                 p.tol_x if tol_x is None else tol_x,
                 p.tol_p if tol_p is None else tol_p, threads, lib=lib, variant=variant)


@dataclasses.dataclass
class Trace:
    perm: np.ndarray  # final order of the set; each node is a contiguous range
    begin: np.ndarray
    end: np.ndarray
    depth: np.ndarray
    axis: np.ndarray  # -1 for leaves
    Q: np.ndarray
    near: int


def trace(pos, mom, w, cell_size=(1.0, 1.0, 1.0), tol_x=0.1, tol_p=0.1, lib=None,
          variant=0) -> Trace:
    """The recursion tree of one particle set (one cell), V1-first preorder."""
    lib = _load(lib)
    pos, mom, w = _f64(pos), _f64(mom), _f64(w)
    m = w.shape[0]
    cs = _f64(list(cell_size)[:3] + [1.0] * (3 - len(cell_size)))
    perm = np.empty(m, np.int64)
    nb, ne, nd = (np.empty(2 * m, np.int64) for _ in range(3))
    na = np.empty(2 * m, np.int32)
    nq = np.empty(2 * m)
    nn = ctypes.c_int64(0)
    near = ctypes.c_uint32(0)
    rc = lib.pma_oracle_trace(m, pos.shape[0], mom.shape[0], _ptr(pos), _ptr(mom), _ptr(w),
                              _ptr(cs), float(tol_x), float(tol_p), _ptr(perm), _ptr(nb),
                              _ptr(ne), _ptr(nd), _ptr(na), _ptr(nq), ctypes.byref(nn),
                              ctypes.byref(near), int(variant))
    if rc != 0:
        raise ValueError("oracle trace failed: %s" % _ERRORS.get(rc, rc))
    k = nn.value
    return Trace(perm, nb[:k].copy(), ne[:k].copy(), nd[:k].copy(), na[:k].copy(),
                 nq[:k].copy(), near.value)


def subset_moments(pos, mom, w, cell_size=(1.0, 1.0, 1.0), idx=None, lib=None, variant=0):
    """Steps 1-2 on one set: returns (W, Q[D], sigma[D], Delta[D])."""
    lib = _load(lib)
    pos, mom, w = _f64(pos), _f64(mom), _f64(w)
    m = w.shape[0]
    D = pos.shape[0] + mom.shape[0]
    cs = _f64(list(cell_size)[:3] + [1.0] * (3 - len(cell_size)))
    W = ctypes.c_double(0.0)
    Q, S, Dl = np.empty(D), np.empty(D), np.empty(D)
    ix = None if idx is None else np.ascontiguousarray(idx, dtype=np.int64)
    mm = m if ix is None else ix.shape[0]
    rc = lib.pma_oracle_subset_moments(mm, pos.shape[0], mom.shape[0], _ptr(pos), _ptr(mom),
                                       m, _ptr(w), _ptr(ix), _ptr(cs), ctypes.byref(W),
                                       _ptr(Q), _ptr(S), _ptr(Dl), int(variant))
    if rc != 0:
        raise ValueError("oracle moments failed: %s" % _ERRORS.get(rc, rc))
    return W.value, Q, S, Dl
