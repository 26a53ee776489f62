"""Thin ctypes binding of the C ABI in ``include/pma.h``.

Functions carry the C names (``pma_create``, ``pma_merge``, ...) and only
marshal arguments: device arrays are torch CUDA tensors whose ``data_ptr()``
is handed to the library, host arrays are numpy arrays or pinned CPU tensors.
Every step of the merge runs in the CUDA library; there is no other code
path, and loading fails loudly when the library cannot be found or built.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

from . import _build

PMA_OK = 0
PMA_ERR_INVALID_ARG = 1
PMA_ERR_INPUT = 2
PMA_ERR_CUDA = 3
PMA_ERR_NOMEM = 4
PMA_ERR_CAPACITY = 5
PMA_ERR_TIMEOUT = 6
PMA_ERR_INTERNAL = 7

PMA_FP64 = 0
PMA_MIXED = 1
PMA_FLAG_NO_INDEX = 1
PMA_FLAG_SPLIT_NORMALIZED = 2
PMA_FLAG_MOMENTUM_NORM = 4
PMA_FLAG_CONSERVE_ENERGY = 8
PMA_FLAG_ENERGY_STATS = 16
PMA_NEAR_STOP = 1
PMA_NEAR_ARGMAX = 2
PMA_NEAR_CUT = 4
PMA_RECHECKED = 8
PMA_NEAR_ANY = PMA_NEAR_STOP | PMA_NEAR_ARGMAX | PMA_NEAR_CUT

SYMBOLS = ("pma_create", "pma_merge", "pma_merge_host", "pma_sync", "pma_get_stats",
           "pma_set_timing", "pma_get_timing", "pma_merge_noalloc", "pma_destroy",
           "pma_error_string", "pma_last_error", "pma_set_wait_limit",
           "pma_test_withhold_status", "pma_test_status_of_bits", "pma_probe_fma",
           "pma_get_classes", "pma_set_classes", "pma_tune", "pma_tune_cache_lookup",
           "pma_tune_cache_store", "pma_checked_build", "pma_check_first")
PMA_NOALLOC_MAX_N = 65536
PMA_NOALLOC_MAX_CELLS = 65536
PMA_N_STAGES = 7
STAGES = ("binning", "big_cells", "warp_cells", "block_cells", "pieces", "emit", "total")


class pma_config(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_int32), ("dp", ctypes.c_int32),
                ("cell_size", ctypes.c_double * 3), ("n_cells", ctypes.c_int64),
                ("n_min", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("capacity", ctypes.c_int64), ("flags", ctypes.c_uint32)]


class pma_output(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_void_p), ("pos", ctypes.c_void_p * 3),
                ("mom", ctypes.c_void_p * 3), ("w", ctypes.c_void_p),
                ("index", ctypes.c_void_p), ("count_dev", ctypes.c_void_p),
                ("cell_flags", ctypes.c_void_p)]


class pma_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in (
        "n_in", "n_out", "cells_merged", "cells_passthrough", "splits", "leaves",
        "depth_sum", "degenerate_cuts", "big_cells", "sorted_input", "near_stop",
        "near_argmax", "near_cut", "fp64_rechecks", "cells_flagged", "cells_tiny",
        "cells_small", "cells_large")] + [("energy_in", ctypes.c_double),
                                           ("energy_out", ctypes.c_double)]


class PmaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("pma status %d (%s): %s" % (code, pma_error_string(code), msg))
        self.code = code


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load ``libpma.so`` (building it with nvcc when absent or stale).  The
    environment variable PMA_LIBRARY names another build of the library to
    load instead, such as the bounds-checked one (``_build.build_checked``)."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("PMA_LIBRARY") or _build.LIB
            if build_if_missing and not os.environ.get("PMA_LIBRARY"):
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libpma.so not found at %s; run __graft_entry__.build()" % path)
            lib = ctypes.CDLL(path)
            P = ctypes.c_void_p
            lib.pma_create.argtypes = [ctypes.POINTER(pma_config), ctypes.POINTER(P)]
            lib.pma_create.restype = ctypes.c_int
            args = [P, ctypes.c_int64, P, P, P, P, ctypes.c_double, ctypes.c_double,
                    ctypes.POINTER(pma_output), ctypes.POINTER(ctypes.c_int64), P]
            lib.pma_merge.argtypes = args
            lib.pma_merge.restype = ctypes.c_int
            lib.pma_merge_host.argtypes = args
            lib.pma_merge_host.restype = ctypes.c_int
            lib.pma_sync.argtypes = [P]
            lib.pma_sync.restype = ctypes.c_int
            lib.pma_get_stats.argtypes = [P, ctypes.POINTER(pma_stats)]
            lib.pma_get_stats.restype = ctypes.c_int
            lib.pma_set_timing.argtypes = [P, ctypes.c_int]
            lib.pma_set_timing.restype = ctypes.c_int
            lib.pma_get_timing.argtypes = [P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]
            lib.pma_get_timing.restype = ctypes.c_int
            lib.pma_merge_noalloc.argtypes = [ctypes.POINTER(pma_config)] + args[1:]
            lib.pma_merge_noalloc.restype = ctypes.c_int
            lib.pma_set_wait_limit.argtypes = [P, ctypes.c_int64]
            lib.pma_set_wait_limit.restype = ctypes.c_int
            lib.pma_checked_build.argtypes = []
            lib.pma_checked_build.restype = ctypes.c_int
            lib.pma_check_first.argtypes = [P, ctypes.POINTER(ctypes.c_uint64)]
            lib.pma_check_first.restype = ctypes.c_int
            lib.pma_test_withhold_status.argtypes = [P, ctypes.c_int]
            lib.pma_test_withhold_status.restype = ctypes.c_int
            caps = ctypes.POINTER(ctypes.c_int32)
            lib.pma_get_classes.argtypes = [P, caps]
            lib.pma_get_classes.restype = ctypes.c_int
            lib.pma_set_classes.argtypes = [P, caps]
            lib.pma_set_classes.restype = ctypes.c_int
            lib.pma_tune.argtypes = [P, ctypes.c_int64, P, P, P, P, ctypes.c_double,
                                     ctypes.c_double, ctypes.POINTER(pma_output), P]
            lib.pma_tune.restype = ctypes.c_int
            lib.pma_tune_cache_lookup.argtypes = [ctypes.c_char_p, ctypes.c_char_p, caps]
            lib.pma_tune_cache_lookup.restype = ctypes.c_int
            lib.pma_tune_cache_store.argtypes = [ctypes.c_char_p, ctypes.c_char_p, caps,
                                                 ctypes.c_double]
            lib.pma_tune_cache_store.restype = ctypes.c_int
            lib.pma_probe_fma.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int)]
            lib.pma_probe_fma.restype = ctypes.c_int
            lib.pma_test_status_of_bits.argtypes = [ctypes.c_uint]
            lib.pma_test_status_of_bits.restype = ctypes.c_int
            lib.pma_destroy.argtypes = [P]
            lib.pma_destroy.restype = ctypes.c_int
            lib.pma_error_string.argtypes = [ctypes.c_int]
            lib.pma_error_string.restype = ctypes.c_char_p
            lib.pma_last_error.argtypes = [P]
            lib.pma_last_error.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def pma_error_string(code: int) -> str:
    return load().pma_error_string(code).decode()


def pma_last_error(handle) -> str:
    return load().pma_last_error(handle).decode()


def _check(rc, handle=None):
    if rc != PMA_OK:
        raise PmaError(rc, pma_last_error(handle) if handle else "")


def pma_create(cfg: pma_config):
    h = ctypes.c_void_p()
    _check(load().pma_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def pma_destroy(handle) -> None:
    _check(load().pma_destroy(handle))


def _ptrs(arrs, n=3):
    out = (ctypes.c_void_p * n)()
    for i, a in enumerate(arrs):
        out[i] = a
    return out


def pma_merge(handle, n, cells, pos, mom, weights, tol_x, tol_p, out: pma_output,
              count_host=True, stream=0):
    """Raw call: every array argument is a device pointer (int)."""
    cnt = ctypes.c_int64(-1)
    rc = load().pma_merge(handle, n, cells, _ptrs(pos), _ptrs(mom), weights, tol_x, tol_p,
                          ctypes.byref(out), ctypes.byref(cnt) if count_host else None, stream)
    _check(rc, handle)
    return cnt.value


def pma_merge_host(handle, n, cells, pos, mom, weights, tol_x, tol_p, out: pma_output,
                   stream=0):
    """Raw call: every array argument is a host pointer (int)."""
    cnt = ctypes.c_int64(-1)
    rc = load().pma_merge_host(handle, n, cells, _ptrs(pos), _ptrs(mom), weights, tol_x, tol_p,
                               ctypes.byref(out), ctypes.byref(cnt), stream)
    _check(rc, handle)
    return cnt.value


def pma_merge_noalloc(cfg: pma_config, n, cells, pos, mom, weights, tol_x, tol_p,
                      out: pma_output, stream=0):
    """Raw call of the allocation-free entry point (device pointers as ints).

    For callers that must not allocate device memory: no handle, scratch in
    a fixed array inside the library, n <= PMA_NOALLOC_MAX_N particles
    grouped by cell, n_cells <= PMA_NOALLOC_MAX_CELLS.  Waits for `stream`.
    """
    cnt = ctypes.c_int64(-1)
    rc = load().pma_merge_noalloc(ctypes.byref(cfg), n, cells, _ptrs(pos), _ptrs(mom), weights,
                                  tol_x, tol_p, ctypes.byref(out), ctypes.byref(cnt), stream)
    if rc != PMA_OK:
        raise PmaError(rc, "pma_merge_noalloc")
    return cnt.value


def pma_sync(handle) -> None:
    _check(load().pma_sync(handle), handle)


def pma_set_wait_limit(handle, wait_ns: int) -> None:
    _check(load().pma_set_wait_limit(handle, int(wait_ns)), handle)


def pma_checked_build() -> bool:
    """True when the loaded library is the bounds-checked build."""
    return load().pma_checked_build() == 1


def pma_check_first(handle):
    """(site, index) of the first failed bounds check of the handle's last
    synchronised call, or None (always None in the normal build)."""
    v = ctypes.c_uint64(0)
    _check(load().pma_check_first(handle, ctypes.byref(v)), handle)
    return None if v.value == 0 else (v.value >> 48, v.value & ((1 << 48) - 1))


def pma_test_withhold_status(handle, tile: int) -> None:
    _check(load().pma_test_withhold_status(handle, int(tile)), handle)


def pma_probe_fma(precision: str):
    """Measured independent-FMA rate per second ("mixed": FP32, "fp64") and
    the SM count of the current device."""
    r, sms = ctypes.c_double(0.0), ctypes.c_int(0)
    _check(load().pma_probe_fma(PMA_MIXED if precision == "mixed" else PMA_FP64,
                                ctypes.byref(r), ctypes.byref(sms)))
    return r.value, sms.value


def pma_get_classes(handle):
    """(cap_t, cap_w, cap, base, widen): the population limits of the
    one-warp, 4-warp and 8-warp (or 12-warp) team paths, the class base of the subset size
    classes, and whether sparse rounds widen the lane groups."""
    c = (ctypes.c_int32 * 5)()
    _check(load().pma_get_classes(handle, c), handle)
    return tuple(c)


def pma_set_classes(handle, caps) -> None:
    """caps = (cap_t, cap_w, cap[, base[, widen]]); entries left out keep the
    handle's current values."""
    caps = tuple(caps)
    caps = caps + pma_get_classes(handle)[len(caps):]
    c = (ctypes.c_int32 * 5)(*caps)
    _check(load().pma_set_classes(handle, c), handle)


def pma_tune(handle, n, cells, pos, mom, weights, tol_x, tol_p, out: pma_output, stream=0):
    """Raw call (device pointers as ints): time the candidate classes on the
    input and keep the fastest (see include/pma.h)."""
    _check(load().pma_tune(handle, n, cells, _ptrs(pos), _ptrs(mom), weights, tol_x, tol_p,
                           ctypes.byref(out), stream), handle)


def pma_tune_cache_lookup(path: str, key: str):
    c = (ctypes.c_int32 * 5)()
    rc = load().pma_tune_cache_lookup(path.encode(), key.encode(), c)
    return tuple(c) if rc == PMA_OK else None


def pma_tune_cache_store(path: str, key: str, caps, ms: float) -> None:
    c = (ctypes.c_int32 * 5)(*caps)
    _check(load().pma_tune_cache_store(path.encode(), key.encode(), c, float(ms)))


def pma_get_stats(handle) -> dict:
    s = pma_stats()
    _check(load().pma_get_stats(handle, ctypes.byref(s)), handle)
    return {k: getattr(s, k) for k, _ in pma_stats._fields_}


def pma_set_timing(handle, enable: bool) -> None:
    _check(load().pma_set_timing(handle, 1 if enable else 0), handle)


def pma_get_timing(handle) -> dict:
    ms = (ctypes.c_float * PMA_N_STAGES)()
    _check(load().pma_get_timing(handle, ms, PMA_N_STAGES), handle)
    return dict(zip(STAGES, [float(x) for x in ms]))


# ---------------------------------------------------------------- helpers

@dataclasses.dataclass
class Output:
    """Device output buffers (torch tensors of `capacity` entries)."""
    cell: "object"
    pos: list
    mom: list
    w: "object"
    index: "object"
    count_dev: "object"
    cell_flags: "object" = None

    def struct(self) -> pma_output:
        o = pma_output()
        o.cell = self.cell.data_ptr()
        for a, t in enumerate(self.pos):
            o.pos[a] = t.data_ptr()
        for a, t in enumerate(self.mom):
            o.mom[a] = t.data_ptr()
        o.w = self.w.data_ptr()
        o.index = self.index.data_ptr() if self.index is not None else None
        o.count_dev = self.count_dev.data_ptr() if self.count_dev is not None else None
        o.cell_flags = self.cell_flags.data_ptr() if self.cell_flags is not None else None
        return o


class Merger:
    """Owns one handle; ``merge`` takes torch CUDA tensors in SoA layout."""

    def __init__(self, dx, dp, n_cells, capacity, cell_size=(1.0, 1.0, 1.0), n_min=0,
                 precision="fp64", flags=0):
        import torch
        self.torch = torch
        self.dx, self.dp, self.n_cells, self.capacity = dx, dp, int(n_cells), int(capacity)
        self.mixed = precision == "mixed"
        cfg = pma_config()
        cfg.dx, cfg.dp = dx, dp
        for a in range(3):
            cfg.cell_size[a] = float(cell_size[a]) if a < len(cell_size) else 1.0
        cfg.n_cells = int(n_cells)
        cfg.n_min = int(n_min)
        cfg.precision = PMA_MIXED if self.mixed else PMA_FP64
        cfg.capacity = int(capacity)
        cfg.flags = flags
        self.handle = pma_create(cfg)
        self.dtype = torch.float32 if self.mixed else torch.float64

    def close(self):
        if self.handle is not None:
            pma_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def alloc_output(self, device="cuda", index=True) -> Output:
        t = self.torch
        N = max(self.capacity, 1)
        return Output(t.empty(N, dtype=t.int32, device=device),
                      [t.empty(N, dtype=self.dtype, device=device) for _ in range(self.dx)],
                      [t.empty(N, dtype=t.float64, device=device) for _ in range(self.dp)],
                      t.empty(N, dtype=t.float64, device=device),
                      t.empty(N, dtype=t.int32, device=device) if index else None,
                      t.zeros(1, dtype=t.int64, device=device),
                      t.zeros(self.n_cells, dtype=t.int32, device=device))

    def merge(self, cells, pos, mom, w, tol_x, tol_p, out: Output = None, sync=True,
              stream=None):
        """Merge device tensors; returns (M or None, out)."""
        if out is None:
            out = self.alloc_output(cells.device)
        n = int(cells.shape[0])
        if stream is None:
            stream = self.torch.cuda.current_stream(cells.device)
        m = pma_merge(self.handle, n, cells.data_ptr(), [p.data_ptr() for p in pos],
                      [p.data_ptr() for p in mom], w.data_ptr(), float(tol_x), float(tol_p),
                      out.struct(), count_host=sync, stream=stream.cuda_stream)
        return (m if sync else None), out

    def sync(self):
        pma_sync(self.handle)

    def stats(self) -> dict:
        return pma_get_stats(self.handle)

    def tune(self, cells, pos, mom, w, tol_x, tol_p, out: Output = None, stream=None):
        """Time the population classes, the class base and group widening on
        these particles and keep the fastest; returns
        (cap_t, cap_w, cap, base, widen)."""
        if out is None:
            out = self.alloc_output(cells.device)
        if stream is None:
            stream = self.torch.cuda.current_stream(cells.device)
        pma_tune(self.handle, int(cells.shape[0]), cells.data_ptr(), [p.data_ptr() for p in pos],
                 [p.data_ptr() for p in mom], w.data_ptr(), float(tol_x), float(tol_p),
                 out.struct(), stream=stream.cuda_stream)
        return pma_get_classes(self.handle)

    def classes(self):
        return pma_get_classes(self.handle)

    def set_classes(self, caps) -> None:
        pma_set_classes(self.handle, caps)

    def set_timing(self, enable: bool = True) -> None:
        pma_set_timing(self.handle, enable)

    def timing(self) -> dict:
        return pma_get_timing(self.handle)
