"""The C ABI library loads and exports every function include/pma.h declares,
and rejects bad configurations before touching any device."""
import ctypes
import os
import re

import pytest

from paper_1504_00636_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pma.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pma_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("pma_create", "pma_merge", "pma_destroy"):
        assert n in names


def test_library_exports_every_declared_function():
    lib = binding.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(binding.SYMBOLS)


def test_error_strings():
    assert binding.pma_error_string(0) == "ok"
    assert "capacity" in binding.pma_error_string(binding.PMA_ERR_CAPACITY)
    assert binding.pma_error_string(12345) == "unknown status"


@pytest.mark.parametrize("field,value", [("dx", 0), ("dx", 4), ("dp", 0), ("n_cells", 0),
                                         ("n_min", -1), ("precision", 7), ("capacity", -5)])
def test_create_rejects_bad_config_without_device(field, value):
    cfg = binding.pma_config()
    cfg.dx, cfg.dp, cfg.n_cells, cfg.capacity = 1, 3, 4, 16
    cfg.cell_size[0] = 1.0
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    rc = binding.load().pma_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == binding.PMA_ERR_INVALID_ARG
    assert not h.value


def test_create_rejects_bad_cell_size():
    cfg = binding.pma_config()
    cfg.dx, cfg.dp, cfg.n_cells, cfg.capacity = 2, 3, 4, 16
    cfg.cell_size[0] = 1.0
    cfg.cell_size[1] = 0.0
    h = ctypes.c_void_p()
    assert binding.load().pma_create(ctypes.byref(cfg), ctypes.byref(h)) == binding.PMA_ERR_INVALID_ARG


def test_null_handle_calls_are_rejected():
    lib = binding.load()
    assert lib.pma_sync(None) == binding.PMA_ERR_INVALID_ARG
    assert lib.pma_destroy(None) == binding.PMA_OK
    assert lib.pma_last_error(None) == b""


def test_struct_layouts_match_the_header(tmp_path):
    # the ctypes mirrors of pma_config, pma_output and pma_stats have the C
    # layout: sizes and field offsets from a C program compiled against pma.h
    import subprocess
    structs = {"pma_config": binding.pma_config, "pma_output": binding.pma_output,
               "pma_stats": binding.pma_stats}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pma.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (name, f)]) == getattr(cls, f).offset, (name, f)
