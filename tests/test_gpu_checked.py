"""The bounds-checked build (compiled with -DPMA_CHECKED, in place of a memory
sanitizer, which is closed on this machine): parity cases that cross every
kernel path (grouped and ungrouped input, tiny, small and big cells, both
precisions, a merge-heavy variant, the energy-conserving replacement) run
with every index check passing and results equal to the oracle's.  The
normal build compiles no checks and says so."""
import os
import subprocess
import sys

import pytest

from paper_1504_00636_gb300 import _build, binding

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_normal_build_has_no_checks():
    assert not binding.pma_checked_build()


def test_checked_build_passes_every_check():
    lib = _build.build_checked()
    env = dict(os.environ, PMA_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env,
                       capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count("ok ") == 8, r.stdout
