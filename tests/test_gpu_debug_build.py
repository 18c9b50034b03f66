"""The checked build (libhn_debug.so, HN_DEBUG_CHECKS=1; include/hn_debug.h): the per-kernel and
solver tests run against it in a child process, where every kernel checks its work-list items and
level descriptors (a failed check fails the solve) and every hierarchy's and operator's guard bytes
are verified when the tests destroy them; a damaged guard is reported."""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import require_gpu
from paper_0904_4152_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_small_level_tests_pass_on_the_checked_build():
    hn = require_gpu()
    if hn.hn_debug_build():
        pytest.skip("already the checked build")
    env = dict(os.environ, HN_DEBUG_CHECKS="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-m", "gpu", "-p", "no:cacheprovider", "-x",
           "tests/test_gpu_kernels.py", "tests/test_gpu_solve.py", "tests/test_gpu_mixed_bc.py",
           "tests/test_gpu_pcg.py", "tests/test_gpu_debug_build.py::test_guard_damage_is_reported"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and " failed" not in r.stdout


def test_guard_damage_is_reported():
    hn = require_gpu()
    if not hn.hn_debug_build():
        pytest.skip("runs in the checked build (the child process above)")
    L = 5
    A = hn.hn_band_create(L)
    mg = hn.hn_mg_setup(A, prec=1)
    hn.hn_band_destroy(A)
    x, st, status = hn.hn_mg_solve(mg, L, I.rhs_uniform(L, 3))
    assert status == hn.HN_OK
    hn.hn_debug_check_mg(mg)                        # intact after a solve
    hn.hn_debug_overwrite_guard(mg)
    with pytest.raises(hn.HnError) as e:
        hn.hn_debug_check_mg(mg)
    assert e.value.status == hn.HN_ERR_STATE and "guard" in str(e.value)
    with pytest.raises(hn.HnError):
        hn.hn_mg_destroy(mg)                        # frees the block, then reports the damage
