"""The C-ABI library builds, loads and exports every entry point declared in include/*.h; host-side
argument checks that need no GPU.  No compute call here touches a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(hn_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_0904_4152_gb300 import hn
    return hn.lib()


def test_headers_declare_the_boundary():
    names = declared_functions()
    for n in ("hn_band_create", "hn_mg_setup", "hn_mg_solve", "hn_mg_submit", "hn_mg_poll"):
        assert n in names
    from paper_0904_4152_gb300 import hn
    assert sorted(hn.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(lib, n)


def test_library_is_self_contained(lib):
    # cudart is linked statically: the library needs no CUDA runtime on the loader path
    out = subprocess.run(["ldd", lib._name], capture_output=True, text=True).stdout
    assert "libcudart" not in out
    assert "sm_103a" in lib.hn_version().decode()


def test_host_side_argument_checks(lib):
    from paper_0904_4152_gb300 import hn
    h = ctypes.c_void_p()
    assert lib.hn_band_create(1, None, ctypes.byref(h)) == hn.HN_ERR_ARG
    assert lib.hn_band_create(hn.HN_MAX_LEVEL + 1, None, ctypes.byref(h)) == hn.HN_ERR_ARG
    assert "level" in hn.hn_last_error()
    assert lib.hn_band_create(3, None, None) == hn.HN_ERR_ARG
    import numpy as np
    bad = np.ones(64)
    bad[5] = -1.0
    assert lib.hn_band_create(3, ctypes.c_void_p(bad.ctypes.data), ctypes.byref(h)) == hn.HN_ERR_ARG
    bad[5] = np.nan
    assert lib.hn_band_create(3, ctypes.c_void_p(bad.ctypes.data), ctypes.byref(h)) == hn.HN_ERR_ARG
    o = hn.hn_mg_opts_default()
    assert (o.coarse_L, o.pre, o.post, o.omega, o.tol, o.inner_tol) == (2, 2, 2, 0.7, 1e-8, 1e-2)
    assert (o.dirichlet_sides, o.solver, o.coarse_solver) == (15, hn.HN_SOLVER_MG, hn.HN_COARSE_EXACT)
    assert lib.hn_mg_setup(None, ctypes.byref(o), ctypes.byref(h)) == hn.HN_ERR_ARG
    assert lib.hn_server_create(0, 4, ctypes.byref(h)) == hn.HN_ERR_ARG
    assert lib.hn_mg_poll(None, 1, 0, None, None) == hn.HN_ERR_ARG


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    # no CPU path stands in for the CUDA library: without it every call raises
    from paper_0904_4152_gb300 import hn
    monkeypatch.setattr(hn, "LIB_PATH", str(tmp_path / "libhn.so"))
    monkeypatch.setattr(hn, "_lib", None)
    with pytest.raises(ImportError, match="not built"):
        hn.lib()
    with pytest.raises(ImportError):
        hn.hn_band_create(4)
