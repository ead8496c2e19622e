"""The C-ABI library builds for sm_103a, loads, and exports every function the
headers in include/ declare (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\([^;{]*\)\s*;", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2404_04441_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for need in ("wave_create", "wave_step", "wave_propagate", "wave_get_field",
                 "wave_set_state", "wave_reset", "wave_destroy", "wave_strerror",
                 "wave_cfl_dt", "wave_synchronize"):
        assert need in names, names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(libpath):
    import paper_2404_04441_gb300 as gw
    gw.load(libpath)
    assert gw.wave_strerror(0) == "ok"
    assert gw.wave_strerror(-4).startswith("dt above")
    assert gw.wave_cfl_dt((10.0, 10.0, 10.0), -1.0) < 0
    assert gw.wave_cfl_dt((0.0, 10.0, 10.0), 3000.0) < 0
    # Courant number v dt / h of the scheme on a cubic grid: 2 / sqrt(3 S)
    S = 205 / 72 + 2 * (8 / 5 + 1 / 5 + 8 / 315 + 1 / 560)
    assert gw.wave_cfl_dt((10.0, 10.0, 10.0), 3500.0) * 3500.0 / 10.0 == pytest.approx(
        2.0 / (3.0 * S) ** 0.5, rel=1e-14)


def test_sm103a_build_fits_register_budget(libpath):
    log = open(os.path.join(os.path.dirname(libpath), "ptxas.log")).read()
    assert "sm_103a" in log
    # no sweep variant spills registers to local memory
    blocks = re.split(r"Compiling entry function", log)
    for b in blocks:
        if "wave_sweep_kernel" in b:
            m = re.search(r"(\d+) bytes spill stores", b)
            assert m and int(m.group(1)) == 0, b[:300]
