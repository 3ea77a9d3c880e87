"""The C-ABI library builds, loads and exports every entry point include/sidp.h declares;
host-side argument validation (no GPU needed: invalid configs fail before any CUDA call)."""
import ctypes

import pytest

from paper_2004_08503_gb300 import build, sidp


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sidp.load()


def test_exports_every_declared_symbol(lib):
    names = sidp.header_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps every one of them
    assert set(names) <= set(sidp._SIGS)


def test_status_strings(lib):
    assert sidp.sidp_status_str(0) == "ok"
    assert "argument" in sidp.sidp_status_str(1)
    assert sidp.sidp_status_str(99) == "unknown status"


@pytest.mark.parametrize("bad", [
    dict(p=0), dict(p=8), dict(nx=0), dict(domain=(0, 1, 0, 2)), dict(cfl=0.0), dict(cfl=1.5),
    dict(law="euler", gamma=1.0), dict(law="euler", gamma=2.0),
    dict(bc=("periodic", "outflow", "periodic", "periodic")), dict(limiter="none", precision="fp64", nx=-3),
])
def test_create_rejects_invalid_config(lib, bad):
    kw = dict(law="burgers", p=3, nx=4, ny=4)
    kw.update(bad)
    cfg = sidp.make_config(**kw)
    h = ctypes.c_void_p()
    st = lib.sidp_create(ctypes.byref(h), ctypes.byref(cfg), None)
    assert st == 1 and not h.value
    assert len(lib.sidp_last_error(None)) > 0


def test_null_arguments(lib):
    assert lib.sidp_create(None, None, None) == 1
    assert lib.sidp_set_state(None, None) == 1
    assert lib.sidp_step(None, 1) == 1
    assert lib.sidp_destroy(None) == 0


def test_plain_c_client_compiles_links_and_runs(lib, tmp_path):
    """The header is valid C99 and the library is usable from C without Python: a C client of
    sidp_curved_metrics (host only) built with gcc -std=c99 -Wall -Werror against libsidp.so."""
    import os
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no gcc")
    here = os.path.dirname(os.path.abspath(__file__))
    root = os.path.dirname(here)
    pkg = os.path.dirname(sidp.LIB_PATH)
    exe = str(tmp_path / "metrics_client")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                    os.path.join(here, "c_abi", "metrics_client.c"), "-o", exe, "-L", pkg, "-lsidp",
                    "-Wl,-rpath," + pkg, "-lm"], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    area, err = float(out[0].split()[1]), float(out[0].split()[3])
    assert abs(area - 6.0) < 1e-13 and err < 1e-14, out
    assert out[1] == "mirrored invalid argument"
