"""The C-ABI library builds, loads and exports every entry point its header
declares; argument checks that return before any CUDA call work without a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "tpcfit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tpcfit_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_17018_gb300 import build, tpcfit
    build.build()
    return tpcfit.load()


def test_header_declares_entry_points():
    names = declared_entry_points()
    for n in ("tpcfit_create", "tpcfit_fit", "tpcfit_destroy", "tpcfit_set_mode", "tpcfit_get_status"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2511_17018_gb300 import tpcfit
    out = subprocess.run(["nm", "-D", "--defined-only", tpcfit.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (tpcfit_\w+)", out))
    declared = set(declared_entry_points())
    assert declared <= exported, declared - exported
    assert exported <= declared, exported - declared   # nothing undocumented
    for n in declared:
        assert hasattr(lib, n)


def test_status_strings_and_version(lib):
    from paper_2511_17018_gb300 import tpcfit
    assert tpcfit.status_string(0) == "ok"
    assert "invalid" in tpcfit.status_string(1)
    assert tpcfit.tpcfit_version() >= 10000


def test_argument_errors_before_any_cuda_call(lib):
    from paper_2511_17018_gb300 import tpcfit
    h = C.c_void_p()
    # null geometry / null output handle
    assert lib.tpcfit_create(None, 0.5, C.byref(h)) == tpcfit.EINVAL
    assert lib.tpcfit_create(None, 0.5, None) == tpcfit.EINVAL
    # bad geometry: wrong sector count, non-ascending rows
    rx = (C.c_double * 3)(85.0, 84.0, 86.0)
    g = tpcfit._Geometry(36, 3, C.cast(rx, C.POINTER(C.c_double)), 20.0, 250.0)
    assert lib.tpcfit_create(C.byref(g), 0.5, C.byref(h)) == tpcfit.EINVAL
    g = tpcfit._Geometry(35, 3, C.cast(rx, C.POINTER(C.c_double)), 20.0, 250.0)
    assert lib.tpcfit_create(C.byref(g), 0.5, C.byref(h)) == tpcfit.EINVAL
    # the other geometry rules: 1..152 rows at positive ascending x, 20-degree
    # sectors (18 per side cover the circle), a finite field
    good = (C.c_double * 153)(*[85.0 + i for i in range(153)])
    gp = C.cast(good, C.POINTER(C.c_double))
    for n_rows, width, bz in ((0, 20.0, 0.5), (153, 20.0, 0.5), (152, 10.0, 0.5), (152, 20.5, 0.5),
                              (152, 20.0, float("nan")), (152, 20.0, float("inf"))):
        g = tpcfit._Geometry(36, n_rows, gp, width, 250.0)
        assert lib.tpcfit_create(C.byref(g), bz, C.byref(h)) == tpcfit.EINVAL, (n_rows, width, bz)
    neg = (C.c_double * 2)(-1.0, 85.0)
    g = tpcfit._Geometry(36, 2, C.cast(neg, C.POINTER(C.c_double)), 20.0, 250.0)
    assert lib.tpcfit_create(C.byref(g), 0.5, C.byref(h)) == tpcfit.EINVAL
    assert lib.tpcfit_rtc_build(C.byref(tpcfit._Geometry(36, 152, gp, 10.0, 250.0)), 0.5, 0, 4, 24, 0, 0,
                                None) == tpcfit.EINVAL
    # null handle everywhere
    assert lib.tpcfit_set_mode(None, 1) == tpcfit.EINVAL
    assert lib.tpcfit_set_config(None, 1, 4, 8, 1) == tpcfit.EINVAL
    assert lib.tpcfit_reserve(None, 10, 10) == tpcfit.EINVAL
    assert lib.tpcfit_set_det_reduction(None, 0) == tpcfit.EINVAL
    assert lib.tpcfit_fit(None, None, None, 0, None, None, None, None, None, None) == tpcfit.EINVAL
    assert lib.tpcfit_get_status(None, None, None, None) == tpcfit.EINVAL
    assert lib.tpcfit_fit_host(None, None, None, None, 0, None, 1, None, None, None, None, None, None) == tpcfit.EINVAL
    assert lib.tpcfit_fit_adjoint_host(None, None, None, None, 0, None, 1, None, None, None, None, None, None,
                                       None) == tpcfit.EINVAL
    lib.tpcfit_destroy(None)


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "tpcfit.h"

int main(void) {
  double rx[3] = {85.0, 84.0, 86.0};          /* not ascending: rejected */
  tpcfit_geometry g = {36, 3, rx, 20.0, 250.0};
  tpcfit_handle* h = NULL;
  if (tpcfit_version() < 10000) return 1;
  if (strcmp(tpcfit_status_string(TPCFIT_OK), "ok") != 0) return 2;
  if (tpcfit_create(&g, 0.5, &h) != TPCFIT_EINVAL || h != NULL) return 3;
  if (tpcfit_create(NULL, 0.5, &h) != TPCFIT_EINVAL) return 4;
  if (tpcfit_set_mode(NULL, 1) != TPCFIT_EINVAL) return 5;
  if (tpcfit_fit(NULL, NULL, NULL, 0, NULL, NULL, NULL, NULL, NULL, NULL) != TPCFIT_EINVAL) return 6;
  tpcfit_destroy(NULL);
  printf("c client ok\n");
  return 0;
}
"""


def test_header_compiles_as_c_and_links(lib, tmp_path):
    # a plain C99 client: the header needs no C++ and no CUDA header, and the
    # library links and answers without a GPU
    import shutil
    from paper_2511_17018_gb300 import tpcfit
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "client"
    libdir = os.path.dirname(tpcfit.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", f"-I{os.path.join(ROOT, 'include')}",
                    str(src), "-o", str(exe), f"-L{libdir}", "-ltpcfit", f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and "c client ok" in r.stdout, (r.returncode, r.stdout, r.stderr)
