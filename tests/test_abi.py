"""The C-ABI library builds, loads without a GPU, and exports every function
include/asp.h declares, with a matching ctypes declaration in the binding."""
import ctypes
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "asp.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(asp_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1606_07872_gb300 import build
    return build.build()


def test_header_declares_the_paper_calls():
    names = _declared()
    for must in ("asp_init", "asp_find_peak", "asp_fit_active_set", "asp_subtract", "asp_minor_cycle"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (asp_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_declares_every_symbol(libpath):
    from paper_1606_07872_gb300 import _lib
    lib = _lib.load(libpath)
    for n in _declared():
        assert n in _lib.SIGNATURES, n
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr)


def test_struct_sizes_match_header(libpath):
    """Layout of the public structs as the C compiler sees them."""
    from paper_1606_07872_gb300 import _lib
    src = f"""
#include <stdio.h>
#include "asp.h"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(asp_gauss), sizeof(asp_component),
         sizeof(asp_peak), sizeof(asp_fit_info), sizeof(asp_params), sizeof(asp_cycle_stats),
         sizeof(asp_iter_record), sizeof(asp_batch_tuning), sizeof(asp_kernel_time), sizeof(asp_alu_peaks),
         sizeof(asp_gauss_ell), sizeof(asp_component_ell));
  return 0;
}}
"""
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    mine = [ctypes.sizeof(t) for t in (_lib.asp_gauss, _lib.asp_component, _lib.asp_peak, _lib.asp_fit_info,
                                       _lib.asp_params, _lib.asp_cycle_stats, _lib.asp_iter_record,
                                       _lib.asp_batch_tuning, _lib.asp_kernel_time, _lib.asp_alu_peaks,
                                       _lib.asp_gauss_ell, _lib.asp_component_ell)]
    assert sizes == mine


def test_default_params_and_status_strings(libpath):
    import paper_1606_07872_gb300 as m
    p = m.default_params()
    assert p.gain == pytest.approx(0.35) and p.k_max == 5 and p.lm_max_iter == 50 and p.n_scales == 6
    assert p.area_frac == pytest.approx(0.05)
    assert m.lib().asp_status_string(0) == b"ok"


def test_null_and_bad_arguments_rejected_without_gpu(libpath):
    import paper_1606_07872_gb300 as m
    L = m.lib()
    h = ctypes.c_void_p()
    p = m.default_params(k_max=0)
    assert L.asp_init(ctypes.byref(p), 8, 8, None, None, None, ctypes.byref(h)) == 1
    p = m.default_params(k_max=m.ASP_KMAX + 1)
    assert L.asp_init(ctypes.byref(p), 8, 8, 1, 1, None, ctypes.byref(h)) == 8
    assert L.asp_destroy(None) == 1
    assert L.asp_minor_cycle(None, 1, None) == 1


def test_binding_constants_match_header():
    """Every #define of include/asp.h that the binding mirrors has the same
    value there."""
    from paper_1606_07872_gb300 import _lib
    defs = dict(re.findall(r"#define\s+(ASP_[A-Z_0-9]+)\s+(\d+)", open(HEADER).read()))
    assert defs, "no numeric #define found"
    for name, val in defs.items():
        assert hasattr(_lib, name), name
        assert getattr(_lib, name) == int(val), name
