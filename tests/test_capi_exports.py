"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/aqs.h declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "aqs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(aqs_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libaqs():
    from paper_2507_20802_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary_calls():
    names = _declared_functions()
    for required in ["aqs_create_system", "aqs_affine_shear", "aqs_minimize",
                     "aqs_parallel_step", "aqs_compare_configs"]:
        assert required in names


def test_library_exports_every_declared_symbol(libaqs):
    missing = [n for n in _declared_functions() if not hasattr(libaqs, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2507_20802_gb300 import aqs
    assert sorted(aqs._SIGS) == _declared_functions()


def test_defaults_and_error_path_without_gpu(libaqs):
    """Pure host entry points work on a machine without a GPU."""
    from paper_2507_20802_gb300 import aqs
    f = aqs.aqs_fire_params()
    aqs.lib().aqs_fire_params_default(ctypes.byref(f))
    assert f.dt0 == 0.005 and f.alpha0 == 0.1 and f.f_inc == 1.1 and f.f_dec == 0.5
    assert f.tol == 1e-10
    # invalid arguments are rejected before any device work
    h = ctypes.c_void_p()
    st = aqs.lib().aqs_create_system(None, ctypes.byref(h))
    assert st == aqs.AQS_ERR_INVALID_ARG
    assert b"null" in aqs.lib().aqs_last_error()


def test_struct_layouts_match_header():
    """sizeof of the ctypes mirrors equals the C layout (checked by compiling
    a probe with the host compiler)."""
    import subprocess
    import tempfile
    from paper_2507_20802_gb300 import aqs
    src = r'''
#include <stdio.h>
#include "aqs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(aqs_potential), sizeof(aqs_system_desc),
         sizeof(aqs_fire_params), sizeof(aqs_min_result), sizeof(aqs_parallel_params),
         sizeof(aqs_parallel_result), sizeof(aqs_kernel_stats));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                                check=True).stdout.split()]
    mine = [ctypes.sizeof(t) for t in (aqs.aqs_potential, aqs.aqs_system_desc,
                                       aqs.aqs_fire_params, aqs.aqs_min_result,
                                       aqs.aqs_parallel_params, aqs.aqs_parallel_result,
                                       aqs.aqs_kernel_stats)]
    assert sizes == mine
