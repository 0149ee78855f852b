"""The C ABI library loads and exports every entry point include/*.h declares.

CPU only: no call here reaches the GPU.
"""
import ctypes
import glob
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names.update(re.findall(r"^ULP_API\s+[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2203_13675_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["unwrap_lp", "ulp_plan_create", "ulp_unwrap", "ulp_unwrap_batched", "ulp_plan_destroy",
                 "ulp_last_error", "ulp_weights", "ulp_matvec", "ulp_precond_apply", "ulp_pcg",
                 "ulp_wrapped_diffs"]:
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), f"{name} declared but not exported"


def test_only_declared_symbols_are_exported(lib):
    from paper_2203_13675_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported <= _declared() | {"_init", "_fini"}, exported - _declared()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc missing")
def test_header_compiles_as_c_and_cpp(tmp_path):
    src = tmp_path / "t.c"
    src.write_text('#include "unwrap_lp.h"\nint main(void){ulp_options o; ulp_options_default(&o); return o.stop_mode;}\n')
    for std in (["gcc", "-std=c99"], ["g++", "-x", "c++", "-std=c++17"]):
        subprocess.check_call([*std, "-fsyntax-only", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                               str(src)])


def test_binding_names_match_abi():
    from paper_2203_13675_gb300 import native
    assert set(native.EXPORTED) == _declared()


def test_host_side_validation_without_gpu(lib):
    # argument checks that fail before any CUDA call
    from paper_2203_13675_gb300 import native
    L = native.load()
    h = ctypes.c_void_p()
    assert L.ulp_plan_create(1, 5, None, ctypes.byref(h)) == native.ULP_ERR_INVALID
    assert b"H=1" in L.ulp_last_error()
    assert L.unwrap_lp(None, 4, 4, 1.0, 0.01, 1, 1e-6, 5, 0, None) == native.ULP_ERR_INVALID
    o = native.ulp_options_default()
    assert o.stop_mode == 0 and o.outer_tol == 1e-6 and o.omega == 1.0 and o.spin_timeout_s == 2.0
