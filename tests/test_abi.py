"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
entry point that include/rpr.h declares, the Python binding declares exactly those,
and the ctypes mirrors of the structs have the C layout (compared against gcc)."""
import os
import re
import subprocess
import tempfile

import pytest

from paper_1803_00430_gb300 import build as cuda_build
from paper_1803_00430_gb300 import rpr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rpr.h")


def _declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(rp_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return rpr.load()


def test_library_exports_every_declared_entry_point(lib):
    declared = _declared_functions()
    assert len(declared) >= 15
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(rpr.exported_symbols()) == declared


def test_status_strings(lib):
    for code in rpr.STATUS:
        assert lib.rp_status_string(code)
    assert lib.rp_status_string(-4) == b"internal buffer capacity exceeded"


def test_struct_layout_matches_c(lib):
    structs = ["rp_mesh_desc", "rp_scene_info", "rp_trace_params", "rp_direct", "rp_trace_stats",
               "rp_estimate_params", "rp_reverb_params", "rp_kernel_time", "rp_debug_limits", "rp_batch_item",
               "rp_batch_tuning", "rp_batch_info", "rp_mlp_config"]
    fields = {s: [f[0] for f in getattr(rpr, s)._fields_] for s in structs}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for s, fs in fields.items():
        lines.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            lines.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("return 0;}")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-std=c11", c, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    import ctypes as C
    for line in out:
        if not line:
            continue
        name, val = line.split()
        if "." in name:
            s, f = name.split(".")
            assert getattr(getattr(rpr, s), f).offset == int(val), name
        else:
            assert C.sizeof(getattr(rpr, name)) == int(val), name


def test_create_without_device_fails_cleanly(lib):
    import ctypes as C
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.rp_create(C.byref(h), 0, None) == rpr.RP_ERR["RP_ERR_NO_DEVICE"]
    assert lib.rp_sync_status(None) == rpr.RP_ERR["RP_ERR_INVALID_ARG"]
    assert lib.rp_trace(None, None, None, None, 0, None, None, None, None) == rpr.RP_ERR["RP_ERR_INVALID_ARG"]
    assert lib.rp_set_debug_limits(None, None) == rpr.RP_ERR["RP_ERR_INVALID_ARG"]


def test_bounds_checked_build_compiles_and_exports_the_same_entry_points():
    import ctypes as C
    path = cuda_build.build(checked=True)
    assert path.endswith(os.path.join("checked", "librpr.so"))
    lib2 = C.CDLL(path)
    missing = [n for n in _declared_functions() if not hasattr(lib2, n)]
    assert not missing, missing
