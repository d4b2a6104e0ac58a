"""The C-ABI library builds, loads and exports every entry point that
include/gcp.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gcp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gcp_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1906_01687_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gcp_sample", "gcp_grad", "gcp_loss_est", "gcp_adam_step"):
        assert required in names


def test_library_exports_every_declared_function(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (gcp_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported


def test_binding_covers_every_declared_function(lib_path):
    from paper_1906_01687_gb300 import gcp
    assert set(declared_functions()) == set(gcp.EXPORTED)


def test_host_side_validation_without_gpu(lib_path):
    """Pure host calls: status strings, sample counts, invalid arguments."""
    from paper_1906_01687_gb300 import gcp
    assert "invalid" in gcp._lib.gcp_status_string(gcp.ERR_INVALID_ARG).decode()
    assert gcp.Sampling(gcp.SAMPLER_UNIFORM, 0, 1000, 1).count() == 1000
    assert gcp.Sampling(gcp.SAMPLER_STRATIFIED, 300, 700, 1).count() == 1000
    assert gcp.Sampling(9, 3, 4, 1).count() == -1
    # a NULL tensor descriptor is rejected before any CUDA call
    h = ctypes.c_void_p()
    assert gcp._lib.gcp_create(ctypes.byref(h), None, None) == gcp.ERR_INVALID_ARG
    t = gcp.gcp_tensor()
    t.d = 0
    assert gcp._lib.gcp_create(ctypes.byref(h), ctypes.byref(t), None) == gcp.ERR_INVALID_ARG
    t.d = 9
    assert gcp._lib.gcp_create(ctypes.byref(h), ctypes.byref(t), None) == gcp.ERR_INVALID_ARG
    # one mode: rejected (Eq. (4.3) has no leave-one-out product), even with a valid-looking descriptor
    buf = (ctypes.c_float * 50)()
    t.d, t.dims[0], t.vals = 1, 50, ctypes.addressof(buf)
    assert gcp._lib.gcp_create(ctypes.byref(h), ctypes.byref(t), None) == gcp.ERR_INVALID_ARG
    assert gcp._lib.gcp_state_init(None, ctypes.c_float(0.1), None) == gcp.ERR_INVALID_ARG


def test_struct_layouts_match_header():
    from paper_1906_01687_gb300 import gcp
    assert ctypes.sizeof(gcp.gcp_tensor) == 160
    assert ctypes.sizeof(gcp.gcp_factors) == 144
    assert ctypes.sizeof(gcp.gcp_sampling) == 56
    assert ctypes.sizeof(gcp.gcp_samples) == 96
    assert ctypes.sizeof(gcp.gcp_adam_params) == 24
    assert ctypes.sizeof(gcp.gcp_epoch_params) == 16
    assert ctypes.sizeof(gcp.gcp_tuning) == 44
    assert ctypes.sizeof(gcp.gcp_launch_info) == 68


def test_ctypes_layouts_match_the_c_compiler(tmp_path):
    """Every struct of include/gcp.h has the same size in C (gcc) and in the binding."""
    from paper_1906_01687_gb300 import gcp
    names = ["gcp_tensor", "gcp_factors", "gcp_sampling", "gcp_samples", "gcp_adam_params", "gcp_epoch_params",
             "gcp_adam_state", "gcp_tuning", "gcp_launch_info", "gcp_batch_problem"]
    src = tmp_path / "sizes.c"
    src.write_text('#include "gcp.h"\n#include <stdio.h>\nint main(void){\n' +
                   "".join(f'printf("%zu\\n", sizeof({n}));\n' for n in names) + "return 0;}\n")
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    sizes = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    for n, size in zip(names, sizes):
        if hasattr(gcp, n):
            assert ctypes.sizeof(getattr(gcp, n)) == size, n
    assert dict(zip(names, sizes))["gcp_adam_state"] == 64
