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
    assert ctypes.sizeof(gcp.gcp_tuning) == 56
    assert ctypes.sizeof(gcp.gcp_launch_info) == 80


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


def _no_gpu():
    try:
        import torch
        return not torch.cuda.is_available()
    except ImportError:
        return True


@pytest.mark.skipif(not _no_gpu(), reason="hands the library fake device addresses: CPU-only machines")
def test_invalid_descriptors_rejected_before_any_launch(lib_path):
    """Each call gets one invalid field (all else well-formed, with fake but
    aligned device addresses that nothing dereferences) and must return
    GCP_ERR_INVALID_ARG from its host-side checks.  Without a GPU a call
    that got past them would fail in CUDA instead (GCP_ERR_CUDA)."""
    from paper_1906_01687_gb300 import gcp
    lib, BAD = gcp._lib, gcp.ERR_INVALID_ARG
    base = 1 << 20
    dims3 = (ctypes.c_int64 * 3)(4, 5, 6)

    def factors(rank=3, ld=4, misalign=0):
        F = gcp.gcp_factors()
        F.rank, F.ld = rank, ld
        for k in range(3):
            F.A[k] = base * (k + 1) + misalign
        return F

    def p8(offset=0, null_mode=None):
        a = gcp._P8()
        for k in range(3):
            a[k] = None if k == null_mode else base * (10 + k) + offset
        return a

    prm = gcp.gcp_adam_params(0.9, 0.999, 1e-8, float("-inf"), 1, 0)
    state = ctypes.c_void_p(base * 50)

    def adam(F=None, d=3, dims=dims3, G=None, prm_=prm, st=state):
        return lib.gcp_adam_step(ctypes.byref(F or factors()), d, dims, G or p8(), p8(), p8(), ctypes.byref(prm_), st,
                                 None)

    assert adam() == gcp.ERR_CUDA  # the control: well-formed, so it reaches CUDA, which has no device here
    assert adam(d=0) == BAD and adam(d=9) == BAD
    assert adam(F=factors(rank=0)) == BAD and adam(F=factors(rank=257, ld=260)) == BAD
    assert adam(F=factors(rank=5, ld=4)) == BAD and adam(F=factors(ld=6)) == BAD
    assert adam(F=factors(misalign=4)) == BAD  # rows must be 16-byte aligned
    assert adam(dims=(ctypes.c_int64 * 3)(4, 0, 6)) == BAD
    assert adam(dims=(ctypes.c_int64 * 3)(4, 2**31, 6)) == BAD
    assert adam(G=p8(null_mode=1)) == BAD and adam(G=p8(offset=8)) == BAD
    assert adam(prm_=gcp.gcp_adam_params(1.0, 0.999, 1e-8, 0.0, 1, 0)) == BAD
    assert adam(prm_=gcp.gcp_adam_params(0.9, -0.1, 1e-8, 0.0, 1, 0)) == BAD
    assert adam(prm_=gcp.gcp_adam_params(0.9, 0.999, -1.0, 0.0, 1, 0)) == BAD
    assert adam(st=ctypes.c_void_p(base * 50 + 4)) == BAD and adam(st=None) == BAD
    # a factor set of 2^31 float4 chunks or more
    assert adam(dims=(ctypes.c_int64 * 3)(2**31 - 1, 2**31 - 1, 4), F=factors(rank=8, ld=8)) == BAD

    ep = gcp.gcp_epoch_params(10, 0.1, 1)
    assert lib.gcp_epoch_end(ctypes.byref(factors()), 3, dims3, p8(), p8(), p8(), p8(), p8(),
                             ctypes.byref(gcp.gcp_epoch_params(-1, 0.1, 1)), state, None) == BAD
    assert lib.gcp_epoch_end(ctypes.byref(factors()), 3, dims3, p8(), p8(), p8(), p8(), p8(),
                             ctypes.byref(gcp.gcp_epoch_params(10, 0.1, -1)), state, None) == BAD
    assert lib.gcp_epoch_end(ctypes.byref(factors()), 3, dims3, p8(), p8(), p8(), p8(), p8(null_mode=2),
                             ctypes.byref(ep), state, None) == BAD
    assert lib.gcp_state_init(ctypes.c_void_p(base + 4), ctypes.c_float(0.1), None) == BAD

    # the handle-free loss estimate
    L = gcp.gcp_samples()
    L.n = 100
    for k in range(3):
        L.idx[k] = base * (20 + k)
    L.x, L.w, L.cls = base * 30, base * 31, base * 32
    out = ctypes.c_void_p(base * 40)

    def noalloc(d=3, F=None, loss=0, L_=L, out_=out):
        return lib.gcp_loss_est_noalloc(d, ctypes.byref(F or factors()), loss, ctypes.byref(L_), out_, None)

    assert noalloc() == gcp.ERR_CUDA
    assert noalloc(d=0) == BAD and noalloc(d=1) == BAD and noalloc(loss=7) == BAD and noalloc(loss=-1) == BAD
    assert noalloc(F=factors(ld=3)) == BAD and noalloc(out_=ctypes.c_void_p(base * 40 + 4)) == BAD
    L2 = gcp.gcp_samples.from_buffer_copy(L)
    L2.n = 262_145  # more than one entry per thread of 1024 blocks of 256
    assert noalloc(L_=L2) == BAD
    L3 = gcp.gcp_samples.from_buffer_copy(L)
    L3.idx[2] = None
    assert noalloc(L_=L3) == BAD

    # handles and batches
    assert lib.gcp_profile(None, 1, 16) == BAD
    assert lib.gcp_refresh(None, None) == BAD
    spec = gcp.Sampling(gcp.SAMPLER_UNIFORM, 0, 10, 1)._c()
    assert lib.gcp_grad_range(None, ctypes.byref(factors()), 0, ctypes.byref(spec), 0, 5, None, p8(), None) == BAD
    assert lib.gcp_set_tuning(None, None) == BAD
    assert lib.gcp_get_device_status(None, None) == BAD
    b = ctypes.c_void_p()
    assert lib.gcp_batch_create(ctypes.byref(b), None, 1, None) == BAD
    probs = (gcp.gcp_batch_problem * 1)()
    assert lib.gcp_batch_create(ctypes.byref(b), probs, 0, None) == BAD
    assert lib.gcp_batch_create(ctypes.byref(b), probs, 1025, None) == BAD
    assert lib.gcp_batch_create(ctypes.byref(b), probs, 1, None) == BAD  # an all-zero problem: d = 0


def header_prototypes():
    """{name: [parameter declarations]} of every function include/gcp.h declares."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"\b([a-z_0-9]+\s*\**)\s*\b(gcp_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        params = [p.strip() for p in m.group(3).replace("\n", " ").split(",")]
        protos[m.group(2)] = [] if params == ["void"] else params
        RETURNS[m.group(2)] = m.group(1).replace(" ", "")
    return protos


RETURNS = {}


def test_binding_signatures_follow_the_header(lib_path):
    """Every ctypes signature has the header's parameter count, and each
    parameter the ctypes type its C type calls for."""
    from paper_1906_01687_gb300 import gcp
    P = ctypes.POINTER
    protos = header_prototypes()
    assert set(protos) == set(gcp._SIGS)

    def expected(decl):
        decl = re.sub(r"\bconst\b", "", decl)
        decl = re.sub(r"\s+", " ", decl).strip()
        ty = decl.rsplit(" ", 1)[0] if not decl.endswith("]") else decl.split("[")[0].rsplit(" ", 1)[0]
        if decl.endswith("[GCP_MAX_MODES]"):
            return {gcp._P8}
        stars = decl.count("*")
        base = ty.replace("*", "").strip()
        if stars == 2:
            return {P(ctypes.c_void_p)}
        if stars == 1:
            structs = {"gcp_factors": gcp.gcp_factors, "gcp_sampling": gcp.gcp_sampling,
                       "gcp_samples": gcp.gcp_samples, "gcp_adam_params": gcp.gcp_adam_params,
                       "gcp_epoch_params": gcp.gcp_epoch_params, "gcp_tensor": gcp.gcp_tensor,
                       "gcp_tuning": gcp.gcp_tuning, "gcp_launch_info": gcp.gcp_launch_info,
                       "gcp_batch_problem": gcp.gcp_batch_problem}
            if base in structs:
                return {P(structs[base])}
            if base in ("int32_t",):
                return {P(ctypes.c_int32), ctypes.c_void_p}
            if base in ("int64_t",):
                return {P(ctypes.c_int64), ctypes.c_void_p}
            if base == "double":
                return {P(ctypes.c_double), ctypes.c_void_p}
            return {ctypes.c_void_p}  # opaque handles, device buffers, the optimizer state
        scalars = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "float": ctypes.c_float,
                   "gcp_loss": ctypes.c_int, "gcp_status": ctypes.c_int, "gcp_stream_t": ctypes.c_void_p,
                   "uint64_t": ctypes.c_uint64}
        return {scalars[base]}

    ret = {"gcp_status": {ctypes.c_int}, "int64_t": {ctypes.c_int64}, "int32_t": {ctypes.c_int32},
           "char*": {ctypes.c_char_p}}
    for name, params in protos.items():
        args, res = gcp._SIGS[name]
        assert res in ret[RETURNS[name]], f"{name} returns {RETURNS[name]}, bound as {res}"
        assert len(args) == len(params), name
        for k, (decl, got) in enumerate(zip(params, args)):
            assert got in expected(decl), f"{name} parameter {k} ({decl}): {got}"


def test_c_example_compiles():
    """The C example (examples/fit_dense.c) is valid C11 against include/gcp.h."""
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "examples", "fit_dense.c")])
