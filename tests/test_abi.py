"""The C-ABI library builds, loads and exports every symbol include/glm.h declares.

These tests make no compute call: they run on a machine without a GPU.
"""
import os
import re

import pytest

import paper_1310_1537_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^GLM_API\s+[\w\s\*]+?\b(glm_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_loads_and_exports_every_declared_symbol():
    lib = pkg.load()
    declared = _declared_symbols()
    assert {"glm_create", "glm_logpost_grad", "glm_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(pkg.EXPORTS)


def test_library_has_no_cuda_runtime_or_torch_dependency():
    import subprocess
    out = subprocess.run(["ldd", pkg.LIB_PATH], capture_output=True, text=True).stdout
    assert "libcudart" not in out and "libtorch" not in out and "libc10" not in out


def test_status_strings():
    assert pkg.glm_status_str(0) == "ok"
    assert pkg.glm_status_str(pkg.GLM_ERR_TIMEOUT) == "device wait timed out"
    assert pkg.glm_status_str(99) == "unknown status"


def test_create_rejects_bad_descriptors_without_touching_a_device():
    import ctypes as C
    lib = pkg.load()
    h = C.c_void_p()
    assert lib.glm_create(None, C.byref(h)) == pkg.GLM_ERR_INVALID_ARG
    bad = [
        dict(n_rows=-1, p=4, ld=4, k_max=1, xtype=0),
        dict(n_rows=10, p=0, ld=4, k_max=1, xtype=0),
        dict(n_rows=10, p=5, ld=4, k_max=1, xtype=0),      # ld < p
        dict(n_rows=10, p=5, ld=5, k_max=1, xtype=0),      # 20-byte rows
        dict(n_rows=10, p=5, ld=6, k_max=1, xtype=1),      # 12-byte rows
        dict(n_rows=10, p=5, ld=8, k_max=1, xtype=2),      # 8-byte rows
        dict(n_rows=10, p=4, ld=4, k_max=0, xtype=0),
        dict(n_rows=10, p=4, ld=4, k_max=1, xtype=7),
    ]
    for b in bad:
        d = pkg.glm_desc_t(b["n_rows"], b["p"], b["ld"], b["k_max"], b["xtype"], 10.0, 0, 0)
        assert lib.glm_create(C.byref(d), C.byref(h)) == pkg.GLM_ERR_INVALID_ARG, b
        assert h.value is None
    d = pkg.glm_desc_t(10, 4, 4, 1, 0, -1.0, 0, 0)
    assert lib.glm_create(C.byref(d), C.byref(h)) == pkg.GLM_ERR_INVALID_ARG


def test_entry_points_reject_null_handle():
    lib = pkg.load()
    assert lib.glm_logpost_grad(None, None, None, None, None, 1, None, None, None) == 1
    assert lib.glm_sync(None, None) == 1
    assert lib.glm_destroy(None) == 0


@pytest.mark.skipif(__import__("tests.conftest", fromlist=["gpu_available"]).gpu_available(),
                    reason="checks the no-device path")
def test_create_without_device_reports_no_device():
    try:
        pkg.glm_create(100, 4, 4, 1)
    except pkg.GLMError as e:
        assert e.status == pkg.GLM_ERR_NO_DEVICE
    else:
        pytest.fail("glm_create succeeded without a device")


def test_server_rejects_bad_descriptors_and_null_arguments():
    import ctypes as C
    lib = pkg.load()
    s = C.c_void_p()
    assert lib.glm_server_create(None, C.byref(s)) == pkg.GLM_ERR_INVALID_ARG
    for b in [(0, 0, 8, 16, 0), (0, 17, 8, 16, 0), (0, 2, 0, 16, 0), (0, 2, 1025, 16, 0),
              (0, 2, 8, 0, 0), (0, 2, 8, 16, -1), (-1, 2, 8, 16, 0)]:
        d = pkg.glm_server_desc_t(*b)
        assert lib.glm_server_create(C.byref(d), C.byref(s)) == pkg.GLM_ERR_INVALID_ARG, b
        assert s.value is None
    rid = C.c_uint64()
    ds = C.c_int32()
    assert lib.glm_server_submit(None, 0, None, 1, C.byref(rid)) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_server_add_dataset(None, None, None, None, 1, 1, 4, 0, 10.0,
                                      C.byref(ds)) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_server_poll(None, 1, None, None, None) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_server_stats(None, None) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_server_remove_dataset(None, 0) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_server_destroy(None) == pkg.GLM_OK
    assert pkg.glm_status_str(pkg.GLM_PENDING) == "pending"


@pytest.mark.skipif(__import__("tests.conftest", fromlist=["gpu_available"]).gpu_available(),
                    reason="checks the no-device path")
def test_server_without_device_reports_no_device():
    with pytest.raises(pkg.GLMError) as e:
        pkg.glm_server_create(0, 2, 8, 16)
    assert e.value.status == pkg.GLM_ERR_NO_DEVICE


def test_slice_sampler_rejects_bad_descriptors_without_a_device():
    import ctypes as C
    lib = pkg.load()
    s = C.c_void_p()
    assert lib.glm_slice_create(None, C.byref(s)) == pkg.GLM_ERR_INVALID_ARG
    good = dict(n_rows=1000, ld=1000, p=5, m=4, s_max=30, device=0, w=1.0, spec=0,
                prior_sigma=10.0)
    bad = [dict(n_rows=0), dict(ld=999), dict(ld=1002), dict(p=0), dict(m=0), dict(m=17),
           dict(s_max=0), dict(s_max=65), dict(w=0.0), dict(w=float("inf")),
           dict(prior_sigma=0.0), dict(device=-1), dict(spec=-1), dict(spec=17)]
    for b in bad:
        d = dict(good, **b)
        desc = pkg.glm_slice_desc_t(d["n_rows"], d["ld"], d["p"], d["m"], d["s_max"],
                                    d["device"], d["w"], d["spec"], d["prior_sigma"])
        assert lib.glm_slice_create(C.byref(desc), C.byref(s)) == pkg.GLM_ERR_INVALID_ARG, b
        assert s.value is None
    assert lib.glm_slice_run(None, None, None, None, None, None, 0, 0, None, None, None, None,
                             None, None) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_slice_destroy(None) == pkg.GLM_OK


def test_ising_entry_points_reject_bad_arguments_without_a_device():
    lib = pkg.load()
    # null pointers, odd or too-small sizes, bad element size: refused before
    # any device call
    assert lib.glm_ising_sweeps(None, None, None, None, 4, 8, 1.0, 1, None, None, None) == \
        pkg.GLM_ERR_INVALID_ARG
    for rows, cols, eb in [(0, 8, 1), (4, 7, 1), (4, 0, 1), (4, 8, 2)]:
        assert lib.glm_ising_split(1, eb, rows, cols, 1, 1, None) == pkg.GLM_ERR_INVALID_ARG
        assert lib.glm_ising_merge(1, 1, eb, rows, cols, 1, None) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_ising_sweeps(16, 16, 16, 16, 4, 8, 1.0, -1, 16, None, None) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_ising_sweeps(16, 16, 16, 16, 4, 8, float("nan"), 1, 16, None, None) == \
        pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_ising_sweeps(16, 16, 16, 16, 4, 8, 1.0, 1, 16, 12, None) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_ising_sweeps(16, 16, 16, 16, 4, 8, 1.0, 0, None, None, None) == pkg.GLM_OK


def test_hessian_evaluator_rejects_bad_shapes_without_a_device():
    import ctypes as C
    lib = pkg.load()
    h = C.c_void_p()
    for n, p, ld, s in [(-1, 4, 4, 1.0), (10, 0, 4, 1.0), (10, 65, 68, 1.0), (10, 8, 6, 1.0),
                        (10, 8, 4, 1.0), (10, 8, 68, 1.0), (10, 8, 8, 0.0), (10, 8, 8, float("inf"))]:
        assert lib.glm_hess_create(n, p, ld, s, 0, C.byref(h)) == pkg.GLM_ERR_INVALID_ARG
        assert h.value is None
    assert lib.glm_hess_create(10, 8, 8, 1.0, 0, None) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_hess_eval(None, None, None, None, None, None, None, None) == pkg.GLM_ERR_INVALID_ARG
    assert lib.glm_hess_destroy(None) == pkg.GLM_OK


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every structure the binding mirrors has the header's size and field
    offsets, as a C compiler lays them out."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [pkg.glm_desc_t, pkg.glm_info_t, pkg.glm_server_desc_t, pkg.glm_request_info_t,
               pkg.glm_server_stats_t, pkg.glm_slice_desc_t]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "glm.h"', 'int main(void) {']
    for st in structs:
        t = st.__name__
        lines.append(f'printf("{t} size %zu\\n", sizeof({t}));')
        for name, _ in st._fields_:
            lines.append(f'printf("{t} {name} %zu\\n", offsetof({t}, {name}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(line.rsplit(" ", 1) for line in
               subprocess.run([str(exe)], capture_output=True, text=True, check=True)
               .stdout.splitlines())
    for st in structs:
        t = st.__name__
        assert int(got[f"{t} size"]) == C_sizeof(st), t
        for name, _ in st._fields_:
            assert int(got[f"{t} {name}"]) == getattr(st, name).offset, (t, name)


def C_sizeof(st):
    import ctypes
    return ctypes.sizeof(st)
