"""CPU checks of the C ABI: the library builds, loads, exports every function
include/crk.h declares, and the binding's structures have the header's
layout.  No compute call is made (there is no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2510_03557_gb300 import build as build_mod

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "crk.h")


@pytest.fixture(scope="module")
def libcrk():
    build_mod.build()
    from paper_2510_03557_gb300 import crk

    return crk


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(crk_[a-z_]+)\s*\(", src)))


def test_header_declares_the_abi(libcrk):
    names = _declared_functions()
    assert set(names) == set(libcrk.ABI)


def test_library_exports_every_declared_symbol(libcrk):
    L = libcrk.lib()
    for name in _declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libcrk.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (crk_[a-z_]+)", out))
    assert set(_declared_functions()) <= exported


def test_error_message_is_available_without_gpu(libcrk):
    assert isinstance(libcrk.crk_last_error(), str)


STRUCTS = (("crk_physics", "Physics"), ("crk_params", "Params"), ("crk_outputs", "Outputs"),
           ("crk_timings", "Timings"), ("crk_service_params", "ServiceParams"), ("crk_job", "Job"),
           ("crk_job_snapshot", "JobSnapshot"), ("crk_job_result", "JobResult"), ("crk_tree", "Tree"))


def test_struct_layouts_match_header(libcrk, tmp_path):
    """Every field of every binding structure exists in the header's struct
    under the same name, at the same offset and with the same size, and the
    structs have the same size: gcc's layout of the header against ctypes'."""
    lines = []
    for cname, pyname in STRUCTS:
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f in getattr(libcrk, pyname)._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu %zu\\n", offsetof({cname}, {f[0]}), '
                         f"sizeof((({cname} *)0)->{f[0]}));")
    prog = tmp_path / "layout.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "crk.h"\nint main(void){\n'
                    + "\n".join(lines) + "\nreturn 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    want = []
    for cname, pyname in STRUCTS:
        cls = getattr(libcrk, pyname)
        want.append(f"{cname} sizeof {ctypes.sizeof(cls)}")
        for f in cls._fields_:
            d = getattr(cls, f[0])
            want.append(f"{cname} {f[0]} {d.offset} {d.size}")
    assert got == want


def test_binding_has_every_header_struct_field(libcrk):
    """No header field is missing from the binding (names in order)."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for cname, pyname in STRUCTS:
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + cname + r"\s*;", src).group(1)
        names = re.findall(r"(\w+)\s*(?:\[[^\]]*\])?\s*[,;]", body)
        assert names == [f[0] for f in getattr(libcrk, pyname)._fields_], cname


def test_binding_rejects_mixed_memory_kinds(libcrk):
    import numpy as np

    with pytest.raises(TypeError):
        libcrk._mem_of(libcrk.CRK_MEM_HOST, libcrk.CRK_MEM_DEVICE)
    assert libcrk._mem_of(None, libcrk.CRK_MEM_HOST) == libcrk.CRK_MEM_HOST
    p, m, keep = libcrk._ptr(np.zeros(4), np.float64)
    assert m == libcrk.CRK_MEM_HOST and keep.dtype == np.float64


@pytest.mark.parametrize("pm_grid", [-2, 2, 7, 2048])
def test_create_rejects_bad_mesh_sizes_before_touching_the_device(libcrk, pm_grid):
    """pm_grid is 0 or an even number in [4, 1024]; the check runs before
    any CUDA call, so it answers here without a GPU."""
    p = libcrk.params(pm_grid=pm_grid)
    h = ctypes.c_void_p()
    rc = libcrk.lib().crk_create(ctypes.byref(p), None, ctypes.byref(h))
    assert rc == libcrk.CRK_EINVAL and "pm_grid" in libcrk.crk_last_error()


@pytest.mark.parametrize("field,value,word", [("leaf_cap", 48, "leaf_cap"), ("precision", 2, "precision"),
                                              ("kernel", 1, "kernel"), ("cm_level", 11, "cm_level"),
                                              ("cm_level", -1, "cm_level"),
                                              ("rebuild_every", -1, "rebuild_every"),
                                              ("flags", 1, "flags"), ("flags", 16, "flags"),
                                              ("graph_margin_pct", -1, "graph_margin_pct")])
def test_create_rejects_bad_params_before_touching_the_device(libcrk, field, value, word):
    """Every create-time parameter is checked before the first CUDA call."""
    p = libcrk.params()
    setattr(p, field, value)
    h = ctypes.c_void_p()
    rc = libcrk.lib().crk_create(ctypes.byref(p), None, ctypes.byref(h))
    assert rc == libcrk.CRK_EINVAL and word in libcrk.crk_last_error()


def test_null_arguments_are_rejected_without_a_device(libcrk):
    L = libcrk.lib()
    h = ctypes.c_void_p()
    assert L.crk_create(None, None, ctypes.byref(h)) == libcrk.CRK_EINVAL
    p = libcrk.params()
    assert L.crk_create(ctypes.byref(p), None, None) == libcrk.CRK_EINVAL
    assert L.crk_get_timings(None, None) == libcrk.CRK_EINVAL
    assert L.crk_get_tree(None, None) == libcrk.CRK_EINVAL
    assert L.crk_destroy(None) == libcrk.CRK_OK


@pytest.mark.parametrize("kw,word", [(dict(max_slots=0), "max_slots"), (dict(max_slots=70000), "max_slots"),
                                     (dict(hbm_budget_bytes=0), "hbm_budget_bytes"),
                                     (dict(snapshot_every=-1), "snapshot_every"),
                                     (dict(size_classes=-1), "size_classes"),
                                     (dict(size_classes=9), "size_classes"),
                                     (dict(lane_priority=2), "lane_priority")])
def test_service_create_rejects_bad_params_before_touching_the_device(libcrk, kw, word):
    args = dict(hbm_budget_bytes=1 << 30, max_slots=4)
    args.update(kw)
    with pytest.raises(libcrk.CrkError) as e:
        libcrk.crk_service_create(**args)
    assert e.value.code == libcrk.CRK_EINVAL and word in str(e.value)


def test_noalloc_argument_checks_without_a_device(libcrk):
    """The allocation-free entry point answers bad sizes, a bad box and null
    arrays (and n = 0) before any CUDA call."""
    f = libcrk.lib().crk_neighbours_noalloc
    i64, dbl = ctypes.c_int64, ctypes.c_double
    assert f(i64(-1), None, None, None, dbl(1.0), None, None, None) == libcrk.CRK_EINVAL
    assert f(i64(libcrk.CRK_NOALLOC_MAX_N + 1), None, None, None, dbl(1.0), None, None, None) == libcrk.CRK_EINVAL
    assert f(i64(8), None, None, None, dbl(0.0), None, None, None) == libcrk.CRK_EINVAL
    assert f(i64(8), None, None, None, dbl(1.0), None, None, None) == libcrk.CRK_EINVAL
    assert f(i64(0), None, None, None, dbl(1.0), None, None, None) == libcrk.CRK_OK


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    """There is no CPU fallback: with libcrk.so missing the binding raises
    instead of computing anything."""
    from paper_2510_03557_gb300 import crk

    monkeypatch.setattr(crk, "_lib", None)
    monkeypatch.setattr(crk, "LIB_PATH", str(tmp_path / "missing" / "libcrk.so"))
    with pytest.raises(ImportError):
        crk.lib()
    with pytest.raises(ImportError):
        crk.crk_create(crk.params())


def test_product_package_never_imports_the_oracle():
    """Only the tests, the smoke check and the bench's CPU legs may use the
    oracle: no module of the package names it."""
    pkg = os.path.join(ROOT, "paper_2510_03557_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath or "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "crk_oracle" not in src and "orc_" not in src, f


def test_oracle_never_uses_the_cuda_path():
    """The oracle shares no code with the CUDA path: it imports nothing of the
    package and loads none of its libraries."""
    odir = os.path.join(ROOT, "oracle")
    for f in os.listdir(odir):
        if f.endswith((".py", ".c", ".h")):
            src = open(os.path.join(odir, f)).read()
            assert "paper_2510_03557_gb300" not in src, f
            assert not re.search(r"libcrk\.so|crk_api|passes\.cu", src), f


def test_build_compiles_every_source_for_sm_103a_only():
    srcs = {f for f in os.listdir(build_mod.CSRC) if f.endswith((".cu", ".cpp"))}
    assert srcs == set(build_mod.SOURCES)
    assert build_mod.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert "-lineinfo" in build_mod.FLAGS and "-O3" in build_mod.FLAGS
