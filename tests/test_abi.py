"""The C ABI: libenp_dg.so builds for sm_103a, loads without a GPU, and exports
every function include/enp_dg.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

import paper_2112_09271_gb300 as enp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(enp_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_operator_entry_points():
    d = _declared()
    for name in ("enp_dg_create", "enp_residual", "enp_jvp", "enp_vjp"):
        assert name in d


def test_library_builds_loads_and_exports_every_declared_symbol():
    path = enp.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a prototype for every exported entry point
    assert sorted(enp.exported_names()) == _declared()


def test_create_rejects_bad_descriptors_without_gpu_work():
    lib = enp.load()
    h = ctypes.c_void_p()
    assert lib.enp_dg_create(ctypes.byref(h), None, None, None, None) == enp.ENP_ERR_INVALID_ARG
    assert lib.enp_dg_create(None, None, None, None, None) == enp.ENP_ERR_INVALID_ARG
    m, ph, dd = enp.MeshDesc(), enp.PhysicsDesc(), enp.DiscDesc()
    m.dim = 4
    assert lib.enp_dg_create(ctypes.byref(h), ctypes.byref(m), ctypes.byref(ph),
                             ctypes.byref(dd), None) == enp.ENP_ERR_INVALID_ARG
    assert not h.value
    assert lib.enp_residual(None, None, None) == enp.ENP_ERR_INVALID_ARG


STRUCTS = [("enp_mesh_desc", "MeshDesc"), ("enp_physics_desc", "PhysicsDesc"),
           ("enp_disc_desc", "DiscDesc"), ("enp_krylov_opts", "KrylovOpts"),
           ("enp_krylov_stats", "KrylovStats"), ("enp_newton_opts", "NewtonOpts"),
           ("enp_newton_stats", "NewtonStats"), ("enp_continuation_opts", "ContinuationOpts"),
           ("enp_continuation_stats", "ContinuationStats")]


def test_binding_structs_match_the_header_layout(tmp_path):
    """Size and every field offset of each ctypes structure equal those the C
    compiler gives the header's struct (a field added on one side only fails)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "enp_dg.h"', "int main(void) {"]
    for cname, pyname in STRUCTS:
        cls = getattr(enp, pyname)
        lines.append(f'printf("{pyname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            cf = f.rstrip("_")  # ctypes names a C field that is a Python keyword with a trailing _
            lines.append(f'printf("{pyname} {f} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    # the header declares the enp_status enum and plain C types only
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        a, b, c = line.split()
        got[(a, b)] = int(c)
    for _, pyname in STRUCTS:
        cls = getattr(enp, pyname)
        assert got[(pyname, "size")] == ctypes.sizeof(cls), pyname
        for f, _ in cls._fields_:
            assert got[(pyname, f)] == getattr(cls, f).offset, (pyname, f)
