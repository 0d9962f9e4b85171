"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/alelb.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

from paper_2002_04353_gb300 import alelb, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "alelb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(alelb_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["alelb_mesh_create", "alelb_mesh_move", "alelb_lb_init", "alelb_lb_step",
              "alelb_moments", "alelb_forces"]:
        assert n in names


def test_library_loads_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for n in _declared():
        assert hasattr(lib, n), n
    assert sorted(_declared()) == sorted(alelb.EXPORTS)


def test_binding_fails_loudly_without_the_library(tmp_path):
    import pytest
    old = alelb._lib
    alelb._lib = None
    try:
        with pytest.raises(RuntimeError):
            alelb.load(str(tmp_path / "missing.so"))
    finally:
        alelb._lib = old


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of alelb_params and alelb_mesh_desc have the
    header's size and field offsets (the host compiler lays out the C
    structs; a field added on one side only would shift the others)."""
    import subprocess
    fields = {"alelb_params": (alelb.Params, ["gamma", "Pr", "mu", "rho_inf", "T_inf", "u_inf", "chord",
                                               "precision", "flags", "stream", "shift"]),
              "alelb_mesh_desc": (alelb.MeshDesc, [f[0] for f in alelb.MeshDesc._fields_])}
    src = ['#include <stddef.h>', '#include <stdio.h>', '#include "alelb.h"', "int main(void) {"]
    for struct, (_, names) in fields.items():
        src.append(f'printf("{struct} size %zu\\n", sizeof({struct}));')
        for n in names:
            src.append(f'printf("{struct} {n} %zu\\n", offsetof({struct}, {n}));')
    src.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line}
    for struct, (cls, names) in fields.items():
        assert got[(struct, "size")] == ctypes.sizeof(cls), struct
        for n in names:
            assert got[(struct, n)] == getattr(cls, n).offset, f"{struct}.{n}"


def test_empty_and_oversize_inputs_are_refused_on_the_host():
    """An empty mesh and a batch of 0 or more than 32 cases are refused with
    ALELB_ERR_ARG before anything reaches a device (no GPU needed)."""
    import numpy as np
    L = alelb.load(build.build())
    d = alelb.MeshDesc()
    X = np.zeros(2, dtype=np.float64)
    conn = np.zeros(6, dtype=np.int32)
    ek = np.zeros(3, dtype=np.uint8)
    d.n_nodes, d.X, d.n_elems = 0, X.ctypes.data, 0
    d.conn, d.edge_kind = conn.ctypes.data, ek.ctypes.data
    for et in (alelb.ELEM_P2TRI, alelb.ELEM_Q2QUAD):
        d.elem_type = et
        h = ctypes.c_void_p()
        assert L.alelb_mesh_create(ctypes.byref(d), ctypes.byref(h)) == -1
        assert b"empty" in L.alelb_mesh_last_error(h)
        L.alelb_mesh_destroy(h)
    d.elem_type = 7
    h = ctypes.c_void_p()
    assert L.alelb_mesh_create(ctypes.byref(d), ctypes.byref(h)) == -1
    L.alelb_mesh_destroy(h)
    arr = (ctypes.c_void_p * 33)()
    out = ctypes.c_void_p()
    assert L.alelb_batch_create(arr, 0, None, ctypes.byref(out)) == -1
    assert L.alelb_batch_create(arr, 33, None, ctypes.byref(out)) == -1
    assert not out.value
