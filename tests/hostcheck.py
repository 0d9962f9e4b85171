"""CPU run of the kernels' element walk (hostcheck.cu beside this file): the
same location routine k_locate runs, compiled for the host.  Test tooling."""
import ctypes as C
import os
import subprocess

import numpy as np

from paper_2002_04353_gb300 import alelb, build

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hostcheck.cu")
OUT = os.path.join(HERE, "_build", "libalelb_hostcheck.so")
_lib = None


def build_lib(force=False):
    deps = build.DEPS + [SRC]
    if force or not os.path.exists(OUT) or any(os.path.getmtime(d) > os.path.getmtime(OUT) for d in deps):
        os.makedirs(os.path.dirname(OUT), exist_ok=True)
        tmp = OUT + f".{os.getpid()}.tmp"
        subprocess.run(["nvcc", "-O2", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared",
                        "-I", os.path.join(build.ROOT, "include"), "-I", build.CSRC, "-o", tmp, SRC], check=True)
        os.replace(tmp, OUT)
    return OUT


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build_lib())
        _lib.alelb_hostcheck_locate.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                                C.c_char_p, C.c_int]
        _lib.alelb_hostcheck_locate_q2.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                                   C.c_char_p, C.c_int]
        _lib.alelb_hostcheck_fast_q2.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                                 C.c_void_p]
        _lib.alelb_hostcheck_inside.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                                C.c_void_p]
        _lib.alelb_hostcheck_fast.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_void_p, C.c_void_p,
                                              C.c_void_p]
        _lib.alelb_hostcheck_orient.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
        _lib.alelb_hostcheck_orient.restype = None
    return _lib


def _desc(mesh, motion):
    X = np.ascontiguousarray(mesh.X, dtype=np.float64).reshape(-1)
    conn = np.ascontiguousarray(mesh.conn, dtype=np.int32).reshape(-1)
    ek = np.ascontiguousarray(mesh.edge_kind, dtype=np.uint8).reshape(-1)
    d = alelb.MeshDesc()
    d.n_nodes, d.X, d.n_elems = mesh.n_nodes, X.ctypes.data, mesh.n_elems
    d.conn, d.edge_kind = conn.ctypes.data, ek.ctypes.data
    d.period[0], d.period[1] = float(mesh.period[0]), float(mesh.period[1])
    d.motion_kind = int(motion.kind)
    for k in range(16):
        d.motion[k] = float(motion.params[k])
    d.renumber = alelb.RENUMBER_MORTON
    d.elem_type = int(getattr(mesh, "elem_type", 0))
    return d, (X, conn, ek)


def inside_f32(mesh, elem, px, py):
    """The FP32 strict-containment filter for points (px, py) in elements elem."""
    from paper_2002_04353_gb300 import inputs as I
    d, keep = _desc(mesh, I.Motion.make(0))
    elem = np.ascontiguousarray(elem, dtype=np.int32)
    px = np.ascontiguousarray(px, dtype=np.float64)
    py = np.ascontiguousarray(py, dtype=np.float64)
    out = np.zeros(len(elem), dtype=np.int8)
    st = lib().alelb_hostcheck_inside(C.byref(d), len(elem), elem.ctypes.data, px.ctypes.data,
                                      py.ctypes.data, out.ctypes.data)
    assert st == 0
    return out.astype(bool)


def locate(mesh, motion, t, literal=False):
    """Element choices of the library's walk on the host (triangles or
    quadrilaterals, after the mesh's element type)."""
    d, keep = _desc(mesh, motion)
    e = np.empty((9, mesh.n_nodes), dtype=np.int32)
    k = np.empty((9, mesh.n_nodes), dtype=np.int8)
    err = C.create_string_buffer(256)
    fn = lib().alelb_hostcheck_locate_q2 if getattr(mesh, "elem_type", 0) == 1 else lib().alelb_hostcheck_locate
    st = fn(C.byref(d), float(t), int(literal), e.ctypes.data, k.ctypes.data, err, 256)
    return st, e, k


def locate_fast(mesh, motion, t_prev, t):
    """Element decisions of the FP32-deviation propagation at time t with the
    cache an exact walk at t_prev leaves; returns (status, elem, kind, fast)."""
    d, keep = _desc(mesh, motion)
    e = np.empty((9, mesh.n_nodes), dtype=np.int32)
    k = np.empty((9, mesh.n_nodes), dtype=np.int8)
    f = np.empty((9, mesh.n_nodes), dtype=np.int8)
    fn = lib().alelb_hostcheck_fast_q2 if getattr(mesh, "elem_type", 0) == 1 else lib().alelb_hostcheck_fast
    st = fn(C.byref(d), float(t_prev), float(t), e.ctypes.data, k.ctypes.data, f.ctypes.data)
    return st, e, k, f.astype(bool)


def orient(pts):
    """The library's exact orientation sign for rows (ax, ay, bx, by, cx, cy),
    and the integer stage's answer alone (2 where it does not apply)."""
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 6)
    out = np.empty(len(pts), dtype=np.int32)
    stage = np.empty(len(pts), dtype=np.int32)
    lib().alelb_hostcheck_orient(pts.ctypes.data, len(pts), out.ctypes.data, stage.ctypes.data)
    return out, stage
