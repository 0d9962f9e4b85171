"""Plain FP64 CPU oracle of the ALE compressible lattice Boltzmann step.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It builds
``alelb_oracle.c`` with the host C compiler (no FMA contraction) and wraps
it with ctypes.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "alelb_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

NQ = 9
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])

FLAG_PHI_OFF = 1
FLAG_COLLIDE_OFF = 2
FLAG_LITERAL_VG = 4
FLAG_BC_EQUILIBRIUM = 8
FLAG_SLIP_WALL = 16
FLAG_MIDPOINT = 32
FLAG_EXACT_CHAR = 64
FLAG_OFFWALL_VG = 256


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (plain C99, -O2,
    -ffp-contract=off so that every FP64 operation rounds as written;
    OpenMP over the independent node loops of a step)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-D_GNU_SOURCE", "-ffp-contract=off", "-fPIC", "-fopenmp",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i, p = C.c_double, C.c_int, C.c_void_p
            dp = np.ctypeslib.ndpointer(np.float64, flags="C")
            ip = np.ctypeslib.ndpointer(np.int32, flags="C")
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
            i8p = np.ctypeslib.ndpointer(np.int8, flags="C")
            L.orc_create.restype = p
            L.orc_create.argtypes = [i, dp, i, ip, u8p, i, d, d, i, dp, dp, C.POINTER(C.c_int)]
            L.orc_destroy.argtypes = [p]
            L.orc_init.argtypes = [p]
            L.orc_step.argtypes = [p, i]
            L.orc_step.restype = i
            L.orc_set_state.argtypes = [p, dp, dp, dp, dp, dp, dp, d]
            L.orc_get_state.argtypes = [p, dp, dp, dp, dp, dp, dp, C.POINTER(C.c_double)]
            L.orc_locate.argtypes = [p, d, ip, i8p]
            L.orc_locate.restype = i
            L.orc_departures.argtypes = [p, d, dp, dp]
            L.orc_departures.restype = i
            L.orc_departures_exact.argtypes = [p, d, dp, dp]
            L.orc_departures_exact.restype = i
            L.orc_map.argtypes = [p, d, i, dp]
            L.orc_fe_grad.argtypes = [p, d, dp, dp, dp]
            L.orc_fe_grad.restype = i
            L.orc_interp.argtypes = [p, d, d, dp, dp]
            L.orc_interp.restype = i
            L.orc_forces.argtypes = [p, dp]
            L.orc_owner.argtypes = [p, ip, ip]
            L.orc_wall_info.argtypes = [p, u8p, dp, ip, dp]
            L.orc_wall_info.restype = i
            L.orc_orient.argtypes = [d] * 6
            L.orc_orient.restype = i
            L.orc_feq.argtypes = [d, d, d, d, dp]
            L.orc_geq.argtypes = [d, d, d, d, d, dp]
            L.orc_gqe.argtypes = [d, d, d, d, d, d, d, d, dp]
            L.orc_feq_shift.argtypes = [d, d, d, d, d, d, dp]
            L.orc_geq_shift.argtypes = [d, d, d, d, d, d, d, dp]
            L.orc_gqe_shift.argtypes = [d, d, d, d, d, d, d, d, d, d, dp]
            L.orc_collide.argtypes = [dp, dp, dp, d, d, dp, dp]
            L.orc_grad_bc.argtypes = [dp, d, d, d, d, dp, dp, dp, dp]
            L.orc_shape.argtypes = [d, d, dp]
            L.orc_shape_q2.argtypes = [d, d, dp]
            L.orc_local.argtypes = [p, i, d, d, dp]
            L.orc_local.restype = i
            L.orc_status.argtypes = [p]
            L.orc_status.restype = i
            L.orc_threads.argtypes = [i]
            L.orc_threads.restype = i
            _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _kin(flow, flags=None):
    k = flow.as_array().copy()
    if flags is not None:
        k[8] = float(flags)
    return k


class Oracle:
    """One solver instance of the oracle on one mesh."""

    def __init__(self, mesh, motion, flow, flags=None):
        L = lib()
        self.mesh, self.motion, self.flow = mesh, motion, flow
        self.kin = _kin(flow, flags)
        st = C.c_int(0)
        X = np.ascontiguousarray(mesh.X, dtype=np.float64).reshape(-1)
        conn = np.ascontiguousarray(mesh.conn, dtype=np.int32).reshape(-1)
        ek = np.ascontiguousarray(mesh.edge_kind, dtype=np.uint8).reshape(-1)
        self.h = L.orc_create(mesh.n_nodes, X, mesh.n_elems, conn, ek, int(getattr(mesh, "elem_type", 0)),
                              float(mesh.period[0]), float(mesh.period[1]), int(motion.kind),
                              np.ascontiguousarray(motion.params, dtype=np.float64), self.kin,
                              C.byref(st))
        self.nn = mesh.n_nodes
        if st.value != 0:
            L.orc_destroy(self.h)
            self.h = None
            raise OracleError(f"oracle mesh preparation failed: status {st.value}")
        L.orc_init(self.h)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_destroy(self.h)
            self.h = None

    def step(self, n=1):
        st = lib().orc_step(self.h, int(n))
        if st:
            raise OracleError(f"oracle step failed: status {st}")

    def set_state(self, f, g, rho, ux, uy, T, t=0.0):
        c = lambda a: np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        lib().orc_set_state(self.h, c(f), c(g), c(rho), c(ux), c(uy), c(T), float(t))

    def state(self):
        nn = self.nn
        f = np.empty(NQ * nn)
        g = np.empty(NQ * nn)
        rho, ux, uy, T = (np.empty(nn) for _ in range(4))
        t = C.c_double(0)
        lib().orc_get_state(self.h, f, g, rho, ux, uy, T, C.byref(t))
        return dict(f=f.reshape(NQ, nn), g=g.reshape(NQ, nn), rho=rho, ux=ux, uy=uy, T=T,
                    t=t.value)

    def locate(self, t):
        e = np.empty(NQ * self.nn, dtype=np.int32)
        k = np.empty(NQ * self.nn, dtype=np.int8)
        st = lib().orc_locate(self.h, float(t), e, k)
        if st:
            raise OracleError(f"oracle locate failed: status {st}")
        return e.reshape(NQ, self.nn), k.reshape(NQ, self.nn)

    def departures(self, t):
        px = np.empty(NQ * self.nn)
        py = np.empty(NQ * self.nn)
        st = lib().orc_departures(self.h, float(t), px, py)
        if st:
            raise OracleError(f"oracle departures failed: status {st}")
        return px.reshape(NQ, self.nn), py.reshape(NQ, self.nn)

    def departures_exact(self, t1):
        """Departure points on the exact characteristic of a step arriving at t1."""
        px = np.empty(NQ * self.nn)
        py = np.empty(NQ * self.nn)
        st = lib().orc_departures_exact(self.h, float(t1), px, py)
        if st:
            raise OracleError(f"oracle exact departures failed: status {st}")
        return px.reshape(NQ, self.nn), py.reshape(NQ, self.nn)

    def map(self, t, a):
        out = np.empty(8)
        lib().orc_map(self.h, float(t), int(a), out)
        return out

    def fe_grad(self, t, K):
        gx = np.empty(self.nn)
        gy = np.empty(self.nn)
        st = lib().orc_fe_grad(self.h, float(t), np.ascontiguousarray(K, dtype=np.float64), gx, gy)
        if st:
            raise OracleError(f"oracle gradient failed: status {st}")
        return gx, gy

    def interp(self, px, py, K):
        out = np.zeros(1)
        e = lib().orc_interp(self.h, float(px), float(py), np.ascontiguousarray(K, dtype=np.float64),
                             out)
        return e, out[0]

    def local(self, e, px, py):
        """Local coordinates of computational point (px, py) in element e."""
        out = np.empty(2)
        st = lib().orc_local(self.h, int(e), float(px), float(py), out)
        if st:
            raise OracleError(f"oracle local coordinates failed: status {st}")
        return out

    def forces(self):
        out = np.empty(6)
        lib().orc_forces(self.h, out)
        return out

    def owner(self):
        o = np.empty(self.nn, dtype=np.int32)
        loc = np.empty(self.nn, dtype=np.int32)
        lib().orc_owner(self.h, o, loc)
        return o, loc

    def wall_info(self):
        nn = self.nn
        w = np.empty(nn, dtype=np.uint8)
        n = np.empty(2 * nn)
        pe = np.empty(nn, dtype=np.int32)
        px = np.empty(2 * nn)
        nb = lib().orc_wall_info(self.h, w, n, pe, px)
        return dict(is_wall=w.astype(bool), normal=n.reshape(nn, 2), probe_e=pe,
                    probe_xi=px.reshape(nn, 2), n_boundary_edges=nb)


def threads(n=0):
    """Threads of the oracle's node loops: n > 0 sets the count; returns the
    count in use."""
    return lib().orc_threads(int(n))


# ---- node-local hooks -------------------------------------------------------

def orient(ax, ay, bx, by, cx, cy):
    return lib().orc_orient(ax, ay, bx, by, cx, cy)


def feq(rho, ux, uy, T):
    out = np.empty(NQ)
    lib().orc_feq(rho, ux, uy, T, out)
    return out


def geq(rho, ux, uy, T, Cv):
    out = np.empty(NQ)
    lib().orc_geq(rho, ux, uy, T, Cv, out)
    return out


def gqe(rho, ux, uy, T, Cv, Pxx, Pxy, Pyy):
    out = np.empty(NQ)
    lib().orc_gqe(rho, ux, uy, T, Cv, Pxx, Pxy, Pyy, out)
    return out


def feq_shift(rho, ux, uy, T, U):
    """f^eq on the lattice c_i + U (lab-frame velocity u)."""
    out = np.empty(NQ)
    lib().orc_feq_shift(rho, ux, uy, T, float(U[0]), float(U[1]), out)
    return out


def geq_shift(rho, ux, uy, T, Cv, U):
    out = np.empty(NQ)
    lib().orc_geq_shift(rho, ux, uy, T, Cv, float(U[0]), float(U[1]), out)
    return out


def gqe_shift(rho, ux, uy, T, Cv, U, Pxx, Pxy, Pyy):
    """g* on the lattice c_i + U; P the lab-frame second moments of f."""
    out = np.empty(NQ)
    lib().orc_gqe_shift(rho, ux, uy, T, Cv, float(U[0]), float(U[1]), Pxx, Pxy, Pyy, out)
    return out


def collide(flow, f, g, Xx, Xy, flags=None):
    fo = np.empty(NQ)
    go = np.empty(NQ)
    lib().orc_collide(_kin(flow, flags), np.ascontiguousarray(f, dtype=np.float64),
                      np.ascontiguousarray(g, dtype=np.float64), Xx, Xy, fo, go)
    return fo, go


def grad_bc(flow, rho, ux, uy, T, du, dT):
    fo = np.empty(NQ)
    go = np.empty(NQ)
    lib().orc_grad_bc(_kin(flow), rho, ux, uy, T, np.ascontiguousarray(du, dtype=np.float64),
                      np.ascontiguousarray(dT, dtype=np.float64), fo, go)
    return fo, go


def shape(xi, eta):
    out = np.empty(6)
    lib().orc_shape(xi, eta, out)
    return out


def shape_q2(xi, eta):
    """The 9-node quadrilateral's shape functions at (xi, eta) in [-1, 1]^2."""
    out = np.empty(9)
    lib().orc_shape_q2(xi, eta, out)
    return out
