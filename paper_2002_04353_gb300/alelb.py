"""Python binding of the C-ABI in include/alelb.h (argument marshalling only).

Function names mirror the C entry points without the ``alelb_`` prefix.
Every step of the time stepping runs in the CUDA kernels of
``csrc/kernels.cuh``; there is no CPU fallback: loading fails loudly when
the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libalelb.so")

OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_MESH", -5: "ERR_MAP",
          -6: "ERR_LOCATE", -7: "ERR_NONFINITE", -8: "ERR_TIMEOUT", -9: "ERR_STATE"}
PREC_FP64 = 0
PREC_FP32_DEV = 1
PREC_BF16_DEV = 2
PREC_FP16_DEV = 3
RENUMBER_NONE = 0
RENUMBER_MORTON = 1
ELEM_P2TRI = 0
ELEM_Q2QUAD = 1
BATCH_GRAPHS = 0
BATCH_PERSISTENT = 1
FLAG_PHI_OFF = 1
FLAG_COLLIDE_OFF = 2
FLAG_LITERAL_VG = 4
FLAG_BC_EQUILIBRIUM = 8
FLAG_SLIP_WALL = 16
FLAG_MIDPOINT = 32
FLAG_EXACT_CHAR = 64
FLAG_OFFWALL_VG = 256
NQ = 9

# every symbol include/alelb.h declares
EXPORTS = ["alelb_mesh_create", "alelb_mesh_destroy", "alelb_mesh_move", "alelb_lb_init",
           "alelb_solver_destroy", "alelb_lb_step", "alelb_sync", "alelb_moments", "alelb_time",
           "alelb_get_pops", "alelb_set_pops", "alelb_forces", "alelb_locate", "alelb_profile",
           "alelb_kernel_times", "alelb_info", "alelb_last_error", "alelb_mesh_last_error",
           "alelb_lb_step_noalloc", "alelb_batch_create", "alelb_batch_destroy", "alelb_batch_step",
           "alelb_batch_sync", "alelb_batch_tune", "alelb_batch_profile", "alelb_batch_kernel_times",
           "alelb_batch_last_error", "alelb_mlp_create", "alelb_mlp_destroy", "alelb_mlp_get_params",
           "alelb_samples", "alelb_mlp_loss_grad", "alelb_mlp_train", "alelb_mlp_predict",
           "alelb_solver_set_mlp", "alelb_mlp_stats", "alelb_mlp_last_error", "alelb_save", "alelb_load",
           "alelb_checkpoint_info", "alelb_batch_set_mode", "alelb_batch_set_wait", "alelb_batch_set_choice",
           "alelb_batch_set_pops", "alelb_batch_get_pops", "alelb_get_pops_stored", "alelb_set_pops_stored",
           "alelb_batch_set_pops_stored", "alelb_batch_get_pops_stored", "alelb_batch_step_host",
           "alelb_get_pops_dev", "alelb_set_pops_dev", "alelb_moments_dev"]


class AlelbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class MeshDesc(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("X", C.c_void_p), ("n_elems", C.c_int32),
                ("conn", C.c_void_p), ("edge_kind", C.c_void_p), ("period", C.c_double * 2),
                ("motion_kind", C.c_int32), ("motion", C.c_double * 16), ("renumber", C.c_int32),
                ("elem_type", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("Pr", C.c_double), ("mu", C.c_double),
                ("rho_inf", C.c_double), ("T_inf", C.c_double), ("u_inf", C.c_double * 2),
                ("chord", C.c_double), ("precision", C.c_int32), ("flags", C.c_int32),
                ("stream", C.c_void_p), ("shift", C.c_double * 2)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library (build it with paper_2002_04353_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing "
                           "(run `python -m paper_2002_04353_gb300.build`)")
    L = C.CDLL(path)
    p, i32, d = C.c_void_p, C.c_int32, C.c_double
    L.alelb_mesh_create.argtypes = [C.POINTER(MeshDesc), C.POINTER(p)]
    L.alelb_mesh_destroy.argtypes = [p]
    L.alelb_mesh_destroy.restype = None
    L.alelb_mesh_move.argtypes = [p, d]
    L.alelb_lb_init.argtypes = [p, C.POINTER(Params), C.POINTER(p)]
    L.alelb_solver_destroy.argtypes = [p]
    L.alelb_solver_destroy.restype = None
    L.alelb_lb_step.argtypes = [p, i32]
    L.alelb_sync.argtypes = [p]
    L.alelb_moments.argtypes = [p, p, p, p, p]
    L.alelb_time.argtypes = [p, C.POINTER(d), C.POINTER(C.c_int64)]
    L.alelb_get_pops.argtypes = [p, p, p]
    L.alelb_set_pops.argtypes = [p, p, p, p, p, p, p, d]
    L.alelb_forces.argtypes = [p, p]
    L.alelb_locate.argtypes = [p, d, i32, p, p]
    L.alelb_profile.argtypes = [p, i32]
    L.alelb_kernel_times.argtypes = [p, C.POINTER(C.c_char_p), p, p, C.POINTER(i32)]
    L.alelb_info.argtypes = [p, p]
    L.alelb_last_error.argtypes = [p]
    L.alelb_last_error.restype = C.c_char_p
    L.alelb_mesh_last_error.argtypes = [p]
    L.alelb_mesh_last_error.restype = C.c_char_p
    L.alelb_lb_step_noalloc.argtypes = [p, C.POINTER(Params), d, p, p, p, p, p]
    L.alelb_batch_create.argtypes = [C.POINTER(p), i32, p, C.POINTER(p)]
    L.alelb_batch_destroy.argtypes = [p]
    L.alelb_batch_destroy.restype = None
    L.alelb_batch_step.argtypes = [p, i32]
    L.alelb_batch_sync.argtypes = [p]
    L.alelb_batch_tune.argtypes = [p, i32, p]
    L.alelb_batch_profile.argtypes = [p, i32]
    L.alelb_batch_kernel_times.argtypes = [p, C.POINTER(C.c_char_p), p, p, C.POINTER(i32)]
    L.alelb_batch_last_error.argtypes = [p]
    L.alelb_batch_last_error.restype = C.c_char_p
    L.alelb_mlp_create.argtypes = [p, C.c_uint64, C.POINTER(p)]
    L.alelb_mlp_destroy.argtypes = [p]
    L.alelb_mlp_destroy.restype = None
    L.alelb_mlp_get_params.argtypes = [p, i32, p]
    L.alelb_samples.argtypes = [p, d, p, p, p, p]
    L.alelb_mlp_loss_grad.argtypes = [p, p, p, p, p, C.c_int64, C.c_float, C.POINTER(d), p]
    L.alelb_mlp_train.argtypes = [p, p, p, p, p, C.c_int64, i32, i32, C.c_float, C.c_float, C.c_uint64, p]
    L.alelb_mlp_predict.argtypes = [p, p, p, C.c_int64, p, p]
    L.alelb_solver_set_mlp.argtypes = [p, p]
    L.alelb_mlp_stats.argtypes = [p, p]
    L.alelb_mlp_last_error.argtypes = [p]
    L.alelb_mlp_last_error.restype = C.c_char_p
    L.alelb_save.argtypes = [p, C.c_char_p]
    L.alelb_load.argtypes = [p, C.c_char_p]
    L.alelb_checkpoint_info.argtypes = [C.c_char_p, p, p, C.c_char_p, i32]
    L.alelb_batch_set_mode.argtypes = [p, i32]
    L.alelb_batch_set_wait.argtypes = [p, d, i32]
    L.alelb_batch_set_choice.argtypes = [p, p]
    L.alelb_batch_set_pops.argtypes = [p, p, p, p]
    L.alelb_batch_get_pops.argtypes = [p, p, p]
    L.alelb_get_pops_stored.argtypes = [p, p, p]
    L.alelb_set_pops_stored.argtypes = [p, p, p, d]
    L.alelb_batch_set_pops_stored.argtypes = [p, p, p, p]
    L.alelb_batch_get_pops_stored.argtypes = [p, p, p]
    L.alelb_batch_step_host.argtypes = [p, p, p, p, p, p]
    L.alelb_get_pops_dev.argtypes = [p, p, p]
    L.alelb_set_pops_dev.argtypes = [p, p, p, d]
    L.alelb_moments_dev.argtypes = [p, p, p, p, p]
    for name in EXPORTS:
        fn = getattr(L, name)
        if fn.restype is C.c_int:  # default: alelb_status
            fn.restype = C.c_int
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data


def _dptr(t):
    """Device address of a CUDA tensor (or None)."""
    return None if t is None else C.c_void_p(t.data_ptr())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32_out(a, n):
    """A caller's output array: C-contiguous, writable float32 of 9 x n values."""
    if not (isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous
            and a.flags.writeable and a.size == NQ * n):
        raise ValueError(f"a C-contiguous writable float32 array of 9 x {n} values")
    return a


class Mesh:
    """alelb_mesh_create / alelb_mesh_move / alelb_mesh_destroy."""

    def __init__(self, mesh, motion, renumber=RENUMBER_MORTON):
        L = load()
        self._keep = (_f64(mesh.X).reshape(-1), np.ascontiguousarray(mesh.conn, dtype=np.int32).reshape(-1),
                      np.ascontiguousarray(mesh.edge_kind, dtype=np.uint8).reshape(-1))
        X, conn, ek = self._keep
        d = MeshDesc()
        d.n_nodes = mesh.n_nodes
        d.X = X.ctypes.data
        d.n_elems = mesh.n_elems
        d.conn = conn.ctypes.data
        d.edge_kind = ek.ctypes.data
        d.period[0], d.period[1] = float(mesh.period[0]), float(mesh.period[1])
        d.motion_kind = int(motion.kind)
        for k in range(16):
            d.motion[k] = float(motion.params[k])
        d.renumber = int(renumber)
        d.elem_type = int(getattr(mesh, "elem_type", 0))
        h = C.c_void_p()
        st = L.alelb_mesh_create(C.byref(d), C.byref(h))
        if st != OK:
            msg = L.alelb_mesh_last_error(h).decode() if h.value else ""
            if h.value:
                L.alelb_mesh_destroy(h)
            raise AlelbError(st, "mesh_create: " + msg)
        self.h = h
        self.n_nodes = mesh.n_nodes
        self.n_elems = mesh.n_elems

    def move(self, t):
        L = load()
        st = L.alelb_mesh_move(self.h, float(t))
        if st != OK:
            raise AlelbError(st, L.alelb_mesh_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            load().alelb_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mesh_create(mesh, motion, renumber=RENUMBER_MORTON):
    return Mesh(mesh, motion, renumber)


def params_of(flow, precision=PREC_FP64, flags=None, stream=None):
    p = Params()
    p.gamma, p.Pr, p.mu = flow.gamma, flow.Pr, flow.mu
    p.rho_inf, p.T_inf = flow.rho_inf, flow.T_inf
    p.u_inf[0], p.u_inf[1] = flow.u_inf
    p.chord = flow.chord
    p.precision = int(precision)
    p.flags = int(flow.flags if flags is None else flags)
    p.stream = stream
    p.shift[0], p.shift[1] = getattr(flow, "shift", (0.0, 0.0))
    return p


def checkpoint_info(path):
    """alelb_checkpoint_info: checks a checkpoint file on the host; returns
    dict(precision, n_nodes, n_elems, step, t) or raises AlelbError."""
    L = load()
    out = np.zeros(4, dtype=np.int64)
    t = C.c_double()
    msg = C.create_string_buffer(512)
    st = L.alelb_checkpoint_info(os.fsencode(path), _ptr(out), C.byref(t), msg, 512)
    if st != OK:
        raise AlelbError(st, msg.value.decode())
    return dict(precision=int(out[0]), n_nodes=int(out[1]), n_elems=int(out[2]), step=int(out[3]),
                t=t.value)


def lb_step_noalloc(mesh: "Mesh", flow, t, post_ptr, rho_ptr, ux_ptr, uy_ptr, T_ptr, stream=None):
    """One FP64 step on caller-owned device buffers (raw device addresses),
    allocating nothing; see alelb_lb_step_noalloc in include/alelb.h."""
    L = load()
    p = params_of(flow, PREC_FP64, stream=stream)
    st = L.alelb_lb_step_noalloc(mesh.h, C.byref(p), float(t), post_ptr, rho_ptr, ux_ptr, uy_ptr, T_ptr)
    if st != OK:
        raise AlelbError(st, "lb_step_noalloc: " + L.alelb_mesh_last_error(mesh.h).decode())


class Solver:
    """alelb_lb_init and the per-solver entry points."""

    def __init__(self, mesh: Mesh, flow, precision=PREC_FP64, flags=None, stream=None):
        L = load()
        p = params_of(flow, precision, flags, stream)
        h = C.c_void_p()
        st = L.alelb_lb_init(mesh.h, C.byref(p), C.byref(h))
        if st != OK:
            msg = L.alelb_last_error(h).decode() if h.value else ""
            if h.value:
                L.alelb_solver_destroy(h)
            raise AlelbError(st, "lb_init: " + msg)
        self.h = h
        self.mesh = mesh
        self.nn = mesh.n_nodes

    def _check(self, st, what):
        if st != OK:
            raise AlelbError(st, f"{what}: " + load().alelb_last_error(self.h).decode())

    def lb_step(self, n=1):
        self._check(load().alelb_lb_step(self.h, int(n)), "lb_step")

    step = lb_step

    def sync(self):
        self._check(load().alelb_sync(self.h), "sync")

    def moments(self):
        out = [np.empty(self.nn) for _ in range(4)]
        self._check(load().alelb_moments(self.h, *[_ptr(a) for a in out]), "moments")
        return dict(rho=out[0], ux=out[1], uy=out[2], T=out[3])

    def moments_into(self, rho, ux, uy, T):
        self._check(load().alelb_moments(self.h, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T)), "moments")

    def time(self):
        t = C.c_double()
        n = C.c_int64()
        self._check(load().alelb_time(self.h, C.byref(t), C.byref(n)), "time")
        return t.value, n.value

    def get_pops(self, f=None, g=None):
        f = np.empty((NQ, self.nn)) if f is None else f
        g = np.empty((NQ, self.nn)) if g is None else g
        self._check(load().alelb_get_pops(self.h, _ptr(f), _ptr(g)), "get_pops")
        return f, g

    def set_pops(self, f, g, rho=None, ux=None, uy=None, T=None, t=0.0):
        f, g = _f64(f), _f64(g)
        fl = [None if a is None else _f64(a) for a in (rho, ux, uy, T)]
        self._check(load().alelb_set_pops(self.h, _ptr(f), _ptr(g), *[_ptr(a) for a in fl], float(t)),
                    "set_pops")

    def get_pops_stored(self, f=None, g=None):
        """The FP32-deviation form's stored deviations, [9, n] float32 each."""
        f = np.empty((NQ, self.nn), dtype=np.float32) if f is None else _f32_out(f, self.nn)
        g = np.empty((NQ, self.nn), dtype=np.float32) if g is None else _f32_out(g, self.nn)
        self._check(load().alelb_get_pops_stored(self.h, _ptr(f), _ptr(g)), "get_pops_stored")
        return f, g

    def set_pops_stored(self, f, g, t=0.0):
        f = np.ascontiguousarray(f, dtype=np.float32)
        g = np.ascontiguousarray(g, dtype=np.float32)
        if f.size != NQ * self.nn or g.size != NQ * self.nn:
            raise ValueError(f"9 x {self.nn} values per array")
        self._check(load().alelb_set_pops_stored(self.h, _ptr(f), _ptr(g), float(t)), "set_pops_stored")

    def _dev_planes(self, *ts):
        """CUDA float64 tensors of 9 x n values (or n for fields); torch's
        current stream is waited for, so that the caller's writes are in."""
        import torch
        for t in ts:
            if t is not None and not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
                raise ValueError("contiguous float64 CUDA tensors")
        torch.cuda.current_stream().synchronize()
        return [_dptr(t) for t in ts]

    def get_pops_dev(self, f, g):
        """Post-collision populations into CUDA tensors [9, n] (zero-copy)."""
        if f.numel() != NQ * self.nn or g.numel() != NQ * self.nn:
            raise ValueError(f"9 x {self.nn} values per tensor")
        self._check(load().alelb_get_pops_dev(self.h, *self._dev_planes(f, g)), "get_pops_dev")

    def set_pops_dev(self, f, g, t=0.0):
        if f.numel() != NQ * self.nn or g.numel() != NQ * self.nn:
            raise ValueError(f"9 x {self.nn} values per tensor")
        self._check(load().alelb_set_pops_dev(self.h, *self._dev_planes(f, g), float(t)), "set_pops_dev")

    def moments_dev(self, rho=None, ux=None, uy=None, T=None):
        """The fields into CUDA tensors of n values (any may be None)."""
        for t in (rho, ux, uy, T):
            if t is not None and t.numel() != self.nn:
                raise ValueError(f"{self.nn} values per tensor")
        self._check(load().alelb_moments_dev(self.h, *self._dev_planes(rho, ux, uy, T)), "moments_dev")

    def save(self, path):
        self._check(load().alelb_save(self.h, os.fsencode(path)), "save")

    def load(self, path):
        self._check(load().alelb_load(self.h, os.fsencode(path)), "load")

    def forces(self):
        out = np.empty(6)
        self._check(load().alelb_forces(self.h, _ptr(out)), "forces")
        return out

    def locate(self, t, use_cache=False):
        e = np.empty((NQ, self.nn), dtype=np.int32)
        k = np.empty((NQ, self.nn), dtype=np.int8)
        self._check(load().alelb_locate(self.h, float(t), int(bool(use_cache)), _ptr(e), _ptr(k)), "locate")
        return e, k

    def profile(self, enable=True):
        self._check(load().alelb_profile(self.h, int(bool(enable))), "profile")

    def kernel_times(self):
        names = (C.c_char_p * 16)()
        ms = np.zeros(16)
        n_l = np.zeros(16, dtype=np.int64)
        n = C.c_int32(16)
        self._check(load().alelb_kernel_times(self.h, names, _ptr(ms), _ptr(n_l), C.byref(n)),
                    "kernel_times")
        return {names[k].decode(): (float(ms[k]), int(n_l[k])) for k in range(n.value)}

    def samples(self, feat, slot, bary, nring, t=None):
        """Training data of the queries at map time t (default: the next
        step's) into DEVICE tensors (feat [9N, 6] f32, slot [9N] i16,
        bary [9N, 3] f32, nring [9N] u8)."""
        if t is None:
            t = self.time()[0] + 1.0
        self._check(load().alelb_samples(self.h, float(t), _dptr(feat), _dptr(slot), _dptr(bary),
                                         _dptr(nring)), "samples")

    def set_mlp(self, net):
        self._check(load().alelb_solver_set_mlp(self.h, None if net is None else net.h), "set_mlp")
        self._net = net  # keep the network alive while in use

    def mlp_stats(self):
        out = np.zeros(3, dtype=np.int64)
        self._check(load().alelb_mlp_stats(self.h, _ptr(out)), "mlp_stats")
        return dict(exact_path=int(out[0]), proposed=int(out[1]), accepted=int(out[2]))

    def info(self):
        out = np.zeros(8)
        self._check(load().alelb_info(self.h, _ptr(out)), "info")
        return dict(n_nodes=int(out[0]), n_elems=int(out[1]), pop_bytes=out[2],
                    n_wall_nodes=int(out[4]), precision=int(out[5]), n_wall_edges=int(out[6]),
                    walks=int(out[7]))

    def close(self):
        if getattr(self, "h", None):
            load().alelb_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lb_init(mesh, flow, precision=PREC_FP64, flags=None, stream=None):
    return Solver(mesh, flow, precision, flags, stream)


class Batch:
    """alelb_batch_*: one batched step over several solvers (kept alive by
    the batch)."""

    def __init__(self, solvers, stream=None):
        L = load()
        self.solvers = list(solvers)
        arr = (C.c_void_p * max(1, len(self.solvers)))(*[s.h for s in self.solvers])
        h = C.c_void_p()
        st = L.alelb_batch_create(arr, len(self.solvers), stream, C.byref(h))
        if st != OK:
            msg = L.alelb_batch_last_error(h).decode() if h.value else ""
            if h.value:
                L.alelb_batch_destroy(h)
            raise AlelbError(st, "batch_create: " + msg)
        self.h = h

    def _check(self, st, what):
        if st != OK:
            raise AlelbError(st, f"{what}: " + load().alelb_batch_last_error(self.h).decode())

    def step(self, n=1):
        self._check(load().alelb_batch_step(self.h, int(n)), "batch_step")

    def sync(self):
        self._check(load().alelb_batch_sync(self.h), "batch_sync")

    def set_mode(self, mode):
        """BATCH_GRAPHS (launch per phase, CUDA graphs) or BATCH_PERSISTENT
        (one cooperative launch per chunk, bounded grid barriers)."""
        self._check(load().alelb_batch_set_mode(self.h, int(mode)), "batch_set_mode")

    def set_wait(self, limit_seconds=1.0, missing_arrivals=0):
        self._check(load().alelb_batch_set_wait(self.h, float(limit_seconds), int(missing_arrivals)),
                    "batch_set_wait")

    def _planes(self, arrs, writable, dtype=np.float64):
        if len(arrs) != len(self.solvers):
            raise ValueError("one f and one g array per case")
        ptrs = (C.c_void_p * len(arrs))()
        for c, (a, s) in enumerate(zip(arrs, self.solvers)):
            a = np.asarray(a)
            if a.dtype != dtype or not a.flags.c_contiguous or a.size != 9 * s.nn or \
                    (writable and not a.flags.writeable):
                raise ValueError(f"case {c}: a C-contiguous {np.dtype(dtype).name} array of 9 x {s.nn} values")
            ptrs[c] = a.ctypes.data
        return ptrs

    def set_pops(self, f, g, t=None):
        """Every case's populations from host arrays (caller's node order),
        one call; t: the cases' times (or None to keep them)."""
        if len(f) != len(self.solvers) or len(g) != len(self.solvers):
            raise ValueError("one f and one g array per case")
        tt = None if t is None else np.ascontiguousarray(t, dtype=np.float64)
        self._check(load().alelb_batch_set_pops(self.h, self._planes(f, False), self._planes(g, False),
                                                None if tt is None else _ptr(tt)), "batch_set_pops")

    def get_pops(self, f, g):
        """Every case's post-collision populations into host arrays."""
        if len(f) != len(self.solvers) or len(g) != len(self.solvers):
            raise ValueError("one f and one g array per case")
        self._check(load().alelb_batch_get_pops(self.h, self._planes(f, True), self._planes(g, True)),
                    "batch_get_pops")

    def set_pops_stored(self, f, g, t=None):
        """Every case's stored FP32 deviations from host arrays, one call."""
        tt = None if t is None else np.ascontiguousarray(t, dtype=np.float64)
        self._check(load().alelb_batch_set_pops_stored(self.h, self._planes(f, False, np.float32),
                                                      self._planes(g, False, np.float32),
                                                      None if tt is None else _ptr(tt)), "batch_set_pops_stored")

    def get_pops_stored(self, f, g):
        """Every case's stored FP32 deviations into host arrays."""
        self._check(load().alelb_batch_get_pops_stored(self.h, self._planes(f, True, np.float32),
                                                      self._planes(g, True, np.float32)), "batch_get_pops_stored")

    def step_host(self, f_in, g_in, f_out, g_out, t=None):
        """One step with every case's stored FP32 deviations in host arrays:
        uploads, the step and the read-back pipelined by case group (the
        output arrays may be the input arrays)."""
        tt = None if t is None else np.ascontiguousarray(t, dtype=np.float64)
        self._check(load().alelb_batch_step_host(self.h, self._planes(f_in, False, np.float32),
                                                 self._planes(g_in, False, np.float32),
                                                 self._planes(f_out, True, np.float32),
                                                 self._planes(g_out, True, np.float32),
                                                 None if tt is None else _ptr(tt)), "batch_step_host")

    def set_choice(self, choice):
        """Launch shapes in alelb_batch_tune's encoding (8 int32 values)."""
        c = np.ascontiguousarray(choice, dtype=np.int32)
        if c.shape != (8,):
            raise ValueError("choice: 8 values")
        self._check(load().alelb_batch_set_choice(self.h, _ptr(c)), "batch_set_choice")

    def tune(self, reps=3, raw=False):
        """Tunes the launch shapes; the chosen ones by name, or (raw) in the
        8-value encoding that set_choice takes."""
        out = np.zeros(8, dtype=np.int32)
        self._check(load().alelb_batch_tune(self.h, int(reps), _ptr(out)), "batch_tune")
        if raw:
            return out
        keys = ["k_stream", "k_stream_fast", "k_stream_slow", "k_moments", "k_deriv1", "k_collide"]
        d = {k: int(out[i]) for i, k in enumerate(keys)}
        d["k_stream_slow_grid"] = int(out[6])
        d["k_stream_fast_directions_per_thread"] = int(out[7]) & 15
        d["k_deriv1_staged"] = bool(out[7] & 16)
        d["k_collide_staged"] = bool(out[7] & 32)
        d["k_stream_fast_fused_moments"] = bool(out[7] & 256)
        d["case_groups"] = 2 if out[7] & 512 else 4 if out[7] & 1024 else 1
        d["groups_pipelined"] = (int(out[7]) >> 12) & 3
        return d

    def profile(self, enable=True):
        self._check(load().alelb_batch_profile(self.h, int(bool(enable))), "batch_profile")

    def kernel_times(self):
        names = (C.c_char_p * 16)()
        ms = np.zeros(16)
        n_l = np.zeros(16, dtype=np.int64)
        n = C.c_int32(16)
        self._check(load().alelb_batch_kernel_times(self.h, names, _ptr(ms), _ptr(n_l), C.byref(n)),
                    "batch_kernel_times")
        return {names[k].decode(): (float(ms[k]), int(n_l[k])) for k in range(n.value)}

    def close(self):
        if getattr(self, "h", None):
            load().alelb_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



class Mlp:
    """alelb_mlp_*: the learned departure-element proposal network.  Device
    arrays are CUDA tensors (anything with data_ptr())."""
    N_PARAMS = 6883

    def __init__(self, params=None, seed=0):
        L = load()
        h = C.c_void_p()
        arr = None if params is None else np.ascontiguousarray(params, dtype=np.float32)
        st = L.alelb_mlp_create(_ptr(arr), int(seed), C.byref(h))
        if st != OK:
            msg = L.alelb_mlp_last_error(h).decode() if h.value else ""
            if h.value:
                L.alelb_mlp_destroy(h)
            raise AlelbError(st, "mlp_create: " + msg)
        self.h = h

    def _check(self, st, what):
        if st != OK:
            raise AlelbError(st, f"{what}: " + load().alelb_mlp_last_error(self.h).decode())

    def params(self, rounded=False):
        out = np.empty(self.N_PARAMS, dtype=np.float32)
        self._check(load().alelb_mlp_get_params(self.h, int(bool(rounded)), _ptr(out)), "mlp_get_params")
        return out

    def loss_grad(self, feat, slot, bary, nring, w_bary=1.0):
        loss = C.c_double()
        g = np.empty(self.N_PARAMS, dtype=np.float32)
        self._check(load().alelb_mlp_loss_grad(self.h, _dptr(feat), _dptr(slot), _dptr(bary), _dptr(nring),
                                               int(slot.shape[0]), float(w_bary), C.byref(loss), _ptr(g)),
                    "mlp_loss_grad")
        return loss.value, g

    def train(self, feat, slot, bary, nring, epochs=1, batch=4096, lr=1e-3, w_bary=1.0, seed=0):
        out = np.zeros(max(1, epochs))
        self._check(load().alelb_mlp_train(self.h, _dptr(feat), _dptr(slot), _dptr(bary), _dptr(nring),
                                           int(slot.shape[0]), int(epochs), int(batch), float(lr),
                                           float(w_bary), int(seed), _ptr(out)), "mlp_train")
        return out[:epochs]

    def predict(self, feat, nring, slot_out, out=None):
        self._check(load().alelb_mlp_predict(self.h, _dptr(feat), _dptr(nring), int(nring.shape[0]),
                                             _dptr(slot_out), _dptr(out)), "mlp_predict")

    def close(self):
        if getattr(self, "h", None):
            load().alelb_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
