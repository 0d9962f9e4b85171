"""Seeded synthetic inputs: meshes, motions and flow parameters.

This module builds the problems the solver is run on -- the computational
mesh (straight-sided P2 triangles), the mesh-motion description and the
free-stream/fluid parameters -- and nothing else.  It holds none of the
method's arithmetic (no map evaluation, no equilibria, no interpolation):
both the CUDA library and the CPU oracle consume its arrays and derive
everything else on their own.

Conventions shared by every consumer of these arrays
----------------------------------------------------
* ``X``      float64 (n_nodes, 2): computational node coordinates.  Vertex
  coordinates are quantised to multiples of 2**-20 so that periodic
  unwrapping (adding the period) and edge midpoints are exact in FP64.
* ``conn``   int32 (n_elems, 6): ``v0 v1 v2 m01 m12 m20`` -- the three
  vertices counter-clockwise, then the midside node of edge k (v_k, v_k+1);
  for the 9-node quadrilaterals (``elem_type`` 1) int32 (n_elems, 9):
  ``v0 v1 v2 v3 m01 m12 m23 m30 c`` -- four vertices counter-clockwise,
  the midside nodes, then the centre (the mean of the four vertices).
* ``edge_kind`` uint8 (n_elems, 3 or 4): kind of edge k: 0 interior or
  periodic, 1 wall, 2 far field.
* ``period`` (Lx, Ly): > 0 for a periodic direction, 0 otherwise.  Periodic
  coordinates lie in [0, L).

The second-order finite-element mesh of the paper (Sec. III, Fig. 1) is a
9-node quadrilateral mesh; every generator below makes either element: the
6-node triangles split each cell along a diagonal, the 9-node
quadrilaterals keep the cell.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

QUANTUM = 2.0 ** -20

# motion kinds (the integer codes the C-ABI uses)
MOTION_NONE = 0
MOTION_SINE = 1
MOTION_PLUNGE = 2
MOTION_PITCH = 3
MOTION_PITCH_PLUNGE = 4
MOTION_BLENDED_PITCH = 5

EDGE_INTERIOR = 0
EDGE_WALL = 1
EDGE_FARFIELD = 2

ELEM_P2TRI = 0
ELEM_Q2QUAD = 1


def quantize(x):
    return np.round(np.asarray(x, dtype=np.float64) / QUANTUM) * QUANTUM


@dataclasses.dataclass
class Mesh:
    X: np.ndarray
    conn: np.ndarray
    edge_kind: np.ndarray
    period: tuple
    name: str = ""
    meta: dict = dataclasses.field(default_factory=dict)
    elem_type: int = ELEM_P2TRI

    @property
    def n_nodes(self):
        return int(self.X.shape[0])

    @property
    def n_elems(self):
        return int(self.conn.shape[0])

    def permuted(self, seed: int) -> "Mesh":
        """Same mesh with node and element numbering shuffled."""
        rng = np.random.default_rng(seed)
        pn = rng.permutation(self.n_nodes)       # new -> old
        inv = np.empty_like(pn)
        inv[pn] = np.arange(self.n_nodes)
        pe = rng.permutation(self.n_elems)
        conn = inv[self.conn[pe]].astype(np.int32)
        return Mesh(self.X[pn].copy(), conn, self.edge_kind[pe].copy(),
                    self.period, self.name + f"/perm{seed}", dict(self.meta), self.elem_type)


@dataclasses.dataclass
class Motion:
    kind: int
    params: np.ndarray  # float64[16]

    @staticmethod
    def make(kind: int, *vals):
        p = np.zeros(16, dtype=np.float64)
        p[: len(vals)] = vals
        return Motion(kind, p)


@dataclasses.dataclass
class Flow:
    gamma: float = 1.4
    Pr: float = 0.71
    mu: float = 0.025
    rho_inf: float = 1.0
    T_inf: float = 0.2
    u_inf: tuple = (0.0, 0.0)
    chord: float = 1.0
    flags: int = 0
    shift: tuple = (0.0, 0.0)  # lattice shift U (velocities c_i + U)

    def as_array(self):
        return np.array([self.gamma, self.Pr, self.mu, self.rho_inf, self.T_inf,
                         self.u_inf[0], self.u_inf[1], self.chord, float(self.flags),
                         float(self.shift[0]), float(self.shift[1])]
                        + [0.0] * 5, dtype=np.float64)


# --------------------------------------------------------------------------
# P2 assembly from a vertex triangulation
# --------------------------------------------------------------------------

def _unwrap(d, L):
    if L > 0:
        d = np.where(d > 0.5 * L, d - L, d)
        d = np.where(d < -0.5 * L, d + L, d)
    return d


def p2_from_tris(vx, tris, period=(0.0, 0.0), tri_edge_kind=None):
    """Add one midside node per unique edge of a CCW vertex triangulation."""
    vx = np.asarray(vx, dtype=np.float64)
    tris = np.asarray(tris, dtype=np.int64)
    nt = tris.shape[0]
    nv = vx.shape[0]
    a = tris[:, [0, 1, 2]].reshape(-1)
    b = tris[:, [1, 2, 0]].reshape(-1)
    key = np.minimum(a, b) * nv + np.maximum(a, b)
    uniq, inv = np.unique(key, return_inverse=True)
    ea = uniq // nv
    eb = uniq % nv
    d = vx[eb] - vx[ea]
    d[:, 0] = _unwrap(d[:, 0], period[0])
    d[:, 1] = _unwrap(d[:, 1], period[1])
    mid = vx[ea] + 0.5 * d              # exact: quantised inputs
    for ax in range(2):
        if period[ax] > 0:
            mid[:, ax] = np.mod(mid[:, ax], period[ax])
    X = np.concatenate([vx, mid], axis=0)
    conn = np.empty((nt, 6), dtype=np.int32)
    conn[:, :3] = tris
    conn[:, 3:] = (nv + inv).reshape(nt, 3)
    if tri_edge_kind is None:
        tri_edge_kind = np.zeros((nt, 3), dtype=np.uint8)
    return X, conn, np.asarray(tri_edge_kind, dtype=np.uint8)


def q2_from_quads(vx, quads, period=(0.0, 0.0), quad_edge_kind=None):
    """Add one midside node per unique edge and a centre node per cell to a
    counter-clockwise vertex quadrangulation (the paper's 9-node element).
    The centre is the mean of the four vertices, the value of the bilinear
    map at (0, 0), computed from vertices unwrapped about the first."""
    vx = np.asarray(vx, dtype=np.float64)
    quads = np.asarray(quads, dtype=np.int64)
    nq = quads.shape[0]
    nv = vx.shape[0]
    a = quads[:, [0, 1, 2, 3]].reshape(-1)
    b = quads[:, [1, 2, 3, 0]].reshape(-1)
    key = np.minimum(a, b) * nv + np.maximum(a, b)
    uniq, inv = np.unique(key, return_inverse=True)
    ea = uniq // nv
    eb = uniq % nv
    d = vx[eb] - vx[ea]
    d[:, 0] = _unwrap(d[:, 0], period[0])
    d[:, 1] = _unwrap(d[:, 1], period[1])
    mid = vx[ea] + 0.5 * d
    v0 = vx[quads[:, 0]]
    rel = [vx[quads[:, k]] - v0 for k in range(4)]
    for r in rel:
        r[:, 0] = _unwrap(r[:, 0], period[0])
        r[:, 1] = _unwrap(r[:, 1], period[1])
    u = [v0 + r for r in rel]
    cen = 0.25 * (((u[0] + u[1]) + u[2]) + u[3])
    for ax in range(2):
        if period[ax] > 0:
            mid[:, ax] = np.mod(mid[:, ax], period[ax])
            cen[:, ax] = np.mod(cen[:, ax], period[ax])
    X = np.concatenate([vx, mid, cen], axis=0)
    conn = np.empty((nq, 9), dtype=np.int32)
    conn[:, :4] = quads
    conn[:, 4:8] = (nv + inv).reshape(nq, 4)
    conn[:, 8] = nv + uniq.size + np.arange(nq)
    if quad_edge_kind is None:
        quad_edge_kind = np.zeros((nq, 4), dtype=np.uint8)
    return X, conn, np.asarray(quad_edge_kind, dtype=np.uint8)


def _check_convex(vx, quads, period):
    """Every corner of every quadrilateral turns left (strictly convex)."""
    p = [vx[quads[:, k]] for k in range(4)]
    for k in range(4):
        d1 = p[(k + 1) % 4] - p[k]
        d2 = p[(k + 2) % 4] - p[(k + 1) % 4]
        for d in (d1, d2):
            for ax in range(2):
                d[:, ax] = _unwrap(d[:, ax], period[ax])
        cr = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
        if not np.all(cr > 0):
            raise ValueError(f"mesh generator produced {int(np.sum(cr <= 0))} non-convex quadrilaterals")


def _check_ccw(vx, tris, period):
    p0 = vx[tris[:, 0]]
    d1 = vx[tris[:, 1]] - p0
    d2 = vx[tris[:, 2]] - p0
    for ax in range(2):
        d1[:, ax] = _unwrap(d1[:, ax], period[ax])
        d2[:, ax] = _unwrap(d2[:, ax], period[ax])
    area2 = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    if not np.all(area2 > 0):
        raise ValueError(f"mesh generator produced {int(np.sum(area2 <= 0))} inverted triangles")
    return area2


# --------------------------------------------------------------------------
# Periodic boxes
# --------------------------------------------------------------------------

def periodic_box(n: int, L: float, jitter: float = 0.2, seed: int = 0, name="box", elem="p2"):
    """n x n vertices on the periodic square [0, L)^2, jittered by
    U(-jitter*h, jitter*h) per coordinate (h = L/n); each quad cell split
    along its SW-NE diagonal with P2 midside nodes added (elem "p2"), or
    kept as a 9-node quadrilateral (elem "q2")."""
    if n < 3:
        raise ValueError("need at least 3 vertices per side")
    h = L / n
    rng = np.random.default_rng(seed)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    vx = np.stack([i.reshape(-1) * h, j.reshape(-1) * h], axis=1).astype(np.float64)
    if jitter > 0:
        vx = vx + rng.uniform(-jitter * h, jitter * h, size=vx.shape)
    vx = np.mod(quantize(vx), L)
    vx = quantize(vx)
    vid = lambda ii, jj: (ii % n) + n * (jj % n)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    ii = ii.reshape(-1)
    jj = jj.reshape(-1)
    v00, v10, v11, v01 = vid(ii, jj), vid(ii + 1, jj), vid(ii + 1, jj + 1), vid(ii, jj + 1)
    period = (float(L), float(L))
    meta = dict(n=n, L=L, h=h, jitter=jitter, seed=seed)
    if elem == "q2":
        quads = np.stack([v00, v10, v11, v01], 1)
        _check_convex(vx, quads, period)
        X, conn, ek = q2_from_quads(vx, quads, period)
        return Mesh(X, conn, ek, period, name=f"{name}q{n}x{n}_L{L:g}_j{jitter:g}_s{seed}", meta=meta,
                    elem_type=ELEM_Q2QUAD)
    tris = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
    _check_ccw(vx, tris, period)
    X, conn, ek = p2_from_tris(vx, tris, period)
    return Mesh(X, conn, ek, period, name=f"{name}{n}x{n}_L{L:g}_j{jitter:g}_s{seed}", meta=meta)


def lattice_box(n: int, elem="p2"):
    """Unjittered periodic box with vertex spacing 2: every P2 (or Q2) node
    sits on the integer lattice [0, 2n)^2, and every lattice point is a
    node."""
    return periodic_box(n, 2.0 * n, jitter=0.0, seed=0, name="lattice", elem=elem)


# --------------------------------------------------------------------------
# NACA 00xx O-mesh
# --------------------------------------------------------------------------

def naca_half_thickness(xc, t):
    """Four-digit NACA thickness distribution with the closed trailing-edge
    coefficient; xc in [0, 1], returns y/c."""
    return 5.0 * t * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc ** 2
                      + 0.2843 * xc ** 3 - 0.1036 * xc ** 4)


def _smoothstep(s):
    s = np.clip(s, 0.0, 1.0)
    return s * s * (3.0 - 2.0 * s)


def _growth_ratio(first, total, n):
    """q with first*(q^n - 1)/(q - 1) = total."""
    lo, hi = 1.0 + 1e-9, 2.0
    for _ in range(200):
        q = 0.5 * (lo + hi)
        s = first * (q ** n - 1.0) / (q - 1.0)
        if s > total:
            hi = q
        else:
            lo = q
    return 0.5 * (lo + hi)


def naca_omesh(ni: int, nj: int, chord: float = 200.0, thickness: float = 0.12,
               R: float = 4000.0, first: float = 0.2, name="naca", elem="p2"):
    """O-mesh of P2 triangles around a NACA 00xx section (leading edge at the
    origin, chord along +x), outer far-field circle of radius R about
    mid-chord.  ni points around the section (even; spacing half
    cosine-clustered, half uniform), nj
    vertex rings; the first ring sits `first` off the wall along the surface
    normal, ring spacing grows geometrically and blends into concentric
    circles away from the body."""
    if ni % 2 or ni < 16 or nj < 4:
        raise ValueError("ni must be even and >= 16, nj >= 4")
    m = ni // 2
    beta = math.pi * np.arange(m + 1) / m
    # half cosine-clustered, half uniform along the chord: refined at the
    # leading and trailing edges without sub-lattice slivers there
    xc = 0.5 * (0.5 * (1.0 - np.cos(beta))) + 0.5 * (beta / math.pi)
    yt = naca_half_thickness(xc, thickness)
    up = np.stack([xc, yt], 1)                      # LE -> TE over the top
    lo = np.stack([xc[m - 1:0:-1], -yt[m - 1:0:-1]], 1)  # TE -> LE underneath
    P = np.concatenate([up, lo], 0) * chord          # clockwise, ni points
    P[0, 1] = 0.0
    P[m, 1] = 0.0
    t = np.roll(P, -1, 0) - np.roll(P, 1, 0)
    nrm = np.stack([-t[:, 1], t[:, 0]], 1)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)   # outward for clockwise order
    C = np.array([0.5 * chord, 0.0])
    seg = np.linalg.norm(np.roll(P, -1, 0) - P, axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)[:-1]]) / seg.sum()
    phi = math.pi - 2.0 * math.pi * s
    circ = np.stack([np.cos(phi), np.sin(phi)], 1)
    dlast = R - 0.5 * chord
    q = _growth_ratio(first, dlast, nj - 1)
    d = np.concatenate([[0.0], first * (q ** np.arange(1, nj) - 1.0) / (q - 1.0)])
    d[-1] = dlast
    w = _smoothstep((d - 1.0) / (2.0 * chord - 1.0))
    rho = 0.5 * chord + d * (R - 0.5 * chord) / dlast
    V = np.empty((nj, ni, 2))
    for jr in range(nj):
        inner = P + d[jr] * nrm
        outer = C + rho[jr] * circ
        V[jr] = (1.0 - w[jr]) * inner + w[jr] * outer
    V[-1] = C + R * circ
    vx = quantize(V.reshape(-1, 2))
    vid = lambda ii, jr: (ii % ni) + ni * jr
    ii, jr = np.meshgrid(np.arange(ni), np.arange(nj - 1), indexing="xy")
    ii = ii.reshape(-1)
    jr = jr.reshape(-1)
    a, b, c_, e = vid(ii, jr), vid(ii + 1, jr), vid(ii + 1, jr + 1), vid(ii, jr + 1)
    meta = dict(ni=ni, nj=nj, chord=chord, thickness=thickness, R=R, first=first, growth=q)
    if elem == "q2":
        quads = np.stack([a, b, c_, e], 1)
        kind = np.zeros((quads.shape[0], 4), dtype=np.uint8)
        kind[jr == 0, 0] = EDGE_WALL                 # edge a-b on ring 0
        kind[jr == nj - 2, 2] = EDGE_FARFIELD        # edge c-e on the last ring
        _check_convex(vx, quads, (0.0, 0.0))
        X, conn, ek = q2_from_quads(vx, quads, (0.0, 0.0), kind)
        return Mesh(X, conn, ek, (0.0, 0.0), name=f"{name}{int(round(thickness * 100)):02d}_q{ni}x{nj}",
                    meta=meta, elem_type=ELEM_Q2QUAD)
    tris = np.concatenate([np.stack([a, b, c_], 1), np.stack([a, c_, e], 1)], 0)
    nq = ii.size
    kind = np.zeros((2 * nq, 3), dtype=np.uint8)
    kind[:nq][jr == 0, 0] = EDGE_WALL              # edge a-b on ring 0
    kind[nq:][jr == nj - 2, 1] = EDGE_FARFIELD     # edge c-e on the last ring
    _check_ccw(vx, tris, (0.0, 0.0))
    X, conn, ek = p2_from_tris(vx, tris, (0.0, 0.0), kind)
    return Mesh(X, conn, ek, (0.0, 0.0),
                name=f"{name}{int(round(thickness * 100)):02d}_{ni}x{nj}",
                meta=dict(ni=ni, nj=nj, chord=chord, thickness=thickness, R=R,
                          first=first, growth=q))


def wall_channel(nx: int = 12, hx: float = 8.0, first: float = 0.7, growth: float = 1.17,
                 ny: int = 14, name="channel", elem="p2"):
    """Flat channel periodic in x: wall edges at y = 0 and at the top ring,
    nx cells of length hx along the wall, ny layers whose thickness starts
    at `first` and grows by `growth`, each cell split along its SW-NE
    diagonal.  Thin near-wall cells like those of an airfoil O-mesh, in a
    geometry whose uniform-in-x flows stay one-dimensional."""
    ys = [0.0]
    d = first
    for _ in range(ny):
        ys.append(ys[-1] + d)
        d *= growth
    ys = np.array(ys)
    V = quantize(np.array([[i * hx, y] for y in ys for i in range(nx)]))
    vid = lambda i, j: (i % nx) + nx * j
    if elem == "q2":
        quads, qk = [], []
        for j in range(len(ys) - 1):
            for i in range(nx):
                quads.append((vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)))
                qk.append((EDGE_WALL if j == 0 else 0, 0, EDGE_WALL if j == len(ys) - 2 else 0, 0))
        quads = np.array(quads)
        _check_convex(V, quads, (nx * hx, 0.0))
        X, conn, ek = q2_from_quads(V, quads, (nx * hx, 0.0), np.array(qk, dtype=np.uint8))
        return Mesh(X, conn, ek, (nx * hx, 0.0), name=f"{name}_q{nx}x{ny}",
                    meta=dict(hx=hx, first=first, growth=growth, height=float(ys[-1])), elem_type=ELEM_Q2QUAD)
    tris, kinds = [], []
    for j in range(len(ys) - 1):
        for i in range(nx):
            a, b, c, e = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            tris.append((a, b, c))
            kinds.append((EDGE_WALL if j == 0 else 0, 0, 0))
            tris.append((a, c, e))
            kinds.append((0, EDGE_WALL if j == len(ys) - 2 else 0, 0))
    tris = np.array(tris)
    kinds = np.array(kinds, dtype=np.uint8)
    _check_ccw(V, tris, (nx * hx, 0.0))
    X, conn, ek = p2_from_tris(V, tris, (nx * hx, 0.0), kinds)
    return Mesh(X, conn, ek, (nx * hx, 0.0), name=f"{name}_{nx}x{ny}",
                meta=dict(hx=hx, first=first, growth=growth, height=float(ys[-1])))


def omesh_size_for(n_nodes: float, aspect: float = 2.7):
    """(ni, nj) of an O-mesh with about n_nodes P2 nodes and ni/nj ~ aspect.
    A ni x nj vertex O-grid has ni*(4*nj - 2) P2 nodes."""
    nj = max(4, int(round(math.sqrt(n_nodes / (4.0 * aspect)))))
    ni = int(round(n_nodes / (4.0 * nj - 2.0)))
    ni += ni % 2
    return max(16, ni), nj


# --------------------------------------------------------------------------
# Flow parameterisation (Sec. V): Ma = u/sqrt(gamma T), Re = rho u c / mu,
# k = omega c / (2 u), Sr = h omega / u.
# --------------------------------------------------------------------------

def speed_of(Ma, T_inf, gamma=1.4):
    return Ma * math.sqrt(gamma * T_inf)


def flow_params(Ma, T_inf=0.3, Re=None, chord=200.0, angle_deg=0.0, mu=None,
                gamma=1.4, Pr=0.71, rho_inf=1.0, flags=0, shift=(0.0, 0.0)):
    U = speed_of(Ma, T_inf, gamma)
    if mu is None:
        mu = rho_inf * U * chord / Re
    a = math.radians(angle_deg)
    return Flow(gamma=gamma, Pr=Pr, mu=mu, rho_inf=rho_inf, T_inf=T_inf,
                u_inf=(U * math.cos(a), U * math.sin(a)), chord=chord, flags=flags,
                shift=tuple(float(x) for x in shift))


@dataclasses.dataclass
class Case:
    mesh: Mesh
    motion: Motion
    flow: Flow
    steps: int
    name: str


def uniform_flow_case(n=48, L=96.0, jitter=0.2, seed=0, amp_frac=0.05, period_steps=100.0,
                      steps=200, Ma=0.3, angle_deg=15.0, T_inf=0.2, omega_inf=1.6, elem="p2"):
    """Uniform-flow preservation on a deforming periodic box: x += A sin(2 pi Y/L)
    sin(2 pi t/T), y += A sin(2 pi X/L) sin(2 pi t/T) with A = amp_frac*L.
    mu is chosen so that the free-stream relaxation rate is omega_inf."""
    mesh = periodic_box(n, L, jitter, seed, elem=elem)
    motion = Motion.make(MOTION_SINE, amp_frac * L, L, period_steps, 0.0)
    mu = (1.0 / omega_inf - 0.5) * 1.0 * T_inf
    flow = flow_params(Ma, T_inf=T_inf, mu=mu, angle_deg=angle_deg, chord=L)
    return Case(mesh, motion, flow, steps, f"uniform_{mesh.name}")


def plunge_case(ni=320, nj=118, Ma=0.2, T_inf=0.3, Re=1e4, k=1.0, h_frac=0.1, chord=1000.0,
                thickness=0.12, R_frac=20.0, first_frac=1e-3, periods=5.0, elem="p2"):
    """NACA00xx plunging y = Y - h sin(omega t), omega = 2 k U / c.  The
    chord is 1000 lattice units so that the first cell layer (1e-3 c) is one
    lattice unit."""
    mesh = naca_omesh(ni, nj, chord, thickness, R_frac * chord, first_frac * chord, elem=elem)
    flow = flow_params(Ma, T_inf=T_inf, Re=Re, chord=chord)
    U = flow.u_inf[0]
    om = 2.0 * k * U / chord
    motion = Motion.make(MOTION_PLUNGE, h_frac * chord, om)
    steps = int(round(periods * 2.0 * math.pi / om))
    return Case(mesh, motion, flow, steps, f"plunge_{mesh.name}")


def pitch_case(ni=640, nj=235, Ma=0.75, T_inf=0.3, Re=1e4, k=0.08, alpha0_deg=0.1,
               amp_deg=2.5, chord=1000.0, thickness=0.12, R_frac=20.0, first_frac=1e-3,
               blended=True, periods=3.0, plunge_frac=0.0, elem="p2"):
    """NACA00xx pitching about c/4 with alpha(t) = alpha0 + A sin(omega t)
    (nose-up positive, i.e. a clockwise rotation theta = -alpha), rigid or
    blended to zero between 2c and 10c from the pivot."""
    mesh = naca_omesh(ni, nj, chord, thickness, R_frac * chord, first_frac * chord, elem=elem)
    flow = flow_params(Ma, T_inf=T_inf, Re=Re, chord=chord)
    U = flow.u_inf[0]
    om = 2.0 * k * U / chord
    th0, A = -math.radians(alpha0_deg), -math.radians(amp_deg)
    Xc, Yc = 0.25 * chord, 0.0
    if blended:
        motion = Motion.make(MOTION_BLENDED_PITCH, th0, A, om, Xc, Yc, 2.0 * chord, 10.0 * chord)
    elif plunge_frac > 0:
        motion = Motion.make(MOTION_PITCH_PLUNGE, th0, A, om, Xc, Yc, plunge_frac * chord, om)
    else:
        motion = Motion.make(MOTION_PITCH, th0, A, om, Xc, Yc)
    steps = int(round(periods * 2.0 * math.pi / om))
    return Case(mesh, motion, flow, steps, f"pitch_{mesh.name}")


def batched_sweep(n_cases=32, seed=0, n_min=20e3, n_max=300e3, scale=1.0, chord=1000.0):
    """Airfoil sweep: NACA 00xx thickness U(8, 18)%, node count log-uniform
    in [n_min, n_max] (times `scale`), Ma U(0.1, 0.8), pitch amplitude
    U(0, 5) deg, plunge amplitude U(0, 0.2c), k U(0.05, 1), Re 1e4, rigid
    pitch + plunge about c/4."""
    rng = np.random.default_rng(seed)
    cases = []
    for c in range(n_cases):
        th = rng.uniform(0.08, 0.18)
        nn = math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * scale
        Ma = rng.uniform(0.1, 0.8)
        amp = rng.uniform(0.0, 5.0)
        hp = rng.uniform(0.0, 0.2)
        k = rng.uniform(0.05, 1.0)
        ni, nj = omesh_size_for(nn)
        mesh = naca_omesh(ni, nj, chord, th, 20.0 * chord, 1e-3 * chord, name=f"sweep{c}_")
        flow = flow_params(Ma, T_inf=0.3, Re=1e4, chord=chord)
        om = 2.0 * k * flow.u_inf[0] / chord
        motion = Motion.make(MOTION_PITCH_PLUNGE, 0.0, -math.radians(amp), om, 0.25 * chord,
                             0.0, hp * chord, om)
        cases.append(Case(mesh, motion, flow, 1000, f"sweep{c}"))
    return cases


def random_state(n_nodes: int, rho_inf=1.0, T_inf=0.2, u=(0.05, 0.02), amp=0.02, seed=0):
    """Smoothly perturbed macroscopic fields (rho, ux, uy, T) per node, used
    to start solvers away from equilibrium in tests."""
    rng = np.random.default_rng(seed)
    rho = rho_inf * (1.0 + amp * rng.uniform(-1, 1, n_nodes))
    ux = u[0] + amp * rng.uniform(-1, 1, n_nodes)
    uy = u[1] + amp * rng.uniform(-1, 1, n_nodes)
    T = T_inf * (1.0 + amp * rng.uniform(-1, 1, n_nodes))
    return rho, ux, uy, T
