"""Pins of the oracle's 9-node quadrilateral path (Sec. III: Eq. Propagation
with s = 1..9, Eq. NonLinear_Eq), each against something other than the
oracle itself:

* shape functions: partition of unity, Kronecker property, exact
  reproduction of every xi^a eta^b with a, b <= 2;
* local coordinates: Newton's answer mapped forward by an independent
  bilinear map returns the point; exact on parallelograms and at nodes;
* interpolation: fields quadratic in the computational coordinates are
  reproduced exactly on distorted quadrilaterals (a bilinear map keeps them
  inside the biquadratic space);
* point location and the missing-population classification against brute
  force with exact rationals;
* owner elements (larger area, then lower id) and owner-element gradients
  exact for quadratic fields;
* uniform-flow preservation on a deforming mesh (Table GCL_Error), the
  integer-lattice reduction to an array-roll D2Q9, mass and energy
  conservation, shear-wave decay at the kinematic viscosity.
All run on the CPU.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2002_04353_gb300 import inputs as I

CX, CY = O.CX, O.CY
RNG = np.random.default_rng(42)
CV = 2.5
# local coordinates of the 9 nodes: corners, midsides, centre
LOCAL9 = np.array([[-1, -1], [1, -1], [1, 1], [-1, 1], [0, -1], [1, 0], [0, 1], [-1, 0], [0, 0]], float)


def _flow(mu=0.02):
    return I.Flow(gamma=1.4, Pr=0.71, mu=mu, rho_inf=1.0, T_inf=0.3)


def test_q2_shape_functions_unity_kronecker_biquadratics():
    for xi, eta in RNG.uniform(-1, 1, (100, 2)):
        assert abs(O.shape_q2(xi, eta).sum() - 1.0) < 1e-15
    for k, (xi, eta) in enumerate(LOCAL9):
        assert np.array_equal(O.shape_q2(xi, eta), np.eye(9)[k])
    c = RNG.uniform(-1, 1, (3, 3))
    p = lambda x, y: sum(c[i, j] * x ** i * y ** j for i in range(3) for j in range(3))
    vals = np.array([p(*q) for q in LOCAL9])
    for xi, eta in RNG.uniform(-1, 1, (100, 2)):
        assert abs(O.shape_q2(xi, eta) @ vals - p(xi, eta)) < 1e-14


def _bilinear(v, xi, eta):
    n = 0.25 * np.array([(1 - xi) * (1 - eta), (1 + xi) * (1 - eta), (1 + xi) * (1 + eta), (1 - xi) * (1 + eta)])
    return n @ v


def test_q2_local_coordinates_invert_the_bilinear_map():
    mesh = I.periodic_box(6, 12.0, 0.2, seed=3, elem="q2")
    o = O.Oracle(mesh, I.Motion.make(0), _flow())
    worst = 0.0
    for e in range(mesh.n_elems):
        v = mesh.X[mesh.conn[e, :4]]
        if np.ptp(v[:, 0]) > 6 or np.ptp(v[:, 1]) > 6:
            continue  # straddles the periodic seam
        for xi, eta in list(RNG.uniform(-1, 1, (5, 2))) + list(LOCAL9):
            p = _bilinear(v, xi, eta)
            loc = o.local(e, p[0], p[1])
            worst = max(worst, np.abs(_bilinear(v, *loc) - p).max(), np.abs(loc - [xi, eta]).max())
    assert worst < 1e-12
    # a parallelogram: the map is affine and one Newton step is exact
    v = np.array([[0.0, 0.0], [4.0, 1.0], [5.0, 4.0], [1.0, 3.0]])
    mesh1 = _single_quad(v)
    o1 = O.Oracle(mesh1, I.Motion.make(0), _flow())
    for xi, eta in RNG.uniform(-1, 1, (20, 2)):
        p = _bilinear(v, xi, eta)
        assert np.allclose(o1.local(0, *p), [xi, eta], rtol=0, atol=1e-15)


def _single_quad(v):
    """One 9-node quadrilateral with wall edges all round (a closed cell)."""
    X = np.concatenate([v, 0.5 * (v + np.roll(v, -1, 0)), [0.25 * (((v[0] + v[1]) + v[2]) + v[3])]])
    return I.Mesh(X, np.arange(9, dtype=np.int32).reshape(1, 9), np.ones((1, 4), np.uint8), (0.0, 0.0),
                  elem_type=I.ELEM_Q2QUAD)


def test_q2_interpolation_reproduces_quadratic_fields():
    mesh = I.periodic_box(8, 16.0, 0.2, seed=5, elem="q2")
    o = O.Oracle(mesh, I.Motion.make(0), _flow())
    c = RNG.uniform(-1, 1, 6)
    cx, cy = 8.0, 8.0  # keep away from the seam: the field is not periodic
    q = lambda x, y: (c[0] + c[1] * (x - cx) + c[2] * (y - cy) + c[3] * (x - cx) ** 2
                      + c[4] * (x - cx) * (y - cy) + c[5] * (y - cy) ** 2)
    K = q(mesh.X[:, 0], mesh.X[:, 1])
    for px, py in RNG.uniform(4.0, 12.0, (200, 2)):
        e, val = o.interp(px, py, K)
        assert e >= 0
        assert abs(val - q(px, py)) < 1e-11 * (1 + abs(q(px, py)))


def _orient_frac(a, b, c):
    ax, ay, bx, by, cx, cy = (Fraction(v) for v in (*a, *b, *c))
    d = (ax - cx) * (by - cy) - (ay - cy) * (bx - cx)
    return (d > 0) - (d < 0)


def _frames(mesh):
    L = mesh.period
    fr = np.empty((mesh.n_elems, 4, 2))
    for e in range(mesh.n_elems):
        v0 = mesh.X[mesh.conn[e, 0]]
        for k in range(4):
            d = mesh.X[mesh.conn[e, k]] - v0
            for ax in range(2):
                if L[ax] > 0:
                    d[ax] -= L[ax] * np.round(d[ax] / L[ax])
            fr[e, k] = v0 + d
    return fr


def _area2(fr):
    return (fr[:, 2, 0] - fr[:, 0, 0]) * (fr[:, 3, 1] - fr[:, 1, 1]) - (fr[:, 3, 0] - fr[:, 1, 0]) * (fr[:, 2, 1] - fr[:, 0, 1])


def _brute_locate(mesh, fr, a2, p):
    L = mesh.period
    rng_ = (-2, -1, 0, 1, 2)
    shifts = [(sx, sy) for sx in (rng_ if L[0] else (0,)) for sy in (rng_ if L[1] else (0,))]
    best = None
    for e in range(mesh.n_elems):
        for sx, sy in shifts:
            v = fr[e] + np.array([sx * L[0], sy * L[1]])
            if all(_orient_frac(v[k], v[(k + 1) % 4], p) >= 0 for k in range(4)):
                key = (-a2[e], e)
                if best is None or key < best[0]:
                    best = (key, e)
    return -1 if best is None else best[1]


@pytest.mark.parametrize("mesh", [I.periodic_box(4, 8.0, 0.2, seed=3, elem="q2"), I.lattice_box(3, elem="q2"),
                                  I.naca_omesh(16, 4, chord=10.0, R=60.0, first=0.5, elem="q2")],
                         ids=["jittered", "lattice", "omesh"])
def test_q2_point_location_matches_brute_force(mesh):
    o = O.Oracle(mesh, I.Motion.make(0), _flow())
    fr = _frames(mesh)
    a2 = _area2(fr)
    pts = [mesh.X[a] for a in range(0, mesh.n_nodes, max(1, mesh.n_nodes // 40))]
    lo, hi = mesh.X.min(0), mesh.X.max(0)
    pts += list(RNG.uniform(lo, hi, (60, 2)))
    for e in range(0, mesh.n_elems, max(1, mesh.n_elems // 20)):
        pts.append(fr[e, 0] + 0.25 * (fr[e, 1] - fr[e, 0]))  # exactly on an edge
    K = np.zeros(mesh.n_nodes)
    for p in pts:
        e, _ = o.interp(p[0], p[1], K)
        assert e == _brute_locate(mesh, fr, a2, np.asarray(p)), p


def test_q2_owner_is_largest_area_and_gradients_exact_for_quadratics():
    mesh = I.naca_omesh(24, 6, chord=10.0, R=40.0, first=0.4, elem="q2")
    o = O.Oracle(mesh, I.Motion.make(0), _flow())
    owner, loc = o.owner()
    a2 = _area2(_frames(mesh))
    for a in range(mesh.n_nodes):
        inc = np.nonzero((mesh.conn == a).any(1))[0]
        assert owner[a] == min(inc, key=lambda e: (-a2[e], e))
        assert mesh.conn[owner[a], loc[a]] == a
    X, Y = mesh.X[:, 0], mesh.X[:, 1]
    c = RNG.uniform(-1, 1, 6)
    K = c[0] + c[1] * X + c[2] * Y + c[3] * X * X + c[4] * X * Y + c[5] * Y * Y
    gx, gy = o.fe_grad(0.0, K)
    scale = np.abs(K).max() / 10
    assert np.allclose(gx, c[1] + 2 * c[3] * X + c[4] * Y, rtol=0, atol=1e-10 * scale)
    assert np.allclose(gy, c[2] + c[4] * X + 2 * c[5] * Y, rtol=0, atol=1e-10 * scale)


def test_q2_uniform_flow_preserved_on_deforming_mesh():
    """Sec. V.A, Table GCL_Error: the shape functions sum to one, so uniform
    flow stays uniform to round-off on the deforming quadrilateral mesh."""
    case = I.uniform_flow_case(n=12, L=24.0, period_steps=40.0, steps=60, elem="q2")
    o = O.Oracle(case.mesh, case.motion, case.flow)
    o.step(case.steps)
    st = o.state()
    u = case.flow.u_inf
    eps = (np.abs(st["ux"] - u[0]).sum() + np.abs(st["uy"] - u[1]).sum()) / (
        st["ux"].size * (abs(u[0]) + abs(u[1])))
    assert eps < 1e-13


def _lattice_state(mesh, T0, u0, amp, seed):
    rho, ux, uy, T = I.random_state(mesh.n_nodes, 1.0, T0, u0, amp, seed=seed)
    f = np.stack([O.feq(rho[a], ux[a], uy[a], T[a]) for a in range(mesh.n_nodes)], 1)
    g = np.stack([O.geq(rho[a], ux[a], uy[a], T[a], CV) for a in range(mesh.n_nodes)], 1)
    return f, g, rho, ux, uy, T


def test_q2_lattice_reduction_equals_array_roll_d2q9():
    """Nodes of an unjittered quadrilateral mesh with vertex spacing 2 sit on
    the integer lattice; with no motion every departure point is a node and
    propagation is the D2Q9 shift."""
    mesh = I.lattice_box(5, elem="q2")
    L = int(mesh.period[0])
    fl = I.Flow(mu=0.02, T_inf=0.2, u_inf=(0.03, 0.01), flags=O.FLAG_PHI_OFF)
    o = O.Oracle(mesh, I.Motion.make(0), fl)
    f, g, rho, ux, uy, T = _lattice_state(mesh, 0.2, (0.03, 0.01), 0.01, 3)
    o.set_state(f, g, rho, ux, uy, T)
    ix = mesh.X[:, 0].astype(int)
    iy = mesh.X[:, 1].astype(int)
    F = np.zeros((9, L, L))
    G = np.zeros((9, L, L))
    F[:, iy, ix] = f
    G[:, iy, ix] = g
    for step in range(3):
        for i in range(9):
            F[i] = np.roll(F[i], (CY[i], CX[i]), axis=(0, 1))
            G[i] = np.roll(G[i], (CY[i], CX[i]), axis=(0, 1))
        for y in range(L):
            for x in range(L):
                F[:, y, x], G[:, y, x] = O.collide(fl, F[:, y, x], G[:, y, x], 0.0, 0.0)
        o.step(1)
        st = o.state()
        assert np.allclose(st["f"], F[:, iy, ix], rtol=1e-14, atol=1e-16)
        assert np.allclose(st["g"], G[:, iy, ix], rtol=1e-14, atol=1e-16)


def test_q2_lattice_mass_and_energy_conserved_and_shear_wave_decays():
    mesh = I.lattice_box(8, elem="q2")
    n = int(mesh.period[0])
    mu = 0.02
    fl = I.Flow(mu=mu, T_inf=0.3, u_inf=(0.0, 0.0))
    o = O.Oracle(mesh, I.Motion.make(0), fl)
    k = 2 * math.pi / n
    x = mesh.X[:, 0]
    rho = np.ones(mesh.n_nodes)
    ux = np.zeros(mesh.n_nodes)
    uy = 1e-3 * np.sin(k * x)
    T = np.full(mesh.n_nodes, 0.3)
    f = np.stack([O.feq(rho[a], ux[a], uy[a], T[a]) for a in range(mesh.n_nodes)], 1)
    g = np.stack([O.geq(rho[a], ux[a], uy[a], T[a], CV) for a in range(mesh.n_nodes)], 1)
    o.set_state(f, g, rho, ux, uy, T)
    m0, e0 = f.sum(), g.sum()

    def amp():
        st = o.state()
        return 2 * np.mean(st["uy"] * np.sin(k * x))

    o.step(20)
    a1 = amp()
    o.step(100)
    a2 = amp()
    st = o.state()
    assert np.isclose(st["f"].sum(), m0, rtol=1e-14) and np.isclose(st["g"].sum(), e0, rtol=1e-14)
    assert -math.log(a2 / a1) / 100 == pytest.approx(mu * k * k, rel=0.03)


def test_q2_missing_population_classification_matches_brute_force():
    """Reading R6 on a pitching quadrilateral O-mesh: missing iff some point
    of the segment from the node to its departure point is outside the
    closed mesh (exact rationals, the segment split at boundary meetings)."""
    mesh = I.naca_omesh(16, 4, chord=10.0, R=30.0, first=0.6, elem="q2")
    mot = I.Motion.make(I.MOTION_PITCH, 0.2, 0.3, 0.05, 2.5, 0.0)
    o = O.Oracle(mesh, mot, _flow())
    t = 3.0
    elem, kind = o.locate(t)
    px, py = o.departures(t)
    fr = _frames(mesh)
    a2 = _area2(fr)
    bnd = [(fr[e, k], fr[e, (k + 1) % 4], mesh.edge_kind[e, k])
           for e in range(mesh.n_elems) for k in range(4) if mesh.edge_kind[e, k]]
    F = Fraction

    def inside(q):
        for e in range(mesh.n_elems):
            v = [(F(fr[e, k, 0]), F(fr[e, k, 1])) for k in range(4)]
            if all((v[k][0] - q[0]) * (v[(k + 1) % 4][1] - q[1]) - (v[k][1] - q[1]) * (v[(k + 1) % 4][0] - q[0]) >= 0
                   for k in range(4)):
                return True
        return False

    def meets(a, p, u, w):
        ax, ay, px_, py_ = (F(v) for v in (*a, *p))
        ux, uy, wx, wy = (F(v) for v in (*u, *w))
        dx, dy = px_ - ax, py_ - ay
        ex, ey = wx - ux, wy - uy
        den = dx * ey - dy * ex
        if den == 0:
            if (ux - ax) * dy - (uy - ay) * dx != 0:
                return []
            L2 = dx * dx + dy * dy
            ts = [((ux - ax) * dx + (uy - ay) * dy) / L2, ((wx - ax) * dx + (wy - ay) * dy) / L2]
            lo, hi = max(min(ts), F(0)), min(max(ts), F(1))
            return [lo, hi] if lo <= hi else []
        t_ = ((ux - ax) * ey - (uy - ay) * ex) / den
        s_ = ((ux - ax) * dy - (uy - ay) * dx) / den
        return [t_] if 0 <= t_ <= 1 and 0 <= s_ <= 1 else []

    wall_nodes = np.unique(np.concatenate([mesh.conn[e, [k, 4 + k, (k + 1) % 4]]
                                           for e in range(mesh.n_elems) for k in range(4)
                                           if mesh.edge_kind[e, k]]))
    sample = list(wall_nodes) + list(RNG.choice(mesh.n_nodes, 30, replace=False))
    n_missing = 0
    for a in sample:
        for i in range(9):
            p = np.array([px[i, a], py[i, a]])
            Xa = mesh.X[a]
            if np.array_equal(p, Xa) and elem[i, a] == -2:
                continue
            ts = {F(0), F(1)}
            kinds = []
            for (u, w, k) in bnd:
                m_ = meets(Xa, p, u, w)
                ts.update(m_)
                if m_:
                    kinds.append((min(m_), k))
            ts = sorted(ts)
            P0 = (F(Xa[0]), F(Xa[1]))
            D = (F(p[0]) - P0[0], F(p[1]) - P0[1])
            pts = [(P0[0] + D[0], P0[1] + D[1])] + [
                (P0[0] + (t0 + t1) / 2 * D[0], P0[1] + (t0 + t1) / 2 * D[1])
                for t0, t1 in zip(ts[:-1], ts[1:]) if t1 > t0]
            missing = not all(inside(q) for q in pts)
            if missing:
                n_missing += 1
                assert elem[i, a] == -1, (a, i)
                assert kind[i, a] == min(kinds)[1]
            else:
                assert elem[i, a] == _brute_locate(mesh, fr, a2, p), (a, i)
    assert n_missing > 20
