"""Closed-form pins of the oracle's wall quantities (Sec. IV.A, Sec. V.B).

Four parts of the oracle had no pin beyond a rest-state invariant: the
viscous and pressure parts of the wall forces (reading R9), the probe point
B of the wall condition, the element of the wall condition's first-order
gradients (reading R8), and the off-wall target velocity of reading R8c.
Each test below checks one of them against a value the test computes on its
own from the mesh arrays and a closed form:

* forces: with nodal fields that are polynomials of degree <= 2 in the
  physical coordinates, the owner-element P2 gradients are exact, the wall
  integrand is a polynomial of degree <= 2 along each straight edge (so
  Simpson's rule is exact), and the divergence theorem turns the closed
  wall integral into body-area integrals of constant or linear fields;
* probe B: with BC_EQUILIBRIUM and no collision, a wall node's missing
  populations after one step are f^eq and g^eq of the density and
  temperature at B = A + n dt, interpolated from the previous-step fields;
* gradient element and R8c: with no collision, an off-wall node's missing
  populations after one step are the Grad reconstruction (checked on its
  own by the moment pins of test_oracle_pins.py) of its target state and of
  the gradient of the fields inside the element the reading names.

All run on the CPU.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2002_04353_gb300 import inputs as I

CX, CY = O.CX, O.CY
CV = 1.0 / (1.4 - 1.0)


def _flow(mu=0.02, flags=0):
    return I.Flow(gamma=1.4, Pr=0.71, mu=mu, rho_inf=1.0, T_inf=0.3, u_inf=(0.0, 0.0),
                  chord=20.0, flags=flags)


def _eq_state(rho, ux, uy, T):
    f = np.stack([O.feq(rho[a], ux[a], uy[a], T[a]) for a in range(rho.size)], 1)
    g = np.stack([O.geq(rho[a], ux[a], uy[a], T[a], CV) for a in range(rho.size)], 1)
    return f, g


def _nv(mesh):
    return 4 if mesh.elem_type == I.ELEM_Q2QUAD else 3


def _wall_edges(mesh):
    """(element, a, m, b, other vertex) of every wall edge: its end nodes a
    and b, its midside node m, and a vertex of the element off the edge."""
    out, nv = [], _nv(mesh)
    for e in range(mesh.n_elems):
        for k in range(nv):
            if mesh.edge_kind[e, k] == I.EDGE_WALL:
                c = mesh.conn[e]
                out.append((e, c[k], c[nv + k], c[(k + 1) % nv], c[(k + 2) % nv]))
    return out


ELEMS = ["p2", "q2"]


def _rot(th):
    return np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])


# ---------------------------------------------------------------------------
# forces (reading R9): p = rho T, tau = mu (S - (1/Cv) div u I), S = grad u + grad u^T
# ---------------------------------------------------------------------------

def _body_integrals(mesh, x):
    """Area and first moments of the body enclosed by the wall edges, from
    the physical node positions x, with the divergence theorem over the
    straight edges (n pointing out of the body, i.e. into the fluid)."""
    A = Mx = My = 0.0
    for e, a, m, b, c in _wall_edges(mesh):
        pa, pb, pc = x[a], x[b], x[c]
        t = pb - pa
        n = np.array([-t[1], t[0]])
        if np.dot(n, pc - pa) < 0:  # the element (fluid) lies on the side of n
            n = -n
        # int x ds over the edge: |t| (xa + xb)/2; n ds = n_unit |t| ds_unit
        A += 0.5 * (pa[0] + pb[0]) * n[0]
        Mx += 0.5 * (pa[0] ** 2 + pa[0] * pb[0] + pb[0] ** 2) / 3.0 * n[0]
        My += 0.5 * (pa[1] ** 2 + pa[1] * pb[1] + pb[1] ** 2) / 3.0 * n[1]
    # the loop orientation of n is out of the body, so these are the body's
    # integrals up to the sign of the outward normal: int_body 1, x, y dA
    return A, Mx, My


@pytest.mark.parametrize("elem", ELEMS)
@pytest.mark.parametrize("moving", [False, True], ids=["static", "pitched"])
def test_wall_forces_of_quadratic_fields_match_closed_forms(moving, elem):
    """u_x = q1 y^2 + q2 x^2 + (linear), u_y = r1 y^2 + r2 x y + (linear),
    rho = 1 + a.x, T = T0 + b.x on a closed airfoil:
      F_visc = mu A (2 q1 + q2 (4 - 2/Cv) + r2 (1 - 1/Cv),  r1 (4 - 2/Cv)),
      F_pres = -int_body grad(rho T) dA.
    A factor 2 or a sign in S, the 1/Cv term, or a wrong Simpson weight
    changes these."""
    mesh = I.naca_omesh(40, 8, chord=20.0, R=200.0, first=1.0, elem=elem)
    if moving:
        mot = I.Motion.make(I.MOTION_PITCH, 0.2, 0.3, 0.05, 5.0, 0.0)
        t = 9.0
        p = mot.params
        th = p[0] + p[1] * math.sin(p[2] * t)
        x = p[3:5] + (mesh.X - p[3:5]) @ _rot(th).T
    else:
        mot, t = I.Motion.make(I.MOTION_NONE), 0.0
        x = mesh.X.copy()
    mu = 0.03
    o = O.Oracle(mesh, mot, _flow(mu=mu))
    X, Y = x[:, 0], x[:, 1]
    q1, q2, r1, r2 = 2e-4, -3e-4, 1.5e-4, 2.5e-4
    ux = q1 * Y ** 2 + q2 * X ** 2 + 0.01 + 1e-3 * X - 2e-3 * Y
    uy = r1 * Y ** 2 + r2 * X * Y - 0.02 + 3e-3 * X + 1e-3 * Y
    a1, a2, b1, b2, T0 = 1e-3, -2e-3, 4e-4, 6e-4, 0.3
    rho = 1.0 + a1 * X + a2 * Y
    T = T0 + b1 * X + b2 * Y
    f, g = _eq_state(rho, ux, uy, T)
    o.set_state(f, g, rho, ux, uy, T, t)
    F = o.forces()
    A, Mx, My = _body_integrals(mesh, x)
    assert A > 0  # the normals point out of the body
    Fv = mu * A * np.array([2 * q1 + q2 * (4 - 2 / CV) + r2 * (1 - 1 / CV), r1 * (4 - 2 / CV)])
    # grad(rho T) = (a1 T + b1 rho, a2 T + b2 rho), linear in x, y
    c0x, c0y = a1 * T0 + b1, a2 * T0 + b2
    cxx, cxy = 2 * a1 * b1, a1 * b2 + a2 * b1
    cyy = 2 * a2 * b2
    Fp = -np.array([c0x * A + cxx * Mx + cxy * My, c0y * A + cxy * Mx + cyy * My])
    assert np.allclose(F[2:4], Fv, rtol=1e-9, atol=1e-12 * abs(Fv).max())
    assert np.allclose(F[0:2], Fp, rtol=1e-9, atol=1e-12 * abs(Fp).max())


# ---------------------------------------------------------------------------
# probe point B = A + n dt of the wall condition (Sec. IV.A)
# ---------------------------------------------------------------------------

def _wall_normals(mesh):
    """Unit normal into the fluid at each wall node: the normalised sum of
    the unit normals of the wall edges through it."""
    acc = {}
    for e, a, m, b, c in _wall_edges(mesh):
        t = mesh.X[b] - mesh.X[a]
        n = np.array([-t[1], t[0]]) / np.linalg.norm(t)
        if np.dot(n, mesh.X[c] - mesh.X[a]) < 0:
            n = -n
        for v in (a, m, b):
            acc[v] = acc.get(v, np.zeros(2)) + n
    return {v: n / np.linalg.norm(n) for v, n in acc.items()}


def _q2_local(v, p):
    """(xi, eta) of p under the bilinear map of the corners v, by a damped
    least-squares iteration (the test's own solver, not the oracle's)."""
    x = np.zeros(2)
    for _ in range(60):
        n = 0.25 * np.array([(1 - x[0]) * (1 - x[1]), (1 + x[0]) * (1 - x[1]), (1 + x[0]) * (1 + x[1]),
                             (1 - x[0]) * (1 + x[1])])
        dn = 0.25 * np.array([[-(1 - x[1]), -(1 - x[0])], [1 - x[1], -(1 + x[0])], [1 + x[1], 1 + x[0]],
                              [-(1 + x[1]), 1 - x[0]]])
        r = n @ v - p
        J = v.T @ dn
        x = x - np.linalg.lstsq(J, r, rcond=None)[0]
    return x


def _interp_brute(mesh, p, K):
    """Interpolation of nodal field K at point p in an element that contains
    it, found by testing every element (non-periodic mesh): P2 on
    triangles, the products of 1-D quadratic Lagrange polynomials on
    quadrilaterals."""
    for e in range(mesh.n_elems):
        if mesh.elem_type == I.ELEM_Q2QUAD:
            v = mesh.X[mesh.conn[e, :4]]
            if not all((v[(k + 1) % 4, 0] - v[k, 0]) * (p[1] - v[k, 1])
                       - (v[(k + 1) % 4, 1] - v[k, 1]) * (p[0] - v[k, 0]) >= -1e-12 for k in range(4)):
                continue
            xi, eta = _q2_local(v, p)
            L = lambda s: [0.5 * s * (s - 1), (1 - s) * (1 + s), 0.5 * s * (s + 1)]
            I9 = [0, 2, 2, 0, 1, 2, 1, 0, 1]
            J9 = [0, 0, 2, 2, 0, 1, 2, 1, 1]
            N = [L(xi)[I9[k]] * L(eta)[J9[k]] for k in range(9)]
            return float(np.dot(N, K[mesh.conn[e]]))
        v = mesh.X[mesh.conn[e, :3]]
        J = np.stack([v[1] - v[0], v[2] - v[0]], 1)
        xi, eta = np.linalg.solve(J, p - v[0])
        l0 = 1 - xi - eta
        if min(xi, eta, l0) >= -1e-12:
            N = [l0 * (2 * l0 - 1), xi * (2 * xi - 1), eta * (2 * eta - 1),
                 4 * l0 * xi, 4 * xi * eta, 4 * eta * l0]
            return float(np.dot(N, K[mesh.conn[e]]))
    raise AssertionError(f"probe point {p} outside the mesh")


@pytest.mark.parametrize("elem", ELEMS)
@pytest.mark.parametrize("field", ["linear", "random"])
def test_wall_condition_reads_rho_and_T_at_the_probe_point(field, elem):
    """A probe at 2 dt, along the wrong normal, or interpolated in an element
    that does not contain B gives other values (the random field is not
    reproduced by any other element's extrapolation)."""
    mesh = I.naca_omesh(32, 8, chord=20.0, R=200.0, first=1.0, elem=elem)
    fl = _flow(flags=O.FLAG_BC_EQUILIBRIUM | O.FLAG_COLLIDE_OFF)
    o = O.Oracle(mesh, I.Motion.make(0), fl)
    X, Y = mesh.X[:, 0], mesh.X[:, 1]
    rng = np.random.default_rng(3)
    if field == "linear":
        rho = 1.0 + 2e-4 * X - 3e-4 * Y
        T = 0.3 + 1e-4 * X + 2e-4 * Y
    else:
        rho = 1.0 + 0.02 * rng.uniform(-1, 1, mesh.n_nodes)
        T = 0.3 * (1.0 + 0.02 * rng.uniform(-1, 1, mesh.n_nodes))
    zero = np.zeros(mesh.n_nodes)
    f, g = _eq_state(rho, zero, zero, T)
    o.set_state(f, g, rho, zero, zero, T, 0.0)
    _, kind = o.locate(1.0)
    o.step(1)
    st = o.state()
    checked = 0
    for a, n in _wall_normals(mesh).items():
        B = mesh.X[a] + n * 1.0
        if field == "linear":
            rB = 1.0 + 2e-4 * B[0] - 3e-4 * B[1]
            TB = 0.3 + 1e-4 * B[0] + 2e-4 * B[1]
        else:
            rB = _interp_brute(mesh, B, rho)
            TB = _interp_brute(mesh, B, T)
        fe, ge = O.feq(rB, 0.0, 0.0, TB), O.geq(rB, 0.0, 0.0, TB, CV)
        miss = np.nonzero(kind[:, a] == 1)[0]
        assert miss.size > 0
        assert np.allclose(st["f"][miss, a], fe[miss], rtol=1e-12, atol=0)
        assert np.allclose(st["g"][miss, a], ge[miss], rtol=1e-12, atol=0)
        checked += 1
    assert checked == len(_wall_normals(mesh)) > 60


# ---------------------------------------------------------------------------
# element of the wall condition's gradients (reading R8)
# ---------------------------------------------------------------------------

def _areas(mesh):
    if mesh.elem_type == I.ELEM_Q2QUAD:  # twice the area: cross product of the diagonals
        v = mesh.X[mesh.conn[:, :4]]
        d1, d2 = v[:, 2] - v[:, 0], v[:, 3] - v[:, 1]
        return d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    v = mesh.X[mesh.conn[:, :3]]
    d1, d2 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]
    return d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]


def _gradient_elements(mesh):
    """Per node: the owner element (largest incident, then lowest id) and
    the wall-side element of reading R8 (largest incident element with a
    vertex on a wall edge, then lowest id; the owner when there is none)."""
    a2 = _areas(mesh)
    wall = set()
    for e, a, m, b, c in _wall_edges(mesh):
        wall.update((a, m, b))
    owner, side = {}, {}
    for node in range(mesh.n_nodes):
        inc = np.nonzero((mesh.conn == node).any(1))[0]
        owner[node] = min(inc, key=lambda e: (-a2[e], e))
        touch = [e for e in inc if any(v in wall for v in mesh.conn[e, :_nv(mesh)])]
        side[node] = min(touch, key=lambda e: (-a2[e], e)) if touch else owner[node]
    return owner, side, wall


def _vertex_gradient(mesh, e, K, node):
    """Gradient at `node` of the interpolant of K through the vertices of e
    alone: linear on a triangle, bilinear on a quadrilateral."""
    if mesh.elem_type == I.ELEM_Q2QUAD:
        v = mesh.X[mesh.conn[e, :4]]
        xi, eta = _q2_local(v, mesh.X[node])
        dn = 0.25 * np.array([[-(1 - eta), -(1 - xi)], [1 - eta, -(1 + xi)], [1 + eta, 1 + xi],
                              [-(1 + eta), 1 - xi]])
        J = v.T @ dn  # d x / d (xi, eta)
        return np.linalg.solve(J.T, K[mesh.conn[e, :4]] @ dn)
    v = mesh.X[mesh.conn[e, :3]]
    J = np.stack([v[1] - v[0], v[2] - v[0]], 0)
    dK = K[mesh.conn[e, 1:3]] - K[mesh.conn[e, 0]]
    return np.linalg.solve(J, dK)


def _lin(c, x):
    return c[0] + c[1] * x[..., 0] + c[2] * x[..., 1]


@pytest.mark.parametrize("elem", ELEMS)
def test_wall_condition_gradient_is_taken_in_the_wall_side_element(elem):
    """Off-wall nodes one layer from the wall of a channel whose first layer
    (0.7) is thinner than a lattice unit have missing populations.  Fields
    linear inside the node's wall-side element and different linear fields
    at every other node: the reconstruction must carry the gradient of the
    inside fields.  The owner element (larger, one layer out) mixes the two
    and gives another value."""
    mesh = I.wall_channel(elem=elem)
    owner, side, wall = _gradient_elements(mesh)
    L = mesh.period[0]
    probe = I.Flow(gamma=1.4, Pr=0.71, mu=0.02, T_inf=0.3, flags=O.FLAG_COLLIDE_OFF)
    _, kind = O.Oracle(mesh, I.Motion.make(0), probe).locate(1.0)
    cand = [a for a in range(mesh.n_nodes)
            if a not in wall and (kind[:, a] == 1).any() and owner[a] != side[a]
            and all(0.2 * L < mesh.X[v, 0] < 0.8 * L for v in mesh.conn[side[a]])
            and all(0.2 * L < mesh.X[v, 0] < 0.8 * L for v in mesh.conn[owner[a]])]
    assert len(cand) >= 4
    L1, L2 = (0.05, 3e-3, -4e-3), (0.02, -6e-3, 8e-3)
    M1, M2 = (-0.01, 2e-3, 5e-3), (0.03, 1e-3, -7e-3)
    # on the (rectangular) quadrilaterals the inside fields also carry a
    # bilinear term about the cell centre, which the vertex interpolant
    # reproduces: its gradient must be taken at the node, not the centre
    q = 1e-3 if elem == "q2" else 0.0
    for a in cand[:: max(1, len(cand) // 4)][:4]:
        inside = np.zeros(mesh.n_nodes, bool)
        inside[mesh.conn[side[a]]] = True
        xc = mesh.X[mesh.conn[side[a], :_nv(mesh)]].mean(0)
        bil = q * (mesh.X[:, 0] - xc[0]) * (mesh.X[:, 1] - xc[1])
        ux = np.where(inside, _lin(L1, mesh.X) + bil, _lin(L2, mesh.X))
        uy = np.where(inside, _lin(M1, mesh.X) - bil, _lin(M2, mesh.X))
        gb = q * np.array([mesh.X[a, 1] - xc[1], mesh.X[a, 0] - xc[0]])
        du = np.array([L1[1] + gb[0], L1[2] + gb[1], M1[1] - gb[0], M1[2] - gb[1]])
        rho = np.ones(mesh.n_nodes)
        T = np.full(mesh.n_nodes, 0.3)
        f, g = _eq_state(rho, ux, uy, T)
        o = O.Oracle(mesh, I.Motion.make(0), probe)
        o.set_state(f, g, rho, ux, uy, T, 0.0)
        o.step(1)
        st = o.state()
        fe, ge = O.grad_bc(probe, 1.0, ux[a], uy[a], 0.3, du, np.zeros(2))
        miss = np.nonzero(kind[:, a] == 1)[0]
        assert np.allclose(st["f"][miss, a], fe[miss], rtol=1e-12, atol=1e-16)
        assert np.allclose(st["g"][miss, a], ge[miss], rtol=1e-12, atol=1e-16)
        # the owner element's vertex-linear gradient differs, and so does the
        # reconstruction it would give: the check above can fail
        dow = np.concatenate([_vertex_gradient(mesh, owner[a], ux, a), _vertex_gradient(mesh, owner[a], uy, a)])
        assert np.abs(dow - du).max() > 1e-3
        fo, _ = O.grad_bc(probe, 1.0, ux[a], uy[a], 0.3, dow, np.zeros(2))
        assert np.abs(fe[miss] - fo[miss]).max() > 1e-6


# ---------------------------------------------------------------------------
# off-wall target velocity (reading R8c, flag OFFWALL_VG)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("elem", ELEMS)
@pytest.mark.parametrize("offwall_vg", [True, False], ids=["R8c", "R8"])
def test_offwall_target_velocity_next_to_a_receding_wall(offwall_vg, elem):
    """The channel plunges, y = Y - h sin(w t): the walls move with
    V_G = (0, -h w cos w t), away from the fluid above the lower wall.
    After one step without collision, each off-wall node's missing
    populations are the Grad reconstruction of (rho_prev, u_tgt, T_prev)
    with the gradients of the (linear) previous-step velocity, where
    u_tgt = V_G(t_{n+1}) under the flag and the node's own previous
    velocity without it (reading R8)."""
    mesh = I.wall_channel(elem=elem)
    h, w = 2.0, 0.02
    mot = I.Motion.make(I.MOTION_PLUNGE, h, w)
    flags = O.FLAG_COLLIDE_OFF | (O.FLAG_OFFWALL_VG if offwall_vg else 0)
    fl = I.Flow(gamma=1.4, Pr=0.71, mu=0.02, T_inf=0.3, flags=flags)
    o = O.Oracle(mesh, mot, fl)
    L1, M1 = (0.05, 3e-4, -4e-3), (-0.01, 2e-4, 5e-3)
    ux, uy = _lin(L1, mesh.X), _lin(M1, mesh.X)
    rho = np.full(mesh.n_nodes, 1.02)
    T = np.full(mesh.n_nodes, 0.31)
    f, g = _eq_state(rho, ux, uy, T)
    o.set_state(f, g, rho, ux, uy, T, 0.0)
    _, kind = o.locate(1.0)
    o.step(1)
    st = o.state()
    _, _, wall = _gradient_elements(mesh)
    Lx = mesh.period[0]
    Vy = -h * w * math.cos(w * 1.0)
    du = np.array([L1[1], L1[2], M1[1], M1[2]])
    n = 0
    for a in range(mesh.n_nodes):
        miss = np.nonzero(kind[:, a] == 1)[0]
        if a in wall or miss.size == 0 or not (0.2 * Lx < mesh.X[a, 0] < 0.8 * Lx):
            continue
        tx, ty = (0.0, Vy) if offwall_vg else (ux[a], uy[a])
        fe, ge = O.grad_bc(fl, 1.02, tx, ty, 0.31, du, np.zeros(2))
        assert np.allclose(st["f"][miss, a], fe[miss], rtol=1e-12, atol=1e-16), a
        assert np.allclose(st["g"][miss, a], ge[miss], rtol=1e-12, atol=1e-16), a
        n += 1
    assert n >= 10
