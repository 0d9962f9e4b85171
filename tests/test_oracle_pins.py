"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: exact
rational arithmetic, closed forms, the moment conditions the paper states,
textbook special cases (the integer-lattice reduction, shear-wave decay),
the exact characteristic of the map, and invariants (conservation, uniform
flow preservation).  All run on the CPU.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2002_04353_gb300 import inputs as I

CX, CY = O.CX, O.CY
RNG = np.random.default_rng(1234)
CV = 1.0 / (1.4 - 1.0)  # the oracle derives Cv = 1/(gamma - 1) from gamma


# ---------------------------------------------------------------------------
# exact orientation predicate
# ---------------------------------------------------------------------------

def _orient_frac(a, b, c):
    ax, ay, bx, by, cx, cy = (Fraction(v) for v in (*a, *b, *c))
    d = (ax - cx) * (by - cy) - (ay - cy) * (bx - cx)
    return (d > 0) - (d < 0)


def test_orient_exact_against_rationals():
    n_zero = 0
    for k in range(4000):
        a = RNG.uniform(-50, 50, 2)
        b = RNG.uniform(-50, 50, 2)
        if k % 2:
            # nearly or exactly collinear: c on the line a-b, rounded
            t = RNG.uniform(-2, 3)
            c = a + t * (b - a)
            if k % 4 == 1:
                c = a + (b - a) * 0.5  # midpoint of quantised points: exact
                a, b = I.quantize(a), I.quantize(b)
                c = a + (b - a) * 0.5
        else:
            c = RNG.uniform(-50, 50, 2)
        s = O.orient(a[0], a[1], b[0], b[1], c[0], c[1])
        e = _orient_frac(a, b, c)
        n_zero += e == 0
        assert s == e, (a, b, c)
    assert n_zero > 500  # the degenerate branch was exercised


# ---------------------------------------------------------------------------
# equilibria: the moment conditions of Sec. IV / Table I
# ---------------------------------------------------------------------------

def _states(n=50):
    for _ in range(n):
        rho = RNG.uniform(0.5, 2.0)
        ux, uy = RNG.uniform(-0.25, 0.25, 2)
        T = RNG.uniform(0.15, 0.45)
        yield rho, ux, uy, T


def test_feq_moments_and_third_moment_deviation():
    for rho, ux, uy, T in _states():
        f = O.feq(rho, ux, uy, T)
        assert np.isclose(f.sum(), rho, rtol=1e-14)
        assert np.isclose((CX * f).sum(), rho * ux, rtol=1e-13, atol=1e-15)
        assert np.isclose((CY * f).sum(), rho * uy, rtol=1e-13, atol=1e-15)
        assert np.isclose((CX * CX * f).sum(), rho * ux * ux + rho * T, rtol=1e-13)
        assert np.isclose((CX * CY * f).sum(), rho * ux * uy, rtol=1e-13, atol=1e-15)
        assert np.isclose((CY * CY * f).sum(), rho * uy * uy + rho * T, rtol=1e-13)
        # third moment on D2Q9 equals rho u_x; its deviation from the
        # Maxwellian (rho u^3 + 3 rho u T) is Q'_xxx of Eq. DeviationTerms
        m3 = (CX ** 3 * f).sum()
        assert np.isclose(m3 - (rho * ux ** 3 + 3 * rho * ux * T),
                          rho * ux * (1 - 3 * T) - rho * ux ** 3, rtol=1e-12, atol=1e-15)


def _Req(rho, ux, uy, T, E):
    d = np.eye(2)
    u = np.array([ux, uy])
    return 2 * rho * E * (T * d + np.outer(u, u)) + 2 * rho * T * (T * d + 2 * np.outer(u, u))


def _mom2(g):
    return np.array([[(CX * CX * g).sum(), (CX * CY * g).sum()],
                     [(CY * CX * g).sum(), (CY * CY * g).sum()]])


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_geq_moments(gamma):
    Cv = 1.0 / (gamma - 1.0)
    for rho, ux, uy, T in _states():
        g = O.geq(rho, ux, uy, T, Cv)
        E = Cv * T + 0.5 * (ux * ux + uy * uy)
        assert np.isclose(g.sum(), 2 * rho * E, rtol=1e-13)
        q = 2 * rho * np.array([ux, uy]) * (E + T)
        assert np.allclose([(CX * g).sum(), (CY * g).sum()], q, rtol=1e-12, atol=1e-14)
        assert np.allclose(_mom2(g), _Req(rho, ux, uy, T, E), rtol=1e-12, atol=1e-14)


def test_gstar_moments_carry_the_pressure_deviation():
    Cv = 2.5
    for rho, ux, uy, T in _states():
        P = np.array([[rho * ux * ux + rho * T, rho * ux * uy],
                      [rho * ux * uy, rho * uy * uy + rho * T]])
        dP = RNG.uniform(-0.02, 0.02, (2, 2))
        dP = dP + dP.T
        Pn = P + dP
        g = O.gqe(rho, ux, uy, T, Cv, Pn[0, 0], Pn[0, 1], Pn[1, 1])
        E = Cv * T + 0.5 * (ux * ux + uy * uy)
        u = np.array([ux, uy])
        qeq = 2 * rho * u * (E + T)
        assert np.isclose(g.sum(), 2 * rho * E, rtol=1e-13)
        assert np.allclose([(CX * g).sum(), (CY * g).sum()], qeq + 2 * dP @ u, rtol=1e-12,
                           atol=1e-14)
        assert np.allclose(_mom2(g), _Req(rho, ux, uy, T, E), rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------------------
# collision (Eqs. feqn, geqn)
# ---------------------------------------------------------------------------

def _flow(mu=0.02, Pr=0.71, gamma=1.4):
    return I.Flow(gamma=gamma, Pr=Pr, mu=mu, rho_inf=1.0, T_inf=0.3)


def test_collision_conserves_and_adds_correction_momentum():
    fl = _flow()
    Cv = 2.5
    for rho, ux, uy, T in _states(30):
        f = O.feq(rho, ux, uy, T) * (1 + RNG.uniform(-0.05, 0.05, 9))
        g = O.geq(rho, ux, uy, T, Cv) * (1 + RNG.uniform(-0.05, 0.05, 9))
        Xx, Xy = RNG.uniform(-1e-3, 1e-3, 2)
        fo, go = O.collide(fl, f, g, Xx, Xy)
        assert np.isclose(fo.sum(), f.sum(), rtol=1e-14)
        assert np.isclose(go.sum(), g.sum(), rtol=1e-14)
        assert np.isclose((CX * fo).sum(), (CX * f).sum() + Xx, rtol=0, atol=1e-14)
        assert np.isclose((CY * fo).sum(), (CY * f).sum() + Xy, rtol=0, atol=1e-14)


def test_uniform_equilibrium_is_a_fixed_point():
    # holds only with q* = q^eq + 2u.(P - P^eq) (reading of Table I's q*)
    fl = _flow()
    for rho, ux, uy, T in _states(30):
        f = O.feq(rho, ux, uy, T)
        g = O.geq(rho, ux, uy, T, 2.5)
        fo, go = O.collide(fl, f, g, 0.0, 0.0)
        assert np.allclose(fo, f, rtol=1e-13, atol=1e-16)
        assert np.allclose(go, g, rtol=1e-13, atol=1e-16)


def test_relaxation_rates_match_viscosity_and_prandtl():
    # mu = (1/omega - 1/2) rho T dt and Pr = Cp mu / kappa with
    # kappa = Cp (1/omega1 - 1/2) rho T dt (Sec. IV)
    for mu, Pr in [(0.02, 0.71), (0.005, 1.3), (0.08, 0.4)]:
        fl = _flow(mu=mu, Pr=Pr)
        rho, ux, uy, T = 1.1, 0.05, -0.03, 0.28
        f0 = O.feq(rho, ux, uy, T)
        eps = 1e-6
        df = eps * CX * CY  # pure shear stress: no mass, no momentum
        fo, _ = O.collide(fl, f0 + df, O.geq(rho, ux, uy, T, 2.5), 0.0, 0.0)
        ratio = ((CX * CY * fo).sum() - rho * ux * uy) / (4 * eps)
        omega = 1 - ratio
        assert np.isclose((1 / omega - 0.5) * rho * T, mu, rtol=1e-6)
        # heat-flux relaxation with f at equilibrium: g' - g^eq = (1 - omega1)(g - g^eq)
        g0 = O.geq(rho, ux, uy, T, 2.5)
        dg = eps * np.array([0, 1, 0, -1, 0, 0, 0, 0, 0], float)  # x-heat flux, no energy
        _, go = O.collide(fl, f0, g0 + dg, 0.0, 0.0)
        r1 = ((CX * go).sum() - (CX * g0).sum()) / (2 * eps)
        omega1 = 1 - r1
        assert np.isclose((1 / omega - 0.5) / (1 / omega1 - 0.5), Pr, rtol=1e-6)


# ---------------------------------------------------------------------------
# Grad-type missing populations (Sec. IV.A, Table II)
# ---------------------------------------------------------------------------

def test_grad_bc_reduces_to_equilibrium_without_gradients():
    fl = _flow()
    for rho, ux, uy, T in _states(20):
        f, g = O.grad_bc(fl, rho, ux, uy, T, np.zeros(4), np.zeros(2))
        assert np.allclose(f, O.feq(rho, ux, uy, T), rtol=1e-15, atol=0)
        assert np.allclose(g, O.geq(rho, ux, uy, T, CV), rtol=1e-15, atol=0)


def test_grad_bc_rigid_rotation_has_no_nonequilibrium_part():
    # S = du + du^T vanishes for a rigid rotation, div u = 0: f^(1) = 0
    fl = _flow()
    rho, ux, uy, T = 1.0, 0.04, 0.02, 0.3
    w = 0.013
    f, _ = O.grad_bc(fl, rho, ux, uy, T, np.array([0.0, -w, w, 0.0]), np.zeros(2))
    assert np.allclose(f, O.feq(rho, ux, uy, T), rtol=0, atol=1e-15)


def test_grad_bc_nonequilibrium_moments():
    fl = _flow(mu=0.02)
    rho, ux, uy, T = 1.05, 0.03, -0.02, 0.3
    omega = 1 / (fl.mu / (rho * T) + 0.5)
    omega1 = 1 / ((1 / omega - 0.5) / fl.Pr + 0.5)
    s = 0.01
    feq = O.feq(rho, ux, uy, T)
    f, g = O.grad_bc(fl, rho, ux, uy, T, np.array([0.0, s, 0.0, 0.0]), np.zeros(2))
    f1 = f - feq
    assert abs(f1.sum()) < 1e-16 and abs((CX * f1).sum()) < 1e-16 and abs((CY * f1).sum()) < 1e-16
    assert np.isclose((CX * CY * f1).sum(), -(1 / omega) * rho * T * s, rtol=1e-12)
    # temperature gradient at u = 0: first moment of g^(1) = -(2/omega1) rho Cp T dT
    dT = np.array([2e-3, -1e-3])
    g0 = O.geq(rho, 0, 0, T, CV)
    _, g = O.grad_bc(fl, rho, 0.0, 0.0, T, np.zeros(4), dT)
    g1 = g - g0
    q1 = -(2 / omega1) * rho * (CV + 1) * T * dT
    assert np.allclose([(CX * g1).sum(), (CY * g1).sum()], q1, rtol=1e-12)
    assert abs(g1.sum()) < 1e-15


# ---------------------------------------------------------------------------
# P2 shape functions (Eq. Propagation for the 6-node triangle)
# ---------------------------------------------------------------------------

LOCAL = np.array([[0, 0], [1, 0], [0, 1], [0.5, 0], [0.5, 0.5], [0, 0.5]])


def test_shape_functions_unity_kronecker_quadratics():
    for xi, eta in RNG.uniform(0, 0.5, (100, 2)):
        assert np.isclose(O.shape(xi, eta).sum(), 1.0, rtol=0, atol=1e-15)
    for k, (xi, eta) in enumerate(LOCAL):
        N = O.shape(xi, eta)
        assert np.array_equal(N, np.eye(6)[k])
    c = RNG.uniform(-1, 1, 6)
    q = lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y
    vals = np.array([q(*p) for p in LOCAL])
    for xi, eta in RNG.uniform(0, 0.5, (100, 2)):
        assert np.isclose(O.shape(xi, eta) @ vals, q(xi, eta), rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------
# point location against brute force with exact rationals
# ---------------------------------------------------------------------------

def _elem_frames(mesh):
    X, conn, L = mesh.X, mesh.conn, mesh.period
    fr = np.empty((mesh.n_elems, 3, 2))
    for e in range(mesh.n_elems):
        v0 = X[conn[e, 0]]
        for k in range(3):
            d = X[conn[e, k]] - v0
            for ax in range(2):
                if L[ax] > 0:
                    d[ax] -= L[ax] * np.round(d[ax] / L[ax])
            fr[e, k] = v0 + d
    return fr


def _brute_locate(mesh, fr, p):
    L = mesh.period
    rng_ = (-2, -1, 0, 1, 2)
    shifts = [(sx, sy) for sx in (rng_ if L[0] else (0,)) for sy in (rng_ if L[1] else (0,))]
    best = None
    for e in range(mesh.n_elems):
        for sx, sy in shifts:
            v = fr[e] + np.array([sx * L[0], sy * L[1]])
            if all(_orient_frac(v[k], v[(k + 1) % 3], p) >= 0 for k in range(3)):
                d = fr[e, 1] - fr[e, 0]
                d2 = fr[e, 2] - fr[e, 0]
                a2 = d[0] * d2[1] - d2[0] * d[1]
                key = (-a2, e)
                if best is None or key < best[0]:
                    best = (key, e)
    return -1 if best is None else best[1]


@pytest.mark.parametrize("mesh", [I.periodic_box(4, 8.0, 0.2, seed=3), I.lattice_box(3),
                                  I.naca_omesh(16, 4, chord=10.0, R=60.0, first=0.5)],
                         ids=["jittered", "lattice", "omesh"])
def test_point_location_matches_brute_force(mesh):
    o = O.Oracle(mesh, I.Motion.make(0), _flow())
    fr = _elem_frames(mesh)
    pts = [mesh.X[a] for a in range(0, mesh.n_nodes, max(1, mesh.n_nodes // 40))]
    lo, hi = mesh.X.min(0), mesh.X.max(0)
    pts += list(RNG.uniform(lo, hi, (60, 2)))
    # exact points on edges: quarter points of quantised vertices
    for e in range(0, mesh.n_elems, max(1, mesh.n_elems // 20)):
        pts.append(fr[e, 0] + 0.25 * (fr[e, 1] - fr[e, 0]))
    if mesh.period[0] > 0:
        pts += [mesh.X[0] + np.array([mesh.period[0], 0.0]), mesh.X[1] - np.array([0.0, mesh.period[1]])]
    K = np.zeros(mesh.n_nodes)
    for p in pts:
        e, _ = o.interp(p[0], p[1], K)
        assert e == _brute_locate(mesh, fr, np.asarray(p)), p


def test_owner_element_is_largest_area_then_lowest_id():
    mesh = I.periodic_box(5, 10.0, 0.2, seed=7)
    o = O.Oracle(mesh, I.Motion.make(0), _flow())
    owner, loc = o.owner()
    fr = _elem_frames(mesh)
    a2 = np.array([(fr[e, 1, 0] - fr[e, 0, 0]) * (fr[e, 2, 1] - fr[e, 0, 1])
                   - (fr[e, 2, 0] - fr[e, 0, 0]) * (fr[e, 1, 1] - fr[e, 0, 1])
                   for e in range(mesh.n_elems)])
    for a in range(mesh.n_nodes):
        inc = np.nonzero((mesh.conn == a).any(1))[0]
        best = min(inc, key=lambda e: (-a2[e], e))
        assert owner[a] == best
        assert mesh.conn[owner[a], loc[a]] == a


# ---------------------------------------------------------------------------
# FE derivatives (Eqs. Ph_Derivative, FE_Derivative)
# ---------------------------------------------------------------------------

def test_fe_gradient_exact_for_quadratics():
    mesh = I.naca_omesh(24, 5, chord=10.0, R=40.0, first=0.4)
    o = O.Oracle(mesh, I.Motion.make(0), _flow())
    X, Y = mesh.X[:, 0], mesh.X[:, 1]
    c = RNG.uniform(-1, 1, 6)
    K = c[0] + c[1] * X + c[2] * Y + c[3] * X * X + c[4] * X * Y + c[5] * Y * Y
    gx, gy = o.fe_grad(0.0, K)
    ex = c[1] + 2 * c[3] * X + c[4] * Y
    ey = c[2] + c[4] * X + 2 * c[5] * Y
    scale = np.abs(K).max() / 10
    assert np.allclose(gx, ex, rtol=0, atol=1e-10 * scale)
    assert np.allclose(gy, ey, rtol=0, atol=1e-10 * scale)


@pytest.mark.parametrize("kind", [I.MOTION_PITCH, I.MOTION_PITCH_PLUNGE])
def test_physical_gradient_of_a_physically_linear_field(kind):
    # K = b . x(X, t) with an affine map is linear in X: d_x K must equal b.
    mesh = I.naca_omesh(24, 5, chord=10.0, R=40.0, first=0.4)
    mot = I.Motion.make(kind, 0.3, 0.2, 0.05, 2.5, 0.0, 1.0, 0.05)
    o = O.Oracle(mesh, mot, _flow())
    t = 7.0
    x = np.array([o.map(t, a)[6:8] for a in range(mesh.n_nodes)])
    b = np.array([0.7, -1.3])
    gx, gy = o.fe_grad(t, x @ b)
    assert np.allclose(gx, b[0], atol=1e-11) and np.allclose(gy, b[1], atol=1e-11)


# ---------------------------------------------------------------------------
# map, transformed velocity and departure point (Sec. II, reading R1)
# ---------------------------------------------------------------------------

def _G(mot, X, t):
    p = mot.params
    if mot.kind in (I.MOTION_PITCH, I.MOTION_PITCH_PLUNGE):
        th = p[0] + p[1] * math.sin(p[2] * t)
        d = X - p[3:5]
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        x = p[3:5] + R @ d
        if mot.kind == I.MOTION_PITCH_PLUNGE:  # plunge y -= h sin(w_h t)
            x = x + np.array([0.0, -p[5] * math.sin(p[6] * t)])
        return x
    if mot.kind == I.MOTION_PLUNGE:
        return np.array([X[0], X[1] - p[0] * math.sin(p[1] * t)])
    if mot.kind == I.MOTION_SINE:
        A, L, Tp = p[0], p[1], p[2]
        s = math.sin(2 * math.pi * t / Tp)
        return np.array([X[0] + A * math.sin(2 * math.pi * X[1] / L) * s,
                         X[1] + A * math.sin(2 * math.pi * X[0] / L) * s])
    raise ValueError


def _Ginv(mot, x, t, X0):
    Xc = np.array(X0, float)
    for _ in range(50):  # Newton on G(X) = x with a finite-difference Jacobian
        r = _G(mot, Xc, t) - x
        h = 1e-6
        J = np.stack([(_G(mot, Xc + [h, 0], t) - _G(mot, Xc - [h, 0], t)) / (2 * h),
                      (_G(mot, Xc + [0, h], t) - _G(mot, Xc - [0, h], t)) / (2 * h)], 1)
        dX = np.linalg.solve(J, r)
        Xc = Xc - dX
        if np.abs(dX).max() < 1e-13:
            break
    return Xc


@pytest.mark.parametrize("mot", [I.Motion.make(I.MOTION_PITCH, 0.4, 0.3, 0.02, 20.0, 16.0),
                                 I.Motion.make(I.MOTION_SINE, 2.0, 32.0, 40.0, 0.0)],
                         ids=["pitch", "sine"])
def test_transformed_velocity_is_the_characteristic_slope(mot):
    """c^_i must be the velocity dX/dtau of the exact characteristic
    X(tau) = G^-1(G(X_a, t1) - c_i (t1 - tau), tau) at tau = t1."""
    mesh = I.periodic_box(8, 32.0, 0.2, seed=5)
    o = O.Oracle(mesh, mot, _flow())
    ol = O.Oracle(mesh, mot, _flow(), flags=O.FLAG_LITERAL_VG)
    t1 = 13.0
    px, py = o.departures(t1)
    lx, ly = ol.departures(t1)
    worst, worst_lit = 0.0, 0.0
    for a in range(0, mesh.n_nodes, 7):
        Xa = mesh.X[a]
        xa = _G(mot, Xa, t1)
        for i in range(9):
            c = np.array([CX[i], CY[i]], float)
            h = 1e-4
            Xp = _Ginv(mot, xa + c * h, t1 + h, Xa)   # tau = t1 + h: x = x_a + c h
            Xm = _Ginv(mot, xa - c * h, t1 - h, Xa)
            chat_exact = (Xp - Xm) / (2 * h)
            chat = Xa - np.array([px[i, a], py[i, a]])
            chat_lit = Xa - np.array([lx[i, a], ly[i, a]])
            worst = max(worst, np.abs(chat - chat_exact).max())
            worst_lit = max(worst_lit, np.abs(chat_lit - chat_exact).max())
    assert worst < 1e-6
    assert worst_lit > 1e-3  # the printed form differs whenever g != I and V_G != 0


def test_midpoint_variant_follows_the_characteristic_to_third_order():
    """Flag MIDPOINT (reading R2's variant): the transformed velocities of a
    step t_n -> t_{n+1} use g and V_G at t_{n+1/2}.  For the plunge map
    y = Y - h sin(w t) (g = I, V_G = (0, -h w cos w t)), one step of pure
    propagation of a field linear in Y reproduces it at the departure point,
    so the departure offset reads off the result.  Closed forms: the
    midpoint offset is -c_y - h w cos(w t_{n+1/2}), the arrival-time one
    -c_y - h w cos(w t_{n+1}), the exact characteristic's
    -c_y - h (sin w t_{n+1} - sin w t_n); the midpoint error is O(w^3), the
    arrival-time one O(w^2)."""
    L, h, w = 32.0, 2.0, 0.03
    mesh = I.periodic_box(16, L, 0.2, seed=8)
    mot = I.Motion.make(I.MOTION_PLUNGE, h, w)
    fl = _flow()
    Y = mesh.X[:, 1]
    base_f = O.feq(1.0, 0.0, 0.0, 0.3)
    base_g = O.geq(1.0, 0.0, 0.0, 0.3, CV)
    slope = 1e-3 / L
    f = base_f[:, None] * (1.0 + slope * Y[None, :])
    g = base_g[:, None] * (1.0 + slope * Y[None, :])
    n = mesh.n_nodes
    t0 = 7.0
    inner = (Y > 4.0) & (Y < L - 4.0)
    got = {}
    for name, flags in (("mid", O.FLAG_MIDPOINT), ("end", 0), ("exact", O.FLAG_EXACT_CHAR)):
        o = O.Oracle(mesh, mot, fl, flags=flags | O.FLAG_COLLIDE_OFF | O.FLAG_PHI_OFF)
        o.set_state(f, g, np.ones(n), np.zeros(n), np.zeros(n), np.full(n, 0.3), t=t0)
        o.step(1)
        fs = o.state()["f"]
        got[name] = (fs / base_f[:, None] - 1.0) / slope - Y[None, :]  # Y_dp - Y per direction
    t1 = t0 + 1.0
    for i in range(9):
        cy = CY[i]
        mid = -cy - h * w * math.cos(w * (t1 - 0.5))
        end = -cy - h * w * math.cos(w * t1)
        exact = -cy - h * (math.sin(w * t1) - math.sin(w * t0))
        assert np.abs(got["mid"][i, inner] - mid).max() < 1e-9
        assert np.abs(got["end"][i, inner] - end).max() < 1e-9
        assert np.abs(got["exact"][i, inner] - exact).max() < 1e-9  # flag EXACT_CHAR
        assert abs(mid - exact) < 1.01 * h * w ** 3 / 24 + 1e-12
        assert abs(end - exact) > 10 * abs(mid - exact)


def test_departure_variants_against_the_exact_characteristic():
    """Accuracy of the two c^ departures X - c^(t) against the exact
    characteristic's (flag EXACT_CHAR), t = t_{n+1} or t_{n+1/2}, as the
    motion slows.  Plunge (c^ depends on time only): the midpoint departure
    is about a hundred times closer.  Rigid pitch: c^ also varies along the
    characteristic through V_G, which no time level captures, so both stay
    first order in the pitch rate and the midpoint only halves the error."""
    mesh = I.periodic_box(8, 32.0, 0.2, seed=5)
    errs = {}
    for kind in ("plunge", "pitch"):
        for w in (0.04, 0.02):
            mot = (I.Motion.make(I.MOTION_PLUNGE, 3.0, w) if kind == "plunge"
                   else I.Motion.make(I.MOTION_PITCH, 0.05, 0.3, w, 16.0, 16.0))
            o = O.Oracle(mesh, mot, _flow())
            t1 = 9.0
            ex = np.stack(o.departures_exact(t1))
            errs[kind, w] = tuple(np.abs(np.stack(o.departures(t)) - ex).max() for t in (t1, t1 - 0.5))
    for w in (0.04, 0.02):
        end, mid = errs["plunge", w]
        assert mid < end / 50
        end, mid = errs["pitch", w]
        assert 0.4 < mid / end < 0.6
    assert 1.8 < errs["pitch", 0.04][0] / errs["pitch", 0.02][0] < 2.4  # first order in the rate


@pytest.mark.parametrize("kind", ["plunge", "pitch", "pitch_plunge"])
def test_exact_characteristic_departure_inverts_the_map(kind):
    """Flag EXACT_CHAR: X_dp = G^-1(G(X, t1) - c_i, t1 - 1), against the
    map inverted by Newton's method in this file (closed forms of G for
    plunge, rigid pitch and pitch with plunge)."""
    mot = {"plunge": I.Motion.make(I.MOTION_PLUNGE, 3.0, 0.05),
           "pitch": I.Motion.make(I.MOTION_PITCH, 0.05, 0.3, 0.04, 10.0, 2.0),
           "pitch_plunge": I.Motion.make(I.MOTION_PITCH_PLUNGE, 0.05, 0.3, 0.04, 10.0, 2.0, 2.0, 0.03)}[kind]
    mesh = I.periodic_box(8, 32.0, 0.2, seed=5)
    o = O.Oracle(mesh, mot, _flow(), flags=O.FLAG_EXACT_CHAR)
    t1 = 9.0
    px, py = o.departures_exact(t1)
    worst = 0.0
    for a in range(0, mesh.n_nodes, 5):
        Xa = mesh.X[a]
        xa = _G(mot, Xa, t1)
        for i in range(9):
            c = np.array([CX[i], CY[i]], float)
            X0 = _Ginv(mot, xa - c, t1 - 1.0, Xa)
            worst = max(worst, abs(X0[0] - px[i, a]), abs(X0[1] - py[i, a]))
    assert worst < 1e-9
    with pytest.raises(O.OracleError):  # no closed-form inverse: refused
        O.Oracle(mesh, I.Motion.make(I.MOTION_SINE, 1.0, 32.0, 50.0, 0.0), _flow()).departures_exact(t1)


def test_mesh_velocity_is_time_derivative_of_the_map():
    mot = I.Motion.make(I.MOTION_BLENDED_PITCH, 0.1, 0.3, 0.01, 50.0, 0.0, 200.0, 1000.0)
    mesh = I.naca_omesh(32, 12, chord=200.0, R=4000.0, first=1.0)
    o = O.Oracle(mesh, mot, _flow())
    t, h = 11.0, 1e-3
    for a in range(0, mesh.n_nodes, 97):
        m = o.map(t, a)
        dxdt = (o.map(t + h, a)[6:8] - o.map(t - h, a)[6:8]) / (2 * h)
        assert np.allclose(m[4:6], dxdt, rtol=1e-6, atol=1e-9)


# ---------------------------------------------------------------------------
# whole-step invariants
# ---------------------------------------------------------------------------

def _eps(st, u):
    return (np.abs(st["ux"] - u[0]).sum() + np.abs(st["uy"] - u[1]).sum()) / (
        st["ux"].size * (abs(u[0]) + abs(u[1])))


def test_uniform_flow_preserved_on_deforming_mesh():
    """Sec. V.A / Table GCL_Error: uniform flow stays uniform to round-off
    (the paper reports eps ~ 4e-16 .. 1.1e-15)."""
    gold = dict(np.loadtxt(__file__.replace("test_oracle_pins.py", "golden/gcl_table.txt"),
                           comments="#"))
    case = I.uniform_flow_case(n=12, L=24.0, period_steps=40.0, steps=60)
    o = O.Oracle(case.mesh, case.motion, case.flow)
    o.step(case.steps)
    eps = _eps(o.state(), case.flow.u_inf)
    assert eps < 100 * max(gold.values())


def test_uniform_flow_paper_map():
    # x = X + A sin(2 pi X/L) sin(2 pi Y/L) sin(2 pi t/t0), A/L = 500/8000,
    # t0 = 1.5 L / u_inf, Ma 0.2, T 0.2 (Sec. V.A), on a small box
    L = 24.0
    fl = I.flow_params(0.2, T_inf=0.2, mu=0.02, chord=L)
    U = fl.u_inf[0]
    mot = I.Motion.make(I.MOTION_SINE, 500.0 / 8000.0 * L, L, 1.5 * L / U, 1.0)
    mesh = I.periodic_box(12, L, 0.2, seed=2)
    o = O.Oracle(mesh, mot, fl)
    o.step(40)
    assert _eps(o.state(), fl.u_inf) < 1e-13


def _lattice_state(mesh, T0, u0, amp, seed):
    rho, ux, uy, T = I.random_state(mesh.n_nodes, 1.0, T0, u0, amp, seed=seed)
    f = np.stack([O.feq(rho[a], ux[a], uy[a], T[a]) for a in range(mesh.n_nodes)], 1)
    g = np.stack([O.geq(rho[a], ux[a], uy[a], T[a], 2.5) for a in range(mesh.n_nodes)], 1)
    return f, g, rho, ux, uy, T


def test_lattice_reduction_equals_array_roll_d2q9():
    """On an unjittered mesh with nodes on the integer lattice and no motion,
    every departure point is a node: propagation must be the D2Q9 shift."""
    mesh = I.lattice_box(5)   # 10 x 10 lattice
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
    for step in range(4):
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


def test_lattice_mass_and_energy_conserved_with_corrections():
    mesh = I.lattice_box(6)
    fl = I.Flow(mu=0.02, T_inf=0.2, u_inf=(0.02, 0.01))
    o = O.Oracle(mesh, I.Motion.make(0), fl)
    f, g, rho, ux, uy, T = _lattice_state(mesh, 0.2, (0.02, 0.01), 0.01, 4)
    o.set_state(f, g, rho, ux, uy, T)
    m0, e0 = f.sum(), g.sum()
    o.step(15)
    st = o.state()
    assert np.isclose(st["f"].sum(), m0, rtol=1e-14)
    assert np.isclose(st["g"].sum(), e0, rtol=1e-14)


def test_shear_wave_decays_at_the_kinematic_viscosity():
    """A transverse wave u_y = U sin(k x) decays as exp(-(mu/rho) k^2 t):
    checks mu = (1/omega - 1/2) rho T dt (Sec. IV)."""
    n = 16
    mesh = I.lattice_box(n)
    L = 2 * n
    mu = 0.02
    fl = I.Flow(mu=mu, T_inf=0.2, u_inf=(0.0, 0.0))
    o = O.Oracle(mesh, I.Motion.make(0), fl)
    k = 2 * math.pi / L
    X = mesh.X[:, 0]
    U0 = 1e-3
    rho = np.ones(mesh.n_nodes)
    ux = np.zeros(mesh.n_nodes)
    uy = U0 * np.sin(k * X)
    T = np.full(mesh.n_nodes, 0.2)
    f = np.stack([O.feq(rho[a], ux[a], uy[a], T[a]) for a in range(mesh.n_nodes)], 1)
    g = np.stack([O.geq(rho[a], ux[a], uy[a], T[a], 2.5) for a in range(mesh.n_nodes)], 1)
    o.set_state(f, g, rho, ux, uy, T)
    amp = lambda: 2 * (o.state()["uy"] * np.sin(k * X)).mean()
    o.step(40)
    a1 = amp()
    o.step(200)
    a2 = amp()
    rate = -math.log(a2 / a1) / 200
    assert rate == pytest.approx(mu * k * k, rel=0.02)


def test_fluid_at_rest_with_walls_stays_at_rest():
    mesh = I.naca_omesh(32, 8, chord=20.0, R=200.0, first=1.0)
    fl = I.Flow(mu=0.02, T_inf=0.3, u_inf=(0.0, 0.0), chord=20.0)
    o = O.Oracle(mesh, I.Motion.make(0), fl)
    o.step(10)
    st = o.state()
    assert np.abs(st["rho"] - 1).max() < 1e-13
    assert np.abs(st["T"] - 0.3).max() < 1e-13
    assert np.abs(st["ux"]).max() < 1e-13 and np.abs(st["uy"]).max() < 1e-13
    F = o.forces()
    # uniform pressure on a closed straight-edged body: zero net force
    assert np.abs(F[:4]).max() < 1e-12 * 0.3 * 20.0


def test_offwall_mesh_velocity_target_keeps_rest_state():
    """Flag OFFWALL_VG (reading R8c, where the paper is silent): off-wall
    missing populations take the mesh velocity as the target.  Its only
    closed-form consequence: a fluid at rest around a body at rest stays at
    rest exactly (V_G = 0 is then the fluid's velocity)."""
    mesh = I.naca_omesh(32, 8, chord=20.0, R=200.0, first=1.0)
    fl = I.Flow(mu=0.02, T_inf=0.3, u_inf=(0.0, 0.0), chord=20.0)
    o = O.Oracle(mesh, I.Motion.make(0), fl, flags=O.FLAG_OFFWALL_VG)
    o.step(10)
    st = o.state()
    assert np.abs(st["rho"] - 1).max() < 1e-13 and np.abs(st["T"] - 0.3).max() < 1e-13
    assert np.abs(st["ux"]).max() < 1e-13 and np.abs(st["uy"]).max() < 1e-13


def test_missing_population_classification_matches_brute_force():
    """Reading R6: a population is missing iff some point of the segment from
    the node to its departure point lies outside the closed mesh; checked
    with exact rationals (split the segment at every meeting with a boundary
    edge, test one interior point of each piece and the departure point)."""
    mesh = I.naca_omesh(16, 4, chord=10.0, R=30.0, first=0.6)
    mot = I.Motion.make(I.MOTION_PITCH, 0.2, 0.3, 0.05, 2.5, 0.0)
    o = O.Oracle(mesh, mot, _flow())
    t = 3.0
    elem, kind = o.locate(t)
    px, py = o.departures(t)
    fr = _elem_frames(mesh)
    bnd = [(fr[e, k], fr[e, (k + 1) % 3], mesh.edge_kind[e, k])
           for e in range(mesh.n_elems) for k in range(3) if mesh.edge_kind[e, k]]
    F = Fraction

    def inside(q):
        for e in range(mesh.n_elems):
            v = [(F(fr[e, k, 0]), F(fr[e, k, 1])) for k in range(3)]
            if all((v[k][0] - q[0]) * (v[(k + 1) % 3][1] - q[1]) - (v[k][1] - q[1]) * (v[(k + 1) % 3][0] - q[0]) >= 0
                   for k in range(3)):
                return True
        return False

    def meets(a, p, u, w):
        """parameters along a->p where the closed segments meet (exact)"""
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

    rng = np.random.default_rng(0)
    wall_nodes = np.unique(np.concatenate([mesh.conn[e, [k, 3 + k, (k + 1) % 3]]
                                           for e in range(mesh.n_elems) for k in range(3)
                                           if mesh.edge_kind[e, k]]))
    sample = list(wall_nodes) + list(rng.choice(mesh.n_nodes, 30, replace=False))
    n_missing = 0
    for a in sample:
        for i in range(9):
            p = np.array([px[i, a], py[i, a]])
            Xa = mesh.X[a]
            if np.array_equal(p, Xa) and (CX[i], CY[i]) == (0, 0) and elem[i, a] == -2:
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
                assert elem[i, a] == _brute_locate(mesh, fr, p), (a, i)
    assert n_missing > 20


def test_wall_condition_thin_first_layer_stays_bounded():
    """Reading R8 (the wall condition's first-order gradients in the node's
    wall-side, i.e. smallest, incident element).  In a flat channel whose
    first cell layer (0.7) is thinner than one lattice unit, the nodes one
    layer off the wall have missing populations and take their own
    previous-step fields as targets (Sec. IV.A).  A uniform tangential flow
    at Mach 0.2 must then develop a boundary layer: the normal velocity
    stays small (only the weak compression waves of the impulsive start
    and of the growing layer, under 1e-3 against a free stream of 0.13)
    and the density stays within 2% of 1.  The larger-element gradient, a difference taken
    away from the wall at those nodes, blows this case up within 40 steps."""
    mesh = I.wall_channel()
    flow = I.flow_params(0.2, T_inf=0.3, Re=1e4, chord=1000.0)
    o = O.Oracle(mesh, I.Motion.make(0), flow)
    o.step(120)
    st = o.state()
    assert np.isfinite(st["rho"]).all()
    assert np.abs(st["rho"] - 1.0).max() < 0.02
    assert np.abs(st["uy"]).max() < 1e-3
    # no slip: the wall nodes' tangential velocity well below the free stream
    wall = np.abs(mesh.X[:, 1]) < 1e-12
    assert np.abs(st["ux"][wall]).max() < 0.5 * flow.u_inf[0]


def test_slip_walls_keep_uniform_tangential_flow():
    """Slip-wall variant (flag SLIP_WALL; the paper has no inviscid wall, the
    reading takes V_G plus the tangential part of the probe velocity and no
    non-equilibrium part): a uniform flow along the flat walls of a channel
    is an exact solution and must stay uniform to round-off, while the
    no-slip condition of Sec. IV.A slows the wall nodes down."""
    mesh = I.wall_channel(first=1.0)
    flow = I.flow_params(0.2, T_inf=0.3, Re=1e4, chord=1000.0)
    u0 = flow.u_inf[0]
    flow.flags = O.FLAG_SLIP_WALL
    o = O.Oracle(mesh, I.Motion.make(0), flow)
    o.step(50)
    st = o.state()
    assert np.abs(st["ux"] - u0).max() < 1e-12 and np.abs(st["uy"]).max() < 1e-12
    assert np.abs(st["rho"] - 1.0).max() < 1e-12 and np.abs(st["T"] - 0.3).max() < 1e-12
    flow.flags = 0
    o = O.Oracle(mesh, I.Motion.make(0), flow)
    o.step(50)
    wall = np.abs(mesh.X[:, 1]) < 1e-12
    assert np.abs(o.state()["ux"][wall]).max() < 0.5 * u0
