"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Element choices must agree bit for bit; FP64 populations and fields to
1e-12 relative, element by element (entries below 1e-3 of the largest are
compared against that floor; velocities against the largest speed); the
FP32-deviation mode to 2e-4 in density and temperature (relative, node by
node) and velocity (relative to the largest speed).
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
import parity_util
from paper_2002_04353_gb300 import alelb, inputs as I

pytestmark = pytest.mark.gpu

CV = 1.0 / (1.4 - 1.0)
TOL64 = 1e-12
TOL32 = 2e-4


def _eq_state(mesh, flow, amp, seed):
    rho, ux, uy, T = I.random_state(mesh.n_nodes, flow.rho_inf, flow.T_inf, flow.u_inf, amp, seed)
    U = getattr(flow, "shift", (0.0, 0.0))
    if any(U):  # populations of the shifted lattice c_i + U
        f = np.stack([O.feq_shift(rho[a], ux[a], uy[a], T[a], U) for a in range(mesh.n_nodes)], 1)
        g = np.stack([O.geq_shift(rho[a], ux[a], uy[a], T[a], CV, U) for a in range(mesh.n_nodes)], 1)
    else:
        f = np.stack([O.feq(rho[a], ux[a], uy[a], T[a]) for a in range(mesh.n_nodes)], 1)
        g = np.stack([O.geq(rho[a], ux[a], uy[a], T[a], CV) for a in range(mesh.n_nodes)], 1)
    return f, g, rho, ux, uy, T


_rel = parity_util.rel


def _pair(mesh, motion, flow, prec=alelb.PREC_FP64, flags=None, state=None, renumber=alelb.RENUMBER_MORTON):
    o = O.Oracle(mesh, motion, flow, flags=flags)
    m = alelb.Mesh(mesh, motion, renumber)
    s = alelb.Solver(m, flow, prec, flags=flags)
    if state is not None:
        o.set_state(*state)
        s.set_pops(*state)
    return o, m, s


# ---------------------------------------------------------------------------
# element choices
# ---------------------------------------------------------------------------

LOC_CASES = {
    "box_sine": lambda: (I.periodic_box(16, 32.0, 0.2, seed=1), I.Motion.make(I.MOTION_SINE, 1.6, 32.0, 100.0, 0.0)),
    "box_paper_map": lambda: (I.periodic_box(12, 24.0, 0.2, seed=2), I.Motion.make(I.MOTION_SINE, 1.5, 24.0, 60.0, 1.0)),
    "lattice_static": lambda: (I.lattice_box(8), I.Motion.make(I.MOTION_NONE)),
    "omesh_plunge": lambda: (I.naca_omesh(64, 20, chord=200.0, R=4000.0, first=1.0), I.Motion.make(I.MOTION_PLUNGE, 20.0, 0.002)),
    "omesh_pitch": lambda: (I.naca_omesh(64, 20, chord=200.0, R=4000.0, first=1.0), I.Motion.make(I.MOTION_PITCH_PLUNGE, 0.05, 0.05, 0.003, 50.0, 0.0, 20.0, 0.003)),
    "omesh_blended": lambda: (I.naca_omesh(64, 20, chord=200.0, R=4000.0, first=1.0), I.Motion.make(I.MOTION_BLENDED_PITCH, 0.05, 0.05, 0.002, 50.0, 0.0, 400.0, 2000.0)),
    # flat walls along lattice directions: segments run along boundary edges
    "channel_plunge": lambda: (I.wall_channel(), I.Motion.make(I.MOTION_PLUNGE, 2.0, 0.02)),
}


@pytest.mark.parametrize("name", sorted(LOC_CASES))
def test_element_choices_bitwise(name):
    mesh, motion = LOC_CASES[name]()
    flow = I.Flow(mu=0.02, T_inf=0.3, u_inf=(0.1, 0.0))
    o = O.Oracle(mesh, motion, flow)
    m = alelb.Mesh(mesh, motion)
    s = alelb.Solver(m, flow)
    for t in (1.0, 17.0, 33.0):
        eo, ko = o.locate(t)
        eg, kg = s.locate(t)
        assert np.array_equal(eo, eg), f"{name} t={t}: {np.sum(eo != eg)} element choices differ"
        assert np.array_equal(ko, kg)


def test_element_choices_literal_vg_flag():
    mesh, motion = LOC_CASES["omesh_pitch"]()
    flow = I.Flow(mu=0.02, T_inf=0.3, u_inf=(0.1, 0.0), flags=O.FLAG_LITERAL_VG)
    o = O.Oracle(mesh, motion, flow)
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow)
    eo, ko = o.locate(9.0)
    eg, kg = s.locate(9.0)
    assert np.array_equal(eo, eg) and np.array_equal(ko, kg)


# ---------------------------------------------------------------------------
# full step, FP64
# ---------------------------------------------------------------------------

def _compare64(o, s, what=""):
    st = o.state()
    f, g = s.get_pops()
    mo = s.moments()
    ef, eg = _rel(f, st["f"]), _rel(g, st["g"])
    assert ef < TOL64 and eg < TOL64, f"{what}: f {ef:.2e} g {eg:.2e}"
    for k, e in parity_util.field_errors(mo, st).items():
        assert e < TOL64, f"{what}: {k} {e:.2e}"


@pytest.mark.parametrize("flags", [0, O.FLAG_PHI_OFF, O.FLAG_COLLIDE_OFF])
def test_fp64_steps_periodic_deforming_box(flags):
    case = I.uniform_flow_case(n=16, L=32.0, period_steps=50.0)
    st = _eq_state(case.mesh, case.flow, 0.01, seed=3)
    o, m, s = _pair(case.mesh, case.motion, case.flow, flags=flags, state=st)
    for k in range(3):
        o.step(4)
        s.lb_step(4)
        _compare64(o, s, f"box flags={flags} after {4 * (k + 1)} steps")


def test_fp64_steps_lattice_reduction_mesh():
    mesh = I.lattice_box(10)
    flow = I.Flow(mu=0.02, T_inf=0.2, u_inf=(0.02, 0.01))
    st = _eq_state(mesh, flow, 0.01, seed=4)
    o, m, s = _pair(mesh, I.Motion.make(0), flow, state=st)
    o.step(6)
    s.lb_step(6)
    _compare64(o, s, "lattice")


@pytest.mark.parametrize("motion_name", ["omesh_plunge", "omesh_pitch", "omesh_blended", "channel_plunge"])
def test_fp64_steps_airfoil_walls_farfield(motion_name):
    mesh, motion = LOC_CASES[motion_name]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o, m, s = _pair(mesh, motion, flow)
    for k in range(2):
        o.step(3)
        s.lb_step(3)
        _compare64(o, s, f"{motion_name} after {3 * (k + 1)} steps")
    fo = o.forces()
    fg = s.forces()
    # absolute floor: a pressure rho_inf T_inf over a chord (the channel's
    # net forces are round-off)
    assert np.allclose(fg, fo, rtol=1e-10, atol=1e-12 * max(np.abs(fo).max(), flow.rho_inf * flow.T_inf * flow.chord))


def test_fp64_bc_equilibrium_variant():
    mesh, motion = LOC_CASES["omesh_plunge"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    flow.flags = O.FLAG_BC_EQUILIBRIUM
    o, m, s = _pair(mesh, motion, flow)
    o.step(4)
    s.lb_step(4)
    _compare64(o, s, "bc-equilibrium")


@pytest.mark.parametrize("prec", [alelb.PREC_FP64, alelb.PREC_FP32_DEV])
def test_slip_wall_variant(prec):
    """The slip (inviscid) wall variant on a pitching-plunging airfoil: wall
    tangent in the physical frame, probe velocity, no non-equilibrium part."""
    mesh, motion = LOC_CASES["omesh_pitch"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    flow.flags = O.FLAG_SLIP_WALL
    o, m, s = _pair(mesh, motion, flow, prec=prec)
    o.step(6)
    s.lb_step(6)
    if prec == alelb.PREC_FP64:
        _compare64(o, s, "slip wall")
    else:
        _compare_mixed(o, s, "slip wall mixed")


def test_renumbering_does_not_change_results():
    case = I.uniform_flow_case(n=10, L=20.0, period_steps=30.0)
    mesh = case.mesh.permuted(7)
    st = _eq_state(mesh, case.flow, 0.01, seed=5)
    res = []
    for ren in (alelb.RENUMBER_NONE, alelb.RENUMBER_MORTON):
        m = alelb.Mesh(mesh, case.motion, ren)
        s = alelb.Solver(m, case.flow)
        s.set_pops(*st)
        s.lb_step(5)
        res.append(s.get_pops())
    assert _rel(res[0][0], res[1][0]) < 1e-14 and _rel(res[0][1], res[1][1]) < 1e-14


def test_uniform_flow_config_full_size_200_steps():
    """The deforming periodic box at its full size (48 x 48 vertices, 9,216
    P2 nodes, 200 steps): uniform flow preserved to round-off and the state
    equal to the oracle's."""
    case = I.uniform_flow_case()
    o, m, s = _pair(case.mesh, case.motion, case.flow)
    o.step(case.steps)
    s.lb_step(case.steps)
    _compare64(o, s, "config full size")
    mo = s.moments()
    u = case.flow.u_inf
    eps = (np.abs(mo["ux"] - u[0]).sum() + np.abs(mo["uy"] - u[1]).sum()) / (
        mo["ux"].size * (abs(u[0]) + abs(u[1])))
    assert eps < 1e-13


def test_zero_steps_and_tiny_mesh():
    mesh = I.periodic_box(3, 6.0, 0.1, seed=9)
    flow = I.Flow(mu=0.02, T_inf=0.2, u_inf=(0.01, 0.0))
    st = _eq_state(mesh, flow, 0.01, seed=1)
    o, m, s = _pair(mesh, I.Motion.make(I.MOTION_SINE, 0.2, 6.0, 20.0, 0.0), flow, state=st)
    s.lb_step(0)
    _compare64(o, s, "zero steps")
    o.step(3)
    s.lb_step(3)
    _compare64(o, s, "tiny mesh")


def test_mesh_errors_are_reported():
    mesh = I.periodic_box(6, 12.0, 0.2, seed=1)
    bad = I.Mesh(mesh.X.copy(), mesh.conn[:, [1, 0, 2, 3, 5, 4]].copy(), mesh.edge_kind, mesh.period)
    with pytest.raises(alelb.AlelbError) as ex:
        alelb.Mesh(bad, I.Motion.make(0))
    assert ex.value.status == -4
    m = alelb.Mesh(mesh, I.Motion.make(I.MOTION_SINE, 20.0, 12.0, 10.0, 0.0))
    with pytest.raises(alelb.AlelbError) as ex:
        m.move(2.5)  # amplitude large enough to fold the map
    assert ex.value.status == -5


# ---------------------------------------------------------------------------
# FP32-deviation (mixed) mode
# ---------------------------------------------------------------------------

def _compare_mixed(o, s, what):
    errs = parity_util.field_errors(s.moments(), o.state())
    for k, err in errs.items():
        assert err < TOL32, f"{what}: {k} err {err:.2e}"
    return errs


def test_mixed_box_matches_fp64_oracle():
    case = I.uniform_flow_case(n=16, L=32.0, period_steps=50.0)
    st = _eq_state(case.mesh, case.flow, 0.01, seed=6)
    o, m, s = _pair(case.mesh, case.motion, case.flow, prec=alelb.PREC_FP32_DEV, state=st)
    o.step(20)
    s.lb_step(20)
    _compare_mixed(o, s, "mixed box")


def test_mixed_airfoil_matches_fp64_oracle():
    mesh, motion = LOC_CASES["omesh_plunge"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o, m, s = _pair(mesh, motion, flow, prec=alelb.PREC_FP32_DEV)
    o.step(6)
    s.lb_step(6)
    _compare_mixed(o, s, "mixed airfoil")


@pytest.mark.parametrize("name", ["box_sine", "box_paper_map", "omesh_plunge", "omesh_pitch", "omesh_blended", "channel_plunge"])
def test_fast_path_element_choices_bitwise(name):
    """The FP32-deviation propagation settles most populations with the
    previous-step element, verified by certified FP32 arithmetic; its
    decisions must equal the oracle's exhaustive search bit for bit."""
    mesh, motion = LOC_CASES[name]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o = O.Oracle(mesh, motion, flow)
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow, alelb.PREC_FP32_DEV)
    s.lb_step(3)  # fills the per-population element cache
    walks_before = s.info()["walks"]
    s.lb_step(2)
    settled = 1.0 - (s.info()["walks"] - walks_before) / (2 * 9 * mesh.n_nodes)
    assert settled > 0.5, f"fast path settled only {settled:.3f} of the populations"
    t, _ = s.time()
    eo, ko = o.locate(t + 1.0)
    eg, kg = s.locate(t + 1.0, use_cache=True)
    assert np.array_equal(eo, eg), f"{name}: {np.sum(eo != eg)} fast-path element choices differ"
    assert np.array_equal(ko, kg)


# ---------------------------------------------------------------------------
# 16-bit population storage (BF16 and scaled FP16 deviations, FP32 arithmetic)
# ---------------------------------------------------------------------------

# Half a unit in the last place of the stored significand: bfloat16 keeps 8
# significant bits, binary16 11.
U16 = {alelb.PREC_BF16_DEV: 2.0 ** -8, alelb.PREC_FP16_DEV: 2.0 ** -11}
PREC16 = [alelb.PREC_BF16_DEV, alelb.PREC_FP16_DEV]


def _compare16(o, s, prec, flow, n, what):
    """First-order model of the storage error: each step rounds every stored
    deviation twice (streamed and post-collision values), each rounding at
    most U16 times the deviation from the far-field equilibria, which the
    16-bit forms store.  The moments take sums over 9 populations and a
    division by rho, so a field moves by at most 2 n U16 D / rho_min with
    D = max over nodes of sum_i (|f_i - f_inf,i| + |g_i - g_inf,i|); the
    temperature carries one more factor 1/Cv + |u|^2.  The bound drops the
    rounding's propagation through later interpolations (P2 weights sum to
    one) and adds the FP32 bound."""
    st = o.state()
    if any(flow.shift):
        fi = O.feq_shift(flow.rho_inf, flow.u_inf[0], flow.u_inf[1], flow.T_inf, flow.shift)
        gi = O.geq_shift(flow.rho_inf, flow.u_inf[0], flow.u_inf[1], flow.T_inf, CV, flow.shift)
    else:
        fi = O.feq(flow.rho_inf, flow.u_inf[0], flow.u_inf[1], flow.T_inf)
        gi = O.geq(flow.rho_inf, flow.u_inf[0], flow.u_inf[1], flow.T_inf, CV)
    D = (np.abs(st["f"] - fi[:, None]).sum(0) + np.abs(st["g"] - gi[:, None]).sum(0)).max()
    rmin = st["rho"].min()
    base = 2 * n * U16[prec] * D / rmin
    umax = max(np.abs(st["ux"]).max(), np.abs(st["uy"]).max())
    mo = s.moments()
    errs = {}
    for k in ("rho", "ux", "uy", "T"):
        scale = 1.0 if k in ("rho", "T") else umax
        tol = base * (1.0 / CV + umax ** 2 + 1.0 if k == "T" else 1.0) / scale + TOL32
        err = np.abs(mo[k] - st[k]).max() / scale
        errs[k] = err
        assert err < tol, f"{what}: {k} err {err:.2e} > {tol:.2e} (D {D:.2e})"
    return errs


@pytest.mark.parametrize("prec", PREC16)
def test_16bit_box_matches_fp64_oracle(prec):
    case = I.uniform_flow_case(n=16, L=32.0, period_steps=50.0)
    st = _eq_state(case.mesh, case.flow, 0.01, seed=6)
    o, m, s = _pair(case.mesh, case.motion, case.flow, prec=prec, state=st)
    o.step(20)
    s.lb_step(20)
    _compare16(o, s, prec, case.flow, 20, "16-bit box")


@pytest.mark.parametrize("prec", PREC16)
def test_16bit_airfoil_matches_fp64_oracle(prec):
    mesh, motion = LOC_CASES["omesh_pitch"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o, m, s = _pair(mesh, motion, flow, prec=prec)
    o.step(8)
    s.lb_step(8)
    _compare16(o, s, prec, flow, 8, "16-bit airfoil")


@pytest.mark.parametrize("prec", PREC16)
def test_16bit_uniform_flow_preserved(prec):
    """Uniform flow on the deforming box: the stored deviations from the
    far-field equilibria stay at the FP32 rounding of the equilibria."""
    case = I.uniform_flow_case(n=16, L=32.0, period_steps=50.0)
    s = alelb.Solver(alelb.Mesh(case.mesh, case.motion), case.flow, prec)
    s.lb_step(50)
    mo = s.moments()
    u = case.flow.u_inf
    assert np.abs(mo["rho"] - case.flow.rho_inf).max() < 1e-6
    assert np.abs(mo["T"] - case.flow.T_inf).max() < 1e-6
    assert max(np.abs(mo["ux"] - u[0]).max(), np.abs(mo["uy"] - u[1]).max()) < 1e-6


@pytest.mark.parametrize("prec", PREC16)
def test_16bit_element_choices_and_info(prec):
    """Storage does not enter the departure points: the deviation forms take
    the same element decisions, and info() reports 2-byte values."""
    mesh, motion = LOC_CASES["omesh_plunge"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o = O.Oracle(mesh, motion, flow)
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow, prec)
    s.lb_step(4)
    assert s.info()["pop_bytes"] == 2
    t, _ = s.time()
    eo, ko = o.locate(t + 1.0)
    eg, kg = s.locate(t + 1.0, use_cache=True)
    assert np.array_equal(eo, eg) and np.array_equal(ko, kg)


# ---------------------------------------------------------------------------
# transformed velocities at the midpoint time (flag MIDPOINT)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("motion_name", ["omesh_pitch", "omesh_blended", "omesh_plunge"])
def test_midpoint_variant_fp64_and_fp32(motion_name):
    mesh, motion = LOC_CASES[motion_name]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o, m, s = _pair(mesh, motion, flow, flags=O.FLAG_MIDPOINT)
    o.step(4)
    s.lb_step(4)
    _compare64(o, s, f"{motion_name} midpoint FP64")
    o2, m2, s2 = _pair(mesh, motion, flow, prec=alelb.PREC_FP32_DEV, flags=O.FLAG_MIDPOINT)
    o2.step(4)
    s2.lb_step(4)
    _compare_mixed(o2, s2, f"{motion_name} midpoint FP32")
    # the flag changes the result (the map moves between t_{n+1/2} and t_{n+1})
    o3 = O.Oracle(mesh, motion, flow)
    o3.step(4)
    assert _rel(o3.state()["f"], o.state()["f"]) > 1e-12


def test_midpoint_variant_fast_path_decisions_bitwise():
    mesh, motion = LOC_CASES["omesh_pitch"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o = O.Oracle(mesh, motion, flow, flags=O.FLAG_MIDPOINT)
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow, alelb.PREC_FP32_DEV, flags=O.FLAG_MIDPOINT)
    s.lb_step(5)
    t, _ = s.time()
    eo, ko = o.locate(t + 0.5)  # the next step's departure map time
    eg, kg = s.locate(t + 0.5, use_cache=True)
    assert np.array_equal(eo, eg) and np.array_equal(ko, kg)


def test_batch_refuses_the_midpoint_variant():
    mesh, motion = LOC_CASES["omesh_plunge"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow, alelb.PREC_FP32_DEV, flags=O.FLAG_MIDPOINT)
    with pytest.raises(alelb.AlelbError) as ex:
        alelb.Batch([s])
    assert ex.value.status == -1


# ---------------------------------------------------------------------------
# departure on the exact characteristic of a rigid map (flag EXACT_CHAR)
# ---------------------------------------------------------------------------

EXACT_CASES = {
    "omesh_plunge": LOC_CASES["omesh_plunge"],
    "omesh_pitch_plunge": LOC_CASES["omesh_pitch"],
    "omesh_pitch": lambda: (I.naca_omesh(64, 20, chord=200.0, R=4000.0, first=1.0),
                            I.Motion.make(I.MOTION_PITCH, 0.05, 0.05, 0.003, 50.0, 0.0)),
}


@pytest.mark.parametrize("motion_name", sorted(EXACT_CASES))
def test_exact_characteristic_fp64_and_fp32(motion_name):
    mesh, motion = EXACT_CASES[motion_name]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o, m, s = _pair(mesh, motion, flow, flags=O.FLAG_EXACT_CHAR)
    o.step(4)
    s.lb_step(4)
    _compare64(o, s, f"{motion_name} exact characteristic FP64")
    o2, m2, s2 = _pair(mesh, motion, flow, prec=alelb.PREC_FP32_DEV, flags=O.FLAG_EXACT_CHAR)
    o2.step(4)
    s2.lb_step(4)
    _compare_mixed(o2, s2, f"{motion_name} exact characteristic FP32")
    # the flag changes the result (X - c^ is the first-order departure)
    o3 = O.Oracle(mesh, motion, flow)
    o3.step(4)
    assert _rel(o3.state()["f"], o.state()["f"]) > 1e-12


def test_exact_characteristic_refused_where_the_map_has_no_closed_inverse():
    mesh, motion = LOC_CASES["omesh_blended"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    m = alelb.Mesh(mesh, motion)
    with pytest.raises(alelb.AlelbError) as ex:
        alelb.Solver(m, flow, alelb.PREC_FP64, flags=O.FLAG_EXACT_CHAR)
    assert ex.value.status == -1
    mesh, motion = LOC_CASES["omesh_plunge"]()
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow, alelb.PREC_FP32_DEV, flags=O.FLAG_EXACT_CHAR)
    with pytest.raises(alelb.AlelbError) as ex:
        alelb.Batch([s])
    assert ex.value.status == -1


# ---------------------------------------------------------------------------
# shifted lattice (velocities c_i + U; Sec. V.D's transonic case)
# ---------------------------------------------------------------------------

U03 = (float(np.float32(0.3)), 0.0)  # 0.3 rounded to FP32: the library wants U exact in FP32


def _shift_cases():
    mesh, motion = LOC_CASES["omesh_pitch"]()
    yield "pitching airfoil Ma 0.75", mesh, motion, I.flow_params(0.75, T_inf=0.3, Re=500.0, chord=200.0,
                                                                   shift=U03)
    box = I.uniform_flow_case(n=16, L=32.0, period_steps=50.0, Ma=0.85, T_inf=0.3)
    fl = dataclasses.replace(box.flow, shift=(U03[0], float(np.float32(-0.05))))
    st = _eq_state(box.mesh, fl, 0.01, seed=5)
    yield "deforming box Ma 0.85", box.mesh, box.motion, (fl, st)


@pytest.mark.parametrize("which", [0, 1])
def test_shifted_lattice_fp64_fp32_and_16bit(which):
    name, mesh, motion, fl = list(_shift_cases())[which]
    fl, st = fl if isinstance(fl, tuple) else (fl, None)
    o, m, s = _pair(mesh, motion, fl, state=st)
    o.step(4)
    s.lb_step(4)
    _compare64(o, s, f"{name}, shifted, FP64")
    o2, m2, s2 = _pair(mesh, motion, fl, prec=alelb.PREC_FP32_DEV, state=st)
    o2.step(4)
    s2.lb_step(4)
    _compare_mixed(o2, s2, f"{name}, shifted, FP32")
    for prec in PREC16:
        o3, m3, s3 = _pair(mesh, motion, fl, prec=prec, state=st)
        o3.step(4)
        s3.lb_step(4)
        _compare16(o3, s3, prec, fl, 4, f"{name}, shifted")
    # the shift changes the result
    o4 = O.Oracle(mesh, motion, dataclasses.replace(fl, shift=(0.0, 0.0)))
    if st is not None:
        o4.set_state(*_eq_state(mesh, dataclasses.replace(fl, shift=(0.0, 0.0)), 0.01, seed=5))
    o4.step(4)
    assert _rel(o4.state()["ux"], o.state()["ux"]) > 1e-9


@pytest.mark.parametrize("flags", [O.FLAG_EXACT_CHAR, O.FLAG_MIDPOINT, O.FLAG_OFFWALL_VG])
def test_shifted_lattice_with_the_variants(flags):
    """The shift combined with the departure variants and the off-wall
    target reading, FP64 and FP32 against the oracle."""
    mesh, motion = LOC_CASES["omesh_plunge"]()
    fl = I.flow_params(0.5, T_inf=0.3, Re=500.0, chord=200.0, shift=U03)
    o, m, s = _pair(mesh, motion, fl, flags=flags)
    o.step(3)
    s.lb_step(3)
    _compare64(o, s, f"plunging airfoil, shifted, flags {flags}")
    o2, m2, s2 = _pair(mesh, motion, fl, prec=alelb.PREC_FP32_DEV, flags=flags)
    o2.step(3)
    s2.lb_step(3)
    _compare_mixed(o2, s2, f"plunging airfoil, shifted, flags {flags}, FP32")


@pytest.mark.parametrize("motion_name", ["omesh_plunge", "omesh_pitch"])
def test_offwall_mesh_velocity_target(motion_name):
    """Flag OFFWALL_VG (reading R8c): FP64 and FP32 against the oracle on
    moving airfoils, where off-wall nodes have missing populations."""
    mesh, motion = LOC_CASES[motion_name]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o, m, s = _pair(mesh, motion, flow, flags=O.FLAG_OFFWALL_VG)
    o.step(4)
    s.lb_step(4)
    _compare64(o, s, f"{motion_name} off-wall V_G FP64")
    o2, m2, s2 = _pair(mesh, motion, flow, prec=alelb.PREC_FP32_DEV, flags=O.FLAG_OFFWALL_VG)
    o2.step(4)
    s2.lb_step(4)
    _compare_mixed(o2, s2, f"{motion_name} off-wall V_G FP32")
    o3 = O.Oracle(mesh, motion, flow)
    o3.step(4)
    assert _rel(o3.state()["f"], o.state()["f"]) > 1e-14  # the flag acts on these meshes


def test_shifted_lattice_refusals():
    mesh, motion = LOC_CASES["omesh_plunge"]()
    m = alelb.Mesh(mesh, motion)
    for bad in ((0.3, 0.0), (1.5, 0.0), (float("nan"), 0.0)):  # 0.3 is not exact in FP32
        fl = I.flow_params(0.5, T_inf=0.3, Re=500.0, chord=200.0, shift=bad)
        with pytest.raises(alelb.AlelbError) as ex:
            alelb.Solver(m, fl, alelb.PREC_FP32_DEV)
        assert ex.value.status == -1


@pytest.mark.parametrize("prec", [alelb.PREC_FP32_DEV, alelb.PREC_BF16_DEV, alelb.PREC_FP16_DEV])
@pytest.mark.parametrize("flags", [0, O.FLAG_MIDPOINT])
def test_deviation_forms_on_a_tiny_mesh(prec, flags):
    """A 3 x 3 periodic box (18 nodes: every warp partly empty, every
    element touching the periodic seams), zero steps, then three."""
    mesh = I.periodic_box(3, 6.0, 0.1, seed=9)
    flow = I.Flow(mu=0.02, T_inf=0.2, u_inf=(0.01, 0.0))
    st = _eq_state(mesh, flow, 0.01, seed=1)
    motion = I.Motion.make(I.MOTION_SINE, 0.2, 6.0, 20.0, 0.0)
    o, m, s = _pair(mesh, motion, flow, prec=prec, flags=flags, state=st)
    s.lb_step(0)
    o.step(3)
    s.lb_step(3)
    if prec == alelb.PREC_FP32_DEV:
        _compare_mixed(o, s, "tiny mesh")
    else:
        _compare16(o, s, prec, flow, 3, "tiny mesh")
