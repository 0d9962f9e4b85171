"""GPU parity of the paper's 9-node quadrilateral element (Sec. III,
Eq. Propagation with s = 1..9, Eq. NonLinear_Eq) against the FP64 oracle:
element choices bit for bit; FP64 state element by element to 1e-12; the
FP32-deviation form to 2e-4 in rho, u, T; the 16-bit forms within their
storage bound; the full 150,400-node plunging O-mesh; refusals of the
parts that serve triangles only."""
import numpy as np
import pytest

import oracle as O
import parity_util
from paper_2002_04353_gb300 import alelb, inputs as I

pytestmark = pytest.mark.gpu

CV = 1.0 / (1.4 - 1.0)
TOL64 = 1e-12
TOL32 = 2e-4

OM = lambda: I.naca_omesh(64, 20, chord=200.0, R=4000.0, first=1.0, elem="q2")
CASES = {
    "box_sine": lambda: (I.periodic_box(16, 32.0, 0.2, seed=1, elem="q2"), I.Motion.make(I.MOTION_SINE, 1.6, 32.0, 100.0, 0.0)),
    "box_paper_map": lambda: (I.periodic_box(12, 24.0, 0.2, seed=2, elem="q2"), I.Motion.make(I.MOTION_SINE, 1.5, 24.0, 60.0, 1.0)),
    "lattice_static": lambda: (I.lattice_box(8, elem="q2"), I.Motion.make(I.MOTION_NONE)),
    "omesh_plunge": lambda: (OM(), I.Motion.make(I.MOTION_PLUNGE, 20.0, 0.002)),
    "omesh_pitch": lambda: (OM(), I.Motion.make(I.MOTION_PITCH_PLUNGE, 0.05, 0.05, 0.003, 50.0, 0.0, 20.0, 0.003)),
    "omesh_blended": lambda: (OM(), I.Motion.make(I.MOTION_BLENDED_PITCH, 0.05, 0.05, 0.002, 50.0, 0.0, 400.0, 2000.0)),
    "channel_plunge": lambda: (I.wall_channel(elem="q2"), I.Motion.make(I.MOTION_PLUNGE, 2.0, 0.02)),
}


def _eq_state(mesh, flow, amp, seed):
    rho, ux, uy, T = I.random_state(mesh.n_nodes, flow.rho_inf, flow.T_inf, flow.u_inf, amp, seed)
    U = getattr(flow, "shift", (0.0, 0.0))
    if any(U):
        f = np.stack([O.feq_shift(rho[a], ux[a], uy[a], T[a], U) for a in range(mesh.n_nodes)], 1)
        g = np.stack([O.geq_shift(rho[a], ux[a], uy[a], T[a], CV, U) for a in range(mesh.n_nodes)], 1)
    else:
        f = np.stack([O.feq(rho[a], ux[a], uy[a], T[a]) for a in range(mesh.n_nodes)], 1)
        g = np.stack([O.geq(rho[a], ux[a], uy[a], T[a], CV) for a in range(mesh.n_nodes)], 1)
    return f, g, rho, ux, uy, T


def _pair(mesh, motion, flow, prec=alelb.PREC_FP64, state=None):
    o = O.Oracle(mesh, motion, flow)
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow, prec)
    if state is not None:
        o.set_state(*state)
        s.set_pops(*state)
    return o, s


def _check64(o, s, what):
    st = o.state()
    f, g = s.get_pops()
    assert parity_util.rel(f, st["f"]) < TOL64 and parity_util.rel(g, st["g"]) < TOL64, what
    for k, e in parity_util.field_errors(s.moments(), st).items():
        assert e < TOL64, f"{what}: {k} {e:.2e}"


def _check32(o, s, what, tol=TOL32):
    for k, e in parity_util.field_errors(s.moments(), o.state()).items():
        assert e < tol, f"{what}: {k} {e:.2e}"


@pytest.mark.parametrize("name", sorted(CASES))
def test_q2_element_choices_bitwise(name):
    mesh, motion = CASES[name]()
    flow = I.Flow(mu=0.02, T_inf=0.3, u_inf=(0.1, 0.0))
    o = O.Oracle(mesh, motion, flow)
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow)
    for t in (1.0, 17.0, 33.0):
        eo, ko = o.locate(t)
        eg, kg = s.locate(t)
        assert np.array_equal(eo, eg), f"{name} t={t}: {np.sum(eo != eg)} element choices differ"
        assert np.array_equal(ko, kg)


@pytest.mark.parametrize("flags", [0, O.FLAG_PHI_OFF, O.FLAG_COLLIDE_OFF])
def test_q2_fp64_deforming_box(flags):
    case = I.uniform_flow_case(n=16, L=32.0, period_steps=50.0, elem="q2")
    case.flow.flags = flags
    o, s = _pair(case.mesh, case.motion, case.flow, state=_eq_state(case.mesh, case.flow, 0.01, 3))
    for k in range(3):
        o.step(4)
        s.lb_step(4)
        _check64(o, s, f"q2 box flags={flags} after {4 * (k + 1)} steps")


@pytest.mark.parametrize("name", ["omesh_plunge", "omesh_pitch", "omesh_blended", "channel_plunge"])
def test_q2_fp64_walls_and_far_field(name):
    mesh, motion = CASES[name]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o, s = _pair(mesh, motion, flow)
    for k in range(2):
        o.step(3)
        s.lb_step(3)
        _check64(o, s, f"q2 {name} after {3 * (k + 1)} steps")
    fo, fg = o.forces(), s.forces()
    # absolute floor: a pressure rho_inf T_inf over a chord (the channel's
    # net forces are round-off)
    assert np.allclose(fg, fo, rtol=1e-10, atol=1e-12 * max(np.abs(fo).max(), flow.rho_inf * flow.T_inf * flow.chord))


@pytest.mark.parametrize("flags", [O.FLAG_BC_EQUILIBRIUM, O.FLAG_SLIP_WALL, O.FLAG_OFFWALL_VG, O.FLAG_MIDPOINT,
                                   O.FLAG_EXACT_CHAR, O.FLAG_LITERAL_VG],
                         ids=["bc_eq", "slip", "offwall_vg", "midpoint", "exact_char", "literal_vg"])
def test_q2_fp64_run_options(flags):
    mesh, motion = CASES["omesh_pitch"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    flow.flags = flags
    o, s = _pair(mesh, motion, flow)
    o.step(5)
    s.lb_step(5)
    _check64(o, s, f"q2 flags {flags}")


def test_q2_fp64_shifted_lattice_and_uniform_flow_config():
    mesh, motion = CASES["omesh_pitch"]()
    flow = I.flow_params(0.75, T_inf=0.3, Re=1000.0, chord=200.0, shift=(float(np.float32(0.3)), 0.0))
    o, s = _pair(mesh, motion, flow)
    o.step(4)
    s.lb_step(4)
    _check64(o, s, "q2 shifted lattice")
    # the deforming-box configuration at full size (48 x 48 cells, 9,216
    # nodes, 200 steps): uniform flow preserved to round-off, state = oracle
    case = I.uniform_flow_case(elem="q2")
    o, s = _pair(case.mesh, case.motion, case.flow)
    o.step(case.steps)
    s.lb_step(case.steps)
    _check64(o, s, "q2 box full size")
    mo = s.moments()
    u = case.flow.u_inf
    eps = (np.abs(mo["ux"] - u[0]).sum() + np.abs(mo["uy"] - u[1]).sum()) / (mo["ux"].size * (abs(u[0]) + abs(u[1])))
    assert eps < 1e-13


@pytest.mark.parametrize("name", ["box_sine", "omesh_plunge", "omesh_pitch"])
def test_q2_fp32_dev_matches_oracle(name):
    mesh, motion = CASES[name]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0) if name != "box_sine" else \
        I.Flow(mu=0.02, T_inf=0.2, u_inf=(0.05, 0.02))
    state = _eq_state(mesh, flow, 0.01, 6) if name == "box_sine" else None
    o, s = _pair(mesh, motion, flow, prec=alelb.PREC_FP32_DEV, state=state)
    o.step(10)
    s.lb_step(10)
    _check32(o, s, f"q2 fp32 {name}")


@pytest.mark.parametrize("prec", [alelb.PREC_BF16_DEV, alelb.PREC_FP16_DEV], ids=["bf16", "fp16"])
def test_q2_16bit_storage_within_its_bound(prec):
    """Each step rounds every stored deviation twice; the fields then move
    by at most 2 n U D / rho_min (D the largest summed deviation from the
    far-field equilibria at a node; U = 2^-8 bfloat16, 2^-11 binary16)."""
    mesh, motion = CASES["omesh_pitch"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    o, s = _pair(mesh, motion, flow, prec=prec)
    n = 8
    o.step(n)
    s.lb_step(n)
    st = o.state()
    fi = O.feq(flow.rho_inf, flow.u_inf[0], flow.u_inf[1], flow.T_inf)
    gi = O.geq(flow.rho_inf, flow.u_inf[0], flow.u_inf[1], flow.T_inf, CV)
    D = (np.abs(st["f"] - fi[:, None]).sum(0) + np.abs(st["g"] - gi[:, None]).sum(0)).max()
    U = 2.0 ** -8 if prec == alelb.PREC_BF16_DEV else 2.0 ** -11
    base = 2 * n * U * D / st["rho"].min()
    errs = parity_util.field_errors(s.moments(), st)
    umax = max(np.abs(st["ux"]).max(), np.abs(st["uy"]).max())
    assert errs["rho"] < base + TOL32
    assert errs["ux"] < base / umax + TOL32 and errs["uy"] < base / umax + TOL32
    assert errs["T"] < base * (1 / CV + umax ** 2 + 1) / st["T"].min() + TOL32


@pytest.fixture(scope="module")
def plunge150k_q2():
    case = I.plunge_case(elem="q2")
    assert case.mesh.n_nodes == 150400
    o = O.Oracle(case.mesh, case.motion, case.flow)
    o.step(20)
    return case, o.state()


@pytest.mark.parametrize("prec", [alelb.PREC_FP64, alelb.PREC_FP32_DEV], ids=["fp64", "fp32dev"])
def test_q2_plunge150k_matches_oracle_20_steps(plunge150k_q2, prec):
    case, st = plunge150k_q2
    s = alelb.Solver(alelb.Mesh(case.mesh, case.motion), case.flow, prec)
    s.lb_step(20)
    if prec == alelb.PREC_FP64:
        f, g = s.get_pops()
        assert parity_util.rel(f, st["f"]) < TOL64 and parity_util.rel(g, st["g"]) < TOL64
        tol = TOL64
    else:
        tol = TOL32
    for k, e in parity_util.field_errors(s.moments(), st).items():
        assert e < tol, f"q2 plunge150k: {k} {e:.2e}"


def test_q2_checkpoint_resume_and_refusals(tmp_path):
    mesh, motion = CASES["omesh_pitch"]()
    flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0)
    m = alelb.Mesh(mesh, motion)
    ref = alelb.Solver(m, flow, alelb.PREC_FP32_DEV)
    ref.lb_step(12)
    a = alelb.Solver(m, flow, alelb.PREC_FP32_DEV)
    a.lb_step(5)
    a.save(tmp_path / "q2.ck")
    b = alelb.Solver(m, flow, alelb.PREC_FP32_DEV)
    b.load(tmp_path / "q2.ck")
    b.lb_step(7)
    fr, gr = ref.get_pops()
    fb, gb = b.get_pops()
    assert np.array_equal(fr, fb) and np.array_equal(gr, gb)
    # the parts that serve triangle meshes only refuse quadrilaterals
    with pytest.raises(alelb.AlelbError) as e:
        alelb.Batch([a])
    assert e.value.status == -1
    net = alelb.Mlp(seed=0)
    with pytest.raises(alelb.AlelbError) as e:
        a.set_mlp(net)
    assert e.value.status == -1
    net.close()
    with pytest.raises(alelb.AlelbError) as e:
        alelb.lb_step_noalloc(alelb.Mesh(mesh, motion, alelb.RENUMBER_NONE), flow, 0.0, 1, 1, 1, 1, 1)
    assert e.value.status == -1
    # a quadrilateral that is not convex, and a misplaced centre node
    bad = I.naca_omesh(16, 4, chord=10.0, R=30.0, first=0.6, elem="q2")
    X = bad.X.copy()
    X[bad.conn[0, 8]] += 1e-3
    with pytest.raises(alelb.AlelbError) as e:
        alelb.Mesh(I.Mesh(X, bad.conn, bad.edge_kind, bad.period, elem_type=I.ELEM_Q2QUAD), I.Motion.make(0))
    assert e.value.status == -4
