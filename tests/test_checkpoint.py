"""Checkpoints on the GPU (alelb_save / alelb_load): a run interrupted by a
save and continued in a fresh solver from the file gives populations and
fields bit-identical to the uninterrupted run; files of another solver, or
damaged files, are refused and leave the solver as it was."""
import numpy as np
import pytest

from paper_2002_04353_gb300 import alelb, inputs as I

pytestmark = pytest.mark.gpu


def _case():
    mesh = I.naca_omesh(64, 20, chord=200.0, thickness=0.15, R=4000.0, first=1.0)
    motion = I.Motion.make(I.MOTION_PITCH_PLUNGE, 0.05, 0.05, 0.003, 50.0, 0.0, 20.0, 0.003)
    flow = I.flow_params(0.15, T_inf=0.3, Re=800.0, chord=200.0, angle_deg=2.0)
    return mesh, motion, flow


@pytest.mark.parametrize("prec", [alelb.PREC_FP64, alelb.PREC_FP32_DEV, alelb.PREC_BF16_DEV],
                         ids=["fp64", "fp32dev", "bf16dev"])
def test_resume_from_a_checkpoint_is_bit_identical(tmp_path, prec):
    mesh, motion, flow = _case()
    m = alelb.Mesh(mesh, motion)
    N, k = 40, 17
    ref = alelb.Solver(m, flow, prec)
    ref.lb_step(N)
    f_ref, g_ref = ref.get_pops()
    mo_ref = ref.moments()
    a = alelb.Solver(m, flow, prec)
    a.lb_step(k)
    path = tmp_path / "state.ck"
    a.save(path)
    info = alelb.checkpoint_info(path)
    assert info["step"] == k and info["t"] == float(k) and info["n_nodes"] == mesh.n_nodes
    b = alelb.Solver(alelb.Mesh(mesh, motion), flow, prec)  # fresh mesh object, same mesh
    b.load(path)
    assert b.time() == (float(k), k)
    b.lb_step(N - k)
    f, g = b.get_pops()
    mo = b.moments()
    assert np.array_equal(f, f_ref) and np.array_equal(g, g_ref)
    for key in ("rho", "ux", "uy", "T"):
        assert np.array_equal(mo[key], mo_ref[key]), key
    # the element cache and the counters came along: the same walks ran
    assert b.info()["walks"] == ref.info()["walks"]


def test_foreign_or_damaged_checkpoints_are_refused(tmp_path):
    mesh, motion, flow = _case()
    m = alelb.Mesh(mesh, motion)
    a = alelb.Solver(m, flow, alelb.PREC_FP32_DEV)
    a.lb_step(5)
    path = tmp_path / "a.ck"
    a.save(path)
    b = alelb.Solver(m, flow, alelb.PREC_FP32_DEV)
    b.lb_step(3)
    f0, g0 = b.get_pops()
    # another precision, another mesh, another free stream: ALELB_ERR_STATE
    others = [alelb.Solver(m, flow, alelb.PREC_FP64),
              alelb.Solver(alelb.Mesh(I.naca_omesh(64, 20, chord=200.0, thickness=0.12, R=4000.0, first=1.0),
                                      motion), flow, alelb.PREC_FP32_DEV),
              alelb.Solver(m, I.flow_params(0.2, T_inf=0.3, Re=800.0, chord=200.0, angle_deg=2.0),
                           alelb.PREC_FP32_DEV)]
    for s in others:
        with pytest.raises(alelb.AlelbError) as e:
            s.load(path)
        assert e.value.status == -9
    # damaged files: ALELB_ERR_ARG, and b keeps its state
    blob = path.read_bytes()
    for name, data in {"trunc": blob[: len(blob) // 2], "flip": blob[:4000] + bytes([blob[4000] ^ 4]) + blob[4001:]}.items():
        q = tmp_path / name
        q.write_bytes(data)
        with pytest.raises(alelb.AlelbError) as e:
            b.load(q)
        assert e.value.status == -1
    f1, g1 = b.get_pops()
    assert np.array_equal(f0, f1) and np.array_equal(g0, g1)
    assert b.time() == (3.0, 3)
    # a good load after the refusals still works, and a viscosity change is allowed
    c = alelb.Solver(m, I.flow_params(0.15, T_inf=0.3, Re=1600.0, chord=200.0, angle_deg=2.0), alelb.PREC_FP32_DEV)
    c.load(path)
    assert c.time() == (5.0, 5)
    c.lb_step(2)
    c.sync()
