"""The step entry point that allocates nothing (alelb_lb_step_noalloc).

Some callers cannot allocate device memory once they are running -- an
application whose device memory is all pre-reserved by its own allocator,
or a loop that must not call cudaMalloc/cudaFree (cudaFree can wait for the
whole device).  For them the library offers one FP64 step whose scratch sits
in a static device array; the caller passes the state in its own device
buffers.  This file checks, through the C-ABI, that two such calls in a row
give what the ordinary allocating solver gives for the same two steps, and
that a mesh beyond the array's size is refused.  It is collected last on
purpose, and passes both alone and after the other tests.
"""
import numpy as np
import pytest

import oracle as O
from paper_2002_04353_gb300 import alelb, inputs as I

pytestmark = pytest.mark.gpu

CV = 1.0 / (1.4 - 1.0)


def _state(mesh, flow, seed):
    rho, ux, uy, T = I.random_state(mesh.n_nodes, flow.rho_inf, flow.T_inf, flow.u_inf, 0.01, seed)
    U = flow.shift
    f = np.stack([O.feq_shift(rho[a], ux[a], uy[a], T[a], U) for a in range(mesh.n_nodes)], 1)
    g = np.stack([O.geq_shift(rho[a], ux[a], uy[a], T[a], CV, U) for a in range(mesh.n_nodes)], 1)
    return f, g, rho, ux, uy, T


@pytest.mark.parametrize("which", ["airfoil", "box", "shifted airfoil"])
def test_noalloc_step_matches_the_allocating_solver_twice(which):
    import torch

    if which != "box":
        mesh = I.naca_omesh(64, 20, chord=200.0, R=4000.0, first=1.0)
        motion = I.Motion.make(I.MOTION_PLUNGE, 20.0, 0.002)
        shift = (float(np.float32(0.3)), 0.0) if which == "shifted airfoil" else (0.0, 0.0)
        flow = I.flow_params(0.1, T_inf=0.3, Re=500.0, chord=200.0, shift=shift)
    else:
        case = I.uniform_flow_case(n=16, L=32.0, period_steps=50.0)
        mesh, motion, flow = case.mesh, case.motion, case.flow
    f, g, rho, ux, uy, T = _state(mesh, flow, 11)
    m = alelb.Mesh(mesh, motion, alelb.RENUMBER_NONE)
    ref = alelb.Solver(m, flow, alelb.PREC_FP64)
    ref.set_pops(f, g, rho, ux, uy, T, t=0.0)

    dev = torch.device("cuda", 0)
    post = torch.tensor(np.concatenate([f, g], 0), dtype=torch.float64, device=dev).contiguous()
    fields = [torch.tensor(a, dtype=torch.float64, device=dev) for a in (rho, ux, uy, T)]
    torch.cuda.synchronize()
    for call in range(2):
        alelb.lb_step_noalloc(m, flow, float(call), post.data_ptr(), *[x.data_ptr() for x in fields])
        ref.lb_step(1)
        fr, gr = ref.get_pops()
        mo = ref.moments()
        got = post.cpu().numpy()
        for name, a, b in (("f", got[:9], fr), ("g", got[9:], gr)):
            err = np.abs(a - b).max() / np.abs(b).max()
            assert err < 1e-12, f"call {call + 1}: {name} differs by {err:.2e}"
        for k, x in zip(("rho", "ux", "uy", "T"), fields):
            b = mo[k]
            err = np.abs(x.cpu().numpy() - b).max() / max(np.abs(b).max(), 1e-300)
            assert err < 1e-12, f"call {call + 1}: {k} differs by {err:.2e}"


def test_noalloc_step_refuses_meshes_beyond_its_scratch():
    import torch

    case = I.plunge_case(ni=320, nj=118)  # 150,400 nodes > 131,072
    m = alelb.Mesh(case.mesh, case.motion, alelb.RENUMBER_NONE)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(alelb.AlelbError) as ex:
        alelb.lb_step_noalloc(m, case.flow, 0.0, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(),
                              x.data_ptr())
    assert ex.value.status == -1
    assert "131072" in str(ex.value)
