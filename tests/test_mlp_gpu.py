"""The learned departure-element proposal on the GPU.

  * training data: every sample's slot names the exact element (checked
    through its barycentric coordinates against the FP64 oracle's departure
    point and element)
  * the GPU loss and gradient against the FP64 reference network
    (oracle/mlp.py) with the same FP16 weights: loss 1e-5, gradient 1e-3
    relative
  * tensor-core inference against the reference: same slot for nearly every
    sample (FP16 activations), logits within 0.05
  * training lowers the loss and raises the hit rate
  * streamed populations with and without the network: bit-identical
"""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as R
from paper_2002_04353_gb300 import alelb, inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case():
    mesh = I.naca_omesh(96, 30, chord=1000.0, R=20000.0, first=1.0)
    flow = I.flow_params(0.2, T_inf=0.3, Re=1850.0, chord=1000.0)
    motion = I.Motion.make(I.MOTION_PITCH_PLUNGE, 0.0, -0.04, 0.0008, 250.0, 0.0, 60.0, 0.0008)
    return mesh, motion, flow


def _samples(s, n_nodes):
    dev = torch.device("cuda")
    q = 9 * n_nodes
    feat = torch.empty((q, 6), dtype=torch.float32, device=dev)
    slot = torch.empty(q, dtype=torch.int16, device=dev)
    bary = torch.empty((q, 3), dtype=torch.float32, device=dev)
    nring = torch.empty(q, dtype=torch.uint8, device=dev)
    s.samples(feat, slot, bary, nring)
    return feat, slot, bary, nring


def _valid(feat, slot, bary, nring):
    keep = slot >= 0
    return (feat[keep].contiguous(), slot[keep].contiguous(), bary[keep].contiguous(),
            nring[keep].contiguous())


def test_samples_name_the_exact_element():
    mesh, motion, flow = _case()
    m = alelb.Mesh(mesh, motion, alelb.RENUMBER_NONE)
    s = alelb.Solver(m, flow, alelb.PREC_FP32_DEV)
    s.lb_step(2)
    feat, slot, bary, nring = _samples(s, mesh.n_nodes)
    o = O.Oracle(mesh, motion, flow)
    t = 3.0
    elem, kind = o.locate(t)
    px, py = o.departures(t)
    sl = slot.cpu().numpy().reshape(9, -1)
    ba = bary.cpu().numpy().reshape(9, -1, 3)
    ok = sl >= 0
    assert ok.mean() > 0.8, f"only {ok.mean():.3f} of the queries have their element in the ring"
    ii, aa = np.nonzero(ok)
    e = elem[ii, aa]
    assert (e >= 0).all()
    v = mesh.X[mesh.conn[e, :3]]  # [n, 3, 2]
    d1, d2 = v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]
    det = d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0]
    qx, qy = px[ii, aa] - v[:, 0, 0], py[ii, aa] - v[:, 0, 1]
    xi = (d2[:, 1] * qx - d2[:, 0] * qy) / det
    eta = (-d1[:, 1] * qx + d1[:, 0] * qy) / det
    assert np.abs(ba[ii, aa, 1] - xi).max() < 1e-5
    assert np.abs(ba[ii, aa, 2] - eta).max() < 1e-5
    assert np.abs(ba[ii, aa].sum(axis=1) - 1.0).max() < 1e-5
    nr = nring.cpu().numpy().reshape(9, -1)
    assert (sl < nr).all() and nr.max() <= 32


def test_gradient_matches_fp64_reference():
    mesh, motion, flow = _case()
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow, alelb.PREC_FP32_DEV)
    s.lb_step(1)
    feat, slot, bary, nring = _valid(*_samples(s, mesh.n_nodes))
    n = 3000
    feat, slot, bary, nring = feat[:n].contiguous(), slot[:n].contiguous(), bary[:n].contiguous(), nring[:n].contiguous()
    net = alelb.Mlp(seed=11)
    L, g = net.loss_grad(feat, slot, bary, nring, w_bary=0.5)
    th = net.params(rounded=True).astype(np.float64)
    Lr, gr = R.loss_and_grad(th, feat.cpu().numpy().astype(np.float64), slot.cpu().numpy().astype(np.int64),
                             bary.cpu().numpy().astype(np.float64), nring.cpu().numpy().astype(np.int64), 0.5)
    assert abs(L - Lr) <= 1e-5 * abs(Lr)
    assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
    assert np.abs(g - gr).max() <= 1e-3 * np.abs(gr).max()


def test_tensor_core_inference_matches_reference():
    mesh, motion, flow = _case()
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow, alelb.PREC_FP32_DEV)
    s.lb_step(1)
    feat, slot, bary, nring = _valid(*_samples(s, mesh.n_nodes))
    net = alelb.Mlp(seed=5)
    n = feat.shape[0]
    ps = torch.empty(n, dtype=torch.int32, device="cuda")
    out = torch.empty((n, 35), dtype=torch.float32, device="cuda")
    net.predict(feat, nring, ps, out)
    th = net.params(rounded=True).astype(np.float64)
    pr, _ = R.predict(th, feat.cpu().numpy().astype(np.float64), nring.cpu().numpy())
    _, _, Or = R.forward(th, feat.cpu().numpy().astype(np.float64))
    assert np.abs(out.cpu().numpy() - Or).max() < 0.05
    assert (ps.cpu().numpy() == pr).mean() > 0.97


def test_training_lowers_the_loss_and_raises_the_hit_rate():
    mesh, motion, flow = _case()
    s = alelb.Solver(alelb.Mesh(mesh, motion), flow, alelb.PREC_FP32_DEV)
    data = []
    for _ in range(3):
        s.lb_step(5)
        data.append(_valid(*_samples(s, mesh.n_nodes)))
    feat, slot, bary, nring = [torch.cat([d[k] for d in data]).contiguous() for k in range(4)]
    net = alelb.Mlp(seed=3)
    n = feat.shape[0]
    ps = torch.empty(n, dtype=torch.int32, device="cuda")
    net.predict(feat, nring, ps)
    hit0 = (ps == slot.int()).float().mean().item()
    losses = net.train(feat, slot, bary, nring, epochs=6, batch=2048, lr=3e-3, w_bary=0.5, seed=1)
    net.predict(feat, nring, ps)
    hit1 = (ps == slot.int()).float().mean().item()
    assert losses[-1] < 0.7 * losses[0], losses
    assert hit1 > hit0 + 0.2 and hit1 > 0.5, (hit0, hit1)


def test_streamed_populations_identical_with_and_without_network():
    mesh, motion, flow = _case()
    m = alelb.Mesh(mesh, motion)
    plain = alelb.Solver(m, flow, alelb.PREC_FP32_DEV)
    learned = alelb.Solver(m, flow, alelb.PREC_FP32_DEV)
    data = []
    for _ in range(4):
        plain.lb_step(3)
        learned.lb_step(3)
        data.append(_valid(*_samples(plain, mesh.n_nodes)))
    feat, slot, bary, nring = [torch.cat([d[k] for d in data]).contiguous() for k in range(4)]
    net = alelb.Mlp(seed=2)
    net.train(feat, slot, bary, nring, epochs=6, batch=2048, lr=3e-3, w_bary=0.5, seed=4)
    learned.set_mlp(net)
    before = learned.mlp_stats()
    plain.lb_step(12)
    learned.lb_step(12)
    fp, gp = plain.get_pops()
    fl, gl = learned.get_pops()
    assert np.array_equal(fp, fl) and np.array_equal(gp, gl)
    mp, ml = plain.moments(), learned.moments()
    for k in mp:
        assert np.array_equal(mp[k], ml[k])
    st = learned.mlp_stats()
    proposed, accepted = st["proposed"] - before["proposed"], st["accepted"] - before["accepted"]
    assert proposed > 0 and accepted > 0
    assert plain.info()["walks"] == learned.info()["walks"]  # the same populations reach the exact path
