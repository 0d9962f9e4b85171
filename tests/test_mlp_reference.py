"""Pins of the FP64 reference network (oracle/mlp.py) used to check the GPU
training kernels: its analytic gradient against central differences, its
loss against values computed by hand on a tiny case, and its softmax
masking."""
import numpy as np

from oracle import mlp


def _batch(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, mlp.N_IN))
    nring = rng.integers(3, mlp.K + 1, size=n)
    slot = np.array([rng.integers(0, r) for r in nring])
    bary = rng.dirichlet(np.ones(3), size=n)
    return X, slot, bary, nring


def _theta(seed, scale=0.4):
    return np.random.default_rng(seed).normal(scale=scale, size=mlp.N_PARAMS)


def test_gradient_matches_central_differences():
    X, slot, bary, nring = _batch(7, 1)
    th = _theta(2)
    L, g = mlp.loss_and_grad(th, X, slot, bary, nring, 0.7)
    rng = np.random.default_rng(3)
    picks = rng.choice(mlp.N_PARAMS, 60, replace=False)
    h = 1e-6
    for k in picks:
        e = np.zeros_like(th)
        e[k] = h
        fd = (mlp.loss(th + e, X, slot, bary, nring, 0.7) - mlp.loss(th - e, X, slot, bary, nring, 0.7)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, g[k])


def test_loss_of_zero_network_is_log_ring_size_plus_bary_mse():
    """All-zero parameters: every logit 0, so the cross-entropy is
    log(nring); every guess 0, so the squared error is the mean of lambda^2."""
    X, slot, bary, nring = _batch(5, 4)
    th = np.zeros(mlp.N_PARAMS)
    L = mlp.loss(th, X, slot, bary, nring, 2.0)
    want = np.mean(np.log(nring)) + 2.0 * np.mean((bary ** 2).sum(axis=1)) / 3.0
    assert abs(L - want) < 1e-14


def test_masked_slots_get_no_probability():
    X, slot, bary, nring = _batch(4, 5)
    nring[:] = 5
    slot[:] = 2
    th = _theta(6)
    pred, _ = mlp.predict(th, X, nring)
    assert (pred < 5).all()
    # gradient of the logits beyond the ring is zero: W3 rows >= 5 (slots)
    # and b3 entries get no update from the cross-entropy
    _, g = mlp.loss_and_grad(th, X, slot, bary, nring, 0.0)
    P = mlp.unpack(g)
    assert np.abs(P["W3"][5:mlp.K]).max() == 0.0 and np.abs(P["b3"][5:mlp.K]).max() == 0.0


def test_pack_unpack_roundtrip_and_size():
    th = _theta(7)
    assert mlp.N_PARAMS == 6 * 64 + 64 + 64 * 64 + 64 + 35 * 64 + 35
    assert np.array_equal(mlp.pack(mlp.unpack(th)), th)
