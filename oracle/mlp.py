"""FP64 reference of the departure-element proposal network.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline leg may import this module; the library never does.

The network (the learned part of the build; the paper has no counterpart):
6 features -> 64 tanh -> 64 tanh -> 32 slot logits + 3 barycentric guesses.
Loss per sample with a true slot s among the node's n ring elements:
    cross-entropy of softmax over the first n logits at s
    + w * mean over k of (guess_k - lambda_k)^2
averaged over the samples.  Parameters are kept as one flat vector in the
order W1 [64][6], b1 [64], W2 [64][64], b2 [64], W3 [35][64], b3 [35], the
same order as the CUDA library's.  The backward pass is the chain rule
written out; a central-difference test pins it.
"""
import numpy as np

N_IN, N_H, K, N_OUT = 6, 64, 32, 35
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
          ("W3", (N_OUT, N_H)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, k = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(theta[k:k + n], dtype=np.float64).reshape(shp)
        k += n
    return out


def pack(P):
    return np.concatenate([np.asarray(P[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def forward(theta, X):
    P = unpack(theta)
    H1 = np.tanh(X @ P["W1"].T + P["b1"])
    H2 = np.tanh(H1 @ P["W2"].T + P["b2"])
    O = H2 @ P["W3"].T + P["b3"]
    return H1, H2, O


def loss_and_grad(theta, X, slot, bary, nring, w_bary):
    """Mean loss over the samples and its gradient (flat, FP64)."""
    P = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    H1, H2, O = forward(theta, X)
    logits = O[:, :K].copy()
    mask = np.arange(K)[None, :] >= np.asarray(nring)[:, None]
    logits[mask] = -np.inf
    m = logits.max(axis=1, keepdims=True)
    ex = np.exp(logits - m)
    Z = ex.sum(axis=1, keepdims=True)
    p = ex / Z
    idx = np.arange(n)
    ce = -(logits[idx, slot] - m[:, 0] - np.log(Z[:, 0]))
    gd = O[:, K:] - np.asarray(bary, dtype=np.float64)
    L = ce.mean() + w_bary * (gd ** 2).sum(axis=1).mean() / 3.0
    dO = np.zeros_like(O)
    dO[:, :K] = p
    dO[idx, slot] -= 1.0
    dO[:, :K] /= n
    dO[:, K:] = w_bary * 2.0 * gd / (3.0 * n)
    G = {"W3": dO.T @ H2, "b3": dO.sum(axis=0)}
    dA2 = (dO @ P["W3"]) * (1.0 - H2 ** 2)
    G["W2"] = dA2.T @ H1
    G["b2"] = dA2.sum(axis=0)
    dA1 = (dA2 @ P["W2"]) * (1.0 - H1 ** 2)
    G["W1"] = dA1.T @ X
    G["b1"] = dA1.sum(axis=0)
    return L, pack(G)


def loss(theta, X, slot, bary, nring, w_bary):
    return loss_and_grad(theta, X, slot, bary, nring, w_bary)[0]


def round_f16(theta):
    """The parameters as the FP16 copies the network runs with."""
    return np.asarray(theta, dtype=np.float16).astype(np.float64)


def predict(theta, X, nring):
    """Slot of largest logit among the first nring."""
    _, _, O = forward(theta, X)
    logits = O[:, :K].copy()
    logits[np.arange(K)[None, :] >= np.asarray(nring)[:, None]] = -np.inf
    return logits.argmax(axis=1), O[:, K:]
